"""pic_energy against the stored state (needs a GB300).

pic_energy must give the kinetic energy and live count of the particles as
stored: the host sum over pic_particles, m sum w (gamma - 1) dV, in FP64. It
is checked after a load, after steps and after a restore. The cases cover
the two-phase 3D FP32 push, the FP64 push, particles removed at absorbing
walls, and particles handled by the escape kernel.
"""
import numpy as np
import pytest

from paper_1503_02464_gb300 import synth
from paper_1503_02464_gb300.sim import Simulation

pytestmark = pytest.mark.gpu


def _host_energy(s, wl):
    total, alive = 0.0, 0
    for k, sp in enumerate(wl.species):
        p = s.particles(k)
        u2 = p["ux"] ** 2 + p["uy"] ** 2 + p["uz"] ** 2
        total += sp.m * np.sum(p["w"] * u2 / (np.sqrt(1.0 + u2) + 1.0))
        alive += len(p["w"])
    return total * float(np.prod(wl.d)), alive


def _build(wl, precision, **kw):
    s = Simulation.from_workload(wl, precision=precision, **kw)
    for isp, sp in enumerate(wl.species):
        p = wl.particles(isp)
        k = s.add_species(sp.q, sp.m, max(len(p["x"]), 1))
        s.load(k, p)
    if wl.neutralize:
        s.neutralize()
    return s


def _check(s, wl, tol):
    e = s.energy()
    ref, alive = _host_energy(s, wl)
    assert e["n_alive"] == alive
    assert abs(e["energy_kinetic"] - ref) <= tol * ref, (e["energy_kinetic"], ref)
    return e


def _cases():
    thermal3 = synth.small(3, (16, 16, 8), 2, 4, 0.1, 31)
    thermal2 = synth.small(2, (40, 24), 1, 4, 0.2, 32)
    # relativistic: particles outrun their tile's guard cells between sorts
    hot = synth.small(3, (24, 24, 16), 2, 2, 1.0, 33)
    hot.sort_every = 1000
    d = 0.1
    walls = synth.Workload("walls_hot", 2, (48, 16, 1), (d, d, 1.0), 0.9 * synth.courant_limit((d, d), 2), 2, 10,
                           34, [synth.Species("electron", -1.0, 1.0, 4, 0.5, 1.0, (4, 44), 0)],
                           absorbing_x=True, neutralize=False)
    return [("thermal3d", thermal3), ("thermal2d", thermal2), ("relativistic3d", hot), ("walls2d", walls)]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name,wl", _cases(), ids=[c[0] for c in _cases()])
def test_energy_by_product_matches_stored_state(precision, name, wl):
    tol = 1e-6 if precision == "fp32" else 1e-12
    s = _build(wl, precision)
    _check(s, wl, tol)                 # after the load
    s.checkpoint(0)
    for _ in range(4):
        s.step(3)
        _check(s, wl, tol)             # after steps
    d = s.diag()
    if name == "relativistic3d":
        assert d["n_escaped"] > 0      # the escape kernel took part
    if name == "walls2d":
        assert s.energy()["n_alive"] < len(wl.particles(0)["x"])  # some left through the walls
    s.restore(0)
    _check(s, wl, tol)                 # after a restore
    s.step(2)
    _check(s, wl, tol)
    s.close()
