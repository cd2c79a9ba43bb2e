"""Two-stream instability (the test problem of the paper's scaling study,
§4.1) on the GPU path: FP64 parity with the oracle step by step, FP32
parity after 10 steps, and the FP32 growth rate against the closed form of
the cold relativistic two-beam dispersion relation (needs a GB300).

Both beams sit on a quiet-start lattice seeded with the growing eigenmode,
over an explicit uniform background of charge +1 (pic_set_background), with
Ex initialised from Gauss's law.  The problem is electrostatic: B is
round-off on both sides, so E and B errors are measured against the joint
norm max(|E|, |B|).
"""
import numpy as np
import pytest

import oracle
from paper_1503_02464_gb300.sim import Simulation

from _parity import compare_fields, compare_particles, j_floor, rel_inf
from _twostream import fit_rate, gauss_ex, growth_rate, mode_amplitude, workload

pytestmark = pytest.mark.gpu


def _pair(wl, precision):
    parts = [wl.particles(i) for i in range(len(wl.species))]
    ex = gauss_ex(wl, parts)
    o = oracle.OracleSim(wl.dims, wl.n, wl.d, wl.dt, wl.order)
    s = Simulation.from_workload(wl, precision=precision)
    for sp, p in zip(wl.species, parts):
        o.add_particles(p, sp.q, sp.m)
        k = s.add_species(sp.q, sp.m, len(p["x"]))
        s.load(k, p)
    bg = np.ones(o.shape3)
    o.set_background(bg)
    s.set_background(bg)
    o.set_field(oracle.EX, ex)
    s.set_field(oracle.EX, ex)
    return o, s, parts


@pytest.mark.parametrize("dims", [2, 3])
def test_two_stream_fp64_parity(dims):
    if dims == 2:
        wl, _ = workload((32, 16), amp=1e-3, lattice=(4, 2))
        nsteps = 60
    else:
        wl, _ = workload((32, 8, 8), amp=1e-3, lattice=(2, 2, 2))
        nsteps = 20
    o, s, parts = _pair(wl, "fp64")
    # the explicit background enters rho as in the oracle: round-off of the
    # unit background and beam densities (the net charge is 1e-3 of them)
    assert np.abs(s.field(oracle.RHO) - o.rho()).max() <= 1e-12
    jf = j_floor(wl, parts)
    for step in range(1, nsteps + 1):
        o.step(1)
        s.step(1)
        if step % 10 == 0:
            fe = compare_fields(o, s, j_abs=jf, joint_eb=True)
            for key, v in fe.items():
                assert v <= 1e-12 * step, (step, key, v)
            for isp in range(2):
                du, _ = compare_particles(o, s, wl, isp)
                assert du <= 1e-12 * step, (step, isp, du)
    dg, do = s.diag(), o.diag()
    assert dg["gauss_max"] < 1e-10 and do["gauss_max"] < 1e-10
    assert abs(dg["energy_field"] / do["energy_field"] - 1.0) < 1e-10


def test_two_stream_fp32_parity_10_steps():
    wl, _ = workload((32, 8, 8), amp=1e-3, lattice=(2, 2, 2))
    o, s, _ = _pair(wl, "fp32")
    o.step(10)
    s.step(10)
    fe = compare_fields(o, s, ["Ex", "Ey", "Ez", "Bx", "By", "Bz"], joint_eb=True)
    for key, v in fe.items():
        assert v <= 1e-5, (key, v)
    for isp in range(2):
        du, _ = compare_particles(o, s, wl, isp)
        assert du <= 1e-5, (isp, du)


def test_two_stream_growth_fp32():
    """The FP32 path reproduces the linear growth of the seeded mode: rate
    within 1.5 % of the closed form and the amplitude history of the FP64
    oracle within 1e-3 at every step."""
    u0, amp, tmax = 0.2, 1e-4, 10.0
    wl, L = workload((32, 16), u0=u0, amp=amp)
    o, s, _ = _pair(wl, "fp32")
    ts, ag, ao = [0.0], [mode_amplitude(s.field(oracle.EX))], [mode_amplitude(o.get_field(oracle.EX))]
    for k in range(int(tmax / wl.dt)):
        o.step(1)
        s.step(1)
        ts.append((k + 1) * wl.dt)
        ag.append(mode_amplitude(s.field(oracle.EX)))
        ao.append(mode_amplitude(o.get_field(oracle.EX)))
    ag, ao = np.array(ag), np.array(ao)
    gth = growth_rate(2 * np.pi / L, u0)
    g = fit_rate(ts, ag, 1.0, tmax)
    assert abs(g / gth - 1.0) < 0.015, (g, gth)
    assert np.abs(ag / ao - 1.0).max() < 1e-3
    assert ag[-1] > 20 * ag[0]  # it did grow
