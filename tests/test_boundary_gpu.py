"""Absorbing x walls, laser injection and particle removal: GPU path vs the
FP64 oracle on identical inputs (needs a GB300).

Tolerances as for the periodic path: FP64 within 1e-12 relative per step,
FP32 within 1e-5 after 10 steps on fields and momenta.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1503_02464_gb300 import synth
from paper_1503_02464_gb300.sim import Simulation

from _parity import compare_fields, compare_particles, j_floor, j_floor_fp32, rel_inf

pytestmark = pytest.mark.gpu

TAU = 2 * math.pi


def _laser_slab(dims, nx, ny, nz=1, d=0.1, a0=2.0, slab=(20, 28), ppc=2, density=4.0, order=2, angle=0.0, pol=1):
    dd = (d, d, d if dims == 3 else 1.0)
    dt = 0.9 * synth.courant_limit(dd, dims)
    n = (nx, ny, nz if dims == 3 else 1)
    wl = synth.Workload("laser_slab_small", dims, n, dd, dt, order, 50, 77,
                        [synth.Species("electron", -1.0, 1.0, ppc, 0.0, density, slab, 0),
                         synth.Species("proton", 1.0, 1836.0, ppc, 0.0, density, slab, 1)],
                        absorbing_x=True, neutralize=False,
                        laser={"a0": a0, "waist": 0.25 * ny * d, "duration": TAU, "pol": pol, "angle": angle})
    return wl


def _pair(wl, precision):
    """Oracle and GPU simulations of the same workload; also returns the
    oracle's J error floor for these particles."""
    o = oracle.OracleSim(wl.dims, wl.n, wl.d, wl.dt, wl.order)
    o.set_absorbing_x(True)
    L = wl.laser
    o.set_laser(L["a0"], L["waist"], L["duration"], pol=L["pol"], angle=L.get("angle", 0.0))
    s = Simulation.from_workload(wl, precision=precision)
    parts = []
    for isp, sp in enumerate(wl.species):
        p = wl.particles(isp)
        parts.append(p)
        o.add_particles(p, sp.q, sp.m)
        k = s.add_species(sp.q, sp.m, len(p["x"]))
        s.load(k, p)
    return o, s, j_floor(wl, parts)


def _check_fp32(wl, before):
    """FP32 against the FP64 oracle once the pulse has reached the slab
    (``before`` steps) and 10 steps more: every field within 1e-5 of its
    vector field's norm (J above the FP32 position-rounding floor,
    j_floor_fp32) and the momenta of both species within 1e-5 of the
    momentum the fields can have imparted, |q/m| max|E| dt t, as in the FP64
    tests: the target starts cold, so its own max |u| is no scale for the
    error."""
    o, s, jf = _pair(wl, "fp32")
    nsteps = before + 10
    o.step(nsteps)
    s.step(nsteps)
    parts = [wl.particles(i) for i in range(len(wl.species))]
    fe = compare_fields(o, s, j_abs=max(jf, j_floor_fp32(wl, parts)))
    emax = max(np.abs(o.get_field(c)).max() for c in range(3))
    dus = []
    for isp, sp in enumerate(wl.species):
        us = abs(sp.q) / sp.m * emax * wl.dt * nsteps
        dus.append(compare_particles(o, s, wl, isp, u_scale=us)[0])
    print("fp32 fields", fe, "momenta", dus)
    for k, v in fe.items():
        assert v <= 1e-5, (k, v)
    for isp, du in enumerate(dus):
        assert du <= 1e-5, (isp, du)


def test_vacuum_pulse_fp64():
    wl = _laser_slab(2, 96, 16, ppc=0)
    wl.species = []
    o, s, _ = _pair(wl, "fp64")
    for step in range(1, 121):
        o.field_step(1)
        s.step(1)
        if step % 20 == 0:
            fe = compare_fields(o, s, ["Ex", "Ey", "Ez", "Bx", "By", "Bz"])
            for k, v in fe.items():
                assert v <= 1e-12 * step, (step, k, v)
    assert np.abs(s.field(1)).max() > 0.1  # the pulse is in the box


@pytest.mark.parametrize("dims", [2, 3])
def test_laser_slab_fp64(dims):
    wl = _laser_slab(3, 64, 16, 8, slab=(10, 16)) if dims == 3 else _laser_slab(2, 96, 24)
    o, s, jf = _pair(wl, "fp64")
    nsteps = 40 if dims == 3 else 80
    for step in range(1, nsteps + 1):
        o.step(1)
        s.step(1)
        if step % 10 == 0:
            fe = compare_fields(o, s, j_abs=jf)
            for k, v in fe.items():
                assert v <= 1e-12 * step, (step, k, v)
            # momentum scale the fields can impart so far: |q/m| max|E| t
            emax = max(np.abs(o.get_field(c)).max() for c in range(3))
            for isp, sp in enumerate(wl.species):
                us = abs(sp.q) / sp.m * emax * wl.dt * step
                du, dx = compare_particles(o, s, wl, isp, u_scale=us)
                assert du <= 1e-12 * step, (step, isp, du)
    # the laser has reached the slab and pushed electrons
    assert np.abs(s.particles(0)["ux"]).max() > 1e-3


@pytest.mark.parametrize("dims,order", [(2, 2), (2, 1), (3, 2), (3, 1)])
def test_laser_slab_fp32(dims, order):
    if dims == 2:
        wl = _laser_slab(2, 96, 24, order=order)
        before = 50
    else:
        wl = _laser_slab(3, 64, 16, 8, slab=(10, 16), order=order)
        before = 20
    _check_fp32(wl, before)


OBLIQUE = [(2, 1, math.radians(20.0)), (2, 2, math.radians(-15.0)), (3, 1, math.radians(25.0)),
           (3, 2, math.radians(-20.0))]


@pytest.mark.parametrize("dims,pol,angle", OBLIQUE)
def test_oblique_laser_slab_fp64(dims, pol, angle):
    """A laser tilted in the x-y plane: each wall row carries its own delay
    and profile, evaluated on the device; FP64 parity per step."""
    if dims == 3:
        wl = _laser_slab(3, 64, 16, 8, slab=(10, 16), angle=angle, pol=pol)
    else:
        wl = _laser_slab(2, 96, 24, angle=angle, pol=pol)
    o, s, jf = _pair(wl, "fp64")
    nsteps = 40 if dims == 3 else 80
    for step in range(1, nsteps + 1):
        o.step(1)
        s.step(1)
        if step % 10 == 0:
            fe = compare_fields(o, s, j_abs=jf)
            for k, v in fe.items():
                assert v <= 1e-12 * step, (step, k, v)
            emax = max(np.abs(o.get_field(c)).max() for c in range(3))
            for isp, sp in enumerate(wl.species):
                us = abs(sp.q) / sp.m * emax * wl.dt * step
                du, dx = compare_particles(o, s, wl, isp, u_scale=us)
                assert du <= 1e-12 * step, (step, isp, du)
    # the tilted wave reached the slab and pushed electrons (along z for s-polarisation)
    p0 = s.particles(0)
    assert max(np.abs(p0[k]).max() for k in ("ux", "uy", "uz")) > 1e-3
    comp = 1 if pol == 1 else 2
    wall = s.field(comp)[0, :, 1] if dims == 2 else s.field(comp)[wl.n[2] // 2, :, 1]
    assert np.abs(wall).max() > 0


@pytest.mark.parametrize("dims", [2, 3])
def test_oblique_laser_slab_fp32(dims):
    angle = math.radians(20.0)
    if dims == 2:
        wl = _laser_slab(2, 96, 24, angle=angle)
        before = 50
    else:
        wl = _laser_slab(3, 64, 16, 8, slab=(10, 16), angle=angle)
        before = 20
    _check_fp32(wl, before)


def _structured_target(structure):
    d = 0.1
    dt = 0.9 * synth.courant_limit((d, d), 2)
    species = [synth.Species("electron", -1.0, 1.0, 2, 0.0, 4.0, (20, 30), 0, structure=structure),
               synth.Species("proton", 1.0, 1836.0, 2, 0.0, 4.0, (20, 30), 0, structure=structure)]
    return synth.Workload("target_small", 2, (96, 48, 1), (d, d, 1.0), dt, 2, 60, 91, species, absorbing_x=True,
                          neutralize=False, laser={"a0": 2.0, "waist": 1.2, "duration": TAU, "pol": 1,
                                                   "angle": math.radians(30.0)})


STRUCTURES = [("grating", 12, 4), ("foam", 0.4, 99)]


@pytest.mark.parametrize("structure", STRUCTURES, ids=["grating", "foam"])
def test_structured_target_fp64(structure):
    """A laser at 30 degrees on a structured target (a grating front or a
    randomly filled foam): FP64 parity per step."""
    wl = _structured_target(structure)
    o, s, jf = _pair(wl, "fp64")
    for step in range(1, 61):
        o.step(1)
        s.step(1)
        if step % 10 == 0:
            fe = compare_fields(o, s, j_abs=jf)
            for k, v in fe.items():
                assert v <= 1e-12 * step, (step, k, v)
            emax = max(np.abs(o.get_field(c)).max() for c in range(3))
            for isp, sp in enumerate(wl.species):
                us = abs(sp.q) / sp.m * emax * wl.dt * step
                du, dx = compare_particles(o, s, wl, isp, u_scale=us)
                assert du <= 1e-12 * step, (step, isp, du)
    p0 = s.particles(0)
    assert max(np.abs(p0[k]).max() for k in ("ux", "uy")) > 1e-3


@pytest.mark.parametrize("structure", STRUCTURES, ids=["grating", "foam"])
def test_structured_target_fp32(structure):
    """The same targets on the FP32 path: 1e-5 on fields (J above the
    position-rounding floor) and on momenta relative to the field-imparted
    momentum, ten steps after the pulse has reached the target."""
    _check_fp32(_structured_target(structure), 50)


def test_oblique_laser_limits():
    """|angle| must stay below pi/2, and the adjoint covers normal incidence only."""
    from paper_1503_02464_gb300 import capi
    wl = _laser_slab(2, 96, 24, angle=0.5 * math.pi)
    with pytest.raises(capi.PicError):
        Simulation.from_workload(wl, precision="fp64")
    wl = _laser_slab(2, 96, 24, angle=0.3)
    s = Simulation.from_workload(wl, precision="fp64")
    with pytest.raises(capi.PicError):
        s.adjoint_begin(16)
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_particles_removed_at_walls(precision):
    """Fast particles streaming into both walls are removed on the same step
    as in the oracle; the remaining fields agree."""
    nx, ny = 40, 8
    wl = synth.Workload("walls", 2, (nx, ny, 1), (0.1, 0.1, 1.0), 0.06, 2, 10, 5, [], absorbing_x=True)
    rng = np.random.default_rng(3)
    n = 64
    x = rng.uniform(4.0, nx - 5.0, n) * 0.1
    parts = {"x": x, "y": rng.uniform(0, ny, n) * 0.1, "z": np.zeros(n),
             "ux": np.where(x > 2.0, 3.0, -3.0) * rng.uniform(0.5, 1.0, n),
             "uy": rng.normal(0, 0.3, n), "uz": rng.normal(0, 0.3, n), "w": np.full(n, 0.5),
             "id": np.arange(n, dtype=np.uint32)}
    o = oracle.OracleSim(2, wl.n, wl.d, wl.dt, 2)
    o.set_absorbing_x(True)
    o.add_particles(parts, -1.0, 1.0)
    s = Simulation.from_workload(wl, precision=precision)
    k = s.add_species(-1.0, 1.0, n)
    s.load(k, parts)
    for step in range(1, 31):
        o.step(1)
        s.step(1)
        assert s.diag()["n_alive"] == o.diag()["n_alive"], step
    assert o.diag()["n_alive"] < n
    tol = 1e-10 if precision == "fp64" else 1e-4
    fe = compare_fields(o, s, ["Ex", "Ey", "Ez", "Bx", "By", "Bz"])
    for key, v in fe.items():
        assert v <= tol, (key, v)
    assert s.diag()["n_absorbed"] == n - o.diag()["n_alive"]

def _oracle_current_of_moves(wl, before, after):
    """J of the given moves (particle dicts before and after one step, FP64
    copies of the GPU's stored FP32 state, matched by id) deposited by the
    oracle on an empty grid."""
    o = oracle.OracleSim(wl.dims, wl.n, wl.d, wl.dt, wl.order)
    L = np.array([wl.n[a] * wl.d[a] for a in range(3)])
    for sp, p0, p1 in zip(wl.species, before, after):
        i0, i1 = np.argsort(p0["id"]), np.argsort(p1["id"])
        assert np.array_equal(p0["id"][i0], p1["id"][i1])
        for a, b in zip(i0, i1):
            r0 = np.array([p0["x"][a], p0["y"][a], p0["z"][a]])
            r1 = np.array([p1["x"][b], p1["y"][b], p1["z"][b]])
            r1 = r0 + (r1 - r0 + 0.5 * L) % L - 0.5 * L  # undo the periodic wrap
            u = np.array([p1["ux"][b], p1["uy"][b], p1["uz"][b]])
            vz = u[2] / np.sqrt(1.0 + u @ u)
            o.deposit_move(sp.q, p0["w"][a], r0, r1, vz)
    return [o.get_field(c) for c in (oracle.JX, oracle.JY, oracle.JZ)]


@pytest.mark.parametrize("dims,order", [(2, 2), (2, 1), (3, 2), (3, 1)])
def test_fp32_deposit_of_stored_moves(dims, order):
    """The FP32 deposit arithmetic alone: after the pulse has reached the
    slab, the current of one FP32 step equals, to 1e-6 of max|J|, the FP64
    Esirkepov current of the same stored moves (the GPU's positions before
    and after the step), so the FP32 position rounding that j_floor_fp32
    allows for is not what is compared here."""
    if dims == 2:
        wl = _laser_slab(2, 96, 24, order=order)
        before = 59
    else:
        wl = _laser_slab(3, 64, 16, 8, slab=(10, 16), order=order)
        before = 29
    _, s, _ = _pair(wl, "fp32")
    s.step(before)
    p0 = [s.particles(i) for i in range(len(wl.species))]
    s.step(1)
    p1 = [s.particles(i) for i in range(len(wl.species))]
    assert all(len(a["id"]) == len(b["id"]) for a, b in zip(p0, p1))  # nothing absorbed in this step
    want = _oracle_current_of_moves(wl, p0, p1)
    got = [s.field(c) for c in (6, 7, 8)]
    norm = max(np.abs(j).max() for j in want)
    errs = [np.abs(g - w_).max() / norm for g, w_ in zip(got, want)]
    print("fp32 deposit of stored moves:", errs, "max|J|", norm)
    assert norm > 0
    for c, e in enumerate(errs):
        assert e <= 1e-6, (c, e)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 2e-5)])
def test_gauss_law_away_from_the_injection_wall(precision, tol):
    """While the pulse enters, div E - rho is not zero in the wall cells: the
    incoming wave is injected through the x = 0 Mur condition as its
    transverse component alone, and a Gaussian profile across y gives that
    component a y derivative there.  Everywhere else Gauss's law holds to
    round-off of the field norm (max|E| / dx): the Yee update keeps div E and
    the charge-conserving deposit keeps rho in step with it."""
    wl = _laser_slab(2, 96, 24)
    # electrons and protons drawn at the same positions: neutral node by
    # node, so E = 0 satisfies Gauss's law at the start
    for sp in wl.species:
        sp.seed_offset = 0
    s = Simulation.from_workload(wl, precision=precision)
    for isp, sp in enumerate(wl.species):
        p = wl.particles(isp)
        k = s.add_species(sp.q, sp.m, len(p["x"]))
        s.load(k, p)
    rho0 = s.field(9)[0]
    assert np.abs(rho0).max() <= 1e-12 * 4.0
    s.step(60)
    Ex, Ey, rho = s.field(0)[0], s.field(1)[0], s.field(9)[0]
    dx, dy = wl.d[0], wl.d[1]
    div = (Ex - np.roll(Ex, 1, axis=1)) / dx + (Ey - np.roll(Ey, 1, axis=0)) / dy
    res = np.abs(div - rho)
    scale = max(np.abs(Ex).max(), np.abs(Ey).max()) / min(dx, dy)
    wall = res[:, :2].max() / scale
    inner = res[:, 2:wl.n[0] - 2].max() / scale
    print(precision, "gauss residual / (max|E|/dx): wall cells %.2e, elsewhere %.2e" % (wall, inner))
    assert np.abs(Ey).max() > 0.1
    assert inner <= tol, inner
    s.close()
