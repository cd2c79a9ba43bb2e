"""GPU path vs the FP64 oracle on identical seeded inputs (needs a GB300).

Tolerances (stated by the build's target): FP64 path within 1e-12 relative
per step; FP32 path within 1e-5 relative on fields and momenta after 10
steps.  Relative means ||a - b||_inf / ||b||_inf per field component and
max |du| / max |u| for momenta matched by particle id.
"""
import numpy as np
import pytest

from paper_1503_02464_gb300 import synth

from _parity import build_gpu, build_oracle, compare_fields, compare_particles, j_floor

pytestmark = pytest.mark.gpu

FP64_TOL_PER_STEP = 1e-12
FP32_TOL = 1e-5


def _wl(dims, order, n, ppc, uth, seed, dt_frac=0.95):
    return synth.small(dims, n, order, ppc, uth, seed, dt_frac)


CASES = [
    # dims, order, grid, tile, ppc, u_th  (grids not multiples of the tile: ragged tiles)
    (2, 1, (40, 24), (16, 16), 4, 0.2),
    (2, 2, (40, 24), (16, 16), 4, 0.2),
    (3, 1, (12, 10, 9), None, 3, 0.2),
    (3, 2, (12, 10, 9), None, 3, 0.2),
]


@pytest.mark.parametrize("dims,order,n,tile,ppc,uth", CASES)
def test_fp64_per_step(dims, order, n, tile, ppc, uth):
    wl = _wl(dims, order, n, ppc, uth, 21 + dims * 10 + order)
    parts = [wl.particles(0)]
    o = build_oracle(wl, parts)
    s = build_gpu(wl, parts, "fp64", tile=tile)
    worst = []
    for step in range(1, 11):
        o.step(1)
        s.step(1)
        fe = compare_fields(o, s)
        du, dx = compare_particles(o, s, wl)
        tol = FP64_TOL_PER_STEP * step
        worst.append((step, max(fe.values()), du, dx))
        for k, v in fe.items():
            assert v <= tol, (step, k, v, tol)
        assert du <= tol, (step, du)
        assert dx <= tol * 10, (step, dx)
    print("fp64 worst per step:", worst)


# rows of a multiple of four cells take the four-node vector reductions of
# the FP32 J flush; these x sizes take the scalar one
ODD_ROW_CASES = [
    (2, 2, (41, 24), (16, 16), 4, 0.2),
    (3, 2, (13, 10, 9), None, 3, 0.2),
]


@pytest.mark.parametrize("dims,order,n,tile,ppc,uth", CASES + ODD_ROW_CASES)
def test_fp32_after_10_steps(dims, order, n, tile, ppc, uth):
    wl = _wl(dims, order, n, ppc, uth, 41 + dims * 10 + order)
    parts = [wl.particles(0)]
    o = build_oracle(wl, parts)
    s = build_gpu(wl, parts, "fp32", tile=tile)
    o.step(10)
    s.step(10)
    # every field, J included (the fixed-point deposit window is what sets
    # the FP32 current apart from the oracle's FP64 one)
    fe = compare_fields(o, s, j_abs=j_floor(wl, parts))
    du, dx = compare_particles(o, s, wl)
    print("fp32 after 10 steps:", fe, du, dx)
    for k, v in fe.items():
        assert v <= FP32_TOL, (k, v)
    assert du <= FP32_TOL, du


@pytest.mark.parametrize("dims", [2, 3])
@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("npart", [1, 2, 4])
def test_tiny_brute_force(dims, order, npart):
    """1-4 particles on a 4^d grid (smaller than a tile window, so window
    cells alias): every field array and every particle compared."""
    n = (4, 4, 4) if dims == 3 else (4, 4)
    wl = _wl(dims, order, n, 1, 0.4, 7 + npart)
    full = wl.particles(0)
    rng = np.random.default_rng(npart)
    pick = np.sort(rng.choice(len(full["x"]), npart, replace=False))
    parts = [{k: np.ascontiguousarray(v[pick]) for k, v in full.items()}]
    o = build_oracle(wl, parts, neutralize=False)
    s = build_gpu(wl, parts, "fp64", neutralize=False)
    for step in range(1, 6):
        o.step(1)
        s.step(1)
        fe = compare_fields(o, s)
        for k, v in fe.items():
            assert v <= FP64_TOL_PER_STEP * step, (step, k, v)
        du, dx = compare_particles(o, s, wl)
        assert du <= FP64_TOL_PER_STEP * step and dx <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_escape_path(precision):
    """Hot plasma, no re-sorting: particles leave their tile windows and take
    the global-memory path; results still match the oracle."""
    wl = _wl(3, 2, (24, 16, 16), 2, 0.8, 99)
    parts = [wl.particles(0)]
    o = build_oracle(wl, parts)
    s = build_gpu(wl, parts, precision, sort_every=1000)
    for step in range(1, 9):
        o.step(1)
        s.step(1)
    fe = compare_fields(o, s, j_abs=j_floor(wl, parts))
    du, dx = compare_particles(o, s, wl)
    d = s.diag()
    assert d["n_escaped"] > 0
    tol = FP64_TOL_PER_STEP * 8 if precision == "fp64" else FP32_TOL
    print(precision, "escape path after 8 steps:", fe, du)
    for k, v in fe.items():
        assert v <= tol, (k, v)
    assert du <= tol


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("order", [1, 2])
def test_fast_plasma_between_chunk_drain(precision, order):
    """A relativistic 3D plasma (u_th = 1) changes the shape support of about
    half its particles every step, more than the deferred-deposit queue of a
    work item holds: the first push overflows the queue (the overflowing
    particles deposit on the general stencil), the later ones take the
    variant that drains the queue between chunks.  Both stay at parity with
    the oracle, J included."""
    wl = _wl(3, order, (32, 16, 16), 16, 1.0, 61 + order)
    parts = [wl.particles(0)]
    o = build_oracle(wl, parts)
    s = build_gpu(wl, parts, precision)
    for step in range(1, 11):
        o.step(1)
        s.step(1)
        s.sync()  # the job count of each push is read back before the next
    fe = compare_fields(o, s, j_abs=j_floor(wl, parts))
    du, dx = compare_particles(o, s, wl)
    d = s.diag()
    print(precision, order, "fast plasma after 10 steps:", fe, du, d["n_push_mid_drain"])
    assert d["n_push_mid_drain"] >= 5, d
    tol = FP64_TOL_PER_STEP * 10 if precision == "fp64" else FP32_TOL
    for k, v in fe.items():
        assert v <= tol, (k, v)
    assert du <= tol


def test_adaptive_sort_within_one_step_call():
    """The same early sorts when all the steps are enqueued by one pic_step
    call: the host loop runs ahead of the device (2M particles, a push takes
    longer than enqueueing a step), so the escape counts must be waited for
    rather than only polled."""
    wl = _wl(3, 2, (64, 64, 32), 16, 1.0, 47)
    parts = [wl.particles(0)]
    s = build_gpu(wl, parts, "fp32", sort_every=1000)
    s.step(30)
    d = s.diag()
    print("adaptive sorts", d["n_sorts_adaptive"], "escaped", d["n_escaped"])
    assert d["n_sorts_adaptive"] > 0
    assert d["n_escaped"] < 0.2 * 30 * wl.n_particles()
    assert np.isfinite(d["energy_kinetic"]) and d["n_alive"] == wl.n_particles()


def test_thermal2d_64_full_fp64():
    """The 2D3V periodic plasma: 64x64 cells, 16 ppc (65,536 electrons),
    CIC, dt = 0.035, 100 steps in FP64 against the oracle."""
    wl = synth.preset("thermal2d_64")
    parts = [wl.particles(0)]
    o = build_oracle(wl, parts)
    s = build_gpu(wl, parts, "fp64")
    errs = []
    for chunk in range(10):
        o.step(10)
        s.step(10)
        fe = compare_fields(o, s, ["Ex", "Ey", "Ez", "Bx", "By", "Bz"])
        du, dx = compare_particles(o, s, wl)
        errs.append((10 * (chunk + 1), max(fe.values()), du))
    print("thermal2d_64 fp64:", errs)
    for nstep, fe, du in errs:
        assert fe <= FP64_TOL_PER_STEP * nstep and du <= FP64_TOL_PER_STEP * nstep, (nstep, fe, du)
    do, dg = o.diag(), s.diag()
    for k in ("energy_field", "energy_kinetic"):
        assert abs(dg[k] - do[k]) <= 1e-10 * abs(do[k]), (k, dg[k], do[k])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_diagnostics_match_oracle(precision):
    wl = _wl(3, 2, (12, 12, 12), 2, 0.1, 5)
    parts = [wl.particles(0)]
    o = build_oracle(wl, parts)
    s = build_gpu(wl, parts, precision)
    o.step(3)
    s.step(3)
    do, dg = o.diag(), s.diag()
    tol = 1e-11 if precision == "fp64" else 1e-5
    for k in ("energy_field", "energy_kinetic"):
        assert abs(dg[k] - do[k]) <= tol * abs(do[k]), (k, dg[k], do[k])
    assert abs(dg["charge"]) <= 1e-10 * abs(parts[0]["w"]).sum() * np.prod(wl.d)
    assert dg["n_alive"] == do["n_alive"]
    # Gauss's law is kept by the charge-conserving deposit (zero at the start)
    scale = np.abs(s.field(9)).max() + 1e-300
    assert dg["gauss_max"] <= (1e-10 if precision == "fp64" else 1e-4) * max(scale, 1.0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_continuity_on_gpu(precision):
    """(rho^{n+1} - rho^n)/dt + div J^{n+1/2} = 0 at round-off on the GPU."""
    wl = _wl(2, 2, (32, 32), 4, 0.3, 3)
    parts = [wl.particles(0)]
    s = build_gpu(wl, parts, precision)
    s.step(2)
    s.diag()
    s.step(1)
    d = s.diag()
    J = max(np.abs(s.field(i)).max() for i in (6, 7, 8))
    tol = 1e-12 if precision == "fp64" else 1e-5
    assert 0 <= d["continuity_max"] <= tol * J / min(wl.d[:2]), d["continuity_max"]


def test_empty_species_and_zero_steps():
    wl = _wl(3, 2, (8, 8, 8), 1, 0.1, 1)
    from paper_1503_02464_gb300.sim import Simulation
    s = Simulation.from_workload(wl, precision="fp32")
    s.add_species(-1.0, 1.0, 16)
    s.step(0)
    s.step(3)
    d = s.diag()
    assert d["n_alive"] == 0 and d["energy_field"] == 0.0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_energy_readback_matches_diag(precision):
    wl = _wl(3, 2, (12, 12, 12), 2, 0.1, 9)
    parts = [wl.particles(0)]
    s = build_gpu(wl, parts, precision)
    s.step(4)
    d, e = s.diag(), s.energy()
    tol = 1e-12 if precision == "fp64" else 1e-6
    for k in ("energy_e", "energy_b", "energy_kinetic"):
        assert abs(d[k] - e[k]) <= tol * abs(d[k]), (k, d[k], e[k])
    assert d["n_alive"] == e["n_alive"] and e["step"] == 4


def test_adaptive_sort_for_fast_particles():
    """A relativistic plasma (u_th = 1) drifts out of the tile windows long
    before a sort_every = 1000 cadence: the library sorts early once a push
    sends more than 0.5 % of the particles down the escape path, and the run
    stays at FP64 parity with the oracle throughout."""
    wl = _wl(3, 2, (16, 16, 8), 4, 1.0, 45)
    parts = [wl.particles(0)]
    o = build_oracle(wl, parts)
    s = build_gpu(wl, parts, "fp64", sort_every=1000)
    for step in range(1, 31):
        o.step(1)
        s.step(1)
        if step % 10 == 0:
            s.sync()
            fe = compare_fields(o, s, ["Ex", "Ey", "Ez", "Bx", "By", "Bz"])
            for k, v in fe.items():
                assert v <= 1e-12 * step, (step, k, v)
            du, _ = compare_particles(o, s, wl, 0)
            assert du <= 1e-12 * step, (step, du)
    d = s.diag()
    assert d["n_sorts_adaptive"] > 0
    # without the early sorts most particles would take the escape path by now
    assert d["n_escaped"] < 0.2 * 30 * wl.n_particles()
