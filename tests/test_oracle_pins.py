"""Pins of the FP64 oracle to closed forms and invariants (CPU only).

Every check here is fixed by the mathematics of section 2 of the paper and
the published methods it names (Boris pusher, Yee FDTD, Esirkepov deposit),
not by the oracle itself, and each is chosen so that a plausible slip (a
dropped bracket term, a sign, a half-cell stagger, a wrong index) fails it.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import OracleSim, EX, EY, EZ, BX, BY, BZ, JX, JY, JZ


# ---------------------------------------------------------------- shapes (§2, g)
@pytest.mark.parametrize("order", [1, 2])
def test_shape_moments(order):
    """Partition of unity, first moment = X, and the sampled second central
    moment: f(1-f) for CIC (f the in-cell offset), the constant 1/4 for TSC."""
    rng = np.random.default_rng(5)
    for X in rng.uniform(-3, 3, 50):
        f = X - math.floor(X)
        var = f * (1 - f) if order == 1 else 0.25
        nodes = np.arange(math.floor(X) - 3, math.floor(X) + 4)
        s = np.array([oracle.shape(order, X - i) for i in nodes])
        assert np.all(s >= 0)
        assert abs(s.sum() - 1.0) < 1e-15
        assert abs((nodes * s).sum() - X) < 1e-13
        assert abs((((nodes - X) ** 2) * s).sum() - var) < 1e-13


def test_shape_values():
    assert oracle.shape(2, 0.0) == 0.75
    assert oracle.shape(2, 0.5) == 0.5
    assert oracle.shape(2, -1.0) == 0.125
    assert oracle.shape(2, 1.5) == 0.0
    assert oracle.shape(1, 0.25) == 0.75
    assert oracle.shape(1, -1.0) == 0.0


# ---------------------------------------------------------------- Boris (§2 eq. 3, ref [8])
def _rot(u, ang):
    c, s = math.cos(ang), math.sin(ang)
    return np.array([c * u[0] + s * u[1], -s * u[0] + c * u[1], u[2]])


@pytest.mark.parametrize("q,m", [(1.0, 1.0), (-1.0, 1.0), (1.0, 1836.0)])
def test_boris_gyration(q, m):
    """Uniform Bz, E = 0: |u| conserved; the turn per step is exactly
    2 atan(q B dt / (2 m gamma)), clockwise seen from +z for q B > 0."""
    B0, dt = 2.0, 0.1
    u0 = np.array([0.7, -0.2, 0.3])
    gamma = math.sqrt(1 + u0 @ u0)
    theta = 2 * math.atan(q * B0 * dt / (2 * m * gamma))
    p = m * u0
    for n in range(1, 201):
        p = oracle.boris(q, m, dt, [0, 0, 0], [0, 0, B0], p)
        u = p / m
        assert abs(math.sqrt(u @ u) - math.sqrt(u0 @ u0)) < 1e-14
        np.testing.assert_allclose(u, _rot(u0, n * theta), rtol=0, atol=1e-13)
    # phase error relative to the exact gyro-frequency: tan(omega_c dt / 2) law
    wc = q * B0 / (m * gamma)
    assert abs(math.tan(theta / 2) - wc * dt / 2) < 1e-15


def test_boris_gyration_in_sim():
    """Same pin through the full cycle: a zero-weight particle in a uniform
    field on the grid (Yee keeps uniform fields; gather of a uniform field is
    exact by the partition of unity)."""
    B0, dt = 1.5, 0.02
    sim = OracleSim(3, (8, 8, 8), (0.1, 0.1, 0.1), dt, 2)
    sim.set_field(BZ, B0)
    u0 = np.array([0.3, 0.4, 0.1])
    sim.add_species(-1.0, 1.0, [0.37], [0.41], [0.33], [u0[0]], [u0[1]], [u0[2]], [0.0])
    gamma = math.sqrt(1 + u0 @ u0)
    theta = 2 * math.atan(-1.0 * B0 * dt / (2 * gamma))
    sim.step(50)
    p = sim.particles()
    u = np.array([p["ux"][0], p["uy"][0], p["uz"][0]])
    np.testing.assert_allclose(u, _rot(u0, 50 * theta), rtol=0, atol=1e-13)
    np.testing.assert_array_equal(sim.get_field(BZ), B0)


def test_boris_exb_drift():
    """E = E0 y, B = B0 z: the mean velocity tends to E x B / B^2 = (E0/B0) x
    for either charge sign; nonrelativistic drift 1e-3 so gamma corrections
    are ~1e-6; mean taken over whole numbers of discrete gyro-turns."""
    E0, B0, dt = 1e-3, 1.0, 0.05
    for q in (1.0, -1.0):
        p = np.zeros(3)
        theta = 2 * math.atan(B0 * dt / 2)
        nper = 2 * math.pi / theta
        nsteps = int(round(20 * nper))
        vs = []
        for _ in range(nsteps):
            p = oracle.boris(q, 1.0, dt, [0, E0, 0], [0, 0, B0], p)
            vs.append(p / math.sqrt(1 + p @ p))
        vmean = np.mean(vs, axis=0)
        assert abs(vmean[0] - E0 / B0) < 2e-3 * (E0 / B0) + 1e-3 * E0 / B0 * (nper / nsteps) * 10
        assert abs(vmean[1]) < 0.05 * E0 / B0
        assert abs(vmean[2]) == 0.0


def test_boris_exb_fixed_point():
    """Nonrelativistic limit: u = E x B / B^2 is a fixed point of the Boris
    map (the electric and magnetic forces cancel at the time-centred u)."""
    E0, B0, dt = 1e-6, 0.5, 0.3
    vd = E0 / B0
    p = np.array([vd, 0.0, 0.0])
    for _ in range(100):
        p = oracle.boris(-1.0, 1.0, dt, [0, E0, 0], [0, 0, B0], p)
    assert abs(p[0] - vd) < 1e-9 * vd
    assert abs(p[1]) < 1e-9 * vd


# ---------------------------------------------------------------- Yee dispersion (§2, ref [9])
def _yee_mode(sim, kvec, e_amp, t):
    """Real plane-wave eigenmode of the split Yee scheme at integer step t.

    Every operator of the scheme acts on exp(i k.x) as i*kappa with
    kappa_a = (2/dx_a) sin(k_a dx_a / 2) when each component sits at its own
    Yee location; leap-frog in time gives Omega = (2/dt) sin(w dt/2) = |kappa|.
    B = kappa x E / Omega at half steps; B at integer steps is the mean of
    the two neighbouring half-step values, which multiplies it by cos(w dt/2).
    """
    d = np.array(sim.d)
    dims = sim.dims
    kap = 2.0 / d * np.sin(kvec * d / 2.0)
    if dims == 2:
        kap[2] = 0.0
    Om = np.linalg.norm(kap)
    w = 2.0 / sim.dt * math.asin(sim.dt * Om / 2.0)
    b_amp = np.cross(kap, e_amp) / Om
    nz, ny, nx = sim.shape3
    k_, j_, i_ = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    out = {}
    stagE = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5)]
    stagB = [(0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]
    for c in range(3):
        for stag, amp, key, fac in ((stagE[c], e_amp[c], EX + c, 1.0),
                                    (stagB[c], b_amp[c], BX + c, math.cos(w * sim.dt / 2))):
            ph = kvec[0] * (i_ + stag[0]) * d[0] + kvec[1] * (j_ + stag[1]) * d[1]
            if dims == 3:
                ph = ph + kvec[2] * (k_ + stag[2]) * d[2]
            out[key] = fac * amp * np.cos(ph - w * t * sim.dt)
    return out, w


@pytest.mark.parametrize("dims", [2, 3])
def test_yee_dispersion(dims):
    n = (16, 12, 10) if dims == 3 else (16, 12, 1)
    d = (0.1, 0.13, 0.07) if dims == 3 else (0.1, 0.13, 1.0)
    lim = 1.0 / math.sqrt(sum(1.0 / x ** 2 for x in d[:dims]))
    sim = OracleSim(dims, n, d, 0.9 * lim, 2)
    m = np.array([3, -2, 1]) if dims == 3 else np.array([3, -2, 0])
    kvec = 2 * math.pi * m / (np.array(n) * np.array(d))
    if dims == 2:
        kvec[2] = 0.0
    kap = 2.0 / np.array(d) * np.sin(kvec * np.array(d) / 2.0)
    if dims == 2:
        kap[2] = 0.0
    # polarisation perpendicular to the discrete wave vector (discrete div E = 0)
    e_amp = np.cross(kap, [0.3, 0.5, 1.0])
    e_amp /= np.linalg.norm(e_amp)
    init, w = _yee_mode(sim, kvec, e_amp, 0)
    for key, v in init.items():
        sim.set_field(key, v)
    nsteps = 40
    sim.field_step(nsteps)
    want, _ = _yee_mode(sim, kvec, e_amp, nsteps)
    for key, v in want.items():
        np.testing.assert_allclose(sim.get_field(key), v, rtol=0, atol=2e-12)
    # the continuous dispersion w = |k| would be visibly wrong
    assert abs(w - np.linalg.norm(kvec)) * nsteps * sim.dt > 1e-3


@pytest.mark.parametrize("frac,grows", [(1.02, True), (0.98, False)])
def test_courant_limit(frac, grows):
    """The Nyquist mode grows above (sum dx^-2)^(-1/2) and is bounded below it."""
    n, d = (8, 8, 8), (0.1, 0.1, 0.1)
    lim = 1.0 / math.sqrt(3.0 / 0.01)
    sim = OracleSim(3, n, d, frac * lim, 1)
    k_, j_, i_ = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    cb = (-1.0) ** (i_ + j_ + k_)
    sim.set_field(EX, cb)
    sim.set_field(EY, -cb)
    sim.field_step(300)
    amp = max(np.abs(sim.get_field(c)).max() for c in (EX, EY, EZ))
    assert (amp > 100.0) == grows
    if not grows:
        assert amp < 3.0


# ---------------------------------------------------------------- gather (§2)
@pytest.mark.parametrize("dims,order", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_gather_linear_field_exact(dims, order):
    """A field linear in x at its own Yee location is gathered exactly; this
    pins the half-cell stagger of every component."""
    n = (16, 16, 16) if dims == 3 else (16, 16, 1)
    d = (0.2, 0.3, 0.25) if dims == 3 else (0.2, 0.3, 1.0)
    sim = OracleSim(dims, n, d, 0.01, order)
    nz, ny, nx = sim.shape3
    k_, j_, i_ = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    stagE = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5)]
    stagB = [(0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]
    coef = np.array([[1.0, 2.0, -1.0, 0.5], [0.3, -1.0, 0.7, 2.0], [-0.4, 0.2, 1.1, -0.6],
                     [2.0, 0.1, 0.4, 0.9], [0.5, -0.7, -0.2, 1.3], [1.2, 0.6, 0.8, -1.5]])
    for c in range(6):
        st = stagE[c] if c < 3 else stagB[c - 3]
        x = (i_ + st[0]) * d[0]
        y = (j_ + st[1]) * d[1]
        z = (k_ + st[2]) * d[2] if dims == 3 else 0.0
        sim.set_field(EX + c, coef[c, 0] + coef[c, 1] * x + coef[c, 2] * y + coef[c, 3] * z)
    rng = np.random.default_rng(3)
    for _ in range(20):
        # stay 3 cells away from the periodic seam, where the field is not linear
        r = rng.uniform(3, 12, 3) * np.array(d)
        if dims == 2:
            r[2] = 0.0
        E, B = sim.gather(*r)
        F = np.concatenate([E, B])
        want = coef[:, 0] + coef[:, 1] * r[0] + coef[:, 2] * r[1] + coef[:, 3] * r[2]
        np.testing.assert_allclose(F, want, rtol=0, atol=1e-12)


# ---------------------------------------------------------------- deposit (§2 eq. 4 + continuity)
def _divJ(sim, J):
    Jx, Jy, Jz = J
    d = sim.d
    return ((Jx - np.roll(Jx, 1, axis=2)) / d[0] + (Jy - np.roll(Jy, 1, axis=1)) / d[1]
            + (Jz - np.roll(Jz, 1, axis=0)) / d[2])


def _divE(sim):
    d = sim.d
    Ex, Ey, Ez = (sim.get_field(c) for c in (EX, EY, EZ))
    return ((Ex - np.roll(Ex, 1, axis=2)) / d[0] + (Ey - np.roll(Ey, 1, axis=1)) / d[1]
            + (Ez - np.roll(Ez, 1, axis=0)) / d[2])


def test_deposit_cic_one_cell_closed_form():
    """CIC particle on a y,z node moving along x inside one cell: the only
    current is Jx(i+1/2) = q w vx (brute force of the definition)."""
    d = (0.1, 0.1, 0.1)
    dt = 0.02
    sim = OracleSim(3, (6, 6, 6), d, dt, 1)
    q, w = -1.0, 0.37
    r0 = np.array([2.2, 3.0, 1.0]) * 0.1
    r1 = np.array([2.7, 3.0, 1.0]) * 0.1
    sim.deposit_move(q, w, r0, r1)
    Jx, Jy, Jz = (sim.get_field(c) for c in (JX, JY, JZ))
    vx = (r1[0] - r0[0]) / dt
    want = np.zeros_like(Jx)
    want[1, 3, 2] = q * w * vx
    np.testing.assert_allclose(Jx, want, rtol=0, atol=1e-14)
    assert np.abs(Jy).max() < 1e-15 and np.abs(Jz).max() < 1e-15


def test_deposit_tsc_1d_closed_form():
    """TSC particle moving along x with nearest node n unchanged and y,z on
    nodes: Jx(n-1/2) = q w vx (1/2 - dbar), Jx(n+1/2) = q w vx (1/2 + dbar)
    with dbar the mean offset from node n (times the y,z weights 3/4 * 3/4 at
    the node and 1/8 at its neighbours)."""
    d = (0.1, 0.1, 0.1)
    dt = 0.02
    sim = OracleSim(3, (8, 8, 8), d, dt, 2)
    q, w = 1.0, 2.0
    X0, X1 = 4.1, 4.35
    r0 = np.array([X0, 3.0, 5.0]) * 0.1
    r1 = np.array([X1, 3.0, 5.0]) * 0.1
    sim.deposit_move(q, w, r0, r1)
    Jx = sim.get_field(JX)
    vx = (X1 - X0) * d[0] / dt
    dbar = 0.5 * ((X0 - 4) + (X1 - 4))
    wy = {2: 0.125, 3: 0.75, 4: 0.125}
    wz = {4: 0.125, 5: 0.75, 6: 0.125}
    want = np.zeros_like(Jx)
    for j, sy in wy.items():
        for k, sz in wz.items():
            want[k, j, 3] = q * w * vx * (0.5 - dbar) * sy * sz
            want[k, j, 4] = q * w * vx * (0.5 + dbar) * sy * sz
    np.testing.assert_allclose(Jx, want, rtol=0, atol=1e-13)


def _thermal(dims, order, n, ppc, uth, seed, dt_frac=0.95):
    from paper_1503_02464_gb300 import synth
    wl = synth.small(dims, n, order, ppc, uth, seed, dt_frac)
    sim = OracleSim(dims, wl.n, wl.d, wl.dt, order)
    sim.add_particles(wl.particles(0), -1.0, 1.0)
    return sim, wl


@pytest.mark.parametrize("dims,order", [(2, 1), (2, 2), (3, 1), (3, 2)])
def test_continuity_gauss_total_current(dims, order):
    """Per step: (rho1 - rho0)/dt + div J = 0 to round-off, div E - rho is
    conserved (zero from a neutral start), total charge is constant, and the
    grid sum of J equals sum q w v^{n+1/2} (eq. 4 integrated over space)."""
    n = (8, 8, 8) if dims == 3 else (16, 12)
    sim, wl = _thermal(dims, order, n, 4, 0.3, 11)
    sim.neutralize()
    dV = np.prod(sim.d)
    rho0 = sim.rho()
    assert np.abs(_divE(sim) - rho0).max() < 1e-12
    q0 = rho0.sum() * dV
    for step in range(5):
        rho0 = sim.rho()
        sim.step(1)
        rho1 = sim.rho()
        J = [sim.get_field(c) for c in (JX, JY, JZ)]
        scale = max(np.abs(x).max() for x in J) / min(sim.d[:dims])
        res = (rho1 - rho0) / sim.dt + _divJ(sim, J)
        assert np.abs(res).max() < 1e-12 * scale, (step, np.abs(res).max(), scale)
        assert np.abs(_divE(sim) - rho1).max() < 1e-11 * max(1.0, np.abs(rho1).max())
        assert abs(rho1.sum() * dV - q0) < 1e-12 * abs(rho1).sum() * dV + 1e-14
        p = sim.particles()
        g = np.sqrt(1 + p["ux"] ** 2 + p["uy"] ** 2 + p["uz"] ** 2)
        for c, key in enumerate(("ux", "uy", "uz")):
            if dims == 2 and c == 2:
                want = (-1.0 * p["w"] * p["uz"] / g).sum()
            elif c < dims:
                want = (-1.0 * p["w"] * p[key] / g).sum()
            else:
                continue
            got = J[c].sum()
            assert abs(got - want) < 1e-12 * np.abs(p["w"] * p[key] / g).sum(), (c, got, want)


def test_straight_line_and_stationary():
    """Zero fields: straight-line motion; a particle at rest deposits no current."""
    d = (0.1, 0.1, 0.1)
    dt = 0.04
    sim = OracleSim(3, (8, 8, 8), d, dt, 2)
    u = np.array([0.3, -0.2, 0.1])
    sim.add_species(1.0, 1.0, [0.33], [0.44], [0.55], [u[0]], [u[1]], [u[2]], [0.0])
    sim.add_species(1.0, 1.0, [0.31], [0.42], [0.53], [0.0], [0.0], [0.0], [1.0])
    sim.step(7)
    p = sim.particles(0)
    v = u / math.sqrt(1 + u @ u)
    np.testing.assert_allclose([p["x"][0], p["y"][0], p["z"][0]],
                               np.array([0.33, 0.44, 0.55]) + 7 * dt * v, rtol=0, atol=1e-15)
    for c in (JX, JY, JZ):
        assert np.abs(sim.get_field(c)).max() == 0.0


def test_cold_plasma_oscillation():
    """Long-wavelength cold Langmuir oscillation: leap-frog frequency obeys
    sin(w dt/2) = w_p dt/2 with w_p = 1 for n = 1 electrons (§ units)."""
    nx, ny = 64, 4
    d = (0.2, 0.2)
    dt = 0.1
    sim = OracleSim(2, (nx, ny), d, dt, 2)
    from paper_1503_02464_gb300 import synth
    cells = np.arange(nx * ny)
    p = synth.particles_for_cells(cells, (nx, ny, 1), (0.2, 0.2, 1.0), 4, 0.0, 1.0, 77, 2)
    # quiet start: regular positions, small sinusoidal velocity
    i = cells.repeat(4) % nx
    j = cells.repeat(4) // nx
    s = np.tile(np.arange(4), nx * ny)
    p["x"] = (i + 0.125 + 0.25 * s) * d[0]
    p["y"] = (j + 0.5) * d[1]
    L = nx * d[0]
    p["ux"] = 1e-4 * np.sin(2 * math.pi * p["x"] / L)
    sim.add_particles(p, -1.0, 1.0)
    sim.neutralize()
    ue = []
    for _ in range(400):
        sim.step(1)
        ue.append(sim.diag()["energy_e"])
    ue = np.array(ue)
    # electric energy oscillates at twice the plasma frequency: find its minima
    mins = [t for t in range(1, len(ue) - 1) if ue[t] < ue[t - 1] and ue[t] <= ue[t + 1]]
    per = 2 * (mins[-1] - mins[0]) / (len(mins) - 1) * dt
    w = 2 * math.pi / per
    kdx = 2 * math.pi / nx
    w_theory = 2 / dt * math.asin(dt / 2)
    assert abs(w - w_theory) / w_theory < 0.02, (w, w_theory)
    assert kdx < 0.1


# ---------------------------------------------------------------- deposit moments (§2 eq. 4)
def _path_moments(X0, X1, a, b):
    """Time averages over a straight move of 1, x_a, x_b and x_a x_b."""
    p0, p1 = X0[a], X1[a]
    q0, q1 = X0[b], X1[b]
    return (1.0, 0.5 * (p0 + p1), 0.5 * (q0 + q1),
            p0 * q0 + 0.5 * (p0 * (q1 - q0) + (p1 - p0) * q0) + (p1 - p0) * (q1 - q0) / 3.0)


def check_transverse_moments(dims, order, seed=3, nmoves=12):
    """One straight move from X0 to X1 (in cells, |X1 - X0| < 1 per axis).

    The charge-conserving current of a component, summed along its own
    axis (or, for the out-of-plane Jz of 2D3V, taken as it is), equals
    q w v_c times transverse node weights that are the time average, over
    the move, of the products of linearly interpolated node weights
    S0 + t (S1 - S0).  Sampled CIC and TSC weights reproduce constants and
    linear functions exactly (sum_i S(X - i) = 1, sum_i i S(X - i) = X), so
    the weights' moments are path averages:
        sum T = 1,  sum j T = <Y>,  sum k T = <Z>,  sum j k T = <Y Z>
    with <Y Z> = Y0 Z0 + (Y0 dZ + dY Z0)/2 + dY dZ / 3 on the path.  A wrong
    1/3 or 1/2 in the bracket, a dropped term, or the end-point shapes used
    in place of the average all change one of these."""
    rng = np.random.default_rng(seed)
    n = (16, 16, 16) if dims == 3 else (16, 16)
    d = np.array([0.1, 0.13, 0.07])
    dt = 0.02
    for _ in range(nmoves):
        sim = OracleSim(dims, n, tuple(d[:dims]), dt, order)
        X0 = 6.0 + 3.0 * rng.random(3)
        X1 = X0 + rng.uniform(-0.95, 0.95, 3)
        if dims == 2:
            X0[2] = X1[2] = 0.0
        q, w, vz_2d = -1.0 + 2.0 * rng.random(), 0.2 + rng.random(), rng.uniform(-0.8, 0.8)
        sim.deposit_move(q, w, X0 * d, X1 * d, vz_2d)
        v = (X1 - X0) * d / dt
        nz, ny, nx = sim.shape3
        k_, j_, i_ = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        pos = (i_.astype(float), j_.astype(float), k_.astype(float))
        comps = [(JX, 0, 1, 2), (JY, 1, 2, 0), (JZ, 2, 0, 1)] if dims == 3 else [(JZ, 2, 0, 1)]
        for key, c, a, b in comps:
            J = sim.get_field(key)
            qv = q * w * (v[c] if dims == 3 else vz_2d)
            want = _path_moments(X0, X1, a, b)
            got = (J.sum(), (J * pos[a]).sum(), (J * pos[b]).sum(), (J * pos[a] * pos[b]).sum())
            for g, m in zip(got, want):
                assert abs(g - qv * m) <= 1e-12 * abs(qv) * max(1.0, abs(m)), (key, g, qv * m)
        sim.close()


@pytest.mark.parametrize("order", [1, 2])
def test_jz_2d3v_moments(order):
    """The out-of-plane current of 2D3V, which the continuity equation does
    not constrain (nothing varies along z), against the path averages of 1,
    x, y and x y."""
    check_transverse_moments(2, order)


@pytest.mark.parametrize("order", [1, 2])
def test_j3d_transverse_moments(order):
    check_transverse_moments(3, order)


# ---------------------------------------------------------------- energy diagnostics
def check_field_energy_of_eigenmode(dims):
    """A travelling vacuum plane wave (an exact eigenvector of the split Yee
    update) has, at every integer step, electric energy (1/2) dV (N/2) |E0|^2
    and magnetic energy (1/2) dV (N/2) |B0|^2 cos^2(w dt/2): over the whole
    periodic grid, sum cos^2(k.x - w t) = N/2 at any phase when 2k is not a
    multiple of the grid's reciprocal lattice."""
    n = (16, 12, 10) if dims == 3 else (16, 12, 1)
    d = (0.1, 0.13, 0.07) if dims == 3 else (0.1, 0.13, 1.0)
    lim = 1.0 / math.sqrt(sum(1.0 / x ** 2 for x in d[:dims]))
    sim = OracleSim(dims, n, d, 0.9 * lim, 2)
    m = np.array([3, -2, 1]) if dims == 3 else np.array([3, -2, 0])
    kvec = 2 * math.pi * m / (np.array(n) * np.array(d))
    kap = 2.0 / np.array(d) * np.sin(kvec * np.array(d) / 2.0)
    if dims == 2:
        kvec[2] = kap[2] = 0.0
    e_amp = np.cross(kap, [0.3, 0.5, 1.0])
    e_amp *= 0.7 / np.linalg.norm(e_amp)
    init, w = _yee_mode(sim, kvec, e_amp, 0)
    for key, val in init.items():
        sim.set_field(key, val)
    Om = np.linalg.norm(kap)
    b_amp = np.cross(kap, e_amp) / Om * math.cos(w * sim.dt / 2)
    ncell = n[0] * n[1] * n[2]
    dV = d[0] * d[1] * (d[2] if dims == 3 else 1.0)
    want_e = 0.5 * dV * 0.5 * ncell * float(e_amp @ e_amp)
    want_b = 0.5 * dV * 0.5 * ncell * float(b_amp @ b_amp)
    for steps in (0, 7, 13):
        if steps:
            sim.field_step(steps)
        dg = sim.diag()
        assert abs(dg["energy_e"] - want_e) < 1e-12 * want_e, (steps, dg["energy_e"], want_e)
        assert abs(dg["energy_b"] - want_b) < 1e-12 * want_b, (steps, dg["energy_b"], want_b)
        assert abs(dg["energy_field"] - want_e - want_b) < 1e-12 * (want_e + want_b)
    sim.close()


@pytest.mark.parametrize("dims", [2, 3])
def test_field_energy_of_vacuum_eigenmode(dims):
    check_field_energy_of_eigenmode(dims)


def check_kinetic_energy_of_cold_beams(dims):
    """Uniform cold beams of density n_s and momentum u_s per unit mass in a
    box of volume V carry kinetic energy sum_s n_s V m_s (gamma_s - 1)
    (relativistic: u = 1 gives gamma - 1 = 0.414, not u^2/2 = 0.5)."""
    from paper_1503_02464_gb300 import synth
    n = (6, 5, 4) if dims == 3 else (8, 6)
    d = (0.11, 0.07, 0.05) if dims == 3 else (0.11, 0.07)
    sim = OracleSim(dims, n, d, 0.01, 2)
    n3 = tuple(list(n) + [1] * (3 - len(n)))
    d3 = tuple(list(d) + [1.0] * (3 - len(d)))
    cells = np.arange(n3[0] * n3[1] * n3[2])
    V = float(np.prod(np.array(n3) * np.array(d3)))
    want = 0.0
    for (q, mass, dens, u, ppc, seed) in ((-1.0, 1.0, 2.5, (1.0, 0.0, 0.0), 3, 5),
                                          (1.0, 1836.0, 2.5, (0.0, -0.02, 0.01), 2, 6)):
        p = synth.particles_for_cells(cells, n3, d3, ppc, 0.0, dens, seed, dims)
        for key, val in zip(("ux", "uy", "uz"), u):
            p[key] = np.full(len(p["x"]), val)
        sim.add_particles(p, q, mass)
        want += dens * V * mass * (math.sqrt(1.0 + sum(x * x for x in u)) - 1.0)
    got = sim.diag()["energy_kinetic"]
    assert abs(got - want) < 1e-12 * want, (got, want)
    sim.close()


@pytest.mark.parametrize("dims", [2, 3])
def test_kinetic_energy_of_cold_beams(dims):
    check_kinetic_energy_of_cold_beams(dims)


def check_langmuir_energy_exchange():
    """A small cold Langmuir oscillation trades kinetic for electric energy:
    over whole periods the kinetic energy (centred at integer steps as the
    mean of the two half-step values) and the electric energy swing by the
    same amount, and their sum is conserved, both to O((w_p dt)^2) (here
    w_p dt = 0.1).  A missing 1/2 or dV in either energy breaks the balance."""
    nx, ny = 64, 4
    d = (0.2, 0.2)
    dt = 0.1
    sim = OracleSim(2, (nx, ny), d, dt, 2)
    from paper_1503_02464_gb300 import synth
    cells = np.arange(nx * ny)
    p = synth.particles_for_cells(cells, (nx, ny, 1), (0.2, 0.2, 1.0), 4, 0.0, 1.0, 77, 2)
    i = cells.repeat(4) % nx
    j = cells.repeat(4) // nx
    s = np.tile(np.arange(4), nx * ny)
    p["x"] = (i + 0.125 + 0.25 * s) * d[0]
    p["y"] = (j + 0.5) * d[1]
    p["ux"] = 1e-3 * np.sin(2 * math.pi * p["x"] / (nx * d[0]))
    sim.add_particles(p, -1.0, 1.0)
    sim.neutralize()
    kin, ue, ub = [], [], []
    for _ in range(128):
        sim.step(1)
        dg = sim.diag()
        kin.append(dg["energy_kinetic"])
        ue.append(dg["energy_e"])
        ub.append(dg["energy_b"])
    kin, ue, ub = np.array(kin), np.array(ue), np.array(ub)
    kc = 0.5 * (kin[:-1] + kin[1:])  # kinetic energy at the integer step of ue[:-1]
    tot = kc + ue[:-1] + ub[:-1]
    swing_k, swing_e = kc.max() - kc.min(), ue.max() - ue.min()
    assert swing_e > 0.0 and abs(swing_k / swing_e - 1.0) < 0.02, (swing_k, swing_e)
    assert (tot.max() - tot.min()) < 0.02 * swing_e, (tot.max() - tot.min(), swing_e)
    sim.close()


def test_langmuir_energy_exchange():
    check_langmuir_energy_exchange()
