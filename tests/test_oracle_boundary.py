"""Pins of the oracle's boundary readings (CPU only).

The paper names boundary conditions and laser injection but gives no
formulas (§2); the oracle reads them as first-order Mur walls in x with the
laser entering as the incoming wave at x = 0.  These checks pin that reading
to physics fixed independently of the code: a plane pulse enters with the
requested amplitude and transverse profile, travels at c, and leaves through
the far wall with a small first-order Mur reflection.  Bit-level parity of
the boundary arithmetic is otherwise only against the oracle itself.
"""
import math

import numpy as np

from oracle import OracleSim, EY, EZ, BZ

TAU = 2 * math.pi


def _pulse_sim(nx=600, ny=4, d=0.2, a0=1.0, waist=1e9, duration=2 * TAU, pol=1):
    dt = 0.9 * d / math.sqrt(2)
    sim = OracleSim(2, (nx, ny), (d, d), dt, 2)
    sim.set_absorbing_x(True)
    sim.set_laser(a0, waist, duration, pol=pol)
    return sim


def test_laser_enters_with_amplitude_and_speed():
    sim = _pulse_sim()
    probe_i = 200
    x_probe = probe_i * 0.2
    trace = []
    nsteps = int((x_probe + 2 * TAU + 10) / sim.dt)
    for n in range(nsteps):
        sim.field_step(1)
        trace.append(sim.get_field(EY)[0, 2, probe_i])
    trace = np.array(trace)
    t = (np.arange(nsteps) + 1) * sim.dt
    # the travelling wave a0 sin^2(pi tau / T) sin(tau), tau = t - x / c
    tau = t - x_probe
    D = 2 * TAU
    want = np.where((tau > 0) & (tau < D), np.sin(np.pi * tau / D) ** 2 * np.sin(tau), 0.0)
    assert abs(np.abs(trace).max() - np.abs(want).max()) < 0.03 * np.abs(want).max()
    assert np.abs(trace - want).max() < 0.1  # small Yee phase error over 200 cells
    # centre of the envelope arrives at x_probe / c + duration / 2
    centre = (t * trace ** 2).sum() / (trace ** 2).sum()
    assert abs(centre - (x_probe + TAU)) < 0.5, centre


def test_mur_wall_absorbs_pulse():
    sim = _pulse_sim(nx=300)
    energies = []
    L = 300 * 0.2
    nsteps = int((L + 2 * TAU + 20) / sim.dt)
    for n in range(nsteps):
        sim.field_step(1)
        if n % 10 == 0:
            energies.append(sim.diag()["energy_field"])
    peak = max(energies)
    assert peak > 0
    assert energies[-1] < 1e-4 * peak, (energies[-1], peak)


def test_transverse_profile_at_entrance():
    ny, d, w0 = 64, 0.2, 3.0
    sim = OracleSim(2, (200, ny), (d, d), 0.9 * d / math.sqrt(2), 2)
    sim.set_absorbing_x(True)
    sim.set_laser(1.0, w0, 4 * TAU, pol=1)
    best = np.zeros(ny)
    for n in range(int(3 * TAU / sim.dt)):
        sim.field_step(1)
        best = np.maximum(best, np.abs(sim.get_field(EY)[0, :, 5]))
    y = (np.arange(ny) + 0.5) * d
    yc = 0.5 * ny * d
    prof = best / best.max()
    want = np.exp(-((y - yc) / w0) ** 2)
    assert np.abs(prof - want).max() < 0.05


def test_particle_removed_at_absorbing_wall():
    nx = 32
    sim = OracleSim(2, (nx, 8), (0.1, 0.1), 0.06, 2)
    sim.set_absorbing_x(True)
    u = 3.0  # v close to c: crosses a cell in ~2 steps
    sim.add_species(-1.0, 1.0, [0.1 * (nx - 6)], [0.4], None, [u], [0.0], [0.0], [0.5])
    alive = []
    for n in range(12):
        sim.step(1)
        alive.append(sim.diag()["n_alive"])
    assert alive[0] == 1 and alive[-1] == 0
    v = u / math.sqrt(1 + u * u)
    # removed on the first step whose new position reaches nx - 4 cells
    steps_to_wall = math.ceil((2.0 * 0.1) / (v * 0.06))
    assert alive.index(0) + 1 == steps_to_wall


# ---- oblique incidence: a Gaussian beam tilted by `angle` in the x-y plane ----

def _oblique_sim(angle, pol, nx=220, ny=256, d=0.2, w0=4.0, duration=4 * TAU):
    dt = 0.9 * d / math.sqrt(2)
    sim = OracleSim(2, (nx, ny), (d, d), dt, 2)
    sim.set_absorbing_x(True)
    sim.set_laser(1.0, w0, duration, pol=pol, angle=angle)
    return sim


def _traces(sim, points, comp, nsteps):
    """Time traces of one field component at the given (i, j) nodes."""
    out = np.zeros((len(points), nsteps))
    for n in range(nsteps):
        sim.field_step(1)
        f = sim.get_field(comp)[0]
        for p, (i, j) in enumerate(points):
            out[p, n] = f[j, i]
    return out


def _centroid(t, tr):
    e = tr ** 2
    return (t * e).sum() / e.sum()


def test_oblique_pulse_travels_along_its_direction():
    """The envelope of an s-polarised oblique pulse crosses points on the beam
    axis at c along (cos a, sin a): arrival times grow by the path length, and
    the on-axis amplitude follows a 2D Gaussian beam, a0 (w0 / w(s))^(1/2)
    with w(s) = w0 (1 + (s / z_R)^2)^(1/2), z_R = w0^2 / 2 (wavenumber 1)."""
    a = math.radians(15.0)
    w0 = 8.0
    sim = _oblique_sim(a, 2, w0=w0)
    d = 0.2
    yc = 0.5 * 256 * d
    y0 = 0.0  # fronts reach the y = 0 edge first for a > 0
    pts, s_axis = [], []
    for s in (6.0, 14.0, 22.0):  # distance along the axis
        x, y = s * math.cos(a), yc + s * math.sin(a)
        pts.append((int(round(x / d)), int(round(y / d))))  # Ez nodes sit at (i, j)
        s_axis.append(s)
    nsteps = int((25.0 + 4 * TAU + 8.0) / sim.dt)
    tr = _traces(sim, pts, EZ, nsteps)
    t = (np.arange(nsteps) + 1) * sim.dt
    cen = [_centroid(t, tr[p]) for p in range(len(pts))]
    # the envelope centre is at tau = duration / 2: t = duration/2 + k.(x, y - y0)
    for (i, j), c in zip(pts, cen):
        want = 2 * TAU + i * d * math.cos(a) + (j * d - y0) * math.sin(a)
        assert abs(c - want) < 0.5, (i, j, c, want)
    speed = (s_axis[2] - s_axis[0]) / (cen[2] - cen[0])
    assert abs(speed - 1.0) < 0.01, speed
    zr = 0.5 * w0 * w0
    for p, sa in enumerate(s_axis):
        want = (1.0 + (sa / zr) ** 2) ** -0.25
        assert abs(np.abs(tr[p]).max() - want) < 0.03, (sa, np.abs(tr[p]).max(), want)


def test_oblique_fronts_delay_along_the_wall():
    """Two points at the same x, dy apart, see the pulse dy sin(a) apart in
    time (the tilt of the phase fronts)."""
    a = math.radians(-20.0)
    sim = _oblique_sim(a, 2)
    d = 0.2
    jc = 128
    i = 40
    pts = [(i, jc - 10), (i, jc + 10)]
    nsteps = int((i * d + 4 * TAU + 12.0) / sim.dt)
    tr = _traces(sim, pts, EZ, nsteps)
    t = (np.arange(nsteps) + 1) * sim.dt
    dt_arr = _centroid(t, tr[1]) - _centroid(t, tr[0])
    want = 20 * d * math.sin(a)
    assert abs(dt_arr - want) < 0.05, (dt_arr, want)


def test_oblique_p_polarisation_is_transverse():
    """E of a p-polarised oblique wave lies across its direction:
    |Ex| / |Ey| = tan(a) on the beam axis inside the box."""
    a = math.radians(25.0)
    w0 = 8.0
    sim = _oblique_sim(a, 1, w0=w0)
    d = 0.2
    yc = 0.5 * 256 * d
    s = 12.0
    x, y = s * math.cos(a), yc + s * math.sin(a)
    i, j = int(round(x / d)), int(round(y / d))
    nsteps = int((s + 4 * TAU + 6.0) / sim.dt)
    ex = np.zeros(nsteps)
    ey = np.zeros(nsteps)
    for n in range(nsteps):
        sim.field_step(1)
        ex[n] = sim.get_field(0)[0, j, i]   # Ex at (i + 1/2, j)
        ey[n] = sim.get_field(EY)[0, j, i]  # Ey at (i, j + 1/2)
    ratio = np.abs(ex).max() / np.abs(ey).max()
    assert abs(ratio - math.tan(a)) < 0.03 * math.tan(a) + 0.01, (ratio, math.tan(a))
    # the field's magnitude on the axis: a0 times the 2D beam's (w0 / w(s))^(1/2)
    want = (1.0 + (s / (0.5 * w0 * w0)) ** 2) ** -0.25
    assert abs(math.hypot(np.abs(ex).max(), np.abs(ey).max()) - want) < 0.03


def test_zero_angle_is_normal_incidence():
    """angle = 0 gives the normal-incidence wave exactly (same arithmetic)."""
    s0 = _oblique_sim(0.0, 1, nx=64, ny=16, w0=2.0, duration=2 * TAU)
    s1 = OracleSim(2, (64, 16), (0.2, 0.2), 0.9 * 0.2 / math.sqrt(2), 2)
    s1.set_absorbing_x(True)
    s1.set_laser(1.0, 2.0, 2 * TAU, pol=1)
    for _ in range(40):
        s0.field_step(1)
        s1.field_step(1)
    assert np.array_equal(s0.get_field(EY), s1.get_field(EY))


def test_oblique_pulse_3d_profile_and_direction():
    """3D: a tilted s-polarised pulse enters with the Gaussian profile across
    z (its direction lies in the x-y plane) and crosses the axis at c."""
    a = math.radians(20.0)
    d, w0 = 0.25, 5.0   # Rayleigh length w0^2 / 2 = 12.5: little diffraction over the probes
    n = (64, 128, 96)
    dt = 0.9 * d / math.sqrt(3)
    sim = OracleSim(3, n, (d, d, d), dt, 2)
    sim.set_absorbing_x(True)
    sim.set_laser(1.0, w0, 4 * TAU, pol=2, angle=a)
    yc, zc = 0.5 * n[1] * d, 0.5 * n[2] * d
    # Ez nodes at (i, j, k + 1/2); probe the axis at two distances s
    pts = []
    for s in (2.0, 8.0):
        x, y = s * math.cos(a), yc + s * math.sin(a)
        pts.append((int(round(x / d)), int(round(y / d))))
    kc = int(round(zc / d - 0.5))
    nsteps = int((8.0 + 4 * TAU + 4.0) / dt)
    tr = np.zeros((2, nsteps))
    best_z = np.zeros(n[2])
    for m in range(nsteps):
        sim.field_step(1)
        ez = sim.get_field(EZ)
        for p, (i, j) in enumerate(pts):
            tr[p, m] = ez[kc, j, i]
        i0, j0 = pts[0]
        best_z = np.maximum(best_z, np.abs(ez[:, j0, i0]))
    t = (np.arange(nsteps) + 1) * dt
    c0, c1 = _centroid(t, tr[0]), _centroid(t, tr[1])
    path = math.hypot((pts[1][0] - pts[0][0]) * d, (pts[1][1] - pts[0][1]) * d)
    # a focused 3D pulse travels on its axis slower than c by up to about
    # 2 / (k w0)^2 = 8 % here (the 2D test pins the speed to 1 % on a wider beam)
    assert 0.9 < path / (c1 - c0) < 1.0, path / (c1 - c0)
    # across z the beam is Gaussian, exp(-(z - zc)^2 / w(s)^2), w(s) = w0 (1 + (s / z_R)^2)^(1/2)
    z = (np.arange(n[2]) + 0.5) * d
    prof = best_z / best_z.max()
    w = w0 * math.sqrt(1.0 + (2.0 / (0.5 * w0 * w0)) ** 2)
    want = np.exp(-((z - zc) / w) ** 2)
    assert np.abs(prof - want).max() < 0.05
