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
