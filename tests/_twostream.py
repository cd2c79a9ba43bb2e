"""Two-stream instability set-up shared by the oracle pin and the GPU tests.

Two cold electron beams with drift momenta +-u0 along x, each of density
1/2 (so the total plasma frequency is 1), over an immobile background of
charge +1, periodic box.  The linear theory of the cold, relativistic,
electrostatic case: with v = u0/gamma0 and each beam's longitudinal plasma
frequency w1^2 = (1/2)/gamma0^3 (the longitudinal mass is gamma0^3 m), the
dispersion relation 1 = w1^2/(w - k v)^2 + w1^2/(w + k v)^2 is a quadratic
in w^2 whose smaller root is negative for (k v)^2 < 2 w1^2; the growth rate
is then

    gamma(k)^2 = w1 sqrt(w1^2 + 4 (k v)^2) - (k v)^2 - w1^2,

largest (= w1/2, i.e. omega_p / (2 sqrt 2) in the non-relativistic limit) at
k v = (sqrt 3 / 2) w1.  This is the test problem of the paper's scaling runs
(§4.1); the closed form is textbook plasma physics, independent of the PIC
method, which makes it a pin for the whole cycle: gather, push, move,
deposit and Yee together must reproduce it.
"""
import math

import numpy as np

import oracle
from paper_1503_02464_gb300 import synth


def growth_rate(k: float, u0: float) -> float:
    g0 = math.sqrt(1.0 + u0 * u0)
    v = u0 / g0
    w1 = math.sqrt(0.5 / g0 ** 3)
    b2 = (k * v) ** 2
    return math.sqrt(max(w1 * math.sqrt(w1 * w1 + 4.0 * b2) - b2 - w1 * w1, 0.0))


def k_fastest(u0: float) -> float:
    g0 = math.sqrt(1.0 + u0 * u0)
    return math.sqrt(3.0) / 2.0 * math.sqrt(0.5 / g0 ** 3) / (u0 / g0)


def eigen_seeds(k: float, u0: float, amp: float):
    """Beam perturbations of the growing eigenmode with Ex = amp cos(k x) at
    t = 0 (linear cold-fluid theory, Lagrangian displacement xi of each
    beam): (d/dt +- v d/dx)^2 xi = -E / gamma0^3 gives, for w = i gamma,
    xi = amp / (gamma0^3 (w -+ k v)^2) and a velocity change
    (gamma +- i k v) xi, i.e. a momentum change gamma0^3 times that.
    Returned as the two synth ``perturb`` tuples (mode 1)."""
    g0 = math.sqrt(1.0 + u0 * u0)
    v = u0 / g0
    gam = growth_rate(k, u0)
    out = []
    for sgn in (1.0, -1.0):
        xi = amp / (g0 ** 3 * (1j * gam - sgn * k * v) ** 2)
        du = g0 ** 3 * (gam + sgn * 1j * k * v) * xi
        out.append((1, abs(xi), float(np.angle(xi)), abs(du), float(np.angle(du))))
    return tuple(out)


def workload(n, u0=0.2, k_frac=1.0, lattice=(4, 2), amp=1e-6, order=2):
    """Box of one wavelength 2 pi / k, k = k_frac * k_fastest, n cells, the
    growing mode seeded with Ex amplitude ``amp`` (unstable k) or, for a
    stable k, both beams displaced by amp cos(k x)."""
    k = k_frac * k_fastest(u0)
    L = 2.0 * math.pi / k
    d = L / n[0]
    if growth_rate(k, u0) > 0.0:
        seeds = eigen_seeds(k, u0, amp)
    else:
        seeds = ((1, amp, 0.0, 0.0, 0.0),) * 2
    return synth.two_stream(tuple(n), d, u0, lattice, seeds, order=order), L


def gauss_ex(wl, parts_list) -> np.ndarray:
    """Ex satisfying the discrete Gauss law for the loaded charge plus the
    +1 background (charge varies along x only): Ex(i+1/2) - Ex(i-1/2) =
    dx rho_i, zero mean.  Computed from the oracle's charge deposit."""
    o = oracle.OracleSim(wl.dims, wl.n, wl.d, wl.dt, wl.order)
    for sp, p in zip(wl.species, parts_list):
        o.add_particles(p, sp.q, sp.m)
    o.set_background(np.ones(o.shape3))
    r = o.rho().mean(axis=(0, 1))  # average over z, y
    ex = np.cumsum(r) * wl.d[0]
    ex -= ex.mean()
    o.close()
    return np.broadcast_to(ex, (wl.n[2], wl.n[1], wl.n[0])).copy()


def mode_amplitude(ex: np.ndarray) -> float:
    """|first Fourier coefficient| of the y/z-averaged Ex along x."""
    e = ex.mean(axis=(0, 1))
    nx = e.size
    xs = np.arange(nx) + 0.5
    return float(abs((e * np.exp(-2j * math.pi * xs / nx)).sum()) * 2.0 / nx)


def fit_rate(ts, amps, t0, t1) -> float:
    ts, amps = np.asarray(ts), np.asarray(amps)
    m = (ts >= t0) & (ts <= t1)
    return float(np.polyfit(ts[m], np.log(amps[m]), 1)[0])
