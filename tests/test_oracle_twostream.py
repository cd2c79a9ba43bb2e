"""Pin of the whole oracle cycle against the cold two-stream instability
(the test problem of the paper's scaling study, §4.1): seeded with the
growing eigenmode of linear theory, the mode's field amplitude follows
A exp(gamma t) with gamma from the closed form of the cold relativistic
two-beam dispersion relation.

A sign error in the Boris electric kick, a dropped term of the Esirkepov
current, a wrong gather weight or a missing longitudinal mass factor
(gamma0^3, a 3 % change of gamma here) each move the measured rate outside
the 1.5 % band; the run ends far below the trapping amplitude.
"""
import numpy as np
import pytest

import oracle

from _twostream import fit_rate, gauss_ex, growth_rate, mode_amplitude, workload

TMAX = 20.0


def _run_oracle(wl, tmax):
    parts = [wl.particles(i) for i in range(len(wl.species))]
    o = oracle.OracleSim(wl.dims, wl.n, wl.d, wl.dt, wl.order)
    for sp, p in zip(wl.species, parts):
        o.add_particles(p, sp.q, sp.m)
    o.set_background(np.ones(o.shape3))
    o.set_field(oracle.EX, gauss_ex(wl, parts))
    ts, amps = [0.0], [mode_amplitude(o.get_field(oracle.EX))]
    for s in range(int(tmax / wl.dt)):
        o.step(1)
        ts.append((s + 1) * wl.dt)
        amps.append(mode_amplitude(o.get_field(oracle.EX)))
    return o, np.array(ts), np.array(amps)


@pytest.mark.parametrize("order,k_frac", [(2, 1.0), (1, 1.0), (2, 0.7), (2, 0.4)])
def test_two_stream_growth_rate(order, k_frac):
    u0, amp = 0.2, 1e-6
    wl, L = workload((32, 4), u0=u0, k_frac=k_frac, order=order, amp=amp)
    o, ts, amps = _run_oracle(wl, TMAX)
    k = 2 * np.pi / L
    gth = growth_rate(k, u0)
    # the seed is the charge of the eigenmode: Ex starts at amp
    assert abs(amps[0] / amp - 1.0) < 0.01, amps[0]
    g = fit_rate(ts, amps, 2.0, TMAX)
    assert abs(g / gth - 1.0) < 0.015, (g, gth)
    # the whole history is one exponential: no stable roots were excited
    ratio = amps / (amps[0] * np.exp(gth * ts))
    assert 0.92 < ratio.min() and ratio.max() < 1.08, (ratio.min(), ratio.max())
    # still linear at the end: far below the trapping amplitude gamma^2 / k
    assert amps[-1] < 0.1 * gth ** 2 / k
    # Gauss's law holds throughout (charge-conserving deposit)
    assert o.diag()["gauss_max"] < 1e-10


def test_two_stream_stable_mode_does_not_grow():
    """Beyond k v = sqrt(2) w1 the two beams are stable: a displacement seed
    only oscillates (its amplitude stays within a small factor of its
    start)."""
    u0 = 0.2
    wl, L = workload((32, 4), u0=u0, k_frac=1.8, amp=1e-5 * 2 * np.pi / (1.8 * 3.0))
    assert growth_rate(2 * np.pi / L, u0) == 0.0
    _, ts, amps = _run_oracle(wl, TMAX)
    assert amps.max() < 5.0 * amps[: int(2.0 / wl.dt)].max()
