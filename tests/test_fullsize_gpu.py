"""Parity at the full bench size (256^3 cells, 134,217,728 electrons, FP32,
the launch configuration bench.py times), on sampled outputs that the
oracle can compute one by one, plus properties that hold at any size
(needs a GB300).

First step from E = B = 0: every particle moves in a straight line
(x1 = x0 + dt u / gamma, §2 eq. 3), the current at a node comes only from
particles within three cells of it (the oracle deposits those on a local
window), and E^1 = -dt J there.  After the step the discrete continuity
equation and Gauss's law hold to FP32 round-off everywhere.
"""
import numpy as np
import pytest

import oracle
from paper_1503_02464_gb300 import synth
from paper_1503_02464_gb300.sim import Simulation

pytestmark = pytest.mark.gpu


def test_thermal3d_256_first_step_sampled():
    wl = synth.preset("thermal3d_256")
    n = wl.n[0]
    host = synth.SharedParticles(wl, 0)
    try:
        s = Simulation.from_workload(wl, precision="fp32")
        k = s.add_species(-1.0, 1.0, host.n)
        s.load(k, host.arrays)
        s.neutralize()
        d0 = s.diag()
        s.step(1)
        d1 = s.diag()
        # ---- properties at any size
        J = [s.field(6 + c) for c in range(3)]
        jmax = max(np.abs(j).max() for j in J)
        assert d1["n_alive"] == host.n
        assert 0 <= d1["continuity_max"] <= 1e-5 * jmax / wl.d[0], (d1["continuity_max"], jmax)
        assert d1["gauss_max"] <= 1e-5 * max(1.0, abs(d0["gauss_max"]) + 1.0)
        # ---- sampled particles: straight-line move
        rng = np.random.default_rng(0)
        ids = rng.choice(host.n, 4000, replace=False)
        p = s.particles(0)
        pos = np.empty(host.n, dtype=np.int64)
        pos[p["id"]] = np.arange(len(p["id"]))
        sel = pos[ids]
        a = host.arrays
        for key, ax in (("x", 0), ("y", 1), ("z", 2)):
            ukey = "u" + key
            g = np.sqrt(1 + a["ux"][ids] ** 2 + a["uy"][ids] ** 2 + a["uz"][ids] ** 2)
            want = a[key][ids] + wl.dt * a[ukey][ids] / g
            L = n * wl.d[ax]
            diff = (p[key][sel] - want + 0.5 * L) % L - 0.5 * L
            assert np.abs(diff).max() / wl.d[ax] < 2e-6, key
            np.testing.assert_array_equal(p[ukey][sel], a[ukey][ids].astype(np.float32).astype(np.float64))
        # ---- sampled nodes: J from the particles within three cells, E = -dt J
        E = [s.field(c) for c in range(3)]
        for trial in range(12):
            c0 = rng.integers(8, n - 8, 3)
            lo = c0 - 3
            ii, jj, kk = np.meshgrid(np.arange(7) + lo[0], np.arange(7) + lo[1], np.arange(7) + lo[2],
                                     indexing="ij")
            cells = np.sort((ii + n * (jj + n * kk)).reshape(-1))
            part = wl.particles(0, cells)
            o = oracle.OracleSim(3, (14, 14, 14), wl.d, wl.dt, wl.order)
            org = (lo - 4) * np.array(wl.d)
            local = dict(part)
            for key, ax in (("x", 0), ("y", 1), ("z", 2)):
                local[key] = part[key] - org[ax]
            o.add_particles(local, -1.0, 1.0)
            o.step(1)
            ci = c0 - lo + 4  # node index in the local window
            for c in range(3):
                jo = o.get_field(6 + c)[ci[2], ci[1], ci[0]]
                jg = J[c][c0[2], c0[1], c0[0]]
                assert abs(jg - jo) <= 1e-5 * jmax, (trial, c, jg, jo)
                eg = E[c][c0[2], c0[1], c0[0]]
                assert abs(eg + wl.dt * jo) <= 1e-5 * wl.dt * jmax, (trial, c, eg, -wl.dt * jo)
        s.close()
    finally:
        host.close()


def test_thermal3d_256_fp32_tracks_fp64_over_a_sort_cycle():
    """The bench workload over 25 steps (a cadence sort at step 20, particles
    on the escape path before it) in FP32 and in FP64 from the same inputs:
    the FP64 path holds the oracle to 1e-12 per step on the small cases, so
    the FP32 run's energies must follow it, and in both runs the discrete
    continuity equation and Gauss's law hold at the last step."""
    wl = synth.preset("thermal3d_256")
    host = synth.SharedParticles(wl, 0)
    out = {}
    try:
        for precision in ("fp32", "fp64"):
            s = Simulation.from_workload(wl, precision=precision)
            k = s.add_species(-1.0, 1.0, host.n)
            s.load(k, host.arrays)
            s.neutralize()
            s.step(24)
            s.diag()  # the previous step's charge, for the continuity check
            s.step(1)
            d = s.diag()
            jmax = max(np.abs(s.field(6 + c)).max() for c in range(3))
            out[precision] = d
            print(precision, {key: d[key] for key in ("energy_e", "energy_b", "energy_kinetic", "gauss_max",
                                                       "continuity_max", "n_escaped")}, "jmax", jmax)
            assert d["n_alive"] == host.n
            tol = 1e-5 if precision == "fp32" else 1e-12
            assert 0 <= d["continuity_max"] <= tol * jmax / wl.d[0], (precision, d["continuity_max"], jmax)
            assert d["n_escaped"] > 0  # the escape path ran
            s.close()
    finally:
        host.close()
    # measured on GB300: kinetic 1e-10, electric 3e-8, magnetic 4e-8 relative
    a, b = out["fp32"], out["fp64"]
    assert a["n_escaped"] == b["n_escaped"]  # the same particles left their windows
    assert abs(a["energy_kinetic"] / b["energy_kinetic"] - 1) <= 1e-8, (a["energy_kinetic"], b["energy_kinetic"])
    assert abs(a["energy_e"] / b["energy_e"] - 1) <= 1e-6, (a["energy_e"], b["energy_e"])
    assert abs(a["energy_b"] / b["energy_b"] - 1) <= 1e-6, (a["energy_b"], b["energy_b"])
    assert a["gauss_max"] <= 1e-6 and b["gauss_max"] <= 1e-12
