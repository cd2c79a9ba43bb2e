"""The OpenMP build of the oracle (CPU only) matches the serial one.

It runs the same arithmetic per particle; only the order in which the
threads' current arrays are added differs, so fields and particles agree to
round-off after several steps (thermal 3D plasma; 2D laser slab with
absorbing walls, where particles are also removed)."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import OracleSim
from paper_1503_02464_gb300 import synth

from _parity import FIELDS


def _run(wl, parallel, nsteps, laser=None):
    o = OracleSim(wl.dims, wl.n, wl.d, wl.dt, wl.order, parallel=parallel)
    if laser:
        o.set_absorbing_x(True)
        o.set_laser(laser["a0"], laser["waist"], laser["duration"], pol=laser["pol"])
    for isp, sp in enumerate(wl.species):
        o.add_particles(wl.particles(isp), sp.q, sp.m)
    if wl.neutralize:
        o.neutralize()
    o.step(nsteps)
    f = [o.get_field(i) for i in range(9)]
    p = [o.particles(i) for i in range(len(wl.species))]
    d = o.diag()
    o.close()
    return f, p, d


def _cases():
    thermal = synth.small(3, (12, 10, 8), 2, 4, 0.2, 5)
    d = 0.1
    dt = 0.9 * synth.courant_limit((d, d), 2)
    slab = synth.Workload("slab", 2, (96, 24, 1), (d, d, 1.0), dt, 2, 10, 9,
                          [synth.Species("electron", -1.0, 1.0, 4, 0.0, 4.0, (20, 28), 0),
                           synth.Species("proton", 1.0, 1836.0, 4, 0.0, 4.0, (20, 28), 1)],
                          absorbing_x=True, neutralize=False,
                          laser={"a0": 2.0, "waist": 0.6, "duration": 2 * math.pi, "pol": 1})
    return [("thermal3d", thermal, 6), ("laser_slab2d", slab, 70)]


@pytest.mark.parametrize("name,wl,nsteps", _cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_parallel_oracle_matches_serial(name, wl, nsteps):
    if (os.cpu_count() or 1) > 1:
        assert oracle.num_threads(parallel=True) > 1
    fs, ps, ds = _run(wl, False, nsteps, wl.laser)
    fp, pp, dp = _run(wl, True, nsteps, wl.laser)
    for name_f, a, b in zip(FIELDS, fp, fs):
        group = [FIELDS.index(name_f[0] + c) for c in "xyz"]
        norm = max(np.abs(fs[g]).max() for g in group) or 1.0
        assert np.abs(a - b).max() <= 1e-12 * norm, name_f
    for a, b in zip(pp, ps):
        assert np.array_equal(a["id"], b["id"])
        for k in ("x", "y", "z", "ux", "uy", "uz"):
            assert np.abs(a[k] - b[k]).max() <= 1e-12 * max(1.0, np.abs(b[k]).max()), k
    assert ds["n_alive"] == dp["n_alive"]
    assert abs(ds["energy_field"] - dp["energy_field"]) <= 1e-12 * max(ds["energy_field"], 1e-300)
