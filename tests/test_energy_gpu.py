"""Total-energy drift of the FP32 path against the FP64 path over long runs
(needs a GB300).

The momentum-conserving PIC scheme heats slowly in FP64 too, so the bound is
on the difference of the drifts: |dU_fp32(t) - dU_fp64(t)| / U(0) <= 1e-3,
with U = field energy + kinetic energy (FP64 reductions).  Both drifts are
printed.
"""
import numpy as np
import pytest

from paper_1503_02464_gb300 import synth
from paper_1503_02464_gb300.sim import Simulation

pytestmark = pytest.mark.gpu


def _energy_history(wl, precision, nsteps, every):
    s = Simulation.from_workload(wl, precision=precision)
    p = wl.particles(0)
    k = s.add_species(-1.0, 1.0, len(p["x"]))
    s.load(k, p)
    s.neutralize()
    hist = []
    for t in range(0, nsteps + 1, every):
        if t:
            s.step(every)
        d = s.diag()
        hist.append(d["energy_field"] + d["energy_kinetic"])
    s.close()
    return np.array(hist)


@pytest.mark.parametrize("case", ["thermal2d_64", "thermal3d_small"])
def test_fp32_energy_drift_tracks_fp64(case):
    if case == "thermal2d_64":
        wl, nsteps = synth.preset("thermal2d_64"), 2000
    else:
        wl, nsteps = synth.small(3, (32, 32, 32), 2, 8, 0.05, 1003, dt_frac=0.97), 500
    u64 = _energy_history(wl, "fp64", nsteps, 50)
    u32 = _energy_history(wl, "fp32", nsteps, 50)
    d64 = (u64 - u64[0]) / u64[0]
    d32 = (u32 - u32[0]) / u64[0]
    print(case, "relative drift fp64 %.3e fp32 %.3e max diff %.3e" % (d64[-1], d32[-1], np.abs(d32 - d64).max()))
    assert np.abs(d32 - d64).max() <= 1e-3


def _laser_slab_history(wl, precision, nsteps, every):
    """Total energy (fields + both species, FP64 sums) every `every` steps,
    and the FP64 Gauss residual max |div E - rho| at the end."""
    s = Simulation.from_workload(wl, precision=precision)
    for isp, sp in enumerate(wl.species):
        p = wl.particles(isp)
        k = s.add_species(sp.q, sp.m, len(p["x"]))
        s.load(k, p)
    hist = []
    for t in range(0, nsteps + 1, every):
        if t:
            s.step(every)
        e = s.energy()
        hist.append(e["energy_e"] + e["energy_b"] + e["energy_kinetic"])
    d = s.diag()
    s.close()
    return np.array(hist), d


def test_fp32_laser_slab_energy_tracks_fp64():
    """The 2D laser-on-overdense-slab configuration (dx = 0.02 lambda, dt at
    0.9 of the Courant limit, p-polarised Gaussian pulse a0 = 3 from x = 0,
    absorbing x walls, periodic y, a 40 n_c slab of electrons and protons,
    TSC), reduced to 512 x 256 cells, a 20-cell slab, 16 particles per cell
    per species and a 4 lambda pulse so that the whole interaction (entry,
    reflection at the slab, exit through the wall) fits in 2000 steps.
    Energy is not conserved here (the pulse brings it in through x = 0 and
    takes it out again), so the bound is on the FP32 and FP64 histories
    themselves: |U_fp32(t) - U_fp64(t)| <= 1e-3 max U_fp64, every 50 steps.
    Gauss's law holds in both to FP64 round-off of the FP32/FP64 data."""
    lam = 2 * np.pi
    d = 0.02 * lam
    dt = 0.9 * synth.courant_limit((d, d), 2)
    n = (512, 256, 1)
    wl = synth.Workload("laser_slab2d_reduced", 2, n, (d, d, 1.0), dt, 2, 2000, 1002,
                        [synth.Species("electron", -1.0, 1.0, 16, 0.0, 40.0, (256, 276), 0),
                         synth.Species("proton", 1.0, 1836.0, 16, 0.0, 40.0, (256, 276), 1)],
                        absorbing_x=True, neutralize=False,
                        laser={"a0": 3.0, "waist": 1.5 * lam, "duration": 4 * lam, "pol": 1})
    u64, d64 = _laser_slab_history(wl, "fp64", 2000, 50)
    u32, d32 = _laser_slab_history(wl, "fp32", 2000, 50)
    peak = u64.max()
    diff = np.abs(u32 - u64).max() / peak
    print("laser slab: peak energy %.4e, end fp64 %.4e fp32 %.4e, max |dU|/peak %.3e, gauss fp64 %.2e fp32 %.2e"
          % (peak, u64[-1], u32[-1], diff, d64["gauss_max"], d32["gauss_max"]))
    assert u64.argmax() > 0 and peak > 10 * max(u64[0], 1e-30)  # the pulse came in
    assert diff <= 1e-3
