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
