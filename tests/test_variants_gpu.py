"""GPU path with the optional steps beside the deposit -- current smoothing
(binomial passes + compensation) and the energy-conserving gather -- against
the FP64 oracle configured alike (needs a GB300).  Same tolerances as the
standard cycle: FP64 within 1e-12 relative per step, FP32 within 1e-5 on
fields and momenta after 10 steps."""
import numpy as np
import pytest

import oracle
from oracle import OracleSim
from paper_1503_02464_gb300 import synth
from paper_1503_02464_gb300.sim import Simulation

from _parity import compare_fields, compare_particles, j_floor

pytestmark = pytest.mark.gpu

CASES = [  # dims, order, filter passes, compensate, gather
    (2, 1, 2, True, "energy"),
    (2, 2, 1, False, "momentum"),
    (2, 2, 0, False, "energy"),
    (3, 1, 0, False, "energy"),
    (3, 2, 1, True, "energy"),
]


def _pair(dims, order, passes, comp, gather, precision, u_th=0.05, seed=31):
    n = (32, 32) if dims == 2 else (16, 16, 8)
    wl = synth.small(dims, n, order, 4, u_th, seed)
    parts = [wl.particles(0)]
    o = OracleSim(wl.dims, wl.n, wl.d, wl.dt, wl.order)
    o.add_particles(parts[0], -1.0, 1.0)
    o.neutralize()
    o.set_filter(passes, comp)
    o.set_gather(gather == "energy")
    s = Simulation.from_workload(wl, precision=precision, filter_passes=passes, filter_compensate=comp,
                                 gather=gather)
    k = s.add_species(-1.0, 1.0, len(parts[0]["x"]))
    s.load(k, parts[0])
    s.neutralize()
    return wl, parts, o, s


@pytest.mark.parametrize("dims,order,passes,comp,gather", CASES)
def test_variant_parity_fp64(dims, order, passes, comp, gather):
    wl, parts, o, s = _pair(dims, order, passes, comp, gather, "fp64")
    # the compensating pass has weights (1 - a)/2, a, (1 - a)/2 with
    # a = 1 + passes/2: it can amplify the oracle's J floor by (1 + passes/2)
    # per axis
    jf = j_floor(wl, parts) * ((1 + 0.5 * passes) ** dims if comp else 1.0)
    for step in range(1, 21):
        o.step(1)
        s.step(1)
        if step % 5 == 0:
            fe = compare_fields(o, s, j_abs=jf)
            for key, v in fe.items():
                assert v <= 1e-12 * step, (step, key, v)
            du, _ = compare_particles(o, s, wl, 0)
            assert du <= 1e-12 * step, (step, du)
    dg, do = s.diag(), o.diag()
    assert dg["gauss_max"] < 1e-11 and do["gauss_max"] < 1e-11
    assert abs(dg["energy_field"] / do["energy_field"] - 1.0) < 1e-10


@pytest.mark.parametrize("dims,order,passes,comp,gather", [CASES[0], CASES[4]])
def test_variant_fp32_10_steps(dims, order, passes, comp, gather):
    wl, parts, o, s = _pair(dims, order, passes, comp, gather, "fp32")
    o.step(10)
    s.step(10)
    fe = compare_fields(o, s, ["Ex", "Ey", "Ez", "Bx", "By", "Bz"])
    for key, v in fe.items():
        assert v <= 1e-5, (key, v)
    du, _ = compare_particles(o, s, wl, 0)
    assert du <= 1e-5, du


def test_filtered_diagnostics_at_round_off():
    """With smoothing on, Gauss's law and continuity are tested on the
    smoothed charge and hold to FP64 round-off step after step."""
    wl, parts, o, s = _pair(3, 2, 2, True, "momentum", "fp64")
    for _ in range(5):
        s.step(1)
        d = s.diag()
    assert d["gauss_max"] < 1e-11
    assert 0 <= d["continuity_max"] < 1e-9


def test_energy_conserving_gather_heating_fp32():
    """The FP32 path shows the physics the oracle pin fixes: an
    under-resolved thermal plasma heats under the momentum-conserving gather
    and not under the energy-conserving one."""
    drift = {}
    for gather in ("momentum", "energy"):
        wl = synth.small(2, (32, 16), 1, 8, 0.01, 1001, dt_frac=0.5, d=0.05)
        s = Simulation.from_workload(wl, precision="fp32", gather=gather)
        k = s.add_species(-1.0, 1.0, wl.n_particles())
        s.load(k, wl.particles(0))
        s.neutralize()
        d0 = s.diag()
        s.step(400)
        d1 = s.diag()
        u0 = d0["energy_field"] + d0["energy_kinetic"]
        drift[gather] = (d1["energy_field"] + d1["energy_kinetic"] - u0) / u0
    assert drift["momentum"] > 2e-3, drift
    assert abs(drift["energy"]) < 0.05 * drift["momentum"], drift


def test_adjoint_rejects_variants():
    wl = synth.small(2, (32, 32), 2, 2, 0.01, 3)
    s = Simulation.from_workload(wl, precision="fp64", filter_passes=1)
    with pytest.raises(RuntimeError):
        s.adjoint_begin(1024)
