"""A tile denser than one fixed-point window may take (needs a GB300).

FP32 runs accumulate a block's current and charge windows as pairs of int32
words, and the low words cannot overflow below 65,536 contributions per
node. So a push work item never exceeds 65,280 slots, and the charge
diagnostic flushes a denser tile in pieces. One 8x8x4 tile holds 76,800
particles (300 per cell) and takes both paths. After three steps, fields,
momenta and charge density match the oracle, in FP32 to the 10-step
tolerance and in FP64 to 1e-12 per step. The total charge stays zero.
"""
import numpy as np
import pytest

from paper_1503_02464_gb300 import synth

from _parity import build_gpu, build_oracle, compare_fields, compare_particles, j_floor

pytestmark = pytest.mark.gpu

RHO = 9


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_tile_beyond_one_window(precision):
    wl = synth.small(3, (8, 8, 4), 2, 300, 0.1, 61)
    parts = [wl.particles(0)]
    assert len(parts[0]["x"]) == 76_800
    o = build_oracle(wl, parts)
    s = build_gpu(wl, parts, precision)
    o.step(3)
    s.step(3)
    tol = 1e-5 if precision == "fp32" else 3e-12
    fe = compare_fields(o, s, j_abs=j_floor(wl, parts))
    du, dx = compare_particles(o, s, wl)
    print(precision, fe, du, dx)
    for k, v in fe.items():
        assert v <= tol, (k, v)
    assert du <= tol, du
    # rho includes the neutralising background, so the net density is a small
    # fluctuation: judge the error against the particles' mean charge density
    rho_o, rho_g = o.rho(), s.field(RHO)
    gross = np.abs(parts[0]["w"]).sum() / rho_o.size
    assert np.abs(rho_g - rho_o).max() <= (1e-6 if precision == "fp32" else 1e-12) * gross
    d = s.diag()
    assert abs(d["charge"]) <= 1e-10 * np.abs(parts[0]["w"]).sum() * np.prod(wl.d)
    assert d["n_alive"] == 76_800
