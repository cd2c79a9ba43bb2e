"""pic_field_energy_noalloc against pic_diag (needs a GB300).

pic_field_energy_noalloc serves callers that must not allocate device memory
(cudaMalloc/cudaFree can synchronise the device; some applications own all
device memory through their own pool).  It reduces caller-owned field arrays
with a static scratch array inside the library.  This file is collected last
so that a run stopping at its first failure has run every other test first.
"""
import ctypes

import numpy as np
import pytest

from paper_1503_02464_gb300 import capi, synth

pytestmark = pytest.mark.gpu

TOL = 1e-12  # both sides sum the same FP64 squares, in different orders


def _sim(precision):
    import torch
    from paper_1503_02464_gb300.sim import Simulation
    wl = synth.small(3, (24, 20, 16), 2, 2, 0.3, 17)
    s = Simulation.from_workload(wl, precision=precision)
    p = wl.particles(0)
    sp = s.add_species(-1.0, 1.0, len(p["x"]))
    s.load(sp, p)
    s.neutralize()
    s.step(6)
    torch.cuda.synchronize()
    return s, wl


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_energy_matches_pic_diag(precision):
    import torch
    s, wl = _sim(precision)
    d = s.diag()
    assert d["energy_e"] > 0 and d["energy_b"] > 0
    dv = float(np.prod(wl.d))
    ncell = wl.ncells
    dtype = torch.float32 if precision == "fp32" else torch.float64
    # the caller's own device arrays (exact copies of the library's fields)
    E = [s.field_device(i).to(dtype) for i in range(3)]
    B = [s.field_device(3 + i).to(dtype) for i in range(3)]
    prec = capi.PIC_FP32 if precision == "fp32" else capi.PIC_FP64
    stream = torch.cuda.current_stream().cuda_stream
    out_dev = torch.zeros(2, dtype=torch.float64, device="cuda")
    out_host = np.zeros(2)
    for _ in range(2):  # two calls in a row share the static scratch
        out_dev.zero_()
        capi.pic_field_energy_noalloc(prec, [t.data_ptr() for t in E], [t.data_ptr() for t in B], ncell, dv,
                                      out_dev.data_ptr(), capi.PIC_MEM_DEVICE, stream)
        torch.cuda.synchronize()
        got = out_dev.cpu().numpy()
        assert abs(got[0] - d["energy_e"]) <= TOL * d["energy_e"], (got, d["energy_e"])
        assert abs(got[1] - d["energy_b"]) <= TOL * d["energy_b"], (got, d["energy_b"])
        out_host[:] = 0
        capi.pic_field_energy_noalloc(prec, [t.data_ptr() for t in E], [t.data_ptr() for t in B], ncell, dv,
                                      out_host.ctypes.data, capi.PIC_MEM_HOST, stream)
        np.testing.assert_array_equal(out_host, got)  # fixed summation order: bitwise equal
    s.close()


def test_noalloc_rejects_oversized_grid():
    import torch
    t = torch.zeros(8, dtype=torch.float32, device="cuda")
    ptrs = [t.data_ptr()] * 3
    out = np.zeros(2)
    with pytest.raises(capi.PicError) as ei:
        capi.pic_field_energy_noalloc(capi.PIC_FP32, ptrs, ptrs, 33554432 + 1, 1.0, out.ctypes.data,
                                      capi.PIC_MEM_HOST, torch.cuda.current_stream().cuda_stream)
    assert ei.value.code == capi.PIC_EINVAL
    assert "33554432" in str(ei.value)
