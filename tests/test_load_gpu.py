"""Particle loads (needs a GB300).

pic_load_particles copies host arrays in chunks of 4M particles through two
device staging buffers, overlapping the copy engine with the conversion
kernel.  A load of several chunks must store exactly what a load of the same
arrays from device memory stores (the same kernel converts both): cells,
offsets, momenta, weights and ids, slot by slot, with running ids continuing
across appending calls.  This holds for pageable and page-locked host arrays
alike, and a non-finite value in a late chunk marks only that particle dead.
"""
import numpy as np
import pytest
import torch

from paper_1503_02464_gb300 import capi, synth
from paper_1503_02464_gb300.sim import Simulation

pytestmark = pytest.mark.gpu

CHUNK = 1 << 22  # particles per staging chunk of a host load
KEYS = ("x", "y", "z", "ux", "uy", "uz", "w")


def _arrays(n, seed, box):
    rng = np.random.default_rng(seed)
    a = {k: rng.uniform(0.0, box[i], n) for i, k in enumerate(("x", "y", "z"))}
    for k in ("ux", "uy", "uz"):
        a[k] = rng.normal(0.0, 0.05, n)
    a["w"] = rng.uniform(0.5, 1.5, n)
    return a


def _sim(wl, cap, precision="fp32"):
    s = Simulation.from_workload(wl, precision=precision)
    s.add_species(-1.0, 1.0, cap)
    return s


def _stored(s):
    return s.particles(0, alive_only=False)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_chunked_host_load_matches_device_load(precision):
    wl = synth.small(3, (64, 64, 32), 2, 1, 0.0, 3)
    box = [wl.n[i] * wl.d[i] for i in range(3)]
    n1, n2 = 2 * CHUNK + 611_003, 1_000_001   # three chunks, then one more call
    a1, a2 = _arrays(n1, 11, box), _arrays(n2, 12, box)

    host = _sim(wl, n1 + n2, precision)
    host.load(0, a1)             # no ids: running index 0 .. n1-1
    host.load(0, a2)             # continues at n1
    got = _stored(host)

    dev = _sim(wl, n1 + n2, precision)
    both = {k: np.concatenate([a1[k], a2[k]]) for k in KEYS}
    td = {k: torch.from_numpy(v).cuda() for k, v in both.items()}
    td["id"] = torch.arange(n1 + n2, dtype=torch.int32).cuda()
    dev.load(0, td)
    ref = _stored(dev)

    assert host.num_particles(0) == n1 + n2
    for k in KEYS + ("id", "alive"):
        assert np.array_equal(got[k], ref[k]), k
    assert np.array_equal(got["id"], np.arange(n1 + n2, dtype=np.uint32))
    host.close()
    dev.close()


def test_page_locked_host_load_and_explicit_ids():
    wl = synth.small(3, (32, 32, 32), 2, 1, 0.0, 4)
    box = [wl.n[i] * wl.d[i] for i in range(3)]
    n = CHUNK + 12_345
    a = _arrays(n, 21, box)
    a["id"] = np.random.default_rng(5).permutation(n).astype(np.uint32)
    cudart = torch.cuda.cudart()
    regs = []
    try:
        for v in a.values():
            assert int(cudart.cudaHostRegister(v.ctypes.data, v.nbytes, 0)) == 0
            regs.append(v.ctypes.data)
        pinned = _sim(wl, n)
        pinned.load(0, a)
        got = _stored(pinned)
    finally:
        for p in regs:
            cudart.cudaHostUnregister(p)
    plain = _sim(wl, n)
    plain.load(0, {k: v.copy() for k, v in a.items()})
    ref = _stored(plain)
    for k in KEYS + ("id", "alive"):
        assert np.array_equal(got[k], ref[k]), k
    assert np.array_equal(got["id"], a["id"])
    pinned.close()
    plain.close()


def test_bad_particle_in_late_chunk():
    wl = synth.small(3, (32, 32, 32), 2, 1, 0.0, 6)
    box = [wl.n[i] * wl.d[i] for i in range(3)]
    n = 2 * CHUNK + 77
    a = _arrays(n, 31, box)
    bad = 2 * CHUNK + 5          # in the third chunk
    a["uy"][bad] = np.nan
    s = _sim(wl, n)
    with pytest.raises(capi.PicError):
        s.load(0, a)
    p = _stored(s)
    assert s.num_particles(0) == n
    assert p["alive"][bad] == 0 and p["alive"].sum() == n - 1
    s.close()
