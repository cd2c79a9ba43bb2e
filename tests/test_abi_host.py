"""C-ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every entry point include/pic.h declares, and rejects bad
configurations on the host before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1503_02464_gb300 import build, capi
    build.build()
    return capi.load()


def declared_symbols():
    syms = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            syms |= set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(pic_\w+)\s*\(", txt, flags=re.M))
    return sorted(syms)


def test_header_declares_entry_points():
    syms = declared_symbols()
    for s in ("pic_create", "pic_load_particles", "pic_step", "pic_fields", "pic_diag"):
        assert s in syms


def test_every_declared_symbol_exported(lib):
    for s in declared_symbols():
        assert hasattr(lib, s), s
    from paper_1503_02464_gb300 import capi
    assert set(capi.EXPORTED) <= set(declared_symbols())


def _cfg(**kw):
    from paper_1503_02464_gb300.sim import make_config
    base = dict(dims=3, n=(8, 8, 8), d=(0.1, 0.1, 0.1), dt=0.05, order=2, tile=None)
    base.update(kw)
    return make_config(base["dims"], base["n"], base["d"], base["dt"], base["order"], tile=base["tile"])


@pytest.mark.parametrize("kw,code", [
    (dict(dims=4), 1), (dict(order=3), 1), (dict(dt=-1.0), 1),
    (dict(dt=0.0578), 2),           # 3D Yee limit for dx = 0.1 is 0.057735
    (dict(dims=2, n=(8, 8), d=(0.1, 0.1), dt=0.0708), 2),  # 2D limit 0.070711
    (dict(tile=(4, 4, 4)), 1),      # only the compiled tile shape
    (dict(n=(1024, 1024, 1024)), 1),  # 2^30 cells
])
def test_create_rejects_bad_config(lib, kw, code):
    from paper_1503_02464_gb300 import capi
    cfg = _cfg(**kw)
    h = ctypes.c_void_p()
    rc = lib.pic_create(ctypes.byref(cfg), ctypes.byref(h))
    assert rc == code
    assert h.value is None
    msg = lib.pic_last_error(None).decode()
    assert msg
    if code == capi.PIC_ECOURANT:
        assert "Yee limit" in msg


def test_create_fails_loudly_without_device(lib):
    """A valid configuration on a machine without a GPU reports PIC_ECUDA
    (no CPU fallback)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cfg = _cfg(dt=0.05)
    h = ctypes.c_void_p()
    rc = lib.pic_create(ctypes.byref(cfg), ctypes.byref(h))
    assert rc == 4
