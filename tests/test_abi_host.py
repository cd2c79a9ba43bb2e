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


@pytest.mark.parametrize("laser", [
    dict(angle=0.5 * 3.141592653589793),   # grazing: |angle| must stay below pi/2
    dict(angle=float("nan")),
    dict(pol=3),
    dict(waist=0.0),
])
def test_create_rejects_bad_laser(lib, laser):
    """Laser parameters are checked on the host before any device work."""
    from paper_1503_02464_gb300.sim import make_config
    L = dict(a0=1.0, waist=1.0, duration=6.0, pol=1, angle=0.3)
    L.update(laser)
    cfg = make_config(2, (32, 8), (0.1, 0.1), 0.05, 2, absorbing_x=True, laser=L)
    h = ctypes.c_void_p()
    rc = lib.pic_create(ctypes.byref(cfg), ctypes.byref(h))
    assert rc == 1 and h.value is None
    assert "laser" in lib.pic_last_error(None).decode()


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


def test_struct_layouts_match_header(tmp_path):
    """Every struct the binding mirrors has the size and field offsets the C
    compiler gives it from include/pic.h (a field added on one side only
    shifts everything after it)."""
    import shutil
    import subprocess
    from paper_1503_02464_gb300 import capi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [capi.pic_laser, capi.pic_config, capi.pic_output_t, capi.pic_diag_t, capi.pic_energy_t]
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "pic.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        parts = ln.split()
        if len(parts) == 3:
            got[(parts[0], parts[1])] = int(parts[2])
    for st in structs:
        name = st.__name__
        assert got[(name, "size")] == ctypes.sizeof(st), name
        for field, _ in st._fields_:
            assert got[(name, field)] == getattr(st, field).offset, (name, field)
