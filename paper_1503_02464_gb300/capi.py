"""ctypes binding of libpic.so -- argument marshalling only.

Every function here has the name of the C entry point it wraps (declared in
``include/pic.h``) and does nothing but convert arguments: all of the PIC
cycle runs in the CUDA kernels of the library.  There is no fallback: if the
library is missing or cannot be loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

PIC_OK, PIC_EINVAL, PIC_ECOURANT, PIC_ENOMEM, PIC_ECUDA, PIC_EOVERFLOW, PIC_ETIMEOUT, PIC_ENAN = range(8)
PIC_FP32, PIC_FP64 = 0, 1
PIC_BC_PERIODIC, PIC_BC_ABSORBING = 0, 1
PIC_GATHER_MOMENTUM, PIC_GATHER_ENERGY = 0, 1
PIC_OUT_FIELD, PIC_OUT_PARTICLES = 0, 1
PIC_MEM_HOST, PIC_MEM_DEVICE = 0, 1
PIC_EX, PIC_EY, PIC_EZ, PIC_BX, PIC_BY, PIC_BZ, PIC_JX, PIC_JY, PIC_JZ, PIC_RHO = range(10)
KERNEL_CLASSES = ["sort", "zero_j", "push", "yee_b", "yee_e", "boundary", "filter", "adj_field", "adj_push",
                  "tape"]

ERROR_NAMES = {0: "PIC_OK", 1: "PIC_EINVAL", 2: "PIC_ECOURANT", 3: "PIC_ENOMEM", 4: "PIC_ECUDA",
               5: "PIC_EOVERFLOW", 6: "PIC_ETIMEOUT", 7: "PIC_ENAN"}

# every symbol include/pic.h declares
EXPORTED = ["pic_create", "pic_destroy", "pic_last_error", "pic_add_species", "pic_load_particles",
            "pic_neutralize", "pic_set_background", "pic_step", "pic_fields", "pic_set_field", "pic_num_particles", "pic_particles",
            "pic_diag", "pic_energy", "pic_sync", "pic_profile", "pic_timings", "pic_launch_count", "pic_checkpoint",
            "pic_restore", "pic_tape_begin", "pic_adjoint_begin", "pic_adjoint_seed_kinetic", "pic_adjoint_step",
            "pic_grad", "pic_state_size", "pic_state_save", "pic_state_load", "pic_output_due", "pic_output_add", "pic_output_capture", "pic_output_count",
            "pic_output_read", "pic_output_remove", "pic_field_energy_noalloc", "pic_alu_peak",
            "pic_adjoint_field", "pic_adjoint_set_field", "pic_adjoint_momenta", "pic_adjoint_set_momenta",
            "pic_tape_record", "pic_grad_binned"]


class pic_laser(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int), ("a0", ctypes.c_double), ("waist", ctypes.c_double),
                ("duration", ctypes.c_double), ("y_center", ctypes.c_double), ("z_center", ctypes.c_double),
                ("polarization", ctypes.c_int), ("angle", ctypes.c_double)]


class pic_config(ctypes.Structure):
    _fields_ = [("dims", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double * 3),
                ("dt", ctypes.c_double), ("shape_order", ctypes.c_int), ("precision", ctypes.c_int),
                ("bc_lo", ctypes.c_int * 3), ("bc_hi", ctypes.c_int * 3), ("sort_every", ctypes.c_int),
                ("tile", ctypes.c_int * 3), ("drift_guard", ctypes.c_int), ("laser", pic_laser),
                ("stream", ctypes.c_void_p), ("filter_passes", ctypes.c_int), ("filter_compensate", ctypes.c_int),
                ("gather", ctypes.c_int)]


class pic_output_t(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("which", ctypes.c_int), ("lo", ctypes.c_int * 3), ("hi", ctypes.c_int * 3),
                ("first", ctypes.c_int64), ("last", ctypes.c_int64), ("every", ctypes.c_int64),
                ("max_frames", ctypes.c_int64), ("max_particles", ctypes.c_int64)]


class pic_diag_t(ctypes.Structure):
    _fields_ = [("energy_field", ctypes.c_double), ("energy_e", ctypes.c_double), ("energy_b", ctypes.c_double),
                ("energy_kinetic", ctypes.c_double), ("charge", ctypes.c_double), ("gauss_max", ctypes.c_double),
                ("continuity_max", ctypes.c_double), ("n_alive", ctypes.c_int64), ("n_escaped", ctypes.c_int64),
                ("n_clamped", ctypes.c_int64), ("n_absorbed", ctypes.c_int64), ("n_sorts_adaptive", ctypes.c_int64),
                ("step", ctypes.c_int64), ("n_push_mid_drain", ctypes.c_int64),
                ("n_adj_escaped", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class pic_energy_t(ctypes.Structure):
    _fields_ = [("energy_e", ctypes.c_double), ("energy_b", ctypes.c_double), ("energy_kinetic", ctypes.c_double),
                ("n_alive", ctypes.c_int64), ("step", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class PicError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib: Optional[ctypes.CDLL] = None


def library_path() -> str:
    """The release library; with PIC_LIBRARY=checked the build whose kernels
    check every window and slot index (build.py); with PIC_LIBRARY set to the
    path of a .so file, that build of the library."""
    sel = os.environ.get("PIC_LIBRARY", "")
    if sel.endswith(".so"):
        return os.path.abspath(sel)
    name = "libpic_checked.so" if sel == "checked" else "libpic.so"
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", name)


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libpic.so (building it with nvcc first if it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"libpic.so not built ({path}); run paper_1503_02464_gb300/build.py")
        from . import build as _build
        _build.build(checked=os.environ.get("PIC_LIBRARY") == "checked")
    lib = ctypes.CDLL(path)
    vp, dp, i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64
    hp = ctypes.c_void_p
    sig = {
        "pic_create": ([ctypes.POINTER(pic_config), ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
        "pic_destroy": ([hp], ctypes.c_int),
        "pic_last_error": ([hp], ctypes.c_char_p),
        "pic_add_species": ([hp, ctypes.c_double, ctypes.c_double, i64, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "pic_load_particles": ([hp, ctypes.c_int, i64] + [vp] * 8 + [ctypes.c_int], ctypes.c_int),
        "pic_neutralize": ([hp], ctypes.c_int),
        "pic_set_background": ([hp, vp, ctypes.c_int], ctypes.c_int),
        "pic_step": ([hp, ctypes.c_int], ctypes.c_int),
        "pic_fields": ([hp, ctypes.c_int, vp, ctypes.c_int], ctypes.c_int),
        "pic_set_field": ([hp, ctypes.c_int, vp, ctypes.c_int], ctypes.c_int),
        "pic_num_particles": ([hp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "pic_particles": ([hp, ctypes.c_int] + [vp] * 9 + [ctypes.c_int], ctypes.c_int),
        "pic_diag": ([hp, ctypes.POINTER(pic_diag_t)], ctypes.c_int),
        "pic_sync": ([hp], ctypes.c_int),
        "pic_energy": ([hp, ctypes.POINTER(pic_energy_t)], ctypes.c_int),
        "pic_profile": ([hp, ctypes.c_int], ctypes.c_int),
        "pic_timings": ([hp, dp, ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
                        ctypes.c_int),
        "pic_launch_count": ([hp, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "pic_checkpoint": ([hp, ctypes.c_int], ctypes.c_int),
        "pic_restore": ([hp, ctypes.c_int], ctypes.c_int),
        "pic_tape_begin": ([hp, ctypes.c_int], ctypes.c_int),
        "pic_tape_record": ([hp], ctypes.c_int),
        "pic_adjoint_begin": ([hp, i64], ctypes.c_int),
        "pic_adjoint_seed_kinetic": ([hp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp], ctypes.c_int),
        "pic_adjoint_step": ([hp, ctypes.c_int], ctypes.c_int),
        "pic_grad": ([hp, dp, ctypes.c_int, vp, ctypes.c_int], ctypes.c_int),
        "pic_grad_binned": ([hp, ctypes.c_int, vp, i64, ctypes.c_int, vp, ctypes.c_int], ctypes.c_int),
        "pic_field_energy_noalloc": ([ctypes.c_int, ctypes.c_void_p * 3, ctypes.c_void_p * 3, i64, ctypes.c_double,
                                      vp, ctypes.c_int, vp], ctypes.c_int),
        "pic_state_size": ([hp, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        "pic_state_save": ([hp, vp, i64, ctypes.c_int], ctypes.c_int),
        "pic_state_load": ([hp, vp, i64, ctypes.c_int], ctypes.c_int),
        "pic_output_due": ([ctypes.POINTER(pic_output_t), i64], ctypes.c_int),
        "pic_output_add": ([hp, ctypes.POINTER(pic_output_t), ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "pic_output_capture": ([hp, ctypes.c_int], ctypes.c_int),
        "pic_output_count": ([hp, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
                             ctypes.c_int),
        "pic_output_read": ([hp, ctypes.c_int, i64, vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                             ctypes.c_int], ctypes.c_int),
        "pic_output_remove": ([hp, ctypes.c_int], ctypes.c_int),
        "pic_alu_peak": ([dp, dp, vp], ctypes.c_int),
        "pic_adjoint_field": ([hp, ctypes.c_int, vp, ctypes.c_int], ctypes.c_int),
        "pic_adjoint_set_field": ([hp, ctypes.c_int, vp, ctypes.c_int], ctypes.c_int),
        "pic_adjoint_momenta": ([hp, ctypes.c_int, vp, vp, vp, ctypes.c_int], ctypes.c_int),
        "pic_adjoint_set_momenta": ([hp, ctypes.c_int, vp, vp, vp, ctypes.c_int], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def check(handle, rc: int) -> None:
    if rc != PIC_OK:
        msg = load().pic_last_error(handle)
        raise PicError(rc, msg.decode() if msg else "")


def pic_create(cfg: pic_config) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    check(None, load().pic_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h


def pic_destroy(h) -> None:
    check(h, load().pic_destroy(h))


def pic_last_error(h) -> str:
    m = load().pic_last_error(h)
    return m.decode() if m else ""


def pic_add_species(h, q: float, m: float, capacity: int) -> int:
    sp = ctypes.c_int()
    check(h, load().pic_add_species(h, float(q), float(m), int(capacity), ctypes.byref(sp)))
    return sp.value


def pic_load_particles(h, species: int, n: int, x, y, z, ux, uy, uz, w, ids, mem_kind: int) -> None:
    check(h, load().pic_load_particles(h, species, int(n), x, y, z, ux, uy, uz, w, ids, mem_kind))


def pic_neutralize(h) -> None:
    check(h, load().pic_neutralize(h))


def pic_set_background(h, rho_bg_ptr: int, mem_kind: int) -> None:
    check(h, load().pic_set_background(h, rho_bg_ptr, mem_kind))


def pic_step(h, nsteps: int) -> None:
    check(h, load().pic_step(h, int(nsteps)))


def pic_fields(h, which: int, out_ptr, mem_kind: int) -> None:
    check(h, load().pic_fields(h, which, out_ptr, mem_kind))


def pic_set_field(h, which: int, in_ptr, mem_kind: int) -> None:
    check(h, load().pic_set_field(h, which, in_ptr, mem_kind))


def pic_num_particles(h, species: int) -> int:
    n = ctypes.c_int64()
    check(h, load().pic_num_particles(h, species, ctypes.byref(n)))
    return n.value


def pic_particles(h, species: int, x, y, z, ux, uy, uz, w, ids, alive, mem_kind: int) -> None:
    check(h, load().pic_particles(h, species, x, y, z, ux, uy, uz, w, ids, alive, mem_kind))


def pic_diag(h) -> dict:
    d = pic_diag_t()
    check(h, load().pic_diag(h, ctypes.byref(d)))
    return d.as_dict()


def pic_energy(h) -> dict:
    d = pic_energy_t()
    check(h, load().pic_energy(h, ctypes.byref(d)))
    return d.as_dict()


def pic_sync(h) -> None:
    check(h, load().pic_sync(h))


def pic_profile(h, enable: bool) -> None:
    check(h, load().pic_profile(h, 1 if enable else 0))


def pic_timings(h) -> dict:
    nmax = len(KERNEL_CLASSES)
    ms = (ctypes.c_double * nmax)()
    cnt = (ctypes.c_int64 * nmax)()
    nc = ctypes.c_int()
    check(h, load().pic_timings(h, ms, cnt, nmax, ctypes.byref(nc)))
    return {KERNEL_CLASSES[i]: (ms[i], cnt[i]) for i in range(nc.value)}


def pic_checkpoint(h, slot: int) -> None:
    check(h, load().pic_checkpoint(h, int(slot)))


def pic_restore(h, slot: int) -> None:
    check(h, load().pic_restore(h, int(slot)))


def pic_tape_begin(h, nsteps: int) -> None:
    check(h, load().pic_tape_begin(h, int(nsteps)))


def pic_adjoint_begin(h, id_capacity: int) -> None:
    check(h, load().pic_adjoint_begin(h, int(id_capacity)))


def pic_adjoint_seed_kinetic(h, species: int, col_lo: int, col_hi: int) -> float:
    F = ctypes.c_double()
    check(h, load().pic_adjoint_seed_kinetic(h, int(species), int(col_lo), int(col_hi), ctypes.byref(F)))
    return F.value


def pic_adjoint_step(h, nsteps: int) -> None:
    check(h, load().pic_adjoint_step(h, int(nsteps)))


def pic_grad(h, species: int, dw_ptr, mem_kind: int) -> float:
    d_a0 = ctypes.c_double()
    check(h, load().pic_grad(h, ctypes.byref(d_a0), int(species), dw_ptr, int(mem_kind)))
    return d_a0.value


def pic_grad_binned(h, species: int, bin_ptr, n_ids: int, nbins: int, out_ptr, mem_kind: int) -> None:
    check(h, load().pic_grad_binned(h, int(species), bin_ptr, int(n_ids), int(nbins), out_ptr, int(mem_kind)))


def pic_state_size(h) -> int:
    n = ctypes.c_int64()
    check(h, load().pic_state_size(h, ctypes.byref(n)))
    return n.value


def pic_state_save(h, buf_ptr, nbytes: int, mem_kind: int) -> None:
    check(h, load().pic_state_save(h, buf_ptr, int(nbytes), int(mem_kind)))


def pic_state_load(h, buf_ptr, nbytes: int, mem_kind: int) -> None:
    check(h, load().pic_state_load(h, buf_ptr, int(nbytes), int(mem_kind)))


def make_output(kind: int, which: int, lo, hi, first: int, last: int, every: int = 1, max_frames: int = 1,
                max_particles: int = 1) -> pic_output_t:
    r = pic_output_t()
    r.kind, r.which = int(kind), int(which)
    for a in range(3):
        r.lo[a] = int(lo[a]) if a < len(lo) else 0
        r.hi[a] = int(hi[a]) if a < len(hi) else 1
    r.first, r.last, r.every = int(first), int(last), int(every)
    r.max_frames, r.max_particles = int(max_frames), int(max_particles)
    return r


def pic_output_due(req: pic_output_t, step: int) -> bool:
    return bool(load().pic_output_due(ctypes.byref(req), int(step)))


def pic_output_add(h, req: pic_output_t) -> int:
    i = ctypes.c_int()
    check(h, load().pic_output_add(h, ctypes.byref(req), ctypes.byref(i)))
    return i.value


def pic_output_capture(h, oid: int) -> None:
    check(h, load().pic_output_capture(h, int(oid)))


def pic_output_count(h, oid: int):
    n, d = ctypes.c_int64(), ctypes.c_int64()
    check(h, load().pic_output_count(h, int(oid), ctypes.byref(n), ctypes.byref(d)))
    return n.value, d.value


def pic_output_read(h, oid: int, frame: int, out_ptr, mem_kind: int):
    """Returns (count, step); raises PicError (PIC_EOVERFLOW) for a particle
    frame that lost records."""
    n, st = ctypes.c_int64(), ctypes.c_int64()
    check(h, load().pic_output_read(h, int(oid), int(frame), out_ptr, ctypes.byref(n), ctypes.byref(st),
                                    int(mem_kind)))
    return n.value, st.value


def pic_output_remove(h, oid: int) -> None:
    check(h, load().pic_output_remove(h, int(oid)))


def pic_launch_count(h) -> int:
    c = ctypes.c_int64()
    check(h, load().pic_launch_count(h, ctypes.byref(c)))
    return c.value


def pic_field_energy_noalloc(precision: int, E_ptrs, B_ptrs, ncell: int, cell_volume: float, out_ptr,
                             mem_kind: int, stream) -> None:
    """FP64 field energies (electric, magnetic) using no device allocation."""
    e = (ctypes.c_void_p * 3)(*E_ptrs)
    b = (ctypes.c_void_p * 3)(*B_ptrs)
    check(None, load().pic_field_energy_noalloc(int(precision), e, b, int(ncell), float(cell_volume), out_ptr,
                                                int(mem_kind), stream))


def pic_alu_peak(stream=None) -> tuple:
    """Measured FP32 and FP64 FMA throughput of the current device, TFLOP/s."""
    a, b = ctypes.c_double(), ctypes.c_double()
    check(None, load().pic_alu_peak(ctypes.byref(a), ctypes.byref(b), stream))
    return a.value, b.value


def pic_adjoint_field(h, which: int, out_ptr, mem_kind: int) -> None:
    check(h, load().pic_adjoint_field(h, int(which), out_ptr, int(mem_kind)))


def pic_adjoint_set_field(h, which: int, in_ptr, mem_kind: int) -> None:
    check(h, load().pic_adjoint_set_field(h, int(which), in_ptr, int(mem_kind)))


def pic_adjoint_momenta(h, species: int, ptrs, mem_kind: int) -> None:
    check(h, load().pic_adjoint_momenta(h, int(species), *ptrs, int(mem_kind)))


def pic_adjoint_set_momenta(h, species: int, ptrs, mem_kind: int) -> None:
    check(h, load().pic_adjoint_set_momenta(h, int(species), *ptrs, int(mem_kind)))


def pic_tape_record(h) -> None:
    check(h, load().pic_tape_record(h))
