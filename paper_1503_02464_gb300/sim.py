"""Python front end of libpic.so: a Simulation object over the C ABI.

Marshalling only -- every step of the PIC cycle runs in the library's CUDA
kernels.  PyTorch is used for device buffers and the CUDA stream; host data
may be numpy arrays.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import capi

_PREC = {"fp32": capi.PIC_FP32, "fp64": capi.PIC_FP64}


def _ptr(a):
    """Data pointer and mem kind of a numpy array or a torch tensor."""
    if a is None:
        return None, capi.PIC_MEM_HOST
    if isinstance(a, np.ndarray):
        return a.ctypes.data, capi.PIC_MEM_HOST
    # torch tensor
    if a.is_cuda:
        return a.data_ptr(), capi.PIC_MEM_DEVICE
    return a.data_ptr(), capi.PIC_MEM_HOST


def make_config(dims: int, n, d, dt: float, order: int, precision: str = "fp32", sort_every: int = 20,
                tile=None, drift_guard: int = 0, absorbing_x: bool = False, laser: Optional[dict] = None,
                stream: Optional[int] = None, filter_passes: int = 0, filter_compensate: bool = False,
                gather: str = "momentum") -> capi.pic_config:
    cfg = capi.pic_config()
    cfg.dims = dims
    nn = list(n) + [1] * (3 - len(n))
    dd = list(d) + [1.0] * (3 - len(d))
    if dims == 2:
        nn[2], dd[2] = 1, 1.0
    for i in range(3):
        cfg.n[i] = int(nn[i])
        cfg.dx[i] = float(dd[i])
        cfg.tile[i] = int(tile[i]) if tile is not None and i < len(tile) else 0
        cfg.bc_lo[i] = capi.PIC_BC_PERIODIC
        cfg.bc_hi[i] = capi.PIC_BC_PERIODIC
    if absorbing_x:
        cfg.bc_lo[0] = cfg.bc_hi[0] = capi.PIC_BC_ABSORBING
    cfg.dt = float(dt)
    cfg.shape_order = int(order)
    cfg.precision = _PREC[precision] if isinstance(precision, str) else int(precision)
    cfg.sort_every = int(sort_every)
    cfg.drift_guard = int(drift_guard)
    if laser:
        cfg.laser.enabled = 1
        cfg.laser.a0 = float(laser["a0"])
        cfg.laser.waist = float(laser["waist"])
        cfg.laser.duration = float(laser["duration"])
        cfg.laser.y_center = float(laser.get("y_center", 0.5 * nn[1] * dd[1]))
        cfg.laser.z_center = float(laser.get("z_center", 0.5 * nn[2] * dd[2]))
        cfg.laser.polarization = int(laser.get("pol", 1))
        cfg.laser.angle = float(laser.get("angle", 0.0))
    cfg.stream = stream
    cfg.filter_passes = int(filter_passes)
    cfg.filter_compensate = 1 if filter_compensate else 0
    cfg.gather = {"momentum": capi.PIC_GATHER_MOMENTUM, "energy": capi.PIC_GATHER_ENERGY}[gather]
    return cfg


class Simulation:
    """One PIC simulation living on the current CUDA device."""

    def __init__(self, dims: int, n, d, dt: float, order: int, precision: str = "fp32", sort_every: int = 20,
                 tile=None, drift_guard: int = 0, absorbing_x: bool = False, laser: Optional[dict] = None,
                 stream=None, filter_passes: int = 0, filter_compensate: bool = False, gather: str = "momentum"):
        capi.load()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.cfg = make_config(dims, n, d, dt, order, precision, sort_every, tile, drift_guard, absorbing_x,
                               laser, stream, filter_passes, filter_compensate, gather)
        self.dims = dims
        self.n = tuple(self.cfg.n)
        self.d = tuple(self.cfg.dx)
        self.dt = dt
        self.order = order
        self.precision = precision
        self.h = capi.pic_create(self.cfg)
        self.species = []

    @classmethod
    def from_workload(cls, wl, precision: str = "fp32", **kw) -> "Simulation":
        kw.setdefault("sort_every", wl.sort_every)
        kw.setdefault("absorbing_x", wl.absorbing_x)
        kw.setdefault("laser", wl.laser)
        return cls(wl.dims, wl.n, wl.d, wl.dt, wl.order, precision, **kw)

    # -- lifecycle
    def close(self):
        if getattr(self, "h", None):
            capi.pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape3(self):
        return (self.n[2], self.n[1], self.n[0])

    # -- particles
    def add_species(self, q: float, m: float, capacity: int) -> int:
        sp = capi.pic_add_species(self.h, q, m, capacity)
        self.species.append((q, m))
        return sp

    def load(self, species: int, parts: dict) -> None:
        """Append particles given as FP64 arrays x, y, z, ux, uy, uz, w (+ id)."""
        keys = ["x", "y", "z", "ux", "uy", "uz", "w"]
        n = len(parts["x"])
        arrs = []
        kinds = set()
        for k in keys:
            a = parts.get(k)
            if a is None and k == "z":
                arrs.append(None)
                continue
            if isinstance(a, np.ndarray):
                a = np.ascontiguousarray(a, dtype=np.float64)
            arrs.append(a)
        ids = parts.get("id")
        if isinstance(ids, np.ndarray):
            ids = np.ascontiguousarray(ids, dtype=np.uint32)
        ptrs = []
        for a in arrs + [ids]:
            p, kind = _ptr(a)
            ptrs.append(p)
            if a is not None:
                kinds.add(kind)
        if len(kinds) != 1:
            raise ValueError("particle arrays must all be host or all be device memory")
        self._keep = (arrs, ids)
        capi.pic_load_particles(self.h, species, n, *ptrs, kinds.pop())

    def neutralize(self) -> None:
        capi.pic_neutralize(self.h)

    def set_background(self, rho_bg) -> None:
        """Immobile background charge density at the nodes, shaped like a field."""
        a = np.ascontiguousarray(np.broadcast_to(rho_bg, self.shape3), dtype=np.float64)
        capi.pic_set_background(self.h, a.ctypes.data, capi.PIC_MEM_HOST)

    def num_particles(self, species: int = 0) -> int:
        return capi.pic_num_particles(self.h, species)

    def particles(self, species: int = 0, alive_only: bool = True) -> dict:
        n = self.num_particles(species)
        out = {k: np.empty(n, dtype=np.float64) for k in ("x", "y", "z", "ux", "uy", "uz", "w")}
        out["id"] = np.empty(n, dtype=np.uint32)
        out["alive"] = np.empty(n, dtype=np.int32)
        if n:
            capi.pic_particles(self.h, species, *[out[k].ctypes.data for k in ("x", "y", "z", "ux", "uy", "uz", "w")],
                               out["id"].ctypes.data, out["alive"].ctypes.data, capi.PIC_MEM_HOST)
        if alive_only:
            m = out["alive"] == 1
            out = {k: v[m] for k, v in out.items()}
        return out

    # -- stepping
    def step(self, nsteps: int = 1) -> None:
        capi.pic_step(self.h, nsteps)

    def sync(self) -> None:
        capi.pic_sync(self.h)

    # -- fields
    def field(self, which: int) -> np.ndarray:
        out = np.empty(self.shape3, dtype=np.float64)
        capi.pic_fields(self.h, which, out.ctypes.data, capi.PIC_MEM_HOST)
        return out

    def field_device(self, which: int):
        import torch
        out = torch.empty(self.shape3, dtype=torch.float64, device="cuda")
        capi.pic_fields(self.h, which, out.data_ptr(), capi.PIC_MEM_DEVICE)
        return out

    def set_field(self, which: int, arr) -> None:
        a = np.ascontiguousarray(np.broadcast_to(arr, self.shape3), dtype=np.float64)
        capi.pic_set_field(self.h, which, a.ctypes.data, capi.PIC_MEM_HOST)

    # -- state save / resume
    def state(self) -> np.ndarray:
        """The complete state (fields, background, particles, step, counters)
        as a byte array."""
        buf = np.empty(capi.pic_state_size(self.h), dtype=np.uint8)
        capi.pic_state_save(self.h, buf.ctypes.data, buf.nbytes, capi.PIC_MEM_HOST)
        return buf

    def load_state(self, buf) -> None:
        """Resume from a state() of a simulation with the same configuration
        and species."""
        b = np.ascontiguousarray(buf, dtype=np.uint8)
        capi.pic_state_load(self.h, b.ctypes.data, b.nbytes, capi.PIC_MEM_HOST)

    def save_state(self, path: str) -> None:
        with open(path, "wb") as f:
            f.write(self.state().tobytes())

    def resume(self, path: str) -> None:
        self.load_state(np.fromfile(path, dtype=np.uint8))

    # -- output manager (reduced-dimension / sub-domain frames in a time window)
    def output_add(self, kind: str, which, lo, hi, first: int, last: int, every: int = 1, max_frames: int = 1,
                   max_particles: int = 1) -> int:
        """Register an output request; kind "field" (which = field id) or
        "particles" (which = species index); box [lo, hi) in cells."""
        k = {"field": capi.PIC_OUT_FIELD, "particles": capi.PIC_OUT_PARTICLES}[kind]
        req = capi.make_output(k, which, lo, hi, first, last, every, max_frames, max_particles)
        oid = capi.pic_output_add(self.h, req)
        self._outputs = getattr(self, "_outputs", {})
        self._outputs[oid] = req
        return oid

    def output_capture(self, oid: int) -> None:
        capi.pic_output_capture(self.h, oid)

    def output_count(self, oid: int):
        """(frames held, frames dropped)."""
        return capi.pic_output_count(self.h, oid)

    def output_read(self, oid: int, frame: int):
        """(data, step): a (bz, by, bx) FP64 array for a field frame, a dict
        of x, y, z, ux, uy, uz, w, id arrays for a particle frame."""
        req = self._outputs[oid]
        if req.kind == capi.PIC_OUT_FIELD:
            shape = tuple(req.hi[a] - req.lo[a] for a in (2, 1, 0))
            out = np.empty(shape, dtype=np.float64)
            _, step = capi.pic_output_read(self.h, oid, frame, out.ctypes.data, capi.PIC_MEM_HOST)
            return out, step
        buf = np.empty((req.max_particles, 8), dtype=np.float64)
        n, step = capi.pic_output_read(self.h, oid, frame, buf.ctypes.data, capi.PIC_MEM_HOST)
        rec = buf[:n]
        names = ("x", "y", "z", "ux", "uy", "uz", "w")
        d = {k: rec[:, i].copy() for i, k in enumerate(names)}
        d["id"] = rec[:, 7].astype(np.uint32)
        return d, step

    def output_remove(self, oid: int) -> None:
        capi.pic_output_remove(self.h, oid)

    def diag(self) -> dict:
        return capi.pic_diag(self.h)

    def energy(self) -> dict:
        return capi.pic_energy(self.h)

    # -- profiling
    def profile(self, enable: bool = True) -> None:
        capi.pic_profile(self.h, enable)

    def timings(self) -> dict:
        return capi.pic_timings(self.h)

    def launch_count(self) -> int:
        return capi.pic_launch_count(self.h)

    # -- differentiable runs (2D3V TSC)
    def checkpoint(self, slot: int) -> None:
        capi.pic_checkpoint(self.h, slot)

    def restore(self, slot: int) -> None:
        capi.pic_restore(self.h, slot)

    def tape_begin(self, nsteps: int) -> None:
        capi.pic_tape_begin(self.h, nsteps)

    def tape_record(self) -> None:
        """Record the current state as the next tape entry without stepping."""
        capi.pic_tape_record(self.h)

    def adjoint_begin(self, id_capacity: int) -> None:
        capi.pic_adjoint_begin(self.h, id_capacity)

    def adjoint_seed_kinetic(self, species: int, col_lo: int, col_hi: int) -> float:
        return capi.pic_adjoint_seed_kinetic(self.h, species, col_lo, col_hi)

    def adjoint_step(self, nsteps: int) -> None:
        capi.pic_adjoint_step(self.h, nsteps)

    def adjoint_field(self, which: int) -> np.ndarray:
        """The adjoint of field component `which` (EX..BZ, or JX..JZ: of the
        current of the last reversed step), FP64, shaped like field()."""
        out = np.empty(self.shape3, dtype=np.float64)
        capi.pic_adjoint_field(self.h, which, out.ctypes.data, capi.PIC_MEM_HOST)
        return out

    def adjoint_set_field(self, which: int, values) -> None:
        """Seed the adjoint of E or B component `which` (dF/dE, dF/dB)."""
        a = np.ascontiguousarray(np.broadcast_to(values, self.shape3), dtype=np.float64)
        capi.pic_adjoint_set_field(self.h, which, a.ctypes.data, capi.PIC_MEM_HOST)

    def adjoint_momenta(self, species: int, id_capacity: int) -> np.ndarray:
        """dF/du of a species by particle id, shape (3, id_capacity)."""
        out = np.zeros((3, id_capacity), dtype=np.float64)
        capi.pic_adjoint_momenta(self.h, species, [out[d].ctypes.data for d in range(3)], capi.PIC_MEM_HOST)
        return out

    def adjoint_set_momenta(self, species: int, lu) -> None:
        """Seed dF/du of a species by particle id, lu shaped (3, id_capacity)."""
        a = np.ascontiguousarray(lu, dtype=np.float64)
        capi.pic_adjoint_set_momenta(self.h, species, [a[d].ctypes.data for d in range(3)], capi.PIC_MEM_HOST)

    def grad_binned(self, species: int, bin_of_id, nbins: int) -> np.ndarray:
        """dF/dw summed over bins of particle ids on the device: out[b] =
        sum of dF/dw_i over ids i with bin_of_id[i] == b.  bin_of_id is an
        int32 numpy array (copied per call) or a CUDA int32 tensor."""
        if hasattr(bin_of_id, "data_ptr"):
            import torch
            if bin_of_id.dtype != torch.int32 or not bin_of_id.is_cuda or not bin_of_id.is_contiguous():
                raise ValueError("bin_of_id: a contiguous CUDA int32 tensor")
            out = torch.zeros(nbins, dtype=torch.float64, device=bin_of_id.device)
            capi.pic_grad_binned(self.h, species, bin_of_id.data_ptr(), bin_of_id.numel(), nbins, out.data_ptr(),
                                 capi.PIC_MEM_DEVICE)
            return out.cpu().numpy()
        b = np.ascontiguousarray(bin_of_id, dtype=np.int32)
        out = np.zeros(nbins, dtype=np.float64)
        capi.pic_grad_binned(self.h, species, b.ctypes.data, len(b), nbins, out.ctypes.data, capi.PIC_MEM_HOST)
        return out

    def grad_a0(self) -> float:
        """dF/da0 after a reverse sweep."""
        return capi.pic_grad(self.h, 0, None, capi.PIC_MEM_HOST)

    def grad(self, species: int, id_capacity: int):
        """(dF/da0, dF/dw by particle id) after a reverse sweep."""
        dw = np.zeros(id_capacity, dtype=np.float64)
        da0 = capi.pic_grad(self.h, species, dw.ctypes.data, capi.PIC_MEM_HOST)
        return da0, dw
