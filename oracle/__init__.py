"""FP64 CPU oracle of the relativistic PIC cycle -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library
(``paper_1503_02464_gb300``) never imports, links or calls it, and the two
share no code: the oracle is plain C (``pic_oracle.c``) compiled with gcc and
driven through ctypes from here.

What the oracle computes (section 2 of the PICCANTE paper, with the readings
listed in ``pic_oracle.c``): gather of the Yee-staggered fields with the
shape function, Boris push and leap-frog move in global FP64 coordinates,
Esirkepov charge-conserving deposition, Yee FDTD split into half B steps, and
FP64 diagnostics.  Particles are the paper's seven doubles (§3.3).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libpic_oracle.so")
_LIB_OMP = os.path.join(_HERE, "_build", "libpic_oracle_omp.so")

EX, EY, EZ, BX, BY, BZ, JX, JY, JZ, RHO = range(10)
FIELD_NAMES = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz", "rho"]

_lib = None
_lib_omp = None


def build(force: bool = False, parallel: bool = False) -> str:
    """Compile the oracle with gcc (no GPU, no CUDA).  ``parallel`` builds
    the OpenMP variant, whose particle loop runs on every host core with a J
    array per thread (same arithmetic; the per-thread J arrays are summed in
    thread order)."""
    lib_path = _LIB_OMP if parallel else _LIB
    os.makedirs(os.path.dirname(lib_path), exist_ok=True)
    if not force and os.path.exists(lib_path) and os.path.getmtime(lib_path) >= os.path.getmtime(_SRC):
        return lib_path
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c99", "-ffp-contract=off"] + (["-fopenmp"] if parallel else []) \
        + ["-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib_path)
    return lib_path


def _load(parallel: bool = False):
    global _lib, _lib_omp
    if parallel:
        if _lib_omp is None:
            _lib_omp = load_library(build(parallel=True))
        return _lib_omp
    if _lib is None:
        _lib = load_library(build())
    return _lib


def num_threads(parallel: bool = True) -> int:
    """Threads the oracle's particle loop runs on (OMP_NUM_THREADS, else
    every host core, for the OpenMP build; 1 for the serial one)."""
    return int(_load(parallel).oracle_num_threads())


def load_library(path: str):
    """Open a compiled oracle library at ``path`` and declare its entry
    points (the default one comes from ``build()``; the pin tests also open
    copies compiled with a deliberately planted mistake)."""
    lib = ctypes.CDLL(path)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    lib.oracle_create.restype = vp
    lib.oracle_create.argtypes = [ctypes.c_int, ip, dp, ctypes.c_double, ctypes.c_int]
    lib.oracle_destroy.argtypes = [vp]
    lib.oracle_add_species.restype = ctypes.c_int
    lib.oracle_add_species.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_long] + [dp] * 7 + [u32p]
    lib.oracle_num_particles.restype = ctypes.c_long
    lib.oracle_num_particles.argtypes = [vp, ctypes.c_int]
    lib.oracle_get_particles.restype = ctypes.c_long
    lib.oracle_get_particles.argtypes = [vp, ctypes.c_int, dp, u32p]
    lib.oracle_get_field.argtypes = [vp, ctypes.c_int, dp]
    lib.oracle_set_field.argtypes = [vp, ctypes.c_int, dp]
    lib.oracle_step.argtypes = [vp, ctypes.c_int]
    lib.oracle_field_step.argtypes = [vp, ctypes.c_int]
    lib.oracle_step_count.restype = ctypes.c_long
    lib.oracle_step_count.argtypes = [vp]
    lib.oracle_shape.restype = ctypes.c_double
    lib.oracle_shape.argtypes = [ctypes.c_int, ctypes.c_double]
    lib.oracle_boris.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp, dp]
    lib.oracle_gather_point.argtypes = [vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp]
    lib.oracle_deposit_move.argtypes = [vp, ctypes.c_double, ctypes.c_double, dp, dp, ctypes.c_double]
    lib.oracle_compute_rho.argtypes = [vp]
    lib.oracle_neutralize.argtypes = [vp]
    lib.oracle_set_background.argtypes = [vp, dp]
    lib.oracle_set_filter.argtypes = [vp, ctypes.c_int, ctypes.c_int]
    lib.oracle_set_gather.argtypes = [vp, ctypes.c_int]
    lib.oracle_smooth.argtypes = [vp, ctypes.c_int]
    lib.oracle_diag.argtypes = [vp, dp]
    lib.oracle_set_boundary.argtypes = [vp, ctypes.c_int]
    lib.oracle_set_laser.argtypes = [vp, ctypes.c_int] + [ctypes.c_double] * 5 + [ctypes.c_int, ctypes.c_double]
    lib.oracle_laser_field.restype = ctypes.c_double
    lib.oracle_laser_field.argtypes = [vp] + [ctypes.c_double] * 4
    lib.oracle_num_threads.restype = ctypes.c_int
    lib.oracle_num_threads.argtypes = []
    return lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def shape(order: int, xi: float) -> float:
    """Shape function value (1 = CIC, 2 = TSC) at distance xi in cells."""
    return _load().oracle_shape(order, float(xi))


def boris(q: float, m: float, dt: float, E, B, p) -> np.ndarray:
    """One Boris momentum update of p (= m u) in fields E, B (§2 eq. 3)."""
    E, B, p = _f64(E).copy(), _f64(B).copy(), _f64(p).copy()
    _load().oracle_boris(q, m, dt, _dp(E), _dp(B), _dp(p))
    return p


class OracleSim:
    """One simulation held by the C oracle.

    ``dims`` is 2 or 3, ``n`` the cells per axis, ``d`` the cell sizes (c/omega
    units), ``dt`` the time step and ``order`` the shape order (1 CIC, 2 TSC).
    Fields are returned as numpy arrays shaped (nz, ny, nx).  ``parallel``
    runs the particle loop of each step on every host core (OpenMP build).
    """

    def __init__(self, dims, n, d, dt, order, parallel: bool = False):
        lib = self._lib = _load(parallel)
        n3 = list(n) + [1] * (3 - len(n))
        d3 = list(d) + [1.0] * (3 - len(d))
        if dims == 2:
            n3[2], d3[2] = 1, 1.0
        self.dims, self.n, self.d, self.dt, self.order = dims, tuple(n3), tuple(d3), dt, order
        ni = (ctypes.c_int * 3)(*n3)
        dd = (ctypes.c_double * 3)(*d3)
        self._h = lib.oracle_create(dims, ni, dd, float(dt), int(order))
        self._keep = []

    def close(self):
        if self._h:
            self._lib.oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape3(self):
        return (self.n[2], self.n[1], self.n[0])

    def add_species(self, q, m, x, y, z, ux, uy, uz, w, ids=None) -> int:
        n = len(x)
        arrs = [_f64(a) for a in (x, y, z if z is not None else np.zeros(n), ux, uy, uz, w)]
        ids = np.ascontiguousarray(ids if ids is not None else np.arange(n), dtype=np.uint32)
        return self._lib.oracle_add_species(
            self._h, float(q), float(m), n, *[_dp(a) for a in arrs],
            ids.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))

    def add_particles(self, parts: dict, q: float, m: float) -> int:
        return self.add_species(q, m, parts["x"], parts["y"], parts.get("z"), parts["ux"], parts["uy"],
                                parts["uz"], parts["w"], parts.get("id"))

    def set_filter(self, passes: int, compensate: bool = False):
        """Smooth J after every deposit: ``passes`` binomial passes per axis,
        then optionally one compensating pass."""
        self._lib.oracle_set_filter(self._h, int(passes), 1 if compensate else 0)

    def set_gather(self, energy_conserving: bool):
        """Gather variant: one shape order lower at half-integer positions."""
        self._lib.oracle_set_gather(self._h, 1 if energy_conserving else 0)

    def smooth(self, which: int):
        """Apply the configured smoothing to one stored field in place."""
        self._lib.oracle_smooth(self._h, int(which))

    def set_absorbing_x(self, on: bool = True):
        self._lib.oracle_set_boundary(self._h, 1 if on else 0)

    def set_laser(self, a0, waist, duration, y_center=None, z_center=None, pol=1, angle=0.0):
        yc = 0.5 * self.n[1] * self.d[1] if y_center is None else y_center
        zc = 0.5 * self.n[2] * self.d[2] if z_center is None else z_center
        self._lib.oracle_set_laser(self._h, 1, float(a0), float(waist), float(duration), float(yc), float(zc),
                                 int(pol), float(angle))

    def laser_field(self, x, y, z, t) -> float:
        return self._lib.oracle_laser_field(self._h, float(x), float(y), float(z), float(t))

    def step(self, n: int = 1):
        self._lib.oracle_step(self._h, int(n))

    def field_step(self, n: int = 1):
        self._lib.oracle_field_step(self._h, int(n))

    def get_field(self, which: int) -> np.ndarray:
        out = np.empty(self.shape3, dtype=np.float64)
        self._lib.oracle_get_field(self._h, which, _dp(out))
        return out

    def set_field(self, which: int, arr):
        a = _f64(np.broadcast_to(arr, self.shape3))
        self._lib.oracle_set_field(self._h, which, _dp(a))

    def rho(self) -> np.ndarray:
        self._lib.oracle_compute_rho(self._h)
        return self.get_field(RHO)

    def neutralize(self):
        self._lib.oracle_neutralize(self._h)

    def set_background(self, rho_bg):
        """Immobile background charge density at the nodes (shaped like a field)."""
        a = _f64(np.broadcast_to(rho_bg, self.shape3))
        self._lib.oracle_set_background(self._h, _dp(a))

    def particles(self, species: int = 0) -> dict:
        lib = self._lib
        n = lib.oracle_num_particles(self._h, species)
        out = np.empty((max(n, 1), 7), dtype=np.float64)
        ids = np.empty(max(n, 1), dtype=np.uint32)
        lib.oracle_get_particles(self._h, species, _dp(out), ids.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
        out, ids = out[:n], ids[:n]
        return {"x": out[:, 0], "y": out[:, 1], "z": out[:, 2], "ux": out[:, 3], "uy": out[:, 4],
                "uz": out[:, 5], "w": out[:, 6], "id": ids}

    def gather(self, x, y, z=0.0):
        E = np.zeros(3)
        B = np.zeros(3)
        self._lib.oracle_gather_point(self._h, float(x), float(y), float(z), _dp(E), _dp(B))
        return E, B

    def deposit_move(self, q, w, r0, r1, vz=0.0):
        r0, r1 = _f64(r0), _f64(r1)
        self._lib.oracle_deposit_move(self._h, float(q), float(w), _dp(r0), _dp(r1), float(vz))

    def diag(self) -> dict:
        out = np.zeros(8)
        self._lib.oracle_diag(self._h, _dp(out))
        return {"energy_field": out[0], "energy_kinetic": out[1], "charge": out[2], "gauss_max": out[3],
                "n_alive": int(out[4]), "energy_e": out[5], "energy_b": out[6]}

    @property
    def step_count(self) -> int:
        return self._lib.oracle_step_count(self._h)
