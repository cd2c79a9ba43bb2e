"""Seeded synthetic inputs shared by the CUDA path, the tests and the bench.

This module holds none of the PIC method's arithmetic: it only draws
particle positions and momenta and names the workload presets.  Both the
CUDA library and the CPU oracle are fed from it, so their inputs are
identical bit for bit.

Random numbers come from Philox4x64-10 (Salmon et al., SC'11) through
numpy's counter-based ``Philox`` bit generator.  Particle ``g`` (global
index = cell * ppc + slot, cells in row-major order i + nx*(j + ny*k)) owns
the two Philox blocks with counters 2g and 2g+1, i.e. eight raw 64-bit
draws, so any subset of cells can be regenerated on its own (this is what
the sampled full-size parity tests rely on).  Draws -> uniforms in (0, 1)
with 53 random bits; normals by the Box-Muller transform.

In the laser-target presets electrons and protons share their draws (the
same seed), so they start at the same positions: the target is neutral
node by node and E = 0 satisfies Gauss's law at t = 0.

Workload recipe (section 2 of the paper states the model; the sizes below are
the synthetic stand-ins for its laser-plasma and thermal-plasma runs and for
the two-stream test problem of its scaling study, §4.1):
positions uniform inside each cell, ``ppc`` particles per cell, momenta
u = gamma v drawn per component from N(0, u_th) plus a species drift (cold
beams/targets have u_th = 0), weight w = density / ppc, ids = global index.
A species may instead use a quiet start: its particles sit on a regular
sub-lattice of each cell (``lattice`` = points per axis), optionally with a
sinusoidal displacement along x and a sinusoidal change of ux (``perturb``),
which seeds one Fourier mode far above the discreteness noise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

TWO_PI = 2.0 * math.pi


def philox_uniforms(seed: int, first: int, count: int) -> np.ndarray:
    """(count, 8) uniforms in (0,1) for particles first .. first+count-1."""
    if count <= 0:
        return np.zeros((0, 8))
    bg = np.random.Philox(key=int(seed), counter=2 * int(first))
    raw = bg.random_raw(8 * int(count)).reshape(count, 8)
    return ((raw >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def _normals(u1, u2):
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(TWO_PI * u2), r * np.sin(TWO_PI * u2)


def particles_for_cells(cells: np.ndarray, grid: Sequence[int], d: Sequence[float], ppc: int,
                        u_th: float, w: np.ndarray | float, seed: int, dims: int,
                        drift: Sequence[float] = (0.0, 0.0, 0.0), lattice: Optional[Sequence[int]] = None,
                        perturb: Optional[Sequence[float]] = None) -> dict:
    """Particles of the given cells (row-major linear indices).

    Returns global positions (physical units), momenta u, weights and ids.
    ``w`` is a scalar or an array with one weight per listed cell.  With
    ``lattice`` = (lx, ly, lz), lx*ly*lz = ppc, positions are the sub-lattice
    points ((a + 1/2)/lx, ...) of each cell instead of random draws.  With
    ``perturb`` = (m, ax, phx, au, phu) and theta = 2 pi m x / Lx at the
    unperturbed x, x moves by ax cos(theta + phx) (periodic wrap into the
    box) and ux changes by au cos(theta + phu).
    """
    cells = np.asarray(cells, dtype=np.int64)
    nx, ny = int(grid[0]), int(grid[1])
    n = cells.size * ppc
    gidx = (cells[:, None] * ppc + np.arange(ppc)[None, :]).reshape(-1)
    # draws are contiguous per run of consecutive cells; fetch run by run
    u = np.empty((n, 8))
    if cells.size:
        breaks = np.nonzero(np.diff(cells) != 1)[0] + 1
        starts = np.concatenate([[0], breaks])
        ends = np.concatenate([breaks, [cells.size]])
        for s, e in zip(starts, ends):
            u[s * ppc:e * ppc] = philox_uniforms(seed, int(cells[s]) * ppc, int(e - s) * ppc)
    cc = np.repeat(cells, ppc)
    i = cc % nx
    j = (cc // nx) % ny
    k = cc // (nx * ny)
    if lattice is None:
        fx, fy, fz = u[:, 0], u[:, 1], u[:, 2]
    else:
        lx, ly, lz = (int(v) for v in lattice)
        if lx * ly * lz != ppc:
            raise ValueError("lattice points per cell must multiply to ppc")
        slot = np.tile(np.arange(ppc), cells.size)
        fx = (slot % lx + 0.5) / lx
        fy = ((slot // lx) % ly + 0.5) / ly
        fz = (slot // (lx * ly) + 0.5) / lz
    x = (i + fx) * d[0]
    y = (j + fy) * d[1]
    z = (k + fz) * d[2] if dims == 3 else np.zeros(n)
    dux = 0.0
    if perturb is not None:
        m, ax, phx, au, phu = (float(v) for v in perturb)
        lx_box = nx * d[0]
        theta = TWO_PI * m * x / lx_box
        x = np.mod(x + ax * np.cos(theta + phx), lx_box)
        dux = au * np.cos(theta + phu)
    n0, n1 = _normals(u[:, 3], u[:, 4])
    n2, _ = _normals(u[:, 5], u[:, 6])
    ux = u_th * n0 + drift[0] + dux
    uy = u_th * n1 + drift[1]
    uz = u_th * n2 + drift[2]
    wa = np.broadcast_to(np.asarray(w, dtype=np.float64), cells.shape)
    ww = np.repeat(wa, ppc) / ppc
    return {"x": x, "y": y, "z": z, "ux": ux, "uy": uy, "uz": uz, "w": np.ascontiguousarray(ww),
            "id": gidx.astype(np.uint32)}


@dataclass
class Species:
    name: str
    q: float
    m: float
    ppc: int
    u_th: float
    density: float = 1.0
    # columns [x0, x1) holding the species (None = whole box)
    x_range: Optional[tuple] = None
    seed_offset: int = 0
    drift: tuple = (0.0, 0.0, 0.0)      # mean momentum u added to every particle
    lattice: Optional[tuple] = None     # quiet start: sub-lattice points per axis
    perturb: Optional[tuple] = None     # quiet start: (mode, ax, phase_x, au, phase_u)
    # density structure inside x_range (see structure_mask): None (uniform),
    # ("grating", period, depth) or ("foam", fill, seed)
    structure: Optional[tuple] = None


@dataclass
class Workload:
    """A named synthetic configuration (grid, time step, shape, species)."""
    name: str
    dims: int
    n: tuple
    d: tuple
    dt: float
    order: int
    steps: int
    seed: int
    species: list = field(default_factory=list)
    sort_every: int = 20
    absorbing_x: bool = False
    laser: Optional[dict] = None
    neutralize: bool = True
    note: str = ""                      # one-line description of the plasma

    @property
    def ncells(self) -> int:
        return int(np.prod(self.n[:self.dims]))

    def species_cells(self, sp: Species) -> np.ndarray:
        nx, ny = self.n[0], self.n[1]
        nz = self.n[2] if self.dims == 3 else 1
        if sp.x_range is None:
            cells = np.arange(nx * ny * nz, dtype=np.int64)
        else:
            i = np.arange(sp.x_range[0], sp.x_range[1])
            jk = np.arange(ny * nz)
            cells = (i[None, :] + nx * jk[:, None]).reshape(-1)
        if sp.structure is not None:
            cells = cells[structure_mask(sp.structure, cells, self.n, sp.x_range)]
        return cells

    def n_particles(self) -> int:
        return sum(int(self.species_cells(s).size) * s.ppc for s in self.species)

    def particles(self, isp: int, cells: Optional[np.ndarray] = None) -> dict:
        sp = self.species[isp]
        if cells is None:
            cells = self.species_cells(sp)
        return particles_for_cells(cells, self.n, self.d, sp.ppc, sp.u_th, sp.density,
                                   self.seed * 1000 + sp.seed_offset, self.dims, sp.drift, sp.lattice,
                                   sp.perturb)


def structure_mask(structure: tuple, cells: np.ndarray, n: Sequence[int], x_range) -> np.ndarray:
    """Which of the listed cells (row-major linear indices) a structured
    target fills.  The paper shows structured targets (foams, gratings) but
    gives no specification, so these are generic shapes:

    ("grating", period, depth): the target's front surface is modulated
    along y, x_front(j) = x0 + floor(depth (1 + sin(2 pi (j + 1/2) / period)) / 2)
    cells, x0 the first column of x_range; cells in front of it are empty.

    ("foam", fill, seed): each cell is filled with probability `fill`, drawn
    once per cell from Philox (key `seed`, counter 2 * cell), so any subset
    of cells gets the same mask.
    """
    cells = np.asarray(cells, dtype=np.int64)
    kind = structure[0]
    nx, ny = int(n[0]), int(n[1])
    if kind == "grating":
        period, depth = float(structure[1]), float(structure[2])
        x0 = x_range[0] if x_range is not None else 0
        i = cells % nx
        j = (cells // nx) % ny
        front = x0 + np.floor(depth * (1.0 + np.sin(TWO_PI * (j + 0.5) / period)) / 2.0).astype(np.int64)
        return i >= front
    if kind == "foam":
        fill, seed = float(structure[1]), int(structure[2])
        u = np.empty(cells.size)
        if cells.size:
            breaks = np.nonzero(np.diff(cells) != 1)[0] + 1
            starts = np.concatenate([[0], breaks])
            ends = np.concatenate([breaks, [cells.size]])
            for a, b in zip(starts, ends):
                u[a:b] = philox_uniforms(seed, int(cells[a]), int(b - a))[:, 0]
        return u < fill
    raise ValueError(f"unknown target structure {kind!r}")


def courant_limit(d: Sequence[float], dims: int) -> float:
    """Largest stable Yee time step (c = 1): (sum 1/dx_i^2)^(-1/2)."""
    return 1.0 / math.sqrt(sum(1.0 / (x * x) for x in d[:dims]))


_NOTES = {
    "thermal2d_64": "2D3V periodic thermal plasma, electrons over immobile ions, CIC",
    "thermal3d_256": "3D3V periodic thermal plasma, electrons over immobile ions, TSC",
    "thermal3d_128": "3D3V periodic thermal plasma, electrons over immobile ions, TSC",
    "laser_slab2d": "2D3V p-polarised laser on an overdense electron-proton slab, absorbing x, TSC",
    "laser_foil3d": "3D3V linearly polarised laser on a thin electron-proton foil, absorbing x, TSC",
    "twostream3d_512": "3D3V two counter-streaming electron beams (u=+-0.2 along x) over immobile ions, "
                       "periodic, TSC (the paper's scaling test problem)",
    "grating_foil2d": "2D3V p-polarised laser at 30 degrees on a grating-fronted electron-proton foil, "
                      "absorbing x, TSC (generic grating: the paper gives no target specification)",
    "foam_foil2d": "2D3V laser on a near-critical foam layer (cells filled at random) in front of a dense foil, "
                   "absorbing x, TSC (generic foam: the paper gives no target specification)",
}


def preset(name: str) -> Workload:
    """The synthetic workloads (sizes of the paper's laser/thermal plasma runs
    and of the two-stream problem of its scaling study)."""
    wl = _preset(name)
    wl.note = _NOTES.get(name, "")
    return wl


def _preset(name: str) -> Workload:
    lam = TWO_PI  # laser wavelength in c/omega_0 units
    if name == "thermal2d_64":
        # 2D3V periodic plasma 64x64, dx=dy=0.05, dt=0.035, 16 ppc, u_th=0.01, CIC
        return Workload(name, 2, (64, 64, 1), (0.05, 0.05, 1.0), 0.035, 1, 100, 1001,
                        [Species("electron", -1.0, 1.0, 16, 0.01)])
    if name == "thermal3d_256":
        # 3D3V periodic thermal plasma 256^3, 8 ppc, u_th=0.05, TSC, sort every 20
        return Workload(name, 3, (256, 256, 256), (0.05, 0.05, 0.05), 0.028, 2, 50, 1003,
                        [Species("electron", -1.0, 1.0, 8, 0.05)])
    if name == "thermal3d_128":
        # the same plasma on a 128^3 grid (16.8M particles): profiling size
        return Workload(name, 3, (128, 128, 128), (0.05, 0.05, 0.05), 0.028, 2, 50, 1003,
                        [Species("electron", -1.0, 1.0, 8, 0.05)])
    if name == "laser_slab2d":
        d = 0.02 * lam
        dt = 0.9 * courant_limit((d, d), 2)
        return Workload(name, 2, (2048, 1024, 1), (d, d, 1.0), dt, 2, 2000, 1002,
                        [Species("electron", -1.0, 1.0, 64, 0.0, 40.0, (1024, 1064), 0),
                         Species("proton", 1.0, 1836.0, 64, 0.0, 40.0, (1024, 1064), 0)],
                        absorbing_x=True, neutralize=False,
                        laser={"a0": 3.0, "waist": 3 * lam, "duration": 10 * lam, "pol": 1})
    if name == "laser_foil3d":
        d = 0.03 * lam
        dt = 0.9 * courant_limit((d, d, d), 3)
        return Workload(name, 3, (512, 256, 256), (d, d, d), dt, 2, 1000, 1004,
                        [Species("electron", -1.0, 1.0, 27, 0.0, 50.0, (256, 276), 0),
                         Species("proton", 1.0, 1836.0, 27, 0.0, 50.0, (256, 276), 0)],
                        absorbing_x=True, neutralize=False,
                        laser={"a0": 10.0, "waist": 2 * lam, "duration": 8 * lam, "pol": 1})
    if name == "grating_foil2d":
        # foil 40 cells (0.8 lambda) thick at 40 n_c, front surface a sine
        # grating of period 1 lambda (50 cells) and depth 0.2 lambda
        d = 0.02 * lam
        dt = 0.9 * courant_limit((d, d), 2)
        grating = ("grating", 50, 10)
        return Workload(name, 2, (1024, 512, 1), (d, d, 1.0), dt, 2, 2000, 1007,
                        [Species("electron", -1.0, 1.0, 16, 0.0, 40.0, (512, 552), 0, structure=grating),
                         Species("proton", 1.0, 1836.0, 16, 0.0, 40.0, (512, 552), 0, structure=grating)],
                        absorbing_x=True, neutralize=False,
                        laser={"a0": 3.0, "waist": 3 * lam, "duration": 10 * lam, "pol": 1,
                               "angle": math.radians(30.0)})
    if name == "foam_foil2d":
        # a foam layer 2.2 lambda thick whose cells are filled with
        # probability 1/4 at 5 n_c (1.25 n_c on average), then a 0.4 lambda
        # foil at 40 n_c
        d = 0.02 * lam
        dt = 0.9 * courant_limit((d, d), 2)
        foam = ("foam", 0.25, 4242)
        return Workload(name, 2, (1024, 512, 1), (d, d, 1.0), dt, 2, 2000, 1008,
                        [Species("foam_e", -1.0, 1.0, 16, 0.0, 5.0, (400, 512), 0, structure=foam),
                         Species("foam_p", 1.0, 1836.0, 16, 0.0, 5.0, (400, 512), 0, structure=foam),
                         Species("foil_e", -1.0, 1.0, 16, 0.0, 40.0, (512, 532), 1),
                         Species("foil_p", 1.0, 1836.0, 16, 0.0, 40.0, (512, 532), 1)],
                        absorbing_x=True, neutralize=False,
                        laser={"a0": 5.0, "waist": 3 * lam, "duration": 10 * lam, "pol": 1})
    if name == "twostream3d_512":
        # the two-stream problem of the paper's scaling runs: 512x512x128
        # cells, 54 ppc (two counter-streaming electron beams of 27 ppc each,
        # u = +-0.2 along x, small spread), immobile neutralising ions
        return Workload(name, 3, (512, 512, 128), (0.05, 0.05, 0.05), 0.028, 2, 50, 1006,
                        [Species("beam+", -1.0, 1.0, 27, 0.002, 0.5, None, 0, (0.2, 0.0, 0.0)),
                         Species("beam-", -1.0, 1.0, 27, 0.002, 0.5, None, 1, (-0.2, 0.0, 0.0))])
    raise KeyError(name)


def two_stream(n: tuple, d: float, u0: float, ppc_lattice: tuple, seeds=(None, None), order: int = 2,
               dt_frac: float = 0.9, density: float = 1.0, seed: int = 77) -> Workload:
    """Two cold counter-streaming electron beams (drift momentum +-u0 along
    x, each of half the density) on a quiet-start lattice, periodic, 2D3V
    (len(n) == 2) or 3D3V; ``seeds`` gives each beam's ``perturb`` tuple
    (see particles_for_cells).  The neutralising background is the
    caller's (a uniform +density)."""
    dims = len(n)
    dd = (d, d, d if dims == 3 else 1.0)
    dt = dt_frac * courant_limit(dd, dims)
    nn = tuple(n) + (1,) * (3 - dims)
    ppc = int(np.prod(ppc_lattice))
    lat = tuple(ppc_lattice) + (1,) * (3 - len(ppc_lattice))
    return Workload(f"twostream{dims}d", dims, nn, dd, dt, order, 0, seed,
                    [Species("beam+", -1.0, 1.0, ppc, 0.0, 0.5 * density, None, 0, (u0, 0.0, 0.0), lat, seeds[0]),
                     Species("beam-", -1.0, 1.0, ppc, 0.0, 0.5 * density, None, 1, (-u0, 0.0, 0.0), lat,
                             seeds[1])], neutralize=False)


def small(dims: int, n: tuple, order: int, ppc: int, u_th: float, seed: int, dt_frac: float = 0.95,
          d: float = 0.05) -> Workload:
    """A small periodic thermal plasma for parity tests."""
    dd = (d, d, d if dims == 3 else 1.0)
    dt = dt_frac * courant_limit(dd, dims)
    nn = tuple(n) + (1,) * (3 - len(n))
    return Workload(f"small{dims}d", dims, nn, dd, dt, order, 10, seed,
                    [Species("electron", -1.0, 1.0, ppc, u_th)])


# ---------------------------------------------------------------------------
# Parallel generation into file-backed shared arrays (large workloads)
# ---------------------------------------------------------------------------
_FIELDS = (("x", np.float64), ("y", np.float64), ("z", np.float64), ("ux", np.float64), ("uy", np.float64),
           ("uz", np.float64), ("w", np.float64), ("id", np.uint32))


def _fill_chunk(args):
    wl, isp, c0, c1, base, paths, n_total = args
    sp = wl.species[isp]
    cells = wl.species_cells(sp)[c0:c1]
    p = wl.particles(isp, cells)
    for (key, dt), path in zip(_FIELDS, paths):
        arr = np.memmap(path, dtype=dt, mode="r+", shape=(n_total,))
        arr[(c0 - base) * sp.ppc:(c1 - base) * sp.ppc] = p[key]
        arr.flush()
        del arr
    return c1 - c0


def _scratch_dir(nbytes: int):
    """A directory with room for nbytes of scratch files: the temporary
    directory, else /dev/shm; None (the default) when neither has room."""
    import os
    import shutil
    import tempfile
    for d in (tempfile.gettempdir(), "/dev/shm"):
        try:
            if os.path.isdir(d) and shutil.disk_usage(d).free > 1.2 * nbytes:
                return d
        except OSError:
            continue
    return None


class SharedParticles:
    """Particle arrays of one species in memory-mapped temporary files, filled
    by a pool of worker processes (spawned, so it is safe after CUDA has
    started).  ``arrays`` maps x, y, z, ux, uy, uz, w, id to numpy views.
    ``cell_range`` = (c0, c1) restricts it to the species' cells c0 .. c1-1
    (positions in ``Workload.species_cells`` order), so that a very large
    species can be generated and loaded piece by piece; ``pool`` reuses a
    caller's process pool."""

    def __init__(self, wl: Workload, isp: int, nproc: int = 0, chunk_cells: int = 65536,
                 cell_range: Optional[tuple] = None, pool=None):
        import multiprocessing as mp
        import os
        import tempfile
        sp = wl.species[isp]
        ncells = int(wl.species_cells(sp).size)
        c0, c1 = (0, ncells) if cell_range is None else (int(cell_range[0]), int(min(cell_range[1], ncells)))
        self.n = max(c1 - c0, 0) * sp.ppc
        self._dir = tempfile.mkdtemp(prefix="picsynth_", dir=_scratch_dir(self.n * 60))
        self.paths = [os.path.join(self._dir, key + ".bin") for key, _ in _FIELDS]
        for (key, dt), path in zip(_FIELDS, self.paths):
            with open(path, "wb") as f:
                f.truncate(max(self.n, 1) * np.dtype(dt).itemsize)
        jobs = [(wl, isp, c, min(c + chunk_cells, c1), c0, self.paths, self.n) for c in range(c0, c1, chunk_cells)]
        nproc = nproc or min(16, os.cpu_count() or 1)
        if pool is not None and len(jobs) > 1:
            for _ in pool.imap_unordered(_fill_chunk, jobs):
                pass
        elif nproc <= 1 or len(jobs) <= 1:
            for j in jobs:
                _fill_chunk(j)
        else:
            with mp.get_context("spawn").Pool(nproc) as own:
                for _ in own.imap_unordered(_fill_chunk, jobs):
                    pass
        self.arrays = {key: np.memmap(path, dtype=dt, mode="r+", shape=(max(self.n, 1),))[:self.n]
                       for (key, dt), path in zip(_FIELDS, self.paths)}

    def close(self):
        import shutil
        self.arrays = {}
        if getattr(self, "_dir", None):
            shutil.rmtree(self._dir, ignore_errors=True)
            self._dir = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
