"""Differentiable laser-slab run: gradients of the rear-electron kinetic
energy with respect to the laser amplitude and the initial density profile.

The forward run is the 2D3V PIC cycle of the library (FP32 or FP64) with a
laser entering through an absorbing x = 0 wall; the backward pass is the
library's hand-written adjoint (Yee and Mur walls, gather, Boris, move,
Esirkepov deposit), with FP64 gradient accumulation.  The forward state is
checkpointed every `segment` steps; the backward pass restores each
checkpoint, re-runs its segment with the step tape on and reverses it.

Workload (a reading of the paper's laser-target studies, §2 and Fig. 1):
2D grid nx x ny, dx = dy = 0.05 lambda, dt = 0.9 x the 2D Courant limit, TSC;
electrons at `ppc` per cell in every cell with weight n(x column) / ppc
(zero-weight tracers where the profile is zero), immobile neutralising ions;
laser polarised along y, Gaussian waist, sin^2 envelope; objective = FP64
kinetic energy of the electrons in columns [obj_lo, obj_hi) at the end.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import synth
from .sim import Simulation

TAU = 2.0 * math.pi


@dataclass
class SlabRun:
    nx: int = 256
    ny: int = 256
    ppc: int = 16
    steps: int = 200
    segment: int = 20
    slab: tuple = (64, 84)          # columns of the initial slab
    density: float = 20.0           # n / n_c in the slab
    obj: tuple = (84, 116)          # objective columns (behind the slab)
    waist: float = 3 * TAU
    duration: float = 4 * TAU
    seed: int = 1005
    precision: str = "fp32"
    # True: the forward records every step (no recomputation in the reverse
    # sweep; about 38 MB per step at the default size, FP32); False: a
    # checkpoint every `segment` steps, each segment recomputed with its
    # steps recorded during the reverse sweep
    store_all: bool = False

    @property
    def d(self) -> float:
        return 0.05 * TAU

    @property
    def dt(self) -> float:
        return 0.9 * synth.courant_limit((self.d, self.d), 2)

    def default_profile(self) -> np.ndarray:
        prof = np.zeros(self.nx)
        prof[self.slab[0]:self.slab[1]] = self.density
        return prof

    def workload(self, a0: float) -> synth.Workload:
        return synth.Workload("laser_slab_diff", 2, (self.nx, self.ny, 1), (self.d, self.d, 1.0), self.dt, 2,
                              self.steps, self.seed, [synth.Species("electron", -1.0, 1.0, self.ppc, 0.0)],
                              sort_every=self.segment, absorbing_x=True, neutralize=True,
                              laser={"a0": float(a0), "waist": self.waist, "duration": self.duration, "pol": 1})

    def particles(self, profile: np.ndarray) -> dict:
        """Electrons of every cell except the absorbing margins, weights from
        the column profile."""
        wl = self.workload(1.0)
        cols = np.arange(3, self.nx - 4)
        cells = (cols[None, :] + self.nx * np.arange(self.ny)[:, None]).reshape(-1)
        cells.sort()
        w_cell = np.asarray(profile, dtype=np.float64)[cells % self.nx]
        return synth.particles_for_cells(cells, wl.n, wl.d, self.ppc, 0.0, w_cell, wl.seed * 1000, 2)

    @property
    def id_capacity(self) -> int:
        return self.nx * self.ny * self.ppc

    def column_of_id(self, ids: np.ndarray) -> np.ndarray:
        return (ids // self.ppc) % self.nx


_BINS = {}


def _column_bins(run: SlabRun):
    """The initial column of every particle id (int32), kept in device memory
    (a CUDA tensor) once made."""
    key = (run.nx, run.ppc, run.id_capacity)
    if key not in _BINS:
        bins = run.column_of_id(np.arange(run.id_capacity)).astype(np.int32)
        import torch
        _BINS[key] = torch.from_numpy(bins).cuda() if torch.cuda.is_available() else bins
    return _BINS[key]


def build_sim(run: SlabRun, a0: float, profile: np.ndarray) -> Simulation:
    """Simulation of the run with its electrons loaded (no steps taken)."""
    wl = run.workload(a0)
    sim = Simulation.from_workload(wl, precision=run.precision)
    parts = run.particles(profile)
    sp = sim.add_species(-1.0, 1.0, len(parts["x"]))
    sim.load(sp, parts)
    sim.neutralize()
    return sim


def run_forward(run: SlabRun, sim: Simulation) -> float:
    """The forward steps, with a checkpoint at the start of every segment but
    the last, whose steps are recorded (or every step recorded,
    run.store_all); returns F (and leaves the adjoint seeded)."""
    if run.store_all:
        sim.tape_begin(run.steps)
        sim.step(run.steps)
    else:
        nseg = run.steps // run.segment
        for k in range(nseg - 1):
            sim.checkpoint(k)
            sim.step(run.segment)
        # the last segment is recorded as it runs, so that the reverse sweep
        # starts without recomputing it
        sim.tape_begin(run.segment)
        sim.step(run.segment)
    sim.adjoint_begin(run.id_capacity)
    return sim.adjoint_seed_kinetic(0, run.obj[0], run.obj[1])


def forward_objective(run: SlabRun, a0: float, profile: np.ndarray, keep: bool = False):
    """Run the forward pass with checkpoints; returns (F, sim or None)."""
    sim = build_sim(run, a0, profile)
    F = run_forward(run, sim)
    if not keep:
        sim.close()
        return F, None
    return F, sim


def backward_gradients(run: SlabRun, sim: Simulation):
    """Reverse sweep over the recorded steps (run.store_all) or the
    checkpointed segments; returns (dF/da0, dF/dprofile[nx])."""
    if run.store_all:
        # the adjoint was seeded at the end of the forward pass
        sim.adjoint_step(run.steps)
        dprof = sim.grad_binned(0, _column_bins(run), run.nx) / run.ppc
        return sim.grad_a0(), dprof
    nseg = run.steps // run.segment
    # the last segment was recorded by the forward pass, which also seeded
    # the adjoint at the final state
    sim.adjoint_step(run.segment)
    for k in reversed(range(nseg - 1)):
        sim.restore(k)
        sim.tape_begin(run.segment)
        # only the start state of the segment's last step is needed
        sim.step(run.segment - 1)
        sim.tape_record()
        sim.adjoint_step(run.segment)
    # dF/dprofile[k] = sum of dF/dw over the electrons of column k / ppc,
    # summed on the device
    dprof = sim.grad_binned(0, _column_bins(run), run.nx) / run.ppc
    return sim.grad_a0(), dprof


def make_function():
    """torch.autograd.Function: F = PicRun.apply(a0, profile) for a SlabRun."""
    import torch

    class PicRun(torch.autograd.Function):
        @staticmethod
        def forward(ctx, a0, profile, run: SlabRun):
            F, sim = forward_objective(run, float(a0.item()), profile.detach().cpu().numpy(), keep=True)
            ctx.sim, ctx.run = sim, run
            return torch.tensor(F, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gF):
            da0, dprof = backward_gradients(ctx.run, ctx.sim)
            ctx.sim.close()
            g = float(gF)
            return (torch.tensor(g * da0, dtype=torch.float64),
                    torch.as_tensor(g * dprof, dtype=torch.float64), None)

    return PicRun


def main(argv=None):
    """Run the differentiable laser-slab problem once: forward with
    checkpoints, then the adjoint; print the objective, dF/da0, the profile
    gradient's norm and the wall times."""
    import argparse
    import time

    import torch

    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--a0", type=float, default=2.0)
    ap.add_argument("--repeat", type=int, default=2, help="runs (the first warms up)")
    ap.add_argument("--store-all", action="store_true", help="record every forward step (no recomputation)")
    args = ap.parse_args(argv)
    run = SlabRun(precision=args.precision, store_all=args.store_all)
    prof = run.default_profile()
    for _ in range(args.repeat):
        sim = build_sim(run, args.a0, prof)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        F = run_forward(run, sim)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        da0, dprof = backward_gradients(run, sim)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        sim.close()
        print(f"F = {F:.10e}  dF/da0 = {da0:.10e}  |dF/dprofile| = {np.linalg.norm(dprof):.6e}  "
              f"forward {1e3 * (t1 - t0):.1f} ms  backward {1e3 * (t2 - t1):.1f} ms  "
              f"ratio {(t2 - t1) / (t1 - t0):.2f}", flush=True)


if __name__ == "__main__":
    main()
