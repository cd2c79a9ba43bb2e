"""Throughput benchmark of the GB300 PIC hot path.

Default workload: the 3D3V periodic thermal plasma, 256^3 cells, 8 electrons
per cell (134,217,728 macro-particles), u_th = 0.05, TSC shape, dx = 0.05,
dt = 0.028, FP32 cell-relative push/deposit, particle sort every 20 steps.
One "step" is one full PIC cycle (sort when due, J reset, fused
gather/Boris/move/Esirkepov kernel, three Yee updates).  Metric:
particle-steps/s = live particles x steps / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Prints one JSON line (rank 0).  Under torchrun with N > 1 every rank runs an
independent replica of the workload on its own GPU (the path has no exchange
step on one GPU; see the design notes), times are max-reduced over ranks and
`value` is the aggregate over all ranks.

`--impl reference` times the FP64 CPU oracle instead (the only other place
this script runs it), on a bounded sub-box of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1503_02464_gb300 import synth  # noqa: E402

WORKLOAD = "thermal3d_256"
# algorithmic bytes of the fused push kernel (FP32, 3D): per particle it
# reads cell(4) + offset(12) + u(12) + w(4) and writes cell(4) + offset(12) +
# u(12) = 60 B; per cell it reads E, B (24 B) once and adds J (12 B read +
# 12 B write) once = 48 B.
PUSH_BYTES_PER_PARTICLE = {"fp32": 60, "fp64": 4 + 24 + 24 + 8 + 4 + 24 + 24}
PUSH_BYTES_PER_CELL = {"fp32": 48, "fp64": 96}
# DRAM bytes (read + write) per particle of one push launch, from an ncu
# capture of the push kernel on the 128^3 case of the same plasma (scaled by
# the particle count); None for workloads and precisions not captured, and
# once the kernel changes.
# Algorithmic flops of the fused push per particle-step, by (dims, shape
# order): gather weights and staggered sums, Boris and move, Esirkepov
# weights, brackets and the products of the full compact stencil (NW = order
# + 2 nodes per axis, no data-dependent skipping); an FMA counts as 2.  The
# breakdown is in the design notes (section 5).
PUSH_FLOPS_PER_PARTICLE = {(3, 2): 1117, (3, 1): 496, (2, 2): 445, (2, 1): 251}
FP32_LANES_PER_SM = 128  # FP32 FMA lanes per SM (nominal roof, quoted beside the measured one)
PUSH_TRAFFIC_PER_PARTICLE = {("thermal3d_256", "fp32"): 62.8, ("thermal3d_128", "fp32"): 62.8}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            # raw samples (the JSON line carries their summary): PIC_CLOCK_DIR, else the temp directory
            out_dir = os.environ.get("PIC_CLOCK_DIR") or tempfile.gettempdir()
            os.makedirs(out_dir, exist_ok=True)
            self.path = os.path.join(out_dir, f"clocks_{os.getpid()}.csv")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- CPU oracle arm
def oracle_sample_workload(wl, ncell_axis: int):
    """A periodic sub-box of the workload with the same cell size, dt, shape,
    density, temperature and particles per cell."""
    n = (ncell_axis,) * wl.dims + (1,) * (3 - wl.dims)
    return synth.Workload(wl.name + f"_sample{ncell_axis}", wl.dims, n, wl.d, wl.dt, wl.order, wl.steps,
                          wl.seed, wl.species, wl.sort_every)


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


# periodic sub-box edge (cells) of the oracle samples: 3D 64^3, 2D 512^2
ORACLE_SAMPLE_CELLS = {3: 64, 2: 512}


def oracle_baseline(wl, nsteps: int, warmup: int = 0) -> dict:
    """The FP64 oracle (OpenMP build, every host core) on a periodic sub-box
    of the workload: particle-steps/s and a description of the sample."""
    import oracle
    sample = oracle_sample_workload(wl, ORACLE_SAMPLE_CELLS[wl.dims])
    npart, times = time_oracle(sample, nsteps, warmup, parallel=True)
    cores = oracle.num_threads(parallel=True)
    tot = sum(times)
    desc = (f"FP64 C oracle, OpenMP on {cores} threads ({os.cpu_count()} host CPUs, {cpu_model()}), periodic "
            f"{'x'.join(map(str, sample.n[:sample.dims]))} sub-box of {wl.name} ({npart} particles, same dx, dt, "
            f"ppc, u_th, shape), {len(times)} steps, {tot:.1f} s")
    return {"value": npart * len(times) / tot, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
            "sample": desc, "npart": npart, "times": times,
            "shape": "x".join(map(str, sample.n[:sample.dims]))}


def time_oracle(wl, nsteps: int, warmup: int = 0, parallel: bool = False):
    import oracle
    o = oracle.OracleSim(wl.dims, wl.n, wl.d, wl.dt, wl.order, parallel=parallel)
    npart = 0
    for isp, sp in enumerate(wl.species):
        p = wl.particles(isp)
        o.add_particles(p, sp.q, sp.m)
        npart += len(p["x"])
    o.neutralize()
    if warmup:
        o.step(warmup)
    times = []
    for _ in range(nsteps):
        t0 = time.perf_counter()
        o.step(1)
        times.append(time.perf_counter() - t0)
    o.close()
    return npart, times


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    wl = synth.preset(args.workload)
    cpu = oracle_baseline(wl, args.steps, args.warmup)
    value, times = cpu["value"], cpu["times"]
    tot = sum(times)
    line = {"impl": "reference", "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "sample": cpu["shape"], "particles": cpu["npart"]},
            "cpu_baseline": {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU arm
def parse_cpulist(spec: str) -> set:
    """CPUs of a sysfs list such as "0-3,8,10-11"."""
    cpus = set()
    for part in spec.strip().split(","):
        if not part:
            continue
        a, _, b = part.partition("-")
        cpus.update(range(int(a), int(b or a) + 1))
    return cpus


def pci_sysfs_name(bus_id: str) -> str:
    """sysfs device name of an nvidia-smi PCI bus id ("00000009:01:00.0" ->
    "0009:01:00.0")."""
    dom, rest = bus_id.strip().split(":", 1)
    return f"{int(dom, 16):04x}:{rest.lower()}"


def _gpu_local_cpus(gpu: int):
    """CPUs on the NUMA node of the GPU (from sysfs), or None."""
    try:
        bus = subprocess.run(["nvidia-smi", "-i", str(gpu), "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=30).stdout
        with open(f"/sys/bus/pci/devices/{pci_sysfs_name(bus)}/local_cpulist") as f:
            return parse_cpulist(f.read()) or None
    except Exception:
        return None


def _dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _barrier_max(world, value: float) -> float:
    """Max of `value` over the ranks (the slowest replica sets the time)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_workload(name: str, rank: int, world: int):
    """The workload of one rank: the same preset, an independent seed per
    replica (the path does not shard: N GPUs run N replicas)."""
    wl = synth.preset(name)
    if world > 1:
        wl.seed += 7919 * rank
    return wl


def aggregate_rate(world: int, npart: int, steps: int, seconds: float) -> float:
    """Whole-job particle-steps/s: every rank's particles over the max time."""
    return world * npart * steps / seconds


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def generate(wl, isp, nproc, world=1):
    """Host inputs of one species; with N replicas on one host the
    generator processes are shared out between the ranks."""
    nproc = nproc or max(1, min(16, (os.cpu_count() or 1) // max(world, 1)))
    return synth.SharedParticles(wl, isp, nproc=nproc)


# Above STREAM_PARTICLES the inputs are not held on the host in full: each
# species is generated and loaded CHUNK_PARTICLES at a time (appending loads).
STREAM_PARTICLES = 1 << 28
CHUNK_PARTICLES = 1 << 25


def run_gpu(args, rank: int, world: int, local: int):
    import torch
    from paper_1503_02464_gb300 import capi
    from paper_1503_02464_gb300.sim import Simulation

    wl = replica_workload(args.workload, rank, world)
    streamed = wl.n_particles() > STREAM_PARTICLES
    # host inputs first (spawned pool, before the first CUDA call)
    t_gen = time.perf_counter()
    pool = None
    if streamed:
        import multiprocessing as mp
        host = []
        pool = mp.get_context("spawn").Pool(args.nproc or min(16, os.cpu_count() or 1))
        if not args.no_e2e:
            print("bench: e2e leg skipped (inputs of this size are generated piece by piece)", file=sys.stderr)
            args.no_e2e = True
    else:
        host = [generate(wl, isp, args.nproc, world) for isp in range(len(wl.species))]
    t_gen = time.perf_counter() - t_gen

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    capi.load()
    stream = torch.cuda.current_stream()
    npart = wl.n_particles() if streamed else sum(h.n for h in host)
    ncell = wl.ncells

    def make_sim(precision):
        return Simulation.from_workload(wl, precision=precision, stream=stream.cuda_stream)

    def load_device(sim):
        if streamed:
            for isp, sp in enumerate(wl.species):
                ncs = int(wl.species_cells(sp).size)
                s = sim.add_species(sp.q, sp.m, ncs * sp.ppc)
                step = max(CHUNK_PARTICLES // sp.ppc, 1)
                for c0 in range(0, ncs, step):
                    h = synth.SharedParticles(wl, isp, cell_range=(c0, c0 + step), pool=pool)
                    dev = {k: torch.from_numpy(v).to("cuda") for k, v in h.arrays.items()}
                    sim.load(s, dev)
                    del dev
                    h.close()
        else:
            for isp, (sp, h) in enumerate(zip(wl.species, host)):
                s = sim.add_species(sp.q, sp.m, h.n)
                dev = {k: torch.from_numpy(v).to("cuda") for k, v in h.arrays.items()}
                sim.load(s, dev)
                del dev
        if wl.neutralize:
            sim.neutralize()

    def timed_steps(sim, k):
        """K steps between device events on the simulation's stream."""
        _barrier(world)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(k)
        e1.record(stream)
        torch.cuda.synchronize()
        _barrier(world)
        return e0.elapsed_time(e1) / 1e3

    results = {}
    # ---------------- FP32 device-resident run (the headline value)
    sim = make_sim(args.precision)
    t_load = time.perf_counter()
    load_device(sim)
    torch.cuda.synchronize()
    t_load = time.perf_counter() - t_load
    sim.step(args.warmup)
    torch.cuda.synchronize()
    l0 = sim.launch_count()
    sim.profile(True)
    clocks = ClockSampler(local)
    clocks.start()
    dt_s = timed_steps(sim, args.steps)
    clk = clocks.stop()
    tim = sim.timings()
    launches = sim.launch_count() - l0
    td = time.perf_counter()
    d = sim.diag()  # FP64 diagnostics (charge deposit, Gauss, energies), synchronising
    diag_ms = 1e3 * (time.perf_counter() - td)
    sim.profile(False)
    dt_max = _barrier_max(world, dt_s)
    push_ms, push_n = tim["push"]
    results["main"] = dict(dt=dt_max, tim=tim, launches=launches, diag=d, clocks=clk, diag_ms=diag_ms)
    sim.close()
    del sim
    torch.cuda.synchronize()

    # ---------------- FP64 path on the same workload (fewer steps)
    fp64 = None
    # FP64 record: cell 4 + offsets 24 + u 24 + w 8 + id 4 = 64 B, double-buffered, + a 4 B sort rank
    fp64_bytes = npart * (2 * 64 + 4)
    if args.fp64_steps > 0 and fp64_bytes > 0.8 * torch.cuda.get_device_properties(local).total_memory:
        fp64 = {"skipped": f"FP64 particle storage of this workload ({fp64_bytes / 1e9:.0f} GB) exceeds 80 % "
                           f"of device memory"}
    elif args.fp64_steps > 0:
        sim = make_sim("fp64")
        load_device(sim)
        sim.step(min(args.warmup, 3))
        sim.profile(True)
        dt64 = _barrier_max(world, timed_steps(sim, args.fp64_steps))
        t64 = sim.timings()
        sim.profile(False)
        sim.close()
        del sim
        p64_ms, p64_n = t64["push"]
        fp64 = {"value": aggregate_rate(world, npart, args.fp64_steps, dt64), "unit": "particle-steps/s",
                "ms_per_step": 1e3 * dt64 / args.fp64_steps, "steps": args.fp64_steps,
                "push_ms_per_launch": p64_ms / max(p64_n, 1)}
        torch.cuda.synchronize()

    # ---------------- FP64 diagnostics over a long run (optional, after the timed regions)
    history = None
    if args.history > 0 and rank == 0:
        sim = make_sim(args.precision)
        load_device(sim)
        every = max(1, args.history_every)
        hist = []
        for t in range(0, args.history + 1, every):
            if t:
                sim.step(every)
            dg = sim.diag()
            hist.append({k: dg[k] for k in ("step", "energy_field", "energy_kinetic", "charge", "gauss_max",
                                            "continuity_max", "n_alive", "n_absorbed") if k in dg})
        sim.close()
        del sim
        torch.cuda.synchronize()
        history = {"steps": args.history, "every": every, "precision": args.precision, "diag": hist}

    # ---------------- adjoint / forward time of the differentiable run
    adjoint = None
    if not args.no_adjoint and rank == 0:
        import dataclasses

        from paper_1503_02464_gb300 import diff
        run = diff.SlabRun(precision="fp32")
        prof = run.default_profile()

        def timed_runs(r):
            reps = []
            for rep in range(4):  # the first repetition warms up; the median of the other three is reported
                sim = diff.build_sim(r, 2.0, prof)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                F = diff.run_forward(r, sim)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                da0, dprof = diff.backward_gradients(r, sim)
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                sim.close()
                if rep:
                    reps.append((t1 - t0, t2 - t1))
            return reps, F, da0

        reps, F, da0 = timed_runs(run)
        fwd_s, bwd_s = sorted(reps, key=lambda r: r[1] / r[0])[len(reps) // 2]
        # every forward step recorded instead (no recomputation), memory permitting
        store_all = None
        free_b, _ = torch.cuda.mem_get_info()
        tape_b = run.steps * run.id_capacity * (4 * 4 + 4 * 4) + run.steps * 6 * 4 * run.nx * run.ny
        if tape_b < 0.5 * free_b:
            reps_a, _, da0_a = timed_runs(dataclasses.replace(run, store_all=True))
            f_a, b_a = sorted(reps_a, key=lambda r: r[1] / r[0])[len(reps_a) // 2]
            store_all = {"forward_s": f_a, "backward_s": b_a, "ratio": b_a / f_a, "ratios": [b / f for f, b in reps_a],
                         "tape_bytes": tape_b, "dF_da0": da0_a,
                         "note": "forward records all steps (device memory), reverse sweep without recomputation"}
        # one more run with per-kernel-class events, for the breakdown only
        sim = diff.build_sim(run, 2.0, prof)
        sim.profile(True)
        diff.run_forward(run, sim)
        diff.backward_gradients(run, sim)
        adj_kernels = {k: {"ms_total": v[0], "launches": v[1]} for k, v in sim.timings().items() if v[1]}
        sim.profile(False)
        sim.close()
        adjoint = {"workload": f"2D3V laser slab {run.nx}x{run.ny}, {run.ppc} ppc ({run.nx * run.ny * run.ppc} "
                               f"electron slots), TSC, {run.steps} steps, checkpoint every {run.segment}, FP32 "
                               f"forward/adjoint, FP64 gradients",
                   "forward_s": fwd_s, "backward_s": bwd_s, "ratio": bwd_s / fwd_s,
                   "ratios": [b / f for f, b in reps],
                   "note": "backward includes re-running every segment with the tape on; median of three "
                           "repetitions after a warm-up",
                   "kernel_ms": adj_kernels,
                   "objective": F, "dF_da0": da0, "store_all": store_all}

    # ---------------- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        # The inputs start in page-locked host buffers allocated (and first
        # touched) from the CPUs next to this GPU: the generated arrays live in
        # scratch files whose pages may sit on another NUMA node, which made
        # the same copy 5x slower on some runs.
        aff = os.sched_getaffinity(0) if hasattr(os, "sched_getaffinity") else None
        near = _gpu_local_cpus(local)
        if aff is not None and near and near & aff:
            os.sched_setaffinity(0, near & aff)
        pinned = [{k: torch.from_numpy(np.asarray(v).view(np.int32) if v.dtype == np.uint32 else np.asarray(v))
                   .pin_memory() for k, v in h.arrays.items()} for h in host]
        # One untimed load of the same page-locked buffers first: the first
        # copy engine pass over freshly pinned pages ran at 60-130 GB/s, every
        # later one at 205 GB/s (one-time translation set-up of the pages).
        sim = make_sim(args.precision)
        for sp, h in zip(wl.species, host):
            sim.add_species(sp.q, sp.m, h.n)
        for isp in range(len(host)):
            sim.load(isp, pinned[isp])
        sim.close()
        sim = make_sim(args.precision)
        for sp, h in zip(wl.species, host):
            sim.add_species(sp.q, sp.m, h.n)
        Ex = np.empty(sim.shape3, dtype=np.float64)
        torch.cuda.synchronize()
        _barrier(world)
        t0 = time.perf_counter()
        for isp in range(len(host)):
            sim.load(isp, pinned[isp])        # pinned host -> device inside the call
        t_copy = time.perf_counter() - t0
        if wl.neutralize:
            sim.neutralize()
        sim.sync()
        t_load_e2e = time.perf_counter() - t0
        t_diag = 0.0
        for _ in range(args.steps):
            sim.step(1)
            td = time.perf_counter()
            dg = sim.energy()                 # FP64 energies read back every step
            t_diag += time.perf_counter() - td
        sim.sync()
        t1 = time.perf_counter()
        _barrier(world)
        e2e_s = _barrier_max(world, t1 - t0)
        sim.close()
        del sim
        del pinned
        if aff is not None:
            os.sched_setaffinity(0, aff)
        h2d = sum(sum(v.nbytes for v in h.arrays.values()) for h in host)
        d2h = 5 * 8
        e2e = {"value": aggregate_rate(world, npart, args.steps, e2e_s), "unit": "particle-steps/s",
               "h2d_bytes_per_step": int(h2d / args.steps), "d2h_bytes_per_step": d2h,
               "pinned": True,
               "load_s": t_load_e2e, "load_copy_s": t_copy, "diag_wall_ms_per_step": 1e3 * t_diag / args.steps,
               "note": "load from pinned host (chunked copy-engine staging) + neutralize + per-step pic_step + "
                       "pic_energy read-back, wall clock; the same pinned buffers were loaded once before, untimed "
                       "(warm-up)"}

    # ---------------- CPU oracle baseline (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        c = oracle_baseline(wl, args.cpu_steps)
        cpu = {k: c[k] for k in ("value", "unit", "cores", "kind", "sample")}

    for h in host:
        h.close()
    if pool is not None:
        pool.close()
        pool.join()

    alu_peaks = capi.pic_alu_peak(stream.cuda_stream)  # FP32, FP64 FMA TFLOP/s of this device
    if rank != 0:
        return
    r = results["main"]
    value = aggregate_rate(world, npart, args.steps, r["dt"])
    peak, peak_kind = _peaks()
    push_avg_s = push_ms / max(push_n, 1) / 1e3
    # one push launch moves one species (equal sizes here) and its windows of every tile
    alg_bytes = (npart // max(len(wl.species), 1)) * PUSH_BYTES_PER_PARTICLE[args.precision] + \
        ncell * PUSH_BYTES_PER_CELL[args.precision]
    achieved = alg_bytes / push_avg_s / 1e9
    # the ALU roof of the same launch: FMA throughput measured on this device
    # (pic_alu_peak, after the timed regions), the nominal roof beside it
    flops_pp = PUSH_FLOPS_PER_PARTICLE[(wl.dims, wl.order)]
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    sm_max_mhz = (r["clocks"] or {}).get("sm_max_mhz") or 2070.0
    nominal_alu = nsm * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    peak_alu, peak64_alu = alu_peaks
    flops_launch = (npart // max(len(wl.species), 1)) * flops_pp
    achieved_alu = flops_launch / push_avg_s / 1e12
    if fp64 is not None and "push_ms_per_launch" in fp64:
        a64 = flops_launch / (fp64["push_ms_per_launch"] / 1e3) / 1e12
        fp64["alu"] = {"achieved": a64, "peak": peak64_alu, "unit": "TFLOP/s", "frac": a64 / peak64_alu,
                       "peak_kind": "measured FP64 FMA-chain kernel (pic_alu_peak)"}
    tim_out = {k: {"ms_total": v[0], "launches": v[1]} for k, v in r["tim"].items() if v[1]}
    line = {
        "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * r["dt"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": f"{wl.name}: {wl.note}, "
                               f"{'x'.join(map(str, wl.n[:wl.dims]))} cells, "
                               f"{sum(sp.ppc for sp in wl.species)} ppc, {npart} particles, "
                               f"u_th={wl.species[0].u_th}, dx={wl.d[0]}, dt={wl.dt}, "
                               f"sort every {wl.sort_every}",
                   "particles": npart, "cells": ncell, "precision": args.precision,
                   "l2": "inputs larger than L2 (particle arrays > 4 GB, fields 0.6 GB)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": (PUSH_TRAFFIC_PER_PARTICLE.get((wl.name, args.precision)) or 0) *
                                (npart // max(len(wl.species), 1)) or None,
                     "kernel": "k_push (fused gather/Boris/move/Esirkepov)",
                     "peak_kind": f"{peak_kind} HBM copy bandwidth",
                     "bytes_per_launch": alg_bytes, "ms_per_launch": push_avg_s * 1e3},
        # the same launch against the FP32 ALU roof (by arithmetic intensity the
        # 3D TSC push is ALU-bound, not HBM-bound)
        "roofline_alu": {"bound": "alu", "achieved": achieved_alu, "peak": peak_alu, "unit": "TFLOP/s",
                         "frac": achieved_alu / peak_alu, "flops_per_particle": flops_pp,
                         "flops_per_launch": flops_launch,
                         "peak_kind": "measured FP32 FMA-chain kernel (pic_alu_peak)",
                         "nominal": nominal_alu,
                         "nominal_kind": f"{nsm} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                                         f"{sm_max_mhz:.0f} MHz max SM clock"},
        "kernel_times": tim_out,
        # the Yee updates against the same copy bandwidth: a B half reads E, B
        # and writes B (9 arrays of the grid), the E update reads E, B, J and
        # writes E (12 arrays)
        "roofline_fields": {
            k: {"bound": "hbm", "achieved": nb * ncell * (4 if args.precision == "fp32" else 8) /
                (r["tim"][k][0] / r["tim"][k][1] / 1e3) / 1e9,
                "peak": peak, "unit": "GB/s",
                "frac": nb * ncell * (4 if args.precision == "fp32" else 8) /
                (r["tim"][k][0] / r["tim"][k][1] / 1e3) / 1e9 / peak,
                "bytes_per_launch": nb * ncell * (4 if args.precision == "fp32" else 8),
                "ms_per_launch": r["tim"][k][0] / r["tim"][k][1]}
            for k, nb in (("yee_b", 9), ("yee_e", 12)) if r["tim"].get(k, (0, 0))[1]},
        "gpu_launches": int(r["launches"]),
        "clocks": r["clocks"],
        "diag_after": {k: r["diag"][k] for k in ("energy_field", "energy_kinetic", "n_alive", "n_escaped",
                                                   "gauss_max")},
        "diag_ms": r["diag_ms"],
        "setup_s": {"generate": t_gen, "load": t_load,
                    "note": "load = generate + copy piece by piece" if streamed else "load = device copy"},
    }
    if fp64 is not None:
        line["fp64"] = fp64
    if e2e is not None:
        line["e2e"] = e2e
    if adjoint is not None:
        line["adjoint"] = adjoint
    if history is not None:
        line["history"] = history
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--cpu-steps", type=int, default=4)
    ap.add_argument("--nproc", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--history", type=int, default=0,
                    help="after the timed runs, run this many steps with the FP64 diagnostics every --history-every")
    ap.add_argument("--history-every", type=int, default=50)
    args = ap.parse_args()
    world, rank, local = _dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_gpu(args, rank, world, local)


if __name__ == "__main__":
    main()
