"""Adjoint (reverse-mode) gradients of the differentiable laser-slab run
against central finite differences (needs a GB300).

Objective F = FP64 kinetic energy of the electrons in a band of columns at
the final step; parameters: laser amplitude a0 and the column density
profile (through the initial weights).  Checks:
  * FP64 adjoint vs FP64 central differences of the GPU forward, h = 1e-6;
  * FP64 adjoint vs central differences of the FP64 CPU oracle;
  * FP32 adjoint (FP64 accumulation) vs FP64 central differences, 1e-4;
  * the torch.autograd.Function wrapper returns the same gradients.
"""
import math

import numpy as np
import pytest

from paper_1503_02464_gb300 import diff

pytestmark = pytest.mark.gpu

TAU = 2 * math.pi


def _tiny(precision="fp64"):
    run = diff.SlabRun(nx=40, ny=8, ppc=2, steps=30, segment=10, slab=(8, 30), density=1.0, obj=(12, 20),
                       waist=1.5, duration=TAU, seed=7, precision=precision)
    prof = run.default_profile()
    prof[8:30] = 1.0 + 0.3 * np.sin(np.arange(22) * 0.7)
    return run, prof


def _fd(run, a0, prof, h, da=0.0, dv=None):
    """Central difference of F along (da, dv)."""
    dv = np.zeros_like(prof) if dv is None else dv
    Fp, _ = diff.forward_objective(run, a0 + h * da, prof + h * dv)
    Fm, _ = diff.forward_objective(run, a0 - h * da, prof - h * dv)
    return (Fp - Fm) / (2 * h)


def _dir_scale(fd_v, dprof, v):
    """Scale of a directional-derivative error: |fd_v| itself, floored at
    1e-3 of the sum of the terms' magnitudes (a direction along which the
    terms happen to cancel must not make the bound meaningless)."""
    return max(abs(fd_v), 1e-3 * float(np.abs(dprof * v).sum()))


def _adjoint(run, a0, prof):
    F, sim = diff.forward_objective(run, a0, prof, keep=True)
    da0, dprof = diff.backward_gradients(run, sim)
    sim.close()
    return F, da0, dprof


def test_adjoint_fp64_matches_central_differences():
    run, prof = _tiny("fp64")
    a0 = 0.8
    F, da0, dprof = _adjoint(run, a0, prof)
    assert F > 0 and np.abs(dprof).max() > 0
    fd_a0 = _fd(run, a0, prof, 1e-6, da=1.0)
    print("F", F, "dF/da0", da0, fd_a0)
    assert abs(fd_a0) > 1e-3 * F / a0  # the laser reaches the objective band
    assert abs(da0 - fd_a0) <= 1e-6 * abs(fd_a0), (da0, fd_a0)
    v = np.random.default_rng(1).normal(size=prof.size)
    fd_v = _fd(run, a0, prof, 1e-6, dv=v)
    print("dF/dprof . v", dprof @ v, fd_v)
    assert abs(fd_v) > 1e-3 * F / np.abs(prof).max()
    assert abs(dprof @ v - fd_v) <= 1e-6 * _dir_scale(fd_v, dprof, v), (dprof @ v, fd_v)


def test_binned_gradient_matches_per_id_sums():
    """pic_grad_binned (the profile gradient's column sums, on the device)
    against a bincount of the per-id weight gradient of pic_grad, with the
    bin map in host and in device memory; ids with a bin outside [0, nbins)
    are left out."""
    import torch
    run, prof = _tiny("fp64")
    F, sim = diff.forward_objective(run, 0.8, prof, keep=True)
    diff.backward_gradients(run, sim)
    _, dw = sim.grad(0, run.id_capacity)
    ids = np.arange(run.id_capacity)
    bins = run.column_of_id(ids).astype(np.int32)
    ref = np.bincount(bins, weights=dw, minlength=run.nx)
    scale = np.abs(dw).sum()
    assert scale > 0
    host = sim.grad_binned(0, bins, run.nx)
    dev = sim.grad_binned(0, torch.from_numpy(bins).cuda(), run.nx)
    for got in (host, dev):
        assert np.abs(got - ref).max() <= 1e-13 * scale, np.abs(got - ref).max() / scale
    # bins past the end (and negative ones) drop out
    odd = bins.copy()
    odd[::3] = -1
    odd[1::3] += run.nx
    keep = np.bincount(bins[2::3], weights=dw[2::3], minlength=run.nx)
    got = sim.grad_binned(0, odd, run.nx)
    assert np.abs(got - keep).max() <= 1e-13 * scale
    sim.close()


def test_adjoint_fp64_matches_oracle_gradient():
    """Central differences of the CPU oracle's objective on the same run."""
    import oracle
    run, prof = _tiny("fp64")
    a0 = 0.8

    def oracle_F(a, p):
        wl = run.workload(a)
        o = oracle.OracleSim(2, wl.n, wl.d, wl.dt, 2)
        o.set_absorbing_x(True)
        L = wl.laser
        o.set_laser(L["a0"], L["waist"], L["duration"], pol=L["pol"])
        o.add_particles(run.particles(p), -1.0, 1.0)
        o.step(run.steps)
        q = o.particles(0)
        col = np.floor(q["x"] / wl.d[0]).astype(int)
        m = (col >= run.obj[0]) & (col < run.obj[1])
        g = np.sqrt(1 + q["ux"] ** 2 + q["uy"] ** 2 + q["uz"] ** 2)
        return float((q["w"][m] * wl.d[0] * wl.d[1] * (g[m] - 1)).sum())

    F, da0, dprof = _adjoint(run, a0, prof)
    assert abs(F - oracle_F(a0, prof)) <= 1e-10 * F
    h = 1e-5
    fd_a0 = (oracle_F(a0 + h, prof) - oracle_F(a0 - h, prof)) / (2 * h)
    assert abs(da0 - fd_a0) <= 1e-5 * abs(fd_a0), (da0, fd_a0)
    v = np.random.default_rng(2).normal(size=prof.size)
    fd_v = (oracle_F(a0, prof + h * v) - oracle_F(a0, prof - h * v)) / (2 * h)
    assert abs(dprof @ v - fd_v) <= 1e-5 * _dir_scale(fd_v, dprof, v), (dprof @ v, fd_v)


def test_adjoint_fp32_matches_fp64_differences():
    run64, prof = _tiny("fp64")
    run32, _ = _tiny("fp32")
    a0 = 0.8
    _, da0, dprof = _adjoint(run32, a0, prof)
    fd_a0 = _fd(run64, a0, prof, 1e-6, da=1.0)
    assert abs(da0 - fd_a0) <= 1e-4 * abs(fd_a0), (da0, fd_a0)
    v = np.random.default_rng(3).normal(size=prof.size)
    fd_v = _fd(run64, a0, prof, 1e-6, dv=v)
    assert abs(dprof @ v - fd_v) <= 1e-4 * _dir_scale(fd_v, dprof, v), (dprof @ v, fd_v)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_store_all_matches_checkpoints(precision):
    """Recording every forward step (no recomputation in the reverse sweep)
    gives the gradients of the checkpointed sweep: to round-off in FP64; in
    FP32 to the level at which a recomputed segment differs from the first
    run (float atomics in the shared windows change the order of additions)."""
    import dataclasses
    run, prof = _tiny(precision)
    F1, da1, dp1 = _adjoint(run, 0.8, prof)
    F2, da2, dp2 = _adjoint(dataclasses.replace(run, store_all=True), 0.8, prof)
    tol = 1e-11 if precision == "fp64" else 1e-4
    assert abs(F2 - F1) <= 1e-12 * abs(F1)
    assert abs(da2 - da1) <= tol * abs(da1), (da1, da2)
    assert np.abs(dp2 - dp1).max() <= tol * np.abs(dp1).max(), np.abs(dp2 - dp1).max() / np.abs(dp1).max()


def test_autograd_function():
    import torch
    run, prof = _tiny("fp64")
    PicRun = diff.make_function()
    a0 = torch.tensor(0.8, dtype=torch.float64, requires_grad=True)
    p = torch.tensor(prof, dtype=torch.float64, requires_grad=True)
    F = PicRun.apply(a0, p, run)
    F.backward()
    _, da0, dprof = _adjoint(run, 0.8, prof)
    assert abs(a0.grad.item() - da0) <= 1e-12 * abs(da0)
    np.testing.assert_allclose(p.grad.numpy(), dprof, rtol=1e-10, atol=1e-14 * np.abs(dprof).max())


def test_full_size_fp32_adjoint_vs_fp64_differences():
    """The 256x256 laser-slab run (1.02M electrons, 200 steps, checkpoints
    every 20): FP32 adjoint gradients (laser amplitude, and the density
    profile along a random direction) against FP64 central differences."""
    run32 = diff.SlabRun(precision="fp32")
    run64 = diff.SlabRun(precision="fp64")
    prof = run32.default_profile()
    a0 = 2.0
    _, da0, dprof = _adjoint(run32, a0, prof)
    fd_a0 = _fd(run64, a0, prof, 1e-6, da=1.0)
    print("full size dF/da0", da0, fd_a0)
    assert abs(da0 - fd_a0) <= 1e-4 * abs(fd_a0), (da0, fd_a0)
    # the 256-value density profile, along a random direction
    v = np.random.default_rng(4).normal(size=prof.size)
    fd_v = _fd(run64, a0, prof, 1e-6, dv=v)
    print("full size dF/dprof . v", dprof @ v, fd_v)
    assert abs(fd_v) > 0
    assert abs(dprof @ v - fd_v) <= 1e-4 * _dir_scale(fd_v, dprof, v), (dprof @ v, fd_v)
