"""Failure paths of the C ABI, all injected from the host (needs a GB300).

No test faults, traps or hangs the GPU: bad arguments, exhausted capacity,
non-finite inputs and non-finite fields are made on the host and must come
back as status codes (with the simulation still usable afterwards)."""
import numpy as np
import pytest

from paper_1503_02464_gb300 import capi, synth
from paper_1503_02464_gb300.sim import Simulation

pytestmark = pytest.mark.gpu


def _sim(precision="fp32", absorbing=False, n=(32, 32)):
    wl = synth.small(2, n, 2, 2, 0.05, 5)
    wl.absorbing_x = absorbing
    s = Simulation.from_workload(wl, precision=precision)
    return wl, s


def _code(fn, *a, **k):
    with pytest.raises(capi.PicError) as ei:
        fn(*a, **k)
    return ei.value.code


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_capacity_exceeded(precision):
    wl, s = _sim(precision)
    p = wl.particles(0)
    k = s.add_species(-1.0, 1.0, 100)
    part = {key: v[:80] for key, v in p.items()}
    s.load(k, part)
    assert _code(s.load, k, part) == capi.PIC_ENOMEM
    assert s.num_particles(k) == 80
    s.step(2)
    assert s.diag()["n_alive"] == 80


@pytest.mark.parametrize("bad", ["x", "ux", "w"])
def test_non_finite_particles_are_rejected(bad):
    wl, s = _sim()
    p = wl.particles(0)
    n = len(p["x"])
    p[bad] = p[bad].copy()
    p[bad][[3, 17]] = [np.nan, np.inf]
    k = s.add_species(-1.0, 1.0, n)
    assert _code(s.load, k, p) == capi.PIC_EINVAL
    s.step(3)
    d = s.diag()
    assert d["n_alive"] == n - 2
    assert np.isfinite(d["energy_kinetic"]) and np.isfinite(d["energy_field"])


def test_particles_outside_absorbing_walls_are_rejected():
    wl, s = _sim(absorbing=True)
    p = wl.particles(0)
    X = p["x"] / wl.d[0]
    outside = int(((X < 3) | (X >= wl.n[0] - 4)).sum())
    assert outside > 0
    k = s.add_species(-1.0, 1.0, len(X))
    assert _code(s.load, k, p) == capi.PIC_EINVAL
    s.step(1)
    assert s.diag()["n_alive"] <= len(X) - outside


def test_non_finite_field_reported_by_diagnostics():
    wl, s = _sim()
    k = s.add_species(-1.0, 1.0, wl.n_particles())
    s.load(k, wl.particles(0))
    ex = np.zeros(s.shape3)
    ex[0, 5, 7] = np.nan
    s.set_field(0, ex)
    assert _code(s.diag) == capi.PIC_ENAN
    s.step(1)  # the NaN reaches momenta: bounded indices, no fault
    assert _code(s.energy) == capi.PIC_ENAN
    # a clean field restores a usable state for new particles
    s.set_field(0, np.zeros(s.shape3))


def test_bad_arguments():
    wl, s = _sim()
    k = s.add_species(-1.0, 1.0, 10)
    h = s.h
    lib = capi.load()
    assert lib.pic_step(h, -1) == capi.PIC_EINVAL
    assert lib.pic_num_particles(h, 7, None) == capi.PIC_EINVAL
    assert _code(s.num_particles, 5) == capi.PIC_EINVAL
    assert _code(s.field, 11) == capi.PIC_EINVAL
    assert _code(s.set_field, 9, np.zeros(s.shape3)) == capi.PIC_EINVAL   # rho is derived, not settable
    assert _code(s.restore, 3) == capi.PIC_EINVAL
    assert _code(s.adjoint_step, 1) == capi.PIC_EINVAL
    assert _code(s.set_background, np.full(s.shape3, np.nan)) == capi.PIC_EINVAL
    assert "background" in capi.load().pic_last_error(h).decode()
    bins = np.zeros(10, dtype=np.int32)
    assert _code(s.grad_binned, 0, bins, 4) == capi.PIC_EINVAL      # no pic_adjoint_begin
    s.adjoint_begin(10)
    assert _code(s.grad_binned, 3, bins, 4) == capi.PIC_EINVAL      # no such species
    assert _code(s.grad_binned, 0, bins, 0) == capi.PIC_EINVAL      # no bins
    assert _code(s.grad_binned, 0, np.zeros(11, dtype=np.int32), 4) == capi.PIC_EINVAL  # more ids than the capacity
    np.testing.assert_array_equal(s.grad_binned(0, bins, 4), np.zeros(4))  # nothing accumulated yet
    # still usable
    s.load(k, {key: v[:10] for key, v in wl.particles(0).items()})
    s.step(1)
    assert s.diag()["n_alive"] == 10
