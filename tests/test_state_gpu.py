"""State save / resume (needs a GB300): a run saved after a few steps and
resumed in a fresh simulation continues as the uninterrupted run does.

Two identical runs agree only to round-off: each tile adds its current
window to the global J with atomics, and neighbouring windows overlap, so
the order of those additions varies.  The resumed run therefore matches to
round-off: 1e-5 of each field's vector norm in FP32 (the 10-step FP32
tolerance), 1e-13 in FP64.  Particles leave exactly the same count and
ids."""
import numpy as np
import pytest

from paper_1503_02464_gb300 import capi, synth
from paper_1503_02464_gb300.sim import Simulation

from _parity import FIELDS

pytestmark = pytest.mark.gpu


def _make(wl, precision, **kw):
    s = Simulation.from_workload(wl, precision=precision, **kw)
    for sp in wl.species:
        s.add_species(sp.q, sp.m, wl.n_particles())
    return s


def _snapshot(s, nsp):
    f = {name: s.field(i) for i, name in enumerate(FIELDS)}
    parts = []
    for k in range(nsp):
        p = s.particles(k)
        o = np.argsort(p["id"])
        parts.append({key: v[o] for key, v in p.items()})
    return f, parts


def _cases():
    thermal = synth.small(3, (16, 16, 8), 2, 2, 0.1, 21)
    thermal.sort_every = 2
    d = 0.1
    slab = synth.Workload("slab", 2, (64, 32, 1), (d, d, 1.0), 0.9 * synth.courant_limit((d, d), 2), 2, 10, 9,
                          [synth.Species("electron", -1.0, 1.0, 4, 0.0, 4.0, (20, 28), 0),
                           synth.Species("proton", 1.0, 1836.0, 4, 0.0, 4.0, (20, 28), 1)],
                          sort_every=1, absorbing_x=True, neutralize=False,
                          laser={"a0": 2.0, "waist": 0.8, "duration": 6.0, "pol": 1})
    return [("thermal3d", thermal, {}), ("laser_slab2d_filtered", slab, {"filter_passes": 1,
                                                                          "filter_compensate": True})]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("name,wl,kw", _cases(), ids=lambda v: v if isinstance(v, str) else "")
def test_resume_continues_the_run(precision, name, wl, kw, tmp_path):
    a = _make(wl, precision, **kw)
    for k in range(len(wl.species)):
        a.load(k, wl.particles(k))
    if wl.neutralize:
        a.neutralize()
    a.step(4)
    path = str(tmp_path / "state.bin")
    a.save_state(path)
    a.step(6)
    fa, pa = _snapshot(a, len(wl.species))
    da = a.diag()

    b = _make(wl, precision, **kw)
    b.resume(path)
    b.step(6)
    fb, pb = _snapshot(b, len(wl.species))
    db = b.diag()
    tol = 1e-5 if precision == "fp32" else 1e-13
    for key in fa:
        scale = max(np.abs(fa[k]).max() for k in FIELDS if k[0] == key[0]) or 1.0
        assert np.abs(fa[key] - fb[key]).max() <= tol * scale, key
    for k in range(len(wl.species)):
        assert np.array_equal(pa[k]["id"], pb[k]["id"])
        assert np.array_equal(pa[k]["w"], pb[k]["w"])
        for key in ("x", "y", "z", "ux", "uy", "uz"):
            assert np.abs(pa[k][key] - pb[k][key]).max() <= tol * max(np.abs(pa[k][key]).max(), 1.0), (k, key)
    assert da["step"] == db["step"] == 10
    assert da["n_alive"] == db["n_alive"] and da["n_absorbed"] == db["n_absorbed"]


def test_state_rejects_a_different_configuration():
    wl = synth.small(2, (32, 32), 2, 2, 0.1, 3)
    a = _make(wl, "fp32")
    a.load(0, wl.particles(0))
    blob = a.state()
    other = synth.small(2, (32, 32), 1, 2, 0.1, 3)  # CIC instead of TSC
    b = _make(other, "fp32")
    with pytest.raises(capi.PicError) as ei:
        b.load_state(blob)
    assert ei.value.code == capi.PIC_EINVAL
    c = _make(wl, "fp64")
    with pytest.raises(capi.PicError):
        c.load_state(blob)
    with pytest.raises(capi.PicError):
        a.load_state(blob[:100])
