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


def _species0_arrays(blob, ncell, dims, rsize):
    """Byte offsets of the cell array and the first offset array of the only
    species in a state blob: the particle storage is the blob's tail, one
    allocation of 256-byte aligned arrays (cell, offsets, u, w, id), and the
    header stores the species' slot count right after the cell count."""
    head = blob[:1024].tobytes()
    at = head.find(np.int64(ncell).tobytes())
    assert at > 0
    slots = int(np.frombuffer(head[at + 8:at + 16], dtype=np.int64)[0])
    a256 = lambda b: (b + 255) // 256 * 256  # noqa: E731
    pb = a256(slots * 4) + (dims + 4) * a256(slots * rsize) + a256(slots * 4)
    cell0 = len(blob) - pb
    return cell0, cell0 + a256(slots * 4)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_state_rejects_invalid_particles(precision):
    """A blob whose particle storage holds a cell outside the grid or a
    non-finite offset is refused (PIC_EINVAL) before it replaces anything:
    the simulation keeps its own state and steps on."""
    wl = synth.small(2, (32, 32), 2, 2, 0.1, 3)
    a = _make(wl, precision)
    a.load(0, wl.particles(0))
    a.step(2)
    blob = a.state()
    rsize = 4 if precision == "fp32" else 8
    cell0, off0 = _species0_arrays(blob, 32 * 32, 2, rsize)
    cells = np.frombuffer(blob[cell0:cell0 + 4 * 64].tobytes(), dtype=np.int32)
    live = int(np.nonzero(cells >= 0)[0][0])

    b = _make(wl, precision)
    pb = wl.particles(0)
    pb["ux"] = pb["ux"] * 0.5
    b.load(0, pb)
    b.step(1)
    before = b.diag()
    for corrupt in ("cell", "offset"):
        bad = blob.copy()
        if corrupt == "cell":
            bad[cell0 + 4 * live:cell0 + 4 * live + 4] = np.frombuffer(np.int32(32 * 32 + 5).tobytes(), np.uint8)
        else:
            nan = np.float32(np.nan) if rsize == 4 else np.float64(np.nan)
            bad[off0 + rsize * live:off0 + rsize * (live + 1)] = np.frombuffer(nan.tobytes(), np.uint8)
        with pytest.raises(capi.PicError) as ei:
            b.load_state(bad)
        assert ei.value.code == capi.PIC_EINVAL
        assert "invalid particle" in str(ei.value)
        after = b.diag()
        assert after["step"] == before["step"] and after["n_alive"] == before["n_alive"]
        # FP64 sums taken with atomics: equal to round-off
        assert abs(after["energy_kinetic"] - before["energy_kinetic"]) <= 1e-13 * before["energy_kinetic"]
        assert abs(after["energy_field"] - before["energy_field"]) <= 1e-13 * before["energy_field"]
    b.step(1)
    b.load_state(blob)  # the intact blob still loads
    assert b.diag()["step"] == 2
