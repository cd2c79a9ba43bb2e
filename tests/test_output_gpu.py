"""Output manager (§3.1 of the paper: reduced-dimension and sub-domain
outputs in a time window with a frequency), captured on the device inside
pic_step, against the FP64 oracle's state at the same steps (needs a GB300).

The oracle side is the definition: slices of its full field arrays, and its
particles whose cell floor(x / dx) lies in the box."""
import numpy as np
import pytest

import oracle
from oracle import OracleSim
from paper_1503_02464_gb300 import capi, synth
from paper_1503_02464_gb300.sim import Simulation

pytestmark = pytest.mark.gpu


def _pair(precision, n=(16, 16, 8), order=2, ppc=4, seed=17):
    wl = synth.small(len(n), n, order, ppc, 0.05, seed)
    p = wl.particles(0)
    o = OracleSim(wl.dims, wl.n, wl.d, wl.dt, wl.order)
    o.add_particles(p, -1.0, 1.0)
    o.neutralize()
    s = Simulation.from_workload(wl, precision=precision)
    k = s.add_species(-1.0, 1.0, len(p["x"]))
    s.load(k, p)
    s.neutralize()
    return wl, o, s


def _box(a, lo, hi):
    return a[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]]


def _in_box(parts, wl, lo, hi, margin=1e-9):
    """Ids inside the box, and ids within `margin` cells of one of its faces
    (where rounding may place a particle on either side)."""
    X = [parts[c] / wl.d[a] for a, c in enumerate("xyz")]
    inside = np.ones(len(X[0]), bool)
    edge = np.zeros(len(X[0]), bool)
    for a in range(3):
        if a >= wl.dims:
            continue
        inside &= (np.floor(X[a]) >= lo[a]) & (np.floor(X[a]) < hi[a])
        for f in (lo[a], hi[a]):
            edge |= np.abs(X[a] - f) < margin
    return set(parts["id"][inside & ~edge].tolist()), set(parts["id"][edge].tolist())


def test_field_frames_match_oracle_fp64():
    wl, o, s = _pair("fp64")
    plane = s.output_add("field", oracle.EY, (0, 0, 3), (16, 16, 4), first=2, last=10, every=4, max_frames=3)
    line = s.output_add("field", oracle.BZ, (0, 5, 2), (16, 6, 3), first=1, last=3, every=1, max_frames=3)
    rho = s.output_add("field", oracle.RHO, (2, 3, 1), (10, 9, 5), first=5, last=5, every=1, max_frames=1)
    jbox = s.output_add("field", oracle.JX, (4, 0, 0), (12, 16, 8), first=4, last=4, every=1, max_frames=1)
    ref = {}
    for step in range(1, 11):
        o.step(1)
        ref[step] = {w: o.get_field(w) for w in (oracle.EY, oracle.BZ, oracle.JX)}
        if step == 5:
            ref[step][oracle.RHO] = o.rho()
    s.step(10)
    assert s.output_count(plane) == (3, 0)
    for f, step in enumerate((2, 6, 10)):
        got, st = s.output_read(plane, f)
        assert st == step
        full = ref[step][oracle.EY]
        assert np.abs(got - _box(full, (0, 0, 3), (16, 16, 4))).max() <= 1e-12 * step * np.abs(full).max()
    for f, step in enumerate((1, 2, 3)):
        got, st = s.output_read(line, f)
        full = ref[step][oracle.BZ]
        assert st == step and got.shape == (1, 1, 16)
        assert np.abs(got - _box(full, (0, 5, 2), (16, 6, 3))).max() <= 1e-12 * step * max(np.abs(full).max(), 1e-30)
    got, st = s.output_read(rho, 0)
    assert st == 5 and got.shape == (4, 6, 8)
    assert np.abs(got - _box(ref[5][oracle.RHO], (2, 3, 1), (10, 9, 5))).max() <= 1e-12
    got, st = s.output_read(jbox, 0)
    full = ref[4][oracle.JX]
    assert np.abs(got - _box(full, (4, 0, 0), (12, 16, 8))).max() <= 1e-10 * np.abs(full).max()


def test_field_frames_equal_full_readout_fp32():
    """A frame is a copy: bit-identical to the same box of pic_fields."""
    wl, o, s = _pair("fp32")
    oid = s.output_add("field", oracle.EX, (3, 2, 1), (11, 13, 6), first=3, last=3, max_frames=2)
    s.output_capture(oid)  # the initial state, outside the schedule
    s.step(3)
    assert s.output_count(oid) == (2, 0)
    f0, st0 = s.output_read(oid, 1)
    assert st0 == 3
    assert np.array_equal(f0, _box(s.field(oracle.EX), (3, 2, 1), (11, 13, 6)))
    init, st = s.output_read(oid, 0)
    assert st == 0 and np.abs(init).max() == 0.0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_particle_frames_match_oracle(precision):
    wl, o, s = _pair(precision)
    lo, hi = (4, 4, 2), (12, 10, 6)
    oid = s.output_add("particles", 0, lo, hi, first=3, last=7, every=4, max_frames=2, max_particles=20000)
    refs = {}
    for step in range(1, 8):
        o.step(1)
        if step in (3, 7):
            refs[step] = o.particles(0)
    s.step(7)
    tol = 1e-12 if precision == "fp64" else 1e-5
    for f, step in enumerate((3, 7)):
        got, st = s.output_read(oid, f)
        assert st == step
        ref = refs[step]
        inside, edge = _in_box(ref, wl, lo, hi)
        ids = set(got["id"].tolist())
        assert len(ids) == len(got["id"])               # no record twice
        assert inside <= ids and ids <= inside | edge   # the same particles
        order = np.argsort(ref["id"])
        sel = np.searchsorted(ref["id"], got["id"], sorter=order)
        ri = order[sel]
        for key in ("x", "y", "z"):
            assert np.abs(got[key] - ref[key][ri]).max() <= tol * max(wl.n) * max(wl.d)
        umax = max(np.abs(ref[k]).max() for k in ("ux", "uy", "uz"))
        for key in ("ux", "uy", "uz"):
            assert np.abs(got[key] - ref[key][ri]).max() <= tol * step * umax
        assert np.array_equal(got["w"], ref["w"][ri]) or precision == "fp32"


def test_particle_frame_overflow_and_dropped_frames():
    wl, o, s = _pair("fp64")
    lo, hi = (0, 0, 0), (16, 16, 8)
    oid = s.output_add("particles", 0, lo, hi, first=1, last=5, every=1, max_frames=2, max_particles=100)
    s.step(5)
    assert s.output_count(oid) == (2, 3)
    n_all = wl.n_particles()
    with pytest.raises(capi.PicError) as ei:
        s.output_read(oid, 0)
    assert ei.value.code == capi.PIC_EOVERFLOW
    buf = np.empty((100, 8))
    try:
        capi.pic_output_read(s.h, oid, 0, buf.ctypes.data, capi.PIC_MEM_HOST)
    except capi.PicError:
        pass
    ids = buf[:, 7].astype(np.int64)
    assert len(set(ids.tolist())) == 100 and ids.min() >= 0 and ids.max() < n_all
    s.output_remove(oid)
    with pytest.raises(capi.PicError):
        s.output_count(oid)


@pytest.mark.parametrize("kw", [
    dict(kind="field", which=10, lo=(0, 0, 0), hi=(1, 1, 1), first=1, last=1),
    dict(kind="field", which=0, lo=(0, 0, 0), hi=(17, 1, 1), first=1, last=1),
    dict(kind="field", which=0, lo=(3, 0, 0), hi=(3, 1, 1), first=1, last=1),
    dict(kind="field", which=0, lo=(0, 0, 0), hi=(1, 1, 1), first=5, last=4),
    dict(kind="field", which=0, lo=(0, 0, 0), hi=(1, 1, 1), first=1, last=4, every=0),
    dict(kind="particles", which=3, lo=(0, 0, 0), hi=(1, 1, 1), first=1, last=1),
])
def test_output_add_validates(kw):
    wl, o, s = _pair("fp32")
    with pytest.raises(capi.PicError) as ei:
        s.output_add(**kw)
    assert ei.value.code == capi.PIC_EINVAL
