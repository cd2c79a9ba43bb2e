"""The counting sort of the particle slots (needs a GB300).

Particles loaded in a shuffled order are sorted by pic_neutralize (the
first sort of a species).  Checked against what the sort must produce,
independently of the push:
  * a permutation: every id once, and each particle's stored state (FP32
    offsets, momenta, weight) bit-identical before and after;
  * slot order by (tile, cell within the tile) over the live slots, the
    order within one cell being free;
  * dead slots only as the padding at the end of a tile's run (runs padded
    to a multiple of 4 slots).
Then a step moves the particles and the cadence sort (sort_every = 1)
restores the order.
"""
import numpy as np
import pytest

from paper_1503_02464_gb300 import synth
from paper_1503_02464_gb300.sim import Simulation

pytestmark = pytest.mark.gpu

PAD = 4  # slots of a tile's run are padded to a multiple of this


def _keys(p, wl, tile):
    """(tile, cell within the tile) of each particle, from its position.  The
    FP32 path stores a cell and an offset in [0, 1 - 2^-24]; the small nudge
    keeps floor() on the right cell for an offset of exactly 0."""
    dims = wl.dims
    tile = tuple(tile) + (1,) * (3 - len(tile))
    c = [np.floor(p[k] / wl.d[a] + 1e-9).astype(np.int64) for a, k in enumerate("xyz"[:dims])]
    for a in range(dims):
        c[a] %= wl.n[a]
    while len(c) < 3:
        c.append(np.zeros_like(c[0]))
    t = [c[a] // tile[a] for a in range(3)]
    nt = [-(-wl.n[a] // tile[a]) for a in range(3)]
    tid = t[0] + nt[0] * (t[1] + nt[1] * t[2])
    local = (c[0] - t[0] * tile[0]) + tile[0] * ((c[1] - t[1] * tile[1]) + tile[1] * (c[2] - t[2] * tile[2]))
    return tid, tid * (tile[0] * tile[1] * tile[2]) + local


def _check_sorted(s, wl, tile, before):
    raw = s.particles(0, alive_only=False)
    alive = raw["alive"] == 1
    live = {k: v[alive] for k, v in raw.items()}
    tid, key = _keys(live, wl, tile)
    assert np.all(np.diff(key) >= 0), "live slots not in (tile, cell) order"
    # each tile's run (live slots and the padding after them) starts at a
    # multiple of PAD and holds fewer than PAD dead slots
    idx = np.nonzero(alive)[0]
    starts = np.r_[0, np.nonzero(np.diff(tid))[0] + 1]
    for a, b in zip(starts, np.r_[starts[1:], len(idx)]):
        first, last = idx[a], idx[b - 1]
        assert first % PAD == 0, first
        assert np.all(alive[first:last + 1]), "a dead slot inside a tile's run"
        nxt = idx[b] if b < len(idx) else len(alive)
        assert nxt - (last + 1) < PAD, (last, nxt)
    # a permutation, every particle's state unchanged bit for bit
    assert np.array_equal(np.sort(live["id"]), np.sort(before["id"]))
    order_a = np.argsort(live["id"])
    order_b = np.argsort(before["id"])
    for k in ("x", "y", "z", "ux", "uy", "uz", "w"):
        assert np.array_equal(live[k][order_a], before[k][order_b]), k


@pytest.mark.parametrize("dims,n,tile", [
    (3, (24, 16, 12), (8, 8, 4)),
    (3, (20, 12, 10), (8, 8, 4)),   # ragged tiles
    (2, (40, 24), (16, 16)),        # ragged tiles
])
def test_sort_order_and_permutation(dims, n, tile):
    wl = synth.small(dims, n, 2, 5, 0.3, 17 + dims)
    p = wl.particles(0)
    perm = np.random.default_rng(3).permutation(len(p["x"]))
    shuffled = {k: np.ascontiguousarray(v[perm]) for k, v in p.items()}
    s = Simulation.from_workload(wl, precision="fp32", sort_every=1)
    k = s.add_species(-1.0, 1.0, len(p["x"]))
    s.load(k, shuffled)
    before = s.particles(0)          # load order, stored FP32 state
    s.neutralize()                    # sorts the freshly loaded species
    _check_sorted(s, wl, tile, before)
    # a step moves particles across cells and tiles; the cadence sort of the
    # next step (sort_every = 1) puts them back in order
    s.step(1)
    moved = s.particles(0)
    s.step(1)
    _check_sorted_after_step(s, wl, tile, moved)
    s.close()


def _check_sorted_after_step(s, wl, tile, moved):
    """After the second step the slots are sorted by the positions the first
    step produced (the sort runs before the step's push), so the order is
    checked against those positions, matched by id."""
    raw = s.particles(0, alive_only=False)
    alive = raw["alive"] == 1
    ids = raw["id"][alive]
    pos = {int(i): j for j, i in enumerate(moved["id"])}
    sel = np.array([pos[int(i)] for i in ids])
    prev = {k: v[sel] for k, v in moved.items()}
    _, key = _keys(prev, wl, tile)
    assert np.all(np.diff(key) >= 0), "slots not in the order of the positions they were sorted by"
    assert len(ids) == len(moved["id"])
