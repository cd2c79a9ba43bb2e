"""Structured targets of the synthetic inputs (CPU): the grating's front
surface and the foam's random fill follow their definitions, are the same
for any subset of cells, and electrons and ions of a preset fill the same
cells (a neutral target)."""
import math

import numpy as np

from paper_1503_02464_gb300 import synth


def test_grating_front_surface():
    n = (64, 40, 1)
    period, depth, x0, x1 = 10.0, 6.0, 20, 40
    sp = synth.Species("e", -1.0, 1.0, 2, 0.0, 1.0, (x0, x1), 0, structure=("grating", period, depth))
    wl = synth.Workload("g", 2, n, (0.1, 0.1, 1.0), 0.05, 2, 1, 1, [sp])
    cells = wl.species_cells(sp)
    i, j = cells % n[0], cells // n[0]
    for row in range(n[1]):
        cols = np.sort(i[j == row])
        front = x0 + math.floor(depth * (1 + math.sin(2 * math.pi * (row + 0.5) / period)) / 2)
        assert cols[0] == front, (row, cols[0], front)
        assert np.array_equal(cols, np.arange(front, x1))
    # the particles sit inside the kept cells
    p = wl.particles(0)
    ci = np.floor(p["x"] / 0.1).astype(int)
    assert ci.min() >= x0 and ci.max() < x1
    assert len(p["x"]) == cells.size * 2


def test_foam_fill_is_per_cell_and_seeded():
    n = (128, 64, 1)
    fill = 0.3
    cells = np.arange(10, 110)[None, :] + n[0] * np.arange(n[1])[:, None]
    cells = cells.reshape(-1)
    m = synth.structure_mask(("foam", fill, 7), cells, n, (10, 110))
    k = m.sum()
    sigma = math.sqrt(cells.size * fill * (1 - fill))
    assert abs(k - fill * cells.size) < 5 * sigma
    # the same mask for any subset of the cells, in any grouping
    sub = cells[::3]
    assert np.array_equal(synth.structure_mask(("foam", fill, 7), sub, n, (10, 110)), m[::3])
    # another seed gives another mask
    assert not np.array_equal(synth.structure_mask(("foam", fill, 8), cells, n, (10, 110)), m)
    # no spatial correlation to speak of between neighbouring cells
    mm = m.reshape(n[1], -1).astype(float)
    c = np.corrcoef(mm[:, :-1].ravel(), mm[:, 1:].ravel())[0, 1]
    assert abs(c) < 0.05, c


def test_structured_presets_are_neutral():
    for name in ("grating_foil2d", "foam_foil2d"):
        wl = synth.preset(name)
        for a in range(0, len(wl.species), 2):
            e, p = wl.species[a], wl.species[a + 1]
            assert e.q == -p.q and e.density == p.density
            assert np.array_equal(wl.species_cells(e), wl.species_cells(p))
            pe, pp = wl.particles(a, wl.species_cells(e)[:50]), wl.particles(a + 1, wl.species_cells(p)[:50])
            assert np.array_equal(pe["x"], pp["x"]) and np.array_equal(pe["y"], pp["y"])
