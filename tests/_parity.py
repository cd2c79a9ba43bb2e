"""Helpers shared by the parity tests: run the oracle and the CUDA path on the
same seeded inputs and compare them."""
import numpy as np

import oracle
from oracle import OracleSim

FIELDS = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Jx", "Jy", "Jz"]


def rel_inf(a, b):
    """||a - b||_inf / ||b||_inf (absolute when b is zero)."""
    nb = np.abs(b).max()
    d = np.abs(a - b).max()
    return d / nb if nb > 0 else d


def build_oracle(wl, parts_list, neutralize=True):
    o = OracleSim(wl.dims, wl.n, wl.d, wl.dt, wl.order)
    for sp, p in zip(wl.species, parts_list):
        o.add_particles(p, sp.q, sp.m)
    if neutralize:
        o.neutralize()
    return o


def build_gpu(wl, parts_list, precision, neutralize=True, **kw):
    from paper_1503_02464_gb300.sim import Simulation
    s = Simulation.from_workload(wl, precision=precision, **kw)
    for sp, p in zip(wl.species, parts_list):
        isp = s.add_species(sp.q, sp.m, max(len(p["x"]), 1))
        s.load(isp, p)
    if neutralize:
        s.neutralize()
    return s


def compare_fields(o, s, names=FIELDS):
    out = {}
    for i, name in enumerate(FIELDS):
        if name not in names:
            continue
        out[name] = rel_inf(s.field(i), o.get_field(i))
    return out


def compare_particles(o, s, wl, species=0):
    """Match by id; return (max |du| / max|u|, max position error in cells)."""
    po = o.particles(species)
    pg = s.particles(species)
    assert len(po["id"]) == len(pg["id"]), (len(po["id"]), len(pg["id"]))
    io = np.argsort(po["id"])
    ig = np.argsort(pg["id"])
    assert np.array_equal(po["id"][io], pg["id"][ig])
    uo = np.stack([po[k][io] for k in ("ux", "uy", "uz")])
    ug = np.stack([pg[k][ig] for k in ("ux", "uy", "uz")])
    umax = max(np.abs(uo).max(), 1e-300)
    du = np.abs(ug - uo).max() / umax
    dx = 0.0
    for a, k in enumerate(("x", "y", "z")[:wl.dims]):
        L = wl.n[a] * wl.d[a]
        diff = pg[k][ig] - po[k][io]
        diff = (diff + 0.5 * L) % L - 0.5 * L
        dx = max(dx, np.abs(diff).max() / wl.d[a])
    return du, dx
