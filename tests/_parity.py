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


def j_floor(wl, parts_list):
    """Absolute error floor of the oracle's current density.

    The oracle keeps global positions, so each shape difference S(X1) - S(X0)
    carries an absolute rounding error up to about 2 ulp(X) (X in cells, up to
    n); a contribution to J is q w (dx/dt) times that, and a node sums at most
    ppc * 4^dims of them.  Relative comparisons of J are meaningless below
    this floor (cold plasmas barely moving)."""
    qw = max((abs(sp.q) * np.abs(p["w"]).max() for sp, p in zip(wl.species, parts_list) if len(p["w"])),
             default=0.0)
    ppc = max((sp.ppc for sp in wl.species), default=1)
    n = max(wl.n[:wl.dims])
    return 4.0 * qw * max(wl.d[:wl.dims]) / wl.dt * 2 * np.spacing(float(n)) * ppc * 4 ** wl.dims


def j_floor_fp32(wl, parts_list):
    """Absolute floor of the FP32 path's current density against an exact
    trajectory.

    The FP32 path stores each in-cell offset in FP32, so every stored
    position is rounded by up to half an ulp of the offset, 2^-25 cells, and
    the discrete continuity equation ties the current to the stored
    displacement: a contribution q w (dx/dt) (a running sum of S1 - S0, at
    most the displacement in cells) times a bracket of at most 1 moves by up
    to q w (dx/dt) 2^-25 against the current of the unrounded move.  A node
    sums at most ppc * (order + 2)^dims such contributions.  For particles
    that barely move (a cold target that a pulse has just reached) this
    rounding, not the arithmetic, separates the FP32 current from the
    oracle's; the arithmetic itself is checked on the stored moves
    (test_fp32_deposit_of_stored_moves)."""
    qw = max((abs(sp.q) * np.abs(p["w"]).max() for sp, p in zip(wl.species, parts_list) if len(p["w"])),
             default=0.0)
    ppc = max((sp.ppc for sp in wl.species), default=1)
    return qw * max(wl.d[:wl.dims]) / wl.dt * 2.0 ** -25 * ppc * (wl.order + 2) ** wl.dims


def compare_fields(o, s, names=FIELDS, j_abs=0.0, joint_eb=False):
    """Error of each component relative to the max norm of its vector field
    (max over Ex, Ey, Ez for E; likewise B and J), so that a component that
    is zero up to round-off in some geometry is judged against the field it
    belongs to.  With joint_eb, E and B share one norm, max(|E|, |B|) (same
    units for c = 1): for electrostatic problems, where B is round-off.  For
    J the difference is first reduced by the absolute floor j_abs (see
    j_floor)."""
    got = {name: s.field(i) for i, name in enumerate(FIELDS)}
    ref = {name: o.get_field(i) for i, name in enumerate(FIELDS)}
    out = {}
    for name in FIELDS:
        if name not in names:
            continue
        heads = ("E", "B") if joint_eb and name[0] in "EB" else (name[0],)
        group = [g + c for g in heads for c in "xyz"]
        norm = max(np.abs(ref[g]).max() for g in group)
        d = np.abs(got[name] - ref[name]).max()
        if name.startswith("J"):
            d = max(d - j_abs, 0.0)
        out[name] = d / norm if norm > 0 else d
    return out


def compare_particles(o, s, wl, species=0, u_scale=0.0):
    """Match by id; return (max |du| / max(max|u|, u_scale), max position
    error in cells).  u_scale lets a test normalise by the momentum the
    fields can impart when the particles themselves barely move."""
    po = o.particles(species)
    pg = s.particles(species)
    assert len(po["id"]) == len(pg["id"]), (len(po["id"]), len(pg["id"]))
    io = np.argsort(po["id"])
    ig = np.argsort(pg["id"])
    assert np.array_equal(po["id"][io], pg["id"][ig])
    uo = np.stack([po[k][io] for k in ("ux", "uy", "uz")])
    ug = np.stack([pg[k][ig] for k in ("ux", "uy", "uz")])
    umax = max(np.abs(uo).max(), u_scale, 1e-300)
    du = np.abs(ug - uo).max() / umax
    dx = 0.0
    for a, k in enumerate(("x", "y", "z")[:wl.dims]):
        L = wl.n[a] * wl.d[a]
        diff = pg[k][ig] - po[k][io]
        diff = (diff + 0.5 * L) % L - 0.5 * L
        dx = max(dx, np.abs(diff).max() / wl.d[a])
    return du, dx
