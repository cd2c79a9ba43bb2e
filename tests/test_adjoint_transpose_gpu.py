"""The adjoint kernels are exact transposes (needs a GB300): dot-product
identities <A x, y> = <x, A^T y> in FP64 for the parts of one PIC step that
are linear in some input, and a Jacobian check where the step is not.

  * Yee + Mur walls (no particles, laser off): the field update is linear in
    (E, B); the reversed step applied to a seed y must give A^T y.
  * Esirkepov deposit, in the weights: from E = B = 0 the particles move
    ballistically whatever their weights, so the fields after the step are
    linear in w; the weight adjoint of a field seed must give the transpose.
  * Gather of E: with B = 0 the Boris step is u' = u + (q dt/m) E(x_p),
    linear in the grid E; a seed on the momenta must return G^T through the
    field adjoint.
  * Gather and rotation in B: u' is not linear in B, so the directional
    derivative of <u'(B), y> is compared with central differences (h = 1e-5).

The 2D3V TSC cycle is the one the adjoint kernels cover.  The particle
transposes run twice: with the particles in the tiles they were sorted into
(the windowed kernel, nodes in shared memory), and after twelve unsorted
steps of a hot plasma, when some have drifted beyond their tile windows and
take the global-memory kernel.
"""
import numpy as np
import pytest

from paper_1503_02464_gb300 import synth
from paper_1503_02464_gb300.sim import Simulation

pytestmark = pytest.mark.gpu

EB = range(6)  # EX .. BZ
TOL = 1e-13


def _sim(walls=False, n=(32, 24)):
    d = 0.1
    dt = 0.9 * synth.courant_limit((d, d), 2)
    return Simulation(2, (n[0], n[1], 1), (d, d, 1.0), dt, 2, "fp64", sort_every=1000, absorbing_x=walls)


def _particles(s, npart, seed, u_th=0.2, walls=False):
    rng = np.random.default_rng(seed)
    nx, ny = s.n[0], s.n[1]
    lo = 4.0 if walls else 0.0
    hi = nx - 5.0 if walls else float(nx)
    p = {"x": rng.uniform(lo, hi, npart) * s.d[0], "y": rng.uniform(0, ny, npart) * s.d[1], "z": np.zeros(npart),
         "ux": rng.normal(0, u_th, npart), "uy": rng.normal(0, u_th, npart), "uz": rng.normal(0, u_th, npart),
         "w": rng.uniform(0.5, 1.5, npart), "id": np.arange(npart, dtype=np.uint32)}
    k = s.add_species(-1.0, 1.0, npart)
    s.load(k, p)
    return p


def _drift(s, drifted):
    """Twelve steps without a sort (sort_every = 1000), so that a hot plasma
    leaves its tiles, then fields back to zero: the next step starts from
    drifted particles and no field."""
    if not drifted:
        return
    s.step(12)
    zero = np.zeros(s.shape3)
    for c in EB:
        s.set_field(c, zero)


def _check_paths(s, npart, drifted):
    n_esc = s.diag()["n_adj_escaped"]
    if drifted:
        assert 0 < n_esc < npart, n_esc
    else:
        assert n_esc == 0, n_esc


def _momenta_by_id(s, npart):
    q = s.particles(0)
    out = np.zeros((3, npart))
    for d, key in enumerate(("ux", "uy", "uz")):
        out[d, q["id"]] = q[key]
    return out


def _dot(a, b):
    return float(sum((x * y).sum() for x, y in zip(a, b)))


def _scale(a, b):
    return float(sum(np.abs(x * y).sum() for x, y in zip(a, b)))


@pytest.mark.parametrize("walls", [False, True], ids=["periodic", "mur_walls"])
def test_yee_transpose_dot_product(walls):
    s = _sim(walls)
    shape = s.shape3
    rng = np.random.default_rng(11)
    x = [rng.normal(size=shape) for _ in EB]
    y = [rng.normal(size=shape) for _ in EB]
    for c in EB:
        s.set_field(c, x[c])
    s.tape_begin(1)
    s.step(1)
    Ax = [s.field(c) for c in EB]
    s.adjoint_begin(1)
    for c in EB:
        s.adjoint_set_field(c, y[c])
    s.adjoint_step(1)
    ATy = [s.adjoint_field(c) for c in EB]
    lhs, rhs = _dot(Ax, y), _dot(x, ATy)
    scale = _scale(Ax, y) + _scale(x, ATy)
    print("yee", walls, lhs, rhs, abs(lhs - rhs) / scale)
    assert abs(lhs - rhs) <= TOL * scale, (lhs, rhs)
    s.close()


@pytest.mark.parametrize("drifted", [False, True], ids=["in_tiles", "drifted"])
def test_deposit_transpose_in_weights(drifted):
    s = _sim()
    npart = 400
    p = _particles(s, npart, 12, u_th=0.8 if drifted else 0.2)
    _drift(s, drifted)
    s.tape_begin(1)
    s.step(1)
    Lw = [s.field(c) for c in EB]
    assert max(np.abs(f).max() for f in Lw) > 0
    rng = np.random.default_rng(13)
    y = [rng.normal(size=s.shape3) for _ in EB]
    s.adjoint_begin(npart)
    for c in EB:
        s.adjoint_set_field(c, y[c])
    s.adjoint_step(1)
    _, lw = s.grad(0, npart)
    lhs, rhs = _dot(Lw, y), float((p["w"] * lw[p["id"]]).sum())
    scale = _scale(Lw, y) + float(np.abs(p["w"] * lw[p["id"]]).sum())
    print("deposit", lhs, rhs, abs(lhs - rhs) / scale)
    assert abs(lhs - rhs) <= TOL * scale, (lhs, rhs)
    _check_paths(s, npart, drifted)
    s.close()


@pytest.mark.parametrize("drifted", [False, True], ids=["in_tiles", "drifted"])
def test_gather_transpose_in_E(drifted):
    s = _sim()
    npart = 400
    _particles(s, npart, 14, u_th=0.8 if drifted else 0.2)
    _drift(s, drifted)
    rng = np.random.default_rng(15)
    E0 = [rng.normal(size=s.shape3) for _ in range(3)]
    for c in range(3):
        s.set_field(c, E0[c])
    u0 = _momenta_by_id(s, npart)
    s.tape_begin(1)
    s.step(1)
    du = _momenta_by_id(s, npart) - u0  # (q dt/m) G E0, linear in E0
    y = rng.normal(size=(3, npart))
    s.adjoint_begin(npart)
    s.adjoint_set_momenta(0, y)
    s.adjoint_step(1)
    lE = [s.adjoint_field(c) for c in range(3)]
    lhs, rhs = float((du * y).sum()), _dot(E0, lE)
    scale = float(np.abs(du * y).sum()) + _scale(E0, lE)
    print("gather E", lhs, rhs, abs(lhs - rhs) / scale)
    assert abs(lhs - rhs) <= TOL * scale, (lhs, rhs)
    _check_paths(s, npart, drifted)
    s.close()


def test_momentum_jacobian_in_B():
    rng = np.random.default_rng(16)
    npart = 300
    shape = (1, 24, 32)
    E0 = [0.3 * rng.normal(size=shape) for _ in range(3)]
    B0 = [0.5 * rng.normal(size=shape) for _ in range(3)]
    v = [rng.normal(size=shape) for _ in range(3)]
    y = rng.normal(size=(3, npart))

    def run(Bf, adjoint=False):
        s = _sim()
        _particles(s, npart, 17)
        for c in range(3):
            s.set_field(c, E0[c])
            s.set_field(3 + c, Bf[c])
        s.tape_begin(1)
        s.step(1)
        F = float((_momenta_by_id(s, npart) * y).sum())
        lB = None
        if adjoint:
            s.adjoint_begin(npart)
            s.adjoint_set_momenta(0, y)
            s.adjoint_step(1)
            lB = [s.adjoint_field(3 + c) for c in range(3)]
        s.close()
        return F, lB

    h = 1e-5
    _, lB = run(B0, adjoint=True)
    Fp, _ = run([b + h * dv for b, dv in zip(B0, v)])
    Fm, _ = run([b - h * dv for b, dv in zip(B0, v)])
    fd = (Fp - Fm) / (2 * h)
    ad = _dot(v, lB)
    print("jacobian in B", ad, fd, abs(ad - fd) / abs(fd))
    assert abs(fd) > 0
    assert abs(ad - fd) <= 1e-8 * abs(fd), (ad, fd)
