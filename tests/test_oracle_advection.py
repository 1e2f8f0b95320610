"""Pins for the oracle's advection term, Eq. (NSdis1-1): Adv_d = 1/2 (u.D u_d +
D.(u u_d)) in the staggered skew form.

* Consistency: against the exact 1/2 (u.grad u_d + div(u u_d)) of a smooth
  field the error falls as h^2, on a periodic 2D grid (a field that is not
  divergence free, so that both halves matter, and a Taylor-Green vortex, for
  which the exact value is (u.grad) u_d) and on a 3D duct with no-slip walls,
  where the tangential mirror ghost enters.
* Energy: on the paper's collocated grid the skew form with the antisymmetric
  D0 gives sum_x u_k Adv_k = 0 for every field; the staggered form keeps this
  identity, to rounding, for any field (periodic, and with walls whose normal
  faces hold 0).
* A uniform flow has no advection; Adv is homogeneous of degree 2.
A dropped half, a sign slip, a transverse mean taken at the wrong edge or a
wrong mirror fails one of these.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1302_3663_gb300 import workloads as W

from test_oracle_operators import face_mask, mesh

sp = pytest.importorskip("sympy")


def _exact_skew(u, X):
    """1/2 (u.grad u_d + div(u u_d)) for sympy expressions u over coordinates X."""
    D = len(X)
    out = []
    for d in range(D):
        adv = sum(u[e] * sp.diff(u[d], X[e]) for e in range(D))
        cons = sum(sp.diff(u[e] * u[d], X[e]) for e in range(D))
        out.append(sp.Rational(1, 2) * (adv + cons))
    return out


def _faces(o, f, d):
    stag = [1] * o.dim
    stag[d] = 0
    P = mesh(o, stag)
    return f(*P) + 0 * P[0]


def _max_error(o, u_exprs, A_exprs, X, walls):
    D = o.dim
    fu = [sp.lambdify(X, c, "numpy") for c in u_exprs]
    fA = [sp.lambdify(X, c, "numpy") for c in A_exprs]
    u = [np.where(face_mask(o, d), _faces(o, fu[d], d), 0.0) if walls else _faces(o, fu[d], d)
         for d in range(D)]
    A = o.advection(u)
    e = 0.0
    for d in range(D):
        fm = face_mask(o, d)
        e = max(e, np.abs(A[d][fm] - _faces(o, fA[d], d)[fm]).max())
    return e


def _rates(errs):
    errs = np.asarray(errs)
    return np.log2(errs[:-1] / errs[1:])


def test_second_order_periodic_2d_general_field():
    x, y = sp.symbols("x y")
    pi = sp.pi
    u = [sp.sin(2 * pi * x) * sp.cos(2 * pi * y) + sp.Rational(3, 10) * sp.cos(2 * pi * y),
         sp.cos(2 * pi * (x + y)) / 2 + sp.sin(2 * pi * x) / 5]
    assert sp.simplify(sp.diff(u[0], x) + sp.diff(u[1], y)) != 0   # both halves matter
    A = _exact_skew(u, [x, y])
    errs = [_max_error(O.Oracle(W.base_params(2, (n, n), (1, 1), 0, 1.0 / n)), u, A, [x, y], False)
            for n in (16, 32, 64, 128)]
    r = _rates(errs)
    assert np.all(np.abs(r - 2.0) < 0.15), (errs, r)


def test_second_order_taylor_green_equals_u_grad_u():
    x, y = sp.symbols("x y")
    pi = sp.pi
    u = [sp.sin(2 * pi * x) * sp.cos(2 * pi * y), -sp.cos(2 * pi * x) * sp.sin(2 * pi * y)]
    assert sp.simplify(sp.diff(u[0], x) + sp.diff(u[1], y)) == 0
    A = [sum(u[e] * sp.diff(u[d], v) for e, v in enumerate((x, y))) for d in range(2)]
    errs = [_max_error(O.Oracle(W.base_params(2, (n, n), (1, 1), 0, 1.0 / n)), u, A, [x, y], False)
            for n in (16, 32, 64, 128)]
    r = _rates(errs)
    assert np.all(np.abs(r - 2.0) < 0.15), (errs, r)


def test_second_order_3d_duct_with_walls():
    # walls at x, y = 0, 1 (every component vanishes there: no slip), periodic z
    x, y, z = sp.symbols("x y z")
    pi = sp.pi
    env = sp.sin(pi * x) * sp.sin(pi * y)
    u = [env * (1 + sp.Rational(3, 10) * sp.cos(2 * pi * z)),
         sp.sin(2 * pi * x) * sp.sin(pi * y) * (1 + sp.sin(2 * pi * z) / 5) / 2,
         env * (1 + sp.Rational(2, 5) * sp.cos(2 * pi * z + sp.Rational(3, 10)))]
    A = _exact_skew(u, [x, y, z])
    errs = [_max_error(O.Oracle(W.base_params(3, (n, n, n), (0, 0, 1), 2, 1.0 / n)), u, A,
                       [x, y, z], True)
            for n in (16, 32, 64, 128)]
    r = _rates(errs)
    assert np.all(np.abs(r - 2.0) < 0.15), (errs, r)


def _random_field(o, rng):
    return [np.where(face_mask(o, d), rng.normal(size=o.shape()), 0.0) for d in range(o.dim)]


@pytest.mark.parametrize("case", ["periodic2d", "walls2d", "duct3d"])
def test_energy_neutral_for_any_field(case):
    if case == "periodic2d":
        o = O.Oracle(W.base_params(2, (24, 16), (1, 1), 0, 1.0 / 24))
    elif case == "walls2d":
        o = O.Oracle(W.base_params(2, (24, 16), (1, 0), 0, 1.0 / 24))
    else:
        o = O.Oracle(W.base_params(3, (12, 10, 16), (0, 0, 1), 2, 1.0 / 12))
    rng = np.random.default_rng(3)
    for _ in range(3):
        u = _random_field(o, rng)
        A = o.advection(u)
        terms = [u[d][face_mask(o, d)] * A[d][face_mask(o, d)] for d in range(o.dim)]
        E = sum(t.sum() for t in terms)
        S = sum(np.abs(t).sum() for t in terms)
        assert abs(E) <= 1e-13 * S, (E, S)


def test_uniform_flow_has_no_advection_and_degree_two():
    for prm in (W.base_params(2, (16, 12), (1, 1), 0, 1.0 / 16),
                W.base_params(3, (8, 6, 10), (1, 1, 1), 2, 1.0 / 8)):
        o = O.Oracle(prm)
        c = [0.7, -1.3, 0.4][:o.dim]
        A = o.advection([np.full(o.shape(), v) for v in c])
        assert all(np.abs(a).max() == 0.0 for a in A)
        rng = np.random.default_rng(5)
        u = _random_field(o, rng)
        A1 = o.advection(u)
        A3 = o.advection([3.0 * a for a in u])
        for d in range(o.dim):
            assert np.allclose(A3[d], 9.0 * A1[d], rtol=1e-13, atol=1e-13 * np.abs(A1[d]).max())
