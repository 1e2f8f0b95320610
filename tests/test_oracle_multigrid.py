"""Pins for the oracle's multigrid transfers and the viscous V-cycle (Sec. 3.5,
Eq. ViscCoarseGrid).

* Transfers in closed form. Restriction of x^2: the mean of two cell children
  gives X^2 + h^2/4, the (1/4, 1/2, 1/4) face stencil X^2 + h^2/2.
  Prolongation of X^2: the bilinear (3/4, 1/4) cell rule gives x^2 + 3h^2/4
  and a midway face x^2 + h^2 (coincident faces copy). At a wall the pressure's
  even mirror reproduces constants and the velocity's odd mirror reproduces a
  field vanishing linearly on the wall.
* Coefficients on the coarse grids: beta averages the fine faces on the coarse
  face (coincident along d), mu at centres averages the 2^D children and on
  edges the two fine edges along the third axis, each then times gamma.
* Viscous V(2,2) cycle: for constant mu the contraction per cycle stays below
  0.15 and does not grow as h falls (grids 32, 64, 128 in 2D; 16, 32 in 3D);
  with a smooth viscosity contrast of 1e3 (and a density contrast of 2) at the
  workloads' time step it stays below 0.3 with gamma = 1 and with gamma = 0.8.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1302_3663_gb300 import workloads as W

from test_oracle_operators import cell_mask, face_mask, mesh, set_coefficients


def _duct(n=(16, 12, 20), **kw):
    return O.Oracle(W.base_params(3, n, (0, 0, 1), 2, 1.0 / n[0], **kw))


def _chan(n=(16, 12), **kw):
    return O.Oracle(W.base_params(2, n, (1, 0), 0, 1.0 / n[0], **kw))


def _stag_face(D, d):
    s = [1] * D
    s[d] = 0
    return s


def _interior_face_mask(o, d, level):
    """Unknown faces of component d on `level`, without those whose stencil
    along a periodic axis d wraps (face 0 and the last one)."""
    m = face_mask(o, d, level)
    if o.prm["periodic"][d]:
        n, _ = o.dims(level)
        sl = [slice(None)] * o.dim
        sl[o.dim - 1 - d] = 0
        m[tuple(sl)] = False
        sl[o.dim - 1 - d] = n[d] - 1
        m[tuple(sl)] = False
    return m


@pytest.mark.parametrize("make", [_chan, _duct])
def test_restriction_closed_forms(make):
    o = make()
    h = o.prm["h"]
    D = o.dim
    for a in range(D):
        # cell-centred: mean of the 2^D children
        f = mesh(o, [1] * D)[a] ** 2
        got = o.restrict(f, 0, -1)
        want = mesh(o, [1] * D, 1)[a] ** 2 + h * h / 4
        cm = cell_mask(o, 1)
        assert np.abs(got - want)[cm].max() <= 1e-14
        # faces of every component: (1/4, 1/2, 1/4) along d, child mean across
        for d in range(D):
            f = mesh(o, _stag_face(D, d))[a] ** 2
            got = o.restrict(f, 0, d)
            want = mesh(o, _stag_face(D, d), 1)[a] ** 2 + (h * h / 2 if a == d else h * h / 4)
            fm = _interior_face_mask(o, d, 1)
            assert np.abs(got - want)[fm].max() <= 1e-14, (a, d)


def _inner(o, d):
    """Fine points (of component d's faces, or of cells for d < 0) whose
    prolongation stencil neither wraps around a periodic axis nor reaches
    beyond a wall: faces 1..n-2 along d, cells 1..n-2 across."""
    n, _ = o.dims(0)
    m = np.zeros(o.shape(0), bool)
    sl = []
    for b in reversed(range(o.dim)):
        sl.append(slice(1, n[b] - 1))
    m[tuple(sl)] = True
    return m


@pytest.mark.parametrize("make", [_chan, _duct])
def test_prolongation_closed_forms(make):
    o = make()
    h = o.prm["h"]
    D = o.dim
    for a in range(D):
        c = mesh(o, [1] * D, 1)[a] ** 2
        got = o.prolong_add(c, np.zeros(o.shape(0)), 0, -1)
        want = mesh(o, [1] * D)[a] ** 2 + 0.75 * h * h
        m = _inner(o, -1)
        assert np.abs(got - want)[m].max() <= 1e-14
        for d in range(D):
            c = mesh(o, _stag_face(D, d), 1)[a] ** 2
            got = o.prolong_add(c, np.zeros(o.shape(0)), 0, d)
            x = mesh(o, _stag_face(D, d))[a]
            if a == d:   # coincident faces copy, midway faces average two
                even = (np.rint(x / h).astype(int) % 2) == 0
                want = np.where(even, x ** 2, x ** 2 + h * h)
            else:
                want = x ** 2 + 0.75 * h * h
            m = _inner(o, d)
            assert np.abs(got - want)[m].max() <= 1e-13, (a, d)
        if not o.prm["periodic"][a]:
            # next to the lower wall: even mirror for the pressure (constants
            # reproduced), odd mirror for velocity (a field ~ distance to the wall)
            ax = D - 1 - a
            first = tuple(slice(None) if q != ax else 0 for q in range(D))
            got = o.prolong_add(np.full(o.shape(1), 2.5), np.zeros(o.shape(0)), 0, -1)
            assert np.abs(got[first][cell_mask(o)[first]] - 2.5).max() <= 1e-15
            for d in range(D):
                if d == a:
                    continue
                c = mesh(o, _stag_face(D, d), 1)[a]
                got = o.prolong_add(c, np.zeros(o.shape(0)), 0, d)
                x = mesh(o, _stag_face(D, d))[a]
                m = np.roll(_inner(o, d), -1, axis=ax)   # interior across, first row along a
                assert m[first].any()
                assert np.abs(got[first] - x[first])[m[first]].max() <= 1e-15


@pytest.mark.parametrize("make", [_chan, _duct])
def test_coefficient_restriction_with_gamma(make):
    gam = 0.7
    o = make(gamma_coarse=gam)
    h = o.prm["h"]
    D = o.dim
    pairs = [(0, 1)] if D == 2 else [(0, 1), (0, 2), (1, 2)]
    for a in range(D):
        q = lambda *X: 1.0 + X[a] ** 2
        set_coefficients(o, rho_fn=lambda *X: 1.0 / q(*X), mu_fn=q)
        for d in range(D):   # beta = 1 / rho: coincident along d, child mean across
            got = o.get("beta", d, 1)
            want = 1.0 + mesh(o, _stag_face(D, d), 1)[a] ** 2 + (0.0 if a == d else h * h / 4)
            fm = face_mask(o, d, 1)
            assert np.abs(got - want)[fm].max() <= 1e-13
        got = o.get("muc", 0, 1)
        want = gam * (1.0 + mesh(o, [1] * D, 1)[a] ** 2 + h * h / 4)
        assert np.abs(got - want)[cell_mask(o, 1)].max() <= 1e-13
        n, _ = o.dims(1)
        for k, (d, e) in enumerate(pairs):
            stag = [1] * D
            stag[d] = stag[e] = 0
            got = o.get("mue", k, 1)
            third = 3 - d - e if D == 3 else -1
            want = gam * (1.0 + mesh(o, stag, 1)[a] ** 2 + (h * h / 4 if a == third else 0.0))
            m = np.zeros(o.shape(1), bool)
            lim = [n[b] + (0 if (b in (d, e) and o.prm["periodic"][b]) else 1) if b in (d, e) else n[b]
                   for b in range(D)]
            m[tuple(slice(0, lim[b]) for b in reversed(range(D)))] = True
            assert np.abs(got - want)[m].max() <= 1e-13, (a, d, e)


def _visc_factors(o, ncyc):
    rng = np.random.default_rng(1)
    D = o.dim
    for d in range(D):
        o.set("urhs", np.where(face_mask(o, d), rng.normal(size=o.shape()), 0.0), d)
        o.set("ut", np.zeros(o.shape()), d)

    def rnorm():
        r = o.residual_visc()
        return np.sqrt(sum(np.sum(r[d][face_mask(o, d)] ** 2) for d in range(D)))

    norms = [rnorm()]
    for _ in range(ncyc):
        o.vcycle_visc()
        norms.append(rnorm())
    return np.array(norms[1:]) / np.array(norms[:-1])


@pytest.mark.parametrize("dim,n", [(2, 32), (2, 64), (2, 128), (3, 16), (3, 32)])
def test_viscous_vcycle_contraction_constant_mu(dim, n):
    # dt = 1: the viscous term dominates the mass term on every level
    if dim == 2:
        o = O.Oracle(W.base_params(2, (n, n // 2), (1, 0), 0, 1.0 / n, dt=1.0, mu_f=1.0))
    else:
        o = O.Oracle(W.base_params(3, (n, n, n), (0, 0, 1), 2, 1.0 / n, dt=1.0, mu_f=1.0))
    set_coefficients(o, mu_fn=lambda *X: 1.0 + 0 * X[0])
    f = _visc_factors(o, 8)
    assert f[2:].max() <= 0.15, f


def _smooth_blob(*X):
    c = [0.5, 0.0, 0.5][:len(X)]
    r = np.sqrt(sum((x - cc) ** 2 for x, cc in zip(X, c)))
    return 0.5 * (1.0 - np.tanh((r - 0.15) / 0.02))


@pytest.mark.parametrize("gamma", [1.0, 0.8])
@pytest.mark.parametrize("dim,n", [(2, 64), (2, 128), (3, 32)])
def test_viscous_vcycle_contraction_viscosity_ratio_1e3(dim, n, gamma):
    h = 1.0 / n
    if dim == 2:
        prm = W.base_params(2, (n, n // 2), (1, 0), 0, h, dt=0.1 * h, gamma_coarse=gamma)
    else:
        prm = W.base_params(3, (n, n, n), (0, 0, 1), 2, h, dt=0.1 * h, gamma_coarse=gamma)
    o = O.Oracle(prm)
    set_coefficients(o, rho_fn=lambda *X: 1.0 + _smooth_blob(*X),
                     mu_fn=lambda *X: 0.01 * (1.0 + 999.0 * _smooth_blob(*X)))
    f = _visc_factors(o, 10)
    print("viscosity ratio 1e3, %dD n=%d gamma=%.1f: factors %s" % (dim, n, gamma, np.round(f, 3)))
    assert f[2:].max() <= 0.3, f
