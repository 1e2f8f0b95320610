"""Pins for the oracle's discrete operators and multigrid (Sec. 3.4, 3.5, 4.1).

* Pressure operator D.(beta D p) (Eq. divergenceGrad): symmetric, constants in
  its null space, diagonal equal to the assembled matrix diagonal, and a
  manufactured solution converging at O(h^2).
* Viscous operator (Eq. divergenceGrad + Eq. divergencePartial, staggered):
  symmetric; for constant mu and a discretely divergence-free field it equals
  mu times the plain component Laplacian (the constant-viscosity form of
  Eq. NSdis1); truncation error O(h^2) against the analytic
  div(mu (grad u + grad u^T)); manufactured wall-bounded solution O(h^2).
* Multigrid: V(2,2) contraction <= 0.2 per cycle for constant-coefficient
  Poisson, independent of h; relative residual 1e-9 is reached (Sec. 4.1);
  converged multigrid equals a dense LU solve on tiny grids, whose condition
  number grows like h^-2 (Sec. 4.1).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1302_3663_gb300 import workloads as W


def p2(n, periodic=(1, 0), h=None, **kw):
    h = h if h is not None else 1.0 / n[0]
    return W.base_params(2, n, periodic, 0, h, **kw)


def p3(n, periodic=(0, 0, 1), h=None, **kw):
    h = h if h is not None else 1.0 / n[0]
    return W.base_params(3, n, periodic, 2, h, **kw)


def cell_mask(o, level=0):
    n, s = o.dims(level)
    m = np.zeros(o.shape(level), bool)
    if o.dim == 3:
        m[:n[2], :n[1], :n[0]] = True
    else:
        m[:n[1], :n[0]] = True
    return m


def face_mask(o, d, level=0):
    n, s = o.dims(level)
    lo = [0, 0, 0]
    hi = [n[0], n[1], n[2]]
    if not o.prm["periodic"][d]:
        lo[d], hi[d] = 1, n[d]
    m = np.zeros(o.shape(level), bool)
    if o.dim == 3:
        m[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = True
    else:
        m[lo[1]:hi[1], lo[0]:hi[0]] = True
    return m


def coord_axes(o, stag, level=0):
    n, s = o.dims(level)
    h = o.prm["h"] * 2 ** level
    return [(np.arange(s[a]) + 0.5 * stag[a]) * h for a in range(o.dim)]


def mesh(o, stag, level=0):
    ax = coord_axes(o, stag, level)
    if o.dim == 3:
        Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        return X, Y, Z
    Y, X = np.meshgrid(ax[1], ax[0], indexing="ij")
    return X, Y


def set_coefficients(o, rho_fn=None, mu_fn=None):
    """Install rho on the faces and mu at centres and edges, then the hierarchy."""
    D = o.dim
    for d in range(D):
        stag = [1] * D
        stag[d] = 0
        P = mesh(o, stag)
        o.set("rho", rho_fn(*P) if rho_fn else np.ones(o.shape()), d)
    if mu_fn is not None:
        o.set("muc", mu_fn(*mesh(o, [1] * D)))
        pairs = [(0, 1)] if D == 2 else [(0, 1), (0, 2), (1, 2)]
        for q, (d, e) in enumerate(pairs):
            stag = [1] * D
            stag[d] = stag[e] = 0
            o.set("mue", mu_fn(*mesh(o, stag)), q)
    o.build_coefficients()


# ---------------------------------------------------------------------------
# pressure operator
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [2, 3])
def test_pressure_operator_symmetric_nullspace_diag(dim):
    o = O.Oracle(p2((8, 4)) if dim == 2 else p3((4, 4, 4)))
    rng = np.random.default_rng(0)
    set_coefficients(o, rho_fn=lambda *X: 1.0 + rng.uniform(0, 2, size=X[0].shape))
    cm = cell_mask(o)
    idx = np.flatnonzero(cm.ravel())
    A = np.zeros((idx.size, idx.size))
    for c, i in enumerate(idx):
        e = np.zeros(o.shape())
        e.ravel()[i] = 1.0
        A[:, c] = o.apply_p(e).ravel()[idx]
    assert np.allclose(A, A.T, rtol=0, atol=1e-10 * np.abs(A).max())
    assert np.abs(A.sum(axis=0)).max() < 1e-10 * np.abs(A).max()
    ev = np.linalg.eigvalsh(0.5 * (A + A.T))
    assert ev.max() < 1e-9 * np.abs(ev).max() and np.sum(np.abs(ev) < 1e-9 * np.abs(ev).max()) == 1
    n, _ = o.dims()
    for c, i in enumerate(idx[:10]):
        k, rem = divmod(i, o.shape()[-1] * o.shape()[-2]) if dim == 3 else (0, i)
        j, ii = divmod(rem, o.shape()[-1])
        assert abs(o.p_diag(0, ii, j, k) - A[c, c]) < 1e-12 * abs(A[c, c])


def solve_pressure_mms(o, pstar, beta, rhs):
    set_coefficients(o, rho_fn=lambda *X: 1.0 / beta(*X))
    C = mesh(o, [1] * o.dim)
    cm = cell_mask(o)
    b = np.where(cm, rhs(*C), 0.0)
    b[cm] -= b[cm].mean()
    o.set("prhs", b)
    o.set("p", np.zeros(o.shape()))
    o.prm["rtol"] = 1e-12
    cyc = o.solve_p(0)
    p = o.get("p")
    ex = pstar(*C)
    ex = ex - ex[cm].mean()
    return np.abs(p[cm] - ex[cm]).max(), cyc


def test_pressure_mms_second_order_2d():
    # Neumann walls in y, periodic in x; smooth variable beta
    H = 0.5
    pstar = lambda x, y: np.cos(2 * np.pi * x) * np.cos(2 * np.pi * y / H)
    beta = lambda x, y: 1.0 + 0.5 * np.sin(2 * np.pi * x) * np.cos(np.pi * y / H)

    def rhs(x, y):
        bx = 0.5 * 2 * np.pi * np.cos(2 * np.pi * x) * np.cos(np.pi * y / H)
        by = -0.5 * (np.pi / H) * np.sin(2 * np.pi * x) * np.sin(np.pi * y / H)
        px = -2 * np.pi * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y / H)
        py = -(2 * np.pi / H) * np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y / H)
        lap = -((2 * np.pi) ** 2 + (2 * np.pi / H) ** 2) * pstar(x, y)
        return beta(x, y) * lap + bx * px + by * py

    errs = []
    for n in (16, 32, 64, 128):
        prm = p2((n, n // 2), rtol=1e-12, max_cycles=80)
        o = O.Oracle(prm)
        e, cyc = solve_pressure_mms(o, pstar, beta, rhs)
        errs.append(e)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.15), (errs, rates)


def test_pressure_mms_second_order_3d():
    pstar = lambda x, y, z: np.cos(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * z)
    beta = lambda x, y, z: 1.0 + 0.3 * np.sin(np.pi * x) * np.sin(np.pi * y)

    def rhs(x, y, z):
        bx = 0.3 * np.pi * np.cos(np.pi * x) * np.sin(np.pi * y)
        by = 0.3 * np.pi * np.sin(np.pi * x) * np.cos(np.pi * y)
        px = -np.pi * np.sin(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * z)
        py = -np.pi * np.cos(np.pi * x) * np.sin(np.pi * y) * np.cos(np.pi * z)
        return beta(x, y, z) * (-3 * np.pi ** 2) * pstar(x, y, z) + bx * px + by * py

    errs = []
    for n in (8, 16, 32):
        o = O.Oracle(p3((n, n, 2 * n), rtol=1e-12, max_cycles=80))
        errs.append(solve_pressure_mms(o, pstar, beta, rhs)[0])
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.2), (errs, rates)


# ---------------------------------------------------------------------------
# viscous operator
# ---------------------------------------------------------------------------
def unknown_vec(o, rng):
    return [np.where(face_mask(o, d), rng.normal(size=o.shape()), 0.0) for d in range(o.dim)]


@pytest.mark.parametrize("case", ["2d", "3d", "2d_per"])
def test_viscous_operator_symmetric_and_diag(case):
    if case == "2d":
        o = O.Oracle(p2((8, 6)))
    elif case == "2d_per":
        o = O.Oracle(p2((8, 6), periodic=(1, 1)))
    else:
        o = O.Oracle(p3((4, 6, 4)))
    rng = np.random.default_rng(1)
    set_coefficients(o, rho_fn=lambda *X: 1.0 + rng.uniform(0, 1, size=X[0].shape),
                     mu_fn=lambda *X: 0.01 * np.exp(rng.uniform(0, np.log(1e3), size=X[0].shape)))
    for _ in range(3):
        u = unknown_vec(o, rng)
        v = unknown_vec(o, rng)
        Au = o.apply_visc(u)
        Av = o.apply_visc(v)
        lhs = sum(float((Au[d] * v[d]).sum()) for d in range(o.dim))
        rhs = sum(float((u[d] * Av[d]).sum()) for d in range(o.dim))
        assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + abs(rhs))
        # positive definite: m > 0 plus a positive semi-definite viscous part
        assert sum(float((Au[d] * u[d]).sum()) for d in range(o.dim)) > 0
    # diagonal entries match the operator applied to unit vectors
    for d in range(o.dim):
        fm = face_mask(o, d)
        for i in np.flatnonzero(fm.ravel())[::5]:
            e = [np.zeros(o.shape()) for _ in range(o.dim)]
            e[d].ravel()[i] = 1.0
            Ae = o.apply_visc(e)[d].ravel()[i]
            sh = o.shape()
            if o.dim == 3:
                k, rem = divmod(i, sh[1] * sh[2])
            else:
                k, rem = 0, i
            j, ii = divmod(rem, sh[-1])
            assert abs(o.visc_diag(0, d, ii, j, k) - Ae) < 1e-12 * abs(Ae)


def roll(a, shift, axis_xyz, dim):
    return np.roll(a, shift, axis=(dim - 1 - axis_xyz))


@pytest.mark.parametrize("dim", [2, 3])
def test_constant_mu_divfree_reduces_to_laplacian(dim):
    # For constant mu and D.u = 0 the coupled operator equals mu L_h u per
    # component, the paper's constant-viscosity form (Eq. NSdis1).
    n = (16, 8) if dim == 2 else (8, 6, 4)
    o = O.Oracle(p2(n, periodic=(1, 1)) if dim == 2 else p3(n, periodic=(1, 1, 1)))
    h = o.prm["h"]
    mu0 = 0.37
    set_coefficients(o, rho_fn=lambda *X: np.zeros_like(X[0]), mu_fn=lambda *X: mu0 + 0 * X[0])
    rng = np.random.default_rng(4)
    sh = o.shape()
    if dim == 2:
        psi = rng.normal(size=sh)          # at the xy corners
        ux = (roll(psi, -1, 1, 2) - psi) / h
        uy = -(roll(psi, -1, 0, 2) - psi) / h
        u = [ux, uy]
    else:
        Ax, Ay, Az = (rng.normal(size=sh) for _ in range(3))   # yz, xz, xy edges
        ux = (roll(Az, -1, 1, 3) - Az) / h - (roll(Ay, -1, 2, 3) - Ay) / h
        uy = (roll(Ax, -1, 2, 3) - Ax) / h - (roll(Az, -1, 0, 3) - Az) / h
        uz = (roll(Ay, -1, 0, 3) - Ay) / h - (roll(Ax, -1, 1, 3) - Ax) / h
        u = [ux, uy, uz]
    div = sum((roll(u[a], -1, a, dim) - u[a]) / h for a in range(dim))
    assert np.abs(div).max() < 1e-10 * np.abs(u[0]).max() / h
    Au = o.apply_visc(u)
    for d in range(dim):
        lap = sum((roll(u[d], -1, a, dim) - 2 * u[d] + roll(u[d], 1, a, dim)) / h ** 2
                  for a in range(dim))
        assert np.abs(Au[d] + mu0 * lap).max() < 1e-11 * np.abs(mu0 * lap).max()


def _visc_analytic_2d():
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    u = [sp.sin(2 * sp.pi * x) * sp.cos(2 * sp.pi * y), 0.5 * sp.cos(2 * sp.pi * x) * sp.sin(4 * sp.pi * y)]
    mu = 1 + 0.5 * sp.cos(2 * sp.pi * x) * sp.sin(2 * sp.pi * y)
    X = [x, y]
    V = []
    for d in range(2):
        V.append(sum(sp.diff(mu * (sp.diff(u[d], X[e]) + sp.diff(u[e], X[d])), X[e]) for e in range(2)))
    f = lambda ex: sp.lambdify((x, y), ex, "numpy")
    return [f(c) for c in u], f(mu), [f(c) for c in V]


def test_viscous_truncation_second_order_periodic_2d():
    us, mu, Vs = _visc_analytic_2d()
    errs = []
    for n in (32, 64, 128, 256):
        o = O.Oracle(p2((n, n), periodic=(1, 1)))
        set_coefficients(o, rho_fn=lambda *X: np.zeros_like(X[0]), mu_fn=lambda *X: mu(*X) + 0 * X[0])
        u = []
        for d in range(2):
            stag = [1, 1]
            stag[d] = 0
            u.append(us[d](*mesh(o, stag)) + 0 * mesh(o, stag)[0])
        Au = o.apply_visc(u)
        e = 0.0
        for d in range(2):
            stag = [1, 1]
            stag[d] = 0
            e = max(e, np.abs(Au[d] + Vs[d](*mesh(o, stag))).max())
        errs.append(e)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.1), (errs, rates)


def test_viscous_wall_mms_solution_second_order():
    # periodic x, no-slip walls at y = 0 and 0.5: u* = 0 on the walls
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    H = sp.Rational(1, 2)
    u = [sp.sin(sp.pi * y / H) * sp.cos(2 * sp.pi * x), 0.3 * sp.sin(2 * sp.pi * y / H) * sp.sin(2 * sp.pi * x)]
    mu = 0.05 * (1 + 0.5 * sp.cos(2 * sp.pi * x) * sp.cos(sp.pi * y / H))
    m0 = 10.0
    X = [x, y]
    f = [m0 * u[d] - sum(sp.diff(mu * (sp.diff(u[d], X[e]) + sp.diff(u[e], X[d])), X[e])
                         for e in range(2)) for d in range(2)]
    L = lambda ex: sp.lambdify((x, y), ex, "numpy")
    us, fs, mus = [L(c) for c in u], [L(c) for c in f], L(mu)
    errs = []
    for n in (16, 32, 64, 128):
        prm = p2((n, n // 2), rtol=1e-12, max_cycles=100, dt=1.0)
        o = O.Oracle(prm)
        set_coefficients(o, rho_fn=lambda *Xs: m0 + 0 * Xs[0], mu_fn=lambda *Xs: mus(*Xs) + 0 * Xs[0])
        for d in range(2):
            stag = [1, 1]
            stag[d] = 0
            P = mesh(o, stag)
            o.set("urhs", np.where(face_mask(o, d), fs[d](*P) + 0 * P[0], 0.0), d)
            o.set("ut", np.zeros(o.shape()), d)
        o.solve_visc(0)
        e = 0.0
        for d in range(2):
            stag = [1, 1]
            stag[d] = 0
            P = mesh(o, stag)
            fm = face_mask(o, d)
            e = max(e, np.abs(o.get("ut", d)[fm] - (us[d](*P) + 0 * P[0])[fm]).max())
        errs.append(e)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.85), (errs, rates)


# ---------------------------------------------------------------------------
# multigrid
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [32, 64, 128])
def test_mg_contraction_constant_coefficient_poisson(n):
    o = O.Oracle(p2((n, n // 2)))
    set_coefficients(o)
    rng = np.random.default_rng(n)
    cm = cell_mask(o)
    b = np.where(cm, rng.normal(size=o.shape()), 0.0)
    b[cm] -= b[cm].mean()
    o.set("prhs", b)
    o.set("p", np.zeros(o.shape()))
    norms = [np.linalg.norm(o.residual_p()[cm])]
    for k in range(8):
        o.vcycle_p()
        norms.append(np.linalg.norm(o.residual_p()[cm]))
    factors = np.array(norms[1:]) / np.array(norms[:-1])
    assert factors[2:].max() <= 0.2, factors
    assert norms[-1] / norms[0] <= 1e-9


def dense_visc(o):
    idx = [np.flatnonzero(face_mask(o, d).ravel()) for d in range(o.dim)]
    cols = []
    for d in range(o.dim):
        for i in idx[d]:
            e = [np.zeros(o.shape()) for _ in range(o.dim)]
            e[d].ravel()[i] = 1.0
            Ae = o.apply_visc(e)
            cols.append(np.concatenate([Ae[q].ravel()[idx[q]] for q in range(o.dim)]))
    return np.array(cols).T, idx


@pytest.mark.parametrize("dim", [2, 3])
def test_mg_equals_dense_solve_tiny(dim):
    prm = p2((8, 4), rtol=1e-14, max_cycles=200) if dim == 2 else p3((4, 4, 4), rtol=1e-14, max_cycles=200)
    o = O.Oracle(prm)
    rng = np.random.default_rng(9)
    set_coefficients(o, rho_fn=lambda *X: 1.0 + rng.uniform(0, 1, size=X[0].shape),
                     mu_fn=lambda *X: 0.01 * np.exp(rng.uniform(0, np.log(100), size=X[0].shape)))
    # pressure: dense least-norm solution with zero mean
    cm = cell_mask(o)
    idx = np.flatnonzero(cm.ravel())
    A = np.zeros((idx.size, idx.size))
    for c, i in enumerate(idx):
        e = np.zeros(o.shape())
        e.ravel()[i] = 1.0
        A[:, c] = o.apply_p(e).ravel()[idx]
    b = rng.normal(size=idx.size)
    b -= b.mean()
    bb = np.zeros(o.shape())
    bb.ravel()[idx] = b
    o.set("prhs", bb)
    o.set("p", np.zeros(o.shape()))
    o.solve_p(0)
    x = np.linalg.lstsq(A, b, rcond=None)[0]
    x -= x.mean()
    pm = o.get("p").ravel()[idx]
    assert np.abs(pm - x).max() < 1e-12 * np.abs(x).max()
    # viscous
    M, fidx = dense_visc(o)
    rhs = rng.normal(size=M.shape[0])
    off = 0
    for d in range(o.dim):
        a = np.zeros(o.shape())
        a.ravel()[fidx[d]] = rhs[off:off + fidx[d].size]
        off += fidx[d].size
        o.set("urhs", a, d)
        o.set("ut", np.zeros(o.shape()), d)
    o.solve_visc(0)
    sol = np.linalg.solve(M, rhs)
    got = np.concatenate([o.get("ut", d).ravel()[fidx[d]] for d in range(o.dim)])
    assert np.abs(got - sol).max() < 1e-12 * np.abs(sol).max()


def test_condition_number_grows_like_h_minus_2():
    conds = []
    for n in (8, 16, 32):
        o = O.Oracle(p2((n, n // 2)))
        set_coefficients(o)
        cm = cell_mask(o)
        idx = np.flatnonzero(cm.ravel())
        A = np.zeros((idx.size, idx.size))
        for c, i in enumerate(idx):
            e = np.zeros(o.shape())
            e.ravel()[i] = 1.0
            A[:, c] = o.apply_p(e).ravel()[idx]
        ev = np.sort(np.abs(np.linalg.eigvalsh(A)))
        conds.append(ev[-1] / ev[1])  # drop the constant null vector
    r = np.array(conds[1:]) / np.array(conds[:-1])
    assert np.all(np.abs(r - 4.0) < 0.3), conds
