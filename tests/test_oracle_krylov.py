"""The premise of the flexible-CG viscous solve, checked on the oracle alone:
with the oracle's own FP64 V-cycle as preconditioner, a flexible conjugate-
gradient iteration on the viscous system reaches the same relative residual
in fewer V-cycles than plain V-cycle iteration when the viscosity contrast
is large, and converges to the same discrete solution."""
import numpy as np

from oracle import oracle as O
from paper_1302_3663_gb300 import workloads as W


def _setup():
    # a 16 x 16 x 32 duct with a stiff, very viscous mound (ratio 1e3)
    h = 1.0 / 16
    rng = np.random.Generator(np.random.PCG64(4))
    X = W._hemisphere_points(rng, 300, (0.5, 0.0, 1.0), 0.3, 3)
    prm = W._duct_params(16, 32, 0.04, 1.5, 1e3, (2.0 / 3.0 * np.pi * 0.3 ** 3) / 300,
                         vc_visc=0, vc_p=0, rtol=1e-10, max_cycles=200, nu1=2, nu2=2)
    inst = W._instance(prm, X, 0.04, 1.0, 0.3, 1, "krylov")
    o = O.Oracle(prm)
    o.set_nodes(inst["X"])
    o.set_springs(inst["ab"], inst["rest"], inst["K"], inst["brk"])
    o.refresh()
    o.stage("rhs")
    return o


def _dot(a, b):
    return sum(float(np.sum(x * y)) for x, y in zip(a, b))


def test_flexible_cg_needs_fewer_vcycles_than_vcycle_iteration():
    o = _setup()
    D = 3
    f = [o.get("urhs", d).copy() for d in range(D)]
    x0 = [o.get("ut", d).copy() for d in range(D)]
    fn = np.sqrt(_dot(f, f))
    tol = 1e-10

    def resid(x):
        return [fi - ai for fi, ai in zip(f, o.apply_visc(x))]

    # plain V-cycles from x0
    for d in range(D):
        o.set("ut", x0[d], d)
    plain = 0
    while np.sqrt(_dot(r := resid([o.get("ut", d) for d in range(D)]), r)) / fn > tol:
        o.vcycle_visc()
        plain += 1
        assert plain < 200
    x_plain = [o.get("ut", d).copy() for d in range(D)]

    def precondition(r):
        for d in range(D):
            o.set("urhs", r[d], d)
            o.set("ut", np.zeros_like(r[d]), d)
        o.vcycle_visc()
        return [o.get("ut", d).copy() for d in range(D)]

    # flexible CG: z = M r, beta = -(z.q)/(p.q), p = z + beta p, q = A p
    x = [a.copy() for a in x0]
    r = resid(x)
    p = q = None
    cg = 0
    while np.sqrt(_dot(r, r)) / fn > tol:
        z = precondition(r)
        w = o.apply_visc(z)
        if p is None:
            p, q = z, w
        else:
            beta = -_dot(z, q) / pq
            p = [zi + beta * pi for zi, pi in zip(z, p)]
            q = [wi + beta * qi for wi, qi in zip(w, q)]
        pq = _dot(p, q)
        alpha = _dot(p, r) / pq
        x = [xi + alpha * pi for xi, pi in zip(x, p)]
        r = [ri - alpha * qi for ri, qi in zip(r, q)]
        cg += 1
        assert cg < 200
    # the recursive residual is the true one, and both reach the same solution
    rt = resid(x)
    assert np.sqrt(_dot(rt, rt)) / fn <= 2 * tol
    scale = np.sqrt(_dot(x_plain, x_plain))
    diff = np.sqrt(sum(float(np.sum((a - b) ** 2)) for a, b in zip(x, x_plain)))
    assert diff / scale < 1e-8
    print("V-cycles: plain %d, flexible CG %d" % (plain, cg))
    assert cg < plain
