"""Pins for the oracle's momentum right-hand side, Eq. (NSdis1-1):
rhs_d = (rho_d sigma / dt) u_d - rho_d Adv_d(u) + c_f f_d + G [d = flow axis].

Each term is isolated by a special case on a periodic grid, with the others
made to vanish, and compared with a value the test knows without the
oracle's arithmetic:
* a uniform density rho0 and a Taylor-Green vortex: rhs - (rho0 sigma / dt) u
  equals -rho0 (u.grad) u of the analytic field, to O(h^2) (the vortex is
  divergence free, so the skew form is (u.grad) u);
* fluid at rest with a prescribed force field: rhs = c_f f exactly;
* fluid at rest without force: rhs = G on the flow axis' faces, 0 elsewhere.
"""
import numpy as np

from oracle import oracle as O
from paper_1302_3663_gb300 import workloads as W


def periodic_case(n=64, **kw):
    kw = dict(dict(u_center=0.0, body_force=0.0), **kw)
    prm = W.base_params(2, (n, n), (1, 1), 0, 1.0 / n, **kw)
    o = O.Oracle(prm)
    return o, prm


def face_coords(o, d):
    h = o.prm["h"]
    n, s = o.dims()
    x = np.arange(s[0]) * h + (0.0 if d == 0 else 0.5 * h)
    y = np.arange(s[1]) * h + (0.0 if d == 1 else 0.5 * h)
    return np.meshgrid(x, y)


def set_uniform_density(o, rho0):
    for d in range(2):
        o.set("rho", np.full(o.shape(), rho0), d)
    o.build_coefficients()


def test_inertia_and_advection_terms_with_a_uniform_density():
    rho0, sigma, dt = 3.0, 0.5, 0.004
    o, prm = periodic_case(sigma=sigma, dt=dt)
    set_uniform_density(o, rho0)
    tg = [lambda x, y: np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y),
          lambda x, y: -np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y)]
    ugu = [lambda x, y: np.pi * np.sin(4 * np.pi * x),     # (u.grad) u of the vortex
           lambda x, y: np.pi * np.sin(4 * np.pi * y)]
    u = [tg[d](*face_coords(o, d)) for d in range(2)]
    for d in range(2):
        o.set("u", u[d], d)
        o.set("force", np.zeros(o.shape()), d)
    o.stage("rhs")
    m = rho0 * sigma / dt
    for d in range(2):
        adv = -(o.get("urhs", d) - m * u[d]) / rho0
        exact = ugu[d](*face_coords(o, d))
        err = np.abs(adv - exact).max()
        assert err <= 0.01 * np.abs(exact).max(), (d, err)
    o.close()


def test_force_term_at_rest():
    o, prm = periodic_case(c_force=2.5)
    set_uniform_density(o, 1.5)
    rng = np.random.default_rng(3)
    f = [rng.standard_normal(o.shape()) for _ in range(2)]
    for d in range(2):
        o.set("u", np.zeros(o.shape()), d)
        o.set("force", f[d], d)
    o.stage("rhs")
    for d in range(2):
        assert np.array_equal(o.get("urhs", d), 2.5 * f[d])
    o.close()


def test_body_force_at_rest_acts_on_the_flow_axis_only():
    o, prm = periodic_case(body_force=0.7)
    set_uniform_density(o, 1.0)
    for d in range(2):
        o.set("u", np.zeros(o.shape()), d)
        o.set("force", np.zeros(o.shape()), d)
    o.stage("rhs")
    assert np.all(o.get("urhs", 0) == 0.7)
    assert np.all(o.get("urhs", 1) == 0.0)
    o.close()
