"""Flow-level pins for the oracle's time step (Sec. 3.4, 4.3, 4.4).

* Biofilm-free 2D channel: from half the laminar profile the step converges
  to the exact discrete steady state (Sec. 4.3: exact convergence to the
  second-order polynomial). With the mirror ghost at the walls that state is
  u_j = G/(2 mu) y_j (H - y_j) + G h^2 / (8 mu).
* Biofilm-free 3D square duct: the converged velocity matches the series of
  Eq. (3DlaminarFlow), written out here as the paper prints it, at O(h^2)
  (Sec. 4.4).
* Projection (Eq. NSdis2 - NSdis4): max |D.u^{n+1}| = (eps dt / sigma) max |r_p|
  for any pressure residual r_p.
* Stability in the sense of Sec. 4.3.4: the kinetic energy of a biofilm run
  stays near the biofilm-free value.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1302_3663_gb300 import workloads as W


def no_nodes(o):
    o.set_nodes(np.zeros((0, o.dim)))
    o.set_springs(np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(0), np.zeros(0))


def test_poiseuille_2d_exact_discrete_steady_state():
    # the paper's strongly viscous scaling (sigma = 0.05, Re ~ 0.05, dt = 1e-4)
    n = 32
    prm = W.base_params(2, (2 * n, n), (1, 0), 0, 1.0 / (2 * n), ic_scale=0.5, dt=1e-4,
                        sigma=0.05, inv_re=20.0, mu_f=1.0, vc_visc=12, vc_p=2)
    o = O.Oracle(prm)
    no_nodes(o)
    G, mu, h, H = o.body_force, prm["mu_f"] * prm["inv_re"], prm["h"], n * prm["h"]
    assert abs(G - 8 * mu / H ** 2) < 1e-12
    o.step(60)
    u = o.get("u", 0)[:n, :2 * n]
    y = (np.arange(n) + 0.5) * h
    exact = G / (2 * mu) * y * (H - y) + G * h * h / (8 * mu)
    assert np.abs(u - exact[:, None]).max() < 1e-12
    assert np.abs(o.get("u", 1)).max() < 1e-13


def spiga_double_series(x, y, a, G, mu, N=4001):
    """Eq. (3DlaminarFlow) with kappa = -G: u = 16 G a^2/(mu pi^4) sum_{n,m odd}
    sin(n pi x/a) sin(m pi y/a) / (n m (n^2 + m^2))."""
    k = np.arange(1, N + 1, 2, dtype=np.float64)
    Sx = np.sin(np.outer(k, x) * np.pi / a) / k[:, None]
    Sy = np.sin(np.outer(k, y) * np.pi / a) / k[:, None]
    Wt = 1.0 / (k[:, None] ** 2 + k[None, :] ** 2)
    return 16.0 * G * a * a / (mu * np.pi ** 4) * (Sx.T @ Wt @ Sy)


def test_oracle_single_series_matches_paper_double_series():
    o = O.Oracle(W.base_params(3, (8, 8, 8), (0, 0, 1), 2, 1.0 / 8))
    pts = np.array([0.05, 0.2, 0.5, 0.77, 0.93])
    ref = spiga_double_series(pts, pts, 1.0, 1.0, 1.0)
    got = np.array([[o.laminar_unit(x, y) for y in pts] for x in pts])
    assert np.abs(got - ref).max() < 2e-7


@pytest.mark.slow
def test_duct_3d_second_order_vs_series():
    errs = []
    for n in (8, 16, 32):
        prm = W.base_params(3, (n, n, 8), (0, 0, 1), 2, 1.0 / n, dt=1e-4, sigma=0.05,
                            inv_re=20.0, mu_f=1.0, vc_visc=6, vc_p=1, coarse_sweeps=200)
        o = O.Oracle(prm)
        no_nodes(o)
        o.step(40)
        uz = o.get("u", 2)[:, :n, :n]
        xc = (np.arange(n) + 0.5) / n
        ex = spiga_double_series(xc, xc, 1.0, o.body_force, prm["mu_f"] * prm["inv_re"]).T
        errs.append(np.abs(uz - ex[None, :, :]).max())
        assert np.abs(uz - uz[0:1]).max() < 1e-13   # independent of z
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2.0) < 0.2), (errs, rates)


def test_projection_identity_div_equals_scaled_residual():
    c = W.c1()
    prm = dict(c["params"], sigma=0.05, euler=816.0, dt=2e-3)
    o = O.Oracle(prm)
    o.set_nodes(c["X"])
    o.set_springs(c["ab"], c["rest"], c["K"], c["brk"])
    o.refresh()
    o.stage("rhs")
    o.solve_visc(3)
    o.stage("divergence")
    o.solve_p(1)                      # a deliberately loose pressure solve
    rp = o.residual_p()[:32, :64]
    o.stage("project")
    st = o.stats()
    pred = prm["euler"] * prm["dt"] / prm["sigma"] * np.abs(rp).max()
    assert st["div_max"] > 1e-8
    assert abs(st["div_max"] - pred) < 1e-9 * pred


def test_c1_kinetic_energy_stable():
    c = W.c1()
    o = O.Oracle(c["params"])
    o.set_nodes(c["X"])
    o.set_springs(c["ab"], c["rest"], c["K"], c["brk"])
    ref = O.Oracle(c["params"])
    no_nodes(ref)
    o.step(c["steps"])
    ref.step(c["steps"])
    ke, ke0 = o.stats()["kinetic"], ref.stats()["kinetic"]
    assert 0.5 * ke0 < ke < 1.05 * ke0
    X = o.nodes()
    assert np.all(np.isfinite(X))
    assert np.abs(X - c["X"]).max() > 1e-4      # the biofilm moves with the flow


def test_divergence_target_holds_after_every_projection():
    # the relative-residual test alone (rtol 1e-9) leaves max |D.u| above
    # 1e-10; adding (euler dt / sigma) max |r_p| <= div_tol to the pressure
    # solve's stopping test holds it below div_tol after every projection
    c = W.c1()
    divs = {}
    cyc = {}
    for tol in (0.0, 1e-10):
        prm = dict(c["params"], vc_visc=0, vc_p=0, rtol=1e-9, max_cycles=100, div_tol=tol)
        o = O.Oracle(prm)
        o.set_nodes(c["X"])
        o.set_springs(c["ab"], c["rest"], c["K"], c["brk"])
        divs[tol], cyc[tol] = [], []
        for _ in range(3):
            o.step(1)
            st = o.stats()
            divs[tol].append(st["div_max"])
            cyc[tol].append(st["cycles_p"])
    assert max(divs[0.0]) > 1e-10
    assert max(divs[1e-10]) <= 1e-10
    assert sum(cyc[1e-10]) > sum(cyc[0.0])


def test_divergence_target_holds_with_sigma_and_euler_not_one():
    # the pressure solve's second test scales max |r_p| by euler dt / sigma,
    # the factor of the projection (Eq. NSdis2 - NSdis4); with euler / sigma =
    # 80 a test without it stops too early and leaves max |D.u| above div_tol
    c = W.c1()
    prm = dict(c["params"], vc_visc=0, vc_p=0, rtol=1e-9, max_cycles=100, div_tol=1e-10,
               sigma=0.5, euler=40.0)
    o = O.Oracle(prm)
    o.set_nodes(c["X"])
    o.set_springs(c["ab"], c["rest"], c["K"], c["brk"])
    for _ in range(3):
        o.step(1)
        assert o.stats()["div_max"] <= 1e-10
    o.close()


def test_initial_velocity_is_the_laminar_profile_times_ic_scale():
    # reading 4: u^0 = ic_scale x the laminar profile, whatever the scale
    c = W.c1()
    u = {}
    for scale in (1.0, 0.5):
        o = O.Oracle(dict(c["params"], ic_scale=scale))
        u[scale] = [o.get("u", d) for d in range(2)]
        o.close()
    assert np.abs(u[1.0][0]).max() > 0.0
    for d in range(2):
        assert np.array_equal(u[0.5][d], 0.5 * u[1.0][d])
