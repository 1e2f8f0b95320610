"""Pins for the oracle's Lagrangian-Eulerian transfers and springs.

* Eq. (discrForceCouple): total spread force equals the node force times the
  discrete unity sum; springs obey Newton's third law, so a spring network
  spreads (nearly) zero total force; the three-node example of Fig. 3.
* Spreading and interpolation with the same width are adjoint in the h^D
  inner product, for any positions (including the wall truncation rule).
* Eq. (discrVelCouple) with phi1 and width h reproduces linear fields.
* Eq. (ViscExp): mu = mu_max at a node lying on a grid point (Fig. 4 setup).
* Eq. (springF), Eq. (defineK): two-node tension and the breaking rule.
* A time step's spreads: the density adds the biofilm's mass eta (rho_ratio -
  1) rho_f d0^D exactly (phi1, omega a multiple of h); forces reach 2 omega
  and no further, the viscosity 2 omega_mu; near a wall the kernel beyond it
  is dropped, the same at both walls.
* Sec. 3.4 with Eq. (discrVelCouple): a node moves by dt / sigma times the
  velocity interpolated with the width-h delta (a uniform flow moves it
  exactly; the velocity of faces 1.3h-1.9h away moves it, of faces beyond
  2h does not), and a whole step moves it with the velocity its projection
  leaves, interpolated at the old position; a node carried past a wall stops
  on it and is counted.
* A step's viscosity spread: a node on a cell centre or on a corner sets
  mu_c or mu_e there to mu_max, in 2D and on every grid of 3D; in 3D a spring
  stretched along all three axes pulls along its separation and breaks on
  its whole length.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1302_3663_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def grid2(n=(32, 16), periodic=(1, 0), h=1.0 / 32, **kw):
    return W.base_params(2, n, periodic, 0, h, **kw)


def grid3(n=(8, 8, 16), periodic=(0, 0, 1), h=1.0 / 8, **kw):
    return W.base_params(3, n, periodic, 2, h, **kw)


def coords(o, stag, level=0):
    n, s = o.dims(level)
    h = o.prm["h"] * 2 ** level
    ax = []
    for a in range(o.dim):
        ax.append((np.arange(s[a]) + 0.5 * stag[a]) * h)
    return ax


def inner(o, a, b):
    return float((a * b).sum()) * o.prm["h"] ** o.dim


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("width", ["omega", "h"])
def test_spread_interp_adjoint(dim, width):
    prm = grid2(omega=0.021, omega_mu=0.021) if dim == 2 else grid3(omega=0.2, omega_mu=0.2)
    o = O.Oracle(prm)
    rng = np.random.default_rng(7 + dim)
    L = [prm["n"][a] * prm["h"] for a in range(dim)]
    X = rng.uniform(0, 1, size=(40, dim)) * np.array(L)
    X[:5, 1] = rng.uniform(0, 0.6 * prm["h"], 5)      # hugging the y = 0 wall
    X[5:8, 0] = L[0] - rng.uniform(0, prm["h"], 3)    # near the upper x boundary
    o.set_nodes(X)
    w = prm["omega"] if width == "omega" else prm["h"]
    F = rng.normal(size=40)
    kinds = [0, 1, O.KIND_CELL] + ([2, O.KIND_EDGE[(0, 2)], O.KIND_EDGE[(1, 2)]] if dim == 3 else [])
    kinds.append(O.KIND_EDGE[(0, 1)])
    for kind in kinds:
        u = rng.normal(size=o.shape())
        lhs = inner(o, o.spread_sum(kind, F, w), u)
        rhs = float((F * o.interp(kind, u, w)).sum())
        assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + abs(rhs) + 1e-300) + 1e-15


def test_interp_linear_exact_phi1():
    prm = grid2(n=(32, 32), periodic=(1, 1), phi_kind=1)
    o = O.Oracle(prm)
    rng = np.random.default_rng(1)
    X = rng.uniform(0.2, 0.8, size=(20, 2))
    o.set_nodes(X)
    h = prm["h"]
    for kind, stag in ((0, (0, 1)), (1, (1, 0)), (O.KIND_CELL, (1, 1))):
        xs, ys = coords(o, stag)
        u = 0.3 + 1.7 * xs[None, :] - 0.9 * ys[:, None]
        U = o.interp(kind, u, h)
        assert np.max(np.abs(U - (0.3 + 1.7 * X[:, 0] - 0.9 * X[:, 1]))) < 1e-13


def test_interp_constant_exact_phi2():
    prm = grid2(n=(32, 32), periodic=(1, 1), phi_kind=2)
    o = O.Oracle(prm)
    X = np.random.default_rng(2).uniform(0, 1, size=(20, 2))
    o.set_nodes(X)
    U = o.interp(0, np.full(o.shape(), 2.25), prm["h"])
    assert np.max(np.abs(U - 2.25)) < 1e-14


def test_fig3_three_node_force_example():
    g = json.load(open(os.path.join(GOLD, "fig3_force_example.json")))
    Xs = [eval(e, {"pi": math.pi}) for e in g["X_expr"]]
    F = np.array(g["F"])
    assert abs(F.sum()) == 0.0
    totals = []
    for h in g["h"]:
        n = int(round(1.0 / h))
        prm = grid2(n=(n, n), periodic=(1, 1), h=h, omega=g["omega"])
        o = O.Oracle(prm)
        X = np.array([[x, 0.5] for x in Xs])
        o.set_nodes(X)
        f = o.spread_sum(0, F, g["omega"])
        totals.append(abs(f.sum()) * h * h)
        # the spread force is a sum of three bumps of widths 4 omega
        xs, ys = coords(o, (0, 1))
        assert np.all(f[:, (xs < Xs[0] - 2 * g["omega"]) | (xs > Xs[2] + 2 * g["omega"])] == 0.0)
    # Fig. 3: finer grids represent the node forces more accurately; the total
    # tends to sum F = 0
    assert totals[-1] < 1e-3 * np.abs(F).sum()
    assert totals[-1] < totals[0]


def test_spring_network_spreads_zero_force_phi1_exact():
    # Newton's third law per spring + phi1 unity with omega = 2h: zero net force
    prm = grid2(n=(64, 64), periodic=(1, 1), h=1.0 / 64, phi_kind=1, omega=2.0 / 64,
                omega_mu=2.0 / 64)
    o = O.Oracle(prm)
    rng = np.random.default_rng(5)
    X = rng.uniform(0.3, 0.7, size=(60, 2))
    ab, rest = W.springs_within(X, 0.08)
    o.set_nodes(X + rng.normal(scale=0.003, size=X.shape))
    o.set_springs(ab, rest, np.full(len(rest), 2.0), np.full(len(rest), 5.0))
    o.refresh()
    Fn = o.node_forces()
    assert np.abs(Fn).max() > 1e-4
    assert np.abs(Fn.sum(axis=0)).max() < 1e-14 * np.abs(Fn).sum()
    for d in range(2):
        f = o.get("force", d)
        assert abs(f.sum() * prm["h"] ** 2) < 1e-13 * np.abs(Fn).sum()


def test_fig4_mu_max_at_node_on_grid_point():
    g = json.load(open(os.path.join(GOLD, "fig4_viscosity_example.json")))
    Xs = [eval(e, {"pi": math.pi}) for e in g["X_expr"]]
    for h in g["h"]:
        n = int(round(1.0 / h))
        prm = grid2(n=(n, n // 2), periodic=(1, 0), h=h, omega=g["omega"], omega_mu=g["omega"],
                    mu_ratio=100.0)
        o = O.Oracle(prm)
        y0 = 0.25  # a grid line for every h in the list
        o.set_nodes(np.array([[x, y0] for x in Xs]))
        mu_out, mu_max = prm["mu_f"], prm["mu_f"] * prm["mu_ratio"]
        me = o.spread_max(O.KIND_EDGE[(0, 1)], g["omega"], mu_out, mu_max)
        i, j = int(round(Xs[0] / h)), int(round(y0 / h))
        assert abs(me[j, i] - mu_max) <= 1e-14 * mu_max
        assert me.min() == mu_out and me.max() <= mu_max * (1 + 1e-14)
        mc = o.spread_max(O.KIND_CELL, g["omega"], mu_out, mu_max)
        assert mc.max() < mu_max and mc.min() == mu_out


def two_node(dist, rest, K=3.0, brk=0.5, periodic=(1, 1), n=(32, 32)):
    prm = grid2(n=n, periodic=periodic)
    o = O.Oracle(prm)
    X = np.array([[0.375, 0.5], [0.375 + dist[0], 0.5 + dist[1]]])
    o.set_nodes(X)
    o.set_springs(np.array([[0, 1]]), np.array([rest]), np.array([K]), np.array([brk]))
    o.refresh()
    return o


def test_spring_tension_closed_form():
    d = np.array([0.03, 0.04])  # length 0.05
    o = two_node(d, rest=0.04, K=3.0)
    F = o.node_forces()
    T = 3.0 * (0.05 - 0.04)
    assert np.allclose(F[0], T * d / 0.05, rtol=0, atol=1e-15)
    assert np.allclose(F[1], -T * d / 0.05, rtol=0, atol=1e-15)
    # compressed spring pushes the nodes apart
    o = two_node(d, rest=0.06, K=3.0)
    assert np.dot(o.node_forces()[0], d) < 0


def test_spring_breaks_beyond_threshold_and_stays_broken():
    # Sec. 3.2: springs break when stretched beyond (1 + eps_b) of the rest length
    o = two_node(np.array([0.061, 0.0]), rest=0.04, brk=0.5)  # 1.525 r > 1.5 r
    ids, steps = o.broken()
    assert list(ids) == [0] and list(steps) == [0]
    assert np.all(o.node_forces() == 0.0)
    o.set_nodes(np.array([[0.4, 0.5], [0.44, 0.5]]))   # back to rest: still broken
    o.refresh()
    assert np.all(o.node_forces() == 0.0)
    assert len(o.broken()[0]) == 1
    o2 = two_node(np.array([0.0595, 0.0]), rest=0.04, brk=0.5)
    assert len(o2.broken()[0]) == 0


def test_spring_minimum_image_across_periodic_axis():
    prm = grid2(n=(32, 16), periodic=(1, 0))
    o = O.Oracle(prm)
    X = np.array([[0.99, 0.2], [0.02, 0.2]])       # 0.03 apart through x = 1
    o.set_nodes(X)
    o.set_springs(np.array([[0, 1]]), np.array([0.02]), np.array([1.0]), np.array([1.0]))
    o.refresh()
    F = o.node_forces()
    assert abs(F[0, 0] - 0.01) < 1e-15 and abs(F[1, 0] + 0.01) < 1e-15
    assert len(o.broken()[0]) == 0


def test_paper_break_rule_twice_rest_length():
    # Eq. (defineK): K = F_max / r and eps_b = 1 give tension F_max at 2 r
    Fmax, r = 0.75, 1.0 / 32   # binary-exact, so that |d| is exactly 2 r
    o = two_node(np.array([2 * r, 0.0]), rest=r, K=Fmax / r, brk=1.0)
    assert len(o.broken()[0]) == 0
    assert abs(np.linalg.norm(o.node_forces()[0]) - Fmax) < 1e-14
    o = two_node(np.array([2 * r * (1 + 1e-9), 0.0]), rest=r, K=Fmax / r, brk=1.0)
    assert len(o.broken()[0]) == 1


def test_per_level_gamma_scales_coarse_viscosity():
    # Eq. (ViscCoarseGrid): mu_lh = gamma_lh I(mu_(l/2)h). Restriction is
    # linear, so halving gamma on the grid 2h alone halves mu_c there and on
    # every coarser grid (whose own gamma stays 1).
    inst = W.c2()
    mu = []
    for gl in ([], [0.0, 0.5]):
        prm = dict(inst["params"], gamma_coarse=1.0, gamma_levels=gl)
        o = O.Oracle(prm)
        o.set_nodes(inst["X"])
        o.set_springs(inst["ab"], inst["rest"], inst["K"], inst["brk"])
        o.refresh()
        mu.append([o.get("muc", 0, l) for l in range(3)])
    assert np.array_equal(mu[0][0], mu[1][0])
    for l in (1, 2):
        assert np.max(np.abs(mu[1][l] - 0.5 * mu[0][l])) <= 1e-15 * np.max(np.abs(mu[0][l]))


# --------------------------------------------------------------------------
# The node move of one time step (Sec. 3.4, Eq. discrVelCouple): X += (dt /
# sigma) U, U interpolated from each component's own face grid with the delta
# of width h, whatever the spreading width omega.
def advance_case(ux_of, uy_of, X, sigma=0.5, dt=0.003):
    h = 1.0 / 32
    prm = grid2(h=h, sigma=sigma, dt=dt, omega=0.6 * h, omega_mu=0.6 * h)
    o = O.Oracle(prm)
    o.set_nodes(np.array([X]))
    o.set_springs(np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(0), np.zeros(0))
    n, s = o.dims()
    # x-faces at (i h, (j + 1/2) h), y-faces at ((i + 1/2) h, j h)
    xi, yj = np.meshgrid(np.arange(s[0]) * h, (np.arange(s[1]) + 0.5) * h)
    xc, yf = np.meshgrid((np.arange(s[0]) + 0.5) * h, np.arange(s[1]) * h)
    o.set("u", ux_of(xi, yj), 0)
    o.set("u", uy_of(xc, yf), 1)
    o.stage("interp_advance")
    dX = o.nodes()[0] - np.asarray(X)
    o.close()
    return dX, h, dt / sigma


def test_node_moves_by_dt_over_sigma_in_a_uniform_flow():
    # partition of unity: any delta of unit mass returns the uniform velocity
    # (the node sits 8 cells from both walls, so no wall face is in reach)
    U0, V0 = 0.3, -0.2
    dX, h, c = advance_case(lambda x, y: np.full_like(x, U0),
                            lambda x, y: np.where((y > 0) & (y < 0.5), V0, 0.0),
                            (0.41 + 0.3 / 32, 0.25 + 0.2 / 32))
    assert np.allclose(dX, [c * U0, c * V0], rtol=0, atol=1e-15)


def test_node_velocity_uses_the_width_h_support():
    # the delta of width h reaches faces closer than 2h along x and no
    # further: x-velocity on the faces 1.3h-1.9h from the node moves it, and
    # on the faces beyond 2.05h does not (a delta of the spreading width
    # 0.6h would miss the first band)
    X = (0.41 + 0.3 / 32, 0.25 + 0.2 / 32)
    h = 1.0 / 32

    def band(lo, hi):
        return lambda x, y: np.where((np.abs(x - X[0]) > lo * h) & (np.abs(x - X[0]) < hi * h),
                                     1.0, 0.0)

    zero = lambda x, y: np.zeros_like(x)   # noqa: E731
    dX, _, c = advance_case(band(1.3, 1.9), zero, X)
    assert dX[0] > 1e-3 * c and dX[1] == 0.0
    dX, _, _ = advance_case(band(2.05, 100.0), zero, X)
    assert dX[0] == 0.0 and dX[1] == 0.0


# --------------------------------------------------------------------------
# A time step's spreads (Eqs. discrForceCouple, discrDensCouple, ViscExp, with
# the widths of Sec. 3.1): forces and density with omega, viscosity with
# omega_mu; the biofilm's density rho_b = (rho_ratio - 1) rho_f on d0^D.
H32 = 1.0 / 32


def refreshed(**kw):
    h = H32
    prm = grid2(n=(32, 32), periodic=(1, 0), h=h, **kw)
    o = O.Oracle(prm)
    A = np.array([0.5 + 0.3 * h, 0.3 + 0.15 * h])
    B = np.array([0.5 + 0.3 * h, 0.7 + 0.15 * h])   # 12.8 h away along y
    o.set_nodes(np.array([A, B]))
    # a stretched spring: a force of 3 (0.4 - 0.1) along y on each node
    o.set_springs(np.array([[0, 1]]), np.array([0.1]), np.array([3.0]), np.array([100.0]))
    o.refresh()
    return o, prm, A, h


def near_a(o, A, h, stag):
    n, s = o.dims()
    x = (np.arange(s[0]) + 0.5 * stag[0]) * h - A[0]
    y = (np.arange(s[1]) + 0.5 * stag[1]) * h - A[1]
    return np.meshgrid(np.abs(x), np.abs(y))


def test_density_spread_adds_the_biofilm_mass():
    # with phi1 and omega a multiple of h the discrete unity sum is exact:
    # sum over each face grid of (rho_d - rho_f) h^2 = eta rho_b d0^2
    o, prm, A, h = refreshed(phi_kind=1, omega=2 * H32, omega_mu=2 * H32, rho_ratio=2.5,
                             d0_vol=0.7 * H32 * H32)
    mass = 2 * (2.5 - 1.0) * prm["rho_f"] * prm["d0_vol"]
    for d in range(2):
        added = (o.get("rho", d) - prm["rho_f"]).sum() * h * h
        assert abs(added - mass) <= 1e-13 * mass, (d, added, mass)
    o.close()


def test_forces_spread_with_omega_and_viscosity_with_omega_mu():
    # omega = 2h: the force on A reaches y-faces 2.2h-3.8h away along x and
    # nothing 4h or more away; omega_mu = h: the viscosity rises only within
    # 2h of a node, so cells 2.2h-3.8h away along x keep mu_f exactly
    o, prm, A, h = refreshed(omega=2 * H32, omega_mu=H32, mu_ratio=10.0)
    fy = o.get("force", 1)
    dx, dy = near_a(o, A, h, (1, 0))
    band = (dx > 2.2 * h) & (dx < 3.8 * h) & (dy < h)
    assert np.abs(fy[band]).max() > 0.0
    assert np.all(fy[(dx >= 4 * h) & (dy < 5 * h)] == 0.0)
    mc = o.get("muc")
    dx, dy = near_a(o, A, h, (1, 1))
    assert mc[(dx < 0.5 * h) & (dy < 0.5 * h)].min() > prm["mu_f"]
    assert np.all(mc[(dx > 2.2 * h) & (dx < 3.8 * h) & (dy < h)] == prm["mu_f"])
    o.close()


def test_a_step_moves_the_nodes_with_its_projected_velocity():
    # Sec. 3.4's order: the nodes move with u^{n+1}, the velocity the step's
    # projection leaves, interpolated at X^n (the c1 mound: its density and
    # viscosity change the flow within the step, so u^{n+1} != u^n)
    inst = W.c1()
    o = O.Oracle(inst["params"])
    o.set_nodes(inst["X"])
    o.set_springs(inst["ab"], inst["rest"], inst["K"], inst["brk"])
    o.step(1)
    u_before = [o.get("u", d) for d in range(2)]
    X0 = o.nodes()
    o.step(1)
    u1 = [o.get("u", d) for d in range(2)]
    assert max(np.abs(a - b).max() for a, b in zip(u1, u_before)) > 1e-6
    prm = inst["params"]
    at_x0 = O.Oracle(prm)   # the interpolation evaluates at an instance's own nodes
    at_x0.set_nodes(X0)
    for d in range(2):
        step = prm["dt"] / prm["sigma"] * at_x0.interp(O.KIND_FACE[d], u1[d], prm["h"])
        moved = o.nodes()[:, d] - X0[:, d]
        Lx = prm["n"][d] * prm["h"]
        if prm["periodic"][d]:   # across the periodic seam
            moved = (moved + 0.5 * Lx) % Lx - 0.5 * Lx
        assert np.allclose(moved, step, rtol=0, atol=1e-15), d
    at_x0.close()
    o.close()


def test_spreads_drop_the_kernel_beyond_a_wall():
    # grid points beyond a wall do not exist: a node 0.3h from the bottom wall
    # loses the kernel mass beyond it, and by the grid's mirror symmetry a
    # node 0.3h from the top wall loses the same (phi1, omega = 2h, where a
    # node away from the walls adds the whole mass)
    h = H32
    prm = grid2(n=(32, 32), periodic=(1, 0), h=h, phi_kind=1, omega=2 * h, omega_mu=2 * h,
                rho_ratio=2.5, d0_vol=0.7 * h * h)
    full = (2.5 - 1.0) * prm["rho_f"] * prm["d0_vol"]
    added = {}
    for where, Y in (("bottom", 0.3 * h), ("top", 1.0 - 0.3 * h)):
        o = O.Oracle(prm)
        o.set_nodes(np.array([[0.5 + 0.3 * h, Y]]))
        o.set_springs(np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(0), np.zeros(0))
        o.refresh()
        added[where] = [(o.get("rho", d) - prm["rho_f"]).sum() * h * h for d in range(2)]
        o.close()
    for d in range(2):
        assert abs(added["bottom"][d] - added["top"][d]) <= 1e-13 * full, d
        assert added["bottom"][d] < 0.9 * full, d


def test_a_step_spreads_viscosity_on_centres_and_edges():
    # Eq. ViscExp at a node on a grid point of a kind gives mu_max there: a
    # node on a cell centre sets mu_c there to mu_max, a node on a corner
    # (the 2D edge grid) sets mu_e there to mu_max
    h = H32
    for kind, X, field in (("centre", (16.5 * h, 9.5 * h), "muc"), ("edge", (16 * h, 9 * h), "mue")):
        prm = grid2(n=(32, 32), periodic=(1, 0), h=h, omega=1.5 * h, omega_mu=1.5 * h,
                    mu_ratio=50.0)
        o = O.Oracle(prm)
        o.set_nodes(np.array([X]))
        o.set_springs(np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(0), np.zeros(0))
        o.refresh()
        mu = o.get(field, 0)
        mu_max = prm["mu_f"] * prm["mu_ratio"]
        assert abs(mu[9, 16] - mu_max) <= 1e-13 * mu_max, kind
        o.close()


def test_a_node_leaving_through_a_wall_is_clamped_onto_it_and_counted():
    # a strong flow into the bottom wall would carry the node 0.2h from it
    # past the wall: it stops on the wall, and the step counts it
    h = 1.0 / 32
    prm = grid2(h=h, sigma=0.5, dt=0.003, omega=0.6 * h, omega_mu=0.6 * h)
    o = O.Oracle(prm)
    X = np.array([[0.5 + 0.3 * h, 0.2 * h]])
    o.set_nodes(X)
    o.set_springs(np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(0), np.zeros(0))
    n, s = o.dims()
    o.set("u", np.zeros(o.shape()), 0)
    vy = np.full(o.shape(), -10.0)
    vy[0, :] = 0.0     # the wall faces
    vy[n[1]:, :] = 0.0
    o.set("u", vy, 1)
    o.stage("interp_advance")
    Y = o.nodes()[0]
    assert Y[0] == X[0, 0] and Y[1] == 0.0
    assert o.stats()["clamped_total"] == 1
    o.close()


def test_spring_tension_and_break_in_3d():
    # a spring stretched along every axis of a 3D grid: the tension of Eq.
    # (springF) along the separation, and a break once the whole length
    # passes (1 + eps_b) r, whatever axis carries the stretch
    prm = grid3()
    d = np.array([0.02, 0.03, 0.06])   # length 0.07
    for rest, brk, broken in ((0.05, 1.0, False), (0.05, 0.3, True)):
        o = O.Oracle(prm)
        X = np.array([[0.4, 0.45, 0.5], [0.4, 0.45, 0.5] + d])
        o.set_nodes(X)
        o.set_springs(np.array([[0, 1]]), np.array([rest]), np.array([2.0]), np.array([brk]))
        o.refresh()
        F = o.node_forces()
        if broken:   # 0.07 > 1.3 * 0.05
            assert len(o.broken()[0]) == 1 and np.all(F == 0.0)
        else:
            T = 2.0 * (0.07 - rest)
            assert np.allclose(F[0], T * d / 0.07, rtol=0, atol=1e-15)
            assert np.allclose(F[1], -T * d / 0.07, rtol=0, atol=1e-15)
        o.close()


def test_a_step_spreads_viscosity_on_every_3d_grid():
    # Eq. ViscExp in 3D: a node on a point of the centre grid or of one of
    # the three edge grids sets mu there to mu_max
    h = 1.0 / 8
    mu_max = 0.01 * 50.0
    # grid point (i, j, k) of each kind: coordinates i h + s_x h / 2 per axis
    kinds = {"muc": (None, (1, 1, 1)), "mue_xy": (0, (0, 0, 1)), "mue_xz": (1, (0, 1, 0)),
             "mue_yz": (2, (1, 0, 0))}
    for name, (e, stag) in kinds.items():
        prm = grid3(h=h, omega=1.5 * h, omega_mu=1.5 * h, mu_ratio=50.0)
        o = O.Oracle(prm)
        ijk = (4, 3, 8)
        X = [(ijk[a] + 0.5 * stag[a]) * h for a in range(3)]
        o.set_nodes(np.array([X]))
        o.set_springs(np.zeros((0, 2), np.int32), np.zeros(0), np.zeros(0), np.zeros(0))
        o.refresh()
        mu = o.get("muc") if e is None else o.get("mue", e)
        assert abs(mu[ijk[2], ijk[1], ijk[0]] - mu_max) <= 1e-13 * mu_max, name
        o.close()
