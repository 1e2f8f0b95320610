"""GPU parity, stage by stage: the CUDA library (through its C ABI) against
the FP64 oracle on the same seeded inputs. Sizes span several thread blocks
and spread tiles and end in ragged tails; the 3D duct coarsens to odd
extents."""
import numpy as np
import pytest

from paper_1302_3663_gb300 import workloads as W

from helpers import assert_close, cell_mask, face_mask, pair, random_coefficients

pytestmark = pytest.mark.gpu

TOL = 1e-12   # one stage: differences come only from rounding order


def ragged_duct(seed=11, nodes=600):
    """24x20x40 duct (walls in x, y; periodic z), nodes near the y = 0 wall."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 1.0 / 24
    prm = W.base_params(3, (24, 20, 40), (0, 0, 1), 2, h, rho_ratio=1.7, mu_ratio=300.0,
                        omega=0.7 * h, omega_mu=0.7 * h, d0_vol=(0.6 * h) ** 3)
    X = np.column_stack([rng.uniform(0.2, 0.8, nodes), np.abs(rng.normal(0, 0.12, nodes)),
                         rng.uniform(0, 40 * h, nodes)])
    if nodes >= 20:
        X[:10, 1] = 0.0                             # on the wall
        X[10:20, 0] = rng.uniform(0, 0.3 * h, 10)   # hugging the x = 0 wall
    X[:, 1] = np.minimum(X[:, 1], 20 * h)
    X[:, 2] = np.mod(X[:, 2], 40 * h)
    ab, rest = W.springs_within(X, 2.5 * prm["omega"])
    m = ab.shape[0]
    return dict(name="ragged", params=prm, X=X, ab=ab, rest=rest,
                K=np.exp(rng.uniform(np.log(0.1), np.log(10), m)), brk=np.full(m, 0.3), steps=10)


CASES = {"c1": W.c1, "ragged": ragged_duct, "c2": W.c2}


@pytest.fixture(scope="module", params=list(CASES))
def inst(request):
    return CASES[request.param]()


def test_laminar_initial_condition(inst):
    g, o = pair(inst)
    assert abs(g.body_force - o.body_force) <= 1e-14 * abs(o.body_force)
    fa = inst["params"]["flow_axis"]
    assert_close(g.get_field("u", fa), o.get("u", fa), 1e-14, "u flow")


def test_refresh_spread_and_coefficients(inst):
    # move the nodes off their rest configuration so that springs pull
    rng = np.random.default_rng(4)
    X = inst["X"] + rng.normal(scale=0.1 * inst["params"]["omega"], size=inst["X"].shape)
    prm = inst["params"]
    for a in range(prm["dim"]):
        L = prm["n"][a] * prm["h"]
        X[:, a] = np.mod(X[:, a], L) if prm["periodic"][a] else np.clip(X[:, a], 0.0, L)
    inst = dict(inst, X=X)
    g, o = pair(inst)
    g.refresh()
    o.refresh()
    D = g.dim
    assert_close(g.get_node_forces(), o.node_forces(), TOL, "node forces")
    for d in range(D):
        assert_close(g.get_field("force", d), o.get("force", d), TOL, "force %d" % d)
        assert_close(g.get_field("rho", d), o.get("rho", d), TOL, "rho %d" % d)
    for l in range(g.levels):
        assert_close(g.get_field("muc", 0, l), o.get("muc", 0, l), TOL, "muc L%d" % l)
        for e in range(3 if D == 3 else 1):
            assert_close(g.get_field("mue", e, l), o.get("mue", e, l), TOL, "mue L%d" % l)
        for d in range(D):
            assert_close(g.get_field("beta", d, l), o.get("beta", d, l), TOL, "beta L%d" % l)
            assert_close(g.get_field("m", d, l), o.get("m", d, l), TOL, "m L%d" % l)
    # the spread did something
    assert np.abs(o.get("force", 0)).max() > 0 or len(inst["ab"]) == 0
    assert o.get("muc").max() > inst["params"]["mu_f"] * 1.5


@pytest.mark.parametrize("level", [0, 1])
def test_pressure_smoother_and_residual(inst, level):
    g, o = pair(inst, load=False)
    rng = np.random.default_rng(5)
    random_coefficients(g, o, rng)
    cm = cell_mask(g, level)
    for which in ("p", "prhs"):
        a = np.where(cm, rng.normal(size=g.shape(level)), 0.0)
        g.set_field(which, a, 0, level)
        o.set(which, a, 0, level)
    assert_close(g.residual_pressure(level), o.residual_p(level), TOL, "pressure residual")
    g.smooth_pressure(level, 3)   # odd: the out-of-place sweep copies back
    for _ in range(3):
        o.rbgs_p(level)
    assert_close(g.get_field("p", 0, level), o.get("p", 0, level), TOL, "p after 3 sweeps")


@pytest.mark.parametrize("level", [0, 1])
def test_viscous_smoother_and_residual(inst, level):
    g, o = pair(inst, load=False)
    rng = np.random.default_rng(6)
    random_coefficients(g, o, rng)
    for d in range(g.dim):
        fm = face_mask(g, d, level)
        for which in ("ut", "urhs"):
            a = np.where(fm, rng.normal(size=g.shape(level)), 0.0)
            g.set_field(which, a, d, level)
            o.set(which, a, d, level)
    rg = g.residual_viscous(level)
    ro = o.residual_visc(level)
    for d in range(g.dim):
        assert_close(rg[d], ro[d], TOL, "viscous residual %d" % d)
    g.smooth_viscous(level, 3)
    for _ in range(3):
        o.rbgs_visc(level)
    for d in range(g.dim):
        assert_close(g.get_field("ut", d, level), o.get("ut", d, level), TOL, "u~ %d" % d)


def test_fused_and_two_kernel_sweeps_agree(inst):
    from paper_1302_3663_gb300 import bfibm
    a, o = pair(inst)
    b = bfibm.load_instance(inst)
    b.set_option(bfibm.OPT_FUSED, 0)
    a.step(3)
    b.step(3)
    for d in range(a.dim):
        assert_close(a.get_velocity(d), b.get_velocity(d), 1e-12, "u%d fused vs two-kernel" % d)
    assert_close(a.get_pressure(), b.get_pressure(), 1e-12, "p fused vs two-kernel")


def test_multigrid_solves_fixed_cycles(inst):
    g, o = pair(inst, load=False)
    rng = np.random.default_rng(7)
    random_coefficients(g, o, rng, mu_ratio=100.0)
    cm = cell_mask(g)
    b = np.where(cm, rng.normal(size=g.shape()), 0.0)
    b[cm] -= b[cm].mean()
    for c in (g,):
        c.set_field("prhs", b)
        c.set_field("p", np.zeros(g.shape()))
    o.set("prhs", b)
    o.set("p", np.zeros(g.shape()))
    assert g.solve_pressure(3) == 3
    o.solve_p(3)
    assert_close(g.get_field("p"), o.get("p"), 1e-11, "p after 3 V-cycles")
    for d in range(g.dim):
        f = np.where(face_mask(g, d), rng.normal(size=g.shape()), 0.0)
        g.set_field("urhs", f, d)
        o.set("urhs", f, d)
        g.set_field("ut", np.zeros(g.shape()), d)
        o.set("ut", np.zeros(g.shape()), d)
    g.solve_viscous(3)
    o.solve_visc(3)
    for d in range(g.dim):
        assert_close(g.get_field("ut", d), o.get("ut", d), 1e-11, "u~ %d after 3 V-cycles" % d)


def test_rhs_divergence_project(inst):
    g, o = pair(inst)
    g.refresh()
    o.refresh()
    rng = np.random.default_rng(8)
    for d in range(g.dim):   # a non-trivial velocity (zero on the walls)
        u = np.where(face_mask(g, d), o.get("u", d) + 0.1 * rng.normal(size=g.shape()), 0.0)
        g.set_velocity(d, u)
        o.set("u", u, d)
    g.stage("rhs")
    o.stage("rhs")
    for d in range(g.dim):
        assert_close(g.get_field("urhs", d), o.get("urhs", d), TOL, "rhs %d" % d)
        assert_close(g.get_field("ut", d), o.get("ut", d), 0.0, "u~ init %d" % d)
    g.stage("divergence")
    o.stage("divergence")
    assert_close(g.get_field("prhs"), o.get("prhs"), TOL, "divergence rhs")
    p = np.where(cell_mask(g), rng.normal(size=g.shape()), 0.0)
    g.set_field("p", p)
    o.set("p", p)
    g.stage("project")
    o.stage("project")
    for d in range(g.dim):
        assert_close(g.get_field("u", d), o.get("u", d), TOL, "projected u %d" % d)


def test_interp_advance(inst):
    g, o = pair(inst)
    rng = np.random.default_rng(9)
    for d in range(g.dim):
        u = np.where(face_mask(g, d), rng.normal(size=g.shape()), 0.0)
        g.set_velocity(d, u)
        o.set("u", u, d)
    g.stage("interp_advance")
    o.stage("interp_advance")
    Xg, Xo = g.get_nodes(), o.nodes()
    assert np.abs(Xg - Xo).max() <= 1e-14
