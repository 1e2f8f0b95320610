"""Refinement studies (Sec. 4.3.2-4.3.3): the face restriction I_h^2h against
closed forms, and the empirical convergence rates of a smooth flow in time
and in space on the oracle (first order in time for the semi-implicit step,
second order in space for the MAC discretisation); on the GPU the same study
through the C ABI must give the oracle's errors and rates."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1302_3663_gb300 import refinement as R, workloads as W


class oracle_backend:
    """The FP64 oracle behind the three methods the refinement harness calls."""

    def __init__(self, inst, prm):
        self.o = O.Oracle(prm, omp=True)
        self.dim = prm["dim"]
        self.o.set_nodes(inst["X"])
        self.o.set_springs(inst["ab"], inst["rest"], inst["K"], inst["brk"])

    def step(self, n):
        self.o.step(n)

    def velocity(self):
        return [self.o.get("u", d) for d in range(self.dim)]

    def nodes(self):
        return self.o.nodes()

    def close(self):
        pass


SOLVER = {"vc_visc": 0, "vc_p": 0, "rtol": 1e-12, "max_cycles": 300, "precision": 0}


spin_up = W.spin_up_channel


def face_centres(n, h, d, dim, per):
    """Coordinates of the stored entries of face component d, array order
    (z, y, x) / (y, x); wall axes carry one extra entry (the wall face on the
    own axis, a pad across)."""
    ax = []
    for a in range(dim):
        m = n[a] + (0 if per[a] else 1)
        i = np.arange(m, dtype=np.float64)
        ax.append(i * h if a == d else (i + 0.5) * h)
    grids = np.meshgrid(*ax[::-1], indexing="ij")
    return grids[::-1]   # x, y (, z)


@pytest.mark.parametrize("dim", [2, 3])
def test_restriction_reproduces_linear_fields_between_walls(dim):
    n = [8, 6, 4][:dim]
    per = [0] * dim
    h = 0.125
    coef = [0.7, -1.3, 0.4][:dim]
    for d in range(dim):
        xf = face_centres(n, h, d, dim, per)
        xc = face_centres([m // 2 for m in n], 2 * h, d, dim, per)
        f = 0.3 + sum(c * x for c, x in zip(coef, xf))
        want = 0.3 + sum(c * x for c, x in zip(coef, xc))
        got = R.restrict_face(f, d, dim, per)
        assert got.shape == want.shape
        # interior coarse faces; wall faces hold 0 and pads are never read
        sl = [slice(None)] * dim
        for a in range(dim):
            k = dim - 1 - a
            nc = n[a] // 2
            sl[k] = slice(1, nc) if a == d else slice(0, nc)
        np.testing.assert_allclose(got[tuple(sl)], want[tuple(sl)], rtol=0, atol=1e-13)
        own = dim - 1 - d
        assert np.all(np.take(got, [0, n[d] // 2], axis=own) == 0.0)


def test_restriction_of_a_periodic_wave():
    # along the own periodic axis (1/4, 1/2, 1/4) scales cos(k x) by
    # (1 + cos(k h)) / 2; across a periodic axis the two-child mean scales it
    # by cos(k h / 2)
    n, h = [16, 8], 1.0 / 16
    per = [1, 1]
    kx, ky = 2 * np.pi * 2 / (n[0] * h), 2 * np.pi / (n[1] * h)
    for d in range(2):
        xf, yf = face_centres(n, h, d, 2, per)
        xc, yc = face_centres([8, 4], 2 * h, d, 2, per)
        f = np.cos(kx * xf) * np.cos(ky * yf)
        gx = (1 + np.cos(kx * h)) / 2 if d == 0 else np.cos(kx * h / 2)
        gy = (1 + np.cos(ky * h)) / 2 if d == 1 else np.cos(ky * h / 2)
        want = gx * gy * np.cos(kx * xc) * np.cos(ky * yc)
        np.testing.assert_allclose(R.restrict_face(f, d, 2, per), want, rtol=0, atol=1e-14)


def test_temporal_rate_of_the_spin_up_is_first_order():
    r = R.temporal_rates(spin_up(32), T=0.02, dt0=2e-3, nruns=4, backend=oracle_backend,
                         solver=SOLVER)
    e = [x["u_2"] for x in r["errors"]]
    assert e[0] > e[1] > e[2] > 0
    for x in r["rates"]:
        assert 0.85 <= x["u_2"] <= 1.15, r["rates"]
        assert np.isnan(x["X_2"])   # no nodes: no node error


def test_spatial_rate_of_the_spin_up_is_second_order():
    r = R.spatial_rates(spin_up, [16, 32, 64], T=0.02, dt=1e-3, backend=oracle_backend,
                        solver=SOLVER)
    (x,) = r["rates"]
    assert 1.8 <= x["u_2"] <= 2.2, r["rates"]
    assert 1.6 <= x["u_inf"] <= 2.2, r["rates"]


def test_mound_converges_under_grid_refinement():
    """The mound with the same nodes on every grid (Sec. 4.3.3): the errors in
    u and X fall as h halves, at least first order in X for the L2 norm, as
    in the paper's constant-coefficient refinement table."""
    r = R.spatial_rates(W.mound_2d, [16, 32, 64, 128], T=0.01, dt=1e-4,
                        backend=oracle_backend, solver=SOLVER)
    e = r["errors"]
    for a, b in zip(e[:-1], e[1:]):
        assert b["u_2"] < a["u_2"] and b["X_2"] < a["X_2"], e
    for x in r["rates"]:
        assert 1.0 <= x["X_2"] <= 2.5, r["rates"]


def _same_study(a, b, rel):
    for ea, eb in zip(a["errors"], b["errors"]):
        for k in ("u_2", "u_inf", "X_2", "X_inf"):
            assert abs(ea[k] - eb[k]) <= rel * max(abs(eb[k]), 1e-300), (k, ea[k], eb[k])


@pytest.mark.gpu
def test_gpu_temporal_study_matches_the_oracle():
    """Biofilm c1 (nodes and springs, 2D) over a few steps: the errors between
    successive time-step halvings on the GPU equal the oracle's."""
    inst = W.c1()
    args = dict(T=0.004, dt0=2e-3, nruns=3, solver=SOLVER)
    g = R.temporal_rates(inst, backend=R.gpu_backend, **args)
    o = R.temporal_rates(inst, backend=oracle_backend, **args)
    _same_study(g, o, 1e-6)


@pytest.mark.gpu
def test_gpu_spatial_study_matches_the_oracle():
    args = dict(ns=[16, 32, 64], T=0.01, dt=1e-3, solver=SOLVER)
    g = R.spatial_rates(spin_up, backend=R.gpu_backend, **args)
    o = R.spatial_rates(spin_up, backend=oracle_backend, **args)
    _same_study(g, o, 1e-6)
    assert abs(g["rates"][0]["u_2"] - o["rates"][0]["u_2"]) <= 1e-6
