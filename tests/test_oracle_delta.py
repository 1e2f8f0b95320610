"""Pins for the oracle's delta kernels (Sec. 3.1).

phi1 is Peskin's four-point function (Eq. PhiPeskin): it is defined by
partition of unity, zero first moment and sum of squares 3/8 over the integer
lattice, for every shift r. phi2 (Eq. PhiCosAlternative) keeps the partition
of unity but not the first moment. For the width-w delta of Eq. (Dirac Delta
Approx), the paper states that phi1 satisfies both conditions exactly when
w = z h with z a natural number.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1302_3663_gb300 import workloads as W

RS = np.linspace(-1.0, 1.0, 41)[:-1] + 0.013


def lattice_sums(kind, r):
    j = np.arange(-4, 5)
    v = O.phi(kind, r - j)
    return v.sum(), ((r - j) * v).sum(), (v * v).sum()


@pytest.mark.parametrize("r", RS)
def test_phi1_peskin_conditions(r):
    s0, s1, s2 = lattice_sums(1, r)
    assert abs(s0 - 1.0) < 1e-15
    assert abs(s1) < 1e-15
    assert abs(s2 - 3.0 / 8.0) < 1e-15


@pytest.mark.parametrize("r", RS)
def test_phi2_partition_of_unity(r):
    s0, _, _ = lattice_sums(2, r)
    assert abs(s0 - 1.0) < 1e-15


def test_phi2_first_moment_not_zero():
    # Sec. 3.1: phi2 satisfies the unity condition but not the first-moment one
    m = max(abs(lattice_sums(2, r)[1]) for r in RS)
    assert m > 1e-3


def test_phi_values_and_support():
    assert O.phi(1, 0.0) == 0.5 and O.phi(2, 0.0) == 0.5
    # both branches of phi1 meet at |r| = 1 with value 1/4
    assert abs(O.phi(1, 1.0) - 0.25) < 1e-16
    assert abs(O.phi(1, 1.0 - 1e-12) - 0.25) < 1e-11
    for k in (1, 2):
        assert O.phi(k, 2.0) == 0.0 and O.phi(k, -2.5) == 0.0
        assert abs(O.phi(k, 0.7) - O.phi(k, -0.7)) == 0.0
    assert abs(O.phi(2, 1.0) - 0.25) < 1e-16


def eps_unity_mom(kind, omega, h, samples=64):
    """Eq. (PhiErrorUnity) and Eq. (PhiErrorFirstMomentum) in one dimension."""
    Xs = np.linspace(0.0, h, samples, endpoint=False)
    eu = em = 0.0
    R = int(np.ceil(2 * omega / h)) + 2
    for X in Xs:
        x = np.arange(-R, R + 1) * h
        w = O.phi(kind, (x - X) / omega) / omega * h
        eu = max(eu, abs(w.sum() - 1.0))
        em = max(em, abs(((x - X) * w).sum()))
    return eu, em


@pytest.mark.parametrize("z", [1, 2, 3, 5])
def test_paper_exactness_phi1_omega_multiple_of_h(z):
    # Sec. 3.1: with h = omega / z, eps_unity = eps_mom = 0 for phi1
    omega = 1.0 / 100
    eu, em = eps_unity_mom(1, omega, omega / z, samples=16)
    assert eu < 1e-14 and em < 1e-16


def test_fig2_shape_errors_vanish_faster_than_h2():
    # Fig. 2: both errors fall faster than O(h^2) as h -> 0 (omega = 1/100)
    omega = 1.0 / 100
    hs = [1.0 / 130, 1.0 / 260, 1.0 / 520]  # omega / h not an integer
    for kind in (1, 2):
        e = [eps_unity_mom(kind, omega, h)[0] for h in hs]
        assert e[1] < e[0] / 4 and e[2] < e[1] / 4


def _grid2(n, periodic, h):
    return W.base_params(2, n, periodic, 0, h)


@pytest.mark.parametrize("z", [1, 2])
def test_spread_exact_unity_and_moment_with_phi1(z):
    # Eq. (discrForceCouple) with phi1 and omega = z h: sum_x f h^D equals the
    # spread force and the first moment about the node vanishes, exactly.
    h = 1.0 / 32
    prm = _grid2((32, 32), (1, 1), h)
    prm["phi_kind"] = 1
    o = O.Oracle(prm)
    rng = np.random.default_rng(3)
    X = rng.uniform(0.2, 0.8, size=(5, 2))
    for X1 in X:
        o.set_nodes(X1[None, :])
        for kind, stag in ((O.KIND_CELL, (0.5, 0.5)), (0, (0.0, 0.5)), (1, (0.5, 0.0)),
                           (O.KIND_EDGE[(0, 1)], (0.0, 0.0))):
            f = o.spread_sum(kind, np.array([2.5]), z * h)
            ny, nx = f.shape
            xs = (np.arange(nx) + stag[0]) * h
            ys = (np.arange(ny) + stag[1]) * h
            assert abs(f.sum() * h * h - 2.5) < 1e-13
            assert abs((f * (xs[None, :] - X1[0])).sum() * h * h) < 1e-13
            assert abs((f * (ys[:, None] - X1[1])).sum() * h * h) < 1e-13
