"""The seeded input generators: deterministic, and shaped as the workloads are defined."""
import numpy as np
from scipy.spatial import cKDTree

from paper_1302_3663_gb300 import workloads as W


def test_c1_deterministic_and_spaced():
    a, b = W.c1(), W.c1()
    assert np.array_equal(a["X"], b["X"]) and np.array_equal(a["ab"], b["ab"])
    X = a["X"]
    assert X.shape == (150, 2)
    assert np.all(X[:, 1] >= 0) and np.all(np.hypot(X[:, 0] - 0.5, X[:, 1]) < 0.1)
    d, _ = cKDTree(X).query(X, k=2)
    assert d[:, 1].min() >= a["spacing"] * (1 - 1e-12)
    r = a["params"]["omega"]
    assert np.all(a["rest"] < 2.5 * r) and np.all(a["K"] == 1.0) and np.all(a["brk"] == 0.5)
    assert np.allclose(np.linalg.norm(X[a["ab"][:, 1]] - X[a["ab"][:, 0]], axis=1), a["rest"])


def test_c2_shape():
    c = W.c2()
    X = c["X"]
    assert X.shape == (2000, 3) and c["params"]["n"] == [64, 64, 64]
    assert np.all(c["K"] >= 0.1) and np.all(c["K"] <= 10.0)
    assert np.all(np.linalg.norm(X - [0.5, 0.0, 0.5], axis=1) < 0.15)


def test_c3_shape():
    c = W.c3()
    assert c["X"].shape == (20000, 3) and c["params"]["n"] == [128, 128, 256]
    assert np.all(c["X"] >= 0) and np.all(c["X"][:, 2] <= 2.0)
    assert 100000 < c["ab"].shape[0] < 300000


def test_c4_c5_draws():
    for i in (0, 5):
        inst = W.c4_instance(i)
        e = inst["params"]["n"][0]
        assert e in (32, 48, 64, 96) and inst["params"]["n"][2] == 2 * e
        assert 500 <= inst["X"].shape[0] <= 8000
    req = W.c5_request(3)
    e = req["params"]["n"][0]
    assert 48 <= e <= 160 and e % 16 == 0
    t = W.c5_arrivals()
    assert t.shape == (128,) and np.all(np.diff(t) > 0)
    assert 15 < t[-1] < 50   # mean gap 0.25 s


def test_paper_units_duct():
    # the paper's scaling table: sigma = L / (T u0), Euler = dp / (rho0 u0^2),
    # Re = rho0 u0 L / mu; springs K = F_max / r breaking at 2 r (Eq. defineK)
    inst = W.paper_units_duct(e=32, nodes=600, f_max=0.5)
    p = inst["params"]
    assert abs(p["sigma"] - 0.05) < 1e-15
    assert abs(p["euler"] - 816.0320641282565) < 1e-9
    assert abs(1.0 / p["inv_re"] - 0.0499) < 1e-15
    assert np.allclose(inst["K"] * inst["rest"], 0.5) and np.all(inst["brk"] == 1.0)
    assert abs(p["dt"] - 0.1 / 32 * 0.05) < 1e-18


def test_paper_units_duct_stable_in_the_oracle():
    # kinetic energy without extreme growth (the stability notion of Sec. 4.3.4)
    from oracle.oracle import Oracle
    inst = W.paper_units_duct(e=32, nodes=600)
    o = Oracle(inst["params"], omp=True)
    o.set_nodes(inst["X"])
    o.set_springs(inst["ab"], inst["rest"], inst["K"], inst["brk"])
    ke = []
    for _ in range(8):
        o.step(1)
        ke.append(o.stats()["kinetic"])
    assert max(ke) < 1.1 * ke[0] and min(ke) > 0.8 * ke[0]
