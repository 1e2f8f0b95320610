"""Seeded synthetic workloads shaped like the paper's biofilm runs.

This module only draws inputs: node positions, spring lists and parameter
sets. It holds none of the method's arithmetic (no delta kernel, no operator,
no laminar profile); both the CUDA library and the CPU oracle read exactly
what it returns.

The paper's own runs use measured S. epidermidis cell coordinates (Sec. 4.2),
which are not available; seeded mounds stand in for them:

* ``c1``  2D, 64x32 cells on [0,1]x[0,0.5], periodic in x, walls in y; 150
  nodes dart-thrown in a half-disc of radius 0.1 on the bottom wall.
* ``c2``  3D, 64^3 square duct of side 1, walls in x and y, periodic in z;
  2,000 dart-thrown nodes in a hemisphere of radius 0.15 on the y = 0 wall.
* ``c3``  3D, 128x128x256 duct (side 1, length 2); 20,000 nodes in three
  Gaussian mounds (sigma 0.05) on the y = 0 wall.
* ``c4``  64 independent ducts with edges drawn from {32, 48, 64, 96}
  (length twice the edge), 500-8,000 nodes uniform in a hemisphere.
* ``c5``  a Poisson arrival stream (mean 4 per second) of ducts with edges
  48..160 and 500-50,000 nodes in three Gaussian mounds.

Dart throwing keeps candidates at least ``spacing`` apart. When the requested
count cannot fit, the spacing shrinks by 0.9 until it can; spacings whose
hexagonal packing bound is already below the count are skipped without
sampling. Springs join every pair closer than 2.5 r, with rest length equal to
the initial distance.
"""
import math

import numpy as np

PHI_COSINE = 2
PHI_PESKIN = 1


def base_params(dim, n, periodic, flow_axis, h, **kw):
    """Parameter set with the defaults used throughout (model units: sigma =
    Euler number = 1/Re = c_f = 1; mu carries the fluid viscosity)."""
    n = list(n) + [1] * (3 - len(n))
    periodic = list(periodic) + [1] * (3 - len(periodic))
    prm = dict(dim=dim, n=n, periodic=periodic, flow_axis=flow_axis, phi_kind=PHI_COSINE,
               mg_levels_max=6, nu1=2, nu2=2, vc_visc=3, vc_p=3, max_cycles=60,
               coarse_sweeps=16, h=float(h), rho_f=1.0, mu_f=0.01, rho_ratio=1.0,
               mu_ratio=1.0, omega=2.0 * h, omega_mu=2.0 * h, d0_vol=h ** dim,
               dt=0.1 * h, sigma=1.0, euler=1.0, inv_re=1.0, c_force=1.0, body_force=0.0,
               u_center=1.0, ic_scale=1.0, rtol=1e-9, gamma_coarse=1.0, precision=0)
    prm.update(kw)
    return prm


# ---------------------------------------------------------------------------
# samplers
# ---------------------------------------------------------------------------
def _hemisphere_points(rng, m, center, R, dim):
    """m uniform points in the half-ball of radius R on the y = center[1] wall."""
    out = np.empty((0, dim))
    while out.shape[0] < m:
        c = rng.uniform(-R, R, size=(2 * m + 16, dim))
        c[:, 1] = np.abs(c[:, 1])
        c = c[np.sum(c * c, axis=1) < R * R]
        out = np.vstack([out, c + np.asarray(center)[None, :dim]])
    return out[:m]


def _pack_bound(volume, spacing, dim):
    """Largest count of points pairwise >= spacing apart a dense packing allows."""
    if dim == 2:
        return volume / (math.sqrt(3.0) / 2.0 * spacing ** 2)
    return volume / (spacing ** 3 / math.sqrt(2.0))


def dart_throw(rng, count, dim, center, R, spacing, attempts_per_node=30):
    """Seeded Poisson-disc sampling of ``count`` points in a half-ball.

    Returns (points, spacing actually used)."""
    volume = (math.pi * R * R / 2.0) if dim == 2 else (2.0 / 3.0 * math.pi * R ** 3)
    while _pack_bound(volume, spacing, dim) < count:
        spacing *= 0.9
    while True:
        cell = spacing / math.sqrt(dim)
        grid = {}
        pts = []
        cand = _hemisphere_points(rng, attempts_per_node * count, center, R, dim)
        s2 = spacing * spacing
        reach = int(math.ceil(spacing / cell))
        for p in cand:
            key = tuple(int(math.floor(p[a] / cell)) for a in range(dim))
            ok = True
            rngs = [range(key[a] - reach, key[a] + reach + 1) for a in range(dim)]
            if dim == 2:
                for i in rngs[0]:
                    for j in rngs[1]:
                        q = grid.get((i, j))
                        if q is not None and (q[0] - p[0]) ** 2 + (q[1] - p[1]) ** 2 < s2:
                            ok = False
                            break
                    if not ok:
                        break
            else:
                for i in rngs[0]:
                    for j in rngs[1]:
                        for k in rngs[2]:
                            q = grid.get((i, j, k))
                            if q is not None and ((q[0] - p[0]) ** 2 + (q[1] - p[1]) ** 2 +
                                                  (q[2] - p[2]) ** 2) < s2:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
            if ok:
                grid[key] = p
                pts.append(p)
                if len(pts) == count:
                    return np.array(pts), spacing
        spacing *= 0.9


def gaussian_mounds(rng, counts, centers, sig, lo, hi):
    """Gaussian clusters on the y = 0 wall: y reflected to |y|, the rest clipped."""
    parts = []
    for m, c in zip(counts, centers):
        p = rng.normal(0.0, sig, size=(m, 3)) + np.asarray(c)[None, :]
        p[:, 1] = np.abs(p[:, 1] - c[1]) + c[1]
        parts.append(p)
    X = np.vstack(parts)
    for a in range(3):
        X[:, a] = np.clip(X[:, a], lo[a], hi[a])
    return X


def springs_within(X, cutoff):
    """All pairs closer than ``cutoff`` (a < b, sorted), with their distances."""
    from scipy.spatial import cKDTree
    tree = cKDTree(X)
    pairs = np.asarray(tree.query_pairs(cutoff, output_type="ndarray"), dtype=np.int64)
    pairs = pairs.reshape(-1, 2)
    pairs = pairs[np.lexsort((pairs[:, 1], pairs[:, 0]))]
    if pairs.shape[0] == 0:
        return pairs.astype(np.int32), np.zeros(0)
    d = X[pairs[:, 1]] - X[pairs[:, 0]]
    rest = np.sqrt(np.sum(d * d, axis=1))
    return pairs.astype(np.int32), rest


# ---------------------------------------------------------------------------
# configurations
# ---------------------------------------------------------------------------
def _instance(prm, X, r, K, brk, steps, name, extra=None):
    ab, rest = springs_within(X, 2.5 * r)
    m = ab.shape[0]
    Kv = K(m) if callable(K) else np.full(m, float(K))
    inst = dict(name=name, params=prm, X=np.ascontiguousarray(X[:, :prm["dim"]]), ab=ab,
                rest=rest, K=Kv, brk=np.full(m, float(brk)), steps=steps)
    if extra:
        inst.update(extra)
    return inst


def c1(seed=0):
    """2D plain FP64: 64x32, 150 nodes in a half-disc, 20 steps, 3 V-cycles."""
    h = 1.0 / 64
    r = 0.01
    rng = np.random.Generator(np.random.PCG64(seed))
    X, spacing = dart_throw(rng, 150, 2, (0.5, 0.0), 0.1, 2 * r)
    area = math.pi * 0.1 ** 2 / 2.0
    prm = base_params(2, (64, 32), (1, 0), 0, h, rho_ratio=1.5, mu_ratio=100.0, omega=r,
                      omega_mu=r, d0_vol=area / 150, vc_visc=3, vc_p=3)
    return _instance(prm, X, r, 1.0, 0.5, 20, "c1", dict(spacing=spacing))


def _duct_params(e, length_cells, r, rho_ratio, mu_ratio, d0_vol, **kw):
    h = 1.0 / e
    return base_params(3, (e, e, length_cells), (0, 0, 1), 2, h, rho_ratio=rho_ratio,
                       mu_ratio=mu_ratio, omega=r, omega_mu=r, d0_vol=d0_vol, **kw)


def _logu(rng, lo, hi, m):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=m))


def c2(seed=1):
    """3D plain FP64: 64^3 duct, 2,000 nodes in a hemisphere of radius 0.15."""
    r = 0.008
    rng = np.random.Generator(np.random.PCG64(seed))
    R = 0.15
    X, spacing = dart_throw(rng, 2000, 3, (0.5, 0.0, 0.5), R, 2 * r)
    vol = 2.0 / 3.0 * math.pi * R ** 3
    prm = _duct_params(64, 64, r, 1.5, 1e3, vol / 2000)
    return _instance(prm, X, r, lambda m: _logu(rng, 0.1, 10.0, m), 0.3, 50, "c2",
                     dict(spacing=spacing))


def _mound_volume(sig, k):
    # k half-balls of radius 2 sigma: the volume the clusters occupy
    return k * 2.0 / 3.0 * math.pi * (2.0 * sig) ** 3


def c3(seed=2, precision=1):
    """3D mixed precision: 128x128x256 duct, 20,000 nodes in three mounds."""
    r = 0.005
    sig = 0.05
    rng = np.random.Generator(np.random.PCG64(seed))
    X = gaussian_mounds(rng, (6667, 6667, 6666), [(0.5, 0.0, 0.5), (0.5, 0.0, 1.0),
                                                 (0.5, 0.0, 1.5)], sig, (0, 0, 0), (1, 1, 2))
    prm = _duct_params(128, 256, r, 2.0, 1e3, _mound_volume(sig, 3) / 20000,
                       precision=precision)
    return _instance(prm, X, r, lambda m: _logu(rng, 0.1, 10.0, m), 0.3, 100, "c3")


def c4_instance(i, seed0=100):
    """One instance of the batched sweep: edge e from {32,48,64,96}, grid e x e x 2e."""
    rng = np.random.Generator(np.random.PCG64(seed0 + i))
    e = int(rng.choice([32, 48, 64, 96]))
    m = int(rng.integers(500, 8001))
    rho_ratio = float(rng.uniform(1.0, 2.0))
    mu_ratio = float(_logu(rng, 10.0, 1e3, 1)[0])
    # the hemispherical mound of the 64^3 duct workload (radius 0.15, r =
    # 0.008), sampled uniformly: at up to 8,000 nodes per instance the
    # dart-throwing spacing rule would take minutes for 64 instances. Denser
    # mounds (8,000 nodes within radius 0.1) exceed the explicit spring
    # stability limit of Sec. 4.3.4 at dt = 0.1 h on the 32-cell grids.
    r = 0.008
    R = 0.15
    X = _hemisphere_points(rng, m, (0.5, 0.0, 1.0), R, 3)
    prm = _duct_params(e, 2 * e, r, rho_ratio, mu_ratio, (2.0 / 3.0 * math.pi * R ** 3) / m,
                       precision=1)
    return _instance(prm, X, r, lambda q: _logu(rng, 0.1, 10.0, q), 0.3, 50, "c4_%02d" % i)


def c4(count=64):
    return [c4_instance(i) for i in range(count)]


def c5_request(i, seed0=1000):
    """One request of the serving stream: edge 48..160 step 16, grid e x e x 2e."""
    rng = np.random.Generator(np.random.PCG64(seed0 + i))
    e = int(rng.choice(np.arange(48, 161, 16)))
    m = int(rng.integers(500, 50001))
    r = 0.005
    sig = 0.05
    k = [m // 3 + (1 if q < m % 3 else 0) for q in range(3)]
    X = gaussian_mounds(rng, k, [(0.5, 0.0, 0.5), (0.5, 0.0, 1.0), (0.5, 0.0, 1.5)], sig,
                        (0, 0, 0), (1, 1, 2))
    prm = _duct_params(e, 2 * e, r, 2.0, 1e3, _mound_volume(sig, 3) / m, precision=1)
    return _instance(prm, X, r, lambda q: _logu(rng, 0.1, 10.0, q), 0.3, 200, "c5_%03d" % i)


def c5_arrivals(count=128, rate=4.0, seed=999):
    """Seeded exponential inter-arrival gaps (Poisson process of the given rate)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


# The paper's scaling (Appendix, "Scaling Parameters"): L = 50 um, u0 = 1 mm/s,
# T = 1 s, pressure drop 0.8144 Pa, rho0 = 998 kg/m^3, mu = 1e-3 kg/(m s).
PAPER_SIGMA = 50e-6 / (1.0 * 1e-3)                 # L / (T u0) = 0.05
PAPER_EULER = 0.8144 / (998.0 * 1e-3 ** 2)         # dp / (rho0 u0^2), about 816
PAPER_RE = 998.0 * 1e-3 * 50e-6 / 1e-3             # rho0 u0 L / mu, about 0.0499


def paper_units_duct(e=64, nodes=1500, f_max=0.5, seed=7):
    """A 3D duct in the paper's nondimensional units (sigma = 0.05, Euler
    number about 816, Re about 0.05, fluid viscosity 1 = that of water): the
    hemispherical mound of the 64^3 duct, springs with K = F_max / r that break
    at twice their rest length (Eq. defineK, break strain 1), and
    dt = 0.1 h sigma (a node moves a tenth of a cell per step at unit speed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = 0.008
    R = 0.15
    X = _hemisphere_points(rng, nodes, (0.5, 0.0, 0.5), R, 3)
    h = 1.0 / e
    prm = _duct_params(e, e, r, 1.5, 1e3, (2.0 / 3.0 * math.pi * R ** 3) / nodes,
                       sigma=PAPER_SIGMA, euler=PAPER_EULER, inv_re=1.0 / PAPER_RE, mu_f=1.0,
                       dt=0.1 * h * PAPER_SIGMA)
    ab, rest = springs_within(X, 2.5 * r)
    return dict(name="paper_units", params=prm, X=np.ascontiguousarray(X), ab=ab, rest=rest,
                K=f_max / np.maximum(rest, 1e-12), brk=np.full(len(rest), 1.0), steps=20)


def spin_up_channel(n=64):
    """2D channel of n x n/2 cells (periodic along the flow, walls across),
    started from half the Poiseuille profile and driven by the body force
    towards the full one; uniform fluid, no nodes. Smooth in space and time:
    the flow of the refinement studies (Sec. 4.3.2-4.3.3)."""
    h = 1.0 / n
    prm = base_params(2, (n, n // 2), (1, 0), 0, h, rho_ratio=1.5, mu_ratio=100.0,
                      omega=0.01, omega_mu=0.01, ic_scale=0.5, mu_f=1.0)
    return _instance(prm, np.zeros((0, 2)), 0.01, 1.0, 0.5, 20, "spin_up")


def mound_2d(n=64, rho_ratio=1.0, mu_ratio=1.0, omega=0.02, seed=0):
    """The refinement-study mound (Sec. 4.3.3): the 2D channel of c1 on an
    n x n/2 grid with the same 150 nodes in every resolution (the Lagrangian
    points are not refined with the grid), delta width omega = 1/50, and a
    biofilm that is fluid-like (ratios 1), twice as dense (rho_ratio 2) or
    500 times as viscous (mu_ratio 500)."""
    h = 1.0 / n
    r = 0.01
    rng = np.random.Generator(np.random.PCG64(seed))
    X, spacing = dart_throw(rng, 150, 2, (0.5, 0.0), 0.1, 2 * r)
    area = math.pi * 0.1 ** 2 / 2.0
    prm = base_params(2, (n, n // 2), (1, 0), 0, h, rho_ratio=rho_ratio, mu_ratio=mu_ratio,
                      omega=omega, omega_mu=omega, d0_vol=area / 150)
    return _instance(prm, X, r, 1.0, 0.5, 20, "mound_2d", dict(spacing=spacing))


def open_channel_2d(seed=0, n=64):
    """The open channel of Sec. 3.6 in 2D: c1's mound (150 nodes in a half-
    disc of radius 0.1 at x = 0.5 on the y = 0 wall) in a channel of
    2n x n/2 cells on [0, 2] x [0, 0.5], the laminar profile held at the
    inflow x = 0, du/dn = 0 and the pressure held at the outflow x = 2."""
    base = c1(seed)
    h = 1.0 / n
    prm = dict(base["params"], n=[2 * n, n // 2, 1], periodic=[0, 0, 1], open_flow=1, h=h,
               dt=0.1 * h)
    return dict(base, params=prm, name="open_channel_2d")


def open_duct(seed=1, e=64):
    """The open square tube of Sec. 3.6: c2's hemispherical mound (2,000
    nodes, radius 0.15, centred at z = 0.5) in an e x e x 2e duct of side 1
    and length 2, the laminar profile of Eq. (3DlaminarFlow) held at the
    inflow z = 0, du/dn = 0 and the pressure held at the outflow z = 2."""
    base = c2(seed)
    h = 1.0 / e
    prm = dict(base["params"], n=[e, e, 2 * e], periodic=[0, 0, 0], open_flow=1, h=h,
               dt=0.1 * h)
    return dict(base, params=prm, name="open_duct")


CONFIGS = {"c1": c1, "c2": c2, "c3": c3, "paper_units": paper_units_duct,
           "open_duct": open_duct}


def cells(prm):
    n = prm["n"]
    return n[0] * n[1] * (n[2] if prm["dim"] == 3 else 1)
