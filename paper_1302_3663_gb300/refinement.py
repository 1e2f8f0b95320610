"""Refinement studies of Sec. 4.3.2-4.3.3: empirical convergence rates in time
and in space.

Time (Eqs. ErrorTemporal and the temporal convergence rate):
    E_p(q(T); dt) = || q^dt(T) - q^(dt/2)(T) ||_p,
    r_p(q(T); dt) = log2( E_p(q(T); dt) / E_p(q(T); dt/2) ).
Space (Eqs. ErrorSpatial and convergenceRate): the same with h, where the
solution on the grid h/2 is first restricted to the grid h (I_h^2h: along a
face's own axis (1/4, 1/2, 1/4) on the coincident and neighbouring faces,
across it the mean of the two children; the nodes are the same on every
grid, so X needs no restriction).

Norms: for the velocity the discrete L2 norm with weight h^D over every face,
and the maximum; for the nodes the root mean square over nodes and the
maximum, of the coordinate differences.

A run is one simulation advanced to T through a backend: the CUDA library
(`gpu_backend`) or any object with the same three methods, so the same study
can be repeated on a reference implementation.
"""
import math

import numpy as np

from . import bfibm


class gpu_backend:
    """Runs a workload instance through the C ABI."""

    def __init__(self, inst, prm):
        self.ctx = bfibm.load_instance(inst, prm_override=prm)
        self.dim = prm["dim"]

    def step(self, n):
        self.ctx.step(n)

    def velocity(self):
        return [self.ctx.get_velocity(d) for d in range(self.dim)]

    def nodes(self):
        return self.ctx.get_nodes()

    def close(self):
        self.ctx.close()


def _norms(diffs, weight):
    sq = sum(float(np.sum(d * d)) for d in diffs)
    mx = max(float(np.max(np.abs(d))) if d.size else 0.0 for d in diffs)
    return math.sqrt(weight * sq), mx


def _node_norms(dX):
    if len(dX) == 0:
        return 0.0, 0.0
    return (math.sqrt(float(np.mean(np.sum(dX * dX, axis=1)))), float(np.max(np.abs(dX))))


def restrict_face(uf, d, dim, per):
    """I_h^2h of face component d: arrays are (z, y, x) in 3D, (y, x) in 2D,
    with the wall face stored on wall axes (extent 2n + 1 fine, n + 1 coarse)."""
    a = np.asarray(uf)
    # numpy axis of grid axis ax
    npax = lambda ax: dim - 1 - ax
    out = a
    for ax in range(dim):
        k = npax(ax)
        out = np.moveaxis(out, k, 0)
        nf = out.shape[0] - (0 if per[ax] else 1)   # fine cells along ax
        nc = nf // 2
        if ax == d:
            ncs = nc if per[ax] else nc + 1
            res = np.zeros((ncs,) + out.shape[1:])
            for I in range(ncs):
                if not per[ax] and (I == 0 or I == nc):
                    continue   # wall faces hold 0
                acc = 0.0
                for o, w in ((-1, 0.25), (0, 0.5), (1, 0.25)):
                    q = 2 * I + o
                    if per[ax]:
                        q %= nf
                    acc = acc + w * out[q]
                res[I] = acc
        else:
            ncs = nc if per[ax] else nc + 1
            res = np.zeros((ncs,) + out.shape[1:])
            res[:nc] = 0.5 * (out[0:2 * nc:2] + out[1:2 * nc:2])
        out = np.moveaxis(res, 0, k)
    return out


def temporal_rates(inst, T, dt0, nruns=4, backend=gpu_backend, solver=None):
    """Runs at dt0, dt0/2, ..., dt0/2^(nruns-1) to time T; returns the errors
    E_2, E_inf of u and X between consecutive runs and the rates between
    consecutive errors."""
    prm0 = dict(inst["params"], **(solver or {}))
    runs = []
    for k in range(nruns):
        dt = dt0 / 2 ** k
        steps = int(round(T / dt))
        b = backend(inst, dict(prm0, dt=dt))
        b.step(steps)
        runs.append((b.velocity(), b.nodes()))
        b.close()
    h = prm0["h"]
    w = h ** prm0["dim"]
    errs = []
    for (ua, Xa), (ub, Xb) in zip(runs[:-1], runs[1:]):
        eu = _norms([x - y for x, y in zip(ua, ub)], w)
        ex = _node_norms(Xa - Xb)
        errs.append({"dt": dt0 / 2 ** len(errs), "u_2": eu[0], "u_inf": eu[1], "X_2": ex[0],
                     "X_inf": ex[1]})
    rates = []
    for a, b in zip(errs[:-1], errs[1:]):
        rates.append({k: (math.log2(a[k] / b[k]) if a[k] > 0 and b[k] > 0 else float("nan"))
                      for k in ("u_2", "u_inf", "X_2", "X_inf")})
        rates[-1]["dt"] = a["dt"]
    return {"errors": errs, "rates": rates}


def spatial_rates(make_inst, ns, T, dt, backend=gpu_backend, solver=None):
    """make_inst(n) gives the workload on a grid of n cells along x (the other
    axes in proportion) with the same nodes; ns ascending by factors of 2.
    Returns E_2, E_inf of u (restricted) and X between consecutive grids and
    the rates between consecutive errors."""
    runs = []
    for n in ns:
        inst = make_inst(n)
        prm = dict(inst["params"], dt=dt, **(solver or {}))
        b = backend(inst, prm)
        b.step(int(round(T / dt)))
        runs.append((prm, b.velocity(), b.nodes()))
        b.close()
    errs = []
    for (pa, ua, Xa), (pb, ub, Xb) in zip(runs[:-1], runs[1:]):
        dim = pa["dim"]
        per = pa["periodic"][:dim]
        ur = [restrict_face(ub[d], d, dim, per) for d in range(dim)]
        eu = _norms([x - y for x, y in zip(ua, ur)], pa["h"] ** dim)
        ex = _node_norms(Xa - Xb)
        errs.append({"h": pa["h"], "u_2": eu[0], "u_inf": eu[1], "X_2": ex[0], "X_inf": ex[1]})
    rates = []
    for a, b in zip(errs[:-1], errs[1:]):
        rates.append({k: (math.log2(a[k] / b[k]) if a[k] > 0 and b[k] > 0 else float("nan"))
                      for k in ("u_2", "u_inf", "X_2", "X_inf")})
        rates[-1]["h"] = a["h"]
    return {"errors": errs, "rates": rates}
