"""Shared helpers of the GPU parity tests: the same seeded inputs go to the
CUDA library (through its C ABI) and to the CPU oracle."""
import numpy as np

from oracle import oracle as O
from paper_1302_3663_gb300 import bfibm


def pair(inst, prm_override=None, omp=True, load=True):
    prm = dict(inst["params"])
    if prm_override:
        prm.update(prm_override)
    g = bfibm.Context(prm)
    o = O.Oracle(prm, omp=omp)
    if load:
        for c in (g, o):
            c.set_nodes(inst["X"])
            c.set_springs(inst["ab"], inst["rest"], inst["K"], inst["brk"])
    return g, o


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def assert_close(a, b, rel, what=""):
    r = rel_l2(np.asarray(a), np.asarray(b))
    assert r <= rel, "%s: relative L2 %.3e > %.1e" % (what, r, rel)
    return r


def random_coefficients(g, o, rng, mu_ratio=1e3, rho_ratio=2.0):
    """Install the same random rho (faces) and mu (centres, edges) on both."""
    D = g.dim
    sh = g.shape()
    for d in range(D):
        r = 1.0 + (rho_ratio - 1.0) * rng.uniform(size=sh)
        g.set_field("rho", r, d)
        o.set("rho", r, d)
    mu = 0.01 * np.exp(rng.uniform(0, np.log(mu_ratio), size=sh))
    g.set_field("muc", mu)
    o.set("muc", mu)
    for e in range(3 if D == 3 else 1):
        mu = 0.01 * np.exp(rng.uniform(0, np.log(mu_ratio), size=sh))
        g.set_field("mue", mu, e)
        o.set("mue", mu, e)
    g.build_coefficients()
    o.build_coefficients()


def face_mask(ctx, d, level=0):
    n, s = ctx.dims(level)
    lo = [0, 0, 0]
    hi = [n[0], n[1], n[2]]
    if not ctx.prm["periodic"][d]:
        lo[d], hi[d] = 1, n[d]
    m = np.zeros(ctx.shape(level), bool)
    if ctx.dim == 3:
        m[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = True
    else:
        m[lo[1]:hi[1], lo[0]:hi[0]] = True
    return m


def cell_mask(ctx, level=0):
    n, s = ctx.dims(level)
    m = np.zeros(ctx.shape(level), bool)
    if ctx.dim == 3:
        m[:n[2], :n[1], :n[0]] = True
    else:
        m[:n[1], :n[0]] = True
    return m
