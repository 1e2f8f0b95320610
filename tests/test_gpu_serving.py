"""Batched and served forms: independent simulations stepped together give
the same results as each simulation alone, and the service admits requests by
device-memory footprint, queueing the rest until memory frees up.

A time step does not depend on the order of atomic additions (node forces are
summed per node in a fixed order, the spread sums f and rho in fixed point),
so alone and in the mix the results are bit-identical
(test_alone_and_in_batch_bit_identical); the other checks state relative L2
bounds on the scale of the whole field, 1e-12 for FP64 and 1e-9 for mixed
precision, which bit-identical results meet trivially."""
import numpy as np
import pytest

from paper_1302_3663_gb300 import bfibm, serve, workloads as W

from helpers import rel_l2

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-9}


def small_instance(i, e=32, nodes=400, precision=1):
    rng = np.random.Generator(np.random.PCG64(500 + i))
    r = 0.02
    X = W._hemisphere_points(rng, nodes, (0.5, 0.0, 1.0), 0.15, 3)
    prm = W._duct_params(e, 2 * e, r, float(rng.uniform(1, 2)),
                         float(np.exp(rng.uniform(np.log(10), np.log(1e3)))),
                         (2.0 / 3.0 * np.pi * 0.15 ** 3) / nodes, precision=precision)
    return W._instance(prm, X, r, lambda q: W._logu(rng, 0.1, 10.0, q), 0.3, 6, "s%d" % i)


def state(ctx):
    return [ctx.get_velocity(d) for d in range(ctx.dim)] + [ctx.get_pressure(), ctx.get_nodes()]


def same(a, b, precision):
    # velocity components on the scale of the whole velocity, then p, then X
    scale = np.sqrt(sum(np.sum(y * y) for y in b[:-2]))
    for x, y in zip(a[:-2], b[:-2]):
        assert np.linalg.norm(x - y) / scale <= TOL[precision]
    assert rel_l2(a[-2], b[-2]) <= TOL[precision]
    assert np.abs(a[-1] - b[-1]).max() <= TOL[precision]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_alone_with_staggered_members(precision):
    insts = [small_instance(i, e=(32 if i % 2 else 48), precision=precision) for i in range(3)]
    alone = []
    for inst in insts:
        c = bfibm.load_instance(inst)
        c.step(6)
        alone.append(state(c))
        c.close()
    b = bfibm.Batch()
    ctxs = [bfibm.load_instance(inst) for inst in insts]
    slots = [b.add(ctxs[0])]
    b.step()                       # member 0 alone for two steps
    b.step()
    slots.append(b.add(ctxs[1]))
    b.step({slots[0]: 2, slots[1]: 1})
    slots.append(b.add(ctxs[2]))
    for _ in range(6):
        want = {s: (1 if ctxs[k].get_stats()["step"] < 6 else 0) for k, s in enumerate(slots)}
        b.step(want)
        b.wait()
    for k, c in enumerate(ctxs):
        assert c.get_stats()["step"] == 6
        same(state(c), alone[k], precision)
    b.close()


TOL_SOLVER = {"vc_visc": 0, "vc_p": 0, "rtol": 1e-11, "max_cycles": 100, "gamma_coarse": 0.8,
              "inner_cycles": 2, "krylov": 1, "div_tol": 1e-10}


def test_persistent_server_matches_alone_bit_for_bit():
    # requests stepped in lock step (each multigrid level one launch over the
    # admitted ones) while others arrive and leave: each result is the bits
    # of the request alone
    insts = [small_instance(i, e=32 + 16 * (i % 2)) for i in range(4)]
    for inst in insts:
        inst["params"].update(TOL_SOLVER)
    reqs = [serve.Request(i, inst, 3 + i, arrival=0.01 * i) for i, inst in enumerate(insts)]
    budget = int(1.05 * (sorted(r.footprint for r in reqs)[-1] + sorted(r.footprint for r in reqs)[-2]))
    srv = serve.Server(budget, persistent=True)
    done = srv.run(reqs)
    srv.close()
    assert len(done) == 4
    for r in done:
        c = bfibm.load_instance(r.inst)
        c.step(r.steps)
        want = state(c)
        c.close()
        got = r.result["u"] + [r.result["p"], r.result["X"]]
        for x, y in zip(got, want):
            assert np.array_equal(x, y)


def test_server_queues_by_footprint_and_matches_alone():
    insts = [small_instance(i, e=32 + 16 * (i % 2)) for i in range(4)]
    reqs = [serve.Request(i, inst, 5, arrival=0.02 * i) for i, inst in enumerate(insts)]
    # room for about two simulations at a time: the others must wait
    budget = int(1.05 * (sorted(r.footprint for r in reqs)[-1] + sorted(r.footprint for r in reqs)[-2]))
    srv = serve.Server(budget)
    done = srv.run(reqs)
    srv.close()
    assert len(done) == 4
    summary = serve.summarize(done, srv.elapsed)
    assert summary["queue_s_max"] > 0.0
    assert summary["step_ms_p99"] >= summary["step_ms_p50"] > 0.0
    for r in done:
        c = bfibm.load_instance(r.inst)
        c.step(5)
        ref = [c.get_velocity(d) for d in range(3)] + [c.get_pressure(), c.get_nodes()]
        got = r.result["u"] + [r.result["p"], r.result["X"]]
        same(got, ref, 1)
        c.close()


def test_contexts_with_different_spread_regions():
    # the spread's shared-memory size depends on the delta width: a context
    # with a narrower support created after a wider one must leave the wider
    # one able to launch
    base = small_instance(7, e=32, nodes=200, precision=0)
    h = base["params"]["h"]
    wide = dict(base, params=dict(base["params"], omega=1.8 * h, omega_mu=1.8 * h))
    narrow = dict(base, params=dict(base["params"], omega=1.2 * h, omega_mu=1.2 * h))
    ref = bfibm.load_instance(wide)
    ref.step(2)
    want = state(ref)
    ref.close()
    a = bfibm.load_instance(wide)
    b = bfibm.load_instance(narrow)
    b.step(1)
    a.step(2)
    same(state(a), want, 0)
    assert a.get_stats()["nonfinite_total"] == 0
    a.close()
    b.close()


# the served benchmark's solver: relative residual 1e-11, flexible CG around
# two FP32 V(2,2) cycles for the viscous solve
TOL_CG = {"vc_visc": 0, "vc_p": 0, "rtol": 1e-11, "max_cycles": 100, "gamma_coarse": 0.8,
          "nu1": 2, "nu2": 2, "inner_cycles": 2, "krylov": 1}


@pytest.mark.parametrize("precision,solver", [(0, None), (1, None), (1, TOL_CG)],
                         ids=["fp64", "mixed", "mixed_tolerance_cg"])
def test_alone_and_in_batch_bit_identical(precision, solver):
    # node forces are summed per node in a fixed order and the spread sums f
    # and rho as fixed-point integers, so nothing depends on the order of
    # atomic additions: a simulation gives the same bits alone and in a batch
    insts = [small_instance(i, e=(32 if i % 2 else 48), precision=precision) for i in range(3)]
    for inst in insts:
        inst["params"].update(solver or {})
    alone = []
    for inst in insts:
        c = bfibm.load_instance(inst)
        c.step(4)
        alone.append(state(c))
        c.close()
    b = bfibm.Batch()
    ctxs = [bfibm.load_instance(inst) for inst in insts]
    slots = [b.add(c) for c in ctxs]
    b.step({slots[0]: 1, slots[1]: 0, slots[2]: 2})
    for _ in range(4):
        b.step({s: (1 if ctxs[k].get_stats()["step"] < 4 else 0) for k, s in enumerate(slots)})
        b.wait()
    for k, c in enumerate(ctxs):
        assert c.get_stats()["step"] == 4
        for x, y in zip(state(c), alone[k]):
            assert np.array_equal(x, y)
        c.close()
    b.close()
