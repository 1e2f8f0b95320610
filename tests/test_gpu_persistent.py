"""The persistent batch (bfibm_batch_set_option(BFIBM_BATCH_PERSISTENT)):
uneven members stepped in lock step, every multigrid level of their
mixed-precision solves one launch over all of them, each solve's device loop
masked per member.

Per member the batched kernels do the arithmetic of the single-instance
kernels on the same block decompositions (the reductions' partial sums
included) and the loop tests are the same, so every member must come out
bit-identical to itself stepped alone: velocity, pressure, nodes, broken
springs and the V-cycle counts of its solves. Members that converge after
different numbers of iterations check the masks; a change of members checks
that the plan is rebuilt."""
import numpy as np
import pytest

from paper_1302_3663_gb300 import bfibm

from test_gpu_serving import small_instance

pytestmark = pytest.mark.gpu

TOL_SOLVER = {"vc_visc": 0, "vc_p": 0, "rtol": 1e-11, "max_cycles": 100, "gamma_coarse": 0.8,
              "nu1": 2, "nu2": 2, "inner_cycles": 2, "krylov": 1, "div_tol": 1e-10}


def members(edges, **over):
    out = []
    for i, e in enumerate(edges):
        inst = small_instance(i, e=e)
        inst["params"].update(TOL_SOLVER)
        inst["params"].update(over)
        out.append(inst)
    return out


def snapshot(c):
    st = c.get_stats()
    return ([c.get_velocity(d) for d in range(3)] + [c.get_pressure(), c.get_nodes()],
            c.get_broken(), (st["cycles_visc"], st["cycles_p"], st["nonconv_total"],
                             st["div_violations"], st["step"]))


def alone(insts, nsteps):
    out = []
    for inst in insts:
        c = bfibm.load_instance(inst)
        cyc = []
        for _ in range(nsteps):
            c.step(1)
            cyc.append(snapshot(c)[2][:2])
        out.append((snapshot(c), cyc))
        c.close()
    return out


def assert_same(got, want, what):
    (fa, ba, sa), (fb, bb, sb) = got, want
    for k, (x, y) in enumerate(zip(fa, fb)):
        assert np.isfinite(x).all()
        assert np.array_equal(x, y), "%s field %d: max |diff| %.3e" % (what, k, np.abs(x - y).max())
    assert np.array_equal(np.asarray(ba), np.asarray(bb)), what
    assert sa == sb, (what, sa, sb)


def run_persistent(insts, nsteps, tune=False):
    ctxs = [bfibm.load_instance(inst) for inst in insts]
    b = bfibm.Batch(persistent=True, tune=tune)
    for c in ctxs:
        c.set_option(bfibm.OPT_STATS, 0)
        b.add(c)
    cyc = [[] for _ in ctxs]
    for _ in range(nsteps):
        b.step()
        assert b.wait() == bfibm.OK
        for k, c in enumerate(ctxs):
            cyc[k].append(snapshot(c)[2][:2])
    return b, ctxs, cyc


@pytest.mark.parametrize("tune", [False, True])
def test_uneven_members_bit_identical_to_alone(tune):
    insts = members([48, 32, 64, 32])
    want = alone(insts, 3)
    b, ctxs, cyc = run_persistent(insts, 3, tune)
    for k, c in enumerate(ctxs):
        assert_same(snapshot(c), want[k][0], "member %d" % k)
        assert cyc[k] == want[k][1]
    info = b.info()
    assert info["persistent"] == 1 and info["members"] == 4 and info["builds"] == 1
    # the batch loops ran as long as the slowest member's
    assert info["visc_iterations"] == sum(max(c[s][0] for c in cyc) // 2 for s in range(3))
    assert info["p_iterations"] == sum(max(c[s][1] for c in cyc) // 2 for s in range(3))
    for lev in range(3):
        for kind in (0, 1):
            TY, KC, NP, bx, allb, grid, kern = b.sweep_shape(lev, kind)
            assert kern in (0, 1)
            assert TY >= 1 and KC >= 1 and NP in (1, 2) and bx % 32 == 0
            # levels the coarse-level cluster kernel takes over have no sweep launch
            assert grid >= (1 if lev == 0 else 0)
    b.close()
    for c in ctxs:
        c.close()


def test_members_stop_on_their_own_tolerance():
    # a loose tolerance on one member: it leaves the loops early, the others
    # run on, and each matches itself alone
    insts = members([32, 48, 32])
    insts[1]["params"].update(rtol=1e-6, div_tol=0.0)
    want = alone(insts, 2)
    b, ctxs, cyc = run_persistent(insts, 2)
    assert cyc[1][0][0] < cyc[0][0][0]
    for k, c in enumerate(ctxs):
        assert_same(snapshot(c), want[k][0], "member %d" % k)
    b.close()
    for c in ctxs:
        c.close()


def test_defect_correction_and_odd_sweep_counts():
    # plain defect correction for the viscous solve, and V(1,1) cycles, whose
    # odd sweep counts end each smoothing with a copy back
    insts = members([32, 48], krylov=0, nu1=1, nu2=1, inner_cycles=3)
    want = alone(insts, 2)
    b, ctxs, _ = run_persistent(insts, 2)
    for k, c in enumerate(ctxs):
        assert_same(snapshot(c), want[k][0], "member %d" % k)
    b.close()
    for c in ctxs:
        c.close()


def test_plan_rebuilt_when_members_change():
    insts = members([32, 48, 32])
    want = alone(insts, 3)
    ctxs = [bfibm.load_instance(inst) for inst in insts]
    b = bfibm.Batch(persistent=True, tune=False)
    slots = [b.add(c) for c in ctxs]
    b.step()
    b.step({slots[0]: 1, slots[1]: 1, slots[2]: 0})   # member 2 waits one step
    assert b.info()["builds"] == 2
    b.step()
    b.remove(slots[0])                                 # member 0 has its 3 steps...
    b.step({slots[1]: 0, slots[2]: 1})                 # ...member 2 catches up
    b.wait()
    assert b.info()["builds"] == 4
    for k, c in enumerate(ctxs):
        assert_same(snapshot(c), want[k][0], "member %d" % k)
    # unequal step counts are refused
    b.add(ctxs[0])
    with pytest.raises(bfibm.BfibmError) as e:
        b.step({0: 2, slots[1]: 1, slots[2]: 1})
    assert e.value.status == bfibm.EINVAL
    b.close()
    for c in ctxs:
        c.close()


def test_members_outside_its_range_are_refused():
    good = members([32])[0]
    for bad in (dict(precision=0), dict(vc_visc=3, vc_p=3)):
        inst = members([32])[0]
        inst["params"].update(bad)
        b = bfibm.Batch(persistent=True, tune=False)
        cs = [bfibm.load_instance(good), bfibm.load_instance(inst)]
        for c in cs:
            b.add(c)
        with pytest.raises(bfibm.BfibmError) as e:
            b.step()
        assert e.value.status == bfibm.EINVAL
        b.close()
        for c in cs:
            c.close()


def test_unrolled_loops_and_pinned_shapes_give_the_same_bits():
    # loops queued as fixed iterations (the masks still stop each member) and
    # sweep shapes pinned after the plan is built (the ring sweep, then the
    # pair sweep): the same bits again
    insts = members([32, 48])
    want = alone(insts, 3)
    ctxs = [bfibm.load_instance(inst) for inst in insts]
    b = bfibm.Batch(persistent=True, tune=False)
    b.set_option(bfibm.BATCH_UNROLL, 40)
    for c in ctxs:
        b.add(c)
    b.step()
    b.wait()
    b.set_sweep_shape(0, 0, (2, 5, 2, 64, 0))
    b.set_sweep_shape(1, 1, (3, 7, 1, 32, 1))
    assert b.sweep_shape(0, 0)[:5] == (2, 5, 2, 64, 0)
    assert b.sweep_shape(1, 1)[:5] == (3, 7, 1, 32, 1)
    for bad in ((0, 8, 1, 32, 0), (4, 8, 3, 32, 0), (4, 8, 1, 48, 0), (40, 8, 1, 64, 0),
                (4, 8, 2, 64, 1, 1),      # the pair sweep takes one plane per phase
                (40, 8, 1, 64, 1, 1),     # more than 512 threads
                (4, 8, 1, 64, 1, 2)):
        with pytest.raises(bfibm.BfibmError):
            b.set_sweep_shape(0, 0, bad)
    assert b.sweep_shape(0, 0)[:5] == (2, 5, 2, 64, 0)
    b.step()
    b.wait()
    b.set_sweep_shape(0, 0, (4, 7, 1, 64, 1, 1))   # the pair sweeps on the finest level
    b.set_sweep_shape(0, 1, (6, 5, 1, 32, 1, 1))
    assert b.sweep_shape(0, 0)[6] == 1 and b.sweep_shape(0, 1)[6] == 1
    b.step()
    assert b.wait() == bfibm.OK
    for k, c in enumerate(ctxs):
        assert_same(snapshot(c), want[k][0], "member %d" % k)
    b.close()
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("tail", [0, 8192])
def test_batch_coarse_level_threshold_keeps_the_bits(tail):
    # the batch's coarse-level kernel from no level at all to every level of
    # at most 8192 cells: the same bits as alone
    insts = members([32, 48, 64])
    want = alone(insts, 2)
    ctxs = [bfibm.load_instance(inst) for inst in insts]
    b = bfibm.Batch(persistent=True, tune=False)
    b.set_option(bfibm.BATCH_TAIL, tail)
    for c in ctxs:
        b.add(c)
    for _ in range(2):
        b.step()
    assert b.wait() == bfibm.OK
    for k, c in enumerate(ctxs):
        assert_same(snapshot(c), want[k][0], "member %d" % k)
    b.close()
    for c in ctxs:
        c.close()
