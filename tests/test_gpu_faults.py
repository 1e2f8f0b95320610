"""Failure paths, made on the host and never by faulting the GPU: malformed
inputs are refused with BFIBM_EINVAL before anything runs; a solve that
cannot reach its tolerance in max_cycles reports BFIBM_ENOCONV, with the
step graph replayed (the device-side loop counts it) and without, and the
same context keeps stepping; a projection above div_tol reports
BFIBM_ENOCONV; a TMA sweep whose bounded waits are set to run out at once
drains its valid copies, stops, is counted, and makes the step report
BFIBM_ETIMEOUT while the device stays usable; a grid larger than the
device's memory is refused with BFIBM_ENOMEM (a real allocation failure,
caught by the library)."""
import numpy as np
import pytest

from paper_1302_3663_gb300 import bfibm, workloads as W

pytestmark = pytest.mark.gpu


def test_malformed_nodes_and_springs_are_refused():
    inst = W.c1()
    c = bfibm.Context(inst["params"])
    X = inst["X"].copy()
    X[3, 0] = np.nan
    with pytest.raises(bfibm.BfibmError) as e:
        c.set_nodes(X)
    assert e.value.status == bfibm.EINVAL
    X = inst["X"].copy()
    X[5, 1] = -0.1   # below the wall
    with pytest.raises(bfibm.BfibmError) as e:
        c.set_nodes(X)
    assert e.value.status == bfibm.EINVAL
    c.set_nodes(inst["X"])
    ab = inst["ab"].copy()
    ab[0, 1] = inst["X"].shape[0]   # endpoint past the last node
    with pytest.raises(bfibm.BfibmError) as e:
        c.set_springs(ab, inst["rest"], inst["K"], inst["brk"])
    assert e.value.status == bfibm.EINVAL
    K = inst["K"].copy()
    K[2] = np.inf
    with pytest.raises(bfibm.BfibmError) as e:
        c.set_springs(inst["ab"], inst["rest"], K, inst["brk"])
    assert e.value.status == bfibm.EINVAL
    # the refusals left the context as it was: it still steps
    c.set_springs(inst["ab"], inst["rest"], inst["K"], inst["brk"])
    assert c.step(2) == bfibm.OK
    assert all(np.isfinite(c.get_velocity(d)).all() for d in range(2))
    c.close()


@pytest.mark.parametrize("graph", [1, 0])
@pytest.mark.parametrize("precision", [0, 1])
def test_unreachable_tolerance_reports_no_convergence_and_recovers(precision, graph):
    inst = W.c2()
    prm = dict(inst["params"], precision=precision, vc_visc=0, vc_p=0, rtol=1e-30,
               max_cycles=2)
    c = bfibm.load_instance(inst, prm_override=prm)
    c.set_option(bfibm.OPT_GRAPH, graph)
    assert c.step(1) == bfibm.ENOCONV
    st = c.get_stats()
    assert st["cycles_visc"] <= 2 and st["res_visc"] > 1e-30
    if graph:
        assert st["nonconv_total"] == 2   # both device loops stopped at the cap
    # the same context keeps stepping (and keeps reporting) with a valid state
    assert c.step(1) == bfibm.ENOCONV
    assert all(np.isfinite(c.get_velocity(d)).all() for d in range(3))
    c.close()
    # a reachable tolerance converges
    c = bfibm.load_instance(inst, prm_override=dict(prm, rtol=1e-9, max_cycles=60))
    c.set_option(bfibm.OPT_GRAPH, graph)
    assert c.step(2) == bfibm.OK
    st = c.get_stats()
    assert st["res_visc"] <= 1e-9 and st["nonconv_total"] == 0
    c.close()


def test_projection_above_div_tol_reports_no_convergence():
    inst = W.c1()   # 3 fixed V-cycles leave max |D.u| near 1e-4
    c = bfibm.load_instance(inst, prm_override=dict(div_tol=1e-8))
    assert c.step(2) == bfibm.ENOCONV
    st = c.get_stats()
    assert st["div_violations"] == 2 and st["div_max_step"] > 1e-8
    c.close()
    c = bfibm.load_instance(inst, prm_override=dict(div_tol=1.0))
    assert c.step(2) == bfibm.OK
    assert c.get_stats()["div_violations"] == 0
    c.close()


def test_tma_wait_that_runs_out_is_reported_and_the_device_recovers():
    # a small duct whose finest level takes the TMA sweep; waits limited to
    # one test of the barrier, so they give up while the block's own (valid)
    # copies are still in flight; the block drains them and returns
    prm = W.base_params(3, (32, 32, 64), (0, 0, 1), 2, 1.0 / 32, precision=1)
    c = bfibm.Context(prm)
    c.set_option(bfibm.OPT_TMA, 2)
    c.set_option(bfibm.OPT_WAIT_NS, 0)
    for _ in range(4):
        c.smooth_f32(1, 0, 1)
    st = c.get_stats()
    assert st["wait_timeouts"] > 0
    with pytest.raises(bfibm.BfibmError) as e:
        c.step(1)
    assert e.value.status == bfibm.ETIMEOUT
    with pytest.raises(bfibm.BfibmError) as e:   # the context is poisoned
        c.step(1)
    assert e.value.status == bfibm.ESTATE
    c.close()
    # a fresh context with the default limit runs normally
    c = bfibm.Context(prm)
    c.set_option(bfibm.OPT_TMA, 2)
    assert c.step(2) == bfibm.OK
    st = c.get_stats()
    assert st["wait_timeouts"] == 0
    assert all(np.isfinite(c.get_velocity(d)).all() for d in range(3))
    c.close()


def test_a_grid_larger_than_the_device_is_refused_with_enomem():
    import torch
    # 1024^3 cells between walls: about 340 GB of FP64 grids, more than the
    # device holds, so the pool allocation fails and nothing is launched
    h = 1.0 / 1024
    prm = W.base_params(3, (1024, 1024, 1024), (0, 0, 1), 2, h, u_center=0.0, body_force=1.0)
    _, total = torch.cuda.mem_get_info()
    if bfibm.footprint(prm, 0, 0) <= 1.1 * total:
        pytest.skip("this device could hold the grid")
    with pytest.raises(bfibm.BfibmError) as e:
        bfibm.Context(prm)
    assert e.value.status == bfibm.ENOMEM
    # and the device is still usable
    c = bfibm.load_instance(W.c1())
    assert c.step(1) == bfibm.OK
    c.close()
