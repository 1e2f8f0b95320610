"""Failure paths, made on the host and never by faulting the GPU: malformed
inputs are refused with BFIBM_EINVAL before anything runs, a solve that
cannot reach its tolerance in max_cycles reports BFIBM_ENOCONV and leaves
the context usable, and a grid larger than the device's memory is refused
with BFIBM_ENOMEM (a real allocation failure, caught by the library)."""
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


@pytest.mark.parametrize("precision", [0, 1])
def test_unreachable_tolerance_reports_no_convergence_and_recovers(precision):
    inst = W.c2()
    prm = dict(inst["params"], precision=precision, vc_visc=0, vc_p=0, rtol=1e-30,
               max_cycles=2)
    c = bfibm.load_instance(inst, prm_override=prm)
    c.set_option(bfibm.OPT_GRAPH, 0)
    assert c.step(1) == bfibm.ENOCONV
    st = c.get_stats()
    assert st["cycles_visc"] <= 2 and st["res_visc"] > 1e-30
    # the context stays usable: a reachable tolerance converges afterwards
    c.close()
    c = bfibm.load_instance(inst, prm_override=dict(prm, rtol=1e-9, max_cycles=60))
    c.set_option(bfibm.OPT_GRAPH, 0)
    assert c.step(1) == bfibm.OK
    assert c.get_stats()["res_visc"] <= 1e-9
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
