"""The open duct of Sec. 3.6 on the GPU against the oracle.

The inflow holds the laminar profile, and the outflow is an unknown face
with du/dn = 0 and the pressure held there. The FP64 path is compared with
the oracle on the same seeded mounds, with the tolerances of the periodic
duct:
* relative L2 of u and p at most 1e-10, over whole runs with fixed V-cycles
  and in relative-residual mode;
* nodes within 1e-12;
* identical break events.
The mass balance (flux out = flux in) and the per-step divergence check
hold on the device. The open duct runs in FP64 only, and mixed precision is
refused."""
import numpy as np
import pytest

from paper_1302_3663_gb300 import bfibm, workloads as W

from helpers import pair
from test_gpu_steps import compare_state, run_pair

pytestmark = pytest.mark.gpu


def test_open_channel_2d_fixed_cycles():
    run_pair(W.open_channel_2d(), 10)


def test_open_duct_3d_fixed_cycles():
    run_pair(W.open_duct(e=32), 4, chunk=2)


def _flux(u, n, fa, dim, idx):
    sl = [slice(0, n[a]) if a != fa else idx for a in reversed(range(dim))]
    return u[tuple(sl)].sum()


@pytest.mark.parametrize("graph", [1, 0])
def test_open_channel_tolerance_mode(graph):
    inst = W.open_channel_2d()
    over = dict(vc_visc=0, vc_p=0, rtol=1e-11, max_cycles=200, div_tol=1e-10)
    g, o = pair(inst, over)
    g.set_option(bfibm.OPT_GRAPH, graph)
    for k in range(3):
        assert g.step(1) == bfibm.OK
        o.step(1)
        st = g.get_stats()
        assert st["div_max_step"] <= 1e-10
        assert st["cycles_p"] == o.stats()["cycles_p"]
    compare_state(g, o, inst, "open channel, rtol 1e-11")
    n, _ = g.dims()
    u = g.get_velocity(0)
    fin, fout = _flux(u, n, 0, 2, 0), _flux(u, n, 0, 2, n[0])
    assert abs(fout - fin) <= 1e-9 * abs(fin), (fin, fout)
    assert g.get_stats()["div_violations"] == 0
    g.close()


def test_open_duct_graph_equals_direct_launches():
    inst = W.open_duct(e=32)
    a = bfibm.load_instance(inst)
    b = bfibm.load_instance(inst)
    b.set_option(bfibm.OPT_GRAPH, 0)
    a.step(3)
    b.step(3)
    for d in range(3):
        x, y = a.get_velocity(d), b.get_velocity(d)
        assert np.linalg.norm(x - y) <= 1e-13 * max(np.linalg.norm(y), 1e-300)
    a.close()
    b.close()


def test_open_duct_settings_outside_its_range_are_refused():
    inst = W.open_duct(e=32)
    for bad in (dict(precision=1), dict(periodic=[0, 0, 1]), dict(u_center=0.0)):
        with pytest.raises(bfibm.BfibmError) as e:
            bfibm.Context(dict(inst["params"], **bad))
        assert e.value.status == bfibm.EINVAL
    c = bfibm.Context(inst["params"])
    with pytest.raises(bfibm.BfibmError):
        c.set_option(bfibm.OPT_FUSED, 1)
    c.close()
