"""Full-size parity in the exact configuration the benchmark times.

The benchmark steps the 128 x 128 x 256 duct (20,000 nodes, viscosity ratio
1e3, density ratio 2) in mixed precision:
* the viscous solve is flexible CG in FP64 around two FP32 V(2,2) cycles per
  iteration;
* the pressure solve is defect correction with two FP32 V(2,2) cycles per FP64
  residual;
* both solves stop at relative residual 1e-11, and the pressure solve also at
  (euler dt / sigma) max |r_p| <= 1e-10;
* the coarse viscosity scaling is tuned per level by the tuner;
* the FP32 sweeps take the shapes the autotuner chose when the context was
  created.

The oracle runs the paper's plain FP64 V-cycles with the same gamma, the same
tolerances and the same stop rule. Both sides solve the same discrete systems
to the same tests, so they agree to within what the tolerances leave: relative
L2 of u and p at most 1e-10, nodes within 1e-10, the same break events. The
library's own check inside every step also shows max |D.u| <= 1e-10.
"""
import numpy as np
import pytest

import bench
from paper_1302_3663_gb300 import bfibm, tuning, workloads as W

from helpers import pair
from test_gpu_steps import near_threshold

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

U_TOL = 1e-10
X_TOL = 1e-10


def test_benchmark_configuration_matches_the_oracle():
    inst = W.c3()
    prm = dict(inst["params"], **bench.TOL_SOLVER)
    assert prm["precision"] == 1 and prm["krylov"] == 1 and prm["div_tol"] == 1e-10
    # the per-level gamma of Eq. (ViscCoarseGrid) as the benchmark tunes it,
    # on the state after one step
    t = bfibm.load_instance(inst, prm_override=prm)
    t.step(1)
    t.set_option(bfibm.OPT_GRAPH, 0)
    gl, _, _ = tuning.tune_gamma(t)
    t.close()
    prm["gamma_levels"] = gl
    g, o = pair(inst, prm)   # the oracle on every host core
    assert any(sh is not None for sh in (g.sweep_shape(0, d) for d in range(3)))
    skip = set()
    for k in range(2):
        assert g.step(1) == bfibm.OK
        o.step(1)
        skip |= near_threshold(o, inst)
        st = g.get_stats()
        assert st["div_max_step"] <= 1e-10, (k, st["div_max_step"])
        assert st["nonconv_total"] == 0 and st["div_violations"] == 0
    uo = [o.get("u", d) for d in range(3)]
    scale = np.sqrt(sum(np.sum(u * u) for u in uo))
    for d in range(3):
        err = np.linalg.norm(g.get_velocity(d) - uo[d]) / scale
        print("u%d relative L2 %.3e" % (d, err))
        assert err <= U_TOL
    po = o.get("p")
    perr = np.linalg.norm(g.get_pressure() - po) / np.linalg.norm(po)
    print("p relative L2 %.3e" % perr)
    assert perr <= U_TOL
    dx = np.abs(g.get_nodes() - o.nodes()).max()
    print("nodes max difference %.3e" % dx)
    assert dx <= X_TOL
    ig, sg = g.get_broken()
    io, so = o.broken()
    ev_g = {(int(i), int(s)) for i, s in zip(ig, sg) if i not in skip}
    ev_o = {(int(i), int(s)) for i, s in zip(io, so) if i not in skip}
    assert ev_g == ev_o
    g.close()
    o.close()
