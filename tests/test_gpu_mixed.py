"""Mixed precision (FP32 V-cycles inside FP64 defect correction) against the
FP64 oracle. The fine-grid residual, the divergence and the coarsest solve
stay FP64, so the differences are those of FP32 corrections. Stated bounds:
with a fixed number of V-cycles per solve (corrections not iterated to
convergence) relative L2 u and p <= 1e-7 and nodes within 1e-10 over whole
runs; in relative-residual mode u and p agree to 1e-12."""
import numpy as np
import pytest

from paper_1302_3663_gb300 import bfibm, workloads as W

from helpers import assert_close, pair, rel_l2

pytestmark = pytest.mark.gpu

U_TOL, P_TOL, X_TOL = 1e-7, 1e-7, 1e-10


def mixed_pair(inst, steps, extra=None):
    over = {"precision": 1}
    if extra:
        over.update(extra)
    g, o = pair(inst, over)
    g.step(steps)
    o.step(steps)
    return g, o


def report(g, o, what):
    du = max(rel_l2(g.get_velocity(d), o.get("u", d)) for d in range(g.dim))
    dp = rel_l2(g.get_pressure(), o.get("p"))
    dx = np.abs(g.get_nodes() - o.nodes()).max()
    print("%s: u %.2e p %.2e X %.2e" % (what, du, dp, dx))
    return du, dp, dx


def test_c1_mixed_fixed_cycles():
    inst = W.c1()
    g, o = mixed_pair(inst, inst["steps"])
    du, dp, dx = report(g, o, "c1 mixed")
    assert du <= U_TOL and dp <= P_TOL and dx <= X_TOL
    ig, _ = g.get_broken()
    io, _ = o.broken()
    assert set(ig) == set(io)


def test_c2_mixed_fixed_cycles():
    inst = W.c2()
    g, o = mixed_pair(inst, 5)
    du, dp, dx = report(g, o, "c2 mixed")
    assert du <= U_TOL and dp <= P_TOL and dx <= X_TOL


def test_mixed_tolerance_mode_reaches_rtol_and_divergence():
    inst = W.c2()
    over = {"vc_visc": 0, "vc_p": 0, "rtol": 1e-9, "max_cycles": 60}
    g, o = mixed_pair(inst, 2, over)
    sg, so = g.get_stats(), o.stats()
    print("cycles mixed %d/%d oracle %d/%d; res %.2e %.2e div %.2e %.2e" % (
        sg["cycles_visc"], sg["cycles_p"], so["cycles_visc"], so["cycles_p"], sg["res_visc"],
        sg["res_p"], sg["div_max"], so["div_max"]))
    assert sg["res_visc"] <= 1e-9 and sg["res_p"] <= 1e-9
    assert sg["div_max"] <= 10 * so["div_max"] + 1e-12
    du, dp, dx = report(g, o, "c2 mixed rtol")
    assert du <= 1e-12 and dp <= 1e-12


@pytest.mark.slow
def test_c3_mixed_two_steps():
    inst = W.c3(precision=1)
    g, o = mixed_pair(inst, 2)
    du, dp, dx = report(g, o, "c3 mixed")
    assert du <= U_TOL and dp <= P_TOL and dx <= X_TOL
