"""The coarse-level cluster kernel (BFIBM_OPT_TAIL): the FP32 V-cycle levels
of at most a given number of cells, down to and with the FP64 coarsest solve,
in one launch per V-cycle. Its in-place red-black phases use the point
updates of the one-pass sweeps and its transfers and residuals those of the
per-level launches, so a context with it and one without must give the same
bits: whole tolerance-mode steps (flexible CG and defect correction), fixed
V-cycle counts, and a threshold that puts the whole V-cycle in the kernel."""
import numpy as np
import pytest

from paper_1302_3663_gb300 import bfibm, workloads as W

from test_gpu_serving import small_instance

pytestmark = pytest.mark.gpu

TOL_SOLVER = {"vc_visc": 0, "vc_p": 0, "rtol": 1e-11, "max_cycles": 100, "gamma_coarse": 0.8,
              "nu1": 2, "nu2": 2, "inner_cycles": 2, "krylov": 1, "div_tol": 1e-10}


def state(c):
    st = c.get_stats()
    return ([c.get_velocity(d) for d in range(3)] + [c.get_pressure(), c.get_nodes()],
            (st["cycles_visc"], st["cycles_p"], st["nonconv_total"]))


def run(inst, tail, steps):
    c = bfibm.load_instance(inst)
    c.set_option(bfibm.OPT_TAIL, tail)
    c.step(steps)
    out = state(c)
    lc = c.launch_counts()   # kernels of the step graph and of its loop bodies, times their runs
    n = steps * lc["top"] + lc["body_visc"] * lc["iters_visc"] + lc["body_p"] * lc["iters_p"]
    c.close()
    return out, n


def assert_same(a, b):
    for k, (x, y) in enumerate(zip(a[0], b[0])):
        assert np.isfinite(x).all()
        assert np.array_equal(x, y), "field %d: max |diff| %.3e" % (k, np.abs(x - y).max())
    assert a[1] == b[1]


@pytest.mark.parametrize("edge,krylov,tail", [(48, 1, 8192), (32, 0, 8192), (32, 1, 1 << 20),
                                              (48, 1, 60)])
def test_tail_bit_identical_to_launch_per_phase(edge, krylov, tail):
    inst = small_instance(0, e=edge)
    inst["params"].update(TOL_SOLVER, krylov=krylov)
    off, n_off = run(inst, 0, 3)
    on, n_on = run(inst, tail, 3)
    assert_same(on, off)
    assert n_on < n_off


def test_tail_on_the_64_cube_duct():
    inst = W.c2()
    inst["params"].update(TOL_SOLVER, precision=1)
    off, n_off = run(inst, 0, 2)
    on, n_on = run(inst, 8192, 2)
    assert_same(on, off)
    assert n_on < n_off


def test_tail_in_fixed_cycle_solves():
    inst = small_instance(1, e=32)
    inst["params"].update(vc_visc=3, vc_p=3, nu1=1, nu2=2, inner_cycles=1)
    off, _ = run(inst, 0, 2)
    on, _ = run(inst, 1 << 20, 2)   # every level in the cluster kernel
    assert_same(on, off)
