"""GPU parity over whole time steps: the CUDA library against the FP64 oracle
on the same seeded workloads. Tolerances (FP64 path): relative L2 of u and p
at most 1e-10, node positions within 1e-12, identical spring-break events
(springs within 1e-12 of the break threshold in the oracle are reported and
excluded)."""
import numpy as np
import pytest

from paper_1302_3663_gb300 import bfibm, workloads as W

from helpers import assert_close, pair
from test_gpu_stages import ragged_duct

pytestmark = pytest.mark.gpu

U_TOL = 1e-10
X_TOL = 1e-12


def near_threshold(o, inst, tol=1e-12):
    """Springs whose length is within tol (relative) of the break length."""
    X = o.nodes()
    prm = inst["params"]
    d = X[inst["ab"][:, 1]] - X[inst["ab"][:, 0]]
    for a in range(prm["dim"]):
        if prm["periodic"][a]:
            L = prm["n"][a] * prm["h"]
            d[:, a] -= L * np.round(d[:, a] / L)
    ratio = np.linalg.norm(d, axis=1) / ((1 + inst["brk"]) * inst["rest"])
    return set(np.flatnonzero(np.abs(ratio - 1) < tol))


def compare_state(g, o, inst, what):
    # components are compared on the scale of the whole velocity field (a
    # component that is zero up to rounding has no relative error of its own)
    D = g.dim
    uo = [o.get("u", d) for d in range(D)]
    scale = np.sqrt(sum(np.sum(u * u) for u in uo))
    for d in range(D):
        err = np.linalg.norm(g.get_velocity(d) - uo[d]) / scale
        assert err <= U_TOL, "%s u%d: relative L2 %.3e" % (what, d, err)
    assert_close(g.get_pressure(), o.get("p"), U_TOL, "%s p" % what)
    Xg, Xo = g.get_nodes(), o.nodes()
    assert np.abs(Xg - Xo).max() <= X_TOL, "%s nodes %.3e" % (what, np.abs(Xg - Xo).max())


def run_pair(inst, steps, override=None, chunk=1):
    g, o = pair(inst, override)
    skip = set()
    done = 0
    while done < steps:
        k = min(chunk, steps - done)
        g.step(k)
        o.step(k)
        done += k
        skip |= near_threshold(o, inst)
    ig, sg = g.get_broken()
    io, so = o.broken()
    ev_g = {(int(i), int(s)) for i, s in zip(ig, sg) if i not in skip}
    ev_o = {(int(i), int(s)) for i, s in zip(io, so) if i not in skip}
    assert ev_g == ev_o, (sorted(ev_g ^ ev_o)[:10], len(skip))
    compare_state(g, o, inst, inst["name"])
    return g, o, skip


def test_c1_full_run():
    inst = W.c1()
    g, o, skip = run_pair(inst, inst["steps"])
    st_g, st_o = g.get_stats(), o.stats()
    assert st_g["cycles_visc"] == st_o["cycles_visc"] == 3
    assert abs(st_g["kinetic"] - st_o["kinetic"]) <= 1e-12 * st_o["kinetic"]
    assert abs(st_g["res_p"] - st_o["res_p"]) <= 1e-6 * st_o["res_p"]
    assert st_g["step"] == inst["steps"]


def test_c1_breaking_springs():
    # weak springs (break strain 0.02) break within a few steps
    inst = W.c1()
    inst["brk"] = np.full(len(inst["rest"]), 0.02)
    inst["K"] = np.full(len(inst["rest"]), 5.0)
    g, o, skip = run_pair(inst, 12, {"dt": 4e-3})
    assert len(o.broken()[0]) > 5


def test_ragged_duct_run():
    inst = ragged_duct()
    g, o, skip = run_pair(inst, inst["steps"], chunk=5)


def test_c2_ten_steps():
    inst = W.c2()
    run_pair(inst, 10, chunk=5)


def test_no_nodes_duct():
    # without a biofilm the flow stays laminar: the cross components and the
    # pressure are rounding noise, compared in absolute terms
    inst = ragged_duct(nodes=0)
    inst["X"] = np.zeros((0, 3))
    inst["ab"] = np.zeros((0, 2), np.int32)
    inst["rest"] = inst["K"] = inst["brk"] = np.zeros(0)
    g, o = pair(inst)
    g.step(5)
    o.step(5)
    assert_close(g.get_velocity(2), o.get("u", 2), U_TOL, "flow component")
    for d in range(2):
        assert np.abs(g.get_velocity(d) - o.get("u", d)).max() < 1e-12
    assert np.abs(g.get_pressure() - o.get("p")).max() < 1e-10


def test_tolerance_mode_matches():
    inst = W.c1()
    g, o = pair(inst, {"vc_visc": 0, "vc_p": 0, "rtol": 1e-9, "max_cycles": 40})
    for k in range(3):
        g.step(1)
        o.step(1)
    sg, so = g.get_stats(), o.stats()
    assert abs(sg["cycles_p"] - so["cycles_p"]) <= 1 and abs(sg["cycles_visc"] - so["cycles_visc"]) <= 1
    assert sg["res_p"] <= 1e-9 and sg["res_visc"] <= 1e-9
    for d in range(2):
        assert_close(g.get_velocity(d), o.get("u", d), 1e-8, "u%d" % d)


def test_divergence_stop_rule_matches_the_oracle():
    # rtol 1e-9 alone leaves max |D.u| above 1e-10 on c1; with div_tol the
    # pressure solves run until (euler dt / sigma) max |r_p| <= div_tol on
    # both sides, so both take the same V-cycles and every projection of the
    # run stays within div_tol
    inst = W.c1()
    g, o = pair(inst, {"vc_visc": 0, "vc_p": 0, "rtol": 1e-9, "max_cycles": 60,
                       "div_tol": 1e-10})
    for k in range(3):
        assert g.step(1) == bfibm.OK
        o.step(1)
        sg, so = g.get_stats(), o.stats()
        assert sg["cycles_p"] == so["cycles_p"], (k, sg["cycles_p"], so["cycles_p"])
        assert sg["div_max_step"] <= 1e-10 and so["div_max"] <= 1e-10
    assert g.get_stats()["div_violations"] == 0
    compare_state(g, o, inst, "c1 with the divergence stop rule")


def test_graph_replay_equals_direct_launches():
    inst = W.c1()
    a = bfibm.load_instance(inst)
    b = bfibm.load_instance(inst)
    b.set_option(bfibm.OPT_GRAPH, 0)
    a.step(6)
    b.step(6)
    for d in range(2):
        assert_close(a.get_velocity(d), b.get_velocity(d), 1e-13, "graph u%d" % d)
    assert np.abs(a.get_nodes() - b.get_nodes()).max() < 1e-14


@pytest.mark.slow
def test_c3_full_size_two_steps_fp64():
    # the benchmark's grid (128 x 128 x 256, 20,000 nodes) at full size
    inst = W.c3(precision=0)
    run_pair(inst, 2, chunk=2)


@pytest.mark.parametrize("precision", [0, 1])
def test_device_loop_equals_host_loop_tolerance_mode(precision):
    # relative-residual solves run as conditional loops inside the step graph;
    # without the graph the host reads the norm after every cycle
    inst = W.c2()
    over = {"vc_visc": 0, "vc_p": 0, "rtol": 1e-9, "max_cycles": 60, "precision": precision}
    a = bfibm.load_instance(inst, prm_override=over)
    b = bfibm.load_instance(inst, prm_override=over)
    b.set_option(bfibm.OPT_GRAPH, 0)
    a.step(2)
    b.step(2)
    sa, sb = a.get_stats(), b.get_stats()
    assert sa["cycles_visc"] == sb["cycles_visc"] and sa["cycles_p"] == sb["cycles_p"]
    assert sa["cycles_visc"] > 3 and sa["res_visc"] <= 1e-9 and sa["res_p"] <= 1e-9
    for d in range(3):
        assert_close(a.get_velocity(d), b.get_velocity(d), 1e-12, "u%d" % d)
    assert_close(a.get_pressure(), b.get_pressure(), 1e-12, "p")


@pytest.mark.parametrize("precision", [0, 1])
def test_launch_accounting_of_device_loops(precision):
    # the step graph of the relative-residual mode loops on the device: its
    # loop bodies and the iterations they ran are counted
    inst = W.c2()
    over = {"vc_visc": 0, "vc_p": 0, "rtol": 1e-9, "max_cycles": 60, "precision": precision}
    c = bfibm.load_instance(inst, prm_override=over)
    c.step(1)
    a = c.launch_counts()
    c.step(2)
    b = c.launch_counts()
    st = c.get_stats()
    assert a["top"] > 0 and a["body_visc"] > 0 and a["body_p"] > 0
    assert b["iters_visc"] - a["iters_visc"] >= 2 * 3
    assert b["iters_p"] - a["iters_p"] >= 2
    assert b["iters_visc"] - a["iters_visc"] >= st["cycles_visc"]


def breaking_c1():
    inst = W.c1()
    inst["brk"] = np.full(len(inst["rest"]), 0.02)
    inst["K"] = np.full(len(inst["rest"]), 5.0)
    return inst, {"dt": 4e-3}, 12


def c2_plain():
    return W.c2(), {}, 6


@pytest.mark.parametrize("case", [breaking_c1, c2_plain], ids=["c1_breaking", "c2"])
@pytest.mark.parametrize("precision", [0, 1])
def test_repeated_runs_bit_identical(case, precision):
    # two runs of the same input agree bit for bit (node forces summed per node
    # in a fixed order, spread sums in fixed point)
    inst, over, steps = case()
    over = dict(over, precision=precision)
    runs = []
    for _ in range(2):
        c = bfibm.load_instance(inst, prm_override=over)
        c.step(steps)
        runs.append([c.get_velocity(d) for d in range(c.dim)] +
                    [c.get_pressure(), c.get_nodes(), c.get_node_forces(),
                     np.sort(c.get_broken()[0])])
        c.close()
    if case is breaking_c1:
        assert len(runs[0][-1]) > 5
    for x, y in zip(*runs):
        assert np.array_equal(x, y)


def test_paper_units_parity():
    # the paper's nondimensional units (sigma 0.05, Euler ~816, Re ~0.05)
    inst = W.paper_units_duct(e=32, nodes=800)
    run_pair(inst, 8, chunk=4)


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_resume_bit_identical(precision):
    # save the state mid-run, restore it into a fresh context: the resumed run
    # continues bit for bit (breaking springs included)
    inst, over, _ = breaking_c1()
    over = dict(over, precision=precision)
    a = bfibm.load_instance(inst, prm_override=over)
    a.step(5)
    ck = a.save_state()
    a.step(7)
    b = bfibm.load_instance(inst, prm_override=over)
    b.load_state(ck)
    assert b.get_stats()["step"] == 5
    b.step(7)
    assert b.get_stats()["step"] == a.get_stats()["step"] == 12
    for d in range(a.dim):
        assert np.array_equal(a.get_velocity(d), b.get_velocity(d))
    assert np.array_equal(a.get_pressure(), b.get_pressure())
    assert np.array_equal(a.get_nodes(), b.get_nodes())
    ea, eb = a.get_broken(), b.get_broken()
    assert len(ea[0]) > 5
    assert sorted(zip(*ea)) == sorted(zip(*eb))
    # a truncated checkpoint, or one of another grid, is refused
    with pytest.raises(bfibm.BfibmError):
        b.load_state(ck[:100])
    other = bfibm.load_instance(ragged_duct(), prm_override={"precision": precision})
    with pytest.raises(bfibm.BfibmError):
        other.load_state(ck)
    a.close()
    b.close()
    other.close()


def test_per_level_gamma_parity():
    # Eq. (ViscCoarseGrid) with a different gamma_lh on each coarse grid
    inst = W.c2()
    run_pair(inst, 4, {"gamma_levels": [0.0, 0.7, 0.9, 0.8, 1.0, 0.75]}, chunk=2)


def test_gamma_tuner_never_needs_more_cycles():
    from paper_1302_3663_gb300 import tuning
    inst = W.c2()
    c = bfibm.load_instance(inst, prm_override={"vc_visc": 0, "vc_p": 0, "rtol": 1e-9,
                                                "max_cycles": 80, "precision": 1})
    c.set_option(bfibm.OPT_GRAPH, 0)
    c.step(1)
    g, before, after = tuning.tune_gamma(c, candidates=(0.7, 1.0))
    assert after <= before
    assert all(0.0 < x <= 1.0 for x in g[1:c.levels])
    c.step(1)   # the tuned hierarchy steps on
    assert c.get_stats()["res_visc"] <= 1e-9
    c.close()
