"""Solver tuning on the device: the coarse-grid viscosity scaling gamma_lh of
Eq. (ViscCoarseGrid), and the work-unit count of multigrid solves against the
number of levels (Sec. 4.3.1).

Both run whole solves through the C ABI on a live context; nothing here
computes on the host beyond bookkeeping.
"""
import numpy as np

from . import bfibm

GAMMA_CANDIDATES = (0.6, 0.7, 0.8, 0.9, 1.0)


def _viscous_cycles(ctx, u0):
    # the same start every trial: the step's right-hand side (already staged)
    # and the velocity u^n as the initial iterate
    for d in range(ctx.dim):
        ctx.set_field("ut", u0[d], d, 0)
    return ctx.solve_viscous(0)


def tune_gamma(ctx, candidates=GAMMA_CANDIDATES, passes=1):
    """Coordinate descent over gamma_lh, coarse level by coarse level: keep
    the value that needs the fewest viscous V-cycles to reach the context's
    rtol from the current state (the paper finds gamma in [0.7, 1] fastest).
    Leaves the best gamma set on the context and returns (gamma_levels,
    cycles before, cycles after)."""
    nlev = ctx.levels
    base = float(ctx.prm.get("gamma_coarse", 1.0))
    given = list(ctx.prm.get("gamma_levels", [])) + [0.0] * 8
    g = [0.0] * 8
    for l in range(1, nlev):
        g[l] = float(given[l]) if given[l] > 0 else base
    # count single V-cycles (several per FP64 residual would round the counts
    # up to their multiple)
    inner = int(ctx.prm.get("inner_cycles", 1))
    ctx.set_option(bfibm.OPT_INNER, 1)
    ctx.stage("rhs")
    u0 = [ctx.get_velocity(d) for d in range(ctx.dim)]
    ctx.set_gamma(g)
    start = best = _viscous_cycles(ctx, u0)
    for _ in range(passes):
        for l in range(1, nlev):
            for cand in candidates:
                if cand == g[l]:
                    continue
                trial = list(g)
                trial[l] = cand
                ctx.set_gamma(trial)
                cyc = _viscous_cycles(ctx, u0)
                if cyc < best:
                    best, g = cyc, trial
    ctx.set_gamma(g)
    ctx.set_option(bfibm.OPT_INNER, inner)
    # leave the viscous iterate as the step would find it
    for d in range(ctx.dim):
        ctx.set_field("ut", u0[d], d, 0)
    return g, start, best


def work_units_per_cycle(dim, nlev, nu1, nu2, coarse_sweeps):
    """Fine-grid relaxations one V-cycle costs: nu1 + nu2 sweeps on each of
    the first nlev - 1 levels, each coarser level 2^-dim of the one above, and
    the coarsest level's sweeps."""
    wu = sum((nu1 + nu2) * 2.0 ** (-dim * l) for l in range(nlev - 1))
    return wu + coarse_sweeps * 2.0 ** (-dim * (nlev - 1))


def work_units_vs_levels(inst, levels, which="pressure", rtol=1e-10, max_cycles=20000, steps=1):
    """For each allowed level count: the cycles one solve needs to reach rtol
    from the state after `steps` time steps, and their cost in work units."""
    rows = []
    for L in levels:
        prm = dict(inst["params"], mg_levels_max=int(L), vc_visc=0, vc_p=0, rtol=rtol,
                   max_cycles=max_cycles, precision=0)
        ctx = bfibm.load_instance(inst, prm_override=prm)
        ctx.set_option(bfibm.OPT_GRAPH, 0)
        ctx.step(steps)
        ctx.stage("rhs")
        if which == "pressure":
            ctx.solve_viscous(0)
            ctx.stage("divergence")
            cycles = ctx.solve_pressure(0)
            res = ctx.get_stats()["res_p"]
        else:
            cycles = ctx.solve_viscous(0)
            res = ctx.get_stats()["res_visc"]
        nlev = ctx.levels
        p = ctx.prm
        wu = cycles * work_units_per_cycle(p["dim"], nlev, p["nu1"], p["nu2"], p["coarse_sweeps"])
        rows.append({"levels_allowed": int(L), "levels": nlev, "cycles": cycles,
                     "work_units": wu, "rel_residual": res})
        ctx.close()
    return rows
