"""The oracle's pins catch plausible mistakes. Each case plants one mistake
in a copy of the oracle's source (a dropped factor, a wrong sign, a flux
taken at the wrong edge, wrong transfer weights, a wrong kernel period,
spring tension or projection), builds that copy, and runs the pin tests of
the function it touches against it, through the oracle's build override: at
least one pin must fail. A control build of the unchanged source passes the
same pins, so a failure is the planted mistake's."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

from oracle import build as oracle_build
from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ADVECTION = "tests/test_oracle_advection.py"
MULTIGRID = "tests/test_oracle_multigrid.py"
OPERATORS = "tests/test_oracle_operators.py"
DELTA = "tests/test_oracle_delta.py"
TRANSFER = "tests/test_oracle_transfer.py"
FLOW = "tests/test_oracle_flow.py"
RHS = "tests/test_oracle_rhs.py"
OPEN = "tests/test_oracle_open.py"

MUTATIONS = {
    # Eq. NSdis1-1: the skew-symmetric advection is the mean of two halves
    "advection_dropped_half": (
        "  return 0.5 * (adv + cons);", "  return (adv + cons);", ADVECTION),
    "advection_sign_slip": (
        "adv += 0.5 * (Uhi * (up - udF) / h + Ulo * (udF - um) / h);",
        "adv += 0.5 * (Uhi * (up - udF) / h - Ulo * (udF - um) / h);", ADVECTION),
    "advection_upper_flux_at_lower_edge": (
        "Uhi = ue_avg_at_face(S, L, u[e], d, e, F, 1);",
        "Uhi = ue_avg_at_face(S, L, u[e], d, e, F, 0);", ADVECTION),
    # full-weighting restriction along the face axis: (1/4, 1/2, 1/4)
    "restriction_weights": (
        "double wgt = (o == 0) ? 0.5 : 0.25;", "double wgt = (o == 0) ? 0.6 : 0.2;", MULTIGRID),
    # linear prolongation: 3/4 on the parent cell
    "prolongation_parent_weight": (
        "idx[0] = I; w[0] = 0.75;", "idx[0] = I; w[0] = 0.7;", MULTIGRID),
    # a fine face on a coarse face takes its value
    "prolongation_coincident_face": (
        "if ((i & 1) == 0) { idx[0] = per ? wrapi(I, nc) : I; w[0] = 1.0; return 1; }",
        "if ((i & 1) == 0) { idx[0] = per ? wrapi(I, nc) : I; w[0] = 0.9; return 1; }",
        MULTIGRID),
    # the coarse edge viscosity is the mean of its two fine edges (3D)
    "edge_viscosity_mean_halved": (
        "double wt = S->D == 3 ? 0.5 : 1.0;", "double wt = S->D == 3 ? 0.25 : 1.0;", MULTIGRID),
    # Eq. divergenceGrad: the normal stress is 2 mu du_d/dx_d
    "viscous_normal_stress_without_2": (
        "double tau_p = 2.0 * mcp * (ud[LIc(L, Fp)] - ud[iF]) / h;",
        "double tau_p = mcp * (ud[LIc(L, Fp)] - ud[iF]) / h;", OPERATORS),
    # Eq. divergencePartial: the shear stress sums both cross derivatives
    "viscous_shear_sign": (
        "tau[side] = me * (dud_de + due_dd);", "tau[side] = me * (dud_de - due_dd);", OPERATORS),
    # Eq. NSdis4: the divergence of the two face fluxes
    "pressure_flux_sign": (
        "acc += (flux_hi - flux_lo) / h;", "acc += (flux_hi + flux_lo) / h;", OPERATORS),
    # Eq. PhiCosAlternative: the cosine kernel's period
    "phi2_period": (
        "if (a < 2.0) return 0.25 * (1.0 + cos(M_PI * r / 2.0));",
        "if (a < 2.0) return 0.25 * (1.0 + cos(M_PI * r / 2.2));", DELTA),
    # Peskin's phi1 (both branches) and the cosine kernel's amplitude
    "phi1_inner_branch_coefficient": (
        "  if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;",
        "  if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 3.9 * a * a)) / 8.0;", DELTA),
    "phi1_outer_branch_sign": (
        "  if (a < 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;",
        "  if (a < 2.0) return (5.0 - 2.0 * a + sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;", DELTA),
    "phi2_amplitude": (
        "if (a < 2.0) return 0.25 * (1.0 + cos(M_PI * r / 2.0));",
        "if (a < 2.0) return 0.3 * (1.0 + cos(M_PI * r / 2.0));", DELTA),
    # Eq. springF: Hookean tension on the stretch beyond the rest length
    "spring_tension_sign": (
        "double T = S->K[q] * (len - S->rest[q]);", "double T = S->K[q] * (len + S->rest[q]);",
        TRANSFER),
    # Eq. NSdis2: the projection subtracts the scaled pressure gradient
    "projection_sign": (
        "S->uvel[d][iF] = L->u[d][iF] - sc * L->beta[d][iF] * gp;",
        "S->uvel[d][iF] = L->u[d][iF] + sc * L->beta[d][iF] * gp;", FLOW),
    # Eq. NSdis4: the right-hand side sigma / (euler dt) D.u
    "divergence_scale_inverted": (
        "double sc = S->P.sigma / S->P.euler / S->P.dt;",
        "double sc = S->P.euler / S->P.sigma / S->P.dt;", FLOW),
    # reading 4: the initial velocity is ic_scale times the laminar profile
    "initial_velocity_without_ic_scale": (
        "        col[(long)b * n0 + a] = P->ic_scale * S->G / (P->inv_re * P->mu_f) * laminar_unit(S, y);",
        "        col[(long)b * n0 + a] = S->G / (P->inv_re * P->mu_f) * laminar_unit(S, y);", FLOW),
    # the pressure solve's divergence test: (euler dt / sigma) max |r_p|
    "divergence_test_without_euler_over_sigma": (
        "  double dscale = S->P.euler * S->P.dt / S->P.sigma;\n  for (cyc = 1; cyc <= maxc; ++cyc) {",
        "  double dscale = S->P.dt;\n  for (cyc = 1; cyc <= maxc; ++cyc) {", FLOW),
    # Sec. 3.5, the V-cycle: the coarse correction starts from zero, the
    # coarse right-hand side is the restricted residual, and the correction
    # is smoothed after it is added
    "pressure_coarse_guess_not_zeroed": (
        "  memset(Lc->p, 0, sizeof(double) * Lc->size);\n  vcycle_p(S, l + 1);",
        "  vcycle_p(S, l + 1);", OPERATORS),
    "pressure_restricts_the_iterate": (
        "  restrict_cell(S, L, Lc, L->pr, Lc->pf);", "  restrict_cell(S, L, Lc, L->p, Lc->pf);",
        OPERATORS),
    # Sec. 3.4, Eq. discrVelCouple: nodes move by dt / sigma times the
    # velocity interpolated with the delta of width h
    "node_velocity_with_the_spreading_width": (
        "S->U[3 * s + d] = interp_one(S, kind_face(d), S->uvel[d], &S->X[3 * s], P->h);",
        "S->U[3 * s + d] = interp_one(S, kind_face(d), S->uvel[d], &S->X[3 * s], P->omega);",
        TRANSFER),
    "nodes_moved_before_the_projection": (
        "    project(S);\n    interp_advance(S);", "    interp_advance(S);\n    project(S);",
        TRANSFER),
    "node_move_without_sigma": (
        "double c = P->dt / P->sigma;", "double c = P->dt;", TRANSFER),
    # Eqs. discrForceCouple, discrDensCouple, ViscExp with the widths of
    # Sec. 3.1: forces and density spread with omega, viscosity with omega_mu,
    # the biofilm's density (rho_ratio - 1) rho_f on d0^D
    "biofilm_density_without_d0": (
        "amp[s] = rho_b * P->d0_vol;", "amp[s] = rho_b;", TRANSFER),
    "biofilm_density_ratio": (
        "double rho_b = (P->rho_ratio - 1.0) * P->rho_f;",
        "double rho_b = P->rho_ratio * P->rho_f;", TRANSFER),
    "viscosity_spread_with_omega": (
        "spread_max(S, kind_cell(), L0->muc, P->omega_mu, P->mu_f, mu_max);",
        "spread_max(S, kind_cell(), L0->muc, P->omega, P->mu_f, mu_max);", TRANSFER),
    "force_spread_with_h": (
        "spread_sum(S, kind_face(d), S->frc[d], &S->F[d], 3, P->omega);",
        "spread_sum(S, kind_face(d), S->frc[d], &S->F[d], 3, P->h);", TRANSFER),
    # the edge viscosities spread on the edge grid; a node carried past a
    # wall stops on it and is counted
    "edge_viscosity_on_the_cell_grid": (
        "spread_max(S, kind_edge(d, e), me, P->omega_mu, P->mu_f, mu_max);",
        "spread_max(S, kind_cell(), me, P->omega_mu, P->mu_f, mu_max);", TRANSFER),
    "node_reflected_at_the_wall": (
        "        if (x < 0.0) { x = 0.0; S->st.clamped_total++; }",
        "        if (x < 0.0) { x = -x; S->st.clamped_total++; }", TRANSFER),
    # no-slip walls: no pressure flux through them, the tangential velocity's
    # odd mirror ghost at both, and its doubled diagonal weight
    "pressure_flux_through_the_top_wall": (
        "    if (per || c[a] < L->n[a] - 1) {", "    if (per || c[a] < L->n[a]) {", FLOW),
    "tangential_ghost_even_at_the_bottom_wall": (
        "  if (q < 0) { c[e] = 0; return -ud[LIc(L, c)]; }",
        "  if (q < 0) { c[e] = 0; return ud[LIc(L, c)]; }", FLOW),
    "tangential_ghost_zero_at_the_top_wall": (
        "  if (q >= L->n[e]) { c[e] = L->n[e] - 1; return -ud[LIc(L, c)]; }",
        "  if (q >= L->n[e]) { c[e] = L->n[e] - 1; return 0.0; }", FLOW),
    "wall_diagonal_weight_not_doubled": (
        "      double wgt = (e == S->open && q == ne) ? 0.0 : (wall ? 2.0 : 1.0);",
        "      double wgt = (e == S->open && q == ne) ? 0.0 : (wall ? 1.0 : 1.0);", OPERATORS),
    # the open duct of Sec. 3.6: du/dn = 0 beyond the outflow (even ghosts in
    # the restriction and the prolongation), the pressure held at kappa L
    "outflow_restriction_without_the_even_ghost": (
        "              if (d == S->open && q > nf) q = nf - 1;   /* even ghost beyond the outflow */",
        "              if (d == S->open && q > nf) q = nf;", OPEN),
    "outflow_tangential_prolongation_odd": (
        "                                     a == S->open ? 1.0 : -1.0, idx[a], w[a]);",
        "                                     -1.0, idx[a], w[a]);", OPEN),
    "outflow_advecting_velocity_past_the_ghost": (
        "  a1[d] = (d == S->open && F[d] == nd) ? nd - 1 : F[d];   /* even ghost beyond the outflow */",
        "  a1[d] = (d == S->open && F[d] == nd) ? nd : F[d];", OPEN),
    "outflow_plane_edge_in_the_viscous_diagonal": (
        "      double wgt = (e == S->open && q == ne) ? 0.0 : (wall ? 2.0 : 1.0);",
        "      double wgt = (e == S->open && q == ne) ? 1.0 : (wall ? 2.0 : 1.0);", OPEN),
    "inflow_scaled_by_ic_scale": (
        "            double v = P->ic_scale != 0.0 ? col[(long)b * n0 + a] / P->ic_scale",
        "            double v = P->ic_scale != 0.0 ? col[(long)b * n0 + a]", OPEN),
    "open_duct_keeps_the_body_force": (
        "      S->p_out = -S->G / P->euler * (P->n[fa] * P->h);\n      S->G = 0.0;",
        "      S->p_out = -S->G / P->euler * (P->n[fa] * P->h);", OPEN),
    "outflow_pressure_sign": (
        "      S->p_out = -S->G / P->euler * (P->n[fa] * P->h);",
        "      S->p_out = S->G / P->euler * (P->n[fa] * P->h);", OPEN),
    # 3D: the spring length takes all three axes, every edge grid gets its
    # viscosity, and the max-spread's z kernel sits on the grid's own stagger
    "spring_length_without_z": (
        "    len2 = len2 + dv[2] * dv[2];", "    len2 = len2;", TRANSFER),
    "yz_edge_viscosity_not_spread": (
        "    for (int e = d + 1; e < D; ++e) {", "    for (int e = d + 1; e < D - (d == 1); ++e) {",
        TRANSFER),
    "viscosity_z_kernel_stagger": (
        "    const double* X = &S->X[3 * s];\n    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};\n"
        "    for (int ax = 0; ax < D; ++ax) support(L, g, ax, X[ax], w, &lo[ax], &hi[ax]);\n"
        "    for (int k = lo[2]; k <= hi[2]; ++k) {\n      int kk = 0; double pz = 1.0;\n"
        "      if (D == 3) {\n        kk = kind_index(S, L, g, 2, k);\n        if (kk < 0) continue;\n"
        "        pz = phi(kind, ((k + 0.5 * g.stag[2]) * L->h - X[2]) / w);",
        "    const double* X = &S->X[3 * s];\n    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};\n"
        "    for (int ax = 0; ax < D; ++ax) support(L, g, ax, X[ax], w, &lo[ax], &hi[ax]);\n"
        "    for (int k = lo[2]; k <= hi[2]; ++k) {\n      int kk = 0; double pz = 1.0;\n"
        "      if (D == 3) {\n        kk = kind_index(S, L, g, 2, k);\n        if (kk < 0) continue;\n"
        "        pz = phi(kind, ((k + 0.5 * g.stag[1]) * L->h - X[2]) / w);", TRANSFER),
    # grid points beyond a wall do not exist: the kernel is cut there
    "kernel_folded_onto_the_wall": (
        "  if (i < 0 || i > hi) return -1;\n  return i;",
        "  if (i < 0) i = 0;\n  if (i > hi) i = hi;\n  return i;", TRANSFER),
    "cell_point_beyond_the_top_wall_kept": (
        "  int hi = g.stag[a] ? L->n[a] - 1 : L->n[a];", "  int hi = g.stag[a] ? L->n[a] : L->n[a];",
        TRANSFER),
    # Eq. ViscExp: the viscosity bump's amplitude (2 w)^D (mu_max - mu_out)
    "viscosity_amplitude_width": (
        "double coef = pow(2.0 * w, D) * (mu_max - mu_out);",
        "double coef = pow(w, D) * (mu_max - mu_out);", TRANSFER),
    # Eq. NSdis1-1: rhs = (rho sigma / dt) u - rho Adv(u) + c_f f + G
    "rhs_advection_without_density": (
        "S->uvel[d][iF] - S->rho[d][iF] * adv +", "S->uvel[d][iF] - adv +", RHS),
    "rhs_advection_sign": (
        "S->uvel[d][iF] - S->rho[d][iF] * adv +", "S->uvel[d][iF] + S->rho[d][iF] * adv +", RHS),
    "rhs_force_dropped": (
        "                         S->P.c_force * S->frc[d][iF] + g;", "                         g;",
        RHS),
    "mass_without_sigma": (
        "  double msc = S->P.sigma / S->P.dt;", "  double msc = 1.0 / S->P.dt;", RHS),
    "viscous_post_smoothing_skipped": (
        "  for (int d = 0; d < S->D; ++d) prolong_add_face(S, L, Lc, d, Lc->u[d], L->u[d]);\n"
        "  for (int it = 0; it < S->P.nu2; ++it) v_rbgs(S, l);",
        "  for (int d = 0; d < S->D; ++d) prolong_add_face(S, L, Lc, d, Lc->u[d], L->u[d]);",
        MULTIGRID),
}


def build_copy(src, out):
    cmd = (["gcc"] + oracle_build.FLAGS + ["-fopenmp", "-o", str(out), str(src), "-lm"])
    subprocess.run(cmd, check=True, capture_output=True)


def run_pins(lib, test_file):
    # one thread per child: the cases run side by side
    env = dict(os.environ, **{O.OVERRIDE_ENV: str(lib), "OMP_NUM_THREADS": "1"})
    return subprocess.run([sys.executable, "-m", "pytest", test_file, "-x", "-q", "-m", "not gpu",
                           "-p", "no:cacheprovider"], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=900)


def source():
    with open(oracle_build.SRC) as f:
        return f.read()


def run_case(tmp, name, text, test_files):
    """Build `text` as a copy of the oracle and run the pin files against it:
    (name, [(file, exit status, output tail)])."""
    src = os.path.join(tmp, name + ".c")
    with open(src, "w") as f:
        f.write(text)
    lib = os.path.join(tmp, "lib%s.so" % name)
    build_copy(src, lib)
    out = []
    for test_file in test_files:
        r = run_pins(lib, test_file)
        out.append((test_file, r.returncode, r.stdout[-1500:]))
    return name, out


def test_planted_mistakes_fail_a_pin_and_the_unchanged_copy_passes(tmp_path):
    text = source()
    cases = [("unchanged", text, (ADVECTION, MULTIGRID, OPERATORS, DELTA, TRANSFER, FLOW, RHS,
                                  OPEN))]
    for name in sorted(MUTATIONS):
        old, new, test_file = MUTATIONS[name]
        assert text.count(old) == 1, "%s: the mutation site is no longer unique" % name
        cases.append((name, text.replace(old, new), (test_file,)))
    workers = max(2, min(8, os.cpu_count() or 2))
    with ThreadPoolExecutor(workers) as pool:
        results = dict(pool.map(lambda c: run_case(str(tmp_path), *c), cases))
    for test_file, rc, tail in results.pop("unchanged"):
        assert rc == 0, "the unchanged copy fails %s:\n%s" % (test_file, tail)
    escaped = [(name, tail) for name, runs in results.items()
               for _, rc, tail in runs if rc != 1 or "failed" not in tail]
    assert not escaped, "no pin failed for: %s\n%s" % ([e[0] for e in escaped],
                                                      escaped[0][1] if escaped else "")
