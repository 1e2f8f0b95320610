/*
 * bfibm_oracle.c -- plain FP64 CPU oracle for one time step of the biofilm
 * immersed-boundary method of Hammond, Stewart, Younger, Solomon and Bortz,
 * "Spatially heterogeneous biofilm simulations using an immersed boundary
 * method with Lagrangian nodes defined by bacterial locations" (arXiv:1302.3663).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load this library. It shares no code, header, table or
 * helper with the CUDA library; the two meet only through their inputs.
 *
 * Everything is written for clarity, not speed: plain loops over the grid in
 * the order the paper states the algorithm, FP64 throughout, compiled with
 * -ffp-contract=off so that no fused multiply-add changes a rounding.
 * OpenMP (when enabled) only splits loops whose iterations are independent
 * (one colour of a red-black sweep, residuals, transfers); every reduction is
 * serial, so results do not depend on the thread count.
 *
 * What each part follows:
 *   delta kernels phi1, phi2 ........... Eq. (PhiPeskin), Eq. (PhiCosAlternative)
 *   width-w delta ...................... Eq. (Dirac Delta Approx)
 *   force / density spread ............. Eq. (discrForceCouple), Eq. (discrDensCouple)
 *   velocity interpolation (width h) ... Eq. (discrVelCouple), Sec. 3.1
 *   viscosity field (max) .............. Eq. (ViscExp)
 *   Hookean springs and breaking ....... Eq. (springF), Eq. (defineK), Sec. 3.2
 *   momentum step ...................... Eq. (NSdis1-1) with Eq. (divergenceGrad),
 *                                         Eq. (divergencePartial) on a staggered grid
 *   projection ......................... Eq. (NSdis2)-(NSdis4)
 *   multigrid .......................... Sec. 3.5 (red-black Gauss-Seidel, full
 *                                         weighting, linear interpolation, V-cycles)
 *   coarse-grid viscosity scaling ...... Eq. (ViscCoarseGrid)
 *   node update ........................ explicit Euler, Sec. 3.4
 *   laminar initial condition .......... Eq. (2DlaminarSoln), Eq. (3DlaminarFlow)
 *
 * Grid conventions (the paper uses a collocated grid; this oracle uses the
 * staggered MAC grid the benchmark fixes, with these readings):
 *   - n[a] cells of width h along axis a; axis a is periodic or bounded by two
 *     no-slip walls at coordinates 0 and n[a]*h.
 *   - Every array of a level is stored with extent s[a] = n[a] + (wall ? 1 : 0)
 *     along axis a, x fastest. A cell-centred value uses indices [0, n[a]); a
 *     face or edge value along one of its face axes uses [0, s[a]), whose
 *     entries 0 and n[a] lie on the walls.
 *   - p, b, mu_c at cell centres; u_d on d-faces; mu_de on (d,e)-edges.
 *   - Walls: u_d = 0 on wall-normal faces (stored zeros); tangential velocity
 *     takes the mirror ghost -u (no slip); pressure flux through walls is zero.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#define OMP_FOR _Pragma("omp parallel for schedule(static)")
#else
#define OMP_FOR
#endif

#define OR_MAXLEV 8

/* ------------------------------------------------------------------------- */
/* Parameters (mirrored by ctypes in oracle.py; field order matters).        */
/* ------------------------------------------------------------------------- */
typedef struct {
  int32_t dim;            /* 2 or 3 */
  int32_t n[3];           /* cells per axis; n[2] = 1 when dim == 2 */
  int32_t periodic[3];    /* 1 = periodic axis, 0 = a pair of no-slip walls */
  int32_t flow_axis;      /* axis the body force pushes along */
  int32_t phi_kind;       /* 1 = phi1, Eq. (PhiPeskin); 2 = phi2, Eq. (PhiCosAlternative) */
  int32_t mg_levels_max;  /* at most 6 levels are useful, Sec. 4.3.1 */
  int32_t nu1, nu2;       /* pre- and post-smoothing sweeps */
  int32_t vc_visc, vc_p;  /* > 0: fixed V-cycle count; 0: relative-residual mode */
  int32_t max_cycles;     /* cap in relative-residual mode */
  int32_t coarse_sweeps;  /* red-black sweeps on the coarsest grid */
  int32_t pad0;
  double h;
  double rho_f, mu_f, rho_ratio, mu_ratio;
  double omega, omega_mu, d0_vol;
  double dt, sigma, euler, inv_re, c_force;
  double body_force;      /* G, used when u_center <= 0 */
  double u_center;        /* > 0: G such that the laminar centreline speed is u_center */
  double ic_scale;        /* initial velocity = ic_scale * laminar profile */
  double rtol;            /* relative residual target, 1e-9 in Sec. 4.1 */
  double gamma_coarse;    /* gamma of Eq. (ViscCoarseGrid) on every coarse level ... */
  double gamma_levels[8]; /* ... unless gamma_levels[l] > 0: gamma_lh of coarse level l */
  double div_tol;         /* > 0: relative-residual pressure solves also run until the
                             divergence the projection will leave is at most div_tol */
  int32_t open_flow;      /* 1: the flow axis is the open duct of Sec. 3.6 (inflow at 0,
                             outflow at n h) instead of periodic */
} or_params;

typedef struct {
  int32_t cycles_visc, cycles_p;
  int32_t broken_total, clamped_total;
  double res_visc, res_p;      /* final relative residuals ||r||_2 / ||f||_2 */
  double div_max;              /* max |D.u| after projection */
  double kinetic;              /* sum over faces of u_d^2 h^D */
  int64_t step;
} or_stats;

typedef struct {
  int n[3], s[3];
  long st[3];             /* strides: 1, s0, s0*s1 */
  long size;
  double h;
  double *p, *pf, *pr;    /* pressure iterate, right-hand side, residual */
  double *beta[3];        /* 1/rho on faces (restricted on coarse levels) */
  double *u[3], *uf[3], *ur[3];  /* viscous iterate, rhs, residual */
  double *m[3];           /* rho sigma / dt on faces */
  double *muc, *mue[3];   /* viscosity at centres and on edges (xy, xz, yz) */
} or_level;

typedef struct {
  or_params P;
  int D, L;
  or_level lev[OR_MAXLEV];
  double *uvel[3];        /* velocity state u^n */
  double *rho[3];         /* density on the d-faces */
  double *frc[3];         /* Eulerian force density on the d-faces */
  double G;               /* body force actually used (0 in an open duct) */
  int open;               /* the open flow axis, or -1 */
  double p_out;           /* open duct: the pressure held at the outflow */
  long eta;
  double *X, *U, *F;      /* eta x 3 */
  long nspring;
  int32_t *ab;
  double *rest, *K, *brk;
  int32_t *broken;
  long nev, capev;
  int32_t *ev_id, *ev_step;
  long step;
  int dirty;
  or_stats st;
} or_sim;

/* ------------------------------------------------------------------------- */
/* Delta kernels.                                                            */
/* ------------------------------------------------------------------------- */
/* Eq. (PhiPeskin): Peskin's four-point function, support |r| < 2. */
static double phi1(double r) {
  double a = fabs(r);
  if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
  if (a < 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
  return 0.0;
}
/* Eq. (PhiCosAlternative): the cosine function of Zhu and Peskin, |r| <= 2. */
static double phi2(double r) {
  double a = fabs(r);
  if (a < 2.0) return 0.25 * (1.0 + cos(M_PI * r / 2.0));
  return 0.0;
}
static double phi(int kind, double r) { return kind == 1 ? phi1(r) : phi2(r); }

double or_phi(int kind, double r) { return phi(kind, r); }

/* ------------------------------------------------------------------------- */
/* Small helpers.                                                            */
/* ------------------------------------------------------------------------- */
static int wrapi(int i, int n) { return ((i % n) + n) % n; }
static long LI(const or_level* L, int i, int j, int k) { return i + L->st[1] * j + L->st[2] * k; }
static long LIc(const or_level* L, const int c[3]) { return LI(L, c[0], c[1], c[2]); }
static int edge_id(int d, int e) { int a = d < e ? d : e, b = d < e ? e : d; return a + b - 1; }

static double* dalloc(long n) { return (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

static void level_alloc(or_sim* S, int l) {
  or_level* L = &S->lev[l];
  L->size = (long)L->s[0] * L->s[1] * L->s[2];
  L->st[0] = 1; L->st[1] = L->s[0]; L->st[2] = (long)L->s[0] * L->s[1];
  L->p = dalloc(L->size); L->pf = dalloc(L->size); L->pr = dalloc(L->size);
  L->muc = dalloc(L->size);
  for (int a = 0; a < 3; ++a) {
    L->beta[a] = dalloc(L->size); L->u[a] = dalloc(L->size); L->uf[a] = dalloc(L->size);
    L->ur[a] = dalloc(L->size); L->m[a] = dalloc(L->size); L->mue[a] = dalloc(L->size);
  }
}
static void level_free(or_level* L) {
  free(L->p); free(L->pf); free(L->pr); free(L->muc);
  for (int a = 0; a < 3; ++a) {
    free(L->beta[a]); free(L->u[a]); free(L->uf[a]); free(L->ur[a]); free(L->m[a]); free(L->mue[a]);
  }
}

/* Loop bounds of the unknown d-faces. Along an open flow axis the inflow face
   0 holds the prescribed velocity and the outflow face n is an unknown. */
static void face_range(const or_sim* S, const or_level* L, int d, int lo[3], int hi[3]) {
  for (int a = 0; a < 3; ++a) { lo[a] = 0; hi[a] = (a < S->D) ? L->n[a] : 1; }
  if (!S->P.periodic[d]) { lo[d] = 1; hi[d] = L->n[d] + (d == S->open ? 1 : 0); }
}

/* ------------------------------------------------------------------------- */
/* Laminar profile: Eq. (2DlaminarSoln) and Eq. (3DlaminarFlow).             */
/* With a body force G along the flow axis, Re^-1 mu Laplacian(u) = -G, u = 0 */
/* on the walls. 2D: u = G/(2 mu) y (H - y). 3D rectangle [0,a]x[0,b]: the    */
/* double sine series of Eq. (3DlaminarFlow) summed over one index in closed */
/* form, which converges exponentially.                                      */
/* ------------------------------------------------------------------------- */
static double laminar_unit(const or_sim* S, const double y[2]) {
  /* profile for G = 1, mu = 1; y = coordinates along the wall axes */
  const or_params* P = &S->P;
  if (S->D == 2) {
    int w = 1 - P->flow_axis;
    double H = P->n[w] * P->h;
    return 0.5 * y[0] * (H - y[0]);
  }
  int wa[2], q = 0;
  for (int a = 0; a < 3; ++a) if (a != P->flow_axis) wa[q++] = a;
  double A = P->n[wa[0]] * P->h, B = P->n[wa[1]] * P->h;
  double x = y[0], yy = y[1];
  double sum = 0.0;
  for (int n = 1; n <= 999; n += 2) {
    double k = n * M_PI / A;
    /* cosh(k(yy-B/2))/cosh(kB/2) written with exponentials that cannot overflow */
    double t1 = exp(k * (yy - B)) + exp(-k * yy);
    double t2 = 1.0 + exp(-k * B);
    sum += sin(k * x) * (t1 / t2) / ((double)n * n * n);
  }
  return 0.5 * x * (A - x) - 4.0 * A * A / (M_PI * M_PI * M_PI) * sum;
}

static void laminar_center_coords(const or_sim* S, double y[2]) {
  const or_params* P = &S->P;
  int q = 0;
  for (int a = 0; a < S->D; ++a) if (a != P->flow_axis) { y[q++] = 0.5 * P->n[a] * P->h; }
}

double or_laminar_unit(void* sim, double y0, double y1) {
  double y[2] = {y0, y1};
  return laminar_unit((or_sim*)sim, y);
}

static void compute_G(or_sim* S) {
  const or_params* P = &S->P;
  if (P->u_center > 0.0) {
    double yc[2];
    laminar_center_coords(S, yc);
    S->G = P->u_center * P->inv_re * P->mu_f / laminar_unit(S, yc);
  } else {
    S->G = P->body_force;
  }
}

/* ------------------------------------------------------------------------- */
/* Pressure operator: Eq. (divergenceGrad) with a = beta = 1/rho on faces.    */
/* ------------------------------------------------------------------------- */
static double p_apply_point(const or_sim* S, const or_level* L, const double* p,
                            const int c[3], double* diag) {
  double h = L->h, acc = 0.0, dg = 0.0;
  long ic = LIc(L, c);
  for (int a = 0; a < S->D; ++a) {
    int per = S->P.periodic[a];
    double flux_hi = 0.0, flux_lo = 0.0;
    if (per || c[a] < L->n[a] - 1) {
      int cp[3] = {c[0], c[1], c[2]};
      cp[a] = wrapi(c[a] + 1, L->n[a]);
      int fp[3] = {c[0], c[1], c[2]};
      fp[a] = per ? wrapi(c[a] + 1, L->n[a]) : c[a] + 1;
      double b = L->beta[a][LIc(L, fp)];
      flux_hi = b * (p[LIc(L, cp)] - p[ic]) / h;
      dg += b;
    } else if (a == S->open) {
      /* the outflow face: p held there (Sec. 3.6), ghost 2 p_out - p; the
         operator is the homogeneous part (ghost -p), p_out goes to the
         right-hand side */
      int fp[3] = {c[0], c[1], c[2]};
      fp[a] = c[a] + 1;
      double b = L->beta[a][LIc(L, fp)];
      flux_hi = b * (-p[ic] - p[ic]) / h;
      dg += 2.0 * b;
    }
    if (per || c[a] > 0) {
      int cm[3] = {c[0], c[1], c[2]};
      cm[a] = wrapi(c[a] - 1, L->n[a]);
      double b = L->beta[a][ic];
      flux_lo = b * (p[ic] - p[LIc(L, cm)]) / h;
      dg += b;
    }
    acc += (flux_hi - flux_lo) / h;
  }
  if (diag) *diag = -dg / (h * h);
  return acc;
}

void or_apply_p(void* sim, int l, const double* p, double* out) {
  or_sim* S = (or_sim*)sim;
  or_level* L = &S->lev[l];
  int nz = S->D == 3 ? L->n[2] : 1;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i) {
        int c[3] = {i, j, k};
        out[LIc(L, c)] = p_apply_point(S, L, p, c, NULL);
      }
}

static void p_residual(or_sim* S, int l) {
  or_level* L = &S->lev[l];
  int nz = S->D == 3 ? L->n[2] : 1;
  OMP_FOR
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i) {
        int c[3] = {i, j, k};
        long ic = LIc(L, c);
        L->pr[ic] = L->pf[ic] - p_apply_point(S, L, L->p, c, NULL);
      }
}

/* One red-black Gauss-Seidel sweep: colour = parity of i+j+k (Sec. 3.5). */
static void p_rbgs(or_sim* S, int l) {
  or_level* L = &S->lev[l];
  int nz = S->D == 3 ? L->n[2] : 1;
  for (int colour = 0; colour < 2; ++colour) {
    OMP_FOR
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < L->n[1]; ++j)
        for (int i = 0; i < L->n[0]; ++i) {
          if (((i + j + k) & 1) != colour) continue;
          int c[3] = {i, j, k};
          long ic = LIc(L, c);
          double dg;
          double Ap = p_apply_point(S, L, L->p, c, &dg);
          if (dg != 0.0) L->p[ic] += (L->pf[ic] - Ap) / dg;
        }
  }
}

static double cell_mean(const or_sim* S, const or_level* L, const double* a) {
  int nz = S->D == 3 ? L->n[2] : 1;
  double s = 0.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i) s += a[LI(L, i, j, k)];
  return s / ((double)L->n[0] * L->n[1] * nz);
}
static void cell_sub(const or_sim* S, const or_level* L, double* a, double v) {
  int nz = S->D == 3 ? L->n[2] : 1;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i) a[LI(L, i, j, k)] -= v;
}

/* ------------------------------------------------------------------------- */
/* Viscous operator: (m_d u_d - Re^-1 [div(mu (grad u + grad u^T))]_d)(F),    */
/* the staggered form of Eq. (divergenceGrad) + Eq. (divergencePartial):      */
/* tau_dd = 2 mu_c du_d/dx_d at centres, tau_de = mu_de (du_d/dx_e +          */
/* du_e/dx_d) at edges, [div tau]_d = sum_e d tau_de / dx_e.                  */
/* Returns the operator value; *diag receives its diagonal entry.            */
/* ------------------------------------------------------------------------- */
static double ud_at(const or_sim* S, const or_level* L, const double* ud, int d, const int F[3],
                    int e, int q) {
  /* u_d on its own grid at the point F with the e-centre index replaced by q
     (e != d); the no-slip mirror ghost applies beyond a wall along e. */
  int c[3] = {F[0], F[1], F[2]};
  (void)d;
  if (S->P.periodic[e]) { c[e] = wrapi(q, L->n[e]); return ud[LIc(L, c)]; }
  if (q < 0) { c[e] = 0; return -ud[LIc(L, c)]; }
  /* beyond the outflow of an open axis du_d/dx_e = 0 (Sec. 3.6): even ghost */
  if (q >= L->n[e] && e == S->open) { c[e] = L->n[e] - 1; return ud[LIc(L, c)]; }
  if (q >= L->n[e]) { c[e] = L->n[e] - 1; return -ud[LIc(L, c)]; }
  c[e] = q;
  return ud[LIc(L, c)];
}

static double v_apply_point(const or_sim* S, const or_level* L, double* const u[3], int d,
                            const int F[3], double* diag) {
  double h = L->h;
  const double* ud = u[d];
  int nd = L->n[d], perd = S->P.periodic[d];
  long iF = LIc(L, F);
  double dg = 0.0;
  /* normal stress at the two cells beside the face */
  int Cp[3] = {F[0], F[1], F[2]}, Cm[3] = {F[0], F[1], F[2]};
  Cm[d] = perd ? wrapi(F[d] - 1, nd) : F[d] - 1;
  int Fp[3] = {F[0], F[1], F[2]}, Fm[3] = {F[0], F[1], F[2]};
  Fp[d] = perd ? wrapi(F[d] + 1, nd) : F[d] + 1;
  Fm[d] = perd ? wrapi(F[d] - 1, nd) : F[d] - 1;
  /* the outflow face of an open axis: du_d/dx_d = 0 there, so the cell beyond
     mirrors the last cell (viscosity and the face beyond it) */
  const int outflow = d == S->open && F[d] == nd;
  if (outflow) { Cp[d] = nd - 1; Fp[d] = nd - 1; }
  double mcp = L->muc[LIc(L, Cp)], mcm = L->muc[LIc(L, Cm)];
  double tau_p = 2.0 * mcp * (ud[LIc(L, Fp)] - ud[iF]) / h;
  double tau_m = 2.0 * mcm * (ud[iF] - ud[LIc(L, Fm)]) / h;
  double V = (tau_p - tau_m) / h;
  dg += 2.0 * (mcp + mcm);
  /* shear stresses on the edges bounding the face along every other axis */
  for (int e = 0; e < S->D; ++e) {
    if (e == d) continue;
    int pere = S->P.periodic[e], ne = L->n[e];
    const double* ue = u[e];
    const double* mu = L->mue[edge_id(d, e)];
    double tau[2];
    for (int side = 0; side < 2; ++side) {
      int q = F[e] + side;            /* e-face index of this edge */
      int qq = pere ? wrapi(q, ne) : q;
      int E[3] = {F[0], F[1], F[2]};
      E[e] = qq;                      /* edge index: d-face F[d], e-face qq */
      double due_dd;                  /* du_e/dx_d on the edge */
      {
        int a1[3] = {F[0], F[1], F[2]}, a0[3] = {F[0], F[1], F[2]};
        a1[e] = qq; a0[e] = qq;
        a1[d] = outflow ? nd - 1 : F[d];   /* beyond the outflow u_e mirrors (even) */
        a0[d] = perd ? wrapi(F[d] - 1, nd) : F[d] - 1;
        due_dd = (ue[LIc(L, a1)] - ue[LIc(L, a0)]) / h;
      }
      double dud_de = (ud_at(S, L, ud, d, F, e, q) - ud_at(S, L, ud, d, F, e, q - 1)) / h;
      double me = mu[LIc(L, E)];
      tau[side] = me * (dud_de + due_dd);
      int wall = (!pere) && (q == 0 || q == ne);
      /* on the outflow plane the ghost is u_d itself: no diagonal weight */
      double wgt = (e == S->open && q == ne) ? 0.0 : (wall ? 2.0 : 1.0);
      dg += wgt * me;
    }
    V += (tau[1] - tau[0]) / h;
  }
  double m = L->m[d][iF];
  if (diag) *diag = m + S->P.inv_re * dg / (h * h);
  return m * ud[iF] - S->P.inv_re * V;
}

void or_apply_visc(void* sim, int l, double* const u[3], double* out[3]) {
  or_sim* S = (or_sim*)sim;
  or_level* L = &S->lev[l];
  for (int d = 0; d < S->D; ++d) {
    int lo[3], hi[3];
    face_range(S, L, d, lo, hi);
    for (long x = 0; x < L->size; ++x) out[d][x] = 0.0;
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) {
          int F[3] = {i, j, k};
          out[d][LIc(L, F)] = v_apply_point(S, L, u, d, F, NULL);
        }
  }
}

double or_visc_diag(void* sim, int l, int d, int i, int j, int k) {
  or_sim* S = (or_sim*)sim;
  int F[3] = {i, j, k};
  double dg;
  v_apply_point(S, &S->lev[l], S->lev[l].u, d, F, &dg);
  return dg;
}
double or_p_diag(void* sim, int l, int i, int j, int k) {
  or_sim* S = (or_sim*)sim;
  int c[3] = {i, j, k};
  double dg;
  p_apply_point(S, &S->lev[l], S->lev[l].p, c, &dg);
  return dg;
}

static void v_residual(or_sim* S, int l) {
  or_level* L = &S->lev[l];
  for (int d = 0; d < S->D; ++d) {
    int lo[3], hi[3];
    face_range(S, L, d, lo, hi);
    for (long x = 0; x < L->size; ++x) L->ur[d][x] = 0.0;
    OMP_FOR
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) {
          int F[3] = {i, j, k};
          long iF = LIc(L, F);
          L->ur[d][iF] = L->uf[d][iF] - v_apply_point(S, L, L->u, d, F, NULL);
        }
  }
}

/* Block red-black sweep: component x red then black, then y, then z; the
   other components are held at their latest values. */
static void v_rbgs(or_sim* S, int l) {
  or_level* L = &S->lev[l];
  for (int d = 0; d < S->D; ++d) {
    int lo[3], hi[3];
    face_range(S, L, d, lo, hi);
    for (int colour = 0; colour < 2; ++colour) {
      OMP_FOR
      for (int k = lo[2]; k < hi[2]; ++k)
        for (int j = lo[1]; j < hi[1]; ++j)
          for (int i = lo[0]; i < hi[0]; ++i) {
            if (((i + j + k) & 1) != colour) continue;
            int F[3] = {i, j, k};
            long iF = LIc(L, F);
            double dg;
            double Au = v_apply_point(S, L, L->u, d, F, &dg);
            L->u[d][iF] += (L->uf[d][iF] - Au) / dg;
          }
    }
  }
}

/* ------------------------------------------------------------------------- */
/* Grid transfers (Sec. 3.5: full weighting down, linear interpolation up).   */
/* Cell-centred: restriction averages the 2^D children; prolongation is       */
/* bi/trilinear (weights 3/4, 1/4 per axis) with a mirror ghost at walls      */
/* (even for pressure, odd for velocity).                                     */
/* Face-centred along its own axis: restriction (1/4, 1/2, 1/4), prolongation  */
/* linear (coincident face copied, midway face averaged).                      */
/* ------------------------------------------------------------------------- */
static void restrict_cell(const or_sim* S, const or_level* Lf, const or_level* Lc,
                          const double* fine, double* coarse) {
  int nz = S->D == 3 ? Lc->n[2] : 1;
  double w = 1.0 / (S->D == 3 ? 8.0 : 4.0);
  OMP_FOR
  for (int K = 0; K < nz; ++K)
    for (int J = 0; J < Lc->n[1]; ++J)
      for (int I = 0; I < Lc->n[0]; ++I) {
        double s = 0.0;
        int kz = S->D == 3 ? 2 : 1;
        for (int c = 0; c < kz; ++c)
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a)
              s += fine[LI(Lf, 2 * I + a, 2 * J + b, S->D == 3 ? 2 * K + c : 0)];
        coarse[LI(Lc, I, J, K)] = s * w;
      }
}

static void restrict_face(const or_sim* S, const or_level* Lf, const or_level* Lc, int d,
                          const double* fine, double* coarse) {
  int lo[3], hi[3];
  face_range(S, Lc, d, lo, hi);
  for (long x = 0; x < Lc->size; ++x) coarse[x] = 0.0;
  int nf = Lf->n[d], per = S->P.periodic[d];
  double wt = 1.0 / (S->D == 3 ? 4.0 : 2.0);
  OMP_FOR
  for (int K = lo[2]; K < hi[2]; ++K)
    for (int J = lo[1]; J < hi[1]; ++J)
      for (int I = lo[0]; I < hi[0]; ++I) {
        int C[3] = {I, J, K};
        double s = 0.0;
        int t1n = 2, t2n = S->D == 3 ? 2 : 1;
        int ta = -1, tb = -1;
        for (int a = 0; a < S->D; ++a) if (a != d) { if (ta < 0) ta = a; else tb = a; }
        for (int t2 = 0; t2 < t2n; ++t2)
          for (int t1 = 0; t1 < t1n; ++t1) {
            int f[3] = {0, 0, 0};
            f[ta] = 2 * C[ta] + t1;
            if (tb >= 0) f[tb] = 2 * C[tb] + t2;
            double along = 0.0;
            for (int o = -1; o <= 1; ++o) {
              int q = 2 * C[d] + o;
              if (d == S->open && q > nf) q = nf - 1;   /* even ghost beyond the outflow */
              f[d] = per ? wrapi(q, nf) : q;
              double wgt = (o == 0) ? 0.5 : 0.25;
              along += wgt * fine[LIc(Lf, f)];
            }
            s += along;
          }
        coarse[LIc(Lc, C)] = s * wt;
      }
}

/* 1D prolongation stencil for a cell-centred axis: fine index i -> two coarse
   indices and weights; returns the number of coarse points (1 or 2). The
   mirror signs (+1 even, -1 odd) apply beyond the lower and the upper end:
   at a wall +1 for the pressure and -1 for tangential velocity; at the
   outflow of an open axis -1 for the pressure (held there) and +1 for
   tangential velocity (du/dn = 0). */
static int prol_cell_1d(int i, int nc, int per, double mirror_lo, double mirror_hi, int idx[2],
                        double w[2]) {
  int I = i >> 1;
  int o = (i & 1) ? 1 : -1;
  int J = I + o;
  idx[0] = I; w[0] = 0.75;
  if (per) { idx[1] = wrapi(J, nc); w[1] = 0.25; return 2; }
  if (J < 0) { w[0] = 0.75 + 0.25 * mirror_lo; return 1; }
  if (J >= nc) { w[0] = 0.75 + 0.25 * mirror_hi; return 1; }
  idx[1] = J; w[1] = 0.25;
  return 2;
}
/* 1D prolongation along a face axis: fine face i from coarse faces. */
static int prol_face_1d(int i, int nc, int per, int idx[2], double w[2]) {
  int I = i >> 1;
  if ((i & 1) == 0) { idx[0] = per ? wrapi(I, nc) : I; w[0] = 1.0; return 1; }
  idx[0] = I; w[0] = 0.5;
  idx[1] = per ? wrapi(I + 1, nc) : I + 1; w[1] = 0.5;
  return 2;
}

static void prolong_add_cell(const or_sim* S, const or_level* Lf, const or_level* Lc,
                             const double* coarse, double* fine) {
  int nz = S->D == 3 ? Lf->n[2] : 1;
  OMP_FOR
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < Lf->n[1]; ++j)
      for (int i = 0; i < Lf->n[0]; ++i) {
        int fi[3] = {i, j, k};
        int idx[3][2]; double w[3][2]; int cnt[3] = {1, 1, 1};
        idx[2][0] = 0; w[2][0] = 1.0;
        for (int a = 0; a < S->D; ++a)
          cnt[a] = prol_cell_1d(fi[a], Lc->n[a], S->P.periodic[a], 1.0,
                                a == S->open ? -1.0 : 1.0, idx[a], w[a]);
        double v = 0.0;
        for (int c = 0; c < cnt[2]; ++c)
          for (int b = 0; b < cnt[1]; ++b)
            for (int a = 0; a < cnt[0]; ++a)
              v += w[0][a] * w[1][b] * w[2][c] * coarse[LI(Lc, idx[0][a], idx[1][b], idx[2][c])];
        fine[LI(Lf, i, j, k)] += v;
      }
}

static void prolong_add_face(const or_sim* S, const or_level* Lf, const or_level* Lc, int d,
                             const double* coarse, double* fine) {
  int lo[3], hi[3];
  face_range(S, Lf, d, lo, hi);
  OMP_FOR
  for (int k = lo[2]; k < hi[2]; ++k)
    for (int j = lo[1]; j < hi[1]; ++j)
      for (int i = lo[0]; i < hi[0]; ++i) {
        int fi[3] = {i, j, k};
        int idx[3][2]; double w[3][2]; int cnt[3] = {1, 1, 1};
        idx[2][0] = 0; w[2][0] = 1.0;
        for (int a = 0; a < S->D; ++a) {
          if (a == d) cnt[a] = prol_face_1d(fi[a], Lc->n[a], S->P.periodic[a], idx[a], w[a]);
          else cnt[a] = prol_cell_1d(fi[a], Lc->n[a], S->P.periodic[a], -1.0,
                                     a == S->open ? 1.0 : -1.0, idx[a], w[a]);
        }
        double v = 0.0;
        for (int c = 0; c < cnt[2]; ++c)
          for (int b = 0; b < cnt[1]; ++b)
            for (int a = 0; a < cnt[0]; ++a)
              v += w[0][a] * w[1][b] * w[2][c] * coarse[LI(Lc, idx[0][a], idx[1][b], idx[2][c])];
        fine[LI(Lf, i, j, k)] += v;
      }
}

/* ------------------------------------------------------------------------- */
/* Coefficients on the coarse grids: beta and m average the fine faces lying  */
/* on the coarse face; mu averages the fine points on the coarse point and is */
/* then scaled by gamma, Eq. (ViscCoarseGrid).                                */
/* ------------------------------------------------------------------------- */
static void restrict_face_coef(const or_sim* S, const or_level* Lf, const or_level* Lc, int d,
                               const double* fine, double* coarse) {
  int hi[3];
  for (int a = 0; a < 3; ++a) hi[a] = Lc->s[a];
  if (S->D == 2) hi[2] = 1;
  double wt = 1.0 / (S->D == 3 ? 4.0 : 2.0);
  for (int K = 0; K < hi[2]; ++K)
    for (int J = 0; J < hi[1]; ++J)
      for (int I = 0; I < hi[0]; ++I) {
        int C[3] = {I, J, K};
        /* along d the face index must be a stored face; across d, a cell */
        int ok = 1;
        for (int a = 0; a < S->D; ++a) {
          if (a == d) { if (C[a] > (S->P.periodic[a] ? Lc->n[a] - 1 : Lc->n[a])) ok = 0; }
          else if (C[a] >= Lc->n[a]) ok = 0;
        }
        if (!ok) { coarse[LIc(Lc, C)] = 0.0; continue; }
        double s = 0.0;
        int kz = S->D == 3 ? 2 : 1;
        for (int c = 0; c < kz; ++c)
          for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
              int f[3] = {2 * I + a, 2 * J + b, S->D == 3 ? 2 * K + c : 0};
              int off[3] = {a, b, c};
              if (off[d] != 0) continue;
              s += fine[LIc(Lf, f)];
            }
        coarse[LIc(Lc, C)] = s * wt;
      }
}

static void restrict_edge_coef(const or_sim* S, const or_level* Lf, const or_level* Lc, int d,
                               int e, const double* fine, double* coarse, double gamma) {
  int hi[3];
  for (int a = 0; a < 3; ++a) hi[a] = Lc->s[a];
  if (S->D == 2) hi[2] = 1;
  int t = 3 - d - e; /* third axis (3D) */
  double wt = S->D == 3 ? 0.5 : 1.0;
  for (int K = 0; K < hi[2]; ++K)
    for (int J = 0; J < hi[1]; ++J)
      for (int I = 0; I < hi[0]; ++I) {
        int C[3] = {I, J, K};
        int ok = 1;
        for (int a = 0; a < S->D; ++a) {
          int lim = (a == d || a == e) ? (S->P.periodic[a] ? Lc->n[a] - 1 : Lc->n[a]) : Lc->n[a] - 1;
          if (C[a] > lim) ok = 0;
        }
        if (!ok) { coarse[LIc(Lc, C)] = 0.0; continue; }
        double s = 0.0;
        int f[3] = {2 * I, 2 * J, S->D == 3 ? 2 * K : 0};
        if (S->D == 3) {
          for (int c = 0; c < 2; ++c) {
            int g[3] = {f[0], f[1], f[2]};
            g[t] = 2 * C[t] + c;
            s += fine[LIc(Lf, g)];
          }
        } else {
          s = fine[LIc(Lf, f)];
        }
        coarse[LIc(Lc, C)] = gamma * (s * wt);
      }
}

static void restrict_cell_coef(const or_sim* S, const or_level* Lf, const or_level* Lc,
                               const double* fine, double* coarse, double gamma) {
  restrict_cell(S, Lf, Lc, fine, coarse);
  int nz = S->D == 3 ? Lc->n[2] : 1;
  for (int K = 0; K < nz; ++K)
    for (int J = 0; J < Lc->n[1]; ++J)
      for (int I = 0; I < Lc->n[0]; ++I) coarse[LI(Lc, I, J, K)] *= gamma;
}

/* Fine coefficients from rho (Eq. NSdis1-1 and Eq. NSdis4) then the hierarchy. */
static void build_coefficients(or_sim* S) {
  or_level* L0 = &S->lev[0];
  double msc = S->P.sigma / S->P.dt;
  for (int d = 0; d < S->D; ++d)
    for (long x = 0; x < L0->size; ++x) {
      double r = S->rho[d][x];
      L0->beta[d][x] = r != 0.0 ? 1.0 / r : 0.0;
      L0->m[d][x] = r * msc;
    }
  for (int l = 1; l < S->L; ++l) {
    or_level *Lf = &S->lev[l - 1], *Lc = &S->lev[l];
    for (int d = 0; d < S->D; ++d) {
      restrict_face_coef(S, Lf, Lc, d, Lf->beta[d], Lc->beta[d]);
      restrict_face_coef(S, Lf, Lc, d, Lf->m[d], Lc->m[d]);
    }
    /* Eq. (ViscCoarseGrid): gamma_lh may differ per coarse grid lh */
    double gam = (l < 8 && S->P.gamma_levels[l] > 0.0) ? S->P.gamma_levels[l] : S->P.gamma_coarse;
    restrict_cell_coef(S, Lf, Lc, Lf->muc, Lc->muc, gam);
    for (int d = 0; d < S->D; ++d)
      for (int e = d + 1; e < S->D; ++e)
        restrict_edge_coef(S, Lf, Lc, d, e, Lf->mue[edge_id(d, e)], Lc->mue[edge_id(d, e)], gam);
  }
}

void or_build_coefficients(void* sim) { build_coefficients((or_sim*)sim); }

/* ------------------------------------------------------------------------- */
/* Multigrid V-cycles (Sec. 3.5).                                             */
/* ------------------------------------------------------------------------- */
static void vcycle_p(or_sim* S, int l) {
  or_level* L = &S->lev[l];
  if (l == S->L - 1) {
    /* coarsest grid: the singular Neumann/periodic problem needs a
       zero-mean right-hand side (an open duct's outflow pressure makes it
       regular); then a fixed number of sweeps */
    if (S->open < 0) cell_sub(S, L, L->pf, cell_mean(S, L, L->pf));
    /* with the outflow pressure held the slowest coarse mode is no longer the
       constant the mean removes: at least 2 n^2 sweeps along the open axis */
    int sweeps = S->P.coarse_sweeps;
    if (S->open >= 0 && sweeps < 2 * L->n[S->open] * L->n[S->open])
      sweeps = 2 * L->n[S->open] * L->n[S->open];
    for (int it = 0; it < sweeps; ++it) p_rbgs(S, l);
    return;
  }
  for (int it = 0; it < S->P.nu1; ++it) p_rbgs(S, l);
  p_residual(S, l);
  or_level* Lc = &S->lev[l + 1];
  restrict_cell(S, L, Lc, L->pr, Lc->pf);
  memset(Lc->p, 0, sizeof(double) * Lc->size);
  vcycle_p(S, l + 1);
  prolong_add_cell(S, L, Lc, Lc->p, L->p);
  for (int it = 0; it < S->P.nu2; ++it) p_rbgs(S, l);
}

static void vcycle_v(or_sim* S, int l) {
  or_level* L = &S->lev[l];
  if (l == S->L - 1) {
    for (int it = 0; it < S->P.coarse_sweeps; ++it) v_rbgs(S, l);
    return;
  }
  for (int it = 0; it < S->P.nu1; ++it) v_rbgs(S, l);
  v_residual(S, l);
  or_level* Lc = &S->lev[l + 1];
  for (int d = 0; d < S->D; ++d) {
    restrict_face(S, L, Lc, d, L->ur[d], Lc->uf[d]);
    memset(Lc->u[d], 0, sizeof(double) * Lc->size);
  }
  vcycle_v(S, l + 1);
  for (int d = 0; d < S->D; ++d) prolong_add_face(S, L, Lc, d, Lc->u[d], L->u[d]);
  for (int it = 0; it < S->P.nu2; ++it) v_rbgs(S, l);
}

static double norm2_cells(const or_sim* S, const or_level* L, const double* a) {
  int nz = S->D == 3 ? L->n[2] : 1;
  double s = 0.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i) { double v = a[LI(L, i, j, k)]; s += v * v; }
  return s;
}
static double norm2_faces(const or_sim* S, const or_level* L, double* const a[3]) {
  double s = 0.0;
  for (int d = 0; d < S->D; ++d) {
    int lo[3], hi[3];
    face_range(S, L, d, lo, hi);
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) { double v = a[d][LI(L, i, j, k)]; s += v * v; }
  }
  return s;
}

static double maxabs_cells(const or_sim* S, const or_level* L, const double* a) {
  int nz = S->D == 3 ? L->n[2] : 1;
  double m = 0.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i) {
        double v = fabs(a[LI(L, i, j, k)]);
        if (!(v <= m)) m = v;   /* a NaN propagates */
      }
  return m;
}

/* Pressure solve on level 0: ncycles > 0 fixed, else until ||r||/||f|| <= rtol
   and, when div_tol > 0, (euler dt / sigma) max |r| <= div_tol: after the
   projection, Eq. (NSdis2), D.u equals (euler dt / sigma) times the residual of
   Eq. (NSdis4), so this bounds max |D.u| by div_tol. The mean of p is
   re-zeroed after every cycle. Returns cycles used. */
static int solve_p(or_sim* S, int ncycles) {
  or_level* L = &S->lev[0];
  double fn = sqrt(norm2_cells(S, L, L->pf));
  int cyc = 0;
  double rel = 0.0;
  int maxc = ncycles > 0 ? ncycles : S->P.max_cycles;
  double dscale = S->P.euler * S->P.dt / S->P.sigma;
  for (cyc = 1; cyc <= maxc; ++cyc) {
    vcycle_p(S, 0);
    if (S->open < 0) cell_sub(S, L, L->p, cell_mean(S, L, L->p));
    if (ncycles <= 0) {
      p_residual(S, 0);
      rel = fn > 0.0 ? sqrt(norm2_cells(S, L, L->pr)) / fn : 0.0;
      int div_ok = S->P.div_tol <= 0.0 || dscale * maxabs_cells(S, L, L->pr) <= S->P.div_tol;
      if (rel <= S->P.rtol && div_ok) break;
    }
  }
  if (cyc > maxc) cyc = maxc;
  p_residual(S, 0);
  S->st.res_p = fn > 0.0 ? sqrt(norm2_cells(S, L, L->pr)) / fn : 0.0;
  S->st.cycles_p = cyc;
  return cyc;
}

static int solve_v(or_sim* S, int ncycles) {
  or_level* L = &S->lev[0];
  double fn = sqrt(norm2_faces(S, L, L->uf));
  int cyc = 0;
  int maxc = ncycles > 0 ? ncycles : S->P.max_cycles;
  for (cyc = 1; cyc <= maxc; ++cyc) {
    vcycle_v(S, 0);
    if (ncycles <= 0) {
      v_residual(S, 0);
      double rel = fn > 0.0 ? sqrt(norm2_faces(S, L, L->ur)) / fn : 0.0;
      if (rel <= S->P.rtol) break;
    }
  }
  if (cyc > maxc) cyc = maxc;
  v_residual(S, 0);
  S->st.res_visc = fn > 0.0 ? sqrt(norm2_faces(S, L, L->ur)) / fn : 0.0;
  S->st.cycles_visc = cyc;
  return cyc;
}

/* Grid transfers between level l and l+1 (for the pins of the transfers): comp < 0 is the
   cell-centred (pressure) pair, comp = d the face pair of velocity component d. The
   restriction overwrites `coarse`; the prolongation adds into `fine`. */
void or_restrict(void* sim, int l, int comp, const double* fine, double* coarse) {
  or_sim* S = (or_sim*)sim;
  if (comp < 0) restrict_cell(S, &S->lev[l], &S->lev[l + 1], fine, coarse);
  else restrict_face(S, &S->lev[l], &S->lev[l + 1], comp, fine, coarse);
}
void or_prolong_add(void* sim, int l, int comp, const double* coarse, double* fine) {
  or_sim* S = (or_sim*)sim;
  if (comp < 0) prolong_add_cell(S, &S->lev[l], &S->lev[l + 1], coarse, fine);
  else prolong_add_face(S, &S->lev[l], &S->lev[l + 1], comp, coarse, fine);
}
int or_solve_p(void* sim, int ncycles) { return solve_p((or_sim*)sim, ncycles); }
int or_solve_visc(void* sim, int ncycles) { return solve_v((or_sim*)sim, ncycles); }
void or_vcycle_p(void* sim) { vcycle_p((or_sim*)sim, 0); }
void or_vcycle_visc(void* sim) { vcycle_v((or_sim*)sim, 0); }
void or_rbgs_p(void* sim, int l) { p_rbgs((or_sim*)sim, l); }
void or_rbgs_visc(void* sim, int l) { v_rbgs((or_sim*)sim, l); }
void or_residual_p(void* sim, int l) { p_residual((or_sim*)sim, l); }
void or_residual_visc(void* sim, int l) { v_residual((or_sim*)sim, l); }

/* ------------------------------------------------------------------------- */
/* Momentum right-hand side, Eq. (NSdis1-1), explicit part:                    */
/*   rhs_d = (rho_d sigma/dt) u_d - rho_d Adv_d(u) + c_f f_d + G [d = flow]     */
/* Adv_d = 1/2 (u . D u_d + D . (u u_d)). On the paper's collocated grid D0 is  */
/* antisymmetric, so this skew form gives sum_x u_k Adv_k = 0 for every field.  */
/* The staggered reading keeps that: along each axis e, the advecting velocity */
/* U_e sits at the two flux points of the d-face (cell centres for e = d, the  */
/* (d,e)-edges otherwise) as a 2-point mean; the conservative half differences */
/* the fluxes U_e * (2-point mean of u_d); the advective half averages the two  */
/* one-sided products U_e * (one-sided difference of u_d).                      */
/* ------------------------------------------------------------------------- */
static double ue_avg_at_face(const or_sim* S, const or_level* L, const double* ue, int d, int e,
                             const int F[3], int qoff) {
  /* average of u_e over the two d-centres beside the d-face F, at e-face F[e]+qoff */
  int nd = L->n[d], ne = L->n[e];
  int q = F[e] + qoff;
  if (S->P.periodic[e]) q = wrapi(q, ne);
  int a1[3] = {F[0], F[1], F[2]}, a0[3] = {F[0], F[1], F[2]};
  a1[e] = q; a0[e] = q;
  a1[d] = (d == S->open && F[d] == nd) ? nd - 1 : F[d];   /* even ghost beyond the outflow */
  a0[d] = S->P.periodic[d] ? wrapi(F[d] - 1, nd) : F[d] - 1;
  return 0.5 * (ue[LIc(L, a0)] + ue[LIc(L, a1)]);
}

static double advection_point(const or_sim* S, const or_level* L, double* const u[3], int d,
                              const int F[3]) {
  double h = L->h;
  const double* ud = u[d];
  int nd = L->n[d], perd = S->P.periodic[d];
  double udF = ud[LIc(L, F)];
  const int outflow = d == S->open && F[d] == nd;   /* beyond it: even ghost */
  double adv = 0.0, cons = 0.0;
  for (int e = 0; e < S->D; ++e) {
    double up, um, Uhi, Ulo;   /* u_d one step up/down along e; U_e at the flux points */
    if (e == d) {
      int Fp[3] = {F[0], F[1], F[2]}, Fm[3] = {F[0], F[1], F[2]};
      Fp[d] = perd ? wrapi(F[d] + 1, nd) : (outflow ? nd - 1 : F[d] + 1);
      Fm[d] = perd ? wrapi(F[d] - 1, nd) : F[d] - 1;
      up = ud[LIc(L, Fp)];
      um = ud[LIc(L, Fm)];
      Uhi = 0.5 * (udF + up);   /* u_d at the cell centres beside the face */
      Ulo = 0.5 * (um + udF);
    } else {
      up = ud_at(S, L, ud, d, F, e, F[e] + 1);
      um = ud_at(S, L, ud, d, F, e, F[e] - 1);
      Uhi = ue_avg_at_face(S, L, u[e], d, e, F, 1);   /* u_e on the (d,e)-edges */
      Ulo = ue_avg_at_face(S, L, u[e], d, e, F, 0);
    }
    adv += 0.5 * (Uhi * (up - udF) / h + Ulo * (udF - um) / h);
    cons += (Uhi * 0.5 * (udF + up) - Ulo * 0.5 * (um + udF)) / h;
  }
  return 0.5 * (adv + cons);
}

void or_advection(void* sim, double* const u[3], double* out[3]) {
  or_sim* S = (or_sim*)sim;
  or_level* L = &S->lev[0];
  for (int d = 0; d < S->D; ++d) {
    int lo[3], hi[3];
    face_range(S, L, d, lo, hi);
    for (long x = 0; x < L->size; ++x) out[d][x] = 0.0;
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) {
          int F[3] = {i, j, k};
          out[d][LIc(L, F)] = advection_point(S, L, u, d, F);
        }
  }
}

static void momentum_rhs(or_sim* S) {
  or_level* L = &S->lev[0];
  for (int d = 0; d < S->D; ++d) {
    int lo[3], hi[3];
    face_range(S, L, d, lo, hi);
    for (long x = 0; x < L->size; ++x) { L->uf[d][x] = 0.0; L->u[d][x] = S->uvel[d][x]; }
    double g = (d == S->P.flow_axis) ? S->G : 0.0;
    OMP_FOR
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) {
          int F[3] = {i, j, k};
          long iF = LIc(L, F);
          double adv = advection_point(S, L, S->uvel, d, F);
          L->uf[d][iF] = L->m[d][iF] * S->uvel[d][iF] - S->rho[d][iF] * adv +
                         S->P.c_force * S->frc[d][iF] + g;
        }
  }
}

/* ------------------------------------------------------------------------- */
/* Divergence and projection, Eq. (NSdis2)-(NSdis4).                          */
/* ------------------------------------------------------------------------- */
static double div_cell(const or_sim* S, const or_level* L, double* const u[3], const int c[3]) {
  double s = 0.0;
  for (int a = 0; a < S->D; ++a) {
    int up[3] = {c[0], c[1], c[2]};
    up[a] = S->P.periodic[a] ? wrapi(c[a] + 1, L->n[a]) : c[a] + 1;
    s += (u[a][LIc(L, up)] - u[a][LIc(L, c)]) / L->h;
  }
  return s;
}

static void divergence_rhs(or_sim* S) {
  or_level* L = &S->lev[0];
  int nz = S->D == 3 ? L->n[2] : 1;
  double sc = S->P.sigma / S->P.euler / S->P.dt;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i) {
        int c[3] = {i, j, k};
        L->pf[LIc(L, c)] = sc * div_cell(S, L, L->u, c);
      }
  if (S->open < 0) {
    cell_sub(S, L, L->pf, cell_mean(S, L, L->pf));
  } else {
    /* the pressure held at the outflow: D.(beta D p) = b becomes
       A p = b - 2 beta p_out / h^2 in the last cells (A: ghost -p) */
    int o = S->open;
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < L->n[1]; ++j)
        for (int i = 0; i < L->n[0]; ++i) {
          int c[3] = {i, j, k};
          if (c[o] != L->n[o] - 1) continue;
          int f[3] = {i, j, k};
          f[o] = L->n[o];
          L->pf[LIc(L, c)] -= 2.0 * L->beta[o][LIc(L, f)] * S->p_out / (L->h * L->h);
        }
  }
}

static double max_div(const or_sim* S, double* const u[3]) {
  const or_level* L = &S->lev[0];
  int nz = S->D == 3 ? L->n[2] : 1;
  double m = 0.0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < L->n[1]; ++j)
      for (int i = 0; i < L->n[0]; ++i) {
        int c[3] = {i, j, k};
        double v = fabs(div_cell(S, L, u, c));
        if (v > m) m = v;
      }
  return m;
}

static void project(or_sim* S) {
  or_level* L = &S->lev[0];
  double sc = S->P.euler * S->P.dt / S->P.sigma;
  for (int d = 0; d < S->D; ++d) {
    int lo[3], hi[3];
    face_range(S, L, d, lo, hi);
    /* faces that are not unknowns keep the iterate's value: 0 on walls,
       the prescribed inflow on an open axis */
    for (long x = 0; x < L->size; ++x) S->uvel[d][x] = L->u[d][x];
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) {
          int F[3] = {i, j, k};
          int Cm[3] = {i, j, k};
          Cm[d] = S->P.periodic[d] ? wrapi(F[d] - 1, L->n[d]) : F[d] - 1;
          long iF = LIc(L, F);
          /* at the outflow the cell beyond holds the ghost 2 p_out - p */
          double pF = (d == S->open && F[d] == L->n[d]) ? 2.0 * S->p_out - L->p[LIc(L, Cm)]
                                                        : L->p[iF];
          double gp = (pF - L->p[LIc(L, Cm)]) / L->h;
          S->uvel[d][iF] = L->u[d][iF] - sc * L->beta[d][iF] * gp;
        }
  }
  S->st.div_max = max_div(S, S->uvel);
  double ke = 0.0, hD = pow(L->h, S->D);
  ke = norm2_faces(S, L, S->uvel) * hD;
  S->st.kinetic = ke;
}

/* ------------------------------------------------------------------------- */
/* Lagrangian-Eulerian transfers.                                             */
/* A grid "kind" gives, per axis, whether the points sit on faces (stag 0,    */
/* coordinate i h) or centres (stag 1, coordinate (i+1/2) h). Points whose    */
/* coordinate along a wall axis lies outside [0, L] do not exist.             */
/* ------------------------------------------------------------------------- */
typedef struct { int stag[3]; } gkind;

static gkind kind_face(int d) { gkind g = {{1, 1, 1}}; g.stag[d] = 0; return g; }
static gkind kind_cell(void) { gkind g = {{1, 1, 1}}; return g; }
static gkind kind_edge(int d, int e) { gkind g = {{1, 1, 1}}; g.stag[d] = 0; g.stag[e] = 0; return g; }

/* valid index of grid point i along axis a (wrapped), or -1 if it does not exist */
static int kind_index(const or_sim* S, const or_level* L, gkind g, int a, int i) {
  if (S->P.periodic[a]) return wrapi(i, L->n[a]);
  int hi = g.stag[a] ? L->n[a] - 1 : L->n[a];
  if (i < 0 || i > hi) return -1;
  return i;
}

/* support range of the width-w kernel around X along axis a (Eq. Dirac Delta Approx) */
static void support(const or_level* L, gkind g, int a, double X, double w, int* ilo, int* ihi) {
  double q = X / L->h - 0.5 * g.stag[a];
  double R = w / L->h;
  *ilo = (int)floor(q - 2.0 * R) + 1;
  *ihi = (int)ceil(q + 2.0 * R) - 1;
}

/* arr(x) += amp(s) * deltatilde(x - X_s, w) for every node, Eq. (discrForceCouple). */
static void spread_sum(or_sim* S, gkind g, double* arr, const double* amp, int ampstride,
                       double w) {
  const or_level* L = &S->lev[0];
  int D = S->D, kind = S->P.phi_kind;
  double winvD = 1.0 / pow(w, D);
  for (long s = 0; s < S->eta; ++s) {
    const double* X = &S->X[3 * s];
    double a = amp[s * ampstride];
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int ax = 0; ax < D; ++ax) support(L, g, ax, X[ax], w, &lo[ax], &hi[ax]);
    for (int k = lo[2]; k <= hi[2]; ++k) {
      int kk = 0; double pz = 1.0;
      if (D == 3) {
        kk = kind_index(S, L, g, 2, k);
        if (kk < 0) continue;
        pz = phi(kind, ((k + 0.5 * g.stag[2]) * L->h - X[2]) / w);
      }
      for (int j = lo[1]; j <= hi[1]; ++j) {
        int jj = kind_index(S, L, g, 1, j);
        if (jj < 0) continue;
        double py = phi(kind, ((j + 0.5 * g.stag[1]) * L->h - X[1]) / w);
        for (int i = lo[0]; i <= hi[0]; ++i) {
          int ii = kind_index(S, L, g, 0, i);
          if (ii < 0) continue;
          double px = phi(kind, ((i + 0.5 * g.stag[0]) * L->h - X[0]) / w);
          arr[LI(L, ii, jj, kk)] += a * (winvD * (px * py * pz));
        }
      }
    }
  }
}

/* Eq. (ViscExp): mu(x) = max_s [(2w)^D (mu_max - mu_out) deltatilde(x - X_s, w) + mu_out]. */
static void spread_max(or_sim* S, gkind g, double* arr, double w, double mu_out, double mu_max) {
  const or_level* L = &S->lev[0];
  int D = S->D, kind = S->P.phi_kind;
  double winvD = 1.0 / pow(w, D);
  double coef = pow(2.0 * w, D) * (mu_max - mu_out);
  for (long s = 0; s < S->eta; ++s) {
    const double* X = &S->X[3 * s];
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int ax = 0; ax < D; ++ax) support(L, g, ax, X[ax], w, &lo[ax], &hi[ax]);
    for (int k = lo[2]; k <= hi[2]; ++k) {
      int kk = 0; double pz = 1.0;
      if (D == 3) {
        kk = kind_index(S, L, g, 2, k);
        if (kk < 0) continue;
        pz = phi(kind, ((k + 0.5 * g.stag[2]) * L->h - X[2]) / w);
      }
      for (int j = lo[1]; j <= hi[1]; ++j) {
        int jj = kind_index(S, L, g, 1, j);
        if (jj < 0) continue;
        double py = phi(kind, ((j + 0.5 * g.stag[1]) * L->h - X[1]) / w);
        for (int i = lo[0]; i <= hi[0]; ++i) {
          int ii = kind_index(S, L, g, 0, i);
          if (ii < 0) continue;
          double px = phi(kind, ((i + 0.5 * g.stag[0]) * L->h - X[0]) / w);
          double cand = coef * (winvD * (px * py * pz)) + mu_out;
          long x = LI(L, ii, jj, kk);
          if (cand > arr[x]) arr[x] = cand;
        }
      }
    }
  }
}

/* U(s) = sum_x u(x) deltatilde(x - X_s, w) h^D, Eq. (discrVelCouple) (w = h there). */
static double interp_one(const or_sim* S, gkind g, const double* arr, const double* X, double w) {
  const or_level* L = &S->lev[0];
  int D = S->D, kind = S->P.phi_kind;
  double scale = pow(L->h / w, D);
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int ax = 0; ax < D; ++ax) support(L, g, ax, X[ax], w, &lo[ax], &hi[ax]);
  double v = 0.0;
  for (int k = lo[2]; k <= hi[2]; ++k) {
    int kk = 0; double pz = 1.0;
    if (D == 3) {
      kk = kind_index(S, L, g, 2, k);
      if (kk < 0) continue;
      pz = phi(kind, ((k + 0.5 * g.stag[2]) * L->h - X[2]) / w);
    }
    for (int j = lo[1]; j <= hi[1]; ++j) {
      int jj = kind_index(S, L, g, 1, j);
      if (jj < 0) continue;
      double py = phi(kind, ((j + 0.5 * g.stag[1]) * L->h - X[1]) / w);
      for (int i = lo[0]; i <= hi[0]; ++i) {
        int ii = kind_index(S, L, g, 0, i);
        if (ii < 0) continue;
        double px = phi(kind, ((i + 0.5 * g.stag[0]) * L->h - X[0]) / w);
        v += arr[LI(L, ii, jj, kk)] * (px * py * pz);
      }
    }
  }
  return v * scale;
}

/* Test entry: spread amp from the current nodes onto a grid of the given kind
   (kind 0..2 = faces of axis d, 3 = centres, 4.. = edges) with width w. */
static gkind kind_from_id(int id) {
  if (id < 3) return kind_face(id);
  if (id == 3) return kind_cell();
  if (id == 4) return kind_edge(0, 1);
  if (id == 5) return kind_edge(0, 2);
  return kind_edge(1, 2);
}
void or_spread_sum(void* sim, int kind_id, double* arr, const double* amp, double w) {
  or_sim* S = (or_sim*)sim;
  spread_sum(S, kind_from_id(kind_id), arr, amp, 1, w);
}
void or_spread_max(void* sim, int kind_id, double* arr, double w, double mu_out, double mu_max) {
  or_sim* S = (or_sim*)sim;
  spread_max(S, kind_from_id(kind_id), arr, w, mu_out, mu_max);
}
void or_interp(void* sim, int kind_id, const double* arr, double w, double* out) {
  or_sim* S = (or_sim*)sim;
  for (long s = 0; s < S->eta; ++s) out[s] = interp_one(S, kind_from_id(kind_id), arr, &S->X[3 * s], w);
}

/* ------------------------------------------------------------------------- */
/* Springs, Eq. (springF): F(s) = sum_k I_sk (d_sk/|d_sk|) K_sk (|d_sk| - r_sk). */
/* A spring breaks for good once |d| > (1 + eps_b) r (the paper: eps_b = 1,   */
/* i.e. twice the rest length, Sec. 3.2). Minimum image on periodic axes.     */
/* ------------------------------------------------------------------------- */
static void spring_forces(or_sim* S) {
  int D = S->D;
  memset(S->F, 0, sizeof(double) * 3 * S->eta);
  for (long q = 0; q < S->nspring; ++q) {
    if (S->broken[q]) continue;
    int a = S->ab[2 * q], b = S->ab[2 * q + 1];
    double dv[3] = {0.0, 0.0, 0.0};
    for (int ax = 0; ax < D; ++ax) {
      double v = S->X[3 * b + ax] - S->X[3 * a + ax];
      if (S->P.periodic[ax]) {
        double Lx = S->P.n[ax] * S->P.h;
        if (v > 0.5 * Lx) v -= Lx;
        else if (v < -0.5 * Lx) v += Lx;
      }
      dv[ax] = v;
    }
    double len2 = dv[0] * dv[0] + dv[1] * dv[1];
    len2 = len2 + dv[2] * dv[2];
    double thr = (1.0 + S->brk[q]) * S->rest[q];
    if (len2 > thr * thr) {
      S->broken[q] = 1;
      if (S->nev == S->capev) {
        S->capev = S->capev ? 2 * S->capev : 64;
        S->ev_id = (int32_t*)realloc(S->ev_id, sizeof(int32_t) * S->capev);
        S->ev_step = (int32_t*)realloc(S->ev_step, sizeof(int32_t) * S->capev);
      }
      S->ev_id[S->nev] = (int32_t)q;
      S->ev_step[S->nev] = (int32_t)S->step;
      S->nev++;
      continue;
    }
    double len = sqrt(len2);
    if (len == 0.0) continue;
    double T = S->K[q] * (len - S->rest[q]);
    for (int ax = 0; ax < D; ++ax) {
      double f = T * dv[ax] / len;
      S->F[3 * a + ax] += f;
      S->F[3 * b + ax] -= f;
    }
  }
}

/* Break test + forces, then f, rho, mu on the grid (Eqs. discrForceCouple,
   discrDensCouple, ViscExp), then the coefficient hierarchy. */
static void refresh_lagrangian(or_sim* S) {
  or_level* L0 = &S->lev[0];
  const or_params* P = &S->P;
  int D = S->D;
  spring_forces(S);
  double rho_b = (P->rho_ratio - 1.0) * P->rho_f;
  double mu_max = P->mu_ratio * P->mu_f;
  double* amp = dalloc(S->eta);
  for (long s = 0; s < S->eta; ++s) amp[s] = rho_b * P->d0_vol;
  for (int d = 0; d < D; ++d) {
    memset(S->frc[d], 0, sizeof(double) * L0->size);
    spread_sum(S, kind_face(d), S->frc[d], &S->F[d], 3, P->omega);
    for (long x = 0; x < L0->size; ++x) S->rho[d][x] = 0.0;
    spread_sum(S, kind_face(d), S->rho[d], amp, 1, P->omega);
    for (long x = 0; x < L0->size; ++x) S->rho[d][x] += P->rho_f;
  }
  free(amp);
  for (long x = 0; x < L0->size; ++x) L0->muc[x] = P->mu_f;
  spread_max(S, kind_cell(), L0->muc, P->omega_mu, P->mu_f, mu_max);
  for (int d = 0; d < D; ++d)
    for (int e = d + 1; e < D; ++e) {
      double* me = L0->mue[edge_id(d, e)];
      for (long x = 0; x < L0->size; ++x) me[x] = P->mu_f;
      spread_max(S, kind_edge(d, e), me, P->omega_mu, P->mu_f, mu_max);
    }
  build_coefficients(S);
}

/* Interpolate u^{n+1} at X^n with the width-h kernel and move the nodes by
   explicit Euler, X^{n+1} = X^n + (dt/sigma) U^{n+1} (Sec. 3.4). */
static void interp_advance(or_sim* S) {
  int D = S->D;
  const or_params* P = &S->P;
  double c = P->dt / P->sigma;
  for (long s = 0; s < S->eta; ++s)
    for (int d = 0; d < D; ++d) S->U[3 * s + d] = interp_one(S, kind_face(d), S->uvel[d], &S->X[3 * s], P->h);
  for (long s = 0; s < S->eta; ++s)
    for (int d = 0; d < D; ++d) {
      double x = S->X[3 * s + d] + c * S->U[3 * s + d];
      double Lx = P->n[d] * P->h;
      if (P->periodic[d]) {
        if (x >= Lx) x -= Lx;
        else if (x < 0.0) x += Lx;
      } else {
        if (x < 0.0) { x = 0.0; S->st.clamped_total++; }
        else if (x > Lx) { x = Lx; S->st.clamped_total++; }
      }
      S->X[3 * s + d] = x;
    }
}

/* ------------------------------------------------------------------------- */
/* Public oracle API (ctypes).                                                */
/* ------------------------------------------------------------------------- */
void* or_create(const or_params* P) {
  if (!P || (P->dim != 2 && P->dim != 3)) return NULL;
  or_sim* S = (or_sim*)calloc(1, sizeof(or_sim));
  S->P = *P;
  S->D = P->dim;
  if (S->D == 2) { S->P.n[2] = 1; S->P.periodic[2] = 1; }
  /* levels: halve while every axis is even, the halved minimum is >= 2 and
     every halved periodic axis stays even (so that red-black colouring is
     consistent across the periodic wrap) */
  int n[3] = {S->P.n[0], S->P.n[1], S->P.n[2]};
  S->L = 0;
  for (;;) {
    or_level* L = &S->lev[S->L];
    for (int a = 0; a < 3; ++a) {
      L->n[a] = n[a];
      L->s[a] = (a < S->D && !S->P.periodic[a]) ? n[a] + 1 : n[a];
    }
    if (S->D == 2) { L->n[2] = 1; L->s[2] = 1; }
    L->h = P->h * (double)(1 << S->L);
    level_alloc(S, S->L);
    S->L++;
    if (S->L >= P->mg_levels_max || S->L >= OR_MAXLEV) break;
    int ok = 1, mn = 1 << 30;
    for (int a = 0; a < S->D; ++a) {
      if (n[a] % 2) ok = 0;
      if (n[a] / 2 < mn) mn = n[a] / 2;
      if (S->P.periodic[a] && (n[a] / 2) % 2) ok = 0;
    }
    if (!ok || mn < 2) break;
    for (int a = 0; a < S->D; ++a) n[a] /= 2;
  }
  long sz = S->lev[0].size;
  for (int a = 0; a < 3; ++a) { S->uvel[a] = dalloc(sz); S->rho[a] = dalloc(sz); S->frc[a] = dalloc(sz); }
  S->open = (P->open_flow && !S->P.periodic[P->flow_axis]) ? P->flow_axis : -1;
  compute_G(S);
  /* laminar initial velocity along the flow axis, evaluated at the faces; the
     profile depends only on the wall-axis coordinates, so it is summed once
     per column and copied along the flow axis */
  {
    or_level* L = &S->lev[0];
    int fa = P->flow_axis, lo[3], hi[3];
    face_range(S, L, fa, lo, hi);
    int ta[2] = {0, 0}, q = 0;
    for (int a = 0; a < S->D; ++a) if (a != fa) ta[q++] = a;
    int n0 = L->n[ta[0]], n1 = (S->D == 3) ? L->n[ta[1]] : 1;
    double* col = dalloc((long)n0 * n1);
    for (int b = 0; b < n1; ++b)
      for (int a = 0; a < n0; ++a) {
        double y[2] = {(a + 0.5) * L->h, (b + 0.5) * L->h};
        col[(long)b * n0 + a] = P->ic_scale * S->G / (P->inv_re * P->mu_f) * laminar_unit(S, y);
      }
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) {
          int c[3] = {i, j, k};
          int a = c[ta[0]], b = (S->D == 3) ? c[ta[1]] : 0;
          S->uvel[fa][LIc(L, c)] = col[(long)b * n0 + a];
        }
    if (S->open >= 0) {
      /* Sec. 3.6: the inflow face holds the laminar profile itself, and the
         pressure falls linearly along the duct, Eq. (pressLam): p(0) = 0,
         eps kappa = -G (the pressure gradient that drives the same flow as
         the body force G), so p_out = kappa L; no body force acts */
      lo[fa] = 0;
      hi[fa] = 1;
      for (int k = lo[2]; k < hi[2]; ++k)
        for (int j = lo[1]; j < hi[1]; ++j)
          for (int i = lo[0]; i < hi[0]; ++i) {
            int c[3] = {i, j, k};
            int a = c[ta[0]], b = (S->D == 3) ? c[ta[1]] : 0;
            double v = P->ic_scale != 0.0 ? col[(long)b * n0 + a] / P->ic_scale
                                           : S->G / (P->inv_re * P->mu_f) *
                                                 laminar_unit(S, (double[2]){(a + 0.5) * L->h,
                                                                            (b + 0.5) * L->h});
            S->uvel[fa][LIc(L, c)] = v;
          }
      S->p_out = -S->G / P->euler * (P->n[fa] * P->h);
      S->G = 0.0;
    }
    free(col);
  }
  /* uniform fluid until nodes arrive */
  for (int d = 0; d < 3; ++d) for (long x = 0; x < sz; ++x) S->rho[d][x] = P->rho_f;
  for (long x = 0; x < sz; ++x) S->lev[0].muc[x] = P->mu_f;
  for (int e = 0; e < 3; ++e) for (long x = 0; x < sz; ++x) S->lev[0].mue[e][x] = P->mu_f;
  build_coefficients(S);
  S->dirty = 1;
  return S;
}

void or_destroy(void* sim) {
  or_sim* S = (or_sim*)sim;
  if (!S) return;
  for (int l = 0; l < S->L; ++l) level_free(&S->lev[l]);
  for (int a = 0; a < 3; ++a) { free(S->uvel[a]); free(S->rho[a]); free(S->frc[a]); }
  free(S->X); free(S->U); free(S->F);
  free(S->ab); free(S->rest); free(S->K); free(S->brk); free(S->broken);
  free(S->ev_id); free(S->ev_step);
  free(S);
}

int or_levels(void* sim) { return ((or_sim*)sim)->L; }
double or_body_force(void* sim) { return ((or_sim*)sim)->G; }
double or_outflow_pressure(void* sim) { return ((or_sim*)sim)->p_out; }
void or_level_dims(void* sim, int l, int32_t* n, int32_t* s) {
  or_sim* S = (or_sim*)sim;
  for (int a = 0; a < 3; ++a) { n[a] = S->lev[l].n[a]; s[a] = S->lev[l].s[a]; }
}

void or_set_nodes(void* sim, long eta, const double* X) {
  or_sim* S = (or_sim*)sim;
  free(S->X); free(S->U); free(S->F);
  S->eta = eta;
  S->X = dalloc(3 * eta); S->U = dalloc(3 * eta); S->F = dalloc(3 * eta);
  for (long s = 0; s < eta; ++s)
    for (int a = 0; a < S->D; ++a) S->X[3 * s + a] = X[S->D * s + a];
  S->dirty = 1;
}

void or_set_springs(void* sim, long m, const int32_t* ab, const double* rest, const double* K,
                    const double* brk) {
  or_sim* S = (or_sim*)sim;
  free(S->ab); free(S->rest); free(S->K); free(S->brk); free(S->broken);
  S->nspring = m;
  S->ab = (int32_t*)malloc(sizeof(int32_t) * 2 * (m > 0 ? m : 1));
  S->rest = dalloc(m); S->K = dalloc(m); S->brk = dalloc(m);
  S->broken = (int32_t*)calloc((size_t)(m > 0 ? m : 1), sizeof(int32_t));
  if (m > 0) {
    memcpy(S->ab, ab, sizeof(int32_t) * 2 * m);
    memcpy(S->rest, rest, sizeof(double) * m);
    memcpy(S->K, K, sizeof(double) * m);
    memcpy(S->brk, brk, sizeof(double) * m);
  }
  S->dirty = 1;
}

void or_refresh(void* sim) {
  or_sim* S = (or_sim*)sim;
  refresh_lagrangian(S);
  S->dirty = 0;
}

/* One time step in the order of Sec. 3.4: u~ (Eq. NSdis1-1), p (Eq. NSdis4),
   u (Eq. NSdis2), U and X, then F, f, rho and mu at the new positions. */
void or_step(void* sim, int nsteps) {
  or_sim* S = (or_sim*)sim;
  if (S->dirty) or_refresh(S);
  for (int it = 0; it < nsteps; ++it) {
    momentum_rhs(S);
    solve_v(S, S->P.vc_visc);
    divergence_rhs(S);
    solve_p(S, S->P.vc_p);
    project(S);
    interp_advance(S);
    S->step++;
    refresh_lagrangian(S);
  }
  S->st.step = S->step;
}

/* stage entries, for operator-level comparisons */
void or_stage_rhs(void* sim) { momentum_rhs((or_sim*)sim); }
void or_stage_divergence(void* sim) { divergence_rhs((or_sim*)sim); }
void or_stage_project(void* sim) { project((or_sim*)sim); }
void or_stage_interp_advance(void* sim) { interp_advance((or_sim*)sim); }
void or_stage_springs(void* sim) { spring_forces((or_sim*)sim); }

/* Field access. which: 0 U state, 1 viscous iterate, 2 viscous rhs, 3 p iterate,
   4 p rhs, 5 rho, 6 force density, 7 mu_c, 8 mu edge, 9 beta, 10 m,
   11 viscous residual, 12 p residual. Arrays are exchanged in storage layout
   (extent s[a] along every axis, x fastest). */
static double* field_ptr(or_sim* S, int which, int comp, int l) {
  or_level* L = &S->lev[l];
  switch (which) {
    case 0: return S->uvel[comp];
    case 1: return L->u[comp];
    case 2: return L->uf[comp];
    case 3: return L->p;
    case 4: return L->pf;
    case 5: return S->rho[comp];
    case 6: return S->frc[comp];
    case 7: return L->muc;
    case 8: return L->mue[comp];
    case 9: return L->beta[comp];
    case 10: return L->m[comp];
    case 11: return L->ur[comp];
    case 12: return L->pr;
  }
  return NULL;
}
long or_level_size(void* sim, int l) { return ((or_sim*)sim)->lev[l].size; }
int or_get_field(void* sim, int which, int comp, int l, double* out) {
  or_sim* S = (or_sim*)sim;
  double* p = field_ptr(S, which, comp, l);
  if (!p) return -1;
  memcpy(out, p, sizeof(double) * S->lev[l].size);
  return 0;
}
int or_set_field(void* sim, int which, int comp, int l, const double* in) {
  or_sim* S = (or_sim*)sim;
  double* p = field_ptr(S, which, comp, l);
  if (!p) return -1;
  memcpy(p, in, sizeof(double) * S->lev[l].size);
  return 0;
}
void or_get_nodes(void* sim, double* X) {
  or_sim* S = (or_sim*)sim;
  for (long s = 0; s < S->eta; ++s)
    for (int a = 0; a < S->D; ++a) X[S->D * s + a] = S->X[3 * s + a];
}
void or_get_node_forces(void* sim, double* F) {
  or_sim* S = (or_sim*)sim;
  for (long s = 0; s < S->eta; ++s)
    for (int a = 0; a < S->D; ++a) F[S->D * s + a] = S->F[3 * s + a];
}
void or_get_node_velocity(void* sim, double* U) {
  or_sim* S = (or_sim*)sim;
  for (long s = 0; s < S->eta; ++s)
    for (int a = 0; a < S->D; ++a) U[S->D * s + a] = S->U[3 * s + a];
}
long or_get_broken(void* sim, long cap, int32_t* id, int32_t* step) {
  or_sim* S = (or_sim*)sim;
  long n = S->nev < cap ? S->nev : cap;
  for (long q = 0; q < n; ++q) { id[q] = S->ev_id[q]; step[q] = S->ev_step[q]; }
  return S->nev;
}
void or_get_stats(void* sim, or_stats* out) {
  or_sim* S = (or_sim*)sim;
  S->st.broken_total = (int32_t)S->nev;
  S->st.step = S->step;
  *out = S->st;
}
int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
