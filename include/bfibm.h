/*
 * bfibm.h -- C ABI of the GB300 biofilm immersed-boundary time step.
 *
 * One context holds one simulation of the method of Hammond et al.,
 * arXiv:1302.3663: incompressible Navier-Stokes with variable density and
 * viscosity on a staggered grid (Eq. NSdis1-1, Eq. NSdis2-NSdis4), solved by
 * red-black multigrid (Sec. 3.5), coupled to Lagrangian nodes through the
 * width-omega delta of Eq. (Dirac Delta Approx) and joined by breakable
 * Hookean springs (Eq. springF, Sec. 3.2). All arithmetic runs in CUDA
 * kernels on the device that was current when the context was created.
 *
 * Conventions
 *   - Every function returns a bfibm_status and never aborts. After a CUDA
 *     error the context is poisoned: later calls return BFIBM_ESTATE.
 *     bfibm_last_error() gives the message of the last failure.
 *   - Host pointers are caller-owned. Inputs are copied before the call
 *     returns; outputs are written before the call returns (the call
 *     synchronises the context's stream when it reads data back).
 *   - Work is queued on the context's stream: the stream given to
 *     bfibm_create, or a stream the library creates when that is NULL.
 *   - One context is used by one host thread at a time.
 *
 * Grid layout shared by every field exchanged through this interface
 *   - n[a] cells of width h along axis a (n[2] = 1 when dim == 2). Axis a is
 *     periodic or bounded by no-slip walls at 0 and n[a] h.
 *   - A field is exchanged as a dense array of extents s[a] = n[a] + 1 along
 *     each wall axis and s[a] = n[a] along each periodic axis, x fastest
 *     (C order [s2][s1][s0]). Index i along axis a is the point at i h for a
 *     face/edge axis of that field and (i + 1/2) h for a centre axis.
 *   - Pressure p sits at cell centres (entries with some index i_a == n_a are
 *     unused, returned as 0). Velocity component d sits on the d-faces; the
 *     faces on walls (i_d = 0 and n_d) hold 0. mu_de sits on the (d,e)-edges.
 */
#ifndef BFIBM_H
#define BFIBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bfibm_ctx bfibm_ctx;

typedef enum {
  BFIBM_OK = 0,
  BFIBM_EINVAL = 1,   /* bad argument; nothing changed */
  BFIBM_ENOMEM = 2,   /* device or host allocation failed; nothing changed */
  BFIBM_ECUDA = 3,    /* a CUDA call failed; the context is poisoned */
  BFIBM_ENOCONV = 4,  /* a solve stopped above its tolerance or a projection above
                         div_tol; state is valid */
  BFIBM_ETIMEOUT = 5, /* a bounded device wait gave up; the context is poisoned */
  BFIBM_ESTATE = 6    /* the context is poisoned or not ready for the call */
} bfibm_status;

/* Parameters (model units). Eq. (N-SnondimFull): sigma = Strouhal number,
   euler = Euler number, inv_re = 1/Re, c_force = L f0 / (rho0 u0^2). */
typedef struct {
  int32_t dim;            /* 2 or 3 */
  int32_t n[3];           /* cells per axis; n[2] = 1 when dim == 2; each >= 2;
                             a level array (s[a] points per axis, rows padded
                             to 8) holds at most 2^31 - 1 elements */
  int32_t periodic[3];    /* 1: periodic axis, 0: no-slip walls */
  int32_t flow_axis;      /* axis of the body force */
  int32_t phi_kind;       /* 1: Eq. (PhiPeskin), 2: Eq. (PhiCosAlternative) */
  int32_t mg_levels_max;  /* multigrid levels (Sec. 4.3.1: at most 6 help) */
  int32_t nu1, nu2;       /* pre/post red-black sweeps per level */
  int32_t vc_visc, vc_p;  /* > 0: fixed V-cycles per solve; 0: until rtol */
  int32_t max_cycles;     /* cap in rtol mode */
  int32_t coarse_sweeps;  /* red-black sweeps on the coarsest grid */
  int32_t precision;      /* 0: FP64 throughout; 1: FP32 V-cycles inside FP64
                             defect correction (fine residual, divergence and
                             coarsest solve stay FP64) */
  double h;               /* mesh width, equal on every axis */
  double rho_f, mu_f;     /* fluid density and viscosity */
  double rho_ratio;       /* biofilm density ratio: rho_b = (rho_ratio - 1) rho_f */
  double mu_ratio;        /* mu_max = mu_ratio * mu_f, Eq. (ViscExp) */
  double omega;           /* delta width for f and rho, Eq. (discrForceCouple/DensCouple) */
  double omega_mu;        /* delta width in Eq. (ViscExp) */
  double d0_vol;          /* d0^D, mean volume per node, Eq. (discrDensCouple) */
  double dt, sigma, euler, inv_re, c_force;
  double body_force;      /* G along flow_axis, used when u_center <= 0 */
  double u_center;        /* > 0: G chosen so the laminar centreline speed is u_center */
  double ic_scale;        /* initial velocity = ic_scale * laminar profile */
  double rtol;            /* relative residual target (Sec. 4.1 uses 1e-9) */
  double gamma_coarse;    /* gamma of Eq. (ViscCoarseGrid) on every coarse level ... */
  double gamma_levels[8]; /* ... unless gamma_levels[l] > 0: gamma_lh of coarse level l
                             (l = 1 is the grid 2h); entries 0 and past the last level
                             are ignored */
  double div_tol;         /* > 0: every projection (Eq. NSdis2) checks max |D.u| in FP64
                             on the device against it (Eq. NSdis4 makes D.u vanish) and
                             counts a violation; 0: the maximum is still recorded */
  int32_t open_flow;      /* 1: the flow axis is the open duct of Sec. 3.6 instead of
                             periodic (periodic[flow_axis] = 0, precision 0, u_center > 0,
                             walls on the cross axes): face 0 holds the laminar profile
                             (Eq. 2DlaminarSoln / 3DlaminarFlow), the outflow face n is an
                             unknown with du/dn = 0 and the pressure held there at
                             kappa L (Eq. pressLam, euler kappa = -G of the same laminar
                             flow); no body force, no pressure flux through the inflow or
                             the walls */
} bfibm_params;

typedef struct {
  int32_t cycles_visc, cycles_p;     /* V-cycles used by the last solves */
  int32_t broken_total;              /* springs broken so far */
  int32_t clamped_total;             /* node moves clamped back onto a wall */
  double res_visc, res_p;            /* last relative residuals (0 if not collected) */
  double div_max;                    /* max |D.u| of the current velocity */
  double kinetic;                    /* sum over faces of u_d^2 h^D (Sec. 4.3.4) */
  int64_t step;                      /* completed time steps */
  int32_t nonfinite_total;           /* non-finite node coordinates met (a run that
                                        has blown up, e.g. a time step above the
                                        stability limit of Sec. 4.3.4); each is reset
                                        to 0 so that every kernel stays in bounds */
  int32_t wait_timeouts;             /* bounded device waits that ran out (0 unless
                                        the device misbehaves or BFIBM_OPT_WAIT_NS is
                                        set very short); the affected sweep stops early
                                        and its result is not valid */
  int32_t nonconv_total;             /* relative-residual solves that stopped above
                                        their tolerance (at max_cycles, or a flexible-CG
                                        solve whose true FP64 residual exceeds twice
                                        rtol), counted on the device */
  int32_t div_violations;            /* projections whose max |D.u| exceeded div_tol */
  double div_max_step;               /* max |D.u| of the last step's projection,
                                        computed inside the step (FP64) */
  double div_max_steps;              /* the largest such value over all steps */
} bfibm_stats;

/* Field selectors for bfibm_get_field / bfibm_set_field (see layout above). */
enum {
  BFIBM_F_U = 0,       /* velocity u^n, component comp (level 0 only) */
  BFIBM_F_UT = 1,      /* viscous multigrid iterate (level 0: u~), component comp */
  BFIBM_F_URHS = 2,    /* viscous right-hand side, component comp */
  BFIBM_F_P = 3,       /* pressure multigrid iterate (level 0: p) */
  BFIBM_F_PRHS = 4,    /* pressure right-hand side */
  BFIBM_F_RHO = 5,     /* density on the comp-faces (level 0 only) */
  BFIBM_F_FORCE = 6,   /* Eulerian force density, component comp (level 0 only) */
  BFIBM_F_MUC = 7,     /* viscosity at centres */
  BFIBM_F_MUE = 8,     /* viscosity on edges: comp 0 = xy, 1 = xz, 2 = yz */
  BFIBM_F_BETA = 9,    /* 1/rho on the comp-faces (restricted on coarse levels) */
  BFIBM_F_M = 10,      /* rho sigma / dt on the comp-faces */
  BFIBM_F_URES = 11,   /* viscous residual, component comp */
  BFIBM_F_PRES = 12,   /* pressure residual */
  BFIBM_F_IDG = 13     /* FP32 only: 1 / diagonal of the viscous operator, component
                          comp (formed from the FP64 coefficients when they are built;
                          0 on the fixed wall faces) */
};

/* Stage selectors for bfibm_stage. */
enum {
  BFIBM_STAGE_RHS = 0,        /* Eq. (NSdis1-1) right-hand side; u~ <- u^n */
  BFIBM_STAGE_DIVERGENCE = 1, /* b = (sigma/euler) D.u~ / dt, mean removed (Eq. NSdis4) */
  BFIBM_STAGE_PROJECT = 2,    /* u = u~ - (euler dt/sigma) beta D p (Eq. NSdis2) */
  BFIBM_STAGE_INTERP_ADVANCE = 3, /* U by Eq. (discrVelCouple), X += dt/sigma U */
  BFIBM_STAGE_SPRINGS = 4     /* break test and node forces, Eq. (springF) */
};

/* Create a context. p is validated and copied; stream may be NULL (the
   library then creates its own non-blocking stream). Allocates every grid
   array of every multigrid level on the current device, evaluates the
   laminar initial velocity (Eq. 2DlaminarSoln / 3DlaminarFlow) and a uniform
   fluid. Errors: BFIBM_EINVAL (bad parameters), BFIBM_ENOMEM, BFIBM_ECUDA. */
bfibm_status bfibm_create(const bfibm_params* p, void* stream, bfibm_ctx** out);

/* Load eta node positions X (eta x dim doubles, row-major, host). Every
   coordinate must lie in [0, L) on a periodic axis and in [0, L] on a wall
   axis (L = n h), else BFIBM_EINVAL and nothing changes. Load springs after
   nodes: loading a different number of nodes drops the springs. */
bfibm_status bfibm_set_nodes(bfibm_ctx* c, int64_t eta, const double* X);

/* Load m springs: node pairs ab (m x 2 int32), rest lengths, Hookean
   coefficients K and break strains (a spring breaks once its length exceeds
   (1 + break_strain) * rest; Sec. 3.2 uses 1). All host arrays. */
bfibm_status bfibm_set_springs(bfibm_ctx* c, int64_t m, const int32_t* ab, const double* rest,
                               const double* K, const double* break_strain);

/* Overwrite velocity component comp (host array in the field layout). */
bfibm_status bfibm_set_velocity(bfibm_ctx* c, int comp, const double* u);

/* Advance nsteps time steps in the order of Sec. 3.4: u~ (Eq. NSdis1-1), p
   (Eq. NSdis4), u (Eq. NSdis2), U (Eq. discrVelCouple), X, then springs,
   f, rho, mu (Eq. discrForceCouple, discrDensCouple, ViscExp) at the new
   positions. Every projection also records max |D.u| in FP64 on the device
   (bfibm_stats.div_max_step). Returns once the steps are done: it waits for
   the context's stream and reads the device status words. BFIBM_ENOCONV
   (the state is valid) if, since the last report, a relative-residual solve
   stopped above its tolerance or a projection exceeded div_tol;
   BFIBM_ETIMEOUT (the context is poisoned) if a bounded device wait ran out. */
bfibm_status bfibm_step(bfibm_ctx* c, int nsteps);

/* Read results into host buffers (field layout; X as eta x dim). */
bfibm_status bfibm_get_velocity(bfibm_ctx* c, int comp, double* out);
bfibm_status bfibm_get_pressure(bfibm_ctx* c, double* out);
bfibm_status bfibm_get_nodes(bfibm_ctx* c, double* X);
/* Broken springs as (spring id, step) pairs sorted by step then id; at most
   cap pairs are written, *n receives the total count. */
bfibm_status bfibm_get_broken(bfibm_ctx* c, int64_t cap, int64_t* n, int32_t* spring_id,
                              int32_t* step);
bfibm_status bfibm_get_stats(bfibm_ctx* c, bfibm_stats* out);
const char* bfibm_last_error(const bfibm_ctx* c);
void bfibm_destroy(bfibm_ctx* c);

/* Operator-level access, for inspection and verification of single stages.
   Fields use the layout above at multigrid level `level` (0 = finest). */
bfibm_status bfibm_get_field(bfibm_ctx* c, int which, int comp, int level, double* out);
bfibm_status bfibm_set_field(bfibm_ctx* c, int which, int comp, int level, const double* in);
/* Device-to-device variants: `dev` is a device pointer to a dense field array. */
bfibm_status bfibm_get_field_dev(bfibm_ctx* c, int which, int comp, int level, double* dev);
bfibm_status bfibm_set_field_dev(bfibm_ctx* c, int which, int comp, int level, const double* dev);
/* FP32 copies of the multigrid arrays used by the mixed-precision V-cycles
   (precision 1 only): which is one of BFIBM_F_UT, URHS, P, PRHS, MUC, MUE,
   BETA, M, URES, PRES, IDG (on level 0, UT/URHS/P/PRHS hold the FP32 correction
   and its right-hand side). Same layout as bfibm_get_field, in floats; host
   buffers; BFIBM_EINVAL for another selector or an FP64-only context. */
bfibm_status bfibm_get_field_f32(bfibm_ctx* c, int which, int comp, int level, float* out);
bfibm_status bfibm_set_field_f32(bfibm_ctx* c, int which, int comp, int level, const float* in);
/* Node forces F (eta x dim, host) from the last spring stage. */
bfibm_status bfibm_get_node_forces(bfibm_ctx* c, double* F);
/* Break test, forces, spreads and coefficient hierarchy at the current nodes. */
bfibm_status bfibm_refresh(bfibm_ctx* c);
/* beta = 1/rho and m = rho sigma/dt on the fine faces, then every coarse level. */
bfibm_status bfibm_build_coefficients(bfibm_ctx* c);
bfibm_status bfibm_stage(bfibm_ctx* c, int stage);
/* Multigrid solves on level 0 (ncycles > 0 fixed, 0 = until rtol), in the
   context's precision and solver options (FP64 V-cycles; or FP32 V-cycles
   inside FP64 defect correction, BFIBM_OPT_INNER of them per FP64 residual,
   and for the viscous solve inside flexible CG with BFIBM_OPT_KRYLOV); the
   V-cycles used are written to *cycles when cycles is not NULL. */
bfibm_status bfibm_solve_pressure(bfibm_ctx* c, int ncycles, int32_t* cycles);
bfibm_status bfibm_solve_viscous(bfibm_ctx* c, int ncycles, int32_t* cycles);
/* nsweeps red-black sweeps on one level (Sec. 3.5). Asynchronous: returns
   once the kernels are queued on the context's stream. */
bfibm_status bfibm_smooth_pressure(bfibm_ctx* c, int level, int nsweeps);
bfibm_status bfibm_smooth_viscous(bfibm_ctx* c, int level, int nsweeps);
/* Residual on one level (synchronous). */
bfibm_status bfibm_residual_pressure(bfibm_ctx* c, int level);
bfibm_status bfibm_residual_viscous(bfibm_ctx* c, int level);
/* nsweeps FP32 red-black sweeps of the correction iterate of a mixed-precision
   context (which: 0 pressure, 1 viscous) on one level; asynchronous.
   BFIBM_ESTATE for an FP64 context. */
bfibm_status bfibm_smooth_f32(bfibm_ctx* c, int which, int level, int nsweeps);
/* Wait for all work queued on the context's stream. */
bfibm_status bfibm_synchronize(bfibm_ctx* c);
/* Replace the coarse-grid viscosity scaling of Eq. (ViscCoarseGrid):
   gamma_levels[l] > 0 sets gamma_lh of coarse level l (others fall back to
   gamma_coarse). Rebuilds the coefficient hierarchy; the next step captures a
   new step graph. BFIBM_EINVAL for a negative or non-finite entry. */
bfibm_status bfibm_set_gamma(bfibm_ctx* c, const double gamma_levels[8]);
/* Number of multigrid levels and their cell counts / storage extents. */
bfibm_status bfibm_levels(bfibm_ctx* c, int32_t* nlevels);
bfibm_status bfibm_level_dims(bfibm_ctx* c, int level, int32_t n[3], int32_t s[3]);
/* Body force G in use (Eq. 2DlaminarSoln / 3DlaminarFlow when u_center > 0). */
bfibm_status bfibm_body_force(bfibm_ctx* c, double* G);
/* Options: BFIBM_OPT_STATS (1: residual norms after every fixed-count solve,
   default 1), BFIBM_OPT_GRAPH (1: replay fixed-count steps as a CUDA graph,
   default 1), BFIBM_OPT_FUSED (1: one-pass FP64 red-black sweeps; 0, the
   default: one kernel per colour, faster where FP64 arithmetic rather than
   memory bounds the sweep; FP32 sweeps are always one-pass), BFIBM_OPT_TMA
   (3D FP32 sweeps that stage their inputs in shared memory with
   tensor-memory-accelerator copies: 0 never, the one-pass sweep reads them
   from global memory; 1, the default, on the levels and components where the
   autotuner timed them faster; 2 on every level that allows them; all give
   bit-identical results), BFIBM_OPT_INNER (mixed precision: FP32 V-cycles per
   FP64 defect-correction iteration, 1 to 16, default 1; each FP64 residual is
   then followed by that many V-cycles on the FP32 correction equation, so a
   solve computes fewer FP64 residuals for the same V-cycles; a tolerance
   solve stops after a multiple of it). Every option but BFIBM_OPT_INNER gives
   the same results to rounding; BFIBM_OPT_INNER changes the iterates within
   the solver tolerance), BFIBM_OPT_KRYLOV (mixed precision, viscous solve:
   0, the default, FP64 defect correction around the FP32 V-cycles; 1, a
   flexible conjugate-gradient iteration in FP64 with the FP32 V-cycles as
   preconditioner, which needs fewer V-cycles where the viscosity contrast
   slows the V-cycle down; the same discrete system and stopping test, so
   tolerance solves agree within the tolerance), BFIBM_OPT_WAIT_NS (the
   limit in nanoseconds of each wait of the TMA sweep for its staged copies,
   default 2e9; 0 tests the barrier once without waiting. A sweep whose wait
   runs out drains its copies in flight, stops and raises
   bfibm_stats.wait_timeouts; the step then reports BFIBM_ETIMEOUT. Short
   limits exist to exercise that path), BFIBM_OPT_TAIL (3D mixed precision:
   the FP32 V-cycle levels of at most this many cells, down to and with the
   FP64 coarsest solve, run in one launch per V-cycle, a cluster of 8 thread
   blocks with a cluster barrier between phases and in-place red-black sweeps;
   default 8192, 0 keeps one launch per sweep, residual and transfer; the same
   results to the bit either way). */
enum {
  BFIBM_OPT_STATS = 0,
  BFIBM_OPT_GRAPH = 1,
  BFIBM_OPT_FUSED = 2,
  BFIBM_OPT_TMA = 3,
  BFIBM_OPT_INNER = 4,
  BFIBM_OPT_KRYLOV = 5,
  BFIBM_OPT_WAIT_NS = 6,
  BFIBM_OPT_TAIL = 7
};
bfibm_status bfibm_set_option(bfibm_ctx* c, int option, int64_t value);
/* Checkpoint and resume. The state a time step starts from (Sec. 3.4): the
   velocity u^n, the pressure (the next projection's initial guess), the node
   positions X^n, the broken springs with their break events, and the step
   count; forces, spreads and coefficients follow from it. bfibm_state_bytes
   gives the buffer size; bfibm_save_state writes the state into a host
   buffer; bfibm_load_state restores it into a context created with the same
   parameters and the same node and spring counts (BFIBM_EINVAL otherwise).
   Because no part of a step depends on the order of atomic operations, a
   resumed run continues bit for bit as the original would have. The buffer
   starts with a header (magic, version, dim, n, precision, counts) followed
   by the raw level-0 arrays in their padded layout; it is meant for the same
   library version. Checkpoints are not in the paper. */
bfibm_status bfibm_state_bytes(bfibm_ctx* c, int64_t* bytes);
bfibm_status bfibm_save_state(bfibm_ctx* c, void* buf, int64_t bytes);
bfibm_status bfibm_load_state(bfibm_ctx* c, const void* buf, int64_t bytes);

/* Tile plan the autotuner chose for the TMA-staged FP32 sweep of one level
   (kind 0..D-1: viscous component, 3: pressure): out = {tile rows, planes per
   chunk, planes prefetched, columns per strip, grid blocks}. Plans are timed once per level
   shape when a mixed-precision context is created. BFIBM_EINVAL when the
   level does not use the TMA sweep (not allowed, or the one-pass sweep timed
   faster). No counterpart in the paper. */
bfibm_status bfibm_tma_plan(bfibm_ctx* c, int level, int kind, int32_t out[5]);
/* Launch shape the autotuner chose for the one-pass FP32 sweep (the kernels
   that read their inputs from global memory) of one level and kind (0..D-1:
   viscous component, 3: pressure), mixed-precision contexts only: out =
   {tile rows, planes per chunk, planes per phase, threads per row, kernel};
   kernel 0 is the ring sweep (a thread per point pair or per 32-thread row
   group, a ring of new red planes, 0 in the first four fields standing for the
   built-in choice), kernel 1 the pair sweep (a thread per (red, black) pair
   of a row marching over the planes, float2 row loads; planes per phase 1,
   threads per row 0). Both give the same bits. BFIBM_EINVAL for an FP64 context, a bad level or kind,
   or a level shape the tuner has not timed. No counterpart in the paper. */
bfibm_status bfibm_sweep_shape(bfibm_ctx* c, int level, int kind, int32_t out[5]);
/* Pin the one-pass FP32 sweep with shape {tile rows (0: built-in), planes per
   chunk (0: built-in), planes per phase (1 or 2), threads per row (0 or a
   multiple of 32 up to 128), kernel (0 ring sweep; 1 pair sweep, which takes
   tile rows >= 1, planes per chunk >= 1, planes per phase 1, threads per row
   0 and a level with walls in x and y and an even row of at most 256 points)} for the shape of one level and kind, process-wide, in
   place of the autotuner's choice (the TMA sweep is no longer used there);
   the next step captures a new step graph. 3D mixed-precision contexts only;
   BFIBM_EINVAL otherwise or for a shape outside those ranges. Same results to
   the bit as any other shape. No counterpart in the paper. */
bfibm_status bfibm_sweep_set_shape(bfibm_ctx* c, int level, int kind, const int32_t shape[5]);
/* Pin the TMA sweep's plan {tile rows, planes per chunk, planes prefetched
   (1..3), columns per strip (>= n[0]: whole rows), grid blocks (0: as many as
   fit at once)} for the shape of one level, process-wide, in place of the
   tuned one (for example to reuse plans tuned in another process). Takes
   effect for step graphs captured afterwards. BFIBM_EINVAL when the level
   does not allow the TMA sweep or the plan does not fit. No counterpart in
   the paper. */
bfibm_status bfibm_tma_set_plan(bfibm_ctx* c, int level, int kind, const int32_t plan[5]);
/* Kernel launches in one replayed time step (the kernel nodes of the captured
   step graph), or -1 when no graph has been captured yet. */
bfibm_status bfibm_launches_per_step(bfibm_ctx* c, int64_t* n);
/* Kernel launch accounting of the replayed step graph: out = {kernel nodes
   at the top level of the step graph (-1 before the first capture), kernel
   nodes of one iteration of the viscous and of the pressure relative-residual
   loop (0 in fixed-cycle mode), iterations of the viscous and of the pressure
   loop run on the device since the context was created}. Kernels launched
   over n replayed steps = n * out[0] + (growth of out[3]) * out[1] + (growth
   of out[4]) * out[2]. No counterpart in the paper. */
bfibm_status bfibm_launch_counts(bfibm_ctx* c, int64_t out[5]);
/* Allocation-free divergence stage (the paper has no counterpart: this exists
   for callers that cannot let a library allocate device memory, such as
   programs whose device memory is already held by another allocator, services
   that must not hit an out-of-memory error after start-up, or loops that
   cannot afford the device-wide synchronisation cudaMalloc/cudaFree may
   cause). Computes what BFIBM_STAGE_DIVERGENCE computes, from the caller's
   buffers: b = (sigma/euler) D.u / dt at every cell, mean removed.
   u0, u1, u2: device pointers to the velocity components in the dense field
   layout above (u2 ignored when dim == 2); b: device pointer, same layout,
   only the cell entries are written. p supplies dim, n, periodic, h, dt,
   sigma and euler (periodic or walled axes only: an open duct is refused
   with BFIBM_EINVAL). stream: the stream to queue on (NULL = legacy default).
   Returns once the kernels are queued.
   Scratch: a fixed device array in the library (512 KB per GPU, held until
   the process exits); grids of more than 2^24 cells are rejected with
   BFIBM_EINVAL. No cudaMalloc, cudaFree or allocating library call is made.
   The first call on a device looks up that array's device address
   (cudaGetSymbolAddress) with the device current; make that first call before
   any stream capture. Every call shares the array, so calls that overlap on
   the GPU (other streams, other threads) race and must be serialised by the
   caller. BFIBM_ECUDA if the lookup or a launch fails. */
bfibm_status bfibm_divergence_noalloc(const bfibm_params* p, const double* u0, const double* u1,
                                      const double* u2, double* b, void* stream);
/* Batches: step many independent contexts together. Every member replays its
   own step graph on its own stream (create members with stream NULL so that
   each has one), so uneven simulations overlap on the device. A batch does
   not own its members; removing or destroying it leaves them intact. */
typedef struct bfibm_batch bfibm_batch;
bfibm_status bfibm_batch_create(bfibm_batch** out);
/* Add a context; *slot receives its index (freed slots are reused). */
bfibm_status bfibm_batch_add(bfibm_batch* b, bfibm_ctx* c, int32_t* slot);
bfibm_status bfibm_batch_remove(bfibm_batch* b, int32_t slot);
/* Queue nsteps[slot] time steps for every member (NULL: one each; 0 skips a
   member) without waiting, bracketing each member's steps with events. */
bfibm_status bfibm_batch_step(bfibm_batch* b, const int32_t* nsteps);
/* Wait until every member's queued work is done and read each member's
   device status words as bfibm_step does: BFIBM_ENOCONV if any member
   reports it (bfibm_get_stats tells which), BFIBM_ETIMEOUT for the first
   member whose bounded wait ran out. */
bfibm_status bfibm_batch_wait(bfibm_batch* b);
/* Device time of a member's steps in the last bfibm_batch_step (waits for
   them); BFIBM_ESTATE if the member was not stepped. */
bfibm_status bfibm_batch_slot_ms(bfibm_batch* b, int32_t slot, float* ms);
void bfibm_batch_destroy(bfibm_batch* b);
/* Batch options. BFIBM_BATCH_PERSISTENT (default 0): 1 steps the members in
   lock step, one CUDA graph per batch step in which every multigrid level and
   phase of both solves (Sec. 3.5, the mixed-precision form: FP32 V-cycles in
   FP64 defect correction, and flexible CG for the viscous solve when the
   members use it) is one launch over a device work list of (member, block)
   items covering members of different sizes; each solve's device loop runs
   while any member still iterates, and a member whose tolerance test is met
   drops out of the mask every launch of the loop reads. The stages around the
   solves run per member on forked branches of the graph. Every member must be
   3D, mixed precision (precision 1), closed (no open duct), solve to a
   tolerance (vc_visc = vc_p = 0), have a stream of its own, and share nu1,
   nu2, BFIBM_OPT_INNER and BFIBM_OPT_KRYLOV with the others; each member then
   gets the same bits as stepped alone. bfibm_batch_step must then give every
   member it steps the same count; the plan (member table, work lists, graph)
   is rebuilt when the stepped members or their options change.
   BFIBM_BATCH_TUNE (default 1): time the batched sweeps' kernel (ring or pair),
   tile rows, chunk planes, planes per phase and grid on every level of at
   least 2^19 cells in all when a plan is built (0: such levels take the pair
   sweep with up to 6 tile rows and 16-plane chunks where every member can, the
   ring sweep otherwise; smaller levels always keep a built-in ring shape).
   BFIBM_BATCH_UNROLL (default 0): k > 0 queues each solve loop as k
   iterations one after another instead of a device-side loop; the masks
   still stop every member where its tolerance is met, so results are the
   same while k covers the iterations the slowest member needs
   (a member not done after k iterations stops there without being counted as
   unconverged). It serves a profiler that cannot see kernels inside
   conditional graph nodes. BFIBM_BATCH_TAIL (default 4096): the levels of at
   most this many cells, down to and with each member's coarsest solve, run
   in the coarse-level kernel of BFIBM_OPT_TAIL with one thread block per
   member, on a branch of the graph beside the other members' launches (0:
   one launch per level and phase throughout); the members' own
   BFIBM_OPT_TAIL does not apply in the batch, and the results are the same
   to the bit. Every option drops the current plan. */
enum {
  BFIBM_BATCH_PERSISTENT = 0,
  BFIBM_BATCH_TUNE = 1,
  BFIBM_BATCH_UNROLL = 2,
  BFIBM_BATCH_TAIL = 3
};
bfibm_status bfibm_batch_set_option(bfibm_batch* b, int option, int64_t value);
/* out[0] persistent mode, out[1] plans built so far; with a plan: out[2]
   members, out[3] kernel nodes of the batch step graph outside its loops,
   out[4] / out[5] kernel nodes of one iteration of the viscous / pressure
   loop, out[6] / out[7] iterations of those loops so far (waits for the
   batch's work). */
bfibm_status bfibm_batch_info(bfibm_batch* b, int64_t out[8]);
/* The batched sweep of the current plan on a level (kind 0 viscous, 1
   pressure): out = {tile rows, chunk planes, planes per phase, threads per
   row, one block per item (1) or resident blocks striding (0), grid, kernel
   (0 the ring sweep, 1 the pair sweep)}. BFIBM_EINVAL without a plan or for
   a level it does not have. */
bfibm_status bfibm_batch_sweep_shape(bfibm_batch* b, int level, int kind, int32_t out[7]);
/* Pin the batched sweep of the current plan on a level (kind as above):
   shape = {tile rows, chunk planes, planes per phase (1 or 2), threads per row
   (a multiple of 32; rows x (tile rows + 2) threads at most 1024), one block
   per item, kernel (1: the pair sweep, where every member smoothing on the
   level has walls across x and y and even rows the block covers, at most 512
   threads)}; the plan's graph is captured again.
   BFIBM_EINVAL without a plan, for a level it does not have or a shape out of
   range (the plan unchanged). */
bfibm_status bfibm_batch_set_sweep_shape(bfibm_batch* b, int level, int kind,
                                         const int32_t shape[6]);
/* Message of the last batch call that failed on the batch itself. */
const char* bfibm_batch_error(bfibm_batch* b);
/* Device bytes a context with these parameters allocates for its grids. */
bfibm_status bfibm_footprint(const bfibm_params* p, int64_t eta, int64_t nsprings,
                             int64_t* bytes);

#ifdef __cplusplus
}
#endif
#endif /* BFIBM_H */
