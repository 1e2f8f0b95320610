// Context, multigrid driver, time step and C ABI of libbfibm (include/bfibm.h).
//
// Host code here only orchestrates: it validates inputs, lays out device
// memory, queues kernels on the context's stream (optionally as one CUDA
// graph per time step) and copies data in and out. Every arithmetic step of
// the method runs in the kernels of stencil.cu and lagrangian.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/bfibm.h"
#include "common.cuh"

using namespace bf;

namespace {

struct Level {
  Geo g;
  LevelPtrs<double> d;   // FP64 arrays
  LevelPtrs<float> f;    // FP32 arrays of the mixed-precision V-cycles
};

int edge_count(int D) { return D == 3 ? 3 : 1; }

long long round_up(long long v, long long a) { return (v + a - 1) / a * a; }

Geo make_geo(const int n[3], const int per[3], int D, double h, int open) {
  Geo g;
  g.open = open;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = n[a];
    g.per[a] = per[a];
    g.s[a] = (a < D && !per[a]) ? n[a] + 1 : n[a];
  }
  if (D == 2) {
    g.n[2] = 1;
    g.s[2] = 1;
    g.per[2] = 1;
  }
  long long pitch = round_up(g.s[0], 8);
  g.st[0] = 1;
  g.st[1] = pitch;
  g.st[2] = pitch * g.s[1];
  g.h = h;
  return g;
}

long long level_elems(const Geo& g) { return g.st[2] * g.s[2]; }

// arrays per level: p, p2, pf, pr, beta[D], u[D], u2[D], uf[D], ur[D], m[D], muc, mue[E]
int arrays_per_level(int D) { return 4 + 6 * D + 1 + edge_count(D); }

// Multigrid levels: halve while every axis is even, the halved minimum is at
// least 2 and every halved periodic axis stays even (so that red-black
// colouring is consistent across the periodic wrap), up to mg_levels_max.
int build_levels(const bfibm_params& P, Geo out[kMaxLevels]) {
  int D = P.dim;
  int n[3] = {P.n[0], P.n[1], D == 3 ? P.n[2] : 1};
  int per[3] = {P.periodic[0], P.periodic[1], D == 3 ? P.periodic[2] : 1};
  int L = 0;
  double h = P.h;
  const int open = P.open_flow ? P.flow_axis : -1;
  for (;;) {
    out[L] = make_geo(n, per, D, h, open);
    ++L;
    if (L >= P.mg_levels_max || L >= kMaxLevels) break;
    bool ok = true;
    int mn = 1 << 30;
    for (int a = 0; a < D; ++a) {
      if (n[a] % 2) ok = false;
      mn = std::min(mn, n[a] / 2);
      if (per[a] && (n[a] / 2) % 2) ok = false;
    }
    if (!ok || mn < 2) break;
    for (int a = 0; a < D; ++a) n[a] /= 2;
    h *= 2.0;
  }
  return L;
}

size_t grid_pool_bytes(const bfibm_params& P, int* nlev = nullptr) {
  Geo g[kMaxLevels];
  int L = build_levels(P, g);
  size_t bytes = 0;
  for (int l = 0; l < L; ++l) {
    size_t arr = (size_t)round_up(level_elems(g[l]) * 8, 256);
    // level 0: velocity, density, force; mixed precision adds the FP64
    // viscous diagonal and the flexible-CG vectors p, q and z
    int na = arrays_per_level(P.dim) + (l == 0 ? 3 * P.dim : 0) +
             (l == 0 && P.precision == 1 ? 4 * P.dim : 0);
    bytes += arr * na;
    if (P.precision == 1)   // the level's arrays and the inverse viscous diagonals
      bytes += (size_t)round_up(level_elems(g[l]) * 4, 256) * (arrays_per_level(P.dim) + P.dim);
  }
  bytes += 256 * 16;  // G and scalars
  if (nlev) *nlev = L;
  return bytes;
}

const char* validate(const bfibm_params* p) {
  if (!p) return "params is NULL";
  if (p->dim != 2 && p->dim != 3) return "dim must be 2 or 3";
  for (int a = 0; a < p->dim; ++a) {
    if (p->n[a] < 2) return "every n[a] must be >= 2";
    if (p->periodic[a] && (p->n[a] % 2)) return "a periodic axis needs an even cell count";
  }
  if (p->dim == 2 && p->n[2] != 1) return "n[2] must be 1 when dim == 2";
  // the grid kernels index within a level array with 32-bit offsets
  long long elems = 1;
  for (int a = 0; a < 3; ++a) {
    long long ext = a < p->dim ? (long long)p->n[a] + (p->periodic[a] ? 0 : 1) : 1;
    if (a == 0) ext = (ext + 7) / 8 * 8;
    elems *= ext;
    if (elems > 2147483647LL) return "a level array would hold more than 2^31 - 1 elements";
  }
  if (p->flow_axis < 0 || p->flow_axis >= p->dim) return "flow_axis out of range";
  if (!p->periodic[p->flow_axis] && !p->open_flow)
    return "the flow axis must be periodic (or open, with open_flow = 1)";
  if (p->periodic[p->flow_axis] && p->open_flow) return "an open flow axis is not periodic";
  for (int a = 0; a < p->dim; ++a)
    if (a != p->flow_axis && p->periodic[a]) {
      // laminar profile is defined between walls; periodic cross axes are allowed
      // only with u_center <= 0 (explicit body force)
      if (p->u_center > 0.0) return "u_center > 0 needs walls on every cross axis";
    }
  if (p->phi_kind != 1 && p->phi_kind != 2) return "phi_kind must be 1 or 2";
  if (!(p->h > 0.0) || !(p->dt > 0.0) || !(p->sigma > 0.0) || !(p->euler > 0.0))
    return "h, dt, sigma and euler must be positive";
  if (!(p->rho_f > 0.0) || !(p->mu_f > 0.0) || p->rho_ratio < 1.0 || p->mu_ratio < 1.0)
    return "rho_f, mu_f > 0 and ratios >= 1 required";
  if (!(p->omega > 0.0) || !(p->omega_mu > 0.0)) return "omega and omega_mu must be positive";
  if (p->mg_levels_max < 1 || p->nu1 < 0 || p->nu2 < 0 || p->coarse_sweeps < 1)
    return "bad multigrid settings";
  if (p->vc_visc < 0 || p->vc_p < 0 || (p->vc_visc == 0 || p->vc_p == 0) && p->max_cycles < 1)
    return "bad V-cycle counts";
  if (p->precision != 0 && p->precision != 1) return "precision must be 0 or 1";
  if (!(p->inv_re >= 0.0)) return "inv_re must be >= 0";
  if (!(p->gamma_coarse > 0.0) || !std::isfinite(p->gamma_coarse)) return "gamma_coarse must be > 0";
  for (int l = 0; l < 8; ++l)
    if (!(p->gamma_levels[l] >= 0.0) || !std::isfinite(p->gamma_levels[l]))
      return "gamma_levels entries must be >= 0";
  if (!(p->div_tol >= 0.0) || !std::isfinite(p->div_tol)) return "div_tol must be >= 0";
  if (p->open_flow != 0 && p->open_flow != 1) return "open_flow must be 0 or 1";
  if (p->open_flow) {
    if (p->precision != 0) return "the open duct runs in FP64 (precision 0)";
    if (!(p->u_center > 0.0)) return "the open duct needs u_center > 0 (the laminar inflow)";
    for (int a = 0; a < p->dim; ++a)
      if (a != p->flow_axis && p->periodic[a]) return "the open duct needs walls on the cross axes";
    if (p->n[p->flow_axis] % 2) return "the open flow axis needs an even cell count";
  }
  return nullptr;
}

constexpr int kCounters = 8;

}  // namespace

struct bfibm_ctx {
  bfibm_params P;
  int D = 0, L = 0;
  Level lev[kMaxLevels];
  double* uvel[3] = {nullptr, nullptr, nullptr};
  double* vdiag[3] = {nullptr, nullptr, nullptr};   // FP64 viscous diagonal (mixed precision)
  double* cg_p[3] = {nullptr, nullptr, nullptr};    // flexible-CG direction and A times it
  double* cg_q[3] = {nullptr, nullptr, nullptr};
  double* cg_z[3] = {nullptr, nullptr, nullptr};    // the preconditioned residual in FP64
  double* rho[3] = {nullptr, nullptr, nullptr};
  double* frc[3] = {nullptr, nullptr, nullptr};
  double* G_dev = nullptr;
  double p_out = 0.0;             // open duct: the pressure held at the outflow
  Scalars sc{};
  double* host_sc = nullptr;  // pinned mirror of sc.out
  char* pool = nullptr;
  size_t pool_bytes = 0;
  // Lagrangian state
  NodeSet N{};
  SpringSet S{};
  TileGeo tg{};
  long long* step_dev = nullptr;
  int* counters = nullptr;    // [0] clamped, [1] event count, [2] non-finite, [3] wait timeouts,
                              // [4] solves stopped above their tolerance, [5] projections
                              // above div_tol
  int seen[kCounters] = {0};  // counters as last reported by a step or a batch wait
  double* spread_scale = nullptr;   // fixed-point scales of the force and density sums
  std::vector<void*> lag_allocs;
  cudaStream_t stream = nullptr;
  cudaStream_t aux = nullptr;     // captures the bodies of device-side loops
  bool own_stream = false;
  bool capturing = false;         // a step graph is being captured
  int* dev_cycles = nullptr;      // V-cycles used by the last solves (visc, p)
  long long* loop_total = nullptr;   // device-loop iterations so far (visc, p)
  long long body_kernels[2] = {0, 0};   // kernel nodes of one iteration of each loop
  cudaGraphExec_t gexec = nullptr;
  bool use_graph = true;
  bool fused = false;            // one-pass FP64 red-black sweeps (FP32 sweeps always are)
  unsigned long long tma_wait_ns = kTmaWaitNs;   // limit of the TMA sweep's waits
  int tma = 1;                   // 3D FP32 sweeps with TMA-staged inputs: 0 never, 1 where
                                 // the tuner timed them faster, 2 wherever a level allows
  bool collect_stats = true;
  bool dirty = true;
  int poisoned = 0;
  long long step_host = 0;
  int inner = 1;                 // FP32 V-cycles per FP64 defect-correction iteration
  int krylov = 0;                // 1: flexible CG around the FP32 V-cycle (viscous, mixed)
  int cycles_visc = 0, cycles_p = 0;
  int loop_inner[2] = {1, 1};    // V-cycles per device-loop iteration (visc, p) when captured
  long long graph_kernels = -1;   // kernel nodes in the captured step graph
  long long version = 0;          // changes whenever the step graph is dropped: a batch plan
                                  // built on this context is then rebuilt
  long long partial_cap = 0;      // doubles in sc.partial
  long long tail_cells = 8192;    // BFIBM_OPT_TAIL: FP32 V-cycle levels of at most this many
                                  // cells run in the coarse-level cluster kernel (0: none)
  int tail_lev = kMaxLevels;      // the first of them (L: none)
  BMember* self_tab = nullptr;    // this context as the one member of that kernel's table
  int* self_list = nullptr;       // {0}
  std::string err;
};

namespace {

bfibm_status set_err(bfibm_ctx* c, bfibm_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

bfibm_status cuda_fail(bfibm_ctx* c, cudaError_t e, const char* where) {
  c->poisoned = 1;
  cudaGetLastError();  // do not leave the error for the next caller
  return set_err(c, BFIBM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);         \
  } while (0)

#define READY(c)                                                                       \
  do {                                                                                 \
    if (!(c)) return BFIBM_EINVAL;                                                     \
    if ((c)->poisoned) return set_err((c), BFIBM_ESTATE, "context poisoned: " + (c)->err); \
  } while (0)

// Versions come from one counter for the whole process: a context created
// where a destroyed one lived never takes over its version, so a batch plan
// built for the old one is never mistaken for a plan of the new one.
long long next_version() {
  static std::atomic<long long> counter{1};
  return counter.fetch_add(1);
}

void drop_graph(bfibm_ctx* c) {
  c->version = next_version();
  if (c->gexec) {
    cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
  }
}


// ----------------------------------------------------------------- multigrid
// n red-black sweeps of the pressure iterate on level l. The fused sweep is
// out of place: the level's two p buffers swap after every sweep and, after
// an odd count, the result is copied back so that the iterate always ends in
// its own buffer (a replayed step graph then sees the same buffers).
void smooth_p(bfibm_ctx* c, int l, int n) {
  Level& Lv = c->lev[l];
  cudaStream_t s = c->stream;
  if (!c->fused) {
    for (int it = 0; it < n; ++it) {
      launch_p_rbgs<double>(c->D, Lv.g, Lv.d, 0, s);
      launch_p_rbgs<double>(c->D, Lv.g, Lv.d, 1, s);
    }
    return;
  }
  for (int it = 0; it < n; ++it) {
    launch_p_rb_fused<double>(c->D, Lv.g, Lv.d, Lv.d.p2, s);
    std::swap(Lv.d.p, Lv.d.p2);
  }
  if (n & 1) {
    cudaMemcpyAsync(Lv.d.p2, Lv.d.p, (size_t)level_elems(Lv.g) * sizeof(double),
                    cudaMemcpyDeviceToDevice, s);
    std::swap(Lv.d.p, Lv.d.p2);
  }
}

// n block sweeps (component x, y, z in turn) of the viscous iterate.
void smooth_v(bfibm_ctx* c, int l, int n) {
  Level& Lv = c->lev[l];
  cudaStream_t s = c->stream;
  for (int it = 0; it < n; ++it)
    for (int d = 0; d < c->D; ++d) {
      if (!c->fused) {
        launch_v_rbgs<double>(c->D, Lv.g, Lv.d, d, 0, c->P.inv_re, s);
        launch_v_rbgs<double>(c->D, Lv.g, Lv.d, d, 1, c->P.inv_re, s);
      } else {
        launch_v_rb_fused<double>(c->D, Lv.g, Lv.d, d, Lv.d.u2[d], c->P.inv_re, s);
        std::swap(Lv.d.u[d], Lv.d.u2[d]);
      }
    }
  if (c->fused && (n & 1))
    for (int d = 0; d < c->D; ++d) {
      cudaMemcpyAsync(Lv.d.u2[d], Lv.d.u[d], (size_t)level_elems(Lv.g) * sizeof(double),
                      cudaMemcpyDeviceToDevice, s);
      std::swap(Lv.d.u[d], Lv.d.u2[d]);
    }
}

// The face components' transfers: one launch for all three in 3D without an
// open axis, else one per component.
template <typename T>
void restrict_faces(bfibm_ctx* c, const Geo& gf, const Geo& gc, T* const rf[3], T* const fc[3],
                    T* const xc[3]) {
  if (c->D == 3 && gf.open < 0) {
    launch_restrict_face3<T>(gf, gc, rf, fc, xc, c->stream);
    return;
  }
  for (int d = 0; d < c->D; ++d)
    launch_restrict_face<T>(c->D, d, gf, gc, rf[d], fc[d], xc[d], c->stream);
}

template <typename T>
void prolong_faces(bfibm_ctx* c, const Geo& gf, const Geo& gc, T* const ec[3], T* const xf[3]) {
  if (c->D == 3 && gf.open < 0) {
    launch_prolong_face3<T>(gf, gc, ec, xf, c->stream);
    return;
  }
  for (int d = 0; d < c->D; ++d) launch_prolong_face<T>(c->D, d, gf, gc, ec[d], xf[d], c->stream);
}

void vcycle_p(bfibm_ctx* c, int l) {
  Level& Lv = c->lev[l];
  cudaStream_t s = c->stream;
  if (l == c->L - 1) {
    launch_coarse_p<double>(c->D, Lv.g, Lv.d, c->P.coarse_sweeps, s);
    return;
  }
  smooth_p(c, l, c->P.nu1);
  launch_p_residual<double>(c->D, Lv.g, Lv.d, s);
  Level& Lc = c->lev[l + 1];
  launch_restrict_cell<double>(c->D, Lv.g, Lc.g, Lv.d.pr, Lc.d.pf, Lc.d.p, s);
  vcycle_p(c, l + 1);
  launch_prolong_cell<double>(c->D, Lv.g, Lc.g, Lc.d.p, Lv.d.p, s);
  smooth_p(c, l, c->P.nu2);
}

void vcycle_v(bfibm_ctx* c, int l) {
  Level& Lv = c->lev[l];
  cudaStream_t s = c->stream;
  if (l == c->L - 1) {
    launch_coarse_v<double>(c->D, Lv.g, Lv.d, c->P.coarse_sweeps, c->P.inv_re, s);
    return;
  }
  smooth_v(c, l, c->P.nu1);
  launch_v_residual<double>(c->D, Lv.g, Lv.d, c->P.inv_re, s);
  Level& Lc = c->lev[l + 1];
  restrict_faces(c, Lv.g, Lc.g, Lv.d.ur, Lc.d.uf, Lc.d.u);
  vcycle_v(c, l + 1);
  prolong_faces(c, Lv.g, Lc.g, Lc.d.u, Lv.d.u);
  smooth_v(c, l, c->P.nu2);
}

// scalar slots: 0 scratch (means), 2/3 viscous |f|^2,|r|^2, 4/5 pressure, 6/7 div/KE,
// 8-10 flexible CG, 11-13 the divergence check of every projection (accumulator,
// this step's max |D.u|, the max over all steps)
// 14 the max |r| of the pressure residual
enum { SL_VF = 2, SL_VR = 3, SL_PF = 4, SL_PR = 5, SL_DIV = 6, SL_ZQ = 8, SL_PQ = 9, SL_PRR = 10,
       SL_DIVACC = 11, SL_DIVSTEP = 12, SL_DIVALL = 13, SL_PRMAX = 14 };

// The projection leaves D.u = (euler dt / sigma) r_p (Eq. NSdis2 - NSdis4, the
// pressure right-hand side having zero mean), so a pressure solve in
// relative-residual mode with div_tol > 0 also runs until
// (euler dt / sigma) max |r_p| <= div_tol: the divergence target then holds
// after every projection, not only on average.
double div_scale(const bfibm_ctx* c) { return c->P.euler * c->P.dt / c->P.sigma; }

bool p_converged(const bfibm_ctx* c, const double* hs) {
  double fn = std::sqrt(hs[SL_PF]), rn = std::sqrt(hs[SL_PR]);
  double rel = fn > 0.0 ? rn / fn : 0.0;
  return rel <= c->P.rtol && (c->P.div_tol <= 0.0 || div_scale(c) * hs[SL_PRMAX] <= c->P.div_tol);
}

// The true FP64 residual of a flexible-CG solve may drift from the recurrence
// that stops the loop; a solve whose true relative residual exceeds this many
// times rtol is reported as not converged.
constexpr double kTrueResidualSlack = 2.0;

inline int dc_iterations(int vcycles, int inner) { return (vcycles + inner - 1) / inner; }

long long cells_of(const Geo& g) { return (long long)g.n[0] * g.n[1] * g.n[2]; }

// First level of the coarse-level cluster kernel: the first level of at most
// tail_cells cells (3D mixed precision, closed duct), else L.
int tail_level(const bfibm_ctx* c) {
  if (c->D != 3 || c->P.precision != 1 || c->tail_cells <= 0 || c->P.open_flow) return c->L;
  for (int l = 0; l < c->L; ++l)
    if (cells_of(c->lev[l].g) <= c->tail_cells) return l;
  return c->L;
}

// The context as a member of a batched kernel's table.
void fill_member(const bfibm_ctx* c, BMember& B) {
  std::memset(&B, 0, sizeof(B));
  for (int l = 0; l < c->L; ++l) {
    B.g[l] = c->lev[l].g;
    B.f[l] = c->lev[l].f;
    B.d[l] = c->lev[l].d;
  }
  B.L = c->L;
  B.inv_re = c->P.inv_re;
  for (int d = 0; d < 3; ++d) {
    B.vdiag[d] = c->vdiag[d];
    B.cg_p[d] = c->cg_p[d];
    B.cg_q[d] = c->cg_q[d];
    B.cg_z[d] = c->cg_z[d];
  }
  B.sc = c->sc;
  B.cycles = c->dev_cycles;
  B.total = c->loop_total;
  B.nonconv = c->counters + 4;
  B.rtol = c->P.rtol;
  B.maxc = dc_iterations(c->P.max_cycles, c->inner);
  B.dscale = div_scale(c);
  B.div_tol = c->P.div_tol;
  B.coarse_sweeps = c->P.coarse_sweeps;
  B.nu1 = c->P.nu1;
  B.nu2 = c->P.nu2;
  B.tail = c->tail_lev;
  for (int l = 0; l < c->L; ++l) {
    const double h = c->lev[l].g.h;
    B.ir[l] = c->P.inv_re / (h * h);
    B.ih2[l] = 1.0 / (h * h);
  }
}

// the context's own one-member table, with its current settings
cudaError_t upload_self(bfibm_ctx* c) {
  c->tail_lev = tail_level(c);
  if (!c->self_tab) return cudaSuccess;
  BMember B;
  fill_member(c, B);
  cudaError_t e = cudaMemcpyAsync(c->self_tab, &B, sizeof(B), cudaMemcpyHostToDevice, c->stream);
  return e == cudaSuccess ? cudaStreamSynchronize(c->stream) : e;
}

bfibm_status read_scalars(bfibm_ctx* c) {
  CK(cudaMemcpyAsync(c->host_sc, c->sc.out, 16 * sizeof(double), cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return BFIBM_OK;
}

long long count_kernel_nodes(cudaGraph_t graph) {
  size_t nn = 0;
  long long nk = 0;
  if (cudaGraphGetNodes(graph, nullptr, &nn) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn && cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
    for (auto nd : nodes) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
    }
  return nk;
}

// Records into the step graph being captured on c->stream a device-side
// loop: a conditional WHILE node whose body (queued by `body` on c->stream,
// redirected to the auxiliary stream while the body is captured) ends with
// launch_tol_check, which decides whether the body runs again.
template <typename Body>
bfibm_status capture_while(bfibm_ctx* c, int which, Body body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(c->stream, &cs, nullptr, &g, &deps, nullptr, &nd));
  std::vector<cudaGraphNode_t> dv(deps, deps + nd);
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CK(cudaGraphAddNode(&node, g, dv.data(), nullptr, dv.size(), &np));
  CK(cudaStreamUpdateCaptureDependencies(c->stream, &node, nullptr, 1,
                                         cudaStreamSetCaptureDependencies));
  cudaGraph_t bg = np.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(c->aux, bg, nullptr, nullptr, 0,
                                   cudaStreamCaptureModeThreadLocal));
  cudaStream_t main = c->stream;
  c->stream = c->aux;
  body(h);
  c->stream = main;
  cudaGraph_t out = nullptr;
  CK(cudaStreamEndCapture(c->aux, &out));
  c->body_kernels[which] = count_kernel_nodes(bg);
  return BFIBM_OK;
}

// Solve on level 0. Fixed mode only queues work; relative-residual mode
// either loops on the device (inside a captured step graph) or reads the
// residual norm back after every cycle.
bfibm_status solve_p(bfibm_ctx* c, int ncycles, int* used) {
  Level& L0 = c->lev[0];
  cudaStream_t s = c->stream;
  double* one[3] = {L0.d.pf, nullptr, nullptr};
  double* res[3] = {L0.d.pr, nullptr, nullptr};
  bool tol = ncycles <= 0;
  if (tol || c->collect_stats) launch_norm2(c->D, L0.g, one, 0, c->sc, SL_PF, s);
  if (!tol) {
    for (int k = 0; k < ncycles; ++k) {
      vcycle_p(c, 0);
      if (L0.g.open < 0) launch_sub_mean(c->D, L0.g, L0.d.p, c->sc, s);
    }
    if (c->collect_stats) {
      launch_p_residual<double>(c->D, L0.g, L0.d, s);
      launch_norm2(c->D, L0.g, res, 0, c->sc, SL_PR, s);
    }
    *used = ncycles;
    return BFIBM_OK;
  }
  if (c->capturing) {
    cudaMemsetAsync(c->dev_cycles + 1, 0, sizeof(int), s);
    c->loop_inner[1] = 1;
    bfibm_status cs = capture_while(c, 1, [&](cudaGraphConditionalHandle h) {
      vcycle_p(c, 0);
      if (L0.g.open < 0) launch_sub_mean(c->D, L0.g, L0.d.p, c->sc, c->stream);
      launch_p_residual<double>(c->D, L0.g, L0.d, c->stream);
      launch_norm2(c->D, L0.g, res, 0, c->sc, SL_PR, c->stream);
      if (c->P.div_tol > 0.0) launch_absmax_cells(c->D, L0.g, L0.d.pr, c->sc, SL_PRMAX, c->stream);
      launch_tol_check(h, c->sc.out, SL_PF, SL_PR, c->P.rtol, c->P.max_cycles, c->dev_cycles + 1,
                       c->loop_total + 1, c->counters + 4, c->stream, SL_PRMAX, div_scale(c),
                       c->P.div_tol);
    });
    *used = -1;
    return cs;
  }
  bfibm_status st = BFIBM_ENOCONV;
  int k = 0;
  for (k = 1; k <= c->P.max_cycles; ++k) {
    vcycle_p(c, 0);
    if (L0.g.open < 0) launch_sub_mean(c->D, L0.g, L0.d.p, c->sc, s);
    launch_p_residual<double>(c->D, L0.g, L0.d, s);
    launch_norm2(c->D, L0.g, res, 0, c->sc, SL_PR, s);
    if (c->P.div_tol > 0.0) launch_absmax_cells(c->D, L0.g, L0.d.pr, c->sc, SL_PRMAX, s);
    bfibm_status rs = read_scalars(c);
    if (rs != BFIBM_OK) return rs;
    if (p_converged(c, c->host_sc)) {
      st = BFIBM_OK;
      break;
    }
  }
  *used = std::min(k, c->P.max_cycles);
  return st;
}

bfibm_status solve_v(bfibm_ctx* c, int ncycles, int* used) {
  Level& L0 = c->lev[0];
  cudaStream_t s = c->stream;
  bool tol = ncycles <= 0;
  if (tol || c->collect_stats) launch_norm2(c->D, L0.g, L0.d.uf, c->D, c->sc, SL_VF, s);
  if (!tol) {
    for (int k = 0; k < ncycles; ++k) vcycle_v(c, 0);
    if (c->collect_stats) {
      launch_v_residual<double>(c->D, L0.g, L0.d, c->P.inv_re, s);
      launch_norm2(c->D, L0.g, L0.d.ur, c->D, c->sc, SL_VR, s);
    }
    *used = ncycles;
    return BFIBM_OK;
  }
  if (c->capturing) {
    cudaMemsetAsync(c->dev_cycles, 0, sizeof(int), s);
    c->loop_inner[0] = 1;
    bfibm_status cs = capture_while(c, 0, [&](cudaGraphConditionalHandle h) {
      vcycle_v(c, 0);
      launch_v_residual<double>(c->D, L0.g, L0.d, c->P.inv_re, c->stream);
      launch_norm2(c->D, L0.g, L0.d.ur, c->D, c->sc, SL_VR, c->stream);
      launch_tol_check(h, c->sc.out, SL_VF, SL_VR, c->P.rtol, c->P.max_cycles, c->dev_cycles,
                       c->loop_total, c->counters + 4, c->stream);
    });
    *used = -1;
    return cs;
  }
  bfibm_status st = BFIBM_ENOCONV;
  int k = 0;
  for (k = 1; k <= c->P.max_cycles; ++k) {
    vcycle_v(c, 0);
    launch_v_residual<double>(c->D, L0.g, L0.d, c->P.inv_re, s);
    launch_norm2(c->D, L0.g, L0.d.ur, c->D, c->sc, SL_VR, s);
    bfibm_status rs = read_scalars(c);
    if (rs != BFIBM_OK) return rs;
    double fn = std::sqrt(c->host_sc[SL_VF]), rn = std::sqrt(c->host_sc[SL_VR]);
    double rel = fn > 0.0 ? rn / fn : 0.0;
    if (rel <= c->P.rtol) {
      st = BFIBM_OK;
      break;
    }
  }
  *used = std::min(k, c->P.max_cycles);
  return st;
}

// ------------------------------------------------------ mixed precision
// FP32 sweeps on level l (out of place, copied back after an odd count).
bool use_tma(bfibm_ctx* c, int l) { return c->tma && tma_eligible(c->D, c->lev[l].g); }
bool tma_for(bfibm_ctx* c, int l, int K) {
  return use_tma(c, l) && (c->tma == 2 || tma_chosen(K, c->lev[l].g));
}

void smooth_p32(bfibm_ctx* c, int l, int n) {
  Level& Lv = c->lev[l];
  const bool tma = tma_for(c, l, 3);
  for (int it = 0; it < n; ++it) {
    if (tma)
      launch_rb_tma(c->D, Lv.g, Lv.f, 3, Lv.f.p2, c->counters + 3, Lv.g.h * Lv.g.h, c->stream,
                    c->tma_wait_ns);
    else {
      int ty = 0, kc = 0, np = 1, bx = 0;
      int kern = 0;
      ring_shape_of(3, Lv.g, &ty, &kc, &np, &bx, &kern);
      if (kern == 1) launch_p_rb_pair(Lv.g, Lv.f, Lv.f.p2, c->stream, ty, kc);
      else launch_p_rb_fused<float>(c->D, Lv.g, Lv.f, Lv.f.p2, c->stream, ty, kc, np, bx);
    }
    std::swap(Lv.f.p, Lv.f.p2);
  }
  if (n & 1) {
    cudaMemcpyAsync(Lv.f.p2, Lv.f.p, (size_t)level_elems(Lv.g) * sizeof(float),
                    cudaMemcpyDeviceToDevice, c->stream);
    std::swap(Lv.f.p, Lv.f.p2);
  }
}

void smooth_v32(bfibm_ctx* c, int l, int n) {
  Level& Lv = c->lev[l];
  for (int it = 0; it < n; ++it)
    for (int d = 0; d < c->D; ++d) {
      if (tma_for(c, l, d))
        launch_rb_tma(c->D, Lv.g, Lv.f, d, Lv.f.u2[d], c->counters + 3,
                      c->P.inv_re / (Lv.g.h * Lv.g.h), c->stream, c->tma_wait_ns);
      else {
        int ty = 0, kc = 0, np = 1, bx = 0, kern = 0;
        ring_shape_of(d, Lv.g, &ty, &kc, &np, &bx, &kern);
        if (kern == 1)
          launch_v_rb_pair(Lv.g, Lv.f, d, Lv.f.u2[d], c->P.inv_re, c->stream, ty, kc);
        else
          launch_v_rb_fused<float>(c->D, Lv.g, Lv.f, d, Lv.f.u2[d], c->P.inv_re, c->stream, ty,
                                   kc, np, bx);
      }
      std::swap(Lv.f.u[d], Lv.f.u2[d]);
    }
  if (n & 1)
    for (int d = 0; d < c->D; ++d) {
      cudaMemcpyAsync(Lv.f.u2[d], Lv.f.u[d], (size_t)level_elems(Lv.g) * sizeof(float),
                      cudaMemcpyDeviceToDevice, c->stream);
      std::swap(Lv.f.u[d], Lv.f.u2[d]);
    }
}

// FP32 V-cycle for the correction e of A e = r on level l; the coarsest
// level is solved in FP64.
void vcycle_p32(bfibm_ctx* c, int l) {
  Level& Lv = c->lev[l];
  cudaStream_t s = c->stream;
  if (l == c->tail_lev) {
    launch_tail(false, c->self_tab, c->self_list, 1, nullptr,
                tail_smem(c->lev[c->L - 1].g, false), s);
    return;
  }
  if (l == c->L - 1) {
    long long n = level_elems(Lv.g);
    launch_f32_to_f64(Lv.f.pf, Lv.d.pf, n, s);
    cudaMemsetAsync(Lv.d.p, 0, n * sizeof(double), s);
    launch_coarse_p<double>(c->D, Lv.g, Lv.d, c->P.coarse_sweeps, s);
    launch_f64_to_f32(Lv.d.p, Lv.f.p, n, s);
    return;
  }
  smooth_p32(c, l, c->P.nu1);
  launch_p_residual<float>(c->D, Lv.g, Lv.f, s);
  Level& Lc = c->lev[l + 1];
  launch_restrict_cell<float>(c->D, Lv.g, Lc.g, Lv.f.pr, Lc.f.pf, Lc.f.p, s);
  vcycle_p32(c, l + 1);
  launch_prolong_cell<float>(c->D, Lv.g, Lc.g, Lc.f.p, Lv.f.p, s);
  smooth_p32(c, l, c->P.nu2);
}

void vcycle_v32(bfibm_ctx* c, int l) {
  Level& Lv = c->lev[l];
  cudaStream_t s = c->stream;
  if (l == c->tail_lev) {
    launch_tail(true, c->self_tab, c->self_list, 1, nullptr,
                tail_smem(c->lev[c->L - 1].g, true), s);
    return;
  }
  if (l == c->L - 1) {
    long long n = level_elems(Lv.g);
    for (int d = 0; d < c->D; ++d) {
      launch_f32_to_f64(Lv.f.uf[d], Lv.d.uf[d], n, s);
      cudaMemsetAsync(Lv.d.u[d], 0, n * sizeof(double), s);
    }
    launch_coarse_v<double>(c->D, Lv.g, Lv.d, c->P.coarse_sweeps, c->P.inv_re, s);
    for (int d = 0; d < c->D; ++d) launch_f64_to_f32(Lv.d.u[d], Lv.f.u[d], n, s);
    return;
  }
  smooth_v32(c, l, c->P.nu1);
  launch_v_residual<float>(c->D, Lv.g, Lv.f, c->P.inv_re, s);
  Level& Lc = c->lev[l + 1];
  restrict_faces(c, Lv.g, Lc.g, Lv.f.ur, Lc.f.uf, Lc.f.u);
  vcycle_v32(c, l + 1);
  prolong_faces(c, Lv.g, Lc.g, Lc.f.u, Lv.f.u);
  smooth_v32(c, l, c->P.nu2);
}

// Defect correction: r = f - A x in FP64 (handed to FP32), c->inner FP32
// V-cycles for the correction of A e = r (the first from e = 0, each next one
// from the last iterate: the same V-cycles in exact arithmetic, one FP64
// residual per `inner` of them), x += e in FP64. ncycles > 0: that many
// V-cycles; else until rtol, with max_cycles V-cycles at most. Returns the
// V-cycles used (a multiple of c->inner in tolerance mode).
bfibm_status solve_p_mixed(bfibm_ctx* c, int ncycles, int* used) {
  Level& L0 = c->lev[0];
  cudaStream_t s = c->stream;
  double* one[3] = {L0.d.pf, nullptr, nullptr};
  bool tol = ncycles <= 0;
  const int inner = c->inner;
  int nb = red_blocks_3d(c->D, L0.g);
  if (tol || c->collect_stats) launch_norm2(c->D, L0.g, one, 0, c->sc, SL_PF, s);
  int vmax = tol ? c->P.max_cycles : ncycles;
  int maxc = dc_iterations(vmax, inner);
  bfibm_status st = tol ? BFIBM_ENOCONV : BFIBM_OK;
  double* xs[3] = {L0.d.p, nullptr, nullptr};
  float* es[3] = {L0.f.p, nullptr, nullptr};
  if (tol && c->capturing) {
    cudaMemsetAsync(c->dev_cycles + 1, 0, sizeof(int), s);
    launch_p_residual_mixed(c->D, L0.g, L0.d, L0.f.pf, L0.f.p, nullptr, s);
    c->loop_inner[1] = inner;
    bfibm_status cs = capture_while(c, 1, [&](cudaGraphConditionalHandle h) {
      cudaStream_t b = c->stream;
      for (int q = 0; q < inner; ++q) vcycle_p32(c, 0);
      xs[0] = L0.d.p;
      es[0] = L0.f.p;
      launch_add_correction(c->D, L0.g, xs, es, 0, b);
      launch_sub_mean(c->D, L0.g, L0.d.p, c->sc, b);
      launch_p_residual_mixed(c->D, L0.g, L0.d, L0.f.pf, L0.f.p, c->sc.partial, b);
      launch_finalize_sum(c->sc.partial, nb, c->sc.out, SL_PR, 1.0, b);
      if (c->P.div_tol > 0.0) launch_finalize_max(c->sc.partial + nb, nb, c->sc.out, SL_PRMAX, b);
      launch_tol_check(h, c->sc.out, SL_PF, SL_PR, c->P.rtol, maxc, c->dev_cycles + 1,
                       c->loop_total + 1, c->counters + 4, b, SL_PRMAX, div_scale(c),
                       c->P.div_tol);
    });
    *used = -1;
    return cs;
  }
  int k = 0, vdone = 0;
  for (k = 1; k <= maxc; ++k) {
    launch_p_residual_mixed(c->D, L0.g, L0.d, L0.f.pf, L0.f.p, tol ? c->sc.partial : nullptr, s);
    if (tol) {
      launch_finalize_sum(c->sc.partial, nb, c->sc.out, SL_PR, 1.0, s);
      launch_finalize_max(c->sc.partial + nb, nb, c->sc.out, SL_PRMAX, s);
      bfibm_status rs = read_scalars(c);
      if (rs != BFIBM_OK) return rs;
      if (p_converged(c, c->host_sc)) {
        st = BFIBM_OK;
        break;
      }
    }
    const int nv = tol ? inner : std::min(inner, ncycles - vdone);
    for (int q = 0; q < nv; ++q) vcycle_p32(c, 0);
    vdone += nv;
    xs[0] = L0.d.p;
    es[0] = L0.f.p;
    launch_add_correction(c->D, L0.g, xs, es, 0, s);
    launch_sub_mean(c->D, L0.g, L0.d.p, c->sc, s);
  }
  if (c->collect_stats || tol) {
    launch_p_residual_mixed(c->D, L0.g, L0.d, L0.f.pf, L0.f.p, c->sc.partial, s);
    launch_finalize_sum(c->sc.partial, nb, c->sc.out, SL_PR, 1.0, s);
  }
  *used = vdone;
  return st;
}

bfibm_status solve_v_mixed(bfibm_ctx* c, int ncycles, int* used) {
  Level& L0 = c->lev[0];
  cudaStream_t s = c->stream;
  bool tol = ncycles <= 0;
  const int inner = c->inner;
  int nb = red_blocks_3d(c->D, L0.g);
  if (tol || c->collect_stats) launch_norm2(c->D, L0.g, L0.d.uf, c->D, c->sc, SL_VF, s);
  int vmax = tol ? c->P.max_cycles : ncycles;
  int maxc = dc_iterations(vmax, inner);
  bfibm_status st = tol ? BFIBM_ENOCONV : BFIBM_OK;
  if (tol && c->capturing) {
    cudaMemsetAsync(c->dev_cycles, 0, sizeof(int), s);
    launch_v_residual_mixed(c->D, L0.g, L0.d, L0.f.uf, L0.f.u, c->vdiag, c->P.inv_re, nullptr, s);
    c->loop_inner[0] = inner;
    bfibm_status cs = capture_while(c, 0, [&](cudaGraphConditionalHandle h) {
      cudaStream_t b = c->stream;
      for (int q = 0; q < inner; ++q) vcycle_v32(c, 0);
      launch_add_correction(c->D, L0.g, L0.d.u, L0.f.u, c->D, b);
      launch_v_residual_mixed(c->D, L0.g, L0.d, L0.f.uf, L0.f.u, c->vdiag, c->P.inv_re, c->sc.partial, b);
      launch_finalize_sum(c->sc.partial, nb, c->sc.out, SL_VR, 1.0, b);
      launch_tol_check(h, c->sc.out, SL_VF, SL_VR, c->P.rtol, maxc, c->dev_cycles,
                       c->loop_total, c->counters + 4, b);
    });
    *used = -1;
    return cs;
  }
  int k = 0, vdone = 0;
  for (k = 1; k <= maxc; ++k) {
    launch_v_residual_mixed(c->D, L0.g, L0.d, L0.f.uf, L0.f.u, c->vdiag, c->P.inv_re,
                            tol ? c->sc.partial : nullptr, s);
    if (tol) {
      launch_finalize_sum(c->sc.partial, nb, c->sc.out, SL_VR, 1.0, s);
      bfibm_status rs = read_scalars(c);
      if (rs != BFIBM_OK) return rs;
      double fn = std::sqrt(c->host_sc[SL_VF]), rn = std::sqrt(c->host_sc[SL_VR]);
      if ((fn > 0.0 ? rn / fn : 0.0) <= c->P.rtol) {
        st = BFIBM_OK;
        break;
      }
    }
    const int nv = tol ? inner : std::min(inner, ncycles - vdone);
    for (int q = 0; q < nv; ++q) vcycle_v32(c, 0);
    vdone += nv;
    launch_add_correction(c->D, L0.g, L0.d.u, L0.f.u, c->D, s);
  }
  if (c->collect_stats || tol) {
    launch_v_residual_mixed(c->D, L0.g, L0.d, L0.f.uf, L0.f.u, c->vdiag, c->P.inv_re, c->sc.partial, s);
    launch_finalize_sum(c->sc.partial, nb, c->sc.out, SL_VR, 1.0, s);
  }
  *used = vdone;
  return st;
}

// Flexible CG for the mixed-precision viscous solve: the FP32 V-cycle (c->inner
// of them) preconditions an FP64 conjugate-gradient iteration on A x = f. The
// residual r is kept in FP64 (recurrence r -= alpha q) and its norm decides
// convergence; a tolerance solve stops after max_cycles V-cycles at most, a
// fixed one runs ncycles V-cycles. Returns V-cycles used.
bfibm_status solve_v_fcg(bfibm_ctx* c, int ncycles, int* used) {
  Level& L0 = c->lev[0];
  cudaStream_t s = c->stream;
  const int D = c->D;
  const bool tol = ncycles <= 0;
  const int inner = c->inner;
  const int nb = red_blocks_3d(D, L0.g);
  const int nbf = fcg_flat_blocks(L0.g);
  double* w[3] = {L0.d.u2[0], L0.d.u2[1], L0.d.u2[2]};
  double* r[3] = {L0.d.ur[0], L0.d.ur[1], L0.d.ur[2]};
  if (tol || c->collect_stats) launch_norm2(D, L0.g, L0.d.uf, D, c->sc, SL_VF, s);
  const int maxc = dc_iterations(tol ? c->P.max_cycles : ncycles, inner);
  // r = f - A x in FP64 (and as the FP32 right-hand side), the first
  // direction flagged by p.q = 0
  launch_v_residual_mixed(D, L0.g, L0.d, L0.f.uf, L0.f.u, c->vdiag, c->P.inv_re, c->sc.partial,
                          s, r);
  launch_finalize_sum(c->sc.partial, nb, c->sc.out, SL_VR, 1.0, s);
  CK(cudaMemsetAsync(c->sc.out + SL_PQ, 0, sizeof(double), s));
  auto iteration = [&](cudaStream_t b, int nv) {
    for (int q = 0; q < nv; ++q) vcycle_v32(c, 0);
    if (D == 3) launch_f32_to_f64_3(L0.f.u, c->cg_z, level_elems(L0.g), b);
    else
      for (int d = 0; d < D; ++d) launch_f32_to_f64(L0.f.u[d], c->cg_z[d], level_elems(L0.g), b);
    launch_fcg_apply(D, L0.g, L0.d, c->cg_z, c->vdiag, c->P.inv_re, w, c->cg_q, c->sc.partial, b);
    launch_finalize_sum(c->sc.partial, nb, c->sc.out, SL_ZQ, 1.0, b);
    launch_fcg_dir(D, L0.g, c->cg_z, w, c->cg_p, c->cg_q, r, c->sc.out, SL_ZQ, SL_PQ,
                   c->sc.partial, b);
    launch_finalize_sum(c->sc.partial, nbf, c->sc.out, SL_PQ, 1.0, b);
    launch_finalize_sum(c->sc.partial + nbf, nbf, c->sc.out, SL_PRR, 1.0, b);
    launch_fcg_update(D, L0.g, L0.d.u, c->cg_p, c->cg_q, r, L0.f.uf, L0.f.u, c->sc.out, SL_PQ,
                      SL_PRR, c->sc.partial, b);
    launch_finalize_sum(c->sc.partial, nbf, c->sc.out, SL_VR, 1.0, b);
  };
  if (tol && c->capturing) {
    cudaMemsetAsync(c->dev_cycles, 0, sizeof(int), s);
    c->loop_inner[0] = inner;
    bfibm_status cs = capture_while(c, 0, [&](cudaGraphConditionalHandle h) {
      iteration(c->stream, inner);
      launch_tol_check(h, c->sc.out, SL_VF, SL_VR, c->P.rtol, maxc, c->dev_cycles, c->loop_total,
                       c->counters + 4, c->stream);
    });
    if (cs == BFIBM_OK) {   // the true FP64 residual of the final iterate, checked
      launch_v_residual_mixed(D, L0.g, L0.d, L0.f.uf, L0.f.u, c->vdiag, c->P.inv_re,
                              c->sc.partial, s);
      launch_finalize_sum(c->sc.partial, nb, c->sc.out, SL_VR, 1.0, s);
      launch_res_check(c->sc.out, SL_VF, SL_VR, kTrueResidualSlack * c->P.rtol, c->counters + 4,
                       s);
    }
    *used = -1;
    return cs;
  }
  bfibm_status st = tol ? BFIBM_ENOCONV : BFIBM_OK;
  int vdone = 0;
  for (int k = 1; k <= maxc; ++k) {
    if (tol) {
      bfibm_status rs = read_scalars(c);
      if (rs != BFIBM_OK) return rs;
      double fn = std::sqrt(c->host_sc[SL_VF]), rn = std::sqrt(c->host_sc[SL_VR]);
      if ((fn > 0.0 ? rn / fn : 0.0) <= c->P.rtol) {
        st = BFIBM_OK;
        break;
      }
    }
    const int nv = tol ? inner : std::min(inner, ncycles - vdone);
    iteration(s, nv);
    vdone += nv;
  }
  if (tol && st != BFIBM_OK) {
    bfibm_status rs = read_scalars(c);
    if (rs != BFIBM_OK) return rs;
    double fn = std::sqrt(c->host_sc[SL_VF]), rn = std::sqrt(c->host_sc[SL_VR]);
    if ((fn > 0.0 ? rn / fn : 0.0) <= c->P.rtol) st = BFIBM_OK;
  }
  if (c->collect_stats || tol) {   // the true FP64 residual of the final iterate
    launch_v_residual_mixed(D, L0.g, L0.d, L0.f.uf, L0.f.u, c->vdiag, c->P.inv_re,
                            c->sc.partial, s);
    launch_finalize_sum(c->sc.partial, nb, c->sc.out, SL_VR, 1.0, s);
  }
  if (tol && st == BFIBM_OK) {
    bfibm_status rs = read_scalars(c);
    if (rs != BFIBM_OK) return rs;
    double fn = std::sqrt(c->host_sc[SL_VF]), rn = std::sqrt(c->host_sc[SL_VR]);
    if (!((fn > 0.0 ? rn / fn : 0.0) <= kTrueResidualSlack * c->P.rtol)) st = BFIBM_ENOCONV;
  }
  *used = vdone;
  return st;
}

// ------------------------------------------------------------------ stages
void stage_rhs(bfibm_ctx* c) {
  launch_adv_rhs(c->D, c->lev[0].g, c->uvel, c->rho, c->frc, c->lev[0].d, c->P.c_force,
                 c->P.flow_axis, c->G_dev, c->stream);
}
void stage_divergence(bfibm_ctx* c) {
  double scale = c->P.sigma / c->P.euler / c->P.dt;
  const int o = c->lev[0].g.open;
  launch_divergence(c->D, c->lev[0].g, c->lev[0].d.u, c->lev[0].d.pf, scale, c->sc, c->stream,
                    o >= 0 ? c->lev[0].d.beta[o] : nullptr, c->p_out);
}
void stage_project(bfibm_ctx* c) {
  double coef = c->P.euler * c->P.dt / c->P.sigma;
  DivCheck dc{c->sc.out, SL_DIVACC, SL_DIVSTEP, SL_DIVALL, c->P.div_tol, c->counters + 5,
              c->p_out};
  launch_project(c->D, c->lev[0].g, c->lev[0].d.u, c->lev[0].d.p, c->lev[0].d.beta, c->uvel,
                 coef, dc, c->stream);
}
void stage_interp_advance(bfibm_ctx* c) {
  launch_interp_advance(c->D, c->lev[0].g, c->N, c->uvel, c->P.phi_kind, c->P.dt / c->P.sigma,
                        c->stream);
}
void stage_springs(bfibm_ctx* c) { launch_springs(c->D, c->lev[0].g, c->N, c->S, c->stream); }

void build_coefficients(bfibm_ctx* c) {
  Level& L0 = c->lev[0];
  launch_coef_fine(c->D, L0.g, c->rho, L0.d.beta, L0.d.m, c->P.sigma / c->P.dt, c->stream);
  for (int l = 1; l < c->L; ++l) {
    // Eq. (ViscCoarseGrid): gamma_lh may differ per coarse grid
    const double gam = (l < 8 && c->P.gamma_levels[l] > 0.0) ? c->P.gamma_levels[l]
                                                              : c->P.gamma_coarse;
    launch_coef_restrict(c->D, c->lev[l - 1].g, c->lev[l].g, c->lev[l - 1].d, c->lev[l].d, gam,
                         c->stream);
  }
  if (c->P.precision == 1) {
    launch_v_diag(c->D, L0.g, L0.d, c->vdiag, c->P.inv_re, c->stream);
    for (int l = 0; l < c->L; ++l) {
      launch_coef_to_f32(c->D, c->lev[l].g, c->lev[l].d, c->lev[l].f, c->stream);
      const double h = c->lev[l].g.h;
      launch_v_idg32(c->D, c->lev[l].g, c->lev[l].d, c->lev[l].f, c->P.inv_re / (h * h), c->stream);
    }
  }
}

SpreadArgs spread_args(const bfibm_ctx* c) {
  SpreadArgs a;
  a.D = c->D;
  a.phi_kind = c->P.phi_kind;
  a.omega = c->P.omega;
  a.omega_mu = c->P.omega_mu;
  a.amp_rho = (c->P.rho_ratio - 1.0) * c->P.rho_f * c->P.d0_vol;
  a.mu_out = c->P.mu_f;
  double tw = 2.0 * c->P.omega_mu;
  a.mu_coef = (c->D == 3 ? tw * tw * tw : tw * tw) * (c->P.mu_ratio * c->P.mu_f - c->P.mu_f);
  a.rho_f = c->P.rho_f;
  a.scale = c->spread_scale;
  return a;
}

// Break test and forces at the current nodes, then f, rho, mu and the
// coefficient hierarchy.
void refresh(bfibm_ctx* c) {
  Level& L0 = c->lev[0];
  stage_springs(c);
  launch_reset_fields(c->D, L0.g, c->frc, c->rho, L0.d.muc, L0.d.mue, c->P.rho_f, c->P.mu_f,
                      c->stream);
  if (c->N.eta > 0) {
    launch_bin(c->D, L0.g, c->tg, c->N, c->stream);
    launch_spread(c->D, L0.g, c->tg, c->N, spread_args(c), c->frc, c->rho, L0.d.muc, L0.d.mue,
                  c->stream);
  }
  launch_spread_finish(c->D, L0.g, spread_args(c), c->frc, c->rho, c->stream);
  build_coefficients(c);
}

// One time step (Sec. 3.4 order).
bfibm_status queue_step(bfibm_ctx* c) {
  stage_rhs(c);
  bool mixed = c->P.precision == 1;
  bfibm_status st = mixed ? (c->krylov ? solve_v_fcg(c, c->P.vc_visc, &c->cycles_visc)
                                        : solve_v_mixed(c, c->P.vc_visc, &c->cycles_visc))
                          : solve_v(c, c->P.vc_visc, &c->cycles_visc);
  if (st != BFIBM_OK && st != BFIBM_ENOCONV) return st;
  stage_divergence(c);
  bfibm_status st2 = mixed ? solve_p_mixed(c, c->P.vc_p, &c->cycles_p)
                           : solve_p(c, c->P.vc_p, &c->cycles_p);
  if (st2 != BFIBM_OK && st2 != BFIBM_ENOCONV) return st2;
  stage_project(c);
  stage_interp_advance(c);
  launch_step_increment(c->step_dev, c->stream);
  refresh(c);
  return (st == BFIBM_ENOCONV || st2 == BFIBM_ENOCONV) ? BFIBM_ENOCONV : BFIBM_OK;
}

bfibm_status ensure_ready(bfibm_ctx* c) {
  if (c->dirty) {
    refresh(c);
    c->dirty = false;
    CK(cudaGetLastError());
  }
  return BFIBM_OK;
}

// Reads the device status words (waits for the context's stream) and reports
// what happened since the last report: BFIBM_ETIMEOUT (the context is
// poisoned) when a bounded device wait ran out, BFIBM_ENOCONV when a solve
// stopped above its tolerance or a projection left max |D.u| above div_tol.
bfibm_status check_status(bfibm_ctx* c) {
  int cnt[kCounters];
  CK(cudaMemcpyAsync(cnt, c->counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const bool timeout = cnt[3] != c->seen[3];
  const bool nonconv = cnt[4] != c->seen[4];
  const bool div = cnt[5] != c->seen[5];
  for (int q = 0; q < kCounters; ++q) c->seen[q] = cnt[q];
  if (timeout) {
    c->poisoned = 1;
    return set_err(c, BFIBM_ETIMEOUT, "a bounded device wait of the TMA sweep ran out");
  }
  if (nonconv || div)
    return set_err(c, BFIBM_ENOCONV,
                   nonconv ? "a solve stopped above its relative-residual tolerance"
                           : "max |D.u| after a projection exceeded div_tol");
  return BFIBM_OK;
}

// Queues nsteps time steps; with `report` it then waits for them and returns
// what check_status reports (a batch step queues only and reports in
// bfibm_batch_wait).
bfibm_status do_steps(bfibm_ctx* c, int nsteps, bool report) {
  bfibm_status st = ensure_ready(c);
  if (st != BFIBM_OK) return st;
  bfibm_status agg = BFIBM_OK;
  if (c->use_graph) {
    if (!c->gexec) {
      cudaGraph_t graph = nullptr;
      CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      c->capturing = true;
      bfibm_status qs = queue_step(c);
      c->capturing = false;
      cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
      if (qs != BFIBM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return qs;
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
      c->graph_kernels = count_kernel_nodes(graph);
      e = cudaGraphInstantiate(&c->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    for (int k = 0; k < nsteps; ++k) CK(cudaGraphLaunch(c->gexec, c->stream));
  } else {
    for (int k = 0; k < nsteps; ++k) {
      bfibm_status qs = queue_step(c);
      if (qs == BFIBM_ENOCONV) agg = BFIBM_ENOCONV;
      else if (qs != BFIBM_OK) return qs;
    }
  }
  CK(cudaGetLastError());
  c->step_host += nsteps;
  if (report) {
    bfibm_status cs = check_status(c);
    if (cs != BFIBM_OK) return cs;
  }
  return agg;
}

// ------------------------------------------------------------ field access
double* field_ptr(bfibm_ctx* c, int which, int comp, int level) {
  if (level < 0 || level >= c->L) return nullptr;
  int D = c->D;
  bool vec = (which == BFIBM_F_U || which == BFIBM_F_UT || which == BFIBM_F_URHS ||
              which == BFIBM_F_RHO || which == BFIBM_F_FORCE || which == BFIBM_F_BETA ||
              which == BFIBM_F_M || which == BFIBM_F_URES);
  if (vec && (comp < 0 || comp >= D)) return nullptr;
  if (which == BFIBM_F_MUE && (comp < 0 || comp >= edge_count(D))) return nullptr;
  bool fine_only = which == BFIBM_F_U || which == BFIBM_F_RHO || which == BFIBM_F_FORCE;
  if (fine_only && level != 0) return nullptr;
  LevelPtrs<double>& L = c->lev[level].d;
  switch (which) {
    case BFIBM_F_U: return c->uvel[comp];
    case BFIBM_F_UT: return L.u[comp];
    case BFIBM_F_URHS: return L.uf[comp];
    case BFIBM_F_P: return L.p;
    case BFIBM_F_PRHS: return L.pf;
    case BFIBM_F_RHO: return c->rho[comp];
    case BFIBM_F_FORCE: return c->frc[comp];
    case BFIBM_F_MUC: return L.muc;
    case BFIBM_F_MUE: return L.mue[comp];
    case BFIBM_F_BETA: return L.beta[comp];
    case BFIBM_F_M: return L.m[comp];
    case BFIBM_F_URES: return L.ur[comp];
    case BFIBM_F_PRES: return L.pr;
  }
  return nullptr;
}

float* field_ptr32(bfibm_ctx* c, int which, int comp, int level) {
  if (c->P.precision != 1 || level < 0 || level >= c->L) return nullptr;
  int D = c->D;
  bool vec = (which == BFIBM_F_UT || which == BFIBM_F_URHS || which == BFIBM_F_BETA ||
              which == BFIBM_F_M || which == BFIBM_F_URES || which == BFIBM_F_IDG);
  if (vec && (comp < 0 || comp >= D)) return nullptr;
  if (which == BFIBM_F_MUE && (comp < 0 || comp >= edge_count(D))) return nullptr;
  LevelPtrs<float>& L = c->lev[level].f;
  if (which == BFIBM_F_IDG) return L.idg[comp];
  switch (which) {
    case BFIBM_F_UT: return L.u[comp];
    case BFIBM_F_URHS: return L.uf[comp];
    case BFIBM_F_P: return L.p;
    case BFIBM_F_PRHS: return L.pf;
    case BFIBM_F_MUC: return L.muc;
    case BFIBM_F_MUE: return L.mue[comp];
    case BFIBM_F_BETA: return L.beta[comp];
    case BFIBM_F_M: return L.m[comp];
    case BFIBM_F_URES: return L.ur[comp];
    case BFIBM_F_PRES: return L.pr;
  }
  return nullptr;
}

bfibm_status copy_field32(bfibm_ctx* c, int which, int comp, int level, void* ext, bool to_ext) {
  float* p = field_ptr32(c, which, comp, level);
  if (!p || !ext) return set_err(c, BFIBM_EINVAL, "bad FP32 field selector or pointer");
  const Geo& g = c->lev[level].g;
  size_t row = (size_t)g.s[0] * sizeof(float);
  size_t pitch = (size_t)g.st[1] * sizeof(float);
  size_t rows = (size_t)g.s[1] * g.s[2];
  if (to_ext)
    CK(cudaMemcpy2DAsync(ext, row, p, pitch, row, rows, cudaMemcpyDeviceToHost, c->stream));
  else
    CK(cudaMemcpy2DAsync(p, pitch, ext, row, row, rows, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return BFIBM_OK;
}

bfibm_status copy_field(bfibm_ctx* c, int which, int comp, int level, void* ext, bool to_ext,
                        cudaMemcpyKind kind) {
  double* p = field_ptr(c, which, comp, level);
  if (!p || !ext) return set_err(c, BFIBM_EINVAL, "bad field selector or pointer");
  const Geo& g = c->lev[level].g;
  size_t row = (size_t)g.s[0] * sizeof(double);
  size_t pitch = (size_t)g.st[1] * sizeof(double);
  size_t rows = (size_t)g.s[1] * g.s[2];
  if (to_ext)
    CK(cudaMemcpy2DAsync(ext, row, p, pitch, row, rows, kind, c->stream));
  else
    CK(cudaMemcpy2DAsync(p, pitch, ext, row, row, rows, kind, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return BFIBM_OK;
}

void free_lag(bfibm_ctx* c, bool nodes, bool springs) {
  if (nodes) {
    for (void* q : {(void*)c->N.X, (void*)c->N.U, (void*)c->N.F, (void*)c->N.tile, (void*)c->N.perm,
                    (void*)c->N.count, (void*)c->N.start, (void*)c->N.cursor, (void*)c->N.tw,
                    (void*)c->N.tlo})
      if (q) cudaFree(q);
    long long keep_eta = 0;
    int* clamped = c->N.clamped;
    int* nonfinite = c->N.nonfinite;
    c->N = NodeSet{};
    c->N.eta = keep_eta;
    c->N.clamped = clamped;
    c->N.nonfinite = nonfinite;
  }
  if (springs) {
    for (void* q : {(void*)c->S.ab, (void*)c->S.rest, (void*)c->S.K, (void*)c->S.brk,
                    (void*)c->S.broken, (void*)c->S.ev_id, (void*)c->S.ev_step,
                    (void*)c->S.fvec, (void*)c->S.adj_start, (void*)c->S.adj})
      if (q) cudaFree(q);
    int* evc = c->S.ev_count;
    long long* step = c->S.step;
    c->S = SpringSet{};
    c->S.ev_count = evc;
    c->S.step = step;
  }
}

template <typename T>
cudaError_t dmalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count > 0 ? count : 1));
}

// ---------------------------------------------------------- persistent batch
// A batch in persistent mode steps its members in lock step, one CUDA graph
// per batch step. Inside it every level and phase of the mixed-precision
// solves (sweeps, residuals, transfers, coarsest solves, the FP64 level-0
// steps and reductions) is one launch over a device work list of (member,
// block) items, so members of different sizes share each launch; a block
// of a launch strides over the list. Each solve's device loop runs while any
// member still iterates: a member whose test is met leaves the mask that
// every launch of the loop reads, so it stops where it would stop alone. The
// stages around the solves (right-hand side, divergence, projection, nodes,
// springs, spread, coefficients) run per member on forked branches of the
// same graph. Per member the arithmetic, the block decompositions of the
// reductions and the tests are those of its own step graph, so results come
// out bit-identical to the member stepped alone.
struct PList {
  BItem* dev = nullptr;
  int n = 0;
  int grid = 0;   // blocks of a 256-thread launch over the list
};

struct PShape {   // a batched sweep: rows, chunk planes, planes per phase, threads per row
  int TY = 4, KC = 8, NP = 1, bx = 32;
  int all = 0;    // 1: one block per item; 0: the resident blocks stride over the items
  int kern = 0;   // 0 the ring sweep, 1 the pair sweep (viscous; one block per item)
  int perz = 0;   // the pair sweep: the streaming axis is periodic in every member
  size_t smem = 0;
  int grid = 0;
};

struct Persist {
  std::vector<bfibm_ctx*> mem;       // table order: level-0 cells descending
  std::vector<long long> version;    // the members' versions the plan was built for
  BMember* tab = nullptr;
  int* act = nullptr;                // the mask of the solve being run
  long long* iters = nullptr;        // batch device-loop iterations so far (viscous, pressure)
  int depth = 0;                     // levels of the deepest member
  int nu1 = 2, nu2 = 2, inner = 1, krylov = 0;
  int unroll = 0;                    // > 0: each solve loop unrolled to this many iterations
  long long tail_cells = 4096;       // levels of at most this many cells: the coarse-level kernel
  std::vector<int> ptail;            // each member's first level in that kernel (L: none)
  // per level l: the members that smooth on l (l below their coarsest level)
  PList swv[kMaxLevels], swp[kMaxLevels];   // ring-sweep blocks (viscous, pressure shape)
  PShape shv[kMaxLevels], shp[kMaxLevels];
  PList en[kMaxLevels];   // 3D blocks over the cells of l: residuals, prolongations
  PList rs[kMaxLevels];   // over the stored faces of l + 1: face restriction
  PList rn[kMaxLevels];   // over the cells of l + 1: cell restriction
  PList fl[kMaxLevels];   // flat blocks over the elements of l: copies after odd sweep counts
  PList co[kMaxLevels];   // one item per member whose coarsest level is l
  size_t co_smem[kMaxLevels][2] = {};
  int* tail[kMaxLevels] = {};        // members whose coarse-level cluster kernel starts on l
  int ntail[kMaxLevels] = {};
  size_t tail_smem[kMaxLevels][2] = {};
  // that kernel runs on a branch of its own, beside the other members' work on
  // the same and deeper levels
  cudaStream_t tstream[kMaxLevels] = {};
  cudaEvent_t tfork[kMaxLevels] = {}, tjoin[kMaxLevels] = {};
  // level 0, every member
  PList a3, ared, aflat, aconv;      // 3D, cell reductions, flat CG passes, conversions
  PList fin3, finred, finflat;       // one item per member, gx = its producer's blocks
  bool masked = false;               // queuing the body of a device loop
  cudaStream_t stream = nullptr, aux = nullptr;
  cudaEvent_t fork = nullptr, done = nullptr;
  std::vector<cudaEvent_t> join;
  cudaGraphExec_t gexec = nullptr;
  long long graph_kernels = 0, body_kernels[2] = {0, 0};
  std::vector<void*> allocs;
  std::string err;
};

// whether member m smooths on level l with launches (above its coarsest level
// and above the level where its coarse-level cluster kernel starts)
bool p_smooths(const Persist& P, int m, int l) {
  return l < std::min(P.ptail[m], P.mem[m]->L - 1);
}

void persist_free(Persist* P) {
  if (!P) return;
  if (P->stream) cudaStreamSynchronize(P->stream);
  if (P->gexec) cudaGraphExecDestroy(P->gexec);
  for (void* a : P->allocs) cudaFree(a);
  for (cudaEvent_t e : P->join) cudaEventDestroy(e);
  for (int l = 0; l < kMaxLevels; ++l) {
    if (P->tfork[l]) cudaEventDestroy(P->tfork[l]);
    if (P->tjoin[l]) cudaEventDestroy(P->tjoin[l]);
    if (P->tstream[l]) cudaStreamDestroy(P->tstream[l]);
  }
  if (P->fork) cudaEventDestroy(P->fork);
  if (P->done) cudaEventDestroy(P->done);
  if (P->aux) cudaStreamDestroy(P->aux);
  if (P->stream) cudaStreamDestroy(P->stream);
  cudaGetLastError();
  delete P;
}

int device_sms() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 152;
  }
  return n;
}

// Items of the members `use` accepts, each member's blocks in the order
// x, y, z; `grid_of(member)` gives the block grid its single-instance launch
// would use.
template <class Use, class Grid>
bool make_items(int nm, Use use, Grid grid_of, std::vector<BItem>& v) {
  v.clear();
  for (int m = 0; m < nm; ++m) {
    if (!use(m)) continue;
    const dim3 gr = grid_of(m);
    if (gr.x > 65535u || gr.y > 65535u || gr.z > 65535u) return false;
    for (unsigned z = 0; z < gr.z; ++z)
      for (unsigned y = 0; y < gr.y; ++y)
        for (unsigned x = 0; x < gr.x; ++x)
          v.push_back(BItem{m, (unsigned short)x, (unsigned short)y, (unsigned short)z,
                            (unsigned short)gr.x, (unsigned short)gr.y, (unsigned short)gr.z});
  }
  return true;
}

cudaError_t upload(Persist& P, const std::vector<BItem>& v, PList& L) {
  L.n = (int)v.size();
  L.dev = nullptr;
  L.grid = 0;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)&L.dev, v.size() * sizeof(BItem));
  if (e != cudaSuccess) return e;
  P.allocs.push_back(L.dev);
  const int cap = device_sms() * 8;   // 256-thread blocks resident per SM
  L.grid = L.n < cap ? L.n : cap;
  return cudaMemcpy(L.dev, v.data(), v.size() * sizeof(BItem), cudaMemcpyHostToDevice);
}

// The sweep items of level l for a shape, and the launch's grid and shared memory.
cudaError_t sweep_list(Persist& P, int l, int K, PShape& sh, PList& L) {
  const int nm = (int)P.mem.size();
  int W = 0;
  for (int m = 0; m < nm; ++m)
    if (p_smooths(P, m, l))
      W = std::max(W, sh.kern ? P.mem[m]->lev[l].g.n[0] : P.mem[m]->lev[l].g.s[0]);
  sh.smem = sh.kern ? (size_t)4 * (sh.TY + 2) * W * sizeof(float) : b_sweep_smem(sh.NP, sh.TY, W);
  if (sh.kern) sh.all = 1;
  std::vector<BItem> v;
  make_items(nm, [&](int m) { return p_smooths(P, m, l); },
             [&](int m) {
               const Geo& g = P.mem[m]->lev[l].g;
               return dim3((g.n[1] + sh.TY - 1) / sh.TY, (g.n[2] + sh.KC - 1) / sh.KC, 1);
             }, v);
  if (L.dev) {
    cudaFree(L.dev);
    P.allocs.erase(std::remove(P.allocs.begin(), P.allocs.end(), (void*)L.dev), P.allocs.end());
  }
  cudaError_t e = upload(P, v, L);
  if (e != cudaSuccess) return e;
  if (sh.kern) {
    sh.grid = L.n;
    return cudaSuccess;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, b_sweep_kernel(K, sh.NP),
                                                    sh.bx * (sh.TY + 2), sh.smem) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  const int cap = device_sms() * std::max(per_sm, 1);
  sh.grid = sh.all || L.n < cap ? L.n : cap;
  return cudaSuccess;
}

// The built-in sweep shape of level l: one thread per point pair of the
// widest member's rows (at most 128), 4 rows, chunks giving about three
// blocks per SM.
PShape default_shape(const Persist& P, int l) {
  PShape sh;
  int np = 1, nR = 1 << 30;
  long long tiles = 0;
  for (size_t m = 0; m < P.mem.size(); ++m)
    if (p_smooths(P, (int)m, l)) {
      const Geo& g = P.mem[m]->lev[l].g;
      np = std::max(np, (g.n[0] + 1) / 2);
      nR = std::min(nR, g.n[1]);
    }
  sh.bx = std::min(128, (np + 31) / 32 * 32);
  sh.TY = std::max(1, std::min(4, nR));
  for (size_t m = 0; m < P.mem.size(); ++m)
    if (p_smooths(P, (int)m, l)) {
      const Geo& g = P.mem[m]->lev[l].g;
      tiles += (long long)((g.n[1] + sh.TY - 1) / sh.TY) * g.n[2];
    }
  long long KC = tiles / (3LL * device_sms());
  sh.KC = (int)std::max(4LL, std::min(16LL, KC));
  // the pair sweep where every member smoothing here can take it and the
  // level holds at least 2^19 cells in all, in the shape the tuner picks on
  // such levels of uneven ducts: six tile rows (fewer where the rows are
  // wide), 16-plane chunks, one block per item
  int bxu = 0, perz = -1;
  long long cells = 0;
  bool pair_ok = true;
  for (size_t m = 0; pair_ok && m < P.mem.size(); ++m) {
    if (!p_smooths(P, (int)m, l)) continue;
    const Geo& g = P.mem[m]->lev[l].g;
    pair_ok = !g.per[0] && !g.per[1] && !(g.n[0] & 1) && g.n[0] >= 4 && g.n[0] <= 256 &&
              (perz < 0 || perz == g.per[2]);
    perz = g.per[2];
    bxu = std::max(bxu, (g.n[0] / 2 + 31) / 32 * 32);
    cells += (long long)g.n[0] * g.n[1] * g.n[2];
  }
  const int pTY = std::min({6, bxu > 0 ? 512 / bxu - 2 : 0, nR});
  if (pair_ok && perz >= 0 && cells >= (1LL << 19) && pTY >= 1) {
    sh.kern = 1;
    sh.perz = perz;
    sh.TY = pTY;
    sh.KC = 16;
    sh.NP = 1;
    sh.bx = bxu;
    sh.all = 1;
  }
  return sh;
}

BArgs bargs(const Persist& P, const PList& L, int lev, int cur = 0) {
  return BArgs{L.dev, L.n, P.tab, P.masked ? P.act : nullptr, lev, cur};
}

// Time the candidate shapes of the batched sweep of kind K (component x for
// the viscous shape, the pressure for its own) on level l and keep the
// fastest; the sweeps are out of place, so only the second buffers change.
cudaError_t tune_level(Persist& P, int l, int K) {
  PShape& best = K == 3 ? P.shp[l] : P.shv[l];
  PList& L = K == 3 ? P.swp[l] : P.swv[l];
  cudaEvent_t e0, e1;
  cudaError_t st = cudaEventCreate(&e0);
  if (st != cudaSuccess) return st;
  st = cudaEventCreate(&e1);
  if (st != cudaSuccess) {
    cudaEventDestroy(e0);
    return st;
  }
  float best_ms = 1e30f;
  PShape keep = best;
  // the ring sweep: one thread per point pair of the widest row on up to 8
  // rows, or 32 threads per row (several pairs each) on taller tiles
  const int bx0 = best.bx;
  const int rows[7][2] = {{2, 0}, {4, 0}, {6, 0}, {8, 0}, {8, 32}, {12, 32}, {16, 32}};
  for (int NP : {1, 2})
    for (const auto& rw : rows)
      for (int KC : {4, 8, 16, 32})
        for (int all : {0, 1}) {
          const int TY = rw[0];
          PShape sh = best;
          sh.kern = 0;
          sh.NP = NP;
          sh.TY = TY;
          sh.KC = KC;
          sh.all = all;
          sh.bx = rw[1] ? rw[1] : bx0;
          if (rw[1] && rw[1] >= bx0) continue;
          if (sh.bx * (TY + 2) > 1024) continue;
          st = sweep_list(P, l, K, sh, L);
          if (st != cudaSuccess) break;
          if (sh.smem > 48 * 1024) continue;
          const BArgs A = bargs(P, L, l);
          float t = 1e30f;
          for (int round = 0; round < 3 && st == cudaSuccess; ++round) {
            cudaEventRecord(e0, P.stream);
            for (int r = 0; r < 3; ++r)
              launch_b_sweep(A, K, sh.TY, sh.KC, sh.NP, sh.bx, sh.smem, sh.grid, P.stream);
            cudaEventRecord(e1, P.stream);
            st = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (st == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
            if (round > 0 && ms < t) t = ms;   // the first round warms up
          }
          if (st != cudaSuccess) break;
          if (t < best_ms) {
            best_ms = t;
            keep = sh;
          }
        }
  // the pair sweep (viscous): where every member smoothing on the level can
  // take it, with one block width (the widest row's) for all
  int bxu = 0, n1min = 1 << 30, perz = -1;
  bool pair_ok = st == cudaSuccess;
  for (size_t m = 0; pair_ok && m < P.mem.size(); ++m) {
    if (!p_smooths(P, (int)m, l)) continue;
    const Geo& g = P.mem[m]->lev[l].g;
    pair_ok = !g.per[0] && !g.per[1] && !(g.n[0] & 1) && g.n[0] >= 4 && g.n[0] <= 256 &&
              (perz < 0 || perz == g.per[2]);
    perz = g.per[2];
    bxu = std::max(bxu, (g.n[0] / 2 + 31) / 32 * 32);
    n1min = std::min(n1min, g.n[1]);
  }
  if (pair_ok && perz >= 0)
    for (int TY : {2, 4, 6, 8, 10, 14})
      for (int KC : {4, 8, 16, 32}) {
        if (TY > n1min || bxu * (TY + 2) > 512) continue;
        PShape sh = best;
        sh.kern = 1;
        sh.perz = perz;
        sh.TY = TY;
        sh.KC = KC;
        sh.NP = 1;
        sh.bx = bxu;
        st = sweep_list(P, l, K, sh, L);
        if (st != cudaSuccess) break;
        if (sh.smem > 48 * 1024) continue;
        const BArgs A = bargs(P, L, l);
        float t = 1e30f;
        for (int round = 0; round < 3 && st == cudaSuccess; ++round) {
          cudaEventRecord(e0, P.stream);
          for (int r = 0; r < 3; ++r) {
            if (K == 3) launch_b_ppair(A, sh.perz != 0, sh.TY, sh.KC, sh.bx, sh.smem, P.stream);
            else launch_b_pair(A, K, sh.perz != 0, sh.TY, sh.KC, sh.bx, sh.smem, P.stream);
          }
          cudaEventRecord(e1, P.stream);
          st = cudaEventSynchronize(e1);
          float ms = 0.f;
          if (st == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
          if (round > 0 && ms < t) t = ms;
        }
        if (st != cudaSuccess) break;
        if (t < best_ms) {
          best_ms = t;
          keep = sh;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != cudaSuccess) return st;
  best = keep;
  return sweep_list(P, l, K, best, L);
}

bool persist_compatible(const bfibm_ctx* a, const bfibm_ctx* c, std::string& why) {
  if (c->D != 3 || c->P.precision != 1) why = "every member must be a 3D mixed-precision context";
  else if (c->P.open_flow) why = "the open duct is not batched";
  else if (c->P.vc_visc > 0 || c->P.vc_p > 0) why = "members must solve to a tolerance (vc_visc = vc_p = 0)";
  else if ((uintptr_t)c->stream <= 2) why = "members need a stream of their own";
  else if (a && (a->P.nu1 != c->P.nu1 || a->P.nu2 != c->P.nu2 || a->inner != c->inner ||
                 a->krylov != c->krylov))
    why = "members must share nu1, nu2, the inner cycle count and the viscous solver";
  else return true;
  return false;
}

// Builds the member table and the work lists (tuning the sweeps when asked).
bfibm_status persist_build(Persist& P, bool tune) {
  const int nm = (int)P.mem.size();
  const bfibm_ctx* c0 = P.mem[0];
  P.nu1 = c0->P.nu1;
  P.nu2 = c0->P.nu2;
  P.inner = c0->inner;
  P.krylov = c0->krylov;
  auto fail = [&](cudaError_t e, const char* where) {
    cudaGetLastError();
    P.err = std::string(where) + ": " + cudaGetErrorString(e);
    return BFIBM_ECUDA;
  };
#define PK(call)                                     \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return fail(e_, #call);   \
  } while (0)
  // the tuner writes the members' second FP32 buffers: their queued work
  // must be done first
  for (bfibm_ctx* c : P.mem) PK(cudaStreamSynchronize(c->stream));
  PK(cudaStreamCreateWithFlags(&P.stream, cudaStreamNonBlocking));
  PK(cudaStreamCreateWithFlags(&P.aux, cudaStreamNonBlocking));
  PK(cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming));
  PK(cudaEventCreateWithFlags(&P.done, cudaEventDisableTiming));
  for (int l = 0; l < kMaxLevels; ++l) {
    PK(cudaStreamCreateWithFlags(&P.tstream[l], cudaStreamNonBlocking));
    PK(cudaEventCreateWithFlags(&P.tfork[l], cudaEventDisableTiming));
    PK(cudaEventCreateWithFlags(&P.tjoin[l], cudaEventDisableTiming));
  }
  P.join.resize(nm, nullptr);
  for (int m = 0; m < nm; ++m) PK(cudaEventCreateWithFlags(&P.join[m], cudaEventDisableTiming));
  std::vector<BMember> host(nm);
  P.depth = 0;
  P.ptail.assign(nm, 0);
  for (int m = 0; m < nm; ++m) {
    const bfibm_ctx* c = P.mem[m];
    fill_member(c, host[m]);
    // the batch's own threshold: each member's kernel has one CTA here
    int t = c->L;
    for (int l = 0; P.tail_cells > 0 && l < c->L; ++l)
      if (cells_of(c->lev[l].g) <= P.tail_cells) {
        t = l;
        break;
      }
    host[m].tail = P.ptail[m] = t;
    P.depth = std::max(P.depth, c->L);
  }
  PK(cudaMalloc((void**)&P.tab, nm * sizeof(BMember)));
  P.allocs.push_back(P.tab);
  PK(cudaMemcpy(P.tab, host.data(), nm * sizeof(BMember), cudaMemcpyHostToDevice));
  PK(cudaMalloc((void**)&P.act, nm * sizeof(int)));
  P.allocs.push_back(P.act);
  PK(cudaMemset(P.act, 0, nm * sizeof(int)));
  PK(cudaMalloc((void**)&P.iters, 2 * sizeof(long long)));
  P.allocs.push_back(P.iters);
  PK(cudaMemset(P.iters, 0, 2 * sizeof(long long)));
  PK(b_coarse_set_smem());
  PK(tail_set_smem());
  std::vector<BItem> v;
  bool ok = true;   // every grid within the items' 16-bit block coordinates
  auto lev = [&](int m, int l) -> const Geo& { return P.mem[m]->lev[l].g; };
  // member m smooths on level l above both its coarsest level and the level
  // where the coarse-level cluster kernel takes over (tail)
  auto tail_of = [&](int m) { return P.ptail[m]; };
  for (int l = 0; l < P.depth; ++l) {
    auto smooths = [&](int m) { return l < std::min(tail_of(m), P.mem[m]->L - 1); };
    ok &= make_items(nm, smooths, [&](int m) {
      const Geo& g = lev(m, l);
      return stencil_grid3(g.n[0], g.n[1], g.n[2]);
    }, v);
    PK(upload(P, v, P.en[l]));
    ok &= make_items(nm, smooths, [&](int m) {
      const Geo& g = lev(m, l + 1);
      return stencil_grid3(g.s[0], g.s[1], g.s[2]);
    }, v);
    PK(upload(P, v, P.rs[l]));
    ok &= make_items(nm, smooths, [&](int m) {
      const Geo& g = lev(m, l + 1);
      return stencil_grid3(g.n[0], g.n[1], g.n[2]);
    }, v);
    PK(upload(P, v, P.rn[l]));
    ok &= make_items(nm, smooths, [&](int m) {
      return dim3(flat_convert_blocks(level_elems(lev(m, l))), 1, 1);
    }, v);
    PK(upload(P, v, P.fl[l]));
    auto coarse_here = [&](int m) { return tail_of(m) >= P.mem[m]->L && l == P.mem[m]->L - 1; };
    ok &= make_items(nm, coarse_here, [&](int) { return dim3(1, 1, 1); }, v);
    PK(upload(P, v, P.co[l]));
    std::vector<int> tl;
    for (int m = 0; m < nm; ++m)
      if (tail_of(m) == l) tl.push_back(m);
    P.ntail[l] = (int)tl.size();
    if (!tl.empty()) {
      PK(cudaMalloc((void**)&P.tail[l], tl.size() * sizeof(int)));
      P.allocs.push_back(P.tail[l]);
      PK(cudaMemcpy(P.tail[l], tl.data(), tl.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    for (int vis = 0; vis < 2; ++vis) {
      size_t mx = 0, mt = 0;
      for (int m = 0; m < nm; ++m) {
        const Geo& gc = lev(m, P.mem[m]->L - 1);
        if (coarse_here(m)) mx = std::max(mx, b_coarse_smem(gc, vis != 0));
        if (tail_of(m) == l) mt = std::max(mt, tail_smem(gc, vis != 0));
      }
      P.co_smem[l][vis] = mx;
      P.tail_smem[l][vis] = mt;
    }
    P.shv[l] = default_shape(P, l);
    P.shp[l] = P.shv[l];
    PK(sweep_list(P, l, 0, P.shv[l], P.swv[l]));
    PK(sweep_list(P, l, 3, P.shp[l], P.swp[l]));
  }
  auto all = [](int) { return true; };
  ok &= make_items(nm, all, [&](int m) {
    const Geo& g = lev(m, 0);
    return stencil_grid3(g.n[0], g.n[1], g.n[2]);
  }, v);
  PK(upload(P, v, P.a3));
  ok &= make_items(nm, all, [&](int m) { return dim3(red_grid_of(cells_of(lev(m, 0))), 1, 1); },
                   v);
  PK(upload(P, v, P.ared));
  ok &= make_items(nm, all, [&](int m) { return dim3(fcg_flat_blocks(lev(m, 0)), 1, 1); }, v);
  PK(upload(P, v, P.aflat));
  ok &= make_items(nm, all, [&](int m) {
    return dim3(flat_convert_blocks(level_elems(lev(m, 0))), 1, 1);
  }, v);
  PK(upload(P, v, P.aconv));
  auto one_per = [&](auto nb_of) {
    v.clear();
    for (int m = 0; m < nm; ++m)
      v.push_back(BItem{m, 0, 0, 0, (unsigned short)nb_of(m), 1, 1});
  };
  one_per([&](int m) { return red_blocks_3d(3, lev(m, 0)); });
  PK(upload(P, v, P.fin3));
  one_per([&](int m) { return red_grid_of(cells_of(lev(m, 0))); });
  PK(upload(P, v, P.finred));
  one_per([&](int m) { return fcg_flat_blocks(lev(m, 0)); });
  PK(upload(P, v, P.finflat));
  if (!ok) {
    P.err = "a member's grid has more than 65535 blocks along an axis";
    return BFIBM_EINVAL;
  }
  if (tune) {
    // levels of at least 2^19 cells in all are timed; smaller ones keep the
    // built-in shape (a launch of a few microseconds cannot tell them apart)
    for (int l = 0; l < P.depth; ++l) {
      long long cells = 0;
      for (int m = 0; m < nm; ++m)
        if (p_smooths(P, m, l)) cells += cells_of(lev(m, l));
      if (cells < (1LL << 19)) continue;
      PK(tune_level(P, l, 0));
      PK(tune_level(P, l, 3));
    }
  }
#undef PK
  return BFIBM_OK;
}

// n sweeps of the viscous components (or the pressure) on level l of every
// member that smooths there; the current buffer of each iterate is tracked
// here, as the single-instance path swaps its pointers, and an odd count
// ends with a copy back.
void b_smooth(Persist& P, int l, int n, bool V) {
  int cur = 0;
  for (int it = 0; it < n; ++it) {
    if (V) {
      for (int d = 0; d < 3; ++d) {
        const PShape& sh = P.shv[l];
        if (sh.kern)
          launch_b_pair(bargs(P, P.swv[l], l, cur), d, sh.perz != 0, sh.TY, sh.KC, sh.bx, sh.smem,
                        P.stream);
        else
          launch_b_sweep(bargs(P, P.swv[l], l, cur), d, sh.TY, sh.KC, sh.NP, sh.bx, sh.smem,
                         sh.grid, P.stream);
        cur ^= 1 << d;
      }
    } else {
      const PShape& sh = P.shp[l];
      if (sh.kern)
        launch_b_ppair(bargs(P, P.swp[l], l, cur), sh.perz != 0, sh.TY, sh.KC, sh.bx, sh.smem,
                       P.stream);
      else
        launch_b_sweep(bargs(P, P.swp[l], l, cur), 3, sh.TY, sh.KC, sh.NP, sh.bx, sh.smem,
                       sh.grid, P.stream);
      cur ^= 8;
    }
  }
  for (int K = 0; K < 4; ++K)
    if ((cur >> K) & 1) launch_b_copy_back(bargs(P, P.fl[l], l), K, P.fl[l].grid, P.stream);
}

void b_level(Persist& P, int l, bool V);

// One V-cycle from level l for every member still in it.
void b_vcycle(Persist& P, int l, bool V) {
  cudaStream_t s = P.stream;
  if (P.ntail[l]) {   // forked: joined again at the end of this level
    cudaEventRecord(P.tfork[l], s);
    cudaStreamWaitEvent(P.tstream[l], P.tfork[l], 0);
    launch_tail(V, P.tab, P.tail[l], P.ntail[l], P.masked ? P.act : nullptr,
                P.tail_smem[l][V ? 1 : 0], P.tstream[l], 1);
    cudaEventRecord(P.tjoin[l], P.tstream[l]);
  }
  b_level(P, l, V);
  if (P.ntail[l]) cudaStreamWaitEvent(s, P.tjoin[l], 0);
}

// Level l of the members that smooth on it (their coarse levels recursively),
// and the coarsest solve of the members whose coarsest level it is.
void b_level(Persist& P, int l, bool V) {
  cudaStream_t s = P.stream;
  if (P.co[l].n) launch_b_coarse(bargs(P, P.co[l], l), V, P.co_smem[l][V ? 1 : 0], s);
  if (!P.en[l].n) return;
  b_smooth(P, l, P.nu1, V);
  if (V) {
    launch_b_v_residual32(bargs(P, P.en[l], l), P.en[l].grid, s);
    launch_b_restrict_face32(bargs(P, P.rs[l], l), P.rs[l].grid, s);
  } else {
    launch_b_p_residual32(bargs(P, P.en[l], l), P.en[l].grid, s);
    launch_b_restrict_cell32(bargs(P, P.rn[l], l), P.rn[l].grid, s);
  }
  b_vcycle(P, l + 1, V);
  if (V)
    launch_b_prolong_face32(bargs(P, P.en[l], l), P.en[l].grid, s);
  else
    launch_b_prolong_cell32(bargs(P, P.en[l], l), P.en[l].grid, s);
  b_smooth(P, l, P.nu2, V);
}

// A device-side loop in the batch graph being captured on P.stream: a
// conditional WHILE node whose body `body` queues (on P.stream, pointed at
// the auxiliary stream meanwhile) with every launch masked.
template <typename Body>
bfibm_status p_capture_while(Persist& P, int which, Body body) {
  if (P.unroll > 0) {   // the iterations queued one after another; masked members skip them
    const long long k0 = 0;
    cudaGraph_t g = nullptr;
    cudaStreamCaptureStatus cs;
    if (cudaStreamGetCaptureInfo(P.stream, &cs, nullptr, &g) != cudaSuccess) {
      cudaGetLastError();
      P.err = "cudaStreamGetCaptureInfo";
      return BFIBM_ECUDA;
    }
    const long long before = count_kernel_nodes(g);
    P.masked = true;
    for (int k = 0; k < P.unroll; ++k) body((cudaGraphConditionalHandle)k0);
    P.masked = false;
    P.body_kernels[which] = (count_kernel_nodes(g) - before) / P.unroll;
    return BFIBM_OK;
  }
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  auto fail = [&](cudaError_t e, const char* where) {
    cudaGetLastError();
    P.err = std::string(where) + ": " + cudaGetErrorString(e);
    return BFIBM_ECUDA;
  };
  cudaError_t e = cudaStreamGetCaptureInfo(P.stream, &cs, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return fail(e, "cudaStreamGetCaptureInfo");
  std::vector<cudaGraphNode_t> dv(deps, deps + nd);
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return fail(e, "cudaGraphConditionalHandleCreate");
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, dv.data(), nullptr, dv.size(), &np);
  if (e != cudaSuccess) return fail(e, "cudaGraphAddNode");
  e = cudaStreamUpdateCaptureDependencies(P.stream, &node, nullptr, 1,
                                          cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return fail(e, "cudaStreamUpdateCaptureDependencies");
  cudaGraph_t bg = np.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(P.aux, bg, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail(e, "cudaStreamBeginCaptureToGraph");
  cudaStream_t main = P.stream;
  P.stream = P.aux;
  P.masked = true;
  body(h);
  P.masked = false;
  P.stream = main;
  cudaGraph_t out = nullptr;
  e = cudaStreamEndCapture(P.aux, &out);
  if (e != cudaSuccess) return fail(e, "cudaStreamEndCapture");
  P.body_kernels[which] = count_kernel_nodes(bg);
  return BFIBM_OK;
}

// The viscous solve of every member (Eq. NSdis1-1), as solve_v_fcg or
// solve_v_mixed queue it in tolerance mode.
bfibm_status b_solve_v(Persist& P) {
  const int nm = (int)P.mem.size();
  cudaStream_t s = P.stream;
  launch_b_norm2(bargs(P, P.ared, 0), true, P.ared.grid, s);
  launch_b_finalize(bargs(P, P.finred, 0), 0, SL_VF, false, false, s);
  if (P.krylov) {
    launch_b_v_residual_mixed(bargs(P, P.a3, 0), true, true, P.a3.grid, s);
    launch_b_finalize(bargs(P, P.fin3, 0), 0, SL_VR, false, false, s);
    launch_b_begin(P.tab, nm, P.act, 0, SL_PQ, s);
    bfibm_status st = p_capture_while(P, 0, [&](cudaGraphConditionalHandle h) {
      cudaStream_t b = P.stream;
      for (int q = 0; q < P.inner; ++q) b_vcycle(P, 0, true);
      launch_b_z_to_f64(bargs(P, P.aconv, 0), P.aconv.grid, b);
      launch_b_fcg_apply(bargs(P, P.a3, 0), P.a3.grid, b);
      launch_b_finalize(bargs(P, P.fin3, 0), 0, SL_ZQ, false, false, b);
      launch_b_fcg_dir(bargs(P, P.aflat, 0), SL_ZQ, SL_PQ, P.aflat.grid, b);
      launch_b_finalize(bargs(P, P.finflat, 0), 0, SL_PQ, false, false, b);
      launch_b_finalize(bargs(P, P.finflat, 0), 1, SL_PRR, false, false, b);
      launch_b_fcg_update(bargs(P, P.aflat, 0), SL_PQ, SL_PRR, P.aflat.grid, b);
      launch_b_finalize(bargs(P, P.finflat, 0), 0, SL_VR, false, false, b);
      launch_b_tol_check(h, P.tab, nm, P.act, 0, SL_VF, SL_VR, -1, P.iters, b, P.unroll == 0);
    });
    if (st != BFIBM_OK) return st;
    // the true FP64 residual of every member's final iterate, checked
    launch_b_v_residual_mixed(bargs(P, P.a3, 0), true, false, P.a3.grid, s);
    launch_b_finalize(bargs(P, P.fin3, 0), 0, SL_VR, false, false, s);
    launch_b_res_check(P.tab, nm, SL_VF, SL_VR, kTrueResidualSlack, s);
    return BFIBM_OK;
  }
  launch_b_begin(P.tab, nm, P.act, 0, -1, s);
  launch_b_v_residual_mixed(bargs(P, P.a3, 0), false, false, P.a3.grid, s);
  return p_capture_while(P, 0, [&](cudaGraphConditionalHandle h) {
    cudaStream_t b = P.stream;
    for (int q = 0; q < P.inner; ++q) b_vcycle(P, 0, true);
    launch_b_add_correction(bargs(P, P.a3, 0), true, P.a3.grid, b);
    launch_b_v_residual_mixed(bargs(P, P.a3, 0), true, false, P.a3.grid, b);
    launch_b_finalize(bargs(P, P.fin3, 0), 0, SL_VR, false, false, b);
    launch_b_tol_check(h, P.tab, nm, P.act, 0, SL_VF, SL_VR, -1, P.iters, b, P.unroll == 0);
  });
}

// The pressure solve of every member (Eq. NSdis3), as solve_p_mixed queues it
// in tolerance mode.
bfibm_status b_solve_p(Persist& P) {
  const int nm = (int)P.mem.size();
  cudaStream_t s = P.stream;
  launch_b_norm2(bargs(P, P.ared, 0), false, P.ared.grid, s);
  launch_b_finalize(bargs(P, P.finred, 0), 0, SL_PF, false, false, s);
  launch_b_begin(P.tab, nm, P.act, 1, -1, s);
  launch_b_p_residual_mixed(bargs(P, P.a3, 0), false, P.a3.grid, s);
  return p_capture_while(P, 1, [&](cudaGraphConditionalHandle h) {
    cudaStream_t b = P.stream;
    for (int q = 0; q < P.inner; ++q) b_vcycle(P, 0, false);
    launch_b_add_correction(bargs(P, P.a3, 0), false, P.a3.grid, b);
    launch_b_partial_sum_p(bargs(P, P.ared, 0), P.ared.grid, b);
    launch_b_finalize(bargs(P, P.finred, 0), 0, 0, false, true, b);
    launch_b_sub_scalar_p(bargs(P, P.a3, 0), P.a3.grid, b);
    launch_b_p_residual_mixed(bargs(P, P.a3, 0), true, P.a3.grid, b);
    launch_b_finalize(bargs(P, P.fin3, 0), 0, SL_PR, false, false, b);
    launch_b_finalize(bargs(P, P.fin3, 0), 1, SL_PRMAX, true, false, b);
    launch_b_tol_check(h, P.tab, nm, P.act, 1, SL_PF, SL_PR, SL_PRMAX, P.iters, b,
                       P.unroll == 0);
  });
}

// Queues `stage` for every member on a branch of its own (its stream, forked
// from and joined back into the batch stream).
template <typename Stage>
void fork_members(Persist& P, Stage stage) {
  cudaEventRecord(P.fork, P.stream);
  for (size_t m = 0; m < P.mem.size(); ++m) {
    bfibm_ctx* c = P.mem[m];
    cudaStreamWaitEvent(c->stream, P.fork, 0);
    stage(c);
    cudaEventRecord(P.join[m], c->stream);
  }
  for (size_t m = 0; m < P.mem.size(); ++m) cudaStreamWaitEvent(P.stream, P.join[m], 0);
}

// One batch step in the order of queue_step (Sec. 3.4), captured once.
bfibm_status persist_capture(Persist& P) {
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(P.stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGetLastError();
    P.err = std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e);
    return BFIBM_ECUDA;
  }
  fork_members(P, [](bfibm_ctx* c) { stage_rhs(c); });
  bfibm_status st = b_solve_v(P);
  if (st == BFIBM_OK) {
    fork_members(P, [](bfibm_ctx* c) { stage_divergence(c); });
    st = b_solve_p(P);
  }
  if (st == BFIBM_OK)
    fork_members(P, [](bfibm_ctx* c) {
      stage_project(c);
      stage_interp_advance(c);
      launch_step_increment(c->step_dev, c->stream);
      refresh(c);
    });
  e = cudaStreamEndCapture(P.stream, &graph);
  if (st != BFIBM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e == cudaSuccess) {
    P.graph_kernels = count_kernel_nodes(graph);
    e = cudaGraphInstantiate(&P.gexec, graph, 0);
  }
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cudaGetLastError();
    P.err = std::string("batch graph: ") + cudaGetErrorString(e);
    return BFIBM_ECUDA;
  }
  return BFIBM_OK;
}

}  // namespace

// =========================================================================
// C ABI
// =========================================================================
extern "C" {

bfibm_status bfibm_footprint(const bfibm_params* p, int64_t eta, int64_t nsprings,
                             int64_t* bytes) {
  if (!bytes || validate(p)) return BFIBM_EINVAL;
  size_t b = grid_pool_bytes(*p);
  b += (size_t)eta * (3 * 3 * sizeof(double) + 2 * sizeof(int));
  b += (size_t)nsprings * (2 * sizeof(int) + 3 * sizeof(double) + 3 * sizeof(int));
  *bytes = (int64_t)b;
  return BFIBM_OK;
}

bfibm_status bfibm_create(const bfibm_params* p, void* stream, bfibm_ctx** out) {
  if (!out) return BFIBM_EINVAL;
  *out = nullptr;
  if (validate(p)) return BFIBM_EINVAL;
  cudaGetLastError();  // a stale error of an earlier call is not ours
  bfibm_ctx* c = new (std::nothrow) bfibm_ctx();
  if (!c) return BFIBM_ENOMEM;
  c->version = next_version();
  c->P = *p;
  c->D = p->dim;
  Geo geos[kMaxLevels];
  c->L = build_levels(*p, geos);
  for (int l = 0; l < c->L; ++l) c->lev[l].g = geos[l];
  if (stream) {
    c->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return BFIBM_ECUDA;
    }
    c->own_stream = true;
  }
  c->pool_bytes = grid_pool_bytes(*p);
  if (cudaMalloc((void**)&c->pool, c->pool_bytes) != cudaSuccess) {
    cudaGetLastError();
    bfibm_destroy(c);
    return BFIBM_ENOMEM;
  }
  // carve arrays
  char* cur = c->pool;
  auto take = [&](const Geo& g) {
    double* q = (double*)cur;
    cur += round_up(level_elems(g) * 8, 256);
    return q;
  };
  int D = c->D, E = edge_count(D);
  for (int l = 0; l < c->L; ++l) {
    Level& Lv = c->lev[l];
    LevelPtrs<double>& d = Lv.d;
    std::memset(&d, 0, sizeof(d));
    d.p = take(Lv.g);
    d.p2 = take(Lv.g);
    d.pf = take(Lv.g);
    d.pr = take(Lv.g);
    for (int a = 0; a < D; ++a) {
      d.beta[a] = take(Lv.g);
      d.u[a] = take(Lv.g);
      d.u2[a] = take(Lv.g);
      d.uf[a] = take(Lv.g);
      d.ur[a] = take(Lv.g);
      d.m[a] = take(Lv.g);
    }
    d.muc = take(Lv.g);
    for (int e = 0; e < E; ++e) d.mue[e] = take(Lv.g);
    if (l == 0)
      for (int a = 0; a < D; ++a) {
        c->uvel[a] = take(Lv.g);
        c->rho[a] = take(Lv.g);
        c->frc[a] = take(Lv.g);
        if (p->precision == 1) {
          c->vdiag[a] = take(Lv.g);
          c->cg_p[a] = take(Lv.g);
          c->cg_q[a] = take(Lv.g);
          c->cg_z[a] = take(Lv.g);
        }
      }
  }
  if (p->precision == 1) {
    auto take32 = [&](const Geo& g) {
      float* q = (float*)cur;
      cur += round_up(level_elems(g) * 4, 256);
      return q;
    };
    for (int l = 0; l < c->L; ++l) {
      Level& Lv = c->lev[l];
      LevelPtrs<float>& f = Lv.f;
      std::memset(&f, 0, sizeof(f));
      f.p = take32(Lv.g);
      f.p2 = take32(Lv.g);
      f.pf = take32(Lv.g);
      f.pr = take32(Lv.g);
      for (int a = 0; a < D; ++a) {
        f.beta[a] = take32(Lv.g);
        f.u[a] = take32(Lv.g);
        f.u2[a] = take32(Lv.g);
        f.uf[a] = take32(Lv.g);
        f.ur[a] = take32(Lv.g);
        f.m[a] = take32(Lv.g);
        f.idg[a] = take32(Lv.g);
      }
      f.muc = take32(Lv.g);
      for (int e = 0; e < E; ++e) f.mue[e] = take32(Lv.g);
    }
  }
  c->G_dev = (double*)cur;
  cur += 256;
  c->sc.out = (double*)cur;
  cur += 256;
  // remaining scalar room
  c->partial_cap = std::max<long long>(4 * kRedBlocks, 2LL * red_blocks_3d(D, c->lev[0].g) + 64);
  if (cudaMalloc((void**)&c->sc.partial, sizeof(double) * c->partial_cap) != cudaSuccess ||
      cudaMalloc((void**)&c->step_dev, sizeof(long long)) != cudaSuccess ||
      cudaMalloc((void**)&c->counters, sizeof(int) * kCounters) != cudaSuccess ||
      cudaMalloc((void**)&c->dev_cycles, sizeof(int) * 2) != cudaSuccess ||
      cudaMalloc((void**)&c->loop_total, sizeof(long long) * 2) != cudaSuccess ||
      cudaMalloc((void**)&c->spread_scale, sizeof(double) * 2) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMallocHost((void**)&c->host_sc, 16 * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    bfibm_destroy(c);
    return BFIBM_ENOMEM;
  }
  c->N.clamped = c->counters;
  c->N.nonfinite = c->counters + 2;
  c->S.ev_count = c->counters + 1;
  c->S.step = c->step_dev;
  cudaStream_t s = c->stream;
  bool ok = cudaMemsetAsync(c->pool, 0, c->pool_bytes, s) == cudaSuccess &&
            cudaMemsetAsync(c->step_dev, 0, sizeof(long long), s) == cudaSuccess &&
            cudaMemsetAsync(c->counters, 0, sizeof(int) * kCounters, s) == cudaSuccess &&
            cudaMemsetAsync(c->dev_cycles, 0, sizeof(int) * 2, s) == cudaSuccess &&
            cudaMemsetAsync(c->loop_total, 0, sizeof(long long) * 2, s) == cudaSuccess;
  {
    static const double one[2] = {1.0, 1.0};
    ok = ok && cudaMemcpyAsync(c->spread_scale, one, sizeof(one), cudaMemcpyHostToDevice, s) ==
                   cudaSuccess;
  }
  if (!ok) {
    bfibm_destroy(c);
    return BFIBM_ECUDA;
  }
  // tiles for binning: 8^3 cells in 3D, 16^2 in 2D
  for (int a = 0; a < 3; ++a) {
    c->tg.T[a] = (a < D) ? (D == 3 ? 8 : 16) : 1;
    c->tg.nt[a] = (a < D) ? (p->n[a] + c->tg.T[a] - 1) / c->tg.T[a] : 1;
  }
  double wmax = std::max(p->omega, p->omega_mu);
  c->tg.H = (int)std::ceil(2.0 * wmax / p->h) + 1;
  c->tg.ntiles = c->tg.nt[0] * c->tg.nt[1] * c->tg.nt[2];
  {
    size_t smem = spread_smem_bytes(D, c->tg);
    if (smem > 48 * 1024 && smem <= spread_smem_limit() && spread_set_smem(D, smem) != cudaSuccess) {
      cudaGetLastError();
      bfibm_destroy(c);
      return BFIBM_ECUDA;
    }
  }
  if (coarse_set_smem() != cudaSuccess || fused_set_carveout() != cudaSuccess ||
      tail_set_smem() != cudaSuccess) {
    cudaGetLastError();
    bfibm_destroy(c);
    return BFIBM_ECUDA;
  }
  if (p->precision == 1 && D == 3) {
    static const int zero = 0;
    if (cudaMalloc((void**)&c->self_tab, sizeof(BMember)) != cudaSuccess ||
        cudaMalloc((void**)&c->self_list, sizeof(int)) != cudaSuccess ||
        cudaMemcpy(c->self_list, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      bfibm_destroy(c);
      return BFIBM_ENOMEM;
    }
  }
  if (upload_self(c) != cudaSuccess) {
    cudaGetLastError();
    bfibm_destroy(c);
    return BFIBM_ECUDA;
  }
  // uniform fluid, laminar initial velocity
  Level& L0 = c->lev[0];
  double mu_eff = p->inv_re * p->mu_f;
  launch_laminar(D, L0.g, p->flow_axis, mu_eff, p->u_center, p->body_force, p->ic_scale,
                 c->uvel[p->flow_axis], c->G_dev, s);
  if (p->open_flow) {
    // Sec. 3.6: no body force; the pressure falls linearly along the duct,
    // Eq. (pressLam), p(0) = 0 and euler kappa = -G (G the body force that
    // drives the same laminar flow), so p_out = kappa L
    double G = 0.0;
    if (cudaMemcpyAsync(&G, c->G_dev, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess ||
        cudaMemsetAsync(c->G_dev, 0, sizeof(double), s) != cudaSuccess) {
      bfibm_destroy(c);
      return BFIBM_ECUDA;
    }
    c->p_out = -G / p->euler * (p->n[p->flow_axis] * p->h);
  }
  launch_reset_fields(D, L0.g, c->frc, c->rho, L0.d.muc, L0.d.mue, p->rho_f, p->mu_f, s);
  build_coefficients(c);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    bfibm_destroy(c);
    return BFIBM_ECUDA;
  }
  // tile shapes of the TMA-staged FP32 sweeps, timed once per level shape
  // (out of place into the spare buffers, before any stream capture)
  if (c->P.precision == 1 && D == 3) {
    bool ok = tma_set_smem() == cudaSuccess;
    for (int l = 0; ok && l < c->L; ++l) {
      Level& Lv = c->lev[l];
      if (!tma_eligible(D, Lv.g)) continue;
      double hh = Lv.g.h * Lv.g.h;
      ok = tma_autotune(D, Lv.g, Lv.f, 3, Lv.f.p2, c->counters + 3, hh, s) == cudaSuccess;
      for (int d = 0; ok && d < D; ++d)
        ok = tma_autotune(D, Lv.g, Lv.f, d, Lv.f.u2[d], c->counters + 3, p->inv_re / hh, s) ==
             cudaSuccess;
    }
    if (!ok || cudaStreamSynchronize(s) != cudaSuccess) {
      cudaGetLastError();
      bfibm_destroy(c);
      return BFIBM_ECUDA;
    }
  }
  c->dirty = true;
  *out = c;
  return BFIBM_OK;
}

void bfibm_destroy(bfibm_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  drop_graph(c);
  free_lag(c, true, true);
  if (c->pool) cudaFree(c->pool);
  if (c->sc.partial) cudaFree(c->sc.partial);
  if (c->step_dev) cudaFree(c->step_dev);
  if (c->counters) cudaFree(c->counters);
  if (c->spread_scale) cudaFree(c->spread_scale);
  if (c->dev_cycles) cudaFree(c->dev_cycles);
  if (c->loop_total) cudaFree(c->loop_total);
  if (c->aux) cudaStreamDestroy(c->aux);
  if (c->host_sc) cudaFreeHost(c->host_sc);
  if (c->self_tab) cudaFree(c->self_tab);
  if (c->self_list) cudaFree(c->self_list);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* bfibm_last_error(const bfibm_ctx* c) { return c ? c->err.c_str() : "no context"; }

bfibm_status bfibm_set_nodes(bfibm_ctx* c, int64_t eta, const double* X) {
  READY(c);
  if (eta < 0 || (eta > 0 && !X) || eta > (int64_t)0x7fffffff)
    return set_err(c, BFIBM_EINVAL, "bad node count or pointer");
  int D = c->D;
  for (int64_t s = 0; s < eta; ++s)
    for (int a = 0; a < D; ++a) {
      double x = X[s * D + a], L = c->P.n[a] * c->P.h;
      bool ok = std::isfinite(x) && x >= 0.0 && (c->P.periodic[a] ? x < L : x <= L);
      if (!ok) return set_err(c, BFIBM_EINVAL, "node position outside the domain");
    }
  CK(cudaStreamSynchronize(c->stream));
  drop_graph(c);
  free_lag(c, true, false);
  if (c->S.m > 0 && c->S.adj_eta != eta) {   // the springs refer to the old node count
    free_lag(c, false, true);
    c->S.m = 0;
  }
  NodeSet& N = c->N;
  N.eta = eta;
  int nt = c->tg.ntiles;
  long long e3 = 3 * std::max<long long>(eta, 1);
  if (dmalloc(&N.X, e3) || dmalloc(&N.U, e3) || dmalloc(&N.F, e3) ||
      dmalloc(&N.tile, eta) || dmalloc(&N.perm, eta) || dmalloc(&N.count, nt + 1) ||
      dmalloc(&N.start, nt + 1) || dmalloc(&N.cursor, nt + 1) || dmalloc(&N.tw, 48 * (e3 / 3)) ||
      dmalloc(&N.tlo, 24 * (e3 / 3))) {
    cudaGetLastError();
    free_lag(c, true, false);
    c->N.eta = 0;
    return set_err(c, BFIBM_ENOMEM, "node buffers");
  }
  CK(cudaMemsetAsync(N.X, 0, sizeof(double) * 3 * std::max<int64_t>(eta, 1), c->stream));
  CK(cudaMemsetAsync(N.U, 0, sizeof(double) * 3 * std::max<int64_t>(eta, 1), c->stream));
  CK(cudaMemsetAsync(N.F, 0, sizeof(double) * 3 * std::max<int64_t>(eta, 1), c->stream));
  if (eta > 0)
    CK(cudaMemcpy2DAsync(N.X, 3 * sizeof(double), X, D * sizeof(double), D * sizeof(double),
                         (size_t)eta, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->dirty = true;
  return BFIBM_OK;
}

bfibm_status bfibm_set_springs(bfibm_ctx* c, int64_t m, const int32_t* ab, const double* rest,
                               const double* K, const double* brk) {
  READY(c);
  if (m < 0 || (m > 0 && (!ab || !rest || !K || !brk)) || m > (int64_t)0x7fffffff)
    return set_err(c, BFIBM_EINVAL, "bad spring count or pointer");
  for (int64_t q = 0; q < m; ++q) {
    int a = ab[2 * q], b = ab[2 * q + 1];
    if (a < 0 || b < 0 || a >= c->N.eta || b >= c->N.eta || a == b)
      return set_err(c, BFIBM_EINVAL, "spring endpoint out of range (set nodes first)");
    if (!(rest[q] >= 0.0) || !std::isfinite(K[q]) || !(brk[q] >= 0.0))
      return set_err(c, BFIBM_EINVAL, "bad spring constants");
  }
  CK(cudaStreamSynchronize(c->stream));
  drop_graph(c);
  free_lag(c, false, true);
  SpringSet& S = c->S;
  S.m = m;
  const long long eta = c->N.eta;
  if (dmalloc(&S.ab, 2 * m) || dmalloc(&S.rest, m) || dmalloc(&S.K, m) || dmalloc(&S.brk, m) ||
      dmalloc(&S.broken, m) || dmalloc(&S.ev_id, m) || dmalloc(&S.ev_step, m) ||
      dmalloc(&S.fvec, 3 * m) || dmalloc(&S.adj_start, eta + 1) || dmalloc(&S.adj, 2 * m)) {
    cudaGetLastError();
    free_lag(c, false, true);
    c->S.m = 0;
    return set_err(c, BFIBM_ENOMEM, "spring buffers");
  }
  if (m > 0) {
    CK(cudaMemcpyAsync(S.ab, ab, sizeof(int) * 2 * m, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(S.rest, rest, sizeof(double) * m, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(S.K, K, sizeof(double) * m, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(S.brk, brk, sizeof(double) * m, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(S.broken, 0, sizeof(int) * m, c->stream));
  }
  // springs of each node in ascending order (the order the node force sums
  // them in): a counting sort of the 2 m endpoints
  {
    std::vector<int> start(eta + 1, 0), adj(2 * std::max<int64_t>(m, 1));
    for (int64_t q = 0; q < m; ++q) {
      ++start[ab[2 * q] + 1];
      ++start[ab[2 * q + 1] + 1];
    }
    for (long long s = 0; s < eta; ++s) start[s + 1] += start[s];
    std::vector<int> fill(start.begin(), start.end() - 1);
    for (int64_t q = 0; q < m; ++q) {
      adj[fill[ab[2 * q]]++] = (int)(2 * q);
      adj[fill[ab[2 * q + 1]]++] = (int)(2 * q + 1);
    }
    CK(cudaMemcpyAsync(S.adj_start, start.data(), sizeof(int) * (eta + 1), cudaMemcpyHostToDevice,
                       c->stream));
    if (m > 0)
      CK(cudaMemcpyAsync(S.adj, adj.data(), sizeof(int) * 2 * m, cudaMemcpyHostToDevice,
                         c->stream));
    CK(cudaStreamSynchronize(c->stream));
    S.adj_eta = eta;
  }
  CK(cudaMemsetAsync(S.ev_count, 0, sizeof(int), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->dirty = true;
  return BFIBM_OK;
}

bfibm_status bfibm_set_velocity(bfibm_ctx* c, int comp, const double* u) {
  READY(c);
  return copy_field(c, BFIBM_F_U, comp, 0, (void*)u, false, cudaMemcpyHostToDevice);
}

bfibm_status bfibm_step(bfibm_ctx* c, int nsteps) {
  READY(c);
  if (nsteps < 0) return set_err(c, BFIBM_EINVAL, "nsteps < 0");
  return do_steps(c, nsteps, true);
}

bfibm_status bfibm_get_velocity(bfibm_ctx* c, int comp, double* out) {
  READY(c);
  return copy_field(c, BFIBM_F_U, comp, 0, out, true, cudaMemcpyDeviceToHost);
}

bfibm_status bfibm_get_pressure(bfibm_ctx* c, double* out) {
  READY(c);
  return copy_field(c, BFIBM_F_P, 0, 0, out, true, cudaMemcpyDeviceToHost);
}

bfibm_status bfibm_get_nodes(bfibm_ctx* c, double* X) {
  READY(c);
  if (!X && c->N.eta > 0) return set_err(c, BFIBM_EINVAL, "X is NULL");
  if (c->N.eta > 0)
    CK(cudaMemcpy2DAsync(X, c->D * sizeof(double), c->N.X, 3 * sizeof(double),
                         c->D * sizeof(double), (size_t)c->N.eta, cudaMemcpyDeviceToHost,
                         c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return BFIBM_OK;
}

bfibm_status bfibm_get_node_forces(bfibm_ctx* c, double* F) {
  READY(c);
  if (!F && c->N.eta > 0) return set_err(c, BFIBM_EINVAL, "F is NULL");
  if (c->N.eta > 0)
    CK(cudaMemcpy2DAsync(F, c->D * sizeof(double), c->N.F, 3 * sizeof(double),
                         c->D * sizeof(double), (size_t)c->N.eta, cudaMemcpyDeviceToHost,
                         c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return BFIBM_OK;
}

bfibm_status bfibm_get_broken(bfibm_ctx* c, int64_t cap, int64_t* n, int32_t* spring_id,
                              int32_t* step) {
  READY(c);
  if (!n) return set_err(c, BFIBM_EINVAL, "n is NULL");
  int cnt = 0;
  CK(cudaMemcpyAsync(&cnt, c->S.ev_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  cnt = (int)std::min<long long>(cnt, c->S.m);
  *n = cnt;
  if (cap <= 0 || cnt == 0) return BFIBM_OK;
  if (!spring_id || !step) return set_err(c, BFIBM_EINVAL, "output arrays are NULL");
  std::vector<int32_t> id(cnt), st(cnt);
  CK(cudaMemcpyAsync(id.data(), c->S.ev_id, sizeof(int) * cnt, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(st.data(), c->S.ev_step, sizeof(int) * cnt, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  std::vector<int> order(cnt);
  for (int q = 0; q < cnt; ++q) order[q] = q;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    return st[a] != st[b] ? st[a] < st[b] : id[a] < id[b];
  });
  int64_t w = std::min<int64_t>(cap, cnt);
  for (int64_t q = 0; q < w; ++q) {
    spring_id[q] = id[order[q]];
    step[q] = st[order[q]];
  }
  return BFIBM_OK;
}

bfibm_status bfibm_get_stats(bfibm_ctx* c, bfibm_stats* out) {
  READY(c);
  if (!out) return set_err(c, BFIBM_EINVAL, "out is NULL");
  launch_div_ke(c->D, c->lev[0].g, c->uvel, c->sc, SL_DIV, c->stream);
  CK(cudaGetLastError());
  bfibm_status rs = read_scalars(c);
  if (rs != BFIBM_OK) return rs;
  int cnt[kCounters];
  CK(cudaMemcpyAsync(cnt, c->counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  std::memset(out, 0, sizeof(*out));
  out->cycles_visc = c->cycles_visc;
  out->cycles_p = c->cycles_p;
  if (c->cycles_visc < 0 || c->cycles_p < 0) {   // counted on the device
    int cyc[2];
    CK(cudaMemcpyAsync(cyc, c->dev_cycles, sizeof(cyc), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->cycles_visc < 0) out->cycles_visc = cyc[0] * c->loop_inner[0];
    if (c->cycles_p < 0) out->cycles_p = cyc[1] * c->loop_inner[1];
  }
  out->broken_total = std::min<int>(cnt[1], (int)std::max<long long>(c->S.m, 0));
  out->clamped_total = cnt[0];
  out->nonfinite_total = cnt[2];
  out->wait_timeouts = cnt[3];
  auto rel = [](double f2, double r2) { return f2 > 0.0 ? std::sqrt(r2) / std::sqrt(f2) : 0.0; };
  out->res_visc = rel(c->host_sc[SL_VF], c->host_sc[SL_VR]);
  out->res_p = rel(c->host_sc[SL_PF], c->host_sc[SL_PR]);
  out->div_max = c->host_sc[SL_DIV];
  out->kinetic = c->host_sc[SL_DIV + 1];
  out->nonconv_total = cnt[4];
  out->div_violations = cnt[5];
  out->div_max_step = c->host_sc[SL_DIVSTEP];
  out->div_max_steps = c->host_sc[SL_DIVALL];
  out->step = c->step_host;
  return BFIBM_OK;
}

bfibm_status bfibm_get_field(bfibm_ctx* c, int which, int comp, int level, double* out) {
  READY(c);
  return copy_field(c, which, comp, level, out, true, cudaMemcpyDeviceToHost);
}
bfibm_status bfibm_set_field(bfibm_ctx* c, int which, int comp, int level, const double* in) {
  READY(c);
  return copy_field(c, which, comp, level, (void*)in, false, cudaMemcpyHostToDevice);
}
bfibm_status bfibm_get_field_f32(bfibm_ctx* c, int which, int comp, int level, float* out) {
  READY(c);
  return copy_field32(c, which, comp, level, out, true);
}
bfibm_status bfibm_set_field_f32(bfibm_ctx* c, int which, int comp, int level, const float* in) {
  READY(c);
  return copy_field32(c, which, comp, level, (void*)in, false);
}
bfibm_status bfibm_get_field_dev(bfibm_ctx* c, int which, int comp, int level, double* dev) {
  READY(c);
  return copy_field(c, which, comp, level, dev, true, cudaMemcpyDeviceToDevice);
}
bfibm_status bfibm_set_field_dev(bfibm_ctx* c, int which, int comp, int level, const double* dev) {
  READY(c);
  return copy_field(c, which, comp, level, (void*)dev, false, cudaMemcpyDeviceToDevice);
}

bfibm_status bfibm_refresh(bfibm_ctx* c) {
  READY(c);
  refresh(c);
  c->dirty = false;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  return BFIBM_OK;
}

bfibm_status bfibm_build_coefficients(bfibm_ctx* c) {
  READY(c);
  build_coefficients(c);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  return BFIBM_OK;
}

bfibm_status bfibm_stage(bfibm_ctx* c, int stage) {
  READY(c);
  switch (stage) {
    case BFIBM_STAGE_RHS: stage_rhs(c); break;
    case BFIBM_STAGE_DIVERGENCE: stage_divergence(c); break;
    case BFIBM_STAGE_PROJECT: stage_project(c); break;
    case BFIBM_STAGE_INTERP_ADVANCE: stage_interp_advance(c); break;
    case BFIBM_STAGE_SPRINGS: stage_springs(c); break;
    default: return set_err(c, BFIBM_EINVAL, "unknown stage");
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  return BFIBM_OK;
}

bfibm_status bfibm_solve_pressure(bfibm_ctx* c, int ncycles, int32_t* cycles) {
  READY(c);
  int used = 0;
  bfibm_status st = c->P.precision == 1 ? solve_p_mixed(c, ncycles, &used)
                                        : solve_p(c, ncycles, &used);
  if (st != BFIBM_OK && st != BFIBM_ENOCONV) return st;
  c->cycles_p = used;
  if (cycles) *cycles = used;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  return st;
}

bfibm_status bfibm_set_gamma(bfibm_ctx* c, const double gamma_levels[8]) {
  READY(c);
  if (!gamma_levels) return set_err(c, BFIBM_EINVAL, "gamma_levels is NULL");
  for (int l = 0; l < 8; ++l)
    if (!(gamma_levels[l] >= 0.0) || !std::isfinite(gamma_levels[l]))
      return set_err(c, BFIBM_EINVAL, "gamma_levels entries must be >= 0");
  CK(cudaStreamSynchronize(c->stream));
  drop_graph(c);
  for (int l = 0; l < 8; ++l) c->P.gamma_levels[l] = gamma_levels[l];
  build_coefficients(c);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  return BFIBM_OK;
}

bfibm_status bfibm_solve_viscous(bfibm_ctx* c, int ncycles, int32_t* cycles) {
  READY(c);
  int used = 0;
  bfibm_status st = c->P.precision == 1 ? (c->krylov ? solve_v_fcg(c, ncycles, &used)
                                                     : solve_v_mixed(c, ncycles, &used))
                                        : solve_v(c, ncycles, &used);
  if (st != BFIBM_OK && st != BFIBM_ENOCONV) return st;
  c->cycles_visc = used;
  if (cycles) *cycles = used;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  return st;
}

bfibm_status bfibm_smooth_pressure(bfibm_ctx* c, int level, int nsweeps) {
  READY(c);
  if (level < 0 || level >= c->L || nsweeps < 0) return set_err(c, BFIBM_EINVAL, "bad level");
  smooth_p(c, level, nsweeps);
  CK(cudaGetLastError());
  return BFIBM_OK;
}

bfibm_status bfibm_smooth_viscous(bfibm_ctx* c, int level, int nsweeps) {
  READY(c);
  if (level < 0 || level >= c->L || nsweeps < 0) return set_err(c, BFIBM_EINVAL, "bad level");
  smooth_v(c, level, nsweeps);
  CK(cudaGetLastError());
  return BFIBM_OK;
}

bfibm_status bfibm_smooth_f32(bfibm_ctx* c, int which, int level, int nsweeps) {
  READY(c);
  if (c->P.precision != 1) return set_err(c, BFIBM_ESTATE, "not a mixed-precision context");
  if (level < 0 || level >= c->L || nsweeps < 0 || (which != 0 && which != 1))
    return set_err(c, BFIBM_EINVAL, "bad level, count or selector");
  if (which == 0) smooth_p32(c, level, nsweeps);
  else smooth_v32(c, level, nsweeps);
  CK(cudaGetLastError());
  return BFIBM_OK;
}

bfibm_status bfibm_synchronize(bfibm_ctx* c) {
  READY(c);
  CK(cudaStreamSynchronize(c->stream));
  return BFIBM_OK;
}

bfibm_status bfibm_residual_pressure(bfibm_ctx* c, int level) {
  READY(c);
  if (level < 0 || level >= c->L) return set_err(c, BFIBM_EINVAL, "bad level");
  launch_p_residual<double>(c->D, c->lev[level].g, c->lev[level].d, c->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  return BFIBM_OK;
}

bfibm_status bfibm_residual_viscous(bfibm_ctx* c, int level) {
  READY(c);
  if (level < 0 || level >= c->L) return set_err(c, BFIBM_EINVAL, "bad level");
  launch_v_residual<double>(c->D, c->lev[level].g, c->lev[level].d, c->P.inv_re, c->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->stream));
  return BFIBM_OK;
}

bfibm_status bfibm_levels(bfibm_ctx* c, int32_t* nlevels) {
  if (!c || !nlevels) return BFIBM_EINVAL;
  *nlevels = c->L;
  return BFIBM_OK;
}

bfibm_status bfibm_level_dims(bfibm_ctx* c, int level, int32_t n[3], int32_t s[3]) {
  if (!c || !n || !s || level < 0 || level >= c->L) return BFIBM_EINVAL;
  for (int a = 0; a < 3; ++a) {
    n[a] = c->lev[level].g.n[a];
    s[a] = c->lev[level].g.s[a];
  }
  return BFIBM_OK;
}

bfibm_status bfibm_body_force(bfibm_ctx* c, double* G) {
  READY(c);
  if (!G) return BFIBM_EINVAL;
  CK(cudaMemcpyAsync(G, c->G_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return BFIBM_OK;
}

bfibm_status bfibm_launch_counts(bfibm_ctx* c, int64_t out[5]) {
  READY(c);
  if (!out) return set_err(c, BFIBM_EINVAL, "out is NULL");
  long long tot[2] = {0, 0};
  CK(cudaMemcpyAsync(tot, c->loop_total, sizeof(tot), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  out[0] = c->gexec ? c->graph_kernels : -1;
  out[1] = c->body_kernels[0];
  out[2] = c->body_kernels[1];
  out[3] = tot[0];
  out[4] = tot[1];
  return BFIBM_OK;
}

bfibm_status bfibm_launches_per_step(bfibm_ctx* c, int64_t* n) {
  READY(c);
  if (!n) return BFIBM_EINVAL;
  *n = c->gexec ? c->graph_kernels : -1;
  return BFIBM_OK;
}

// ------------------------------------------------------------------ checkpoints
namespace {
struct CkptHeader {
  uint64_t magic;
  int32_t version, dim, n[3], precision;
  int64_t eta, m, step, events, elems;
};
constexpr uint64_t kCkptMagic = 0x31544b504d424942ull;   // "BIBMPKT1"

int64_t ckpt_bytes(const bfibm_ctx* c) {
  const int64_t elems = level_elems(c->lev[0].g);
  return (int64_t)sizeof(CkptHeader) + (int64_t)(c->D + 1) * elems * 8 + c->N.eta * 3 * 8 +
         c->S.m * 3 * 4;
}
}  // namespace

bfibm_status bfibm_state_bytes(bfibm_ctx* c, int64_t* bytes) {
  READY(c);
  if (!bytes) return set_err(c, BFIBM_EINVAL, "bytes is NULL");
  *bytes = ckpt_bytes(c);
  return BFIBM_OK;
}

bfibm_status bfibm_save_state(bfibm_ctx* c, void* buf, int64_t bytes) {
  READY(c);
  if (!buf || bytes < ckpt_bytes(c)) return set_err(c, BFIBM_EINVAL, "buffer too small");
  CkptHeader h;
  std::memset(&h, 0, sizeof(h));
  h.magic = kCkptMagic;
  h.version = 1;
  h.dim = c->D;
  for (int a = 0; a < 3; ++a) h.n[a] = c->P.n[a];
  h.precision = c->P.precision;
  h.eta = c->N.eta;
  h.m = c->S.m;
  h.step = c->step_host;
  h.elems = level_elems(c->lev[0].g);
  int cnt[kCounters];
  CK(cudaMemcpyAsync(cnt, c->counters, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  h.events = std::min<int64_t>(cnt[1], c->S.m);
  unsigned char* q = (unsigned char*)buf;
  std::memcpy(q, &h, sizeof(h));
  q += sizeof(h);
  const size_t fb = (size_t)h.elems * 8;
  for (int d = 0; d < c->D; ++d, q += fb)
    CK(cudaMemcpyAsync(q, c->uvel[d], fb, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(q, c->lev[0].d.p, fb, cudaMemcpyDeviceToHost, c->stream));
  q += fb;
  if (h.eta > 0) CK(cudaMemcpyAsync(q, c->N.X, h.eta * 24, cudaMemcpyDeviceToHost, c->stream));
  q += h.eta * 24;
  if (h.m > 0) {
    CK(cudaMemcpyAsync(q, c->S.broken, h.m * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(q + h.m * 4, c->S.ev_id, h.m * 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(q + h.m * 8, c->S.ev_step, h.m * 4, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return BFIBM_OK;
}

bfibm_status bfibm_load_state(bfibm_ctx* c, const void* buf, int64_t bytes) {
  READY(c);
  if (!buf || bytes < (int64_t)sizeof(CkptHeader)) return set_err(c, BFIBM_EINVAL, "buffer too small");
  CkptHeader h;
  std::memcpy(&h, buf, sizeof(h));
  bool same = h.magic == kCkptMagic && h.version == 1 && h.dim == c->D &&
              h.precision == c->P.precision && h.eta == c->N.eta && h.m == c->S.m &&
              h.elems == level_elems(c->lev[0].g) && h.step >= 0 && h.events >= 0 &&
              h.events <= h.m;
  for (int a = 0; a < 3; ++a) same = same && h.n[a] == c->P.n[a];
  if (!same) return set_err(c, BFIBM_EINVAL, "checkpoint does not match this context");
  if (bytes < ckpt_bytes(c)) return set_err(c, BFIBM_EINVAL, "checkpoint truncated");
  CK(cudaStreamSynchronize(c->stream));
  const unsigned char* q = (const unsigned char*)buf + sizeof(h);
  const size_t fb = (size_t)h.elems * 8;
  for (int d = 0; d < c->D; ++d, q += fb)
    CK(cudaMemcpyAsync(c->uvel[d], q, fb, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->lev[0].d.p, q, fb, cudaMemcpyHostToDevice, c->stream));
  q += fb;
  if (h.eta > 0) CK(cudaMemcpyAsync(c->N.X, q, h.eta * 24, cudaMemcpyHostToDevice, c->stream));
  q += h.eta * 24;
  if (h.m > 0) {
    CK(cudaMemcpyAsync(c->S.broken, q, h.m * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->S.ev_id, q + h.m * 4, h.m * 4, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->S.ev_step, q + h.m * 8, h.m * 4, cudaMemcpyHostToDevice, c->stream));
  }
  long long step = h.step;
  int events = (int)h.events;
  CK(cudaMemcpyAsync(c->step_dev, &step, sizeof(step), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->counters + 1, &events, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->step_host = h.step;
  c->dirty = true;   // forces, spreads and coefficients follow from X on the next step
  return BFIBM_OK;
}

bfibm_status bfibm_tma_plan(bfibm_ctx* c, int level, int kind, int32_t out[5]) {
  READY(c);
  if (!out || level < 0 || level >= c->L || kind < 0 || kind > 3 ||
      (kind < 3 && kind >= c->D) || c->P.precision != 1 || !use_tma(c, level))
    return set_err(c, BFIBM_EINVAL, "no TMA sweep on this level");
  int v[5];
  if (!tma_plan_of(kind, c->lev[level].g, v)) return set_err(c, BFIBM_EINVAL, "level not tuned");
  for (int q = 0; q < 5; ++q) out[q] = v[q];
  return BFIBM_OK;
}

bfibm_status bfibm_sweep_shape(bfibm_ctx* c, int level, int kind, int32_t out[5]) {
  READY(c);
  if (!out || level < 0 || level >= c->L || kind < 0 || kind > 3 ||
      (kind < 3 && kind >= c->D) || c->P.precision != 1)
    return set_err(c, BFIBM_EINVAL, "no FP32 sweep of this kind on this level");
  int ty = 0, kc = 0, np = 1, bx = 0, kern = 0;
  if (!ring_shape_of(kind, c->lev[level].g, &ty, &kc, &np, &bx, &kern))
    return set_err(c, BFIBM_EINVAL, "level not tuned");
  out[0] = ty;
  out[1] = kc;
  out[2] = np;
  out[3] = bx;
  out[4] = kern;
  return BFIBM_OK;
}

bfibm_status bfibm_sweep_set_shape(bfibm_ctx* c, int level, int kind, const int32_t shape[5]) {
  READY(c);
  if (!shape || level < 0 || level >= c->L || kind < 0 || kind > 3 ||
      (kind < 3 && kind >= c->D) || c->P.precision != 1 || c->D != 3)
    return set_err(c, BFIBM_EINVAL, "no FP32 sweep of this kind on this level");
  int v[5] = {shape[0], shape[1], shape[2], shape[3], shape[4]};
  if (!ring_set_shape(kind, c->lev[level].g, v)) return set_err(c, BFIBM_EINVAL, "bad shape");
  CK(cudaStreamSynchronize(c->stream));
  drop_graph(c);
  return BFIBM_OK;
}

bfibm_status bfibm_tma_set_plan(bfibm_ctx* c, int level, int kind, const int32_t plan[5]) {
  READY(c);
  if (!plan || level < 0 || level >= c->L || kind < 0 || kind > 3 ||
      (kind < 3 && kind >= c->D) || !tma_eligible(c->D, c->lev[level].g))
    return set_err(c, BFIBM_EINVAL, "no TMA sweep on this level");
  int v[5] = {plan[0], plan[1], plan[2], plan[3], plan[4]};
  if (!tma_set_plan(kind, c->lev[level].g, v)) return set_err(c, BFIBM_EINVAL, "plan does not fit");
  return BFIBM_OK;
}

bfibm_status bfibm_set_option(bfibm_ctx* c, int option, int64_t value) {
  READY(c);
  if (option == BFIBM_OPT_STATS) {
    c->collect_stats = value != 0;
  } else if (option == BFIBM_OPT_GRAPH) {
    c->use_graph = value != 0;
  } else if (option == BFIBM_OPT_FUSED) {
    if (value != 0 && c->P.open_flow)
      return set_err(c, BFIBM_EINVAL, "the open duct uses one kernel per colour");
    c->fused = value != 0;
  } else if (option == BFIBM_OPT_TMA) {
    if (value < 0 || value > 2) return set_err(c, BFIBM_EINVAL, "BFIBM_OPT_TMA takes 0, 1 or 2");
    c->tma = (int)value;
  } else if (option == BFIBM_OPT_KRYLOV) {
    if (value < 0 || value > 1) return set_err(c, BFIBM_EINVAL, "BFIBM_OPT_KRYLOV takes 0 or 1");
    c->krylov = (int)value;
  } else if (option == BFIBM_OPT_WAIT_NS) {
    if (value < 0) return set_err(c, BFIBM_EINVAL, "BFIBM_OPT_WAIT_NS takes a value >= 0");
    c->tma_wait_ns = (unsigned long long)value;
  } else if (option == BFIBM_OPT_INNER) {
    if (value < 1 || value > 16)
      return set_err(c, BFIBM_EINVAL, "BFIBM_OPT_INNER takes 1 to 16");
    c->inner = (int)value;
  } else if (option == BFIBM_OPT_TAIL) {
    if (value < 0) return set_err(c, BFIBM_EINVAL, "BFIBM_OPT_TAIL takes a value >= 0");
    c->tail_cells = value;
  } else {
    return set_err(c, BFIBM_EINVAL, "unknown option");
  }
  CK(cudaStreamSynchronize(c->stream));
  CK(upload_self(c));
  drop_graph(c);
  return BFIBM_OK;
}

// ------------------------------------------------------------------ batches
struct bfibm_batch {
  struct Slot {
    bfibm_ctx* c = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    bool timed = false;
  };
  std::vector<Slot> slots;
  int persistent = 0;    // BFIBM_BATCH_PERSISTENT
  int tune = 1;          // BFIBM_BATCH_TUNE
  int unroll = 0;        // BFIBM_BATCH_UNROLL
  long long tail = 4096; // BFIBM_BATCH_TAIL
  Persist* ps = nullptr; // the plan of the last persistent step
  long long builds = 0;  // plans built
  std::string err;
};

bfibm_status bfibm_batch_create(bfibm_batch** out) {
  if (!out) return BFIBM_EINVAL;
  *out = new (std::nothrow) bfibm_batch();
  return *out ? BFIBM_OK : BFIBM_ENOMEM;
}

bfibm_status bfibm_batch_add(bfibm_batch* b, bfibm_ctx* c, int32_t* slot) {
  if (!b || !c || !slot) return BFIBM_EINVAL;
  READY(c);
  int k = -1;
  for (size_t q = 0; q < b->slots.size(); ++q)
    if (!b->slots[q].c) {
      k = (int)q;
      break;
    }
  if (k < 0) {
    k = (int)b->slots.size();
    b->slots.emplace_back();
  }
  bfibm_batch::Slot& s = b->slots[k];
  if (!s.e0 && (cudaEventCreate(&s.e0) != cudaSuccess || cudaEventCreate(&s.e1) != cudaSuccess)) {
    cudaGetLastError();
    return BFIBM_ECUDA;
  }
  s.c = c;
  s.timed = false;
  *slot = k;
  return BFIBM_OK;
}

bfibm_status bfibm_batch_remove(bfibm_batch* b, int32_t slot) {
  if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].c) return BFIBM_EINVAL;
  if (b->ps) {   // the plan holds the member's arrays, which may be freed next
    persist_free(b->ps);
    b->ps = nullptr;
  }
  b->slots[slot].c = nullptr;
  b->slots[slot].timed = false;
  return BFIBM_OK;
}

namespace {
// The members stepped by nsteps in table order (level-0 cells descending),
// with a plan built for exactly them, then n launches of its graph.
bfibm_status persist_step(bfibm_batch* b, const int32_t* nsteps) {
  std::vector<int> idx;
  int n = -1;
  for (size_t q = 0; q < b->slots.size(); ++q) {
    bfibm_batch::Slot& s = b->slots[q];
    if (!s.c) continue;
    const int k = nsteps ? nsteps[q] : 1;
    s.timed = false;
    if (k <= 0) continue;
    if (n >= 0 && k != n) {
      b->err = "a persistent batch steps every member it steps the same number of steps";
      return BFIBM_EINVAL;
    }
    n = k;
    idx.push_back((int)q);
  }
  if (idx.empty()) return BFIBM_OK;
  std::vector<bfibm_ctx*> mem;
  for (int q : idx) {
    bfibm_ctx* c = b->slots[q].c;
    READY(c);
    std::string why;
    if (!persist_compatible(mem.empty() ? nullptr : mem[0], c, why)) {
      b->err = why;
      return BFIBM_EINVAL;
    }
    mem.push_back(c);
  }
  std::stable_sort(mem.begin(), mem.end(), [](const bfibm_ctx* x, const bfibm_ctx* y) {
    return cells_of(x->lev[0].g) > cells_of(y->lev[0].g);
  });
  std::vector<long long> ver;
  for (bfibm_ctx* c : mem) ver.push_back(c->version);
  if (!b->ps || b->ps->mem != mem || b->ps->version != ver) {
    persist_free(b->ps);
    b->ps = new (std::nothrow) Persist();
    if (!b->ps) return BFIBM_ENOMEM;
    b->ps->mem = mem;
    b->ps->version = ver;
    b->ps->unroll = b->unroll;
    b->ps->tail_cells = b->tail;
    bfibm_status st = persist_build(*b->ps, b->tune != 0);
    if (st == BFIBM_OK) st = persist_capture(*b->ps);
    if (st != BFIBM_OK) {
      b->err = b->ps->err;
      persist_free(b->ps);
      b->ps = nullptr;
      return st;
    }
    ++b->builds;
  }
  Persist& P = *b->ps;
  for (size_t m = 0; m < mem.size(); ++m) {
    bfibm_ctx* c = mem[m];
    bfibm_status st = ensure_ready(c);
    if (st != BFIBM_OK) return st;
    CK(cudaEventRecord(P.join[m], c->stream));
    CK(cudaStreamWaitEvent(P.stream, P.join[m], 0));
  }
  bfibm_ctx* c = mem[0];   // for the error path of CK
  for (int q : idx) CK(cudaEventRecord(b->slots[q].e0, P.stream));
  for (int k = 0; k < n; ++k) CK(cudaGraphLaunch(P.gexec, P.stream));
  for (int q : idx) {
    CK(cudaEventRecord(b->slots[q].e1, P.stream));
    b->slots[q].timed = true;
  }
  CK(cudaEventRecord(P.done, P.stream));
  for (bfibm_ctx* m : mem) {
    CK(cudaStreamWaitEvent(m->stream, P.done, 0));
    m->step_host += n;
    m->cycles_visc = m->cycles_p = -1;   // counted on the device
    m->loop_inner[0] = m->loop_inner[1] = P.inner;
  }
  return BFIBM_OK;
}
}  // namespace

bfibm_status bfibm_batch_set_option(bfibm_batch* b, int option, int64_t value) {
  if (!b) return BFIBM_EINVAL;
  if (option == BFIBM_BATCH_PERSISTENT) b->persistent = value != 0;
  else if (option == BFIBM_BATCH_TUNE) b->tune = value != 0;
  else if (option == BFIBM_BATCH_UNROLL && value >= 0 && value <= 1000) b->unroll = (int)value;
  else if (option == BFIBM_BATCH_TAIL && value >= 0) b->tail = value;
  else return BFIBM_EINVAL;
  persist_free(b->ps);
  b->ps = nullptr;
  return BFIBM_OK;
}

bfibm_status bfibm_batch_info(bfibm_batch* b, int64_t out[8]) {
  if (!b || !out) return BFIBM_EINVAL;
  std::memset(out, 0, 8 * sizeof(int64_t));
  out[0] = b->persistent;
  out[1] = b->builds;
  if (!b->ps) return BFIBM_OK;
  Persist& P = *b->ps;
  long long it[2] = {0, 0};
  if (cudaMemcpyAsync(it, P.iters, sizeof(it), cudaMemcpyDeviceToHost, P.stream) != cudaSuccess ||
      cudaStreamSynchronize(P.stream) != cudaSuccess) {
    cudaGetLastError();
    return BFIBM_ECUDA;
  }
  out[2] = (int64_t)P.mem.size();
  out[3] = P.graph_kernels;
  out[4] = P.body_kernels[0];
  out[5] = P.body_kernels[1];
  out[6] = it[0];
  out[7] = it[1];
  return BFIBM_OK;
}

bfibm_status bfibm_batch_sweep_shape(bfibm_batch* b, int level, int kind, int32_t out[7]) {
  if (!b || !out || !b->ps || level < 0 || level >= b->ps->depth || kind < 0 || kind > 1)
    return BFIBM_EINVAL;
  const PShape& sh = kind == 0 ? b->ps->shv[level] : b->ps->shp[level];
  out[0] = sh.TY;
  out[1] = sh.KC;
  out[2] = sh.NP;
  out[3] = sh.bx;
  out[4] = sh.all;
  out[5] = sh.grid;
  out[6] = sh.kern;
  return BFIBM_OK;
}

bfibm_status bfibm_batch_set_sweep_shape(bfibm_batch* b, int level, int kind,
                                         const int32_t shape[6]) {
  if (!b || !shape || !b->ps || level < 0 || level >= b->ps->depth || kind < 0 || kind > 1)
    return BFIBM_EINVAL;
  Persist& P = *b->ps;
  PShape sh = kind == 0 ? P.shv[level] : P.shp[level];
  sh.TY = shape[0];
  sh.KC = shape[1];
  sh.NP = shape[2];
  sh.bx = shape[3];
  sh.all = shape[4] != 0;
  sh.kern = shape[5];
  if (sh.TY < 1 || sh.KC < 1 || (sh.NP != 1 && sh.NP != 2) || sh.bx < 32 || sh.bx % 32 ||
      sh.bx * (sh.TY + 2) > 1024 || sh.kern < 0 || sh.kern > 1) {
    b->err = "a sweep shape needs rows >= 1, planes >= 1, 1 or 2 planes per phase, "
             "32 k threads per row, at most 1024 threads and kernel 0 or 1";
    return BFIBM_EINVAL;
  }
  if (sh.kern) {   // the pair sweep: every member eligible, one row width
    bool ok = sh.NP == 1 && sh.bx * (sh.TY + 2) <= 512;
    int perz = -1;
    for (size_t m = 0; ok && m < P.mem.size(); ++m) {
      if (!p_smooths(P, (int)m, level)) continue;
      const Geo& g = P.mem[m]->lev[level].g;
      ok = !g.per[0] && !g.per[1] && !(g.n[0] & 1) && g.n[0] >= 4 && g.n[0] <= 256 &&
           sh.TY <= g.n[1] && (g.n[0] / 2 + 31) / 32 * 32 <= sh.bx && (perz < 0 || perz == g.per[2]);
      perz = g.per[2];
    }
    if (!ok) {
      b->err = "the pair sweep needs walls across x and y, even rows of 4 to 256 points no wider "
               "than the block, rows >= tile rows, one periodicity along z and at most 512 "
               "threads";
      return BFIBM_EINVAL;
    }
    sh.perz = perz > 0;
  }
  if (cudaStreamSynchronize(P.stream) != cudaSuccess) {
    cudaGetLastError();
    return BFIBM_ECUDA;
  }
  PList& L = kind == 0 ? P.swv[level] : P.swp[level];
  cudaError_t e = sweep_list(P, level, kind == 0 ? 0 : 3, sh, L);
  if (e == cudaSuccess && sh.smem > 48 * 1024) {
    b->err = "the sweep shape needs more than 48 KB of shared memory";
    sh = kind == 0 ? P.shv[level] : P.shp[level];
    e = sweep_list(P, level, kind == 0 ? 0 : 3, sh, L);
    if (e == cudaSuccess) return BFIBM_EINVAL;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BFIBM_ECUDA;
  }
  (kind == 0 ? P.shv[level] : P.shp[level]) = sh;
  if (P.gexec) cudaGraphExecDestroy(P.gexec);
  P.gexec = nullptr;
  bfibm_status st = persist_capture(P);
  if (st != BFIBM_OK) {   // a plan without its graph is of no use
    b->err = P.err;
    persist_free(b->ps);
    b->ps = nullptr;
  }
  return st;
}

const char* bfibm_batch_error(bfibm_batch* b) { return b ? b->err.c_str() : ""; }

bfibm_status bfibm_batch_step(bfibm_batch* b, const int32_t* nsteps) {
  if (!b) return BFIBM_EINVAL;
  if (b->persistent) return persist_step(b, nsteps);
  bfibm_status agg = BFIBM_OK;
  for (size_t q = 0; q < b->slots.size(); ++q) {
    bfibm_batch::Slot& s = b->slots[q];
    if (!s.c) continue;
    int n = nsteps ? nsteps[q] : 1;
    if (n <= 0) {
      s.timed = false;
      continue;
    }
    bfibm_ctx* c = s.c;
    READY(c);
    CK(cudaEventRecord(s.e0, c->stream));
    bfibm_status st = do_steps(c, n, false);
    if (st != BFIBM_OK && st != BFIBM_ENOCONV) return st;
    if (st == BFIBM_ENOCONV) agg = st;
    CK(cudaEventRecord(s.e1, c->stream));
    s.timed = true;
  }
  return agg;
}

bfibm_status bfibm_batch_wait(bfibm_batch* b) {
  if (!b) return BFIBM_EINVAL;
  bfibm_status agg = BFIBM_OK;
  for (auto& s : b->slots) {
    if (!s.c) continue;
    bfibm_ctx* c = s.c;
    READY(c);
    bfibm_status st = check_status(c);
    if (st == BFIBM_ENOCONV) agg = BFIBM_ENOCONV;
    else if (st != BFIBM_OK) return st;
  }
  return agg;
}

bfibm_status bfibm_batch_slot_ms(bfibm_batch* b, int32_t slot, float* ms) {
  if (!b || !ms || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].c)
    return BFIBM_EINVAL;
  bfibm_batch::Slot& s = b->slots[slot];
  if (!s.timed) return BFIBM_ESTATE;
  bfibm_ctx* c = s.c;
  CK(cudaEventSynchronize(s.e1));
  CK(cudaEventElapsedTime(ms, s.e0, s.e1));
  return BFIBM_OK;
}

void bfibm_batch_destroy(bfibm_batch* b) {
  if (!b) return;
  persist_free(b->ps);
  for (auto& s : b->slots) {
    if (s.e0) cudaEventDestroy(s.e0);
    if (s.e1) cudaEventDestroy(s.e1);
  }
  delete b;
}

}  // extern "C"
