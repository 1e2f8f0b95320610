// Internal declarations shared by the CUDA translation units of libbfibm.
// Kernels live in stencil.cu (Eulerian grid work) and lagrangian.cu (nodes,
// springs, transfers); solver.cu holds the context, the multigrid driver and
// the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bf {

constexpr int kMaxLevels = 8;
constexpr int kRedBlocks = 1024;   // blocks of every partial-reduction kernel

// Geometry of one multigrid level. Every array of the level shares it.
// Storage extent s[a] = n[a] + 1 on a wall axis (room for the upper wall
// face/edge), n[a] on a periodic axis; x is contiguous, rows are padded to
// st[1] elements.
struct Geo {
  int n[3];
  int s[3];
  int per[3];
  long long st[3];   // strides in elements: 1, pitch, pitch * s[1]
  double h;
  int open;          // the open flow axis of a duct with inflow and outflow (Sec. 3.6), or -1:
                     // face 0 along it holds the prescribed inflow, face n is the outflow (an
                     // unknown with du/dn = 0 and the pressure held there)
};

__host__ __device__ inline long long gidx(const Geo& g, int i, int j, int k) {
  return (long long)i + g.st[1] * j + g.st[2] * k;
}

template <typename T>
struct LevelPtrs {
  T* p;          // pressure iterate
  T* pf;         // pressure rhs
  T* pr;         // pressure residual
  T* beta[3];    // 1/rho on faces (restricted)
  T* u[3];       // viscous iterate
  T* uf[3];      // viscous rhs
  T* ur[3];      // viscous residual
  T* m[3];       // rho sigma / dt on faces
  T* muc;        // mu at centres
  T* mue[3];     // mu on edges: xy, xz, yz
  T* p2;         // second buffer of p for out-of-place sweeps
  T* u2[3];      // second buffers of u
  T* idg[3];     // FP32 sweeps: 1 / diagonal of the viscous operator of component d
};

struct Ptr3d {
  double* a[3];
};

// The FP32 viscous point update, Eq. (NSdis1-1) with Eq. (divergenceGrad) /
// (divergencePartial) on the staggered grid, with every rounding written out
// (each product, difference and fused multiply-add explicit), so that every
// FP32 sweep kernel (ring, pair and TMA-staged) gives the same bits whatever
// the compiler would otherwise contract:
//   cross += mep (u_e(F+e) - u_e(F+e-d)) - mem (u_e(F) - u_e(F-d))
//   off = cross + cdp u_d(F+d) + cdm u_d(F-d) + sum_e (cep u_d(F+e) + cem u_d(F-e))
//   u_d(F) = (rhs + ir off) / diag, with 1 / diag precomputed
__device__ __forceinline__ float vx_cross(float cross, float mep, float uEp, float uEpm, float mem,
                                          float uF, float uFm) {
  return __fadd_rn(cross,
                   __fmaf_rn(mep, __fsub_rn(uEp, uEpm), -__fmul_rn(mem, __fsub_rn(uF, uFm))));
}
__device__ __forceinline__ float vx_off(float cross, float cdp, float up, float cdm, float um) {
  return __fmaf_rn(cdm, um, __fmaf_rn(cdp, up, cross));
}
__device__ __forceinline__ float vx_acc(float off, float w, float u) { return __fmaf_rn(w, u, off); }
__device__ __forceinline__ float vx_final(float rhs, float ir, float off, float idg) {
  return __fmul_rn(__fmaf_rn(ir, off, rhs), idg);
}

// The FP32 pressure point update, Eq. (divergenceGrad) in the order of the
// two-kernel sweep (neighbours axis 0, 1, 2, lower then upper), every
// rounding written out so that every FP32 pressure sweep (ring, pair, TMA,
// the coarse-level kernel) gives the same bits:
//   num = fma(beta_nb, p_nb, num), dg = dg + beta_nb per neighbour,
//   p = fma(-h^2, f, num) / dg
// A neighbour beyond a wall may enter with beta 0 and p 0: it changes no bit.
__device__ __forceinline__ void px_acc(float& num, float& dg, float b, float p) {
  num = __fmaf_rn(b, p, num);
  dg = __fadd_rn(dg, b);
}
__device__ __forceinline__ float px_final(float num, float dg, float h2, float f) {
  return __fdiv_rn(__fmaf_rn(-h2, f, num), dg);
}

struct Scalars {
  double* partial;   // kRedBlocks partial results
  double* out;       // 16 finalized scalars
};

// ------------------------------------------------------- batched launches
// The block a kernel body works on: its coordinates and the extent of the
// grid it belongs to. A single-instance kernel passes its own blockIdx and
// gridDim; a batched kernel passes the block of one member's grid that an
// item of its work list names. Partial sums are indexed by linear(), so a
// member's reductions come out the same in a batch as alone.
struct Blk {
  int x, y, z, gx, gy, gz;
  __device__ __forceinline__ int linear() const { return x + gx * (y + gy * z); }
};
__device__ __forceinline__ Blk own_blk() {
  return Blk{(int)blockIdx.x, (int)blockIdx.y, (int)blockIdx.z,
             (int)gridDim.x,  (int)gridDim.y,  (int)gridDim.z};
}

// One item of a batched launch's work list: block (x, y, z) of the
// gx x gy x gz grid the single-instance launch would use on member m.
struct BItem {
  int m;
  unsigned short x, y, z, gx, gy, gz;
};

// One member of a persistent batch as the batched kernels see it.
struct BMember {
  Geo g[kMaxLevels];
  LevelPtrs<float> f[kMaxLevels];
  LevelPtrs<double> d[kMaxLevels];
  int L;                    // levels
  double inv_re;
  double* vdiag[3];         // FP64 viscous diagonal (level 0)
  double* cg_p[3];          // flexible-CG direction, A times it, preconditioned residual
  double* cg_q[3];
  double* cg_z[3];
  Scalars sc;
  int* cycles;              // device-loop iterations of the last solves (viscous, pressure)
  long long* total;         // device-loop iterations so far (viscous, pressure)
  int* nonconv;             // solves stopped above their tolerance
  double rtol;
  int maxc;                 // outer iterations of a solve at most
  double dscale, div_tol;   // the pressure loop's second test: dscale max |r_p| <= div_tol
  int coarse_sweeps;
  int nu1, nu2;             // sweeps before and after the coarse-grid correction
  int tail;                 // first level of the coarse-level cluster kernel (L: none)
  double ir[kMaxLevels];    // inv_re / h^2 per level and 1 / h^2, formed on the host (IEEE
  double ih2[kMaxLevels];   // division, the same bits as on the device) so that no thread
                            // divides in FP64
};

// What every batched kernel takes: its work list, the member table, the mask
// of members whose solve is still iterating (null: every member), the level,
// and which buffer holds each current iterate (bit e: u_e is in u2[e]; bit 3:
// p is in p2), as the out-of-place sweeps leave them.
struct BArgs {
  const BItem* items;
  int n;
  const BMember* tab;
  const int* act;
  int lev;
  int cur;
};

// The persistent loop of a batched kernel: the launch's blocks stride over
// the work list; a masked member's items are skipped. The barrier after each
// item lets the next one reuse shared memory.
template <class F>
__device__ __forceinline__ void for_items(const BArgs& A, F&& f) {
  for (int w = blockIdx.x; w < A.n; w += gridDim.x) {
    const BItem it = A.items[w];
    if (A.act && !A.act[it.m]) continue;
    f(A.tab[it.m], Blk{it.x, it.y, it.z, it.gx, it.gy, it.gz});
    __syncthreads();
  }
}

// a member's FP32 arrays of one level with the current iterates in front
__device__ __forceinline__ LevelPtrs<float> cur_ptrs(const LevelPtrs<float>& in, int cur) {
  LevelPtrs<float> L = in;
#pragma unroll
  for (int e = 0; e < 3; ++e)
    if ((cur >> e) & 1) {
      L.u[e] = in.u2[e];
      L.u2[e] = in.u[e];
    }
  if ((cur >> 3) & 1) {
    L.p = in.p2;
    L.p2 = in.p;
  }
  return L;
}

// ---------------------------------------------------------------- stencil.cu
// Pressure: one colour of red-black Gauss-Seidel for D.(beta D p) = f.
template <typename T>
void launch_p_rbgs(int D, const Geo& g, const LevelPtrs<T>& L, int colour, cudaStream_t s);
template <typename T>
void launch_p_residual(int D, const Geo& g, const LevelPtrs<T>& L, cudaStream_t s);
// Viscous: one colour of component d.
template <typename T>
void launch_v_rbgs(int D, const Geo& g, const LevelPtrs<T>& L, int d, int colour, double inv_re,
                   cudaStream_t s);
template <typename T>
void launch_v_residual(int D, const Geo& g, const LevelPtrs<T>& L, double inv_re, cudaStream_t s);
// Transfers between level l (fine) and l+1 (coarse).
template <typename T>
void launch_restrict_cell(int D, const Geo& gf, const Geo& gc, const T* rf, T* fc, T* xc,
                          cudaStream_t s);
template <typename T>
void launch_restrict_face(int D, int d, const Geo& gf, const Geo& gc, const T* rf, T* fc, T* xc,
                          cudaStream_t s);
template <typename T>
void launch_prolong_cell(int D, const Geo& gf, const Geo& gc, const T* ec, T* xf, cudaStream_t s);
template <typename T>
void launch_prolong_face(int D, int d, const Geo& gf, const Geo& gc, const T* ec, T* xf,
                         cudaStream_t s);
// the three face components in one launch (3D, no open axis)
template <typename T>
void launch_restrict_face3(const Geo& gf, const Geo& gc, T* const rf[3], T* const fc[3],
                           T* const xc[3], cudaStream_t s);
template <typename T>
void launch_prolong_face3(const Geo& gf, const Geo& gc, T* const ec[3], T* const xf[3],
                          cudaStream_t s);
// Coarsest level: the whole solve in one block.
template <typename T>
void launch_coarse_p(int D, const Geo& g, const LevelPtrs<T>& L, int sweeps, cudaStream_t s);
template <typename T>
void launch_coarse_v(int D, const Geo& g, const LevelPtrs<T>& L, int sweeps, double inv_re,
                     cudaStream_t s);

// Fused sweeps (smooth.cu): both colours in one pass, read L.p / L.u[d],
// write `out`.
template <typename T>
void launch_p_rb_fused(int D, const Geo& g, const LevelPtrs<T>& L, T* out, cudaStream_t s,
                       int TYo = 0, int KCo = 0, int NPo = 1, int BXo = 0);
template <typename T>
void launch_v_rb_fused(int D, const Geo& g, const LevelPtrs<T>& L, int d, T* out, double inv_re,
                       cudaStream_t s, int TYo = 0, int KCo = 0, int NPo = 1, int BXo = 0);
// chunk planes filling `waves` waves of resident blocks (3D FP32 sweeps; 0: none)
int ring_fill_kc(int D, int K, const Geo& g, int TY, int NP, int BX, int waves);
// The pair sweep of a 3D FP32 viscous component (smooth.cu): one thread per
// (red, black) pair of a row, TY rows per block plus two ring rows, KC planes
// per chunk; same arithmetic as the one-pass sweep
bool pair_eligible(int D, const Geo& g, int TY);
void launch_v_rb_pair(const Geo& g, const LevelPtrs<float>& L, int d, float* out, double inv_re,
                      cudaStream_t s, int TY, int KC);
// the pair sweep of the 3D FP32 pressure (same eligibility and shapes)
void launch_p_rb_pair(const Geo& g, const LevelPtrs<float>& L, float* out, cudaStream_t s, int TY,
                      int KC);
// d: 0..2 viscous component, 3 pressure
int pair_fill_kc(const Geo& g, int d, int TY, int waves);

// Mixed precision (mixed.cu).
int red_blocks_3d(int D, const Geo& g);
// (partial, when not null, receives the blocks' sums of r^2 and then their
// maxima of |r|: 2 red_blocks_3d entries)
void launch_p_residual_mixed(int D, const Geo& g, const LevelPtrs<double>& L, float* r32,
                             float* e32, double* partial, cudaStream_t s);
void launch_v_residual_mixed(int D, const Geo& g, const LevelPtrs<double>& L, float* const r32[3],
                             float* const e32[3], double* const diag[3], double inv_re,
                             double* partial, cudaStream_t s, double* const r64[3] = nullptr);
// Flexible CG around the FP32 V-cycle (mixed.cu): z is the V-cycle's result
// converted to FP64; w = A z with partial z.q;
// p = z + beta p, q = w + beta q with partials p.q, p.r (2 nb entries);
// x += alpha p, r -= alpha q, r32 = r, e32 = 0 with partial r.r. beta and
// alpha are read from out[] slots on the device.
void launch_fcg_apply(int D, const Geo& g, const LevelPtrs<double>& L, double* const z[3],
                      double* const diag[3], double inv_re, double* const w[3],
                      double* const q[3], double* partial, cudaStream_t s);
void launch_fcg_dir(int D, const Geo& g, double* const z[3], double* const w[3], double* const p[3],
                    double* const q[3], double* const r[3], const double* out, int sl_zq,
                    int sl_pq, double* partial, cudaStream_t s);
// blocks of the flat direction and update passes (their partial sums)
int fcg_flat_blocks(const Geo& g);
void launch_fcg_update(int D, const Geo& g, double* const x[3], double* const p[3],
                       double* const q[3], double* const r[3], float* const r32[3],
                       float* const e32[3], const double* out, int sl_pq, int sl_pr,
                       double* partial, cudaStream_t s);
// diagonal of the FP64 viscous operator on one level (formed once per step)
void launch_v_diag(int D, const Geo& g, const LevelPtrs<double>& L, double* const diag[3],
                   double inv_re, cudaStream_t s);
void launch_add_correction(int D, const Geo& g, double* const x[3], float* const e[3], int ncomp,
                           cudaStream_t s);
void launch_f32_to_f64(const float* in, double* out, long long n, cudaStream_t s);
// three arrays of n elements each in one launch
void launch_f32_to_f64_3(float* const in[3], double* const out[3], long long n, cudaStream_t s);
void launch_f64_to_f32(const double* in, float* out, long long n, cudaStream_t s);
// 1 / diagonal of the viscous operator per face component, from the FP64
// coefficients of one level, stored in L32.idg (0 on the fixed wall faces)
void launch_v_idg32(int D, const Geo& g, const LevelPtrs<double>& L64,
                    const LevelPtrs<float>& L32, double ir, cudaStream_t s);
void launch_coef_to_f32(int D, const Geo& g, const LevelPtrs<double>& L64,
                        const LevelPtrs<float>& L32, cudaStream_t s);
// out[slot] = scale * sum(partial[0..nb))
void launch_finalize_sum(const double* partial, int nb, double* out, int slot, double scale,
                         cudaStream_t s);

// allow the coarsest-level kernels up to 160 KB of shared memory (call once,
// outside stream capture)
cudaError_t coarse_set_smem();

cudaError_t fused_set_carveout();

// ------------------------------------------- batched kernels (3D, FP32 V-cycles)
// One launch covers a level (or phase) of every member its work list names;
// `grid` blocks stride over the list (for_items). Transfers take A.lev as the
// fine level. Each does, per member, the arithmetic of the single-instance
// launch it mirrors, on that launch's block decomposition.
// stencil.cu
void launch_b_v_residual32(const BArgs& A, int grid, cudaStream_t s);
void launch_b_p_residual32(const BArgs& A, int grid, cudaStream_t s);
void launch_b_restrict_face32(const BArgs& A, int grid, cudaStream_t s);   // 3 components
void launch_b_restrict_cell32(const BArgs& A, int grid, cudaStream_t s);
void launch_b_prolong_face32(const BArgs& A, int grid, cudaStream_t s);    // 3 components
void launch_b_prolong_cell32(const BArgs& A, int grid, cudaStream_t s);
// The coarsest level A.lev of each listed member (one item each): its FP32
// right-hand side converted to FP64, the iterate zeroed, the FP64 coarse
// solve, the result rounded to FP32. smem: the largest b_coarse_smem of the
// members.
void launch_b_coarse(const BArgs& A, bool viscous, size_t smem, cudaStream_t s);
size_t b_coarse_smem(const Geo& g, bool viscous);
cudaError_t b_coarse_set_smem();
// level 0: per-block sums of uf . uf (viscous) or pf^2 into sc.partial
void launch_b_norm2(const BArgs& A, bool viscous, int grid, cudaStream_t s);
// level 0: the two passes of the pressure's mean removal around a finalize
void launch_b_partial_sum_p(const BArgs& A, int grid, cudaStream_t s);
void launch_b_sub_scalar_p(const BArgs& A, int grid, cudaStream_t s);
// one item per member with gx = nb, the partials its producer wrote:
// out[slot] = scale * (sum or max of partial[off nb .. off nb + nb)), scale
// 1, or 1 / cells with `mean`
void launch_b_finalize(const BArgs& A, int off, int slot, bool is_max, bool mean,
                       cudaStream_t s);
// Start of a batched solve: every member active, its loop counter (`which`:
// 0 viscous, 1 pressure) zeroed and out[zero_slot] = 0 when zero_slot >= 0.
void launch_b_begin(const BMember* tab, int nm, int* act, int which, int zero_slot,
                    cudaStream_t s);
// End of an iteration of a batched device loop: for each active member the
// test of the single-instance loop (||r||/||f|| from out[sr], out[sf]; with
// smax >= 0 also dscale out[smax] <= div_tol); a member that stops leaves the
// mask; the loop runs again while any member is active.
// The coarse levels of an FP32 V-cycle in one launch (stencil.cu): one
// cluster of kTailCtas CTAs per listed member runs its levels tail .. L - 1
// (tail from the member table): nu1 in-place red-black sweeps per level,
// residual and restriction down to the coarsest level, the FP64 coarse solve
// there (with its conversions), prolongation and nu2 sweeps back up, with a
// cluster barrier between phases. Same arithmetic, point for point, as the
// launches it replaces. viscous: the viscous components, else the pressure;
// act (may be null) masks members; smem: the largest tail_smem of the members;
// ctas 1 gives each member one CTA (a batch's members then run side by side).
constexpr int kTailCtas = 8;
void launch_tail(bool viscous, const BMember* tab, const int* list, int nlist, const int* act,
                 size_t smem, cudaStream_t s, int ctas = kTailCtas);
size_t tail_smem(const Geo& coarsest, bool viscous);
cudaError_t tail_set_smem();
// iters[which] counts the loop's iterations; use_h false: no loop node to
// steer (an unrolled loop), the masks alone decide.
void launch_b_tol_check(cudaGraphConditionalHandle h, const BMember* tab, int nm, int* act,
                        int which, int sf, int sr, int smax, long long* iters, cudaStream_t s,
                        bool use_h = true);
// counts in each member's nonconv the solves whose ||r||/||f|| exceeds slack rtol
void launch_b_res_check(const BMember* tab, int nm, int sf, int sr, double slack,
                        cudaStream_t s);
// mixed.cu (level 0, FP64)
void launch_b_v_residual_mixed(const BArgs& A, bool partial, bool r64, int grid, cudaStream_t s);
void launch_b_p_residual_mixed(const BArgs& A, bool partial, int grid, cudaStream_t s);
void launch_b_add_correction(const BArgs& A, bool viscous, int grid, cudaStream_t s);
void launch_b_z_to_f64(const BArgs& A, int grid, cudaStream_t s);
void launch_b_fcg_apply(const BArgs& A, int grid, cudaStream_t s);
void launch_b_fcg_dir(const BArgs& A, int sl_zq, int sl_pq, int grid, cudaStream_t s);
void launch_b_fcg_update(const BArgs& A, int sl_pq, int sl_pr, int grid, cudaStream_t s);
// blocks of the single-instance launches the batched ones mirror: the 1D
// reductions over n cells, the 3D launches (32 x 4 x 2 threads) over
// nx x ny x nz points, the flat conversions over n elements
int red_grid_of(long long n);
dim3 stencil_grid3(long long nx, long long ny, long long nz);
int flat_convert_blocks(long long n);
// smooth.cu: one ring sweep of viscous component K (0..2) or the pressure
// (K = 3) on level A.lev of every listed member, out of place (the output
// buffer is the one A.cur marks as not current); TY rows, KC planes, NP
// planes per phase, blocks of bx x (TY + 2) threads
void launch_b_sweep(const BArgs& A, int K, int TY, int KC, int NP, int bx, size_t smem, int grid,
                    cudaStream_t s);
const void* b_sweep_kernel(int K, int NP);
size_t b_sweep_smem(int NP, int TY, int W);
// the pair sweep of viscous component d over a work list of pair-eligible
// members sharing the streaming axis' periodicity (perz); one block of
// bx x (TY + 2) threads per item; smem: 4 (TY + 2) W floats, W the widest row
void launch_b_pair(const BArgs& A, int d, bool perz, int TY, int KC, int bx, size_t smem,
                   cudaStream_t s);
// the same for the pressure
void launch_b_ppair(const BArgs& A, bool perz, int TY, int KC, int bx, size_t smem,
                    cudaStream_t s);
// after an odd count of sweeps: the current iterate of kind K copied back to
// its own buffer (items: flat blocks over the level's elements)
void launch_b_copy_back(const BArgs& A, int K, int grid, cudaStream_t s);

// ---------------------------------------------------------------- smooth_tma.cu
// 3D FP32 red-black sweeps with TMA-staged inputs. Kind K: 0..2 viscous
// component, 3 pressure; coef = inv_re / h^2 (viscous) or h^2 (pressure);
// err counts bounded waits that ran out.
// default limit of the TMA sweep's bounded waits (a context may set its own;
// 0 tests each barrier once without waiting)
constexpr unsigned long long kTmaWaitNs = 2000000000ull;
bool tma_eligible(int D, const Geo& g);
cudaError_t tma_set_smem();
cudaError_t tma_autotune(int D, const Geo& g, const LevelPtrs<float>& L, int K, float* out,
                         int* err, double coef, cudaStream_t s);
cudaError_t launch_rb_tma(int D, const Geo& g, const LevelPtrs<float>& L, int K, float* out,
                          int* err, double coef, cudaStream_t s,
                          unsigned long long wait_ns = kTmaWaitNs);
// pin a plan {TY, KC, PD, SW, grid (0: resident blocks)} for a level shape
bool tma_set_plan(int K, const Geo& g, const int in[5]);
// the one-pass sweep's tuned tile rows, chunk planes, planes per phase,
// threads per row and kernel (0 ring sweep, 1 pair sweep) for a level shape
bool ring_shape_of(int K, const Geo& g, int* TY, int* KC, int* NP, int* BX, int* KERN = nullptr);
bool ring_set_shape(int K, const Geo& g, const int in[5]);
// whether the tuner found the TMA sweep faster than the one-pass sweep
bool tma_chosen(int K, const Geo& g);
// tuned plan of a level shape: tile rows, chunk planes, prefetch planes,
// strip columns, grid
bool tma_plan_of(int K, const Geo& g, int out[5]);

// FP64-only grid stages.
void launch_coef_fine(int D, const Geo& g, double* const rho[3], double* beta[3], double* m[3],
                      double msc, cudaStream_t s);
void launch_coef_restrict(int D, const Geo& gf, const Geo& gc, const LevelPtrs<double>& F,
                          const LevelPtrs<double>& C, double gamma, cudaStream_t s);
void launch_adv_rhs(int D, const Geo& g, double* const uvel[3], double* const rho[3],
                    double* const frc[3], const LevelPtrs<double>& L0, double c_force,
                    int flow_axis, const double* G_dev, cudaStream_t s);
// (an open duct keeps the mean and moves the held outflow pressure p_out into
// the last cells: b -= 2 beta_out p_out / h^2)
void launch_divergence(int D, const Geo& g, double* const u[3], double* b, double scale,
                       Scalars sc, cudaStream_t s, const double* beta_open = nullptr,
                       double p_out = 0.0);
// The divergence check fused into the projection: out[acc] accumulates the
// max |D.u| of the projected velocity (bit pattern of a double); a small
// kernel then copies it to out[step], folds it into out[all] (max over all
// steps), counts a violation in *viol when it exceeds tol (> 0) and clears
// out[acc].
struct DivCheck {
  double* out;
  int acc, step, all;
  double tol;
  int* viol;
  double p_out;   // open duct: the pressure held at the outflow
};
void launch_project(int D, const Geo& g, double* const ut[3], const double* p,
                    double* const beta[3], double* uvel[3], double coef, const DivCheck& dc,
                    cudaStream_t s);
// mean over cells of a (deterministic two-pass) subtracted from a
void launch_sub_mean(int D, const Geo& g, double* a, Scalars sc, cudaStream_t s);
// sum of squares over the unknowns (cells if ncomp == 0, else the faces of
// ncomp components) -> sc.out[slot]
void launch_norm2(int D, const Geo& g, double* const a[3], int ncomp, Scalars sc, int slot,
                  cudaStream_t s);
// max |D.u| -> sc.out[slot], sum u^2 h^D -> sc.out[slot + 1]
void launch_div_ke(int D, const Geo& g, double* const u[3], Scalars sc, int slot, cudaStream_t s);
// laminar initial velocity and body force
void launch_laminar(int D, const Geo& g, int flow_axis, double mu_eff, double u_center,
                    double body_force, double ic_scale, double* ucomp, double* G_dev,
                    cudaStream_t s);
void launch_fill(double* a, long long n, double v, cudaStream_t s);
// device side of a relative-residual while loop in a graph (see solver.cu)
// (smax >= 0 adds a second test, mscale * out[smax] <= mtol when mtol > 0; a
// loop that stops at the cap with a test unmet is counted in *nonconv)
void launch_tol_check(cudaGraphConditionalHandle h, const double* out, int sf, int sr,
                      double rtol, int maxc, int* counter, long long* total, int* nonconv,
                      cudaStream_t s, int smax = -1, double mscale = 0.0, double mtol = 0.0);
// out[slot] = max of partial[0..nb)
void launch_finalize_max(const double* partial, int nb, double* out, int slot, cudaStream_t s);
// out[slot] = max over the cells of |a|
void launch_absmax_cells(int D, const Geo& g, const double* a, Scalars sc, int slot,
                         cudaStream_t s);
// counts ||r||/||f|| (from out[sr], out[sf]) above thresh in *nonconv
void launch_res_check(const double* out, int sf, int sr, double thresh, int* nonconv,
                      cudaStream_t s);

// ------------------------------------------------------------ lagrangian.cu
struct NodeSet {
  long long eta;
  double* X;    // eta x 3
  double* U;    // eta x 3
  double* F;    // eta x 3
  int* tile;    // eta: tile of each node
  int* perm;    // eta: nodes sorted by tile
  int* count;   // ntiles + 1
  int* start;   // ntiles + 1
  int* cursor;  // ntiles
  int* clamped; // 1 counter
  int* nonfinite;  // 1 counter: non-finite coordinates reset to 0
  double* tw;   // eta x 2 widths x 2 staggers x 3 axes x 4: 1D delta weights
  int* tlo;     // eta x 2 x 2 x 3 x (first index, count)
};
struct SpringSet {
  long long m;
  int* ab;          // m x 2
  double* rest;
  double* K;
  double* brk;
  int* broken;      // m flags
  int* ev_id;       // m slots
  int* ev_step;
  int* ev_count;    // 1 counter
  long long* step;  // device step counter
  double* fvec;     // m x 3: the force each spring puts on its first node
  int* adj_start;   // eta + 1: springs of node s are adj[adj_start[s] .. adj_start[s+1])
  int* adj;         // 2 m: 2 * spring + (0: first node, 1: second node), springs ascending
  long long adj_eta;   // node count the adjacency was built for
};
struct TileGeo {
  int T[3];         // cells per tile and axis
  int nt[3];        // tiles per axis
  int H;            // halo (grid points) around a tile in shared memory
  int ntiles;
};
struct SpreadArgs {
  int D;
  int phi_kind;
  double omega, omega_mu;
  double amp_rho;     // rho_b d0^D
  double mu_out, mu_coef;   // (2 w)^D (mu_max - mu_out)
  double rho_f;       // background density
  double* scale;      // device [2]: fixed-point scales of the force and density sums
};

void launch_springs(int D, const Geo& g, const NodeSet& N, const SpringSet& S, cudaStream_t s);
void launch_bin(int D, const Geo& g, const TileGeo& tg, const NodeSet& N, cudaStream_t s);
void launch_reset_fields(int D, const Geo& g, double* frc[3], double* rho[3], double* muc,
                         double* mue[3], double rho_f, double mu_f, cudaStream_t s);
void launch_spread(int D, const Geo& g, const TileGeo& tg, const NodeSet& N, const SpreadArgs& a,
                   double* frc[3], double* rho[3], double* muc, double* mue[3], cudaStream_t s);
// f and rho leave the spread as 64-bit fixed-point sums (see lagrangian.cu);
// this converts them to doubles (run after every spread, and after a reset
// without nodes)
void launch_spread_finish(int D, const Geo& g, const SpreadArgs& a, double* frc[3], double* rho[3],
                          cudaStream_t s);
void launch_interp_advance(int D, const Geo& g, const NodeSet& N, double* const uvel[3],
                           int phi_kind, double dt_over_sigma, cudaStream_t s);
void launch_step_increment(long long* step, cudaStream_t s);
size_t spread_smem_bytes(int D, const TileGeo& tg);
// opt the spread kernel into more than 48 KB of dynamic shared memory (call
// once, outside stream capture)
cudaError_t spread_set_smem(int D, size_t bytes);
size_t spread_smem_limit();

}  // namespace bf
