// Mixed-precision pieces of the defect-correction solves: each outer
// iteration computes the fine-grid residual r = f - A x in FP64, hands it to
// an FP32 V-cycle as the right-hand side of A e = r (e starts at 0), and adds
// the FP32 correction back into the FP64 iterate. The coarsest grid is solved
// in FP64 (its right-hand side and solution are converted at the boundary).
#include <cuda_runtime.h>
#include <math_constants.h>

#include "common.cuh"

namespace bf {

namespace {

constexpr int kBlock1D = 256;

__host__ __device__ constexpr int edge_id(int d, int e) {
  return (d < e ? d : e) + (d < e ? e : d) - 1;
}
__device__ __forceinline__ long long offp(const Geo& g, int a, int ci) {
  return (g.per[a] && ci == g.n[a] - 1) ? -(long long)(g.n[a] - 1) * g.st[a] : g.st[a];
}
__device__ __forceinline__ long long offm(const Geo& g, int a, int ci) {
  return (g.per[a] && ci == 0) ? (long long)(g.n[a] - 1) * g.st[a] : -g.st[a];
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// sum over a block whose size is a multiple of 32; valid in thread 0
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  int t = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  int nt = blockDim.x * blockDim.y * blockDim.z;
  int lane = t & 31, w = t >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  v = (t < (nt + 31) / 32) ? sh[t] : 0.0;
  if (w == 0) v = warp_sum(v);
  __syncthreads();
  return v;
}
// maximum over a block whose size is a multiple of 32; valid in thread 0
__device__ double block_max(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  int t = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  int nt = blockDim.x * blockDim.y * blockDim.z;
  int lane = t & 31, w = t >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  v = (t < (nt + 31) / 32) ? sh[t] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  __syncthreads();
  return v;
}
inline dim3 blk3(int D) { return D == 3 ? dim3(32, 4, 2) : dim3(32, 8, 1); }
inline dim3 grd3(long long nx, long long ny, long long nz, dim3 b) {
  return dim3((unsigned)((nx + b.x - 1) / b.x), (unsigned)((ny + b.y - 1) / b.y),
              (unsigned)((nz + b.z - 1) / b.z));
}

// FP64 pressure residual written as the FP32 right-hand side of the
// correction equation; the FP32 correction is zeroed; per-block partial sums
// of r^2 (for the relative-residual test) in partial[0 .. nb) and per-block
// maxima of |r| (for the divergence the projection will leave, Eq. NSdis2 -
// NSdis4: max |D.u| = (euler dt / sigma) max |r|) in partial[nb .. 2 nb),
// nb the launch's blocks; a non-finite residual counts as infinity.
template <int D>
__device__ __forceinline__ void p_residual_mixed_body(const Blk& B, Geo g, LevelPtrs<double> L,
                                                      float* r32, float* e32, double* partial,
                                                      double ih2) {
  __shared__ double sh[32];
  int i = B.x * blockDim.x + threadIdx.x;
  int j = B.y * blockDim.y + threadIdx.y;
  int k = B.z * blockDim.z + threadIdx.z;
  double r2 = 0.0, ra = 0.0;
  if (i < g.n[0] && j < g.n[1] && k < g.n[2]) {
    int ci[3] = {i, j, k};
    long long c = gidx(g, i, j, k);
    double num = 0.0, dg = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const double* __restrict__ b = L.beta[a];
      if (ci[a] > 0 || g.per[a]) {
        double bb = b[c];
        num += bb * L.p[c + offm(g, a, ci[a])];
        dg += bb;
      }
      if (ci[a] < g.n[a] - 1 || g.per[a]) {
        long long cp = c + offp(g, a, ci[a]);
        double bb = b[cp];
        num += bb * L.p[cp];
        dg += bb;
      }
    }
    double r = L.pf[c] - (num - dg * L.p[c]) * ih2;   // ih2 = 1 / h^2 from the host
    r32[c] = (float)r;
    e32[c] = 0.0f;
    r2 = r * r;
    ra = fabs(r);
    if (!(ra <= CUDART_INF)) ra = CUDART_INF;
  }
  if (partial) {
    r2 = block_sum(r2, sh);
    ra = block_max(ra, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) {
      const int nb = B.gx * B.gy * B.gz;
      partial[B.linear()] = r2;
      partial[nb + B.linear()] = ra;
    }
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_p_residual_mixed(Geo g, LevelPtrs<double> L, float* r32,
                                                          float* e32, double* partial, double ih2) {
  p_residual_mixed_body<D>(own_blk(), g, L, r32, e32, partial, ih2);
}

// Diagonal of the FP64 viscous operator of component d at face F:
// m_d + (inv_re / h^2) * (2 mu_c on both cells + the edge viscosities, an edge
// beyond a wall counted twice for the mirrored tangential neighbour). The
// coefficients stay fixed through a time step's solves, so the diagonal is
// formed once per step instead of in every defect-correction cycle.
template <int D, int d>
__device__ __forceinline__ double v_diag64(const Geo& g, const LevelPtrs<double>& L,
                                           const int ci[3], long long F, double ir) {
  long long od_m = offm(g, d, ci[d]);
  double mcp = L.muc[F], mcm = L.muc[F + od_m];
  double dgV = 2.0 * (mcp + mcm);
#pragma unroll
  for (int e = 0; e < D; ++e) {
    if (e == d) continue;
    const double* __restrict__ me = L.mue[edge_id(d, e)];
    bool pe = g.per[e] != 0;
    bool wp = !pe && ci[e] == g.n[e] - 1;
    bool wm = !pe && ci[e] == 0;
    double mep = me[F + offp(g, e, ci[e])], mem = me[F];
    dgV += (wp ? 2.0 : 1.0) * mep + (wm ? 2.0 : 1.0) * mem;
  }
  return L.m[d][F] + ir * dgV;
}

template <int D>
__global__ void __launch_bounds__(256) k_v_diag(Geo g, LevelPtrs<double> L, Ptr3d diag,
                                                double ir) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) return;
  int ci[3] = {i, j, k};
  long long F = gidx(g, i, j, k);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    double v = 0.0;
    if (g.per[d] || ci[d] != 0) {
      if (d == 0) v = v_diag64<D, 0>(g, L, ci, F, ir);
      else if (d == 1) v = v_diag64<D, 1>(g, L, ci, F, ir);
      else v = v_diag64<D, (D == 3 ? 2 : 1)>(g, L, ci, F, ir);
    }
    diag.a[d][F] = v;
  }
}

struct F32x3 {
  float* a[3];
};

// 1 / diagonal per face component for the FP32 sweeps: formed in FP64 from
// the level's FP64 coefficients, rounded once to FP32.
template <int D>
__global__ void __launch_bounds__(256) k_v_idg32(Geo g, LevelPtrs<double> L, F32x3 idg,
                                                 double ir) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) return;
  int ci[3] = {i, j, k};
  long long F = gidx(g, i, j, k);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    float v = 0.f;
    if (g.per[d] || ci[d] != 0) {
      double dg;
      if (d == 0) dg = v_diag64<D, 0>(g, L, ci, F, ir);
      else if (d == 1) dg = v_diag64<D, 1>(g, L, ci, F, ir);
      else dg = v_diag64<D, (D == 3 ? 2 : 1)>(g, L, ci, F, ir);
      v = (float)(1.0 / dg);
    }
    idg.a[d][F] = v;
  }
}

// FP64 viscous residual of component d at face F with the diagonal read from
// `diag` (the same arithmetic as the FP64 residual kernel). INTERIOR: no
// neighbour lies beyond a wall or across a periodic seam, so the offsets are
// the plain strides and no flag is tested.
template <int D, int d, bool INTERIOR, typename V>
__device__ __forceinline__ double v_off64(const Geo& g, const LevelPtrs<double>& L,
                                          const V* const vec[3], const int ci[3], long long F) {
  const V* __restrict__ ud = vec[d];
  const long long od_p = INTERIOR ? g.st[d] : offp(g, d, ci[d]);
  const long long od_m = INTERIOR ? -g.st[d] : offm(g, d, ci[d]);
  double mcp = L.muc[F], mcm = L.muc[F + od_m];
  double off = 2.0 * (mcp * (double)ud[F + od_p] + mcm * (double)ud[F + od_m]);
#pragma unroll
  for (int e = 0; e < D; ++e) {
    if (e == d) continue;
    const V* __restrict__ ue = vec[e];
    const double* __restrict__ me = L.mue[edge_id(d, e)];
    bool wp = false, wm = false;
    if (!INTERIOR) {
      bool pe = g.per[e] != 0;
      wp = !pe && ci[e] == g.n[e] - 1;
      wm = !pe && ci[e] == 0;
    }
    const long long oep = INTERIOR ? g.st[e] : offp(g, e, ci[e]);
    const long long oem = INTERIOR ? -g.st[e] : offm(g, e, ci[e]);
    long long Ep = F + oep;
    double mep = me[Ep], mem = me[F];
    double cp = (double)ue[Ep] - (double)ue[Ep + od_m];
    double cm = (double)ue[F] - (double)ue[F + od_m];
    double udp = 0.0, udm = 0.0;
    if (!wp) udp = (double)ud[Ep];
    if (!wm) udm = (double)ud[F + oem];
    off += mep * (udp + cp) + mem * (udm - cm);
  }
  return off;
}

// The off-diagonal part of the FP64 viscous operator of component d at face
// F applied to `vec` (FP64 or FP32 components, summed in FP64).
template <int D, int d, bool INTERIOR>
__device__ __forceinline__ double v_res64d(const Geo& g, const LevelPtrs<double>& L,
                                           const double* __restrict__ diag, const int ci[3],
                                           long long F, double ir) {
  const double* const vec[3] = {L.u[0], L.u[1], L.u[2]};
  double off = v_off64<D, d, INTERIOR, double>(g, L, vec, ci, F);
  return L.uf[d][F] - diag[F] * L.u[d][F] + ir * off;
}

template <int D, bool INTERIOR>
__device__ __forceinline__ double v_res_any(const Geo& g, const LevelPtrs<double>& L,
                                            const Ptr3d& diag, int d, const int ci[3],
                                            long long F, double ir) {
  if (d == 0) return v_res64d<D, 0, INTERIOR>(g, L, diag.a[0], ci, F, ir);
  if (d == 1) return v_res64d<D, 1, INTERIOR>(g, L, diag.a[1], ci, F, ir);
  return v_res64d<D, (D == 3 ? 2 : 1), INTERIOR>(g, L, diag.a[D == 3 ? 2 : 1], ci, F, ir);
}

template <int D>
__device__ __forceinline__ void v_residual_mixed_body(const Blk& B, Geo g, LevelPtrs<double> L,
                                                      F32x3 r32, F32x3 e32, Ptr3d diag, double ir,
                                                      double* partial, Ptr3d r64) {
  __shared__ double sh[32];
  int i = B.x * blockDim.x + threadIdx.x;
  int j = B.y * blockDim.y + threadIdx.y;
  int k = B.z * blockDim.z + threadIdx.z;
  double r2 = 0.0;
  if (i < g.n[0] && j < g.n[1] && k < g.n[2]) {
    int ci[3] = {i, j, k};
    long long F = gidx(g, i, j, k);
    bool interior = true;
#pragma unroll
    for (int a = 0; a < D; ++a) interior = interior && ci[a] > 0 && ci[a] < g.n[a] - 1;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      double r = 0.0;
      if (interior) r = v_res_any<D, true>(g, L, diag, d, ci, F, ir);
      else if (g.per[d] || ci[d] != 0) r = v_res_any<D, false>(g, L, diag, d, ci, F, ir);
      r32.a[d][F] = (float)r;
      e32.a[d][F] = 0.0f;
      if (r64.a[0]) r64.a[d][F] = r;
      r2 += r * r;
    }
  }
  if (partial) {
    r2 = block_sum(r2, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0) partial[B.linear()] = r2;
  }
}

template <int D>
__global__ void __launch_bounds__(256, 3) k_v_residual_mixed(Geo g, LevelPtrs<double> L, F32x3 r32,
                                                          F32x3 e32, Ptr3d diag, double ir,
                                                          double* partial, Ptr3d r64) {
  v_residual_mixed_body<D>(own_blk(), g, L, r32, e32, diag, ir, partial, r64);
}

// x += e over the unknowns of ncomp face components (ncomp = 0: cells)
template <int D>
__device__ __forceinline__ void add_correction_body(const Blk& B, Geo g, Ptr3d x, F32x3 e,
                                                    int ncomp) {
  int i = B.x * blockDim.x + threadIdx.x;
  int j = B.y * blockDim.y + threadIdx.y;
  int k = B.z * blockDim.z + threadIdx.z;
  if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) return;
  int ci[3] = {i, j, k};
  long long c = gidx(g, i, j, k);
  if (ncomp == 0) {
    x.a[0][c] += (double)e.a[0][c];
    return;
  }
#pragma unroll
  for (int d = 0; d < 3; ++d)   // compile-time components: no local-memory copies
    if (d < ncomp && (g.per[d] || ci[d] != 0)) x.a[d][c] += (double)e.a[d][c];
}

template <int D>
__global__ void __launch_bounds__(256) k_add_correction(Geo g, Ptr3d x, F32x3 e, int ncomp) {
  add_correction_body<D>(own_blk(), g, x, e, ncomp);
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256) k_convert(const Tin* __restrict__ in, Tout* __restrict__ out,
                                                 long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    out[q] = (Tout)in[q];
}

}  // namespace

// three FP32 arrays to FP64 on every stored element
__global__ void __launch_bounds__(256) k_convert3(F32x3 in, Ptr3d out, long long n) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    for (int d = 0; d < 3; ++d) out.a[d][q] = (double)in.a[d][q];
}

namespace {

struct ConvList {
  const double* in[12];
  float* out[12];
  int n;
};

__global__ void __launch_bounds__(256) k_convert_list(ConvList L, long long elems) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < elems;
       q += (long long)gridDim.x * blockDim.x)
    for (int a = 0; a < L.n; ++a) L.out[a][q] = (float)L.in[a][q];
}

}  // namespace

int red_blocks_3d(int D, const Geo& g) {
  dim3 b = blk3(D);
  dim3 gr = grd3(g.n[0], g.n[1], g.n[2], b);
  return (int)(gr.x * gr.y * gr.z);
}

void launch_p_residual_mixed(int D, const Geo& g, const LevelPtrs<double>& L, float* r32,
                             float* e32, double* partial, cudaStream_t s) {
  dim3 b = blk3(D);
  dim3 gr = grd3(g.n[0], g.n[1], g.n[2], b);
  const double ih2 = 1.0 / (g.h * g.h);
  if (D == 3) k_p_residual_mixed<3><<<gr, b, 0, s>>>(g, L, r32, e32, partial, ih2);
  else k_p_residual_mixed<2><<<gr, b, 0, s>>>(g, L, r32, e32, partial, ih2);
}

void launch_v_residual_mixed(int D, const Geo& g, const LevelPtrs<double>& L, float* const r32[3],
                             float* const e32[3], double* const diag[3], double inv_re,
                             double* partial, cudaStream_t s, double* const r64[3]) {
  dim3 b = blk3(D);
  dim3 gr = grd3(g.n[0], g.n[1], g.n[2], b);
  F32x3 r, e;
  Ptr3d dg, rr;
  for (int d = 0; d < 3; ++d) {
    r.a[d] = r32[d];
    e.a[d] = e32[d];
    dg.a[d] = diag[d];
    rr.a[d] = r64 ? r64[d] : nullptr;
  }
  double ir = inv_re / (g.h * g.h);
  if (D == 3) k_v_residual_mixed<3><<<gr, b, 0, s>>>(g, L, r, e, dg, ir, partial, rr);
  else k_v_residual_mixed<2><<<gr, b, 0, s>>>(g, L, r, e, dg, ir, partial, rr);
}

// ------------------------------------------------------------ flexible CG
// Flexible conjugate gradients for the viscous solve, in FP64 around the
// FP32 V-cycle as preconditioner M (the viscous operator A is symmetric
// positive definite; M is neither symmetric nor fixed, so the update of the
// search direction uses the flexible form, with one previous direction):
//   z = M r,  w = A z,  beta = -(z.q) / (p.q)  (0 at the first iteration),
//   p = z + beta p,  q = w + beta q,  alpha = (p.r) / (p.q),
//   x += alpha p,  r -= alpha q.
// Scalars travel between the kernels in device memory (slots of `out`).
// (z arrives in FP64: converting each FP32 neighbour at every use would put
// about fifteen conversions per face on GB300's small FP64 pipe)
template <int D, int d, bool INTERIOR>
__device__ __forceinline__ double v_apply_z(const Geo& g, const LevelPtrs<double>& L,
                                            const Ptr3d& z, const double* __restrict__ diag,
                                            const int ci[3], long long F, double ir) {
  const double* const vec[3] = {z.a[0], z.a[1], z.a[2]};
  double off = v_off64<D, d, INTERIOR, double>(g, L, vec, ci, F);
  return diag[F] * z.a[d][F] - ir * off;
}

template <int D, bool INTERIOR>
__device__ __forceinline__ double v_apply_any(const Geo& g, const LevelPtrs<double>& L,
                                              const Ptr3d& z, const Ptr3d& diag, int d,
                                              const int ci[3], long long F, double ir) {
  if (d == 0) return v_apply_z<D, 0, INTERIOR>(g, L, z, diag.a[0], ci, F, ir);
  if (d == 1) return v_apply_z<D, 1, INTERIOR>(g, L, z, diag.a[1], ci, F, ir);
  return v_apply_z<D, (D == 3 ? 2 : 1), INTERIOR>(g, L, z, diag.a[D == 3 ? 2 : 1], ci, F, ir);
}

__device__ __forceinline__ bool block_leader() {
  return threadIdx.x == 0 && threadIdx.y == 0 && threadIdx.z == 0;
}

// w = A z on every unknown face (0 on the fixed wall faces); partial sums of z.q.
// GB300's FP64 rate bounds this kernel and the FP64 residual: their launch
// bounds keep 4 and 3 blocks resident per SM (64 and 80 registers) so that
// enough warps hide the FP64 pipe's and the loads' latency. The batched forms
// hold a member's pointers in registers on top and keep 3 at 80 registers:
// their spills (about 110 bytes a thread) cost less than the third block
// gains (1 % of a 64-duct batch step).
template <int D>
__device__ __forceinline__ void fcg_apply_body(const Blk& B, Geo g, LevelPtrs<double> L, Ptr3d z,
                                               Ptr3d diag, double ir, Ptr3d w, Ptr3d q,
                                               double* partial) {
  __shared__ double sh[32];
  int i = B.x * blockDim.x + threadIdx.x;
  int j = B.y * blockDim.y + threadIdx.y;
  int k = B.z * blockDim.z + threadIdx.z;
  double zq = 0.0;
  if (i < g.n[0] && j < g.n[1] && k < g.n[2]) {
    int ci[3] = {i, j, k};
    long long F = gidx(g, i, j, k);
    bool interior = true;
#pragma unroll
    for (int a = 0; a < D; ++a) interior = interior && ci[a] > 0 && ci[a] < g.n[a] - 1;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      double v = 0.0;
      if (interior) v = v_apply_any<D, true>(g, L, z, diag, d, ci, F, ir);
      else if (g.per[d] || ci[d] != 0) v = v_apply_any<D, false>(g, L, z, diag, d, ci, F, ir);
      w.a[d][F] = v;
      zq += z.a[d][F] * q.a[d][F];
    }
  }
  zq = block_sum(zq, sh);
  if (block_leader()) partial[B.linear()] = zq;
}

template <int D>
__global__ void __launch_bounds__(256, 4) k_fcg_apply(Geo g, LevelPtrs<double> L, Ptr3d z,
                                                   Ptr3d diag, double ir, Ptr3d w, Ptr3d q,
                                                   double* partial) {
  fcg_apply_body<D>(own_blk(), g, L, z, diag, ir, w, q, partial);
}

// The direction and update passes touch every stored element of the level
// arrays (pads and fixed wall faces hold 0 in every vector, so they add
// nothing): flat grid-stride loops over pairs of doubles.
constexpr int kFlatBlocks = 1216;   // 8 blocks of 256 threads per SM on 152 SMs

// p = z + beta p, q = w + beta q; partial sums of p.q (first nb) and p.r (next nb)
template <int D>
__device__ __forceinline__ void fcg_dir_body(const Blk& B, long long npair, Ptr3d z, Ptr3d w,
                                             Ptr3d p, Ptr3d q, Ptr3d r,
                                             const double* __restrict__ out, int sl_zq, int sl_pq,
                                             double* partial) {
  __shared__ double sh[32];
  const double pq_old = out[sl_pq];
  // the first direction is z itself: the previous solve's p and q are not read
  const bool first = pq_old == 0.0;
  const double beta = first ? 0.0 : -out[sl_zq] / pq_old;
  double pq = 0.0, pr = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double2* __restrict__ zz = reinterpret_cast<const double2*>(z.a[d]);
    const double2* __restrict__ ww = reinterpret_cast<const double2*>(w.a[d]);
    const double2* __restrict__ rr = reinterpret_cast<const double2*>(r.a[d]);
    double2* pp = reinterpret_cast<double2*>(p.a[d]);
    double2* qq = reinterpret_cast<double2*>(q.a[d]);
    for (long long k = B.x * (long long)blockDim.x + threadIdx.x; k < npair;
         k += (long long)B.gx * blockDim.x) {
      double2 zv = zz[k], wv = ww[k], rv = rr[k], pv = zv, qv = wv;
      if (!first) {
        const double2 po = pp[k], qo = qq[k];
        pv.x += beta * po.x;
        pv.y += beta * po.y;
        qv.x += beta * qo.x;
        qv.y += beta * qo.y;
      }
      pp[k] = pv;
      qq[k] = qv;
      pq += pv.x * qv.x + pv.y * qv.y;
      pr += pv.x * rv.x + pv.y * rv.y;
    }
  }
  pq = block_sum(pq, sh);
  pr = block_sum(pr, sh);
  if (threadIdx.x == 0) {
    partial[B.x] = pq;
    partial[B.gx + B.x] = pr;
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_fcg_dir(long long npair, Ptr3d z, Ptr3d w, Ptr3d p,
                                                 Ptr3d q, Ptr3d r, const double* __restrict__ out,
                                                 int sl_zq, int sl_pq, double* partial) {
  fcg_dir_body<D>(own_blk(), npair, z, w, p, q, r, out, sl_zq, sl_pq, partial);
}

// x += alpha p, r -= alpha q; the new residual as the FP32 right-hand side of
// the next preconditioning (correction zeroed); partial sums of r.r
template <int D>
__device__ __forceinline__ void fcg_update_body(const Blk& B, long long npair, Ptr3d x, Ptr3d p,
                                                Ptr3d q, Ptr3d r, F32x3 r32, F32x3 e32,
                                                const double* __restrict__ out, int sl_pq,
                                                int sl_pr, double* partial) {
  __shared__ double sh[32];
  const double pq = out[sl_pq];
  const double alpha = pq != 0.0 ? out[sl_pr] / pq : 0.0;
  double rs = 0.0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    double2* xx = reinterpret_cast<double2*>(x.a[d]);
    const double2* __restrict__ pp = reinterpret_cast<const double2*>(p.a[d]);
    const double2* __restrict__ qq = reinterpret_cast<const double2*>(q.a[d]);
    double2* rr = reinterpret_cast<double2*>(r.a[d]);
    float2* r2 = reinterpret_cast<float2*>(r32.a[d]);
    float2* e2 = reinterpret_cast<float2*>(e32.a[d]);
    for (long long k = B.x * (long long)blockDim.x + threadIdx.x; k < npair;
         k += (long long)B.gx * blockDim.x) {
      double2 xv = xx[k], pv = pp[k], qv = qq[k], rv = rr[k];
      xv.x += alpha * pv.x;
      xv.y += alpha * pv.y;
      rv.x -= alpha * qv.x;
      rv.y -= alpha * qv.y;
      xx[k] = xv;
      rr[k] = rv;
      r2[k] = make_float2((float)rv.x, (float)rv.y);
      e2[k] = make_float2(0.f, 0.f);
      rs += rv.x * rv.x + rv.y * rv.y;
    }
  }
  rs = block_sum(rs, sh);
  if (threadIdx.x == 0) partial[B.x] = rs;
}

template <int D>
__global__ void __launch_bounds__(256) k_fcg_update(long long npair, Ptr3d x, Ptr3d p, Ptr3d q,
                                                    Ptr3d r, F32x3 r32, F32x3 e32,
                                                    const double* __restrict__ out, int sl_pq,
                                                    int sl_pr, double* partial) {
  fcg_update_body<D>(own_blk(), npair, x, p, q, r, r32, e32, out, sl_pq, sl_pr, partial);
}

namespace {
Ptr3d p3(double* const a[3]) {
  Ptr3d o;
  for (int d = 0; d < 3; ++d) o.a[d] = a[d];
  return o;
}
F32x3 f3(float* const a[3]) {
  F32x3 o;
  for (int d = 0; d < 3; ++d) o.a[d] = a[d];
  return o;
}
}  // namespace

void launch_fcg_apply(int D, const Geo& g, const LevelPtrs<double>& L, double* const z[3],
                      double* const diag[3], double inv_re, double* const w[3],
                      double* const q[3], double* partial, cudaStream_t s) {
  dim3 b = blk3(D);
  dim3 gr = grd3(g.n[0], g.n[1], g.n[2], b);
  double ir = inv_re / (g.h * g.h);
  if (D == 3) k_fcg_apply<3><<<gr, b, 0, s>>>(g, L, p3(z), p3(diag), ir, p3(w), p3(q), partial);
  else k_fcg_apply<2><<<gr, b, 0, s>>>(g, L, p3(z), p3(diag), ir, p3(w), p3(q), partial);
}

// flat loops run over pairs: the level arrays hold an even number of
// elements (rows padded to a multiple of 8) and start on 256-byte boundaries
__host__ __device__ long long flat_elems(const Geo& g) { return g.st[2] * g.s[2]; }

int fcg_flat_blocks(const Geo& g) {
  long long npair = flat_elems(g) / 2;
  long long nb = (npair + 255) / 256;
  return (int)(nb < kFlatBlocks ? (nb < 1 ? 1 : nb) : kFlatBlocks);
}

void launch_fcg_dir(int D, const Geo& g, double* const z[3], double* const w[3], double* const p[3],
                    double* const q[3], double* const r[3], const double* out, int sl_zq,
                    int sl_pq, double* partial, cudaStream_t s) {
  const long long npair = flat_elems(g) / 2;
  const int nb = fcg_flat_blocks(g);
  if (D == 3)
    k_fcg_dir<3><<<nb, 256, 0, s>>>(npair, p3(z), p3(w), p3(p), p3(q), p3(r), out, sl_zq, sl_pq, partial);
  else
    k_fcg_dir<2><<<nb, 256, 0, s>>>(npair, p3(z), p3(w), p3(p), p3(q), p3(r), out, sl_zq, sl_pq, partial);
}

void launch_fcg_update(int D, const Geo& g, double* const x[3], double* const p[3],
                       double* const q[3], double* const r[3], float* const r32[3],
                       float* const e32[3], const double* out, int sl_pq, int sl_pr,
                       double* partial, cudaStream_t s) {
  const long long npair = flat_elems(g) / 2;
  const int nb = fcg_flat_blocks(g);
  if (D == 3)
    k_fcg_update<3><<<nb, 256, 0, s>>>(npair, p3(x), p3(p), p3(q), p3(r), f3(r32), f3(e32), out,
                                       sl_pq, sl_pr, partial);
  else
    k_fcg_update<2><<<nb, 256, 0, s>>>(npair, p3(x), p3(p), p3(q), p3(r), f3(r32), f3(e32), out,
                                       sl_pq, sl_pr, partial);
}

void launch_v_diag(int D, const Geo& g, const LevelPtrs<double>& L, double* const diag[3],
                   double inv_re, cudaStream_t s) {
  dim3 b = blk3(D);
  dim3 gr = grd3(g.n[0], g.n[1], g.n[2], b);
  Ptr3d dg;
  for (int d = 0; d < 3; ++d) dg.a[d] = diag[d];
  double ir = inv_re / (g.h * g.h);
  if (D == 3) k_v_diag<3><<<gr, b, 0, s>>>(g, L, dg, ir);
  else k_v_diag<2><<<gr, b, 0, s>>>(g, L, dg, ir);
}

void launch_add_correction(int D, const Geo& g, double* const x[3], float* const e[3], int ncomp,
                           cudaStream_t s) {
  dim3 b = blk3(D);
  dim3 gr = grd3(g.n[0], g.n[1], g.n[2], b);
  Ptr3d xx;
  F32x3 ee;
  for (int d = 0; d < 3; ++d) {
    xx.a[d] = x[d];
    ee.a[d] = e[d];
  }
  if (D == 3) k_add_correction<3><<<gr, b, 0, s>>>(g, xx, ee, ncomp);
  else k_add_correction<2><<<gr, b, 0, s>>>(g, xx, ee, ncomp);
}

void launch_f32_to_f64(const float* in, double* out, long long n, cudaStream_t s) {
  k_convert<float, double><<<(unsigned)flat_convert_blocks(n), kBlock1D, 0, s>>>(in, out, n);
}

void launch_f32_to_f64_3(float* const in[3], double* const out[3], long long n, cudaStream_t s) {
  F32x3 i;
  Ptr3d o;
  for (int d = 0; d < 3; ++d) {
    i.a[d] = in[d];
    o.a[d] = out[d];
  }
  k_convert3<<<(unsigned)flat_convert_blocks(n), kBlock1D, 0, s>>>(i, o, n);
}

void launch_f64_to_f32(const double* in, float* out, long long n, cudaStream_t s) {
  k_convert<double, float><<<(unsigned)flat_convert_blocks(n), kBlock1D, 0, s>>>(in, out, n);
}

void launch_v_idg32(int D, const Geo& g, const LevelPtrs<double>& L64,
                    const LevelPtrs<float>& L32, double ir, cudaStream_t s) {
  dim3 b = blk3(D);
  dim3 gr = grd3(g.n[0], g.n[1], g.n[2], b);
  F32x3 o;
  for (int d = 0; d < 3; ++d) o.a[d] = L32.idg[d];
  if (D == 3) k_v_idg32<3><<<gr, b, 0, s>>>(g, L64, o, ir);
  else k_v_idg32<2><<<gr, b, 0, s>>>(g, L64, o, ir);
}

void launch_coef_to_f32(int D, const Geo& g, const LevelPtrs<double>& L64,
                        const LevelPtrs<float>& L32, cudaStream_t s) {
  ConvList cl;
  cl.n = 0;
  for (int d = 0; d < D; ++d) {
    cl.in[cl.n] = L64.beta[d];
    cl.out[cl.n++] = L32.beta[d];
    cl.in[cl.n] = L64.m[d];
    cl.out[cl.n++] = L32.m[d];
  }
  cl.in[cl.n] = L64.muc;
  cl.out[cl.n++] = L32.muc;
  for (int e = 0; e < (D == 3 ? 3 : 1); ++e) {
    cl.in[cl.n] = L64.mue[e];
    cl.out[cl.n++] = L32.mue[e];
  }
  long long n = g.st[2] * g.s[2];
  long long nb = (n + kBlock1D - 1) / kBlock1D;
  if (nb > 4096) nb = 4096;
  k_convert_list<<<(unsigned)nb, kBlock1D, 0, s>>>(cl, n);
}

// ------------------------------------------------------------------ batched
// The level-0 FP64 steps of the batched solves: the bodies above over a
// persistent batch's work list, each with a member's own arrays, scalars and
// the block decomposition of its single-instance launch.
__global__ void __launch_bounds__(256, 3) kb_v_residual_mixed(BArgs A, int with_partial, int with_r64) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    const Geo g = M.g[0];
    F32x3 r, e;
    Ptr3d dg, rr;
    for (int d = 0; d < 3; ++d) {
      r.a[d] = M.f[0].uf[d];
      e.a[d] = M.f[0].u[d];
      dg.a[d] = M.vdiag[d];
      rr.a[d] = with_r64 ? M.d[0].ur[d] : nullptr;
    }
    v_residual_mixed_body<3>(B, g, M.d[0], r, e, dg, M.ir[0],
                             with_partial ? M.sc.partial : nullptr, rr);
  });
}

__global__ void __launch_bounds__(256) kb_p_residual_mixed(BArgs A, int with_partial) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    p_residual_mixed_body<3>(B, M.g[0], M.d[0], M.f[0].pf, M.f[0].p,
                             with_partial ? M.sc.partial : nullptr, M.ih2[0]);
  });
}

__global__ void __launch_bounds__(256) kb_add_correction(BArgs A, int viscous) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    Ptr3d x;
    F32x3 e;
    for (int d = 0; d < 3; ++d) {
      x.a[d] = viscous ? M.d[0].u[d] : (d == 0 ? M.d[0].p : nullptr);
      e.a[d] = viscous ? M.f[0].u[d] : (d == 0 ? M.f[0].p : nullptr);
    }
    add_correction_body<3>(B, M.g[0], x, e, viscous ? 3 : 0);
  });
}

// z = the V-cycle's FP32 result in FP64, on every stored element
__global__ void __launch_bounds__(256) kb_z_to_f64(BArgs A) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    const long long n = flat_elems(M.g[0]);
    for (int d = 0; d < 3; ++d) {
      const float* __restrict__ in = M.f[0].u[d];
      double* __restrict__ out = M.cg_z[d];
      for (long long q = B.x * (long long)blockDim.x + threadIdx.x; q < n;
           q += (long long)B.gx * blockDim.x)
        out[q] = (double)in[q];
    }
  });
}

__global__ void __launch_bounds__(256, 3) kb_fcg_apply(BArgs A) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    const Geo g = M.g[0];
    Ptr3d z, dg, w, q;
    for (int d = 0; d < 3; ++d) {
      z.a[d] = M.cg_z[d];
      dg.a[d] = M.vdiag[d];
      w.a[d] = M.d[0].u2[d];
      q.a[d] = M.cg_q[d];
    }
    fcg_apply_body<3>(B, g, M.d[0], z, dg, M.ir[0], w, q, M.sc.partial);
  });
}

__global__ void __launch_bounds__(256) kb_fcg_dir(BArgs A, int sl_zq, int sl_pq) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    Ptr3d z, w, p, q, r;
    for (int d = 0; d < 3; ++d) {
      z.a[d] = M.cg_z[d];
      w.a[d] = M.d[0].u2[d];
      p.a[d] = M.cg_p[d];
      q.a[d] = M.cg_q[d];
      r.a[d] = M.d[0].ur[d];
    }
    fcg_dir_body<3>(B, flat_elems(M.g[0]) / 2, z, w, p, q, r, M.sc.out, sl_zq, sl_pq,
                    M.sc.partial);
  });
}

__global__ void __launch_bounds__(256) kb_fcg_update(BArgs A, int sl_pq, int sl_pr) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    Ptr3d x, p, q, r;
    F32x3 r32, e32;
    for (int d = 0; d < 3; ++d) {
      x.a[d] = M.d[0].u[d];
      p.a[d] = M.cg_p[d];
      q.a[d] = M.cg_q[d];
      r.a[d] = M.d[0].ur[d];
      r32.a[d] = M.f[0].uf[d];
      e32.a[d] = M.f[0].u[d];
    }
    fcg_update_body<3>(B, flat_elems(M.g[0]) / 2, x, p, q, r, r32, e32, M.sc.out, sl_pq, sl_pr,
                       M.sc.partial);
  });
}

int flat_convert_blocks(long long n) {
  long long nb = (n + kBlock1D - 1) / kBlock1D;
  if (nb > 4096) nb = 4096;
  return (int)(nb < 1 ? 1 : nb);
}

void launch_b_v_residual_mixed(const BArgs& A, bool partial, bool r64, int grid, cudaStream_t s) {
  if (A.n > 0) kb_v_residual_mixed<<<grid, blk3(3), 0, s>>>(A, partial ? 1 : 0, r64 ? 1 : 0);
}
void launch_b_p_residual_mixed(const BArgs& A, bool partial, int grid, cudaStream_t s) {
  if (A.n > 0) kb_p_residual_mixed<<<grid, blk3(3), 0, s>>>(A, partial ? 1 : 0);
}
void launch_b_add_correction(const BArgs& A, bool viscous, int grid, cudaStream_t s) {
  if (A.n > 0) kb_add_correction<<<grid, blk3(3), 0, s>>>(A, viscous ? 1 : 0);
}
void launch_b_z_to_f64(const BArgs& A, int grid, cudaStream_t s) {
  if (A.n > 0) kb_z_to_f64<<<grid, kBlock1D, 0, s>>>(A);
}
void launch_b_fcg_apply(const BArgs& A, int grid, cudaStream_t s) {
  if (A.n > 0) kb_fcg_apply<<<grid, blk3(3), 0, s>>>(A);
}
void launch_b_fcg_dir(const BArgs& A, int sl_zq, int sl_pq, int grid, cudaStream_t s) {
  if (A.n > 0) kb_fcg_dir<<<grid, 256, 0, s>>>(A, sl_zq, sl_pq);
}
void launch_b_fcg_update(const BArgs& A, int sl_pq, int sl_pr, int grid, cudaStream_t s) {
  if (A.n > 0) kb_fcg_update<<<grid, 256, 0, s>>>(A, sl_pq, sl_pr);
}

}  // namespace bf
