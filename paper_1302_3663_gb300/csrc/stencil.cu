// Eulerian grid kernels: red-black Gauss-Seidel smoothers, residuals, grid
// transfers and coarse solves of the two multigrid solves (Sec. 3.5), the
// explicit momentum right-hand side (Eq. NSdis1-1), the divergence and the
// projection (Eq. NSdis2 - NSdis4), coefficient hierarchies (Eq.
// ViscCoarseGrid) and deterministic reductions.
//
// Every array of a level shares one layout (see Geo): a wall axis stores one
// extra plane so that the upper wall face/edge has a slot. All stencil
// kernels map one thread to one grid point; the red-black kernels map one
// thread to one point of the colour being updated, so a warp covers 64
// consecutive x positions.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "common.cuh"
#include "point.cuh"

namespace bf {

namespace {

constexpr int kBlock1D = 256;

__host__ __device__ constexpr int edge_id(int d, int e) {
  return (d < e ? d : e) + (d < e ? e : d) - 1;
}

inline dim3 blk3(int D) { return D == 3 ? dim3(32, 4, 2) : dim3(32, 8, 1); }
inline dim3 grd3(long long nx, long long ny, long long nz, dim3 b) {
  return dim3((unsigned)((nx + b.x - 1) / b.x), (unsigned)((ny + b.y - 1) / b.y),
              (unsigned)((nz + b.z - 1) / b.z));
}
// extent of the points a kernel covers along axis a: the cells, plus the
// outflow plane of an open axis when `outflow` (its faces are unknowns)
inline int ext(const Geo& g, int a, bool outflow) {
  return g.n[a] + (outflow && g.open == a ? 1 : 0);
}
inline int red_grid(long long n) {
  long long b = (n + kBlock1D - 1) / kBlock1D;
  return (int)(b < kRedBlocks ? (b > 0 ? b : 1) : kRedBlocks);
}

// offset to the +1 / -1 neighbour along axis a (wrapping on periodic axes;
// on wall axes the caller decides whether the neighbour exists)
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
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
// block-wide sum/max; the result is valid in thread 0
__device__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) v = warp_sum(v);
  __syncthreads();
  return v;
}
__device__ double block_max(double v, double* sh) {
  v = warp_max(v);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) v = warp_max(v);
  __syncthreads();
  return v;
}

// Tests of the open axis written with compile-time indices only: an array
// index taken from g.open (or from a value the compiler knows equals it)
// would put the whole geometry into local memory.
__device__ __forceinline__ bool is_open(const Geo& g, int a) {
  return (a == 0 && g.open == 0) || (a == 1 && g.open == 1) || (a == 2 && g.open == 2);
}
__device__ __forceinline__ long long st_of(const Geo& g, int a) {
  return a == 0 ? g.st[0] : (a == 1 ? g.st[1] : g.st[2]);
}
// a point on the plane beyond the last cells of an open axis other than d
template <int d>
__device__ __forceinline__ bool beyond_outflow(const Geo& g, const int ci[3]) {
  return (d != 0 && g.open == 0 && ci[0] == g.n[0]) || (d != 1 && g.open == 1 && ci[1] == g.n[1]) ||
         (d != 2 && g.open == 2 && ci[2] == g.n[2]);
}
// a cell in the last layer along the open axis
__device__ __forceinline__ bool last_open_cell(const Geo& g, const int ci[3]) {
  return (g.open == 0 && ci[0] == g.n[0] - 1) || (g.open == 1 && ci[1] == g.n[1] - 1) ||
         (g.open == 2 && ci[2] == g.n[2] - 1);
}

// decode a flattened cell index over n[0] x n[1] x n[2]
__device__ __forceinline__ void decode(const Geo& g, long long idx, int& i, int& j, int& k) {
  i = (int)(idx % g.n[0]);
  long long r = idx / g.n[0];
  j = (int)(r % g.n[1]);
  k = (int)(r / g.n[1]);
}

// ---------------------------------------------------------------------------
// Pressure operator D.(beta D p), Eq. (divergenceGrad). num = sum of
// beta_nb p_nb over the existing neighbours, dg = sum of beta_nb; then
// (A p)(c) = (num - dg p(c)) / h^2. No flux crosses a wall.
// ---------------------------------------------------------------------------
template <int D, typename T, bool COH = false>
__device__ __forceinline__ void p_terms(const Geo& g, const LevelPtrs<T>& L, const int ci[3],
                                        long long c, T& num, T& dg) {
  num = T(0);
  dg = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const T* __restrict__ b = L.beta[a];
    if (ci[a] > 0 || g.per[a]) {
      long long cm = c + offm(g, a, ci[a]);
      T bb = b[c];
      num += bb * ldm<COH>(L.p + cm);
      dg += bb;
    }
    if (ci[a] < g.n[a] - 1 || g.per[a]) {
      long long cp = c + offp(g, a, ci[a]);
      T bb = b[cp];
      num += bb * ldm<COH>(L.p + cp);
      dg += bb;
    } else if (is_open(g, a)) {
      // the outflow face, pressure held there: the homogeneous ghost -p
      // (the held value is in the right-hand side)
      dg += T(2) * b[c + st_of(g, a)];
    }
  }
}

template <int D, typename T>
__global__ void __launch_bounds__(256) k_p_rbgs(Geo g, LevelPtrs<T> L, int colour) {
  int ih = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (j >= g.n[1] || k >= g.n[2]) return;
  int i = 2 * ih + ((j + k + colour) & 1);
  if (i >= g.n[0]) return;
  int ci[3] = {i, j, k};
  long long c = gidx(g, i, j, k);
  T num, dg;
  p_terms<D, T>(g, L, ci, c, num, dg);
  T h2 = (T)(g.h * g.h);
  L.p[c] = (num - h2 * L.pf[c]) / dg;
}

// ih2 = (T)(1 / h^2), formed once on the host
template <int D, typename T, bool COH = false>
__device__ __forceinline__ void p_residual_at(const Geo& g, const LevelPtrs<T>& L,
                                              const int ci[3], long long c, T ih2) {
  T num, dg;
  p_terms<D, T, COH>(g, L, ci, c, num, dg);
  L.pr[c] = ldm<COH>(L.pf + c) - (num - dg * ldm<COH>(L.p + c)) * ih2;
}

template <int D, typename T>
__device__ __forceinline__ void p_residual_body(const Blk& B, Geo g, LevelPtrs<T> L, T ih2) {
  int i = B.x * blockDim.x + threadIdx.x;
  int j = B.y * blockDim.y + threadIdx.y;
  int k = B.z * blockDim.z + threadIdx.z;
  if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) return;
  int ci[3] = {i, j, k};
  p_residual_at<D, T>(g, L, ci, gidx(g, i, j, k), ih2);
}

template <int D, typename T>
__global__ void __launch_bounds__(256) k_p_residual(Geo g, LevelPtrs<T> L, T ih2) {
  p_residual_body<D, T>(own_blk(), g, L, ih2);
}

// ---------------------------------------------------------------------------
// Viscous operator for component d at face F (Eq. divergenceGrad +
// Eq. divergencePartial on the staggered grid): tau_dd = 2 mu_c du_d/dx_d at
// the cells beside F, tau_de = mu_de (du_d/dx_e + du_e/dx_d) on the edges
// bounding F. Returns off and dgV with h^2 [div tau]_d = off - dgV u_d(F).
// Beyond a wall along e the tangential u_d takes the mirror ghost -u_d(F),
// which doubles that edge's weight in dgV; u_e on the wall is a stored 0.
// ---------------------------------------------------------------------------
// On the outflow face of an open axis (d = open, index n) du/dn = 0: the face
// beyond mirrors the face n - 1, the cell beyond mirrors the last cell (its
// viscosity) and the tangential components mirror too (du_e/dx_d = 0 there).
// Across the outflow (e = open, last cell) the tangential u_d mirrors evenly:
// that edge contributes its cross term only.
// q: the point's neighbour offsets and wall flags (make_pt), formed once per
// point and shared by the components of a residual.
template <int D, int d, typename T, bool COH = false>
__device__ __forceinline__ void v_terms_q(const Geo& g, const LevelPtrs<T>& L, const int ci[3],
                                          const Pt& q, T& off, T& dgV) {
  const T* __restrict__ ud = L.u[d];
  const int F = q.F;
  const bool outflow = d == g.open && ci[d] == g.n[d];
  const int od_m = q.om[d];
  const int od_p = outflow ? od_m : q.op[d];
  T mcp = outflow ? L.muc[F + od_m] : L.muc[F], mcm = L.muc[F + od_m];
  off = T(2) * (mcp * ldm<COH>(ud + F + od_p) + mcm * ldm<COH>(ud + F + od_m));
  dgV = T(2) * (mcp + mcm);
#pragma unroll
  for (int e = 0; e < D; ++e) {
    if (e == d) continue;
    const T* __restrict__ ue = L.u[e];
    const T* __restrict__ me = L.mue[edge_id(d, e)];
    const bool wp = q.wp[e];
    const bool wm = q.wm[e];
    bool neu = wp && e == g.open;   // beyond the outflow: even ghost, no weight
    const int Ep = F + q.op[e];     // e-face index ci[e] + 1
    T mep = me[Ep], mem = me[F];
    T cp = outflow ? T(0) : ldm<COH>(ue + Ep) - ldm<COH>(ue + Ep + od_m);
    T cm = outflow ? T(0) : ldm<COH>(ue + F) - ldm<COH>(ue + F + od_m);
    T udp = T(0), udm = T(0);
    if (!wp) udp = ldm<COH>(ud + Ep);
    if (!wm) udm = ldm<COH>(ud + F + q.om[e]);
    off += mep * (udp + cp) + mem * (udm - cm);
    dgV += (neu ? T(0) : (wp ? T(2) : T(1))) * mep + (wm ? T(2) : T(1)) * mem;
  }
}

template <int D, int d, typename T, bool COH = false>
__device__ __forceinline__ void v_terms(const Geo& g, const LevelPtrs<T>& L, const int ci[3],
                                        long long F, T& off, T& dgV) {
  Pt q;
  make_pt<D>(g, ci, q);
  v_terms_q<D, d, T, COH>(g, L, ci, q, off, dgV);
}

template <int D, int d, typename T>
__global__ void __launch_bounds__(256) k_v_rbgs(Geo g, LevelPtrs<T> L, int colour, T ir) {
  int ih = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z * blockDim.z + threadIdx.z;
  // the faces of component d: along an open axis d the outflow face n too
  const int e0 = g.n[0] + (d == 0 && g.open == 0), e1 = g.n[1] + (d == 1 && g.open == 1),
            e2 = g.n[2] + (d == 2 && g.open == 2);
  if (j >= e1 || k >= e2) return;
  int i = 2 * ih + ((j + k + colour) & 1);
  if (i >= e0) return;
  int ci[3] = {i, j, k};
  if (!g.per[d] && ci[d] == 0) return;   // wall face
  long long F = gidx(g, i, j, k);
  T off, dgV;
  v_terms<D, d, T>(g, L, ci, F, off, dgV);
  L.u[d][F] = (L.uf[d][F] + ir * off) / (L.m[d][F] + ir * dgV);
}

template <int D, int d, typename T, bool COH = false>
__device__ __forceinline__ void v_residual_point(const Geo& g, const LevelPtrs<T>& L,
                                                 const int ci[3], const Pt& q, T ir) {
  const int F = q.F;
  // the plane beyond the last cells of an open axis holds only its outflow faces
  if (beyond_outflow<d>(g, ci)) return;
  if (!g.per[d] && ci[d] == 0) {
    L.ur[d][F] = T(0);
    return;
  }
  T off, dgV;
  v_terms_q<D, d, T, COH>(g, L, ci, q, off, dgV);
  L.ur[d][F] = ldm<COH>(L.uf[d] + F) - (L.m[d][F] + ir * dgV) * ldm<COH>(L.u[d] + F) + ir * off;
}

template <int D, typename T>
__device__ __forceinline__ void v_residual_body(const Blk& B, Geo g, LevelPtrs<T> L, T ir) {
  int i = B.x * blockDim.x + threadIdx.x;
  int j = B.y * blockDim.y + threadIdx.y;
  int k = B.z * blockDim.z + threadIdx.z;
  if (i >= g.n[0] + (g.open == 0) || j >= g.n[1] + (g.open == 1) || k >= g.n[2] + (g.open == 2))
    return;
  int ci[3] = {i, j, k};
  Pt q;
  make_pt<D>(g, ci, q);
  v_residual_point<D, 0, T>(g, L, ci, q, ir);
  v_residual_point<D, 1, T>(g, L, ci, q, ir);
  if constexpr (D == 3) v_residual_point<D, 2, T>(g, L, ci, q, ir);
}

template <int D, typename T>
__global__ void __launch_bounds__(256) k_v_residual(Geo g, LevelPtrs<T> L, T ir) {
  v_residual_body<D, T>(own_blk(), g, L, ir);
}

// ---------------------------------------------------------------------------
// Grid transfers (Sec. 3.5).
// Cell-centred restriction: mean of the 2^D children. Face restriction along
// its own axis: (1/4, 1/2, 1/4) on the faces 2I-1, 2I, 2I+1; across the other
// axes the mean of the two children. Both zero the coarse iterate.
// ---------------------------------------------------------------------------
template <int D, typename T, bool COH = false>
__device__ __forceinline__ void restrict_cell_at(const Geo& gf, const Geo& gc,
                                                 const T* __restrict__ rf, T* __restrict__ fc,
                                                 T* __restrict__ xc, int I, int J, int K) {
  long long f0 = gidx(gf, 2 * I, 2 * J, D == 3 ? 2 * K : 0);
  long long sy = gf.st[1], sz = gf.st[2];
  T s = ldm<COH>(rf + f0) + ldm<COH>(rf + f0 + 1);
  s += ldm<COH>(rf + f0 + sy);
  s += ldm<COH>(rf + f0 + sy + 1);
  if constexpr (D == 3) {
    s += ldm<COH>(rf + f0 + sz);
    s += ldm<COH>(rf + f0 + sz + 1);
    s += ldm<COH>(rf + f0 + sz + sy);
    s += ldm<COH>(rf + f0 + sz + sy + 1);
  }
  long long c = gidx(gc, I, J, K);
  fc[c] = s * (D == 3 ? T(0.125) : T(0.25));
  xc[c] = T(0);
}

template <int D, typename T>
__device__ __forceinline__ void restrict_cell_body(const Blk& B, Geo gf, Geo gc,
                                                   const T* __restrict__ rf, T* __restrict__ fc,
                                                   T* __restrict__ xc) {
  int I = B.x * blockDim.x + threadIdx.x;
  int J = B.y * blockDim.y + threadIdx.y;
  int K = B.z * blockDim.z + threadIdx.z;
  if (I >= gc.n[0] || J >= gc.n[1] || K >= gc.n[2]) return;
  restrict_cell_at<D, T>(gf, gc, rf, fc, xc, I, J, K);
}

template <int D, typename T>
__global__ void __launch_bounds__(256) k_restrict_cell(Geo gf, Geo gc, const T* __restrict__ rf,
                                                       T* __restrict__ fc, T* __restrict__ xc) {
  restrict_cell_body<D, T>(own_blk(), gf, gc, rf, fc, xc);
}

// one coarse face C (a stored face along d, a cell across it)
template <int D, int d, typename T, bool COH = false>
__device__ __forceinline__ void restrict_face_at(const Geo& gf, const Geo& gc,
                                                 const T* __restrict__ rf, T* __restrict__ fc,
                                                 T* __restrict__ xc, const int C[3]) {
  long long c = gidx(gc, C[0], C[1], C[2]);
  xc[c] = T(0);
  bool wallface = !gc.per[d] && (C[d] == 0 || (C[d] == gc.n[d] && d != gc.open));
  if (wallface) {
    fc[c] = T(0);
    return;
  }
  constexpr int ta = (d == 0) ? 1 : 0;
  constexpr int tb = (D == 3) ? ((d == 2) ? 1 : 2) : -1;
  int nf = gf.n[d];
  int f[3] = {0, 0, 0};
  T s = T(0);
#pragma unroll
  for (int t2 = 0; t2 < (D == 3 ? 2 : 1); ++t2) {
#pragma unroll
    for (int t1 = 0; t1 < 2; ++t1) {
      f[ta] = 2 * C[ta] + t1;
      if constexpr (tb >= 0) f[tb] = 2 * C[tb] + t2;
      T along = T(0);
#pragma unroll
      for (int o = -1; o <= 1; ++o) {
        int q = 2 * C[d] + o;
        if (gf.per[d]) q = q < 0 ? q + nf : (q >= nf ? q - nf : q);
        if (d == gf.open && q > nf) q = nf - 1;   // even ghost beyond the outflow
        f[d] = q;
        T w = (o == 0) ? T(0.5) : T(0.25);
        along += w * ldm<COH>(rf + gidx(gf, f[0], f[1], f[2]));
      }
      s += along;
    }
  }
  fc[c] = s * (D == 3 ? T(0.25) : T(0.5));
}

template <int D, int d, typename T>
__device__ __forceinline__ void restrict_face_body(const Blk& B, Geo gf, Geo gc,
                                                   const T* __restrict__ rf, T* __restrict__ fc,
                                                   T* __restrict__ xc) {
  int C[3];
  C[0] = B.x * blockDim.x + threadIdx.x;
  C[1] = B.y * blockDim.y + threadIdx.y;
  C[2] = B.z * blockDim.z + threadIdx.z;
  // along d cover the stored faces (walls included), across d the cells
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int lim = (a == d && a < D) ? gc.s[a] : gc.n[a];
    if (C[a] >= lim) return;
  }
  restrict_face_at<D, d, T>(gf, gc, rf, fc, xc, C);
}

template <int D, int d, typename T>
__global__ void __launch_bounds__(256) k_restrict_face(Geo gf, Geo gc, const T* __restrict__ rf,
                                                       T* __restrict__ fc, T* __restrict__ xc) {
  restrict_face_body<D, d, T>(own_blk(), gf, gc, rf, fc, xc);
}

template <typename T>
struct Faces3 {
  T* a[3];
};

// the three components in one pass over the coarse level's stored extent (3D)
template <typename T>
__device__ __forceinline__ void restrict_face3_body(const Blk& B, const Geo& gf, const Geo& gc,
                                                    const Faces3<T>& rf, const Faces3<T>& fc,
                                                    const Faces3<T>& xc) {
  const int C[3] = {(int)(B.x * blockDim.x + threadIdx.x), (int)(B.y * blockDim.y + threadIdx.y),
                    (int)(B.z * blockDim.z + threadIdx.z)};
  if (C[0] < gc.s[0] && C[1] < gc.n[1] && C[2] < gc.n[2])
    restrict_face_at<3, 0, T>(gf, gc, rf.a[0], fc.a[0], xc.a[0], C);
  if (C[0] < gc.n[0] && C[1] < gc.s[1] && C[2] < gc.n[2])
    restrict_face_at<3, 1, T>(gf, gc, rf.a[1], fc.a[1], xc.a[1], C);
  if (C[0] < gc.n[0] && C[1] < gc.n[1] && C[2] < gc.s[2])
    restrict_face_at<3, 2, T>(gf, gc, rf.a[2], fc.a[2], xc.a[2], C);
}

template <typename T>
__global__ void __launch_bounds__(256) k_restrict_face3(Geo gf, Geo gc, Faces3<T> rf, Faces3<T> fc,
                                                        Faces3<T> xc) {
  restrict_face3_body<T>(own_blk(), gf, gc, rf, fc, xc);
}

// 1D prolongation weights. Cell-centred axis: 3/4 on the parent, 1/4 on the
// next coarse cell toward the child; beyond a wall the mirror ghost
// (sign `mirror`) folds that 1/4 into the parent. Face axis: the coincident
// coarse face, or the mean of the two coarse faces around a midway face.
// The weights are exact binary fractions in any precision.
template <typename T>
__device__ __forceinline__ int prol_cell_1d(int i, int nc, int per, int mirror_lo, int mirror_hi,
                                            int idx[2], T w[2]) {
  int I = i >> 1;
  int J = I + ((i & 1) ? 1 : -1);
  idx[0] = I;
  w[0] = T(0.75);
  w[1] = T(0);
  if (per) {
    idx[1] = J < 0 ? J + nc : (J >= nc ? J - nc : J);
    w[1] = T(0.25);
    return 2;
  }
  if (J < 0 || J >= nc) {
    const int mirror = J < 0 ? mirror_lo : mirror_hi;
    w[0] = mirror > 0 ? T(1) : T(0.5);
    idx[1] = I;   // weight 0: any valid index
    return 1;
  }
  idx[1] = J;
  w[1] = T(0.25);
  return 2;
}
template <typename T>
__device__ __forceinline__ int prol_face_1d(int i, int nc, int per, int idx[2], T w[2]) {
  int I = i >> 1;
  w[1] = T(0);
  if ((i & 1) == 0) {
    idx[0] = I;   // a fine face index is below 2 nc, so I < nc
    idx[1] = I;   // weight 0: any valid index
    w[0] = T(1);
    return 1;
  }
  idx[0] = I;
  w[0] = T(0.5);
  idx[1] = (per && I + 1 == nc) ? 0 : I + 1;
  w[1] = T(0.5);
  return 2;
}

// Roundings of the prolongation written out, so that every form of it (one
// point per thread, two points per thread, the coarse-level cluster kernel)
// gives the same bits whatever the compiler would contract.
__device__ __forceinline__ float pmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double pmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float pfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double pfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float padd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double padd(double a, double b) { return __dadd_rn(a, b); }

// separable tensor-product sum: x-rows first, then y, then z, each pair of
// terms as w1 t1 + (w0 t0) with one rounding of the product and one of the
// fused sum. Every axis takes two terms; a missing term has weight 0 and a
// valid index, and adding its exact zero leaves the sum unchanged, so the
// loops unroll fully and the index and weight arrays stay in registers.
template <typename T, bool COH = false>
__device__ __forceinline__ T prol_sum(const Geo& gc, const T* __restrict__ ec, const int idx[3][2],
                                      const T w[3][2]) {
  T col[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    T row[2];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      long long r = gidx(gc, 0, idx[1][b], idx[2][c]);
      row[b] = pfma(w[0][1], ldm<COH>(ec + r + idx[0][1]), pmul(w[0][0], ldm<COH>(ec + r + idx[0][0])));
    }
    col[c] = pfma(w[1][1], row[1], pmul(w[1][0], row[0]));
  }
  return pfma(w[2][1], col[1], pmul(w[2][0], col[0]));
}

// the coarse correction added at one fine cell fi
template <int D, typename T, bool COH = false>
__device__ __forceinline__ void prolong_cell_at(const Geo& gf, const Geo& gc,
                                                const T* __restrict__ ec, T* __restrict__ xf,
                                                const int fi[3]) {
  int idx[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  T w[3][2] = {{T(1), T(0)}, {T(1), T(0)}, {T(1), T(0)}};
  // the pressure correction mirrors evenly at walls and the inflow, oddly at
  // the outflow, where the pressure is held
#pragma unroll
  for (int a = 0; a < D; ++a)
    prol_cell_1d<T>(fi[a], gc.n[a], gc.per[a], +1, a == gc.open ? -1 : +1, idx[a], w[a]);
  const long long x = gidx(gf, fi[0], fi[1], fi[2]);
  xf[x] = padd(ldm<COH>(xf + x), prol_sum<T, COH>(gc, ec, idx, w));
}

template <int D, typename T>
__device__ __forceinline__ void prolong_cell_body(const Blk& B, Geo gf, Geo gc,
                                                  const T* __restrict__ ec, T* __restrict__ xf) {
  int fi[3];
  fi[0] = B.x * blockDim.x + threadIdx.x;
  fi[1] = B.y * blockDim.y + threadIdx.y;
  fi[2] = B.z * blockDim.z + threadIdx.z;
  if (fi[0] >= gf.n[0] || fi[1] >= gf.n[1] || fi[2] >= gf.n[2]) return;
  prolong_cell_at<D, T>(gf, gc, ec, xf, fi);
}

template <int D, typename T>
__global__ void __launch_bounds__(256) k_prolong_cell(Geo gf, Geo gc, const T* __restrict__ ec,
                                                      T* __restrict__ xf) {
  prolong_cell_body<D, T>(own_blk(), gf, gc, ec, xf);
}

// the coarse correction added at one fine face fi of component d (not a wall face)
template <int D, int d, typename T, bool COH = false>
__device__ __forceinline__ void prolong_face_at(const Geo& gf, const Geo& gc,
                                                const T* __restrict__ ec, T* __restrict__ xf,
                                                const int fi[3]) {
  int idx[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  T w[3][2] = {{T(1), T(0)}, {T(1), T(0)}, {T(1), T(0)}};
#pragma unroll
  for (int a = 0; a < D; ++a) {
    if (a == d)
      prol_face_1d<T>(fi[a], gc.n[a], gc.per[a], idx[a], w[a]);
    else   // tangential velocity: odd at walls and the inflow, even beyond the outflow
      prol_cell_1d<T>(fi[a], gc.n[a], gc.per[a], -1, a == gc.open ? +1 : -1, idx[a], w[a]);
  }
  const long long x = gidx(gf, fi[0], fi[1], fi[2]);
  xf[x] = padd(ldm<COH>(xf + x), prol_sum<T, COH>(gc, ec, idx, w));
}

template <int D, int d, typename T>
__device__ __forceinline__ void prolong_face_body(const Blk& B, Geo gf, Geo gc,
                                                  const T* __restrict__ ec, T* __restrict__ xf) {
  int fi[3];
  fi[0] = B.x * blockDim.x + threadIdx.x;
  fi[1] = B.y * blockDim.y + threadIdx.y;
  fi[2] = B.z * blockDim.z + threadIdx.z;
  // along an open axis d the outflow face n is an unknown too
  if (fi[0] >= gf.n[0] + (d == 0 && gf.open == 0) || fi[1] >= gf.n[1] + (d == 1 && gf.open == 1) ||
      fi[2] >= gf.n[2] + (d == 2 && gf.open == 2))
    return;
  if (!gf.per[d] && fi[d] == 0) return;
  prolong_face_at<D, d, T>(gf, gc, ec, xf, fi);
}

template <int D, int d, typename T>
__global__ void __launch_bounds__(256) k_prolong_face(Geo gf, Geo gc, const T* __restrict__ ec,
                                                      T* __restrict__ xf) {
  prolong_face_body<D, d, T>(own_blk(), gf, gc, ec, xf);
}

// the three components in one pass over the fine cells (3D, no open axis).
// Each axis's 1D weights and indices are formed once per cell, by the cell
// rule (a tangential axis, odd mirror at walls) and by the face rule (the
// component's own axis), and shared by the components; the sums are those of
// prolong_face_at, term for term.
template <typename T>
__device__ __forceinline__ void prolong_face3_body(const Blk& B, const Geo& gf, const Geo& gc,
                                                   const Faces3<T>& ec, const Faces3<T>& xf) {
  const int fi[3] = {(int)(B.x * blockDim.x + threadIdx.x), (int)(B.y * blockDim.y + threadIdx.y),
                     (int)(B.z * blockDim.z + threadIdx.z)};
  if (fi[0] >= gf.n[0] || fi[1] >= gf.n[1] || fi[2] >= gf.n[2]) return;
  int cidx[3][2], fidx[3][2];
  T cw[3][2], fw[3][2];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    prol_cell_1d<T>(fi[a], gc.n[a], gc.per[a], -1, -1, cidx[a], cw[a]);
    prol_face_1d<T>(fi[a], gc.n[a], gc.per[a], fidx[a], fw[a]);
  }
  const long long x = gidx(gf, fi[0], fi[1], fi[2]);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    if (!gf.per[d] && fi[d] == 0) continue;   // the wall face
    int idx[3][2];
    T w[3][2];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        idx[a][t] = a == d ? fidx[a][t] : cidx[a][t];
        w[a][t] = a == d ? fw[a][t] : cw[a][t];
      }
    xf.a[d][x] = padd(xf.a[d][x], prol_sum<T>(gc, ec.a[d], idx, w));
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_face3(Geo gf, Geo gc, Faces3<T> ec, Faces3<T> xf) {
  prolong_face3_body<T>(own_blk(), gf, gc, ec, xf);
}

// The same corrections, two fine points along x per thread: cells or faces
// 2I and 2I + 1 share the coarse x index I and every y and z index and
// weight, so each coarse row is addressed once and its value at I loaded once
// for both; each point's sum is prol_sum's, term for term. The fine x extent
// is even (twice the coarse one).
template <typename T>
__device__ __forceinline__ void prol_pair_sum(const Geo& gc, const T* __restrict__ e, int I,
                                              const int xa[2], const T wa[2], const int xb[2],
                                              const T wb[2], const int iy[2], const T wy[2],
                                              const int iz[2], const T wz[2], T& va, T& vb) {
  T cola[2], colb[2];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    T rowa[2], rowb[2];
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const T* __restrict__ r = e + gidx(gc, 0, iy[b], iz[c]);
      const T e0 = r[I];   // xa[0] == xb[0] == I
      rowa[b] = pfma(wa[1], r[xa[1]], pmul(wa[0], e0));
      rowb[b] = pfma(wb[1], r[xb[1]], pmul(wb[0], e0));
    }
    cola[c] = pfma(wy[1], rowa[1], pmul(wy[0], rowa[0]));
    colb[c] = pfma(wy[1], rowb[1], pmul(wy[0], rowb[0]));
  }
  va = pfma(wz[1], cola[1], pmul(wz[0], cola[0]));
  vb = pfma(wz[1], colb[1], pmul(wz[0], colb[0]));
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_face3_pair(Geo gf, Geo gc, Faces3<T> ec,
                                                           Faces3<T> xf) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z * blockDim.z + threadIdx.z;
  const int i0 = 2 * I;
  if (i0 >= gf.n[0] || j >= gf.n[1] || k >= gf.n[2]) return;
  // per axis the cell-centred and the face weights (x: both points)
  int cxa[2], cxb[2], fxa[2], fxb[2], cy[2], fy[2], cz[2], fz[2];
  T wcxa[2], wcxb[2], wfxa[2], wfxb[2], wcy[2], wfy[2], wcz[2], wfz[2];
  prol_cell_1d<T>(i0, gc.n[0], gc.per[0], -1, -1, cxa, wcxa);
  prol_cell_1d<T>(i0 + 1, gc.n[0], gc.per[0], -1, -1, cxb, wcxb);
  prol_face_1d<T>(i0, gc.n[0], gc.per[0], fxa, wfxa);
  prol_face_1d<T>(i0 + 1, gc.n[0], gc.per[0], fxb, wfxb);
  prol_cell_1d<T>(j, gc.n[1], gc.per[1], -1, -1, cy, wcy);
  prol_face_1d<T>(j, gc.n[1], gc.per[1], fy, wfy);
  prol_cell_1d<T>(k, gc.n[2], gc.per[2], -1, -1, cz, wcz);
  prol_face_1d<T>(k, gc.n[2], gc.per[2], fz, wfz);
  const long long x = gidx(gf, i0, j, k);
  T va, vb;
  // x-faces: the wall face 0 (the first point of the first pair) is fixed
  prol_pair_sum<T>(gc, ec.a[0], I, fxa, wfxa, fxb, wfxb, cy, wcy, cz, wcz, va, vb);
  if (gf.per[0] || i0 != 0) xf.a[0][x] = padd(xf.a[0][x], va);
  xf.a[0][x + 1] = padd(xf.a[0][x + 1], vb);
  if (gf.per[1] || j != 0) {   // y-faces
    prol_pair_sum<T>(gc, ec.a[1], I, cxa, wcxa, cxb, wcxb, fy, wfy, cz, wcz, va, vb);
    xf.a[1][x] = padd(xf.a[1][x], va);
    xf.a[1][x + 1] = padd(xf.a[1][x + 1], vb);
  }
  if (gf.per[2] || k != 0) {   // z-faces
    prol_pair_sum<T>(gc, ec.a[2], I, cxa, wcxa, cxb, wcxb, cy, wcy, fz, wfz, va, vb);
    xf.a[2][x] = padd(xf.a[2][x], va);
    xf.a[2][x + 1] = padd(xf.a[2][x + 1], vb);
  }
}

// ---------------------------------------------------------------------------
// Coarsest level: one block does the whole solve (the grid holds at most a
// few thousand points and stays in L2). Colour phases are separated by
// block barriers.
// ---------------------------------------------------------------------------
// The coarsest level's arrays are copied to shared memory when they fit
// (nel elements each); the sweeps then run on the copies.
constexpr size_t kCoarseSmemMax = 160 * 1024;
__host__ __device__ inline size_t coarse_bytes(int D, const Geo& g, int elem, bool viscous) {
  long long nel = g.st[2] * g.s[2];
  int narr = viscous ? 3 * D + 1 + (D == 3 ? 3 : 1) : 2 + D;
  return (size_t)narr * nel * elem;
}
template <typename T>
__device__ __forceinline__ void stage_in(T* dst, const T* src, long long nel) {
  for (long long q = threadIdx.x; q < nel; q += blockDim.x) dst[q] = src[q];
}
template <typename T>
__device__ __forceinline__ void stage_out(T* dst, const T* src, long long nel) {
  for (long long q = threadIdx.x; q < nel; q += blockDim.x) dst[q] = src[q];
}

template <int D, typename T>
__device__ __forceinline__ void coarse_p_body(const Blk& B, Geo g, LevelPtrs<T> Lg, int sweeps,
                                              long long nel, int use_smem) {
  extern __shared__ __align__(16) unsigned char csm[];
  __shared__ double sh[32];
  LevelPtrs<T> L = Lg;
  if (use_smem) {
    T* b = reinterpret_cast<T*>(csm);
    L.p = b;
    L.pf = b + nel;
    stage_in(L.p, Lg.p, nel);
    stage_in(L.pf, Lg.pf, nel);
    for (int a = 0; a < D; ++a) {
      L.beta[a] = b + (2 + a) * nel;
      stage_in(L.beta[a], Lg.beta[a], nel);
    }
    __syncthreads();
  }
  long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  if (g.open < 0) {   // the singular problem needs a zero-mean right-hand side
    double s = 0.0;
    for (long long q = threadIdx.x; q < ncell; q += blockDim.x) {
      int i, j, k;
      decode(g, q, i, j, k);
      s += (double)L.pf[gidx(g, i, j, k)];
    }
    s = block_sum(s, sh);
    __shared__ double mean;
    if (threadIdx.x == 0) mean = s / (double)ncell;
    __syncthreads();
    for (long long q = threadIdx.x; q < ncell; q += blockDim.x) {
      int i, j, k;
      decode(g, q, i, j, k);
      L.pf[gidx(g, i, j, k)] -= (T)mean;
    }
    __syncthreads();
  }
  int nh = (g.n[0] + 1) >> 1;
  long long npts = (long long)nh * g.n[1] * g.n[2];
  T h2 = (T)(g.h * g.h);
  for (int it = 0; it < sweeps; ++it) {
    for (int colour = 0; colour < 2; ++colour) {
      for (long long q = threadIdx.x; q < npts; q += blockDim.x) {
        int ih = (int)(q % nh);
        long long r = q / nh;
        int j = (int)(r % g.n[1]);
        int k = (int)(r / g.n[1]);
        int i = 2 * ih + ((j + k + colour) & 1);
        if (i >= g.n[0]) continue;
        int ci[3] = {i, j, k};
        long long c = gidx(g, i, j, k);
        T num, dg;
        p_terms<D, T>(g, L, ci, c, num, dg);
        L.p[c] = (num - h2 * L.pf[c]) / dg;
      }
      __syncthreads();
    }
  }
  if (use_smem) {
    stage_out(Lg.p, L.p, nel);
    stage_out(Lg.pf, L.pf, nel);
  }
}

template <int D, typename T>
__global__ void __launch_bounds__(1024) k_coarse_p(Geo g, LevelPtrs<T> Lg, int sweeps,
                                                   long long nel, int use_smem) {
  coarse_p_body<D, T>(own_blk(), g, Lg, sweeps, nel, use_smem);
}

// One colour of component d on the coarsest grid. INV: L.m[d] holds the
// inverse of the whole diagonal (formed once per solve in shared memory), so
// the update multiplies instead of forming the diagonal and dividing.
template <int D, int d, typename T, bool INV>
__device__ __forceinline__ void coarse_v_phase(const Geo& g, const LevelPtrs<T>& L, int colour,
                                               T ir) {
  // the faces of component d (the outflow face too along an open axis d)
  const int e0 = g.n[0] + (d == 0 && g.open == 0), e1 = g.n[1] + (d == 1 && g.open == 1),
            e2 = g.n[2] + (d == 2 && g.open == 2);
  const int nh = (e0 + 1) >> 1;
  const int npts = nh * e1 * e2;   // a few thousand at most on the coarsest grid
  for (int q = threadIdx.x; q < npts; q += blockDim.x) {
    int ih = q % nh;
    int r = q / nh;
    int j = r % e1;
    int k = r / e1;
    int i = 2 * ih + ((j + k + colour) & 1);
    if (i >= e0) continue;
    int ci[3] = {i, j, k};
    if (!g.per[d] && ci[d] == 0) continue;
    long long F = gidx(g, i, j, k);
    T off, dgV;
    v_terms<D, d, T>(g, L, ci, F, off, dgV);
    if constexpr (INV) L.u[d][F] = (L.uf[d][F] + ir * off) * L.m[d][F];
    else L.u[d][F] = (L.uf[d][F] + ir * off) / (L.m[d][F] + ir * dgV);
  }
  __syncthreads();
}

// m_d -> 1 / (m_d + ir dgV) in place on the staged copy (each point reads
// only its own m_d)
template <int D, int d, typename T>
__device__ __forceinline__ void coarse_v_invert(const Geo& g, const LevelPtrs<T>& L, T ir) {
  const int e0 = g.n[0] + (d == 0 && g.open == 0), e1 = g.n[1] + (d == 1 && g.open == 1),
            e2 = g.n[2] + (d == 2 && g.open == 2);
  const int ncell = e0 * e1 * e2;
  for (int q = threadIdx.x; q < ncell; q += blockDim.x) {
    int i = q % e0;
    int r = q / e0;
    int j = r % e1;
    int k = r / e1;
    int ci[3] = {i, j, k};
    if (!g.per[d] && ci[d] == 0) continue;
    long long F = gidx(g, i, j, k);
    T off, dgV;
    v_terms<D, d, T>(g, L, ci, F, off, dgV);
    L.m[d][F] = T(1) / (L.m[d][F] + ir * dgV);
  }
}

template <int D, typename T>
__device__ __forceinline__ void coarse_v_body(const Blk& B, Geo g, LevelPtrs<T> Lg, int sweeps,
                                              T ir, long long nel, int use_smem) {
  extern __shared__ __align__(16) unsigned char csm[];
  LevelPtrs<T> L = Lg;
  if (use_smem) {
    T* b = reinterpret_cast<T*>(csm);
    int q = 0;
    for (int d = 0; d < D; ++d) {
      L.u[d] = b + (q++) * nel;
      stage_in(L.u[d], Lg.u[d], nel);
      L.uf[d] = b + (q++) * nel;
      stage_in(L.uf[d], Lg.uf[d], nel);
      L.m[d] = b + (q++) * nel;
      stage_in(L.m[d], Lg.m[d], nel);
    }
    L.muc = b + (q++) * nel;
    stage_in(L.muc, Lg.muc, nel);
    for (int e = 0; e < (D == 3 ? 3 : 1); ++e) {
      L.mue[e] = b + (q++) * nel;
      stage_in(L.mue[e], Lg.mue[e], nel);
    }
    __syncthreads();
    // the coefficients are fixed through the solve: invert each diagonal once
    coarse_v_invert<D, 0, T>(g, L, ir);
    coarse_v_invert<D, 1, T>(g, L, ir);
    if constexpr (D == 3) coarse_v_invert<D, 2, T>(g, L, ir);
    __syncthreads();
    for (int it = 0; it < sweeps; ++it) {
      coarse_v_phase<D, 0, T, true>(g, L, 0, ir);
      coarse_v_phase<D, 0, T, true>(g, L, 1, ir);
      coarse_v_phase<D, 1, T, true>(g, L, 0, ir);
      coarse_v_phase<D, 1, T, true>(g, L, 1, ir);
      if constexpr (D == 3) {
        coarse_v_phase<D, 2, T, true>(g, L, 0, ir);
        coarse_v_phase<D, 2, T, true>(g, L, 1, ir);
      }
    }
    for (int d = 0; d < D; ++d) stage_out(Lg.u[d], L.u[d], nel);
    return;
  }
  for (int it = 0; it < sweeps; ++it) {
    coarse_v_phase<D, 0, T, false>(g, L, 0, ir);
    coarse_v_phase<D, 0, T, false>(g, L, 1, ir);
    coarse_v_phase<D, 1, T, false>(g, L, 0, ir);
    coarse_v_phase<D, 1, T, false>(g, L, 1, ir);
    if constexpr (D == 3) {
      coarse_v_phase<D, 2, T, false>(g, L, 0, ir);
      coarse_v_phase<D, 2, T, false>(g, L, 1, ir);
    }
  }
}

template <int D, typename T>
__global__ void __launch_bounds__(1024) k_coarse_v(Geo g, LevelPtrs<T> Lg, int sweeps, T ir,
                                                   long long nel, int use_smem) {
  coarse_v_body<D, T>(own_blk(), g, Lg, sweeps, ir, nel, use_smem);
}

// ---------------------------------------------------------------------------
// Coefficients: beta = 1/rho and m = rho sigma/dt on every stored fine face;
// coarse levels average the fine faces on each coarse face, and the fine
// points on each coarse centre/edge for mu, scaled by gamma (Eq.
// ViscCoarseGrid).
// ---------------------------------------------------------------------------
struct Ptr3 {
  double* a[3];
};

__global__ void __launch_bounds__(256) k_coef_fine(Geo g, int D, Ptr3 rho, Ptr3 beta, Ptr3 m,
                                                   double msc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= g.s[0] || j >= g.s[1] || k >= g.s[2]) return;
  long long c = gidx(g, i, j, k);
  for (int d = 0; d < D; ++d) {
    double r = rho.a[d][c];
    beta.a[d][c] = r != 0.0 ? 1.0 / r : 0.0;
    m.a[d][c] = r * msc;
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_coef_restrict(Geo gf, Geo gc, LevelPtrs<double> F,
                                                       LevelPtrs<double> Cc, double gamma) {
  int C[3];
  C[0] = blockIdx.x * blockDim.x + threadIdx.x;
  C[1] = blockIdx.y * blockDim.y + threadIdx.y;
  C[2] = blockIdx.z * blockDim.z + threadIdx.z;
  if (C[0] >= gc.s[0] || C[1] >= gc.s[1] || C[2] >= gc.s[2]) return;
  long long c = gidx(gc, C[0], C[1], C[2]);
  // faces
#pragma unroll
  for (int d = 0; d < D; ++d) {
    bool ok = true;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      if (a == d) {
        if (C[a] > (gc.per[a] ? gc.n[a] - 1 : gc.n[a])) ok = false;
      } else if (C[a] >= gc.n[a]) {
        ok = false;
      }
    }
    double sb = 0.0, sm = 0.0;
    if (ok) {
      for (int z = 0; z < (D == 3 ? 2 : 1); ++z)
        for (int y = 0; y < 2; ++y)
          for (int x = 0; x < 2; ++x) {
            int off[3] = {x, y, z};
            if (off[d] != 0) continue;
            long long f = gidx(gf, 2 * C[0] + x, 2 * C[1] + y, D == 3 ? 2 * C[2] + z : 0);
            sb += F.beta[d][f];
            sm += F.m[d][f];
          }
    }
    double wt = (D == 3) ? 0.25 : 0.5;
    Cc.beta[d][c] = ok ? sb * wt : 0.0;
    Cc.m[d][c] = ok ? sm * wt : 0.0;
  }
  // centres
  {
    bool ok = C[0] < gc.n[0] && C[1] < gc.n[1] && C[2] < gc.n[2];
    if (ok) {
      long long f0 = gidx(gf, 2 * C[0], 2 * C[1], D == 3 ? 2 * C[2] : 0);
      long long sy = gf.st[1], sz = gf.st[2];
      double s = F.muc[f0] + F.muc[f0 + 1];
      s += F.muc[f0 + sy];
      s += F.muc[f0 + sy + 1];
      if (D == 3) {
        s += F.muc[f0 + sz];
        s += F.muc[f0 + sz + 1];
        s += F.muc[f0 + sz + sy];
        s += F.muc[f0 + sz + sy + 1];
      }
      Cc.muc[c] = (s * (D == 3 ? 0.125 : 0.25)) * gamma;
    } else {
      Cc.muc[c] = 0.0;
    }
  }
  // edges
#pragma unroll
  for (int d = 0; d < D; ++d)
#pragma unroll
    for (int e = d + 1; e < D; ++e) {
      int t = 3 - d - e;
      bool ok = true;
#pragma unroll
      for (int a = 0; a < D; ++a) {
        int lim = (a == d || a == e) ? (gc.per[a] ? gc.n[a] - 1 : gc.n[a]) : gc.n[a] - 1;
        if (C[a] > lim) ok = false;
      }
      double v = 0.0;
      if (ok) {
        int f[3] = {2 * C[0], 2 * C[1], D == 3 ? 2 * C[2] : 0};
        if (D == 3) {
          double s = 0.0;
          for (int q = 0; q < 2; ++q) {
            int gi[3] = {f[0], f[1], f[2]};
            gi[t] = 2 * C[t] + q;
            s += F.mue[edge_id(d, e)][gidx(gf, gi[0], gi[1], gi[2])];
          }
          v = gamma * (s * 0.5);
        } else {
          v = gamma * (F.mue[edge_id(d, e)][gidx(gf, f[0], f[1], f[2])] * 1.0);
        }
      }
      Cc.mue[edge_id(d, e)][c] = v;
    }
}

// ---------------------------------------------------------------------------
// Momentum right-hand side, Eq. (NSdis1-1):
//   rhs_d = m_d u_d - rho_d Adv_d(u) + c_f f_d + G [d = flow axis]
// Adv_d = 1/2 (u.D u_d + D.(u u_d)) in the staggered skew form that keeps the
// property of the paper's D0 form, sum over faces of u_d Adv_d = 0: along each
// axis e the advecting velocity U_e is a 2-point mean at the two flux points
// of the face (cell centres for e = d, edges otherwise), and the mean of the
// conservative half (fluxes U_e x 2-point mean of u_d) and the advective half
// (mean of U_e x one-sided differences) collapses to
//   Adv_d = sum_e (U_e+ u_d(F + e) - U_e- u_d(F - e)) / (2h).
// The iterate u~ starts from u^n.
// ---------------------------------------------------------------------------
// U_e = s / 2 with s a sum of two values, so each term is s u / (4h): one
// product per point (FP64 throughput is scarce).
template <int D, int d>
__device__ __forceinline__ void adv_rhs_point(const Geo& g, const Ptr3& uv, const Ptr3& rho,
                                              const Ptr3& frc, const LevelPtrs<double>& L0,
                                              const int ci[3], long long F, double c_force,
                                              double gflow, double c4) {
  if (!g.per[d] && ci[d] == 0) {   // not an unknown: 0 on a wall, the inflow on an open axis
    L0.uf[d][F] = 0.0;
    L0.u[d][F] = d == g.open ? uv.a[d][F] : 0.0;
    return;
  }
  // the plane beyond the last cells of an open axis holds only its outflow faces
  if (beyond_outflow<d>(g, ci)) return;
  const double* __restrict__ ud = uv.a[d];
  // on the outflow face everything beyond mirrors evenly (du/dn = 0)
  const bool outflow = d == g.open && ci[d] == g.n[d];
  long long od_m = offm(g, d, ci[d]), od_p = outflow ? od_m : offp(g, d, ci[d]);
  long long oc = outflow ? od_m : 0;   // the cell beyond the outflow is the last cell
  double udF = ud[F], udp = ud[F + od_p], udm = ud[F + od_m];
  // 4 h Adv_d, one axis at a time
  double a4 = (udF + udp) * udp - (udm + udF) * udm;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    if (e == d) continue;
    const double* __restrict__ ue = uv.a[e];
    bool pe = g.per[e] != 0;
    long long oe_p = offp(g, e, ci[e]);
    double up = -udF, um = -udF;   // mirror ghosts beyond a wall (U_e = 0 there)
    if (pe || ci[e] != g.n[e] - 1) up = ud[F + oe_p];
    else if (e == g.open) up = udF;   // beyond the outflow: even ghost
    if (pe || ci[e] != 0) um = ud[F + offm(g, e, ci[e])];
    double s_lo = ue[F + od_m] + ue[F + oc];                 // 2 x u_e on the lower edge
    double s_hi = ue[F + oe_p + od_m] + ue[F + oe_p + oc];   // 2 x u_e on the upper edge
    a4 += s_hi * up - s_lo * um;
  }
  double A = c4 * a4;
  L0.uf[d][F] = L0.m[d][F] * udF - rho.a[d][F] * A + c_force * frc.a[d][F] + gflow;
  L0.u[d][F] = udF;
}

template <int D>
__global__ void __launch_bounds__(256) k_adv_rhs(Geo g, Ptr3 uv, Ptr3 rho, Ptr3 frc,
                                                 LevelPtrs<double> L0, double c_force, int flow,
                                                 const double* __restrict__ G_dev) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= g.n[0] + (g.open == 0) || j >= g.n[1] + (g.open == 1) || k >= g.n[2] + (g.open == 2))
    return;
  int ci[3] = {i, j, k};
  long long F = gidx(g, i, j, k);
  double G = *G_dev;
  const double c4 = 0.25 / g.h;
  adv_rhs_point<D, 0>(g, uv, rho, frc, L0, ci, F, c_force, flow == 0 ? G : 0.0, c4);
  adv_rhs_point<D, 1>(g, uv, rho, frc, L0, ci, F, c_force, flow == 1 ? G : 0.0, c4);
  if constexpr (D == 3)
    adv_rhs_point<D, 2>(g, uv, rho, frc, L0, ci, F, c_force, flow == 2 ? G : 0.0, c4);
}

// ---------------------------------------------------------------------------
// Divergence, projection and reductions.
// ---------------------------------------------------------------------------
template <int D>
__device__ __forceinline__ double div_at(const Geo& g, const Ptr3& u, const int ci[3],
                                         long long c) {
  double s = 0.0;
#pragma unroll
  for (int a = 0; a < D; ++a) s += (u.a[a][c + offp(g, a, ci[a])] - u.a[a][c]) / g.h;
  return s;
}

template <int D>
__global__ void __launch_bounds__(256) k_divergence(Geo g, Ptr3 u, double* __restrict__ b,
                                                    double scale, double* __restrict__ partial,
                                                    const double* __restrict__ beta_open,
                                                    double pbc) {
  __shared__ double sh[32];
  long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  double acc = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncell;
       q += (long long)gridDim.x * blockDim.x) {
    int ci[3];
    decode(g, q, ci[0], ci[1], ci[2]);
    long long c = gidx(g, ci[0], ci[1], ci[2]);
    double v = scale * div_at<D>(g, u, ci, c);
    // the held outflow pressure: b -= 2 beta_out p_out / h^2 (pbc = 2 p_out / h^2)
    if (last_open_cell(g, ci)) v -= beta_open[c + st_of(g, g.open)] * pbc;
    b[c] = v;
    acc += v;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__device__ __forceinline__ void partial_sum_body(const Blk& B, Geo g, const double* __restrict__ a,
                                                 double* __restrict__ partial) {
  __shared__ double sh[32];
  long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  double acc = 0.0;
  for (long long q = B.x * (long long)blockDim.x + threadIdx.x; q < ncell;
       q += (long long)B.gx * blockDim.x) {
    int i, j, k;
    decode(g, q, i, j, k);
    acc += a[gidx(g, i, j, k)];
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[B.x] = acc;
}

__global__ void __launch_bounds__(256) k_partial_sum(Geo g, const double* __restrict__ a,
                                                     double* __restrict__ partial) {
  partial_sum_body(own_blk(), g, a, partial);
}

// out[slot] = scale * (sum or max of partial[0..nb)), in a fixed order
__device__ __forceinline__ void finalize_body(const Blk& B, const double* __restrict__ partial,
                                              int nb, double* __restrict__ out, int slot,
                                              double scale, int is_max) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int q = threadIdx.x; q < nb; q += blockDim.x) v = is_max ? fmax(v, partial[q]) : v + partial[q];
  v = is_max ? block_max(v, sh) : block_sum(v, sh);
  if (threadIdx.x == 0) out[slot] = v * scale;
}

__global__ void __launch_bounds__(1024) k_finalize(const double* __restrict__ partial, int nb,
                                                   double* __restrict__ out, int slot,
                                                   double scale, int is_max) {
  finalize_body(own_blk(), partial, nb, out, slot, scale, is_max);
}

__device__ __forceinline__ void sub_scalar_body(const Blk& B, Geo g, double* __restrict__ a,
                                                const double* __restrict__ s) {
  int i = B.x * blockDim.x + threadIdx.x;
  int j = B.y * blockDim.y + threadIdx.y;
  int k = B.z * blockDim.z + threadIdx.z;
  if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) return;
  a[gidx(g, i, j, k)] -= *s;
}

__global__ void __launch_bounds__(256) k_sub_scalar(Geo g, double* __restrict__ a,
                                                    const double* __restrict__ s) {
  sub_scalar_body(own_blk(), g, a, s);
}

// u_d on one face after the projection, Eq. (NSdis2); pM is p of the cell
// below the face along d. One function for the face a thread owns and for
// the upper faces it recomputes, so both round alike.
__device__ __forceinline__ double proj_face(double ut, double beta, double pF, double pM,
                                            double coef, double h) {
  return ut - coef * beta * ((pF - pM) / h);
}

// Projection, Eq. (NSdis2), with the check of Eq. (NSdis4) fused in: each
// thread owns the lower faces of its cell, writes them, recomputes the upper
// ones (owned by the neighbours) and takes |D.u| of its cell in FP64. The
// block maximum goes to *divacc as the bit pattern of a non-negative double
// (unsigned max: order-independent, hence deterministic); a non-finite
// divergence counts as infinity.
template <int D>
__global__ void __launch_bounds__(256) k_project(Geo g, Ptr3 ut, const double* __restrict__ p,
                                                 Ptr3 beta, Ptr3 uv, double coef,
                                                 unsigned long long* __restrict__ divacc,
                                                 double p_out) {
  __shared__ double sh[32];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z * blockDim.z + threadIdx.z;
  double mx = 0.0;
  if (g.open >= 0) {   // the outflow faces, one plane beyond the last cells
    const int ci[3] = {i, j, k};
#pragma unroll
    for (int o = 0; o < D; ++o) {   // the open axis, as a compile-time index (see is_open)
      if (!is_open(g, o)) continue;
      bool beyond = ci[o] == g.n[o];
#pragma unroll
      for (int a = 0; a < D; ++a)
        if (a != o && ci[a] >= g.n[a]) beyond = false;
      if (beyond) {
        long long F = gidx(g, i, j, k);
        const double pm = p[F - g.st[o]];
        uv.a[o][F] = proj_face(ut.a[o][F], beta.a[o][F], 2.0 * p_out - pm, pm, coef, g.h);
      }
    }
  }
  if (i < g.n[0] && j < g.n[1] && k < g.n[2]) {
    int ci[3] = {i, j, k};
    long long F = gidx(g, i, j, k);
    const double pF = p[F];
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      double lo = 0.0;
      if (!g.per[d] && ci[d] == 0) {
        // not an unknown: 0 on a wall, the prescribed inflow on an open axis
        lo = ut.a[d][F];
        uv.a[d][F] = lo;
      } else {
        lo = proj_face(ut.a[d][F], beta.a[d][F], pF, p[F + offm(g, d, ci[d])], coef, g.h);
        uv.a[d][F] = lo;
      }
      double hi = 0.0;   // the upper wall face holds 0
      if (g.per[d] || ci[d] != g.n[d] - 1) {
        long long Fu = F + offp(g, d, ci[d]);
        hi = proj_face(ut.a[d][Fu], beta.a[d][Fu], p[Fu], pF, coef, g.h);
      } else if (is_open(g, d)) {   // the outflow face: ghost 2 p_out - p
        long long Fu = F + st_of(g, d);
        hi = proj_face(ut.a[d][Fu], beta.a[d][Fu], 2.0 * p_out - pF, pF, coef, g.h);
      }
      s += (hi - lo) / g.h;
    }
    mx = fabs(s);
    if (!(mx <= CUDART_INF)) mx = CUDART_INF;
  }
  // block maximum over the linear thread index (a 3D block)
  const int t = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  const int nt = blockDim.x * blockDim.y * blockDim.z;
  mx = warp_max(mx);
  if ((t & 31) == 0) sh[t >> 5] = mx;
  __syncthreads();
  if (t < 32) {
    mx = t < ((nt + 31) >> 5) ? sh[t] : 0.0;
    mx = warp_max(mx);
    if (t == 0 && mx > 0.0) atomicMax(divacc, (unsigned long long)__double_as_longlong(mx));
  }
}

// After a projection: this step's max |D.u| to out[step], the maximum over
// all steps to out[all], a violation counted when it exceeds tol (> 0), and
// the accumulator cleared for the next projection.
__global__ void k_div_check(double* __restrict__ out, int acc, int step, int all, double tol,
                            int* __restrict__ viol) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned long long* a = reinterpret_cast<unsigned long long*>(out + acc);
  const double v = __longlong_as_double((long long)*a);
  out[step] = v;
  out[all] = fmax(out[all], v);
  if (tol > 0.0 && !(v <= tol)) ++(*viol);
  *a = 0ull;
}

template <int D>
__device__ __forceinline__ void norm2_body(const Blk& B, Geo g, Ptr3 a, int ncomp,
                                           double* __restrict__ partial) {
  __shared__ double sh[32];
  long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  double acc = 0.0;
  for (long long q = B.x * (long long)blockDim.x + threadIdx.x; q < ncell;
       q += (long long)B.gx * blockDim.x) {
    int ci[3];
    decode(g, q, ci[0], ci[1], ci[2]);
    long long c = gidx(g, ci[0], ci[1], ci[2]);
    if (ncomp == 0) {
      double v = a.a[0][c];
      acc += v * v;
    } else {
#pragma unroll
      for (int d = 0; d < 3; ++d) {   // compile-time components (see is_open)
        if (d >= ncomp) break;
        if (is_open(g, d) && ci[d] == g.n[d] - 1) {   // the outflow face is an unknown too
          double v = a.a[d][c + st_of(g, d)];
          acc += v * v;
        }
        if (!g.per[d] && ci[d] == 0) continue;
        double v = a.a[d][c];
        acc += v * v;
      }
    }
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[B.x] = acc;
}

template <int D>
__global__ void __launch_bounds__(256) k_norm2(Geo g, Ptr3 a, int ncomp,
                                               double* __restrict__ partial) {
  norm2_body<D>(own_blk(), g, a, ncomp, partial);
}

template <int D>
__global__ void __launch_bounds__(256) k_div_ke(Geo g, Ptr3 u, double* __restrict__ pmax,
                                                double* __restrict__ psum) {
  __shared__ double sh[32];
  long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  double mx = 0.0, acc = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncell;
       q += (long long)gridDim.x * blockDim.x) {
    int ci[3];
    decode(g, q, ci[0], ci[1], ci[2]);
    long long c = gidx(g, ci[0], ci[1], ci[2]);
    mx = fmax(mx, fabs(div_at<D>(g, u, ci, c)));
    for (int d = 0; d < D; ++d) {
      if (d == g.open && ci[d] == g.n[d] - 1) {   // the outflow face
        double v = u.a[d][c + g.st[d]];
        acc += v * v;
      }
      if (!g.per[d] && ci[d] == 0) continue;
      double v = u.a[d][c];
      acc += v * v;
    }
  }
  mx = block_max(mx, sh);
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) {
    pmax[blockIdx.x] = mx;
    psum[blockIdx.x] = acc;
  }
}

// ---------------------------------------------------------------------------
// Laminar profile (Eq. 2DlaminarSoln, Eq. 3DlaminarFlow) for G = 1 and an
// effective viscosity of 1. In 3D the double series of Eq. (3DlaminarFlow)
// is summed over one index in closed form: x(A-x)/2 minus a single series in
// cosh, summed over the odd n below 1000.
// ---------------------------------------------------------------------------
__device__ double laminar_unit(int D, double A, double B, double x, double y) {
  if (D == 2) return 0.5 * x * (A - x);
  double sum = 0.0;
  for (int n = 1; n <= 999; n += 2) {
    double k = n * CUDART_PI / A;
    double t1 = exp(k * (y - B)) + exp(-k * y);
    double t2 = 1.0 + exp(-k * B);
    sum += sin(k * x) * (t1 / t2) / ((double)n * n * n);
  }
  return 0.5 * x * (A - x) - 4.0 * A * A / (CUDART_PI * CUDART_PI * CUDART_PI) * sum;
}

__global__ void k_body_force(int D, double A, double B, double mu_eff, double u_center,
                             double body_force, double* G_dev) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (u_center > 0.0)
    *G_dev = u_center * mu_eff / laminar_unit(D, A, B, 0.5 * A, 0.5 * B);
  else
    *G_dev = body_force;
}

// one thread per column across the flow axis; the value is copied along it
__global__ void k_laminar(Geo g, int D, int fa, int ta0, int ta1, double mu_eff, double ic_scale,
                          const double* __restrict__ G_dev, double* __restrict__ u) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  int b = blockIdx.y * blockDim.y + threadIdx.y;
  int n0 = g.n[ta0], n1 = (D == 3) ? g.n[ta1] : 1;
  if (a >= n0 || b >= n1) return;
  double A = g.n[ta0] * g.h, B = (D == 3) ? g.n[ta1] * g.h : 0.0;
  double full = (*G_dev) / mu_eff * laminar_unit(D, A, B, (a + 0.5) * g.h, (b + 0.5) * g.h);
  double v = ic_scale * full;
  int lo = g.per[fa] ? 0 : 1, hi = g.n[fa] + (fa == g.open ? 1 : 0);
  for (int q = lo; q < hi; ++q) {
    int c[3] = {0, 0, 0};
    c[fa] = q;
    c[ta0] = a;
    if (D == 3) c[ta1] = b;
    u[gidx(g, c[0], c[1], c[2])] = v;
  }
  if (fa == g.open) {   // the inflow face holds the laminar profile itself (Sec. 3.6)
    int c[3] = {0, 0, 0};
    c[ta0] = a;
    if (D == 3) c[ta1] = b;
    u[gidx(g, c[0], c[1], c[2])] = full;
  }
}

// One iteration of a device-side relative-residual loop has finished:
// count it and keep looping while ||r||/||f|| > rtol (or, with mtol > 0,
// mscale * out[smax] > mtol) and the cap is not hit. A loop that stops at
// the cap with either test unmet is counted in *nonconv.
__global__ void k_tol_check(cudaGraphConditionalHandle h, const double* __restrict__ out, int sf,
                            int sr, double rtol, int maxc, int* __restrict__ counter,
                            long long* __restrict__ total, int* __restrict__ nonconv, int smax,
                            double mscale, double mtol) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int n = ++(*counter);
  ++(*total);
  double f2 = out[sf], r2 = out[sr];
  double rel = f2 > 0.0 ? sqrt(r2) / sqrt(f2) : 0.0;
  const bool met = rel <= rtol && (mtol <= 0.0 || mscale * out[smax] <= mtol);
  const bool again = !met && n < maxc;
  if (!again && !met) ++(*nonconv);
  cudaGraphSetConditional(h, again ? 1u : 0u);
}

// max over cells of |a| (a non-finite value counts as infinity), per block
__global__ void __launch_bounds__(256) k_absmax_cells(Geo g, const double* __restrict__ a,
                                                      double* __restrict__ partial) {
  __shared__ double sh[32];
  long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  double mx = 0.0;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ncell;
       q += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    decode(g, q, i, j, k);
    double v = fabs(a[gidx(g, i, j, k)]);
    mx = (v <= CUDART_INF) ? fmax(mx, v) : CUDART_INF;
  }
  mx = block_max(mx, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = mx;
}

// ||r||/||f|| from out[sr], out[sf]: counted in *nonconv when above thresh
__global__ void k_res_check(const double* __restrict__ out, int sf, int sr, double thresh,
                            int* __restrict__ nonconv) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double f2 = out[sf], r2 = out[sr];
  double rel = f2 > 0.0 ? sqrt(r2) / sqrt(f2) : 0.0;
  if (!(rel <= thresh)) ++(*nonconv);
}

__global__ void k_fill(double* a, long long n, double v) {
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
       q += (long long)gridDim.x * blockDim.x)
    a[q] = v;
}


// ===========================================================================
// Batched kernels: the bodies above, run over a persistent batch's work list
// (3D, FP32 V-cycle arrays; FP64 on level 0 and the coarsest level). Each
// copies a member's geometry and pointers out of the table before the body
// runs, so the body's stores cannot alias them.
// ===========================================================================
__global__ void __launch_bounds__(256) kb_v_residual32(BArgs A) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    v_residual_body<3, float>(B, M.g[A.lev], cur_ptrs(M.f[A.lev], A.cur), (float)M.ir[A.lev]);
  });
}

__global__ void __launch_bounds__(256) kb_p_residual32(BArgs A) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    p_residual_body<3, float>(B, M.g[A.lev], cur_ptrs(M.f[A.lev], A.cur), (float)M.ih2[A.lev]);
  });
}

__global__ void __launch_bounds__(256) kb_restrict_face32(BArgs A) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    const int l = A.lev;
    Faces3<float> rf, fc, xc;
    for (int d = 0; d < 3; ++d) {
      rf.a[d] = M.f[l].ur[d];
      fc.a[d] = M.f[l + 1].uf[d];
      xc.a[d] = M.f[l + 1].u[d];
    }
    restrict_face3_body<float>(B, M.g[l], M.g[l + 1], rf, fc, xc);
  });
}

__global__ void __launch_bounds__(256) kb_restrict_cell32(BArgs A) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    const int l = A.lev;
    restrict_cell_body<3, float>(B, M.g[l], M.g[l + 1], M.f[l].pr, M.f[l + 1].pf, M.f[l + 1].p);
  });
}

__global__ void __launch_bounds__(256) kb_prolong_face32(BArgs A) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    const int l = A.lev;
    Faces3<float> ec, xf;
    for (int d = 0; d < 3; ++d) {
      ec.a[d] = M.f[l + 1].u[d];
      xf.a[d] = M.f[l].u[d];
    }
    prolong_face3_body<float>(B, M.g[l], M.g[l + 1], ec, xf);
  });
}

__global__ void __launch_bounds__(256) kb_prolong_cell32(BArgs A) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    const int l = A.lev;
    prolong_cell_body<3, float>(B, M.g[l], M.g[l + 1], M.f[l + 1].p, M.f[l].p);
  });
}

// The coarsest level of one member per block, as the single-instance
// V-cycle does it in four launches: the FP32 right-hand side converted to
// FP64 and the FP64 iterate zeroed on every stored element, the FP64 coarse
// solve (staged in shared memory under the same size rule), the result
// rounded to FP32.
template <bool V>
__global__ void __launch_bounds__(1024) kb_coarse(BArgs A) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    const Geo g = M.g[A.lev];
    const LevelPtrs<double> Ld = M.d[A.lev];
    const LevelPtrs<float> Lf = M.f[A.lev];
    const long long nel = g.st[2] * g.s[2];
    for (long long q = threadIdx.x; q < nel; q += blockDim.x) {
      if (V) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          Ld.uf[d][q] = (double)Lf.uf[d][q];
          Ld.u[d][q] = 0.0;
        }
      } else {
        Ld.pf[q] = (double)Lf.pf[q];
        Ld.p[q] = 0.0;
      }
    }
    __syncthreads();
    const int use = coarse_bytes(3, g, (int)sizeof(double), V) <= kCoarseSmemMax;
    if (V) coarse_v_body<3, double>(B, g, Ld, M.coarse_sweeps, M.ir[A.lev], nel, use);
    else coarse_p_body<3, double>(B, g, Ld, M.coarse_sweeps, nel, use);
    __syncthreads();
    for (long long q = threadIdx.x; q < nel; q += blockDim.x) {
      if (V) {
#pragma unroll
        for (int d = 0; d < 3; ++d) Lf.u[d][q] = (float)Ld.u[d][q];
      } else {
        Lf.p[q] = (float)Ld.p[q];
      }
    }
  });
}

__global__ void __launch_bounds__(256) kb_norm2(BArgs A, int viscous) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    Ptr3 a;
    for (int d = 0; d < 3; ++d) a.a[d] = viscous ? M.d[0].uf[d] : (d == 0 ? M.d[0].pf : nullptr);
    norm2_body<3>(B, M.g[0], a, viscous ? 3 : 0, M.sc.partial);
  });
}

__global__ void __launch_bounds__(256) kb_partial_sum_p(BArgs A) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    partial_sum_body(B, M.g[0], M.d[0].p, M.sc.partial);
  });
}

__global__ void __launch_bounds__(256) kb_sub_scalar_p(BArgs A) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    sub_scalar_body(B, M.g[0], M.d[0].p, M.sc.out);
  });
}

__global__ void __launch_bounds__(1024) kb_finalize(BArgs A, int off, int slot, int is_max,
                                                    int mean) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    const int nb = B.gx;
    const Geo& g = M.g[0];
    const double scale = mean ? 1.0 / (double)((long long)g.n[0] * g.n[1] * g.n[2]) : 1.0;
    finalize_body(B, M.sc.partial + (long long)off * nb, nb, M.sc.out, slot, scale, is_max);
  });
}

__global__ void kb_begin(const BMember* __restrict__ tab, int nm, int* __restrict__ act,
                         int which, int zero_slot) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < nm; m += gridDim.x * blockDim.x) {
    act[m] = 1;
    tab[m].cycles[which] = 0;
    if (zero_slot >= 0) tab[m].sc.out[zero_slot] = 0.0;
  }
}

// the test of k_tol_check per active member; one block
__global__ void __launch_bounds__(1024) kb_tol_check(cudaGraphConditionalHandle h,
                                                     const BMember* __restrict__ tab, int nm,
                                                     int* __restrict__ act, int which, int sf,
                                                     int sr, int smax, long long* iters,
                                                     int use_h) {
  int any = 0;
  for (int m = threadIdx.x; m < nm; m += blockDim.x) {
    if (!act[m]) continue;
    const BMember& M = tab[m];
    const int n = ++M.cycles[which];
    ++M.total[which];
    const double f2 = M.sc.out[sf], r2 = M.sc.out[sr];
    const double rel = f2 > 0.0 ? sqrt(r2) / sqrt(f2) : 0.0;
    const double mtol = smax >= 0 ? M.div_tol : 0.0;
    const bool met = rel <= M.rtol && (mtol <= 0.0 || M.dscale * M.sc.out[smax] <= mtol);
    const bool again = !met && n < M.maxc;
    if (!again && !met) ++(*M.nonconv);
    act[m] = again ? 1 : 0;
    any |= again ? 1 : 0;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    ++iters[which];
    if (use_h) cudaGraphSetConditional(h, any ? 1u : 0u);
  }
}

__global__ void kb_res_check(const BMember* __restrict__ tab, int nm, int sf, int sr,
                             double slack) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < nm; m += gridDim.x * blockDim.x) {
    const BMember& M = tab[m];
    const double f2 = M.sc.out[sf], r2 = M.sc.out[sr];
    const double rel = f2 > 0.0 ? sqrt(r2) / sqrt(f2) : 0.0;
    if (!(rel <= slack * M.rtol)) ++(*M.nonconv);
  }
}


// ===========================================================================
// Coarse-level V-cycle in one launch (one cluster per member). The levels
// below a few thousand cells cost a launch per sweep, residual, transfer and
// conversion, each a few microseconds of mostly idle GPU; here one cluster of
// kTailCtas CTAs runs them all, phase after phase, with a cluster barrier
// (release / acquire) between phases. Sweeps are in place: all red points of
// a component, a barrier, all black points. The red update reads the old
// black neighbours and the black update the new red ones, as in the one-pass
// sweeps, with the same point function (v_red / p_red), so the bits are those
// of the launches it replaces. Every array a phase writes is read back through
// L2 (the COH point functions), never through the read-only cache.
// ===========================================================================
// the barrier between phases: the cluster's (release / acquire at cluster
// scope), or the block's when the member has one CTA
template <int C>
__device__ __forceinline__ void tail_sync() {
  if constexpr (C == 1) {
    __syncthreads();
  } else {
    asm volatile("barrier.cluster.arrive.release;\n\t"
                 "barrier.cluster.wait.acquire;" ::: "memory");
  }
}

// one colour of viscous component d on level g, in place
template <int d>
__device__ __forceinline__ void tail_v_colour(const Geo& g, const LevelPtrs<float>& L, float ir,
                                              int colour, int t0, int T) {
  const int nh = (g.n[0] + 1) >> 1;
  const int npts = nh * g.n[1] * g.n[2];
  for (int q = t0; q < npts; q += T) {
    const int ih = q % nh, r = q / nh;
    const int j = r % g.n[1], k = r / g.n[1];
    const int i = 2 * ih + ((j + k + colour) & 1);
    if (i >= g.n[0]) continue;
    const int ci[3] = {i, j, k};
    if (!g.per[d] && ci[d] == 0) continue;   // the wall face stays 0
    Pt pt;
    make_pt<3>(g, ci, pt);
    L.u[d][pt.F] = v_red<3, d, float, true>(L, pt, ir);
  }
}

__device__ __forceinline__ void tail_p_colour(const Geo& g, const LevelPtrs<float>& L, float h2,
                                              int colour, int t0, int T) {
  const int nh = (g.n[0] + 1) >> 1;
  const int npts = nh * g.n[1] * g.n[2];
  for (int q = t0; q < npts; q += T) {
    const int ih = q % nh, r = q / nh;
    const int j = r % g.n[1], k = r / g.n[1];
    const int i = 2 * ih + ((j + k + colour) & 1);
    if (i >= g.n[0]) continue;
    const int ci[3] = {i, j, k};
    Pt pt;
    make_pt<3>(g, ci, pt);
    L.p[pt.F] = p_red<3, float, true>(L, pt, h2);
  }
}

template <bool V, int C>
__device__ __forceinline__ void tail_smooth(const BMember& M, int l, int n, int t0, int T) {
  const Geo g = M.g[l];
  const LevelPtrs<float> L = M.f[l];
  for (int it = 0; it < n; ++it) {
    if (V) {
      const float ir = (float)M.ir[l];
      for (int c = 0; c < 2; ++c) {
        tail_v_colour<0>(g, L, ir, c, t0, T);
        tail_sync<C>();
      }
      for (int c = 0; c < 2; ++c) {
        tail_v_colour<1>(g, L, ir, c, t0, T);
        tail_sync<C>();
      }
      for (int c = 0; c < 2; ++c) {
        tail_v_colour<2>(g, L, ir, c, t0, T);
        tail_sync<C>();
      }
    } else {
      const float h2 = (float)(g.h * g.h);
      for (int c = 0; c < 2; ++c) {
        tail_p_colour(g, L, h2, c, t0, T);
        tail_sync<C>();
      }
    }
  }
}

// residual on level l, restricted to level l + 1 (whose iterate it zeroes)
template <bool V, int C>
__device__ __forceinline__ void tail_down(const BMember& M, int l, int t0, int T) {
  const Geo g = M.g[l], gc = M.g[l + 1];
  const LevelPtrs<float> L = M.f[l], Lc = M.f[l + 1];
  const int ncell = g.n[0] * g.n[1] * g.n[2];
  const float ir = (float)M.ir[l];
  for (int q = t0; q < ncell; q += T) {
    const int ci[3] = {q % g.n[0], (q / g.n[0]) % g.n[1], q / (g.n[0] * g.n[1])};
    Pt pt;
    make_pt<3>(g, ci, pt);
    if (V) {
      v_residual_point<3, 0, float, true>(g, L, ci, pt, ir);
      v_residual_point<3, 1, float, true>(g, L, ci, pt, ir);
      v_residual_point<3, 2, float, true>(g, L, ci, pt, ir);
    } else {
      p_residual_at<3, float, true>(g, L, ci, pt.F, (float)M.ih2[l]);
    }
  }
  tail_sync<C>();
  if (V) {
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      // along d the stored faces (walls included), across d the cells
      const int e0 = d == 0 ? gc.s[0] : gc.n[0], e1 = d == 1 ? gc.s[1] : gc.n[1],
                e2 = d == 2 ? gc.s[2] : gc.n[2];
      for (int q = t0; q < e0 * e1 * e2; q += T) {
        const int cc[3] = {q % e0, (q / e0) % e1, q / (e0 * e1)};
        if (d == 0) restrict_face_at<3, 0, float, true>(g, gc, L.ur[0], Lc.uf[0], Lc.u[0], cc);
        else if (d == 1) restrict_face_at<3, 1, float, true>(g, gc, L.ur[1], Lc.uf[1], Lc.u[1], cc);
        else restrict_face_at<3, 2, float, true>(g, gc, L.ur[2], Lc.uf[2], Lc.u[2], cc);
      }
    }
  } else {
    const int nc = gc.n[0] * gc.n[1] * gc.n[2];
    for (int q = t0; q < nc; q += T)
      restrict_cell_at<3, float, true>(g, gc, L.pr, Lc.pf, Lc.p, q % gc.n[0],
                                       (q / gc.n[0]) % gc.n[1], q / (gc.n[0] * gc.n[1]));
  }
  tail_sync<C>();
}

// the correction of level l + 1 prolonged onto level l
template <bool V, int C>
__device__ __forceinline__ void tail_up(const BMember& M, int l, int t0, int T) {
  const Geo g = M.g[l], gc = M.g[l + 1];
  const LevelPtrs<float> L = M.f[l], Lc = M.f[l + 1];
  const int ncell = g.n[0] * g.n[1] * g.n[2];
  for (int q = t0; q < ncell; q += T) {
    const int fi[3] = {q % g.n[0], (q / g.n[0]) % g.n[1], q / (g.n[0] * g.n[1])};
    if (V) {
      if (g.per[0] || fi[0] != 0) prolong_face_at<3, 0, float, true>(g, gc, Lc.u[0], L.u[0], fi);
      if (g.per[1] || fi[1] != 0) prolong_face_at<3, 1, float, true>(g, gc, Lc.u[1], L.u[1], fi);
      if (g.per[2] || fi[2] != 0) prolong_face_at<3, 2, float, true>(g, gc, Lc.u[2], L.u[2], fi);
    } else {
      prolong_cell_at<3, float, true>(g, gc, Lc.p, L.p, fi);
    }
  }
  tail_sync<C>();
}

// the coarsest level, on the cluster's first CTA: as kb_coarse
template <bool V, int C>
__device__ __forceinline__ void tail_coarse(const BMember& M, int rank) {
  const int l = M.L - 1;
  if (rank == 0) {
    const Geo g = M.g[l];
    const LevelPtrs<double> Ld = M.d[l];
    const LevelPtrs<float> Lf = M.f[l];
    const long long nel = g.st[2] * g.s[2];
    for (long long q = threadIdx.x; q < nel; q += blockDim.x) {
      if (V) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          Ld.uf[d][q] = (double)__ldcg(Lf.uf[d] + q);
          Ld.u[d][q] = 0.0;
        }
      } else {
        Ld.pf[q] = (double)__ldcg(Lf.pf + q);
        Ld.p[q] = 0.0;
      }
    }
    __syncthreads();
    const int use = coarse_bytes(3, g, (int)sizeof(double), V) <= kCoarseSmemMax;
    const Blk B{0, 0, 0, 1, 1, 1};
    if (V) coarse_v_body<3, double>(B, g, Ld, M.coarse_sweeps, M.ir[l], nel, use);
    else coarse_p_body<3, double>(B, g, Ld, M.coarse_sweeps, nel, use);
    __syncthreads();
    for (long long q = threadIdx.x; q < nel; q += blockDim.x) {
      if (V) {
#pragma unroll
        for (int d = 0; d < 3; ++d) Lf.u[d][q] = (float)Ld.u[d][q];
      } else {
        Lf.p[q] = (float)Ld.p[q];
      }
    }
  }
  tail_sync<C>();
}

// one member per C CTAs (a cluster when C > 1)
template <bool V, int C>
__device__ __forceinline__ void tail_run(const BMember* __restrict__ tab,
                                         const int* __restrict__ list, int nlist,
                                         const int* __restrict__ act) {
  const int item = blockIdx.x / C;
  if (item >= nlist) return;
  const int m = list[item];
  if (act && !act[m]) return;               // all C CTAs leave together
  const BMember& M = tab[m];
  const int rank = blockIdx.x % C;
  const int t0 = rank * blockDim.x + threadIdx.x, T = C * blockDim.x;
  const int ls = M.tail, lc = M.L - 1;
  for (int l = ls; l < lc; ++l) {
    tail_smooth<V, C>(M, l, M.nu1, t0, T);
    tail_down<V, C>(M, l, t0, T);
  }
  tail_coarse<V, C>(M, rank);
  for (int l = lc - 1; l >= ls; --l) {
    tail_up<V, C>(M, l, t0, T);
    tail_smooth<V, C>(M, l, M.nu2, t0, T);
  }
}

// Threads per CTA: the pressure's coarsest solve sums the right-hand side's
// mean over 1024 threads, as the one-block coarse kernel does (the same order,
// the same bits); the viscous kernel has no block reduction and takes 512
// threads, so that each may hold 128 registers.
template <bool V>
constexpr int kTailThreads = V ? 512 : 1024;

template <bool V>
__global__ void __cluster_dims__(kTailCtas, 1, 1) __launch_bounds__(kTailThreads<V>)
    k_tail(const BMember* __restrict__ tab, const int* __restrict__ list, int nlist,
           const int* __restrict__ act) {
  tail_run<V, kTailCtas>(tab, list, nlist, act);
}

// one CTA per member: many members side by side in one wave
template <bool V>
__global__ void __launch_bounds__(kTailThreads<V>) k_tail1(const BMember* __restrict__ tab,
                                                           const int* __restrict__ list,
                                                           int nlist, const int* __restrict__ act) {
  tail_run<V, 1>(tab, list, nlist, act);
}

}  // namespace

// ===========================================================================
// launchers
// ===========================================================================
template <typename T>
void launch_p_rbgs(int D, const Geo& g, const LevelPtrs<T>& L, int colour, cudaStream_t s) {
  dim3 b = blk3(D);
  dim3 gr = grd3((g.n[0] + 1) / 2, g.n[1], g.n[2], b);
  if (D == 3) k_p_rbgs<3, T><<<gr, b, 0, s>>>(g, L, colour);
  else k_p_rbgs<2, T><<<gr, b, 0, s>>>(g, L, colour);
}

template <typename T>
void launch_p_residual(int D, const Geo& g, const LevelPtrs<T>& L, cudaStream_t s) {
  dim3 b = blk3(D);
  dim3 gr = grd3(g.n[0], g.n[1], g.n[2], b);
  const T ih2 = (T)(1.0 / (g.h * g.h));
  if (D == 3) k_p_residual<3, T><<<gr, b, 0, s>>>(g, L, ih2);
  else k_p_residual<2, T><<<gr, b, 0, s>>>(g, L, ih2);
}

template <typename T>
void launch_v_rbgs(int D, const Geo& g, const LevelPtrs<T>& L, int d, int colour, double inv_re,
                   cudaStream_t s) {
  dim3 b = blk3(D);
  dim3 gr = grd3((ext(g, 0, d == 0) + 1) / 2, ext(g, 1, d == 1), ext(g, 2, d == 2), b);
  T ir = (T)(inv_re / (g.h * g.h));
  if (D == 3) {
    if (d == 0) k_v_rbgs<3, 0, T><<<gr, b, 0, s>>>(g, L, colour, ir);
    else if (d == 1) k_v_rbgs<3, 1, T><<<gr, b, 0, s>>>(g, L, colour, ir);
    else k_v_rbgs<3, 2, T><<<gr, b, 0, s>>>(g, L, colour, ir);
  } else {
    if (d == 0) k_v_rbgs<2, 0, T><<<gr, b, 0, s>>>(g, L, colour, ir);
    else k_v_rbgs<2, 1, T><<<gr, b, 0, s>>>(g, L, colour, ir);
  }
}

template <typename T>
void launch_v_residual(int D, const Geo& g, const LevelPtrs<T>& L, double inv_re, cudaStream_t s) {
  dim3 b = blk3(D);
  dim3 gr = grd3(ext(g, 0, true), ext(g, 1, true), ext(g, 2, true), b);
  T ir = (T)(inv_re / (g.h * g.h));
  if (D == 3) k_v_residual<3, T><<<gr, b, 0, s>>>(g, L, ir);
  else k_v_residual<2, T><<<gr, b, 0, s>>>(g, L, ir);
}

template <typename T>
void launch_restrict_cell(int D, const Geo& gf, const Geo& gc, const T* rf, T* fc, T* xc,
                          cudaStream_t s) {
  dim3 b = blk3(D);
  dim3 gr = grd3(gc.n[0], gc.n[1], gc.n[2], b);
  if (D == 3) k_restrict_cell<3, T><<<gr, b, 0, s>>>(gf, gc, rf, fc, xc);
  else k_restrict_cell<2, T><<<gr, b, 0, s>>>(gf, gc, rf, fc, xc);
}

template <typename T>
void launch_restrict_face(int D, int d, const Geo& gf, const Geo& gc, const T* rf, T* fc, T* xc,
                          cudaStream_t s) {
  dim3 b = blk3(D);
  dim3 gr = grd3(gc.s[0], gc.s[1], gc.s[2], b);
  if (D == 3) {
    if (d == 0) k_restrict_face<3, 0, T><<<gr, b, 0, s>>>(gf, gc, rf, fc, xc);
    else if (d == 1) k_restrict_face<3, 1, T><<<gr, b, 0, s>>>(gf, gc, rf, fc, xc);
    else k_restrict_face<3, 2, T><<<gr, b, 0, s>>>(gf, gc, rf, fc, xc);
  } else {
    if (d == 0) k_restrict_face<2, 0, T><<<gr, b, 0, s>>>(gf, gc, rf, fc, xc);
    else k_restrict_face<2, 1, T><<<gr, b, 0, s>>>(gf, gc, rf, fc, xc);
  }
}

template <typename T>
void launch_prolong_cell(int D, const Geo& gf, const Geo& gc, const T* ec, T* xf, cudaStream_t s) {
  dim3 b = blk3(D);
  dim3 gr = grd3(gf.n[0], gf.n[1], gf.n[2], b);
  if (D == 3) k_prolong_cell<3, T><<<gr, b, 0, s>>>(gf, gc, ec, xf);
  else k_prolong_cell<2, T><<<gr, b, 0, s>>>(gf, gc, ec, xf);
}

template <typename T>
void launch_prolong_face(int D, int d, const Geo& gf, const Geo& gc, const T* ec, T* xf,
                         cudaStream_t s) {
  dim3 b = blk3(D);
  dim3 gr = grd3(ext(gf, 0, d == 0), ext(gf, 1, d == 1), ext(gf, 2, d == 2), b);
  if (D == 3) {
    if (d == 0) k_prolong_face<3, 0, T><<<gr, b, 0, s>>>(gf, gc, ec, xf);
    else if (d == 1) k_prolong_face<3, 1, T><<<gr, b, 0, s>>>(gf, gc, ec, xf);
    else k_prolong_face<3, 2, T><<<gr, b, 0, s>>>(gf, gc, ec, xf);
  } else {
    if (d == 0) k_prolong_face<2, 0, T><<<gr, b, 0, s>>>(gf, gc, ec, xf);
    else k_prolong_face<2, 1, T><<<gr, b, 0, s>>>(gf, gc, ec, xf);
  }
}

template <typename T>
void launch_restrict_face3(const Geo& gf, const Geo& gc, T* const rf[3], T* const fc[3],
                           T* const xc[3], cudaStream_t s) {
  Faces3<T> r, f, x;
  for (int d = 0; d < 3; ++d) {
    r.a[d] = rf[d];
    f.a[d] = fc[d];
    x.a[d] = xc[d];
  }
  dim3 b = blk3(3);
  k_restrict_face3<T><<<grd3(gc.s[0], gc.s[1], gc.s[2], b), b, 0, s>>>(gf, gc, r, f, x);
}

template <typename T>
void launch_prolong_face3(const Geo& gf, const Geo& gc, T* const ec[3], T* const xf[3],
                          cudaStream_t s) {
  Faces3<T> e, x;
  for (int d = 0; d < 3; ++d) {
    e.a[d] = ec[d];
    x.a[d] = xf[d];
  }
  dim3 b = blk3(3);
  if (gf.n[0] % 2 == 0)
    k_prolong_face3_pair<T><<<grd3(gf.n[0] / 2, gf.n[1], gf.n[2], b), b, 0, s>>>(gf, gc, e, x);
  else
    k_prolong_face3<T><<<grd3(gf.n[0], gf.n[1], gf.n[2], b), b, 0, s>>>(gf, gc, e, x);
}
template void launch_restrict_face3<float>(const Geo&, const Geo&, float* const[3],
                                           float* const[3], float* const[3], cudaStream_t);
template void launch_restrict_face3<double>(const Geo&, const Geo&, double* const[3],
                                            double* const[3], double* const[3], cudaStream_t);
template void launch_prolong_face3<float>(const Geo&, const Geo&, float* const[3],
                                          float* const[3], cudaStream_t);
template void launch_prolong_face3<double>(const Geo&, const Geo&, double* const[3],
                                           double* const[3], cudaStream_t);

size_t coarse_smem_bytes(int D, const Geo& g, int elem, bool viscous) {
  return coarse_bytes(D, g, elem, viscous);
}

template <typename T>
void launch_coarse_p(int D, const Geo& g, const LevelPtrs<T>& L, int sweeps, cudaStream_t s) {
  // with the outflow pressure held the slowest coarse mode is no longer the
  // constant the mean removes: at least 2 n^2 sweeps along the open axis
  if (g.open >= 0 && sweeps < 2 * g.n[g.open] * g.n[g.open]) sweeps = 2 * g.n[g.open] * g.n[g.open];
  long long nel = g.st[2] * g.s[2];
  size_t smem = coarse_smem_bytes(D, g, sizeof(T), false);
  int use = smem <= kCoarseSmemMax;
  if (!use) smem = 0;
  if (D == 3) k_coarse_p<3, T><<<1, 1024, smem, s>>>(g, L, sweeps, nel, use);
  else k_coarse_p<2, T><<<1, 1024, smem, s>>>(g, L, sweeps, nel, use);
}

template <typename T>
void launch_coarse_v(int D, const Geo& g, const LevelPtrs<T>& L, int sweeps, double inv_re,
                     cudaStream_t s) {
  T ir = (T)(inv_re / (g.h * g.h));
  long long nel = g.st[2] * g.s[2];
  size_t smem = coarse_smem_bytes(D, g, sizeof(T), true);
  int use = smem <= kCoarseSmemMax;
  if (!use) smem = 0;
  if (D == 3) k_coarse_v<3, T><<<1, 1024, smem, s>>>(g, L, sweeps, ir, nel, use);
  else k_coarse_v<2, T><<<1, 1024, smem, s>>>(g, L, sweeps, ir, nel, use);
}

cudaError_t coarse_set_smem() {
  cudaError_t e = cudaSuccess;
  int b = (int)kCoarseSmemMax;
  auto set = [&](const void* f) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  };
  set((const void*)k_coarse_p<3, double>);
  set((const void*)k_coarse_p<2, double>);
  set((const void*)k_coarse_v<3, double>);
  set((const void*)k_coarse_v<2, double>);
  set((const void*)k_coarse_p<3, float>);
  set((const void*)k_coarse_p<2, float>);
  set((const void*)k_coarse_v<3, float>);
  set((const void*)k_coarse_v<2, float>);
  return e;
}

#define BF_INST(T)                                                                           \
  template void launch_p_rbgs<T>(int, const Geo&, const LevelPtrs<T>&, int, cudaStream_t);   \
  template void launch_p_residual<T>(int, const Geo&, const LevelPtrs<T>&, cudaStream_t);    \
  template void launch_v_rbgs<T>(int, const Geo&, const LevelPtrs<T>&, int, int, double,     \
                                 cudaStream_t);                                              \
  template void launch_v_residual<T>(int, const Geo&, const LevelPtrs<T>&, double,           \
                                     cudaStream_t);                                          \
  template void launch_restrict_cell<T>(int, const Geo&, const Geo&, const T*, T*, T*,       \
                                        cudaStream_t);                                       \
  template void launch_restrict_face<T>(int, int, const Geo&, const Geo&, const T*, T*, T*,  \
                                        cudaStream_t);                                       \
  template void launch_prolong_cell<T>(int, const Geo&, const Geo&, const T*, T*,            \
                                       cudaStream_t);                                        \
  template void launch_prolong_face<T>(int, int, const Geo&, const Geo&, const T*, T*,       \
                                       cudaStream_t);                                        \
  template void launch_coarse_p<T>(int, const Geo&, const LevelPtrs<T>&, int, cudaStream_t); \
  template void launch_coarse_v<T>(int, const Geo&, const LevelPtrs<T>&, int, double,        \
                                   cudaStream_t);
BF_INST(double)
BF_INST(float)
#undef BF_INST

static Ptr3 ptr3(double* const a[3]) {
  Ptr3 p;
  for (int d = 0; d < 3; ++d) p.a[d] = a[d];
  return p;
}

void launch_coef_fine(int D, const Geo& g, double* const rho[3], double* beta[3], double* m[3],
                      double msc, cudaStream_t s) {
  dim3 b = blk3(D);
  dim3 gr = grd3(g.s[0], g.s[1], g.s[2], b);
  k_coef_fine<<<gr, b, 0, s>>>(g, D, ptr3(rho), ptr3(beta), ptr3(m), msc);
}

void launch_coef_restrict(int D, const Geo& gf, const Geo& gc, const LevelPtrs<double>& F,
                          const LevelPtrs<double>& C, double gamma, cudaStream_t s) {
  dim3 b = blk3(D);
  dim3 gr = grd3(gc.s[0], gc.s[1], gc.s[2], b);
  if (D == 3) k_coef_restrict<3><<<gr, b, 0, s>>>(gf, gc, F, C, gamma);
  else k_coef_restrict<2><<<gr, b, 0, s>>>(gf, gc, F, C, gamma);
}

void launch_adv_rhs(int D, const Geo& g, double* const uvel[3], double* const rho[3],
                    double* const frc[3], const LevelPtrs<double>& L0, double c_force,
                    int flow_axis, const double* G_dev, cudaStream_t s) {
  dim3 b = blk3(D);
  dim3 gr = grd3(ext(g, 0, true), ext(g, 1, true), ext(g, 2, true), b);
  if (D == 3)
    k_adv_rhs<3><<<gr, b, 0, s>>>(g, ptr3(uvel), ptr3(rho), ptr3(frc), L0, c_force, flow_axis, G_dev);
  else
    k_adv_rhs<2><<<gr, b, 0, s>>>(g, ptr3(uvel), ptr3(rho), ptr3(frc), L0, c_force, flow_axis, G_dev);
}

void launch_divergence(int D, const Geo& g, double* const u[3], double* b, double scale,
                       Scalars sc, cudaStream_t s, const double* beta_open, double p_out) {
  long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  int nb = red_grid(ncell);
  const double pbc = 2.0 * p_out / (g.h * g.h);
  if (D == 3) k_divergence<3><<<nb, kBlock1D, 0, s>>>(g, ptr3(u), b, scale, sc.partial, beta_open, pbc);
  else k_divergence<2><<<nb, kBlock1D, 0, s>>>(g, ptr3(u), b, scale, sc.partial, beta_open, pbc);
  if (g.open >= 0) return;   // a regular problem: the mean stays
  k_finalize<<<1, 1024, 0, s>>>(sc.partial, nb, sc.out, 0, 1.0 / (double)ncell, 0);
  dim3 bb = blk3(D);
  k_sub_scalar<<<grd3(g.n[0], g.n[1], g.n[2], bb), bb, 0, s>>>(g, b, sc.out);
}

void launch_sub_mean(int D, const Geo& g, double* a, Scalars sc, cudaStream_t s) {
  long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  int nb = red_grid(ncell);
  k_partial_sum<<<nb, kBlock1D, 0, s>>>(g, a, sc.partial);
  k_finalize<<<1, 1024, 0, s>>>(sc.partial, nb, sc.out, 0, 1.0 / (double)ncell, 0);
  dim3 bb = blk3(D);
  k_sub_scalar<<<grd3(g.n[0], g.n[1], g.n[2], bb), bb, 0, s>>>(g, a, sc.out);
}

void launch_project(int D, const Geo& g, double* const ut[3], const double* p,
                    double* const beta[3], double* uvel[3], double coef, const DivCheck& dc,
                    cudaStream_t s) {
  dim3 b = blk3(D);
  dim3 gr = grd3(ext(g, 0, true), ext(g, 1, true), ext(g, 2, true), b);
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(dc.out + dc.acc);
  if (D == 3)
    k_project<3><<<gr, b, 0, s>>>(g, ptr3(ut), p, ptr3(beta), ptr3(uvel), coef, acc, dc.p_out);
  else
    k_project<2><<<gr, b, 0, s>>>(g, ptr3(ut), p, ptr3(beta), ptr3(uvel), coef, acc, dc.p_out);
  k_div_check<<<1, 32, 0, s>>>(dc.out, dc.acc, dc.step, dc.all, dc.tol, dc.viol);
}

void launch_norm2(int D, const Geo& g, double* const a[3], int ncomp, Scalars sc, int slot,
                  cudaStream_t s) {
  long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  int nb = red_grid(ncell);
  if (D == 3) k_norm2<3><<<nb, kBlock1D, 0, s>>>(g, ptr3(a), ncomp, sc.partial);
  else k_norm2<2><<<nb, kBlock1D, 0, s>>>(g, ptr3(a), ncomp, sc.partial);
  k_finalize<<<1, 1024, 0, s>>>(sc.partial, nb, sc.out, slot, 1.0, 0);
}

void launch_div_ke(int D, const Geo& g, double* const u[3], Scalars sc, int slot, cudaStream_t s) {
  long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  int nb = red_grid(ncell);
  double* pmax = sc.partial;
  double* psum = sc.partial + kRedBlocks;
  if (D == 3) k_div_ke<3><<<nb, kBlock1D, 0, s>>>(g, ptr3(u), pmax, psum);
  else k_div_ke<2><<<nb, kBlock1D, 0, s>>>(g, ptr3(u), pmax, psum);
  double hD = D == 3 ? g.h * g.h * g.h : g.h * g.h;
  k_finalize<<<1, 1024, 0, s>>>(pmax, nb, sc.out, slot, 1.0, 1);
  k_finalize<<<1, 1024, 0, s>>>(psum, nb, sc.out, slot + 1, hD, 0);
}

void launch_laminar(int D, const Geo& g, int flow_axis, double mu_eff, double u_center,
                    double body_force, double ic_scale, double* ucomp, double* G_dev,
                    cudaStream_t s) {
  int ta[2] = {0, 0}, q = 0;
  for (int a = 0; a < D; ++a)
    if (a != flow_axis) ta[q++] = a;
  double A = g.n[ta[0]] * g.h, B = (D == 3) ? g.n[ta[1]] * g.h : 0.0;
  k_body_force<<<1, 32, 0, s>>>(D, A, B, mu_eff, u_center, body_force, G_dev);
  int n0 = g.n[ta[0]], n1 = (D == 3) ? g.n[ta[1]] : 1;
  dim3 b(32, 8, 1);
  dim3 gr((n0 + 31) / 32, (n1 + 7) / 8, 1);
  k_laminar<<<gr, b, 0, s>>>(g, D, flow_axis, ta[0], ta[1], mu_eff, ic_scale, G_dev, ucomp);
}

void launch_finalize_sum(const double* partial, int nb, double* out, int slot, double scale,
                         cudaStream_t s) {
  k_finalize<<<1, 1024, 0, s>>>(partial, nb, out, slot, scale, 0);
}

void launch_tol_check(cudaGraphConditionalHandle h, const double* out, int sf, int sr,
                      double rtol, int maxc, int* counter, long long* total, int* nonconv,
                      cudaStream_t s, int smax, double mscale, double mtol) {
  k_tol_check<<<1, 32, 0, s>>>(h, out, sf, sr, rtol, maxc, counter, total, nonconv,
                               smax < 0 ? 0 : smax, mscale, smax < 0 ? 0.0 : mtol);
}

void launch_finalize_max(const double* partial, int nb, double* out, int slot,
                         cudaStream_t s) {
  k_finalize<<<1, 1024, 0, s>>>(partial, nb, out, slot, 1.0, 1);
}

void launch_absmax_cells(int D, const Geo& g, const double* a, Scalars sc, int slot,
                         cudaStream_t s) {
  long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  int nb = red_grid(ncell);
  k_absmax_cells<<<nb, kBlock1D, 0, s>>>(g, a, sc.partial);
  k_finalize<<<1, 1024, 0, s>>>(sc.partial, nb, sc.out, slot, 1.0, 1);
}

void launch_res_check(const double* out, int sf, int sr, double thresh, int* nonconv,
                      cudaStream_t s) {
  k_res_check<<<1, 32, 0, s>>>(out, sf, sr, thresh, nonconv);
}

void launch_fill(double* a, long long n, double v, cudaStream_t s) {
  if (n <= 0) return;
  int nb = red_grid(n);
  k_fill<<<nb, kBlock1D, 0, s>>>(a, n, v);
}

// the block decompositions the single-instance launches use, for the work
// lists of batched launches
int red_grid_of(long long n) { return red_grid(n); }
dim3 stencil_grid3(long long nx, long long ny, long long nz) { return grd3(nx, ny, nz, blk3(3)); }

// ------------------------------------------------------------------ batched
void launch_b_v_residual32(const BArgs& A, int grid, cudaStream_t s) {
  if (A.n > 0) kb_v_residual32<<<grid, blk3(3), 0, s>>>(A);
}
void launch_b_p_residual32(const BArgs& A, int grid, cudaStream_t s) {
  if (A.n > 0) kb_p_residual32<<<grid, blk3(3), 0, s>>>(A);
}
void launch_b_restrict_face32(const BArgs& A, int grid, cudaStream_t s) {
  if (A.n > 0) kb_restrict_face32<<<grid, blk3(3), 0, s>>>(A);
}
void launch_b_restrict_cell32(const BArgs& A, int grid, cudaStream_t s) {
  if (A.n > 0) kb_restrict_cell32<<<grid, blk3(3), 0, s>>>(A);
}
void launch_b_prolong_face32(const BArgs& A, int grid, cudaStream_t s) {
  if (A.n > 0) kb_prolong_face32<<<grid, blk3(3), 0, s>>>(A);
}
void launch_b_prolong_cell32(const BArgs& A, int grid, cudaStream_t s) {
  if (A.n > 0) kb_prolong_cell32<<<grid, blk3(3), 0, s>>>(A);
}
size_t b_coarse_smem(const Geo& g, bool viscous) {
  const size_t b = coarse_bytes(3, g, (int)sizeof(double), viscous);
  return b <= kCoarseSmemMax ? b : 0;
}
void launch_b_coarse(const BArgs& A, bool viscous, size_t smem, cudaStream_t s) {
  if (A.n <= 0) return;
  if (viscous) kb_coarse<true><<<A.n, 1024, smem, s>>>(A);
  else kb_coarse<false><<<A.n, 1024, smem, s>>>(A);
}
cudaError_t b_coarse_set_smem() {
  cudaError_t e = cudaFuncSetAttribute((const void*)kb_coarse<true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kCoarseSmemMax);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)kb_coarse<false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCoarseSmemMax);
  return e;
}
void launch_b_norm2(const BArgs& A, bool viscous, int grid, cudaStream_t s) {
  if (A.n > 0) kb_norm2<<<grid, kBlock1D, 0, s>>>(A, viscous ? 1 : 0);
}
void launch_b_partial_sum_p(const BArgs& A, int grid, cudaStream_t s) {
  if (A.n > 0) kb_partial_sum_p<<<grid, kBlock1D, 0, s>>>(A);
}
void launch_b_sub_scalar_p(const BArgs& A, int grid, cudaStream_t s) {
  if (A.n > 0) kb_sub_scalar_p<<<grid, blk3(3), 0, s>>>(A);
}
void launch_b_finalize(const BArgs& A, int off, int slot, bool is_max, bool mean,
                       cudaStream_t s) {
  if (A.n > 0) kb_finalize<<<A.n, 1024, 0, s>>>(A, off, slot, is_max ? 1 : 0, mean ? 1 : 0);
}
void launch_b_begin(const BMember* tab, int nm, int* act, int which, int zero_slot,
                    cudaStream_t s) {
  if (nm > 0) kb_begin<<<(nm + 255) / 256, 256, 0, s>>>(tab, nm, act, which, zero_slot);
}
void launch_b_tol_check(cudaGraphConditionalHandle h, const BMember* tab, int nm, int* act,
                        int which, int sf, int sr, int smax, long long* iters, cudaStream_t s,
                        bool use_h) {
  kb_tol_check<<<1, 1024, 0, s>>>(h, tab, nm, act, which, sf, sr, smax, iters, use_h ? 1 : 0);
}
void launch_b_res_check(const BMember* tab, int nm, int sf, int sr, double slack,
                        cudaStream_t s) {
  if (nm > 0) kb_res_check<<<(nm + 255) / 256, 256, 0, s>>>(tab, nm, sf, sr, slack);
}

size_t tail_smem(const Geo& coarsest, bool viscous) { return b_coarse_smem(coarsest, viscous); }

cudaError_t tail_set_smem() {
  cudaError_t e = cudaSuccess;
  for (const void* f : {(const void*)k_tail<true>, (const void*)k_tail<false>,
                        (const void*)k_tail1<true>, (const void*)k_tail1<false>})
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kCoarseSmemMax);
  return e;
}

void launch_tail(bool viscous, const BMember* tab, const int* list, int nlist, const int* act,
                 size_t smem, cudaStream_t s, int ctas) {
  if (nlist <= 0) return;
  if (ctas == 1) {
    if (viscous) k_tail1<true><<<nlist, kTailThreads<true>, smem, s>>>(tab, list, nlist, act);
    else k_tail1<false><<<nlist, kTailThreads<false>, smem, s>>>(tab, list, nlist, act);
  } else {
    if (viscous)
      k_tail<true><<<nlist * kTailCtas, kTailThreads<true>, smem, s>>>(tab, list, nlist, act);
    else
      k_tail<false><<<nlist * kTailCtas, kTailThreads<false>, smem, s>>>(tab, list, nlist, act);
  }
}

}  // namespace bf
