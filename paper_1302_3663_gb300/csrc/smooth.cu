// Fused red-black Gauss-Seidel sweeps (Sec. 3.5): one kernel pass updates
// both colours, so every array is read from DRAM once per sweep instead of
// once per colour.
//
// A block owns full x rows, TY rows of the row axis (y in 3D) and a chunk of
// planes along the streaming axis (z in 3D, y in 2D). It walks the chunk
// plane by plane: first the new red values of plane k on its rows plus one
// ring row on each side (red points depend only on old black values), kept in
// a three-plane shared-memory ring; then the black values of plane k-1, which
// need the new red values of planes k-2, k-1, k. The sweep is out of place:
// old values are read from one buffer and both colours are written to
// another, so neighbouring blocks (which recompute the shared ring rows and
// the first plane of a chunk) never read a value another block has already
// replaced. The arithmetic of every point update is that of the two-kernel
// sweep in stencil.cu.
#include <cuda_runtime.h>

#include "common.cuh"

namespace bf {

namespace {

__host__ __device__ constexpr int edge_id(int d, int e) {
  return (d < e ? d : e) + (d < e ? e : d) - 1;
}

__device__ __forceinline__ long long offp(const Geo& g, int a, int ci) {
  return (g.per[a] && ci == g.n[a] - 1) ? -(long long)(g.n[a] - 1) * g.st[a] : g.st[a];
}
__device__ __forceinline__ long long offm(const Geo& g, int a, int ci) {
  return (g.per[a] && ci == 0) ? (long long)(g.n[a] - 1) * g.st[a] : -g.st[a];
}
__device__ __forceinline__ int wrapi(int i, int n) { return ((i % n) + n) % n; }

template <int D>
struct Ax {
  static constexpr int R = (D == 3) ? 1 : 2;   // row axis (a size-1 dummy in 2D)
  static constexpr int S = (D == 3) ? 2 : 1;   // streaming axis
  static constexpr int RING = (D == 3) ? 1 : 0;
};

// Per-thread view of the three-plane ring of new red values.
template <typename T>
struct Ring {
  T* buf;
  int nrow, W;
  __device__ __forceinline__ T* row(int slot, int r) const { return buf + (slot * nrow + r) * W; }
};

__device__ __forceinline__ int slot_of(int k) { return ((k % 3) + 3) % 3; }

// ---------------------------------------------------------------------------
// Pressure: red from the old black values (global), black from the new red
// values (shared). Neighbours are summed axis 0, 1, 2, lower then upper, as
// in the two-kernel sweep.
// ---------------------------------------------------------------------------
template <int D, typename T>
__device__ __forceinline__ T p_red(const Geo& g, const LevelPtrs<T>& L, const int ci[3],
                                   long long c, T h2) {
  T num = T(0), dg = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const T* __restrict__ b = L.beta[a];
    if (ci[a] > 0 || g.per[a]) {
      T bb = b[c];
      num += bb * L.p[c + offm(g, a, ci[a])];
      dg += bb;
    }
    if (ci[a] < g.n[a] - 1 || g.per[a]) {
      long long cp = c + offp(g, a, ci[a]);
      T bb = b[cp];
      num += bb * L.p[cp];
      dg += bb;
    }
  }
  return (num - h2 * L.pf[c]) / dg;
}

template <int D, typename T>
__device__ __forceinline__ T p_black(const Geo& g, const LevelPtrs<T>& L, const Ring<T>& rg,
                                     const int ci[3], long long c, int r, int sl_m, int sl_0,
                                     int sl_p, T h2) {
  constexpr int RA = Ax<D>::R, SA = Ax<D>::S;
  T num = T(0), dg = T(0);
  const T* here = rg.row(sl_0, r);
  int i = ci[0], n0 = g.n[0];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const T* __restrict__ b = L.beta[a];
    bool hm = ci[a] > 0 || g.per[a];
    bool hp = ci[a] < g.n[a] - 1 || g.per[a];
    T vm = T(0), vp = T(0);
    if (a == 0) {
      if (hm) vm = here[i > 0 ? i - 1 : n0 - 1];
      if (hp) vp = here[i < n0 - 1 ? i + 1 : 0];
    } else if (a == RA) {
      if (hm) vm = rg.row(sl_0, r - 1)[i];
      if (hp) vp = rg.row(sl_0, r + 1)[i];
    } else {  // a == SA
      if (hm) vm = rg.row(sl_m, r)[i];
      if (hp) vp = rg.row(sl_p, r)[i];
    }
    if (hm) {
      T bb = b[c];
      num += bb * vm;
      dg += bb;
    }
    if (hp) {
      T bb = b[c + offp(g, a, ci[a])];
      num += bb * vp;
      dg += bb;
    }
  }
  (void)SA;
  return (num - h2 * L.pf[c]) / dg;
}

template <int D, typename T>
__global__ void __launch_bounds__(1024) k_p_rb_fused(Geo g, LevelPtrs<T> L, T* __restrict__ out,
                                                     int TY, int KC) {
  constexpr int RA = Ax<D>::R, SA = Ax<D>::S, RING = Ax<D>::RING;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  Ring<T> rg{reinterpret_cast<T*>(sm_raw), TY + 2 * RING, g.s[0]};
  const int n0 = g.n[0], nR = g.n[RA], nS = g.n[SA];
  const int j0 = blockIdx.x * TY;
  const int k0 = blockIdx.y * KC;
  const int k1 = min(k0 + KC, nS);
  const int r = threadIdx.y;
  const int j = j0 + r - RING;
  int jw = j;
  bool rowvalid = true;
  if (g.per[RA]) jw = wrapi(j, nR);
  else rowvalid = (j >= 0 && j < nR);
  const bool tilerow = (r >= RING && r < RING + TY && j < nR);
  const T h2 = (T)(g.h * g.h);
  const int nthr = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int q = tid; q < 3 * rg.nrow * rg.W; q += nthr) rg.buf[q] = T(0);
  __syncthreads();
  for (int k = k0 - 1; k <= k1; ++k) {
    // new red values of plane k on every row of the block (ring included)
    T* row = rg.row(slot_of(k), r);
    int kw = k;
    bool planevalid = true;
    if (g.per[SA]) kw = wrapi(k, nS);
    else planevalid = (k >= 0 && k < nS);
    if (planevalid && rowvalid) {
      for (int ip = threadIdx.x; 2 * ip < n0; ip += blockDim.x) {
        int ci[3];
        ci[RA] = jw;
        ci[SA] = kw;
        int par = (ci[1] + ci[2]) & 1;
        ci[0] = 2 * ip + par;          // the red point of this pair
        if (ci[0] < n0) row[ci[0]] = p_red<D, T>(g, L, ci, gidx(g, ci[0], ci[1], ci[2]), h2);
      }
    } else {
      for (int i = threadIdx.x; i < rg.W; i += blockDim.x) row[i] = T(0);
    }
    __syncthreads();
    // black values of plane k - 1 on the block's own rows; both colours out
    const int kb = k - 1;
    if (kb >= k0 && tilerow) {
      const int sl_m = slot_of(kb - 1), sl_0 = slot_of(kb), sl_p = slot_of(kb + 1);
      const T* here = rg.row(sl_0, r);
      for (int ip = threadIdx.x; 2 * ip < n0; ip += blockDim.x) {
        int ci[3];
        ci[RA] = jw;
        ci[SA] = kb;
        int par = (ci[1] + ci[2]) & 1;
        int ir = 2 * ip + par, ib = 2 * ip + (par ^ 1);
        if (ir < n0) out[gidx(g, ir, ci[1], ci[2])] = here[ir];
        if (ib < n0) {
          ci[0] = ib;
          long long c = gidx(g, ib, ci[1], ci[2]);
          out[c] = p_black<D, T>(g, L, rg, ci, c, r, sl_m, sl_0, sl_p, h2);
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Viscous component d. Neighbour coefficients and the cross-component part
// come from the coefficient arrays and the (fixed) other components; the u_d
// neighbours come from the old buffer (red) or the ring (black).
// ---------------------------------------------------------------------------
template <int D, int d, typename T>
struct VC {
  T cdp, cdm;          // 2 mu_c on the cells beside the face
  T cep[2], cem[2];    // edge mu per other axis (the neighbour beyond a wall is unused)
  bool wp[2], wm[2];   // that neighbour lies beyond a wall (mirror ghost)
  T cross, diag;
};

template <int D, int d, typename T>
__device__ __forceinline__ void v_coef(const Geo& g, const LevelPtrs<T>& L, const int ci[3],
                                       long long F, T ir, VC<D, d, T>& v) {
  long long od_m = offm(g, d, ci[d]);
  T mcp = L.muc[F], mcm = L.muc[F + od_m];
  v.cdp = T(2) * mcp;
  v.cdm = T(2) * mcm;
  T dgV = T(2) * (mcp + mcm);
  v.cross = T(0);
  int q = 0;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    if (e == d) continue;
    const T* __restrict__ ue = L.u[e];
    const T* __restrict__ me = L.mue[edge_id(d, e)];
    bool pe = g.per[e] != 0;
    bool wp = !pe && ci[e] == g.n[e] - 1;
    bool wm = !pe && ci[e] == 0;
    long long Ep = F + offp(g, e, ci[e]);
    T mep = me[Ep], mem = me[F];
    v.cross += mep * (ue[Ep] - ue[Ep + od_m]) - mem * (ue[F] - ue[F + od_m]);
    v.cep[q] = mep;
    v.cem[q] = mem;
    v.wp[q] = wp;
    v.wm[q] = wm;
    dgV += (wp ? T(2) : T(1)) * mep + (wm ? T(2) : T(1)) * mem;
    ++q;
  }
  v.diag = L.m[d][F] + ir * dgV;
}

template <int D, int d, typename T>
__device__ __forceinline__ T v_red(const Geo& g, const LevelPtrs<T>& L, const int ci[3],
                                   long long F, T ir) {
  VC<D, d, T> v;
  v_coef<D, d, T>(g, L, ci, F, ir, v);
  const T* __restrict__ ud = L.u[d];
  T off = v.cross + v.cdp * ud[F + offp(g, d, ci[d])] + v.cdm * ud[F + offm(g, d, ci[d])];
  int q = 0;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    if (e == d) continue;
    if (!v.wp[q]) off += v.cep[q] * ud[F + offp(g, e, ci[e])];
    if (!v.wm[q]) off += v.cem[q] * ud[F + offm(g, e, ci[e])];
    ++q;
  }
  return (L.uf[d][F] + ir * off) / v.diag;
}

// u_d at the neighbour of ci one step along axis a (side +1/-1) from the ring
template <int D, typename T>
__device__ __forceinline__ T ring_nb(const Geo& g, const Ring<T>& rg, const int ci[3], int a,
                                     int side, int r, int sl_m, int sl_0, int sl_p) {
  constexpr int RA = Ax<D>::R;
  if (a == 0) {
    int i = ci[0] + side;
    if (g.per[0]) i = wrapi(i, g.n[0]);
    return rg.row(sl_0, r)[i];
  }
  if (a == RA) return rg.row(sl_0, r + side)[ci[0]];
  return rg.row(side > 0 ? sl_p : sl_m, r)[ci[0]];
}

template <int D, int d, typename T>
__device__ __forceinline__ T v_black(const Geo& g, const LevelPtrs<T>& L, const Ring<T>& rg,
                                     const int ci[3], long long F, T ir, int r, int sl_m,
                                     int sl_0, int sl_p) {
  VC<D, d, T> v;
  v_coef<D, d, T>(g, L, ci, F, ir, v);
  T off = v.cross + v.cdp * ring_nb<D, T>(g, rg, ci, d, +1, r, sl_m, sl_0, sl_p) +
          v.cdm * ring_nb<D, T>(g, rg, ci, d, -1, r, sl_m, sl_0, sl_p);
  int q = 0;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    if (e == d) continue;
    if (!v.wp[q]) off += v.cep[q] * ring_nb<D, T>(g, rg, ci, e, +1, r, sl_m, sl_0, sl_p);
    if (!v.wm[q]) off += v.cem[q] * ring_nb<D, T>(g, rg, ci, e, -1, r, sl_m, sl_0, sl_p);
    ++q;
  }
  return (L.uf[d][F] + ir * off) / v.diag;
}

template <int D, int d, typename T>
__global__ void __launch_bounds__(1024) k_v_rb_fused(Geo g, LevelPtrs<T> L, T* __restrict__ out,
                                                     int TY, int KC, T ir) {
  constexpr int RA = Ax<D>::R, SA = Ax<D>::S, RING = Ax<D>::RING;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  Ring<T> rg{reinterpret_cast<T*>(sm_raw), TY + 2 * RING, g.s[0]};
  const int n0 = g.n[0], nR = g.n[RA], nS = g.n[SA];
  const int j0 = blockIdx.x * TY;
  const int k0 = blockIdx.y * KC;
  const int k1 = min(k0 + KC, nS);
  const int r = threadIdx.y;
  const int j = j0 + r - RING;
  int jw = j;
  bool rowvalid = true;
  if (g.per[RA]) jw = wrapi(j, nR);
  else rowvalid = (j >= 0 && j < nR);
  const bool tilerow = (r >= RING && r < RING + TY && j < nR);
  const bool wall_d = !g.per[d];
  const int nthr = blockDim.x * blockDim.y, tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int q = tid; q < 3 * rg.nrow * rg.W; q += nthr) rg.buf[q] = T(0);
  __syncthreads();
  for (int k = k0 - 1; k <= k1; ++k) {
    T* row = rg.row(slot_of(k), r);
    int kw = k;
    bool planevalid = true;
    if (g.per[SA]) kw = wrapi(k, nS);
    else planevalid = (k >= 0 && k < nS);
    if (planevalid && rowvalid) {
      for (int ip = threadIdx.x; 2 * ip < n0; ip += blockDim.x) {
        int ci[3];
        ci[RA] = jw;
        ci[SA] = kw;
        int par = (ci[1] + ci[2]) & 1;
        ci[0] = 2 * ip + par;
        if (ci[0] >= n0) continue;
        T v = T(0);   // wall faces hold 0
        if (!(wall_d && ci[d] == 0)) v = v_red<D, d, T>(g, L, ci, gidx(g, ci[0], ci[1], ci[2]), ir);
        row[ci[0]] = v;
      }
    } else {
      for (int i = threadIdx.x; i < rg.W; i += blockDim.x) row[i] = T(0);
    }
    __syncthreads();
    const int kb = k - 1;
    if (kb >= k0 && tilerow) {
      const int sl_m = slot_of(kb - 1), sl_0 = slot_of(kb), sl_p = slot_of(kb + 1);
      const T* here = rg.row(sl_0, r);
      for (int ip = threadIdx.x; 2 * ip < n0; ip += blockDim.x) {
        int ci[3];
        ci[RA] = jw;
        ci[SA] = kb;
        int par = (ci[1] + ci[2]) & 1;
        int irr = 2 * ip + par, ib = 2 * ip + (par ^ 1);
        if (irr < n0) out[gidx(g, irr, ci[1], ci[2])] = here[irr];
        if (ib < n0) {
          ci[0] = ib;
          long long F = gidx(g, ib, ci[1], ci[2]);
          T v = T(0);
          if (!(wall_d && ci[d] == 0)) v = v_black<D, d, T>(g, L, rg, ci, F, ir, r, sl_m, sl_0, sl_p);
          out[F] = v;
        }
      }
    }
    __syncthreads();
  }
}

struct FusedShape {
  dim3 grid, block;
  int TY, KC;
  size_t smem;
};

template <typename T>
FusedShape fused_shape(int D, const Geo& g) {
  FusedShape f;
  int RA = (D == 3) ? 1 : 2, SA = (D == 3) ? 2 : 1;
  int ring = (D == 3) ? 1 : 0;
  int npairs = (g.n[0] + 1) / 2;
  int bx = ((npairs + 31) / 32) * 32;
  if (bx > 128) bx = 128;
  f.TY = (D == 3) ? (g.n[RA] >= 8 ? 8 : g.n[RA]) : 1;
  while (bx * (f.TY + 2 * ring) > 1024 && f.TY > 1) --f.TY;
  while ((size_t)3 * (f.TY + 2 * ring) * g.s[0] * sizeof(T) > 48 * 1024 && f.TY > 1) --f.TY;
  int nrt = (g.n[RA] + f.TY - 1) / f.TY;
  // aim for several blocks per SM while keeping the recomputed first plane of
  // each chunk a small fraction of the work
  long long want = 4LL * 152;
  int KC = (int)((long long)g.n[SA] * nrt / want);
  if (KC < 4) KC = 4;
  if (KC > g.n[SA]) KC = g.n[SA];
  f.KC = KC;
  f.block = dim3(bx, f.TY + 2 * ring, 1);
  f.grid = dim3(nrt, (g.n[SA] + KC - 1) / KC, 1);
  f.smem = (size_t)3 * (f.TY + 2 * ring) * g.s[0] * sizeof(T);
  return f;
}

}  // namespace

template <typename T>
void launch_p_rb_fused(int D, const Geo& g, const LevelPtrs<T>& L, T* out, cudaStream_t s) {
  FusedShape f = fused_shape<T>(D, g);
  if (D == 3) k_p_rb_fused<3, T><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC);
  else k_p_rb_fused<2, T><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC);
}

template <typename T>
void launch_v_rb_fused(int D, const Geo& g, const LevelPtrs<T>& L, int d, T* out, double inv_re,
                       cudaStream_t s) {
  FusedShape f = fused_shape<T>(D, g);
  T ir = (T)(inv_re / (g.h * g.h));
  if (D == 3) {
    if (d == 0) k_v_rb_fused<3, 0, T><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC, ir);
    else if (d == 1) k_v_rb_fused<3, 1, T><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC, ir);
    else k_v_rb_fused<3, 2, T><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC, ir);
  } else {
    if (d == 0) k_v_rb_fused<2, 0, T><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC, ir);
    else k_v_rb_fused<2, 1, T><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC, ir);
  }
}

size_t fused_smem_bytes(int D, const Geo& g, int elem) {
  return elem == 8 ? fused_shape<double>(D, g).smem : fused_shape<float>(D, g).smem;
}

template void launch_p_rb_fused<double>(int, const Geo&, const LevelPtrs<double>&, double*,
                                        cudaStream_t);
template void launch_p_rb_fused<float>(int, const Geo&, const LevelPtrs<float>&, float*,
                                       cudaStream_t);
template void launch_v_rb_fused<double>(int, const Geo&, const LevelPtrs<double>&, int, double*,
                                        double, cudaStream_t);
template void launch_v_rb_fused<float>(int, const Geo&, const LevelPtrs<float>&, int, float*,
                                       double, cudaStream_t);

}  // namespace bf
