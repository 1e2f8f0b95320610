// Fused red-black Gauss-Seidel sweeps (Sec. 3.5): one kernel pass updates
// both colours, so every array is read from DRAM once per sweep instead of
// once per colour.
//
// A block owns full x rows, TY rows of the row axis (y in 3D) and a chunk of
// planes along the streaming axis (z in 3D, y in 2D). It walks the chunk NP
// planes at a time: first the new red values of NP planes on its rows plus
// one ring row on each side (red points depend only on old black values, so
// the NP updates are independent), kept in a ring of NP + 2 planes in shared
// memory; then the black values of the NP planes one behind, which need the
// new red values of the planes below, at and above them. The sweep is out of
// place: old values are read from one buffer and both colours are written to
// another, so neighbouring blocks (which recompute the shared ring rows and
// the first plane of a chunk) never read a value another block has already
// replaced. The arithmetic of every point update is that of the two-kernel
// sweep in stencil.cu, except that FP32 viscous updates multiply by a
// precomputed inverse diagonal instead of dividing by the diagonal.
#include <cuda_runtime.h>

#include "common.cuh"

namespace bf {

namespace {

__host__ __device__ constexpr int edge_id(int d, int e) {
  return (d < e ? d : e) + (d < e ? e : d) - 1;
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

// Offsets (32-bit, within one level array) of a point's six neighbours and
// its wall flags, computed once per point update. op/om wrap on periodic
// axes; on a wall axis om of the first and op of the last index point beyond
// the grid and are flagged by wm/wp.
struct Pt {
  int F;
  int op[3], om[3];
  bool wp[3], wm[3];
};

template <int D>
__device__ __forceinline__ void make_pt(const Geo& g, const int ci[3], Pt& q) {
  const int st[3] = {1, (int)g.st[1], (int)g.st[2]};
  q.F = ci[0] + st[1] * ci[1] + st[2] * ci[2];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a >= D) {
      q.op[a] = q.om[a] = 0;
      q.wp[a] = q.wm[a] = true;
      continue;
    }
    bool last = ci[a] == g.n[a] - 1, first = ci[a] == 0;
    bool per = g.per[a] != 0;
    q.op[a] = (per && last) ? -(g.n[a] - 1) * st[a] : st[a];
    q.om[a] = (per && first) ? (g.n[a] - 1) * st[a] : -st[a];
    q.wp[a] = !per && last;
    q.wm[a] = !per && first;
  }
}

// ---------------------------------------------------------------------------
// Pressure: red from the old black values (global), black from the new red
// values (shared). Neighbours are summed axis 0, 1, 2, lower then upper, as
// in the two-kernel sweep.
// ---------------------------------------------------------------------------
template <int D, typename T>
__device__ __forceinline__ T p_red(const LevelPtrs<T>& L, const Pt& q, T h2) {
  T num = T(0), dg = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const T* __restrict__ b = L.beta[a];
    if (!q.wm[a]) {
      T bb = b[q.F];
      num += bb * L.p[q.F + q.om[a]];
      dg += bb;
    }
    if (!q.wp[a]) {
      T bb = b[q.F + q.op[a]];
      num += bb * L.p[q.F + q.op[a]];
      dg += bb;
    }
  }
  return (num - h2 * L.pf[q.F]) / dg;
}

// the new red value of a neighbour of the black point: from the ring row of
// this plane (x, row axis) or of the planes before and after (streaming axis)
template <int D, typename T>
__device__ __forceinline__ T ring_nb(const Ring<T>& rg, const Pt& q, int i, int n0, int a,
                                     int side, int r, int sl_m, int sl_0, int sl_p) {
  constexpr int RA = Ax<D>::R;
  if (a == 0) {
    int ii = i + side;
    if (ii < 0) ii += n0;
    else if (ii >= n0 && q.op[0] < 0) ii -= n0;   // periodic wrap (op < 0 only then)
    return rg.row(sl_0, r)[ii];
  }
  if (a == RA) return rg.row(sl_0, r + side)[i];
  return rg.row(side > 0 ? sl_p : sl_m, r)[i];
}

template <int D, typename T>
__device__ __forceinline__ T p_black(const LevelPtrs<T>& L, const Ring<T>& rg, const Pt& q,
                                     int i, int n0, int r, int sl_m, int sl_0, int sl_p, T h2) {
  T num = T(0), dg = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const T* __restrict__ b = L.beta[a];
    if (!q.wm[a]) {
      T bb = b[q.F];
      num += bb * ring_nb<D, T>(rg, q, i, n0, a, -1, r, sl_m, sl_0, sl_p);
      dg += bb;
    }
    if (!q.wp[a]) {
      T bb = b[q.F + q.op[a]];
      num += bb * ring_nb<D, T>(rg, q, i, n0, a, +1, r, sl_m, sl_0, sl_p);
      dg += bb;
    }
  }
  return (num - h2 * L.pf[q.F]) / dg;
}

// NP planes per iteration: the red values of planes k .. k+NP-1 (independent
// of one another, so their loads overlap), a barrier, then the black values
// of planes k-1 .. k+NP-2; the ring holds NP + 2 planes.
__device__ __forceinline__ int add_mod(int s, int o, int R) {
  int v = s + o;
  return v >= R ? v - R : (v < 0 ? v + R : v);
}

template <int D, typename T, int NP>
__global__ void __launch_bounds__(1024) k_p_rb_fused(Geo g, LevelPtrs<T> L, T* __restrict__ out,
                                                     int TY, int KC) {
  constexpr int RA = Ax<D>::R, SA = Ax<D>::S, RING = Ax<D>::RING;
  constexpr int R = NP + 2;
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
  for (int q = tid; q < R * rg.nrow * rg.W; q += nthr) rg.buf[q] = T(0);
  __syncthreads();
  // ring slot and wrapped index of plane k, advanced by NP planes per
  // iteration (no division per point); plane k0 - 2 sits in slot 0
  int sk = 1;
  int kw = g.per[SA] ? wrapi(k0 - 1, nS) : k0 - 1;
  for (int k = k0 - 1; k <= k1; k += NP) {
    // new red values of planes k .. k + NP - 1 on every row of the block
    bool live[NP];
    int kwo[NP];
#pragma unroll
    for (int o = 0; o < NP; ++o) {
      const int p = k + o;
      kwo[o] = (g.per[SA] && kw + o >= nS) ? kw + o - nS : kw + o;
      live[o] = p <= k1 && rowvalid && (g.per[SA] || (p >= 0 && p < nS));
      if (p <= k1 && !live[o]) {
        T* row = rg.row(add_mod(sk, o, R), r);
        for (int i = threadIdx.x; i < rg.W; i += blockDim.x) row[i] = T(0);
      }
    }
    for (int ip = threadIdx.x; 2 * ip < n0; ip += blockDim.x) {
#pragma unroll
      for (int o = 0; o < NP; ++o) {
        if (!live[o]) continue;
        int ci[3];
        ci[RA] = jw;
        ci[SA] = kwo[o];
        ci[0] = 2 * ip + ((ci[1] + ci[2]) & 1);   // the red point of this pair
        if (ci[0] < n0) {
          Pt q;
          make_pt<D>(g, ci, q);
          rg.row(add_mod(sk, o, R), r)[ci[0]] = p_red<D, T>(L, q, h2);
        }
      }
    }
    __syncthreads();
    // black values of planes k - 1 .. k + NP - 2 on the block's own rows;
    // both colours out
    if (tilerow) {
      for (int ip = threadIdx.x; 2 * ip < n0; ip += blockDim.x) {
#pragma unroll
        for (int o = 0; o < NP; ++o) {
          const int kb = k - 1 + o;
          if (kb < k0 || kb >= k1) continue;
          const int sl_m = add_mod(sk, o - 2, R), sl_0 = add_mod(sk, o - 1, R),
                    sl_p = add_mod(sk, o, R);
          const T* here = rg.row(sl_0, r);
          int ci[3];
          ci[RA] = jw;
          ci[SA] = kb;
          int par = (ci[1] + ci[2]) & 1;
          int ir = 2 * ip + par, ib = 2 * ip + (par ^ 1);
          if (ir < n0) out[ir + (int)g.st[1] * ci[1] + (int)g.st[2] * ci[2]] = here[ir];
          if (ib < n0) {
            ci[0] = ib;
            Pt q;
            make_pt<D>(g, ci, q);
            out[q.F] = p_black<D, T>(L, rg, q, ib, n0, r, sl_m, sl_0, sl_p, h2);
          }
        }
      }
    }
    __syncthreads();
    sk = add_mod(sk, NP, R);
    kw += NP;
    if (g.per[SA] && kw >= nS) kw -= nS;
  }
}

// ---------------------------------------------------------------------------
// Viscous component d. Neighbour coefficients and the cross-component part
// come from the coefficient arrays and the (fixed) other components; the u_d
// neighbours come from the old buffer (red) or the ring (black).
// ---------------------------------------------------------------------------
// FP32 sweeps multiply by the precomputed 1 / diagonal (L.idg, formed in
// FP64 once per step); FP64 sweeps form the diagonal and divide, as the
// two-kernel sweep does.
template <typename T>
constexpr bool kIdg = sizeof(T) == 4;

template <int D, int d, typename T>
struct VC {
  T cdp, cdm;          // 2 mu_c on the cells beside the face
  T cep[2], cem[2];    // edge mu per other axis (the neighbour beyond a wall is unused)
  T cross, diag;       // diag: the diagonal (FP64) or its inverse (FP32)
};

template <int D, int d, typename T>
__device__ __forceinline__ void v_coef(const LevelPtrs<T>& L, const Pt& q, T ir, VC<D, d, T>& v) {
  const int F = q.F, od_m = q.om[d];
  T mcp = L.muc[F], mcm = L.muc[F + od_m];
  v.cdp = T(2) * mcp;
  v.cdm = T(2) * mcm;
  T dgV = T(2) * (mcp + mcm);
  v.cross = T(0);
  int k = 0;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    if (e == d) continue;
    const T* __restrict__ ue = L.u[e];
    const T* __restrict__ me = L.mue[edge_id(d, e)];
    const int Ep = F + q.op[e];
    T mep = me[Ep], mem = me[F];
    v.cross += mep * (ue[Ep] - ue[Ep + od_m]) - mem * (ue[F] - ue[F + od_m]);
    v.cep[k] = mep;
    v.cem[k] = mem;
    if constexpr (!kIdg<T>) dgV += (q.wp[e] ? T(2) : T(1)) * mep + (q.wm[e] ? T(2) : T(1)) * mem;
    ++k;
  }
  if constexpr (kIdg<T>) v.diag = L.idg[d][F];
  else v.diag = L.m[d][F] + ir * dgV;
}

template <typename T>
__device__ __forceinline__ T v_solve(T num, T diag) {
  if constexpr (kIdg<T>) return num * diag;
  else return num / diag;
}

template <int D, int d, typename T>
__device__ __forceinline__ T v_red(const LevelPtrs<T>& L, const Pt& q, T ir) {
  VC<D, d, T> v;
  v_coef<D, d, T>(L, q, ir, v);
  const T* __restrict__ ud = L.u[d];
  T off = v.cross + v.cdp * ud[q.F + q.op[d]] + v.cdm * ud[q.F + q.om[d]];
  int k = 0;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    if (e == d) continue;
    if (!q.wp[e]) off += v.cep[k] * ud[q.F + q.op[e]];
    if (!q.wm[e]) off += v.cem[k] * ud[q.F + q.om[e]];
    ++k;
  }
  return v_solve<T>(L.uf[d][q.F] + ir * off, v.diag);
}

template <int D, int d, typename T>
__device__ __forceinline__ T v_black(const LevelPtrs<T>& L, const Ring<T>& rg, const Pt& q,
                                     int i, int n0, T ir, int r, int sl_m, int sl_0, int sl_p) {
  VC<D, d, T> v;
  v_coef<D, d, T>(L, q, ir, v);
  // along d a wall neighbour is the stored zero face: the ring holds 0 there
  T off = v.cross + v.cdp * ring_nb<D, T>(rg, q, i, n0, d, +1, r, sl_m, sl_0, sl_p) +
          v.cdm * ring_nb<D, T>(rg, q, i, n0, d, -1, r, sl_m, sl_0, sl_p);
  int k = 0;
#pragma unroll
  for (int e = 0; e < D; ++e) {
    if (e == d) continue;
    if (!q.wp[e]) off += v.cep[k] * ring_nb<D, T>(rg, q, i, n0, e, +1, r, sl_m, sl_0, sl_p);
    if (!q.wm[e]) off += v.cem[k] * ring_nb<D, T>(rg, q, i, n0, e, -1, r, sl_m, sl_0, sl_p);
    ++k;
  }
  return v_solve<T>(L.uf[d][q.F] + ir * off, v.diag);
}

template <int D, int d, typename T, int NP>
__global__ void __launch_bounds__(1024) k_v_rb_fused(Geo g, LevelPtrs<T> L, T* __restrict__ out,
                                                     int TY, int KC, T ir) {
  constexpr int RA = Ax<D>::R, SA = Ax<D>::S, RING = Ax<D>::RING;
  constexpr int R = NP + 2;
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
  for (int q = tid; q < R * rg.nrow * rg.W; q += nthr) rg.buf[q] = T(0);
  __syncthreads();
  int sk = 1;
  int kw = g.per[SA] ? wrapi(k0 - 1, nS) : k0 - 1;
  for (int k = k0 - 1; k <= k1; k += NP) {
    bool live[NP];
    int kwo[NP];
#pragma unroll
    for (int o = 0; o < NP; ++o) {
      const int p = k + o;
      kwo[o] = (g.per[SA] && kw + o >= nS) ? kw + o - nS : kw + o;
      live[o] = p <= k1 && rowvalid && (g.per[SA] || (p >= 0 && p < nS));
      if (p <= k1 && !live[o]) {
        T* row = rg.row(add_mod(sk, o, R), r);
        for (int i = threadIdx.x; i < rg.W; i += blockDim.x) row[i] = T(0);
      }
    }
    for (int ip = threadIdx.x; 2 * ip < n0; ip += blockDim.x) {
#pragma unroll
      for (int o = 0; o < NP; ++o) {
        if (!live[o]) continue;
        int ci[3];
        ci[RA] = jw;
        ci[SA] = kwo[o];
        ci[0] = 2 * ip + ((ci[1] + ci[2]) & 1);
        if (ci[0] >= n0) continue;
        T v = T(0);   // wall faces hold 0
        if (!(wall_d && ci[d] == 0)) {
          Pt q;
          make_pt<D>(g, ci, q);
          v = v_red<D, d, T>(L, q, ir);
        }
        rg.row(add_mod(sk, o, R), r)[ci[0]] = v;
      }
    }
    __syncthreads();
    if (tilerow) {
      for (int ip = threadIdx.x; 2 * ip < n0; ip += blockDim.x) {
#pragma unroll
        for (int o = 0; o < NP; ++o) {
          const int kb = k - 1 + o;
          if (kb < k0 || kb >= k1) continue;
          const int sl_m = add_mod(sk, o - 2, R), sl_0 = add_mod(sk, o - 1, R),
                    sl_p = add_mod(sk, o, R);
          const T* here = rg.row(sl_0, r);
          int ci[3];
          ci[RA] = jw;
          ci[SA] = kb;
          int par = (ci[1] + ci[2]) & 1;
          int irr = 2 * ip + par, ib = 2 * ip + (par ^ 1);
          if (irr < n0) out[irr + (int)g.st[1] * ci[1] + (int)g.st[2] * ci[2]] = here[irr];
          if (ib < n0) {
            ci[0] = ib;
            Pt q;
            make_pt<D>(g, ci, q);
            T v = T(0);
            if (!(wall_d && ci[d] == 0))
              v = v_black<D, d, T>(L, rg, q, ib, n0, ir, r, sl_m, sl_0, sl_p);
            out[q.F] = v;
          }
        }
      }
    }
    __syncthreads();
    sk = add_mod(sk, NP, R);
    kw += NP;
    if (g.per[SA] && kw >= nS) kw -= nS;
  }
}

struct FusedShape {
  dim3 grid, block;
  int TY, KC;
  size_t smem;
};

// Tile rows TYo, chunk planes KCo and threads per row BXo (3D) come from the
// autotuner when it has timed this level shape; 0 selects the built-in
// heuristic. A row of fewer threads than point pairs has each thread update
// several pairs per phase.
template <typename T>
FusedShape fused_shape(int D, const Geo& g, int TYo = 0, int KCo = 0, int NP = 1, int BXo = 0) {
  FusedShape f;
  int RA = (D == 3) ? 1 : 2, SA = (D == 3) ? 2 : 1;
  int ring = (D == 3) ? 1 : 0;
  int npairs = (g.n[0] + 1) / 2;
  int bx = ((npairs + 31) / 32) * 32;
  if (bx > 128) bx = 128;
  if (D == 3 && BXo >= 32 && BXo < bx) bx = BXo / 32 * 32;
  // 4 rows (+2 ring rows) keep blocks small enough for several per SM
  f.TY = (D == 3) ? (g.n[RA] >= 4 ? 4 : g.n[RA]) : 1;
  if (D == 3 && TYo > 0) f.TY = TYo < g.n[RA] ? TYo : g.n[RA];
  while (bx * (f.TY + 2 * ring) > 1024 && f.TY > 1) --f.TY;
  while ((size_t)(NP + 2) * (f.TY + 2 * ring) * g.s[0] * sizeof(T) > 48 * 1024 && f.TY > 1) --f.TY;
  int nrt = (g.n[RA] + f.TY - 1) / f.TY;
  // about three blocks per SM in flight, with chunks of at most 16 planes so
  // that the recomputed first plane of a chunk stays a small fraction
  long long want = 3LL * 152;
  int KC = (int)((long long)g.n[SA] * nrt / want);
  if (KC < 4) KC = 4;
  if (KC > 16) KC = 16;
  if (D == 3 && KCo > 0) KC = KCo;
  if (KC > g.n[SA]) KC = g.n[SA];
  f.KC = KC;
  f.block = dim3(bx, f.TY + 2 * ring, 1);
  f.grid = dim3(nrt, (g.n[SA] + KC - 1) / KC, 1);
  f.smem = (size_t)(NP + 2) * (f.TY + 2 * ring) * g.s[0] * sizeof(T);
  return f;
}

}  // namespace

template <typename T>
void launch_p_rb_fused(int D, const Geo& g, const LevelPtrs<T>& L, T* out, cudaStream_t s, int TYo,
                       int KCo, int NPo, int BXo) {
  const int NP = (D == 3 && NPo == 2) ? 2 : 1;
  FusedShape f = fused_shape<T>(D, g, TYo, KCo, NP, BXo);
  if (D == 3 && NP == 2) k_p_rb_fused<3, T, 2><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC);
  else if (D == 3) k_p_rb_fused<3, T, 1><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC);
  else k_p_rb_fused<2, T, 1><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC);
}

template <typename T>
void launch_v_rb_fused(int D, const Geo& g, const LevelPtrs<T>& L, int d, T* out, double inv_re,
                       cudaStream_t s, int TYo, int KCo, int NPo, int BXo) {
  const int NP = (D == 3 && NPo == 2) ? 2 : 1;
  FusedShape f = fused_shape<T>(D, g, TYo, KCo, NP, BXo);
  T ir = (T)(inv_re / (g.h * g.h));
  if (D == 3) {
    if (NP == 2) {
      if (d == 0) k_v_rb_fused<3, 0, T, 2><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC, ir);
      else if (d == 1) k_v_rb_fused<3, 1, T, 2><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC, ir);
      else k_v_rb_fused<3, 2, T, 2><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC, ir);
    } else {
      if (d == 0) k_v_rb_fused<3, 0, T, 1><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC, ir);
      else if (d == 1) k_v_rb_fused<3, 1, T, 1><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC, ir);
      else k_v_rb_fused<3, 2, T, 1><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC, ir);
    }
  } else {
    if (d == 0) k_v_rb_fused<2, 0, T, 1><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC, ir);
    else k_v_rb_fused<2, 1, T, 1><<<f.grid, f.block, f.smem, s>>>(g, L, out, f.TY, f.KC, ir);
  }
}

// Let the fused sweeps run several blocks per SM: ask for a shared-memory
// carveout of a quarter of the unified L1/shared storage for the FP64 sweeps
// and half of it for the FP32 sweeps, whose taller tiles (up to 18 ring rows)
// need more (call once, outside stream capture).
cudaError_t fused_set_carveout() {
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* f) {
    const bool f32 = f == (const void*)k_p_rb_fused<3, float, 1> ||
                     f == (const void*)k_p_rb_fused<3, float, 2> ||
                     f == (const void*)k_v_rb_fused<3, 0, float, 1> ||
                     f == (const void*)k_v_rb_fused<3, 1, float, 1> ||
                     f == (const void*)k_v_rb_fused<3, 2, float, 1> ||
                     f == (const void*)k_v_rb_fused<3, 0, float, 2> ||
                     f == (const void*)k_v_rb_fused<3, 1, float, 2> ||
                     f == (const void*)k_v_rb_fused<3, 2, float, 2>;
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, f32 ? 50 : 25);
  };
  set((const void*)k_p_rb_fused<3, float, 1>);
  set((const void*)k_p_rb_fused<3, float, 2>);
  set((const void*)k_p_rb_fused<2, float, 1>);
  set((const void*)k_p_rb_fused<3, double, 1>);
  set((const void*)k_p_rb_fused<3, double, 2>);
  set((const void*)k_p_rb_fused<2, double, 1>);
  set((const void*)k_v_rb_fused<3, 0, float, 1>);
  set((const void*)k_v_rb_fused<3, 1, float, 1>);
  set((const void*)k_v_rb_fused<3, 2, float, 1>);
  set((const void*)k_v_rb_fused<3, 0, float, 2>);
  set((const void*)k_v_rb_fused<3, 1, float, 2>);
  set((const void*)k_v_rb_fused<3, 2, float, 2>);
  set((const void*)k_v_rb_fused<2, 0, float, 1>);
  set((const void*)k_v_rb_fused<2, 1, float, 1>);
  set((const void*)k_v_rb_fused<3, 0, double, 1>);
  set((const void*)k_v_rb_fused<3, 1, double, 1>);
  set((const void*)k_v_rb_fused<3, 2, double, 1>);
  set((const void*)k_v_rb_fused<3, 0, double, 2>);
  set((const void*)k_v_rb_fused<3, 1, double, 2>);
  set((const void*)k_v_rb_fused<3, 2, double, 2>);
  set((const void*)k_v_rb_fused<2, 0, double, 1>);
  set((const void*)k_v_rb_fused<2, 1, double, 1>);
  return e;
}

// Chunk planes that give `waves` full waves of resident blocks for the 3D
// FP32 sweep of kind K (0..2 viscous components, 3 pressure) with TY tile
// rows; 0 where the occupancy cannot be had.
int ring_fill_kc(int D, int K, const Geo& g, int TY, int NP, int BX, int waves) {
  if (D != 3) return 0;
  FusedShape f = fused_shape<float>(D, g, TY, 0, NP, BX);
  const void* fn;
  if (K == 3) fn = NP == 2 ? (const void*)k_p_rb_fused<3, float, 2> : (const void*)k_p_rb_fused<3, float, 1>;
  else if (K == 0) fn = NP == 2 ? (const void*)k_v_rb_fused<3, 0, float, 2> : (const void*)k_v_rb_fused<3, 0, float, 1>;
  else if (K == 1) fn = NP == 2 ? (const void*)k_v_rb_fused<3, 1, float, 2> : (const void*)k_v_rb_fused<3, 1, float, 1>;
  else fn = NP == 2 ? (const void*)k_v_rb_fused<3, 2, float, 2> : (const void*)k_v_rb_fused<3, 2, float, 1>;
  int bps = 0, dev = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, (int)(f.block.x * f.block.y * f.block.z),
                                                    f.smem) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  long long chunks = (long long)waves * nsm * bps / (long long)f.grid.x;
  if (chunks < 1) return 0;
  int KC = (int)((g.n[2] + chunks - 1) / chunks);
  return KC < 2 ? 2 : KC;
}

size_t fused_smem_bytes(int D, const Geo& g, int elem) {
  return elem == 8 ? fused_shape<double>(D, g).smem : fused_shape<float>(D, g).smem;
}

template void launch_p_rb_fused<double>(int, const Geo&, const LevelPtrs<double>&, double*,
                                        cudaStream_t, int, int, int, int);
template void launch_p_rb_fused<float>(int, const Geo&, const LevelPtrs<float>&, float*,
                                       cudaStream_t, int, int, int, int);
template void launch_v_rb_fused<double>(int, const Geo&, const LevelPtrs<double>&, int, double*,
                                        double, cudaStream_t, int, int, int, int);
template void launch_v_rb_fused<float>(int, const Geo&, const LevelPtrs<float>&, int, float*,
                                       double, cudaStream_t, int, int, int, int);

}  // namespace bf
