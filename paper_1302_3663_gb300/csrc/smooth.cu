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

#include <type_traits>

#include "common.cuh"
#include "point.cuh"

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

// ---------------------------------------------------------------------------
// Pressure: red from the old black values (global), black from the new red
// values (shared). Neighbours are summed axis 0, 1, 2, lower then upper, as
// in the two-kernel sweep.
// ---------------------------------------------------------------------------
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
      const T pn = ring_nb<D, T>(rg, q, i, n0, a, -1, r, sl_m, sl_0, sl_p);
      if constexpr (sizeof(T) == 4) px_acc(num, dg, bb, pn);
      else {
        num += bb * pn;
        dg += bb;
      }
    }
    if (!q.wp[a]) {
      T bb = b[q.F + q.op[a]];
      const T pn = ring_nb<D, T>(rg, q, i, n0, a, +1, r, sl_m, sl_0, sl_p);
      if constexpr (sizeof(T) == 4) px_acc(num, dg, bb, pn);
      else {
        num += bb * pn;
        dg += bb;
      }
    }
  }
  if constexpr (sizeof(T) == 4) return px_final(num, dg, h2, L.pf[q.F]);
  else return (num - h2 * L.pf[q.F]) / dg;
}

// NP planes per iteration: the red values of planes k .. k+NP-1 (independent
// of one another, so their loads overlap), a barrier, then the black values
// of planes k-1 .. k+NP-2; the ring holds NP + 2 planes.
__device__ __forceinline__ int add_mod(int s, int o, int R) {
  int v = s + o;
  return v >= R ? v - R : (v < 0 ? v + R : v);
}

template <int D, typename T, int NP>
__device__ __forceinline__ void p_rb_fused_body(const Blk& B, Geo g, LevelPtrs<T> L,
                                                T* __restrict__ out, int TY, int KC) {
  constexpr int RA = Ax<D>::R, SA = Ax<D>::S, RING = Ax<D>::RING;
  constexpr int R = NP + 2;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  Ring<T> rg{reinterpret_cast<T*>(sm_raw), TY + 2 * RING, g.s[0]};
  const int n0 = g.n[0], nR = g.n[RA], nS = g.n[SA];
  const int j0 = B.x * TY;
  const int k0 = B.y * KC;
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

template <int D, typename T, int NP>
__global__ void __launch_bounds__(1024) k_p_rb_fused(Geo g, LevelPtrs<T> L, T* __restrict__ out,
                                                     int TY, int KC) {
  p_rb_fused_body<D, T, NP>(own_blk(), g, L, out, TY, KC);
}

// ---------------------------------------------------------------------------
// Viscous component d. Neighbour coefficients and the cross-component part
// come from the coefficient arrays and the (fixed) other components; the u_d
// neighbours come from the old buffer (red) or the ring (black).
template <int D, int d, typename T>
__device__ __forceinline__ T v_black(const LevelPtrs<T>& L, const Ring<T>& rg, const Pt& q,
                                     int i, int n0, T ir, int r, int sl_m, int sl_0, int sl_p) {
  VC<D, d, T> v;
  v_coef<D, d, T>(L, q, ir, v);
  // along d a wall neighbour is the stored zero face: the ring holds 0 there
  if constexpr (kIdg<T>) {
    float off = vx_off(v.cross, v.cdp, ring_nb<D, T>(rg, q, i, n0, d, +1, r, sl_m, sl_0, sl_p),
                       v.cdm, ring_nb<D, T>(rg, q, i, n0, d, -1, r, sl_m, sl_0, sl_p));
    int k = 0;
#pragma unroll
    for (int e = 0; e < D; ++e) {
      if (e == d) continue;
      if (!q.wp[e])
        off = vx_acc(off, v.cep[k], ring_nb<D, T>(rg, q, i, n0, e, +1, r, sl_m, sl_0, sl_p));
      if (!q.wm[e])
        off = vx_acc(off, v.cem[k], ring_nb<D, T>(rg, q, i, n0, e, -1, r, sl_m, sl_0, sl_p));
      ++k;
    }
    return vx_final(L.uf[d][q.F], ir, off, v.diag);
  } else {
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
}

template <int D, int d, typename T, int NP>
__device__ __forceinline__ void v_rb_fused_body(const Blk& B, Geo g, LevelPtrs<T> L,
                                                T* __restrict__ out, int TY, int KC, T ir) {
  constexpr int RA = Ax<D>::R, SA = Ax<D>::S, RING = Ax<D>::RING;
  constexpr int R = NP + 2;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  Ring<T> rg{reinterpret_cast<T*>(sm_raw), TY + 2 * RING, g.s[0]};
  const int n0 = g.n[0], nR = g.n[RA], nS = g.n[SA];
  const int j0 = B.x * TY;
  const int k0 = B.y * KC;
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

template <int D, int d, typename T, int NP>
__global__ void __launch_bounds__(1024) k_v_rb_fused(Geo g, LevelPtrs<T> L, T* __restrict__ out,
                                                     int TY, int KC, T ir) {
  v_rb_fused_body<D, d, T, NP>(own_blk(), g, L, out, TY, KC, ir);
}

// ---------------------------------------------------------------------------
// Pair sweep (3D FP32 viscous component d, walls in x and y). One thread owns
// the two points (x0, x0 + 1), x0 = 2 ip, of a row: one red, one black. It
// walks the planes of a chunk. Every input row is read as one float2, plus
// the value left (x0 - 1) or right (x0 + 2) of the pair where a stencil
// reaches there. Rows that the next planes need again (the plane above
// becomes the plane itself, then the plane below) stay in registers, so a
// pair costs 15 to 17 loads per plane.
//
// At plane k the thread computes the coefficient sets of both points, that
// is, everything of the update but the u_d neighbours. The red point is then
// solved from the old u_d values, and the black point's set is kept. After
// one barrier the black point of plane k - 1 is solved from its kept set and
// the ring of new red values. The ring has four plane slots, so the next
// plane's red values never overwrite a slot still being read. Then the pair
// of plane k - 1 is stored. The expressions and their order are those of
// v_red / v_black; a term the ring sweep skips at a wall gets a zero weight
// here (adding 0 * x changes no bit).
// ---------------------------------------------------------------------------
struct PRow {        // a row at the pair: v = (x0, x0 + 1), l = x0 - 1, r = x0 + 2
  float2 v;
  float l, r;
};

template <int o>     // the value at x0 + o, o in -1 .. 2
__device__ __forceinline__ float pe(const PRow& q) {
  if constexpr (o == -1) return q.l;
  else if constexpr (o == 0) return q.v.x;
  else if constexpr (o == 1) return q.v.y;
  else return q.r;
}

__device__ __forceinline__ float2 ldp(const float* __restrict__ a, int o) {
  return __ldg(reinterpret_cast<const float2*>(a + o));
}
// bring a line towards L1 for the next plane's load (no register is tied up)
__device__ __forceinline__ void pf1(const float* a, int o) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(a + o));
}

struct PSet {
  float cross, cdp, cdm, cep0, cem0, cep1, cem1, uf, idg;
};

// The coefficient set of element e from the rows of its plane: pc (u_d's own
// centre row is not needed here), for every e2 != d pairs of rows at F and at
// F + e, each with the row shifted by -d.
template <int d, int e>
__device__ __forceinline__ PSet pset(const PRow& mc, const PRow& mcm, const PRow& me0_F,
                                     const PRow& me0_P, const PRow& ue0_F, const PRow& ue0_Fm,
                                     const PRow& ue0_P, const PRow& ue0_Pm, const PRow& me1_F,
                                     const PRow& me1_P, const PRow& ue1_F, const PRow& ue1_Fm,
                                     const PRow& ue1_P, const PRow& ue1_Pm, const PRow& uf,
                                     const PRow& idg, bool wp0, bool wm0, bool wp1, bool wm1) {
  constexpr int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
  constexpr int sd = d == 0 ? -1 : 0;        // x shift of F - d
  constexpr int s1 = e1 == 0 ? 1 : 0, s2 = e2 == 0 ? 1 : 0;   // x shift of F + e
  PSet c;
  float mcp = pe<e>(mc), mcmv = pe<e + sd>(mcm);
  c.cdp = 2.f * mcp;
  c.cdm = 2.f * mcmv;
  c.cross = 0.f;
  {
    float mep = pe<e + s1>(me0_P), mem = pe<e>(me0_F);
    c.cross = vx_cross(c.cross, mep, pe<e + s1>(ue0_P), pe<e + s1 + sd>(ue0_Pm), mem, pe<e>(ue0_F),
                       pe<e + sd>(ue0_Fm));
    c.cep0 = wp0 ? 0.f : mep;
    c.cem0 = wm0 ? 0.f : mem;
  }
  {
    float mep = pe<e + s2>(me1_P), mem = pe<e>(me1_F);
    c.cross = vx_cross(c.cross, mep, pe<e + s2>(ue1_P), pe<e + s2 + sd>(ue1_Pm), mem, pe<e>(ue1_F),
                       pe<e + sd>(ue1_Fm));
    c.cep1 = wp1 ? 0.f : mep;
    c.cem1 = wm1 ? 0.f : mem;
  }
  c.uf = pe<e>(uf);
  c.idg = pe<e>(idg);
  return c;
}

__device__ __forceinline__ float psolve(const PSet& c, float ir, float up_d, float um_d,
                                        float up_1, float um_1, float up_2, float um_2) {
  float off = vx_off(c.cross, c.cdp, up_d, c.cdm, um_d);
  off = vx_acc(off, c.cep0, up_1);
  off = vx_acc(off, c.cem0, um_1);
  off = vx_acc(off, c.cep1, up_2);
  off = vx_acc(off, c.cem1, um_2);
  return vx_final(c.uf, ir, off, c.idg);
}

template <int d, bool PERZ>
__device__ __forceinline__ void v_rb_pair_body(const Blk& B, Geo g, LevelPtrs<float> L,
                                               float* __restrict__ out, int TY, int KC, float ir) {
  constexpr int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float* ring = reinterpret_cast<float*>(sm_raw);
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int W = n0;                        // ring row pitch
  const int plane = (TY + 2) * W;
  const int x0 = 2 * threadIdx.x, r = threadIdx.y;
  const int j0 = B.x * TY;
  const int k0 = B.y * KC, k1 = min(k0 + KC, n2);
  const int j = j0 - 1 + r;
  const bool lane_ok = x0 < n0;
  const bool rowvalid = lane_ok && j >= 0 && j < n1;
  const bool own = rowvalid && r >= 1 && r <= TY;
  const int st1 = (int)g.st[1], st2 = (int)g.st[2];
  const int xl = x0 > 0 ? x0 - 1 : 0;     // left of the pair (clamped at the wall: zero weight)
  // wall flags of the row and of the two x positions
  const bool wpy = j == n1 - 1, wmy = j == 0;
  const bool wmx0 = x0 == 0, wpx1 = x0 + 1 == n0 - 1;
  for (int q = threadIdx.y * blockDim.x + threadIdx.x; q < 4 * plane; q += blockDim.x * blockDim.y)
    ring[q] = 0.f;
  const float* __restrict__ ud = L.u[d];
  const float* __restrict__ ua = L.u[e1];
  const float* __restrict__ ub = L.u[e2];
  const float* __restrict__ ma = L.mue[edge_id(d, e1)];
  const float* __restrict__ mb = L.mue[edge_id(d, e2)];
  const float* __restrict__ mc = L.muc;
  const float* __restrict__ uf = L.uf[d];
  const float* __restrict__ ig = L.idg[d];
  // row offsets (elements, x0 included): this row, the rows below and above
  const int jm = j > 0 ? j - 1 : j;
  const int oy0 = j * st1 + x0, oym = jm * st1 + x0, oyp = (j + 1) * st1 + x0;
  // plane index of plane k (wrapped on a periodic axis, clamped into the
  // storage on a wall axis: planes outside are never used)
  auto pz = [&](int k) -> int {
    if constexpr (PERZ) return k < 0 ? k + n2 : (k >= n2 ? k - n2 : k);
    else return k < 0 ? 0 : (k > n2 ? n2 : k);
  };
  auto row = [&](const float* __restrict__ a, int oy, int kz, bool left, bool right) -> PRow {
    PRow q;
    const int o = oy + kz * st2;
    q.v = ldp(a, o);
    q.l = left ? __ldg(a + o - x0 + xl) : 0.f;
    q.r = right ? __ldg(a + o + 2) : 0.f;
    return q;
  };
  // register queues along z: rows of plane k - 1 and k
  PRow UDm{}, UDc{};
  PRow Q0c{}, Q1c{}, Q2c{};     // the component-specific rows of plane k (see below)
  const bool ld = rowvalid;
  {
    const int km = pz(k0 - 2), kc = pz(k0 - 1);
    if (ld) {
      UDm = row(ud, oy0, km, false, false);
      UDc = row(ud, oy0, kc, false, false);
      if constexpr (d == 0) {          // u_z and mu_xz at F (plane k)
        Q0c = row(ub, oy0, kc, true, false);
        Q1c = row(mb, oy0, kc, false, false);
      } else if constexpr (d == 1) {   // u_z at F and F - y, mu_yz at F (plane k)
        Q0c = row(ub, oy0, kc, false, false);
        Q1c = row(ub, oym, kc, false, false);
        Q2c = row(mb, oy0, kc, false, false);
      } else {                         // u_x at F, u_y at F and F + y, mu_c at F (plane k - 1)
        Q0c = row(ua, oy0, km, false, true);
        Q1c = row(ub, oy0, km, false, false);
        Q2c = row(ub, oyp, km, false, false);
      }
    }
  }
  PRow MCzm{};
  if constexpr (d == 2) {
    if (ld) MCzm = row(mc, oy0, pz(k0 - 2), false, false);
  }
  __syncthreads();
  int sk = 0;                                // ring slot of plane k
  PSet keep{};                               // the black point's set of plane k - 1
  float red_prev = 0.f;
  // One plane. PAR is the element of the red point, (j + k) & 1: a warp
  // holds one row, so it is the same in every lane, and the black point of
  // plane k - 1 is element PAR as well.
  auto step = [&](auto par_tag, const int k) {
    constexpr int PAR = decltype(par_tag)::value;
    const bool planevalid = PERZ || (k >= 0 && k < n2);
    const int kw = pz(k), kp = pz(k + 1);
    // the z walls of plane k (unused by the z component: z is its own axis)
    [[maybe_unused]] const bool wpz = !PERZ && kw == n2 - 1, wmz = !PERZ && kw == 0;
    float redv = 0.f;
    PSet blk{};
    PRow UDp{};
    if (ld) UDp = row(ud, oy0, kp, false, false);
    if (ld && k < k1) {
      // the rows the next plane loads: one plane further along z
      const int kn = pz(k + 1) * st2, kn2 = pz(k + 2) * st2;
      pf1(ud, oy0 + kn2);
      pf1(ud, oym + kn);
      pf1(ud, oyp + kn);
      pf1(mc, oy0 + kn);
      pf1(uf, oy0 + kn);
      pf1(ig, oy0 + kn);
      if constexpr (d == 0) {
        pf1(ma, oy0 + kn);
        pf1(ma, oyp + kn);
        pf1(ua, oy0 + kn);
        pf1(ua, oyp + kn);
        pf1(ub, oy0 + kn2);
        pf1(mb, oy0 + kn2);
      } else if constexpr (d == 1) {
        pf1(mc, oym + kn);
        pf1(ma, oy0 + kn);
        pf1(ua, oy0 + kn);
        pf1(ua, oym + kn);
        pf1(ub, oy0 + kn2);
        pf1(ub, oym + kn2);
        pf1(mb, oy0 + kn2);
      } else {
        pf1(ma, oy0 + kn);
        pf1(ua, oy0 + kn);
        pf1(mb, oy0 + kn);
        pf1(mb, oyp + kn);
        pf1(ub, oy0 + kn);
        pf1(ub, oyp + kn);
      }
    }
    PRow N0{}, N1{};
    [[maybe_unused]] PRow N2{}, N3{};   // the y and z components queue more rows
    if (ld && planevalid) {
      // u_d at the rows beside (old values) and the value beside the red point
      const PRow UDym = row(ud, oym, kw, false, false), UDyp = row(ud, oyp, kw, false, false);
      PRow UDx = UDc;
      const int ox = oy0 + kw * st2;
      if constexpr (PAR == 1) UDx.r = __ldg(ud + ox + 2);
      else UDx.l = __ldg(ud + ox - x0 + xl);
      PSet c0, c1;
      if constexpr (d == 0) {
        // e1 = y: mu_xy at F, F + y; u_y at F, F + y (and x - 1)
        // e2 = z: mu_xz at F, F + z; u_z at F, F + z (and x - 1)
        const PRow MC = row(mc, oy0, kw, true, false);
        const PRow MAF = row(ma, oy0, kw, false, false), MAP = row(ma, oyp, kw, false, false);
        const PRow UAF = row(ua, oy0, kw, true, false), UAP = row(ua, oyp, kw, true, false);
        const PRow UBP = row(ub, oy0, kp, true, false), MBP = row(mb, oy0, kp, false, false);
        const PRow UF = row(uf, oy0, kw, false, false), IG = row(ig, oy0, kw, false, false);
        c0 = pset<0, 0>(MC, MC, MAF, MAP, UAF, UAF, UAP, UAP, Q1c, MBP, Q0c, Q0c, UBP, UBP, UF, IG,
                        wpy, wmy, wpz, wmz);
        c1 = pset<0, 1>(MC, MC, MAF, MAP, UAF, UAF, UAP, UAP, Q1c, MBP, Q0c, Q0c, UBP, UBP, UF, IG,
                        wpy, wmy, wpz, wmz);
        N0 = UBP;
        N1 = MBP;
      } else if constexpr (d == 1) {
        // e1 = x: mu_xy at F, F + x; u_x at F, F + x and the row below
        // e2 = z: mu_yz at F, F + z; u_z at F, F + z and the row below
        const PRow MC = row(mc, oy0, kw, false, false), MCm = row(mc, oym, kw, false, false);
        const PRow MA = row(ma, oy0, kw, false, true);
        const PRow UA = row(ua, oy0, kw, false, true), UAm = row(ua, oym, kw, false, true);
        const PRow UBP = row(ub, oy0, kp, false, false), UBPm = row(ub, oym, kp, false, false);
        const PRow MBP = row(mb, oy0, kp, false, false);
        const PRow UF = row(uf, oy0, kw, false, false), IG = row(ig, oy0, kw, false, false);
        c0 = pset<1, 0>(MC, MCm, MA, MA, UA, UAm, UA, UAm, Q2c, MBP, Q0c, Q1c, UBP, UBPm, UF, IG,
                        false, wmx0, wpz, wmz);
        c1 = pset<1, 1>(MC, MCm, MA, MA, UA, UAm, UA, UAm, Q2c, MBP, Q0c, Q1c, UBP, UBPm, UF, IG,
                        wpx1, false, wpz, wmz);
        N0 = UBP;
        N1 = UBPm;
        N2 = MBP;
      } else {
        // e1 = x: mu_xz at F, F + x; u_x at F, F + x and the plane below
        // e2 = y: mu_yz at F, F + y; u_y at F, F + y and the plane below
        const PRow MC = row(mc, oy0, kw, false, false);
        const PRow MA = row(ma, oy0, kw, false, true);
        const PRow UA = row(ua, oy0, kw, false, true);
        const PRow MBF = row(mb, oy0, kw, false, false), MBP = row(mb, oyp, kw, false, false);
        const PRow UBF = row(ub, oy0, kw, false, false), UBP = row(ub, oyp, kw, false, false);
        const PRow UF = row(uf, oy0, kw, false, false), IG = row(ig, oy0, kw, false, false);
        c0 = pset<2, 0>(MC, MCzm, MA, MA, UA, Q0c, UA, Q0c, MBF, MBP, UBF, Q1c, UBP, Q2c, UF, IG,
                        false, wmx0, wpy, wmy);
        c1 = pset<2, 1>(MC, MCzm, MA, MA, UA, Q0c, UA, Q0c, MBF, MBP, UBF, Q1c, UBP, Q2c, UF, IG,
                        wpx1, false, wpy, wmy);
        N0 = UA;
        N1 = UBF;
        N2 = UBP;
        N3 = MC;
      }
      // the red point: its set and its old neighbours along d, e1, e2
      float np_[3], nm_[3];
      np_[0] = pe<PAR + 1>(UDx);
      nm_[0] = pe<PAR - 1>(UDx);
      np_[1] = pe<PAR>(UDyp);
      nm_[1] = pe<PAR>(UDym);
      np_[2] = pe<PAR>(UDp);
      nm_[2] = pe<PAR>(UDm);
      redv = psolve(PAR ? c1 : c0, ir, np_[d], nm_[d], np_[e1], nm_[e1], np_[e2], nm_[e2]);
      const bool wall_red = (d == 0 && x0 + PAR == 0) || (d == 1 && j == 0) ||
                            (d == 2 && !PERZ && kw == 0);
      if (wall_red) redv = 0.f;
      blk = PAR ? c0 : c1;
    }
    if (lane_ok) {
      const float2 rv = PAR ? make_float2(0.f, redv) : make_float2(redv, 0.f);
      *reinterpret_cast<float2*>(ring + sk * plane + r * W + x0) = rv;
    }
    __syncthreads();
    // the black point (element PAR) of plane k - 1 on the block's own rows;
    // the pair out
    const int kb = k - 1;
    if (own && kb >= k0 && kb < k1) {
      const int kbw = pz(kb);
      const int s_m = (sk + 2) & 3, s_0 = (sk + 3) & 3;   // planes k - 2, k - 1 (k: sk)
      const int xb = x0 + PAR;
      const float* R0 = ring + s_0 * plane + r * W;
      float np_[3], nm_[3];
      np_[0] = xb + 1 < n0 ? R0[xb + 1] : 0.f;
      nm_[0] = xb > 0 ? R0[xb - 1] : 0.f;
      np_[1] = R0[W + xb];
      nm_[1] = R0[-W + xb];
      np_[2] = ring[sk * plane + r * W + xb];
      nm_[2] = ring[s_m * plane + r * W + xb];
      float bv = psolve(keep, ir, np_[d], nm_[d], np_[e1], nm_[e1], np_[e2], nm_[e2]);
      const bool wall_blk = (d == 0 && xb == 0) || (d == 1 && j == 0) ||
                            (d == 2 && !PERZ && kbw == 0);
      if (wall_blk) bv = 0.f;
      const float2 o = PAR ? make_float2(red_prev, bv) : make_float2(bv, red_prev);
      *reinterpret_cast<float2*>(out + oy0 + kbw * st2) = o;
    }
    // advance the queues by one plane
    keep = blk;
    red_prev = redv;
    sk = (sk + 1) & 3;
    UDm = UDc;
    UDc = UDp;
    if (ld) {
      if constexpr (d == 0) {
        if (planevalid) {
          Q0c = N0;
          Q1c = N1;
        } else {
          Q0c = row(ub, oy0, kp, true, false);
          Q1c = row(mb, oy0, kp, false, false);
        }
      } else if constexpr (d == 1) {
        if (planevalid) {
          Q0c = N0;
          Q1c = N1;
          Q2c = N2;
        } else {
          Q0c = row(ub, oy0, kp, false, false);
          Q1c = row(ub, oym, kp, false, false);
          Q2c = row(mb, oy0, kp, false, false);
        }
      } else {
        if (planevalid) {
          Q0c = N0;
          Q1c = N1;
          Q2c = N2;
          MCzm = N3;
        } else {
          Q0c = row(ua, oy0, kw, false, true);
          Q1c = row(ub, oy0, kw, false, false);
          Q2c = row(ub, oyp, kw, false, false);
          MCzm = row(mc, oy0, kw, false, false);
        }
      }
    }
  };
  using P0 = std::integral_constant<int, 0>;
  using P1 = std::integral_constant<int, 1>;
  int k = k0 - 1;
  for (; k + 1 <= k1; k += 2) {   // two planes per iteration: the parity alternates
    if ((j + k) & 1) {
      step(P1{}, k);
      step(P0{}, k + 1);
    } else {
      step(P0{}, k);
      step(P1{}, k + 1);
    }
  }
  if (k <= k1) {
    if ((j + k) & 1) step(P1{}, k);
    else step(P0{}, k);
  }
}

template <int d, bool PERZ>
__global__ void __launch_bounds__(512, 2) k_v_rb_pair(Geo g, LevelPtrs<float> L,
                                                   float* __restrict__ out, int TY, int KC,
                                                   float ir) {
  v_rb_pair_body<d, PERZ>(own_blk(), g, L, out, TY, KC, ir);
}

struct FusedShape {
  dim3 grid, block;
  int TY, KC;
  size_t smem;
};

// ---------------------------------------------------------------------------
// Batched ring sweep: the one-pass sweep above over a persistent batch's work
// list. Each item is a (row tile, plane chunk) block of one member's level;
// the ring is sized for the widest member's rows. K 0..2: viscous component,
// 3: pressure. The output is the buffer that A.cur marks as not current.
// ---------------------------------------------------------------------------
template <int K, int NP>
__global__ void __launch_bounds__(1024) kb_sweep(BArgs A, int TY, int KC) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    const Geo g = M.g[A.lev];
    const LevelPtrs<float> L = cur_ptrs(M.f[A.lev], A.cur);
    if constexpr (K == 3) {
      p_rb_fused_body<3, float, NP>(B, g, L, L.p2, TY, KC);
    } else {
      v_rb_fused_body<3, K, float, NP>(B, g, L, L.u2[K], TY, KC, (float)M.ir[A.lev]);
    }
  });
}

// Batched pair sweep of viscous component d: block b does item b of the list
// (one block per item, so no work-list loop adds registers to a kernel at its
// limit); the block is as wide as the widest member's row needs, and the lanes
// past a narrower member's row only take part in the barriers.
template <int d, bool PERZ>
__global__ void __launch_bounds__(512, 2) kb_pair(BArgs A, int TY, int KC) {
  const BItem it = A.items[blockIdx.x];
  if (A.act && !A.act[it.m]) return;
  const BMember& M = A.tab[it.m];
  const Geo g = M.g[A.lev];
  const LevelPtrs<float> L = cur_ptrs(M.f[A.lev], A.cur);
  v_rb_pair_body<d, PERZ>(Blk{it.x, it.y, it.z, it.gx, it.gy, it.gz}, g, L, L.u2[d], TY, KC,
                          (float)M.ir[A.lev]);
}

// ---------------------------------------------------------------------------
// Pair sweep of the pressure (3D FP32, walls in x and y), built like the
// viscous pair sweep: one thread per (red, black) pair of a row, TY rows plus
// two ring rows per block, marching over a chunk of planes. At plane k the
// red point is solved from old black values: the p rows of its plane and of
// the rows below and above, and p of the planes below and above from a
// register queue. The black point's weights (its six betas, 0 beyond a wall)
// and right-hand side are kept; after one barrier the black point of plane
// k - 1 is solved from the four-slot ring of new red values. The point
// arithmetic is px_acc / px_final in the order of p_red; a neighbour beyond a
// wall enters with beta 0 and p 0, which changes no bit.
// ---------------------------------------------------------------------------
struct PPSet {
  float b[6];   // beta of the x-, x+, y-, y+, z-, z+ neighbours
  float f;      // right-hand side
};

__device__ __forceinline__ float ppsolve(const PPSet& c, float h2, const float nb[6]) {
  float num = 0.f, dg = 0.f;
#pragma unroll
  for (int t = 0; t < 6; ++t) px_acc(num, dg, c.b[t], nb[t]);
  return px_final(num, dg, h2, c.f);
}

template <bool PERZ>
__device__ __forceinline__ void p_rb_pair_body(const Blk& B, Geo g, LevelPtrs<float> L,
                                               float* __restrict__ out, int TY, int KC, float h2) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float* ring = reinterpret_cast<float*>(sm_raw);
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const int W = n0;
  const int plane = (TY + 2) * W;
  const int x0 = 2 * threadIdx.x, r = threadIdx.y;
  const int j0 = B.x * TY;
  const int k0 = B.y * KC, k1 = min(k0 + KC, n2);
  const int j = j0 - 1 + r;
  const bool lane_ok = x0 < n0;
  const bool rowvalid = lane_ok && j >= 0 && j < n1;
  const bool own = rowvalid && r >= 1 && r <= TY;
  const int st1 = (int)g.st[1], st2 = (int)g.st[2];
  const int xl = x0 > 0 ? x0 - 1 : 0;
  const bool wpy = j == n1 - 1, wmy = j == 0;
  const bool wmx0 = x0 == 0, wpx1 = x0 + 1 == n0 - 1;
  for (int q = threadIdx.y * blockDim.x + threadIdx.x; q < 4 * plane; q += blockDim.x * blockDim.y)
    ring[q] = 0.f;
  const float* __restrict__ pp = L.p;
  const float* __restrict__ bx = L.beta[0];
  const float* __restrict__ by = L.beta[1];
  const float* __restrict__ bz = L.beta[2];
  const float* __restrict__ pf = L.pf;
  const int jm = j > 0 ? j - 1 : j;
  const int oy0 = j * st1 + x0, oym = jm * st1 + x0, oyp = (j + 1) * st1 + x0;
  auto pz = [&](int k) -> int {
    if constexpr (PERZ) return k < 0 ? k + n2 : (k >= n2 ? k - n2 : k);
    else return k < 0 ? 0 : (k > n2 ? n2 : k);
  };
  const bool ld = rowvalid;
  // register queues along z: p of planes k - 1 and k, beta_z of plane k
  float2 Pm = make_float2(0.f, 0.f), Pc = Pm, BZc = Pm;
  if (ld) {
    Pm = ldp(pp, oy0 + pz(k0 - 2) * st2);
    Pc = ldp(pp, oy0 + pz(k0 - 1) * st2);
    BZc = ldp(bz, oy0 + pz(k0 - 1) * st2);
  }
  __syncthreads();
  int sk = 0;
  PPSet keep{};
  float red_prev = 0.f;
  auto step = [&](auto par_tag, const int k) {
    constexpr int PAR = decltype(par_tag)::value;
    const bool planevalid = PERZ || (k >= 0 && k < n2);
    const int kw = pz(k), kp = pz(k + 1);
    const bool wpz = !PERZ && kw == n2 - 1, wmz = !PERZ && kw == 0;
    float redv = 0.f;
    PPSet blk{};
    float2 Pp = make_float2(0.f, 0.f), BZp = Pp;
    if (ld) {
      Pp = ldp(pp, oy0 + kp * st2);
      BZp = ldp(bz, oy0 + kp * st2);
    }
    if (ld && k < k1) {   // the rows the next plane loads
      const int kn = pz(k + 1) * st2, kn2 = pz(k + 2) * st2;
      pf1(pp, oy0 + kn2);
      pf1(bz, oy0 + kn2);
      pf1(pp, oym + kn);
      pf1(pp, oyp + kn);
      pf1(bx, oy0 + kn);
      pf1(by, oy0 + kn);
      pf1(by, oyp + kn);
      pf1(pf, oy0 + kn);
    }
    if (ld && planevalid) {
      const int oz = kw * st2;
      // p of this row (queued) with the value left (red at x0 + 1) or right (red at x0)
      const float2 P0 = Pc;
      const float Pl = PAR ? 0.f : __ldg(pp + oy0 + oz - x0 + xl);
      const float Pr = PAR ? __ldg(pp + oy0 + oz + 2) : 0.f;
      const float2 PYm = ldp(pp, oym + oz), PYp = ldp(pp, oyp + oz);
      const float2 BX = ldp(bx, oy0 + oz);
      const float BXr = __ldg(bx + oy0 + oz + 2);
      const float2 BY = ldp(by, oy0 + oz), BYp = ldp(by, oyp + oz);
      const float2 F = ldp(pf, oy0 + oz);
      // the two points' weights: x at x0 uses beta_x(x0), beta_x(x0 + 1); x0 + 1
      // uses beta_x(x0 + 1), beta_x(x0 + 2)
      PPSet c0, c1;
      c0.b[0] = wmx0 ? 0.f : BX.x;
      c0.b[1] = BX.y;
      c1.b[0] = BX.y;
      c1.b[1] = wpx1 ? 0.f : BXr;
      c0.b[2] = wmy ? 0.f : BY.x;
      c1.b[2] = wmy ? 0.f : BY.y;
      c0.b[3] = wpy ? 0.f : BYp.x;
      c1.b[3] = wpy ? 0.f : BYp.y;
      c0.b[4] = wmz ? 0.f : BZc.x;
      c1.b[4] = wmz ? 0.f : BZc.y;
      c0.b[5] = wpz ? 0.f : BZp.x;
      c1.b[5] = wpz ? 0.f : BZp.y;
      c0.f = F.x;
      c1.f = F.y;
      // the red point (element PAR): its old neighbours, 0 beyond a wall
      float nb[6];
      if constexpr (PAR == 0) {
        nb[0] = wmx0 ? 0.f : Pl;
        nb[1] = P0.y;
        nb[2] = wmy ? 0.f : PYm.x;
        nb[3] = wpy ? 0.f : PYp.x;
        nb[4] = wmz ? 0.f : Pm.x;
        nb[5] = wpz ? 0.f : Pp.x;
      } else {
        nb[0] = P0.x;
        nb[1] = wpx1 ? 0.f : Pr;
        nb[2] = wmy ? 0.f : PYm.y;
        nb[3] = wpy ? 0.f : PYp.y;
        nb[4] = wmz ? 0.f : Pm.y;
        nb[5] = wpz ? 0.f : Pp.y;
      }
      redv = ppsolve(PAR ? c1 : c0, h2, nb);
      blk = PAR ? c0 : c1;
    }
    if (lane_ok) {
      const float2 rv = PAR ? make_float2(0.f, redv) : make_float2(redv, 0.f);
      *reinterpret_cast<float2*>(ring + sk * plane + r * W + x0) = rv;
    }
    __syncthreads();
    // the black point (element PAR) of plane k - 1 on the block's own rows;
    // the pair out
    const int kb = k - 1;
    if (own && kb >= k0 && kb < k1) {
      const int kbw = pz(kb);
      const int s_m = (sk + 2) & 3, s_0 = (sk + 3) & 3;
      const int xb = x0 + PAR;
      const float* R0 = ring + s_0 * plane + r * W;
      float nb[6];
      nb[0] = xb > 0 ? R0[xb - 1] : 0.f;
      nb[1] = xb + 1 < n0 ? R0[xb + 1] : 0.f;
      nb[2] = R0[-W + xb];
      nb[3] = R0[W + xb];
      nb[4] = ring[s_m * plane + r * W + xb];
      nb[5] = ring[sk * plane + r * W + xb];
      const float bv = ppsolve(keep, h2, nb);
      const float2 o = PAR ? make_float2(red_prev, bv) : make_float2(bv, red_prev);
      *reinterpret_cast<float2*>(out + oy0 + kbw * st2) = o;
    }
    keep = blk;
    red_prev = redv;
    sk = (sk + 1) & 3;
    Pm = Pc;
    Pc = Pp;
    BZc = BZp;
  };
  using P0t = std::integral_constant<int, 0>;
  using P1t = std::integral_constant<int, 1>;
  int k = k0 - 1;
  for (; k + 1 <= k1; k += 2) {   // two planes per iteration: the parity alternates
    if ((j + k) & 1) {
      step(P1t{}, k);
      step(P0t{}, k + 1);
    } else {
      step(P0t{}, k);
      step(P1t{}, k + 1);
    }
  }
  if (k <= k1) {
    if ((j + k) & 1) step(P1t{}, k);
    else step(P0t{}, k);
  }
}

template <bool PERZ>
__global__ void __launch_bounds__(512, 2) k_p_rb_pair(Geo g, LevelPtrs<float> L,
                                                   float* __restrict__ out, int TY, int KC,
                                                   float h2) {
  p_rb_pair_body<PERZ>(own_blk(), g, L, out, TY, KC, h2);
}

// the batched pressure pair sweep: one block per item, as kb_pair
template <bool PERZ>
__global__ void __launch_bounds__(512, 2) kb_ppair(BArgs A, int TY, int KC) {
  const BItem it = A.items[blockIdx.x];
  if (A.act && !A.act[it.m]) return;
  const BMember& M = A.tab[it.m];
  const Geo g = M.g[A.lev];
  const LevelPtrs<float> L = cur_ptrs(M.f[A.lev], A.cur);
  p_rb_pair_body<PERZ>(Blk{it.x, it.y, it.z, it.gx, it.gy, it.gz}, g, L, L.p2, TY, KC,
                       (float)(g.h * g.h));
}

// after an odd count of sweeps the current iterate (in the second buffer) is
// copied to its own buffer, on every stored element
template <int K>
__global__ void __launch_bounds__(256) kb_copy_back(BArgs A) {
  for_items(A, [&](const BMember& M, const Blk& B) {
    const Geo& g = M.g[A.lev];
    const long long n = g.st[2] * g.s[2];
    const float* __restrict__ src = K == 3 ? M.f[A.lev].p2 : M.f[A.lev].u2[K];
    float* __restrict__ dst = K == 3 ? M.f[A.lev].p : M.f[A.lev].u[K];
    for (long long q = B.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)B.gx * blockDim.x)
      dst[q] = src[q];
  });
}

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

// Pair sweep: blocks of (pairs of a row rounded up to 32) x (TY + 2) threads
// over (row tiles, plane chunks); 3D, walls in x and y, an even row of at
// most 256 points.
bool pair_eligible(int D, const Geo& g, int TY) {
  if (D != 3 || g.per[0] || g.per[1] || (g.n[0] & 1) || g.n[0] < 4 || g.n[0] > 256) return false;
  const int bx = ((g.n[0] / 2 + 31) / 32) * 32;
  return TY >= 1 && TY <= g.n[1] && bx * (TY + 2) <= 512;
}

const void* pair_kernel(int d, bool perz) {
  if (perz)
    return d == 0 ? (const void*)k_v_rb_pair<0, true>
                  : (d == 1 ? (const void*)k_v_rb_pair<1, true> : (const void*)k_v_rb_pair<2, true>);
  return d == 0 ? (const void*)k_v_rb_pair<0, false>
                : (d == 1 ? (const void*)k_v_rb_pair<1, false> : (const void*)k_v_rb_pair<2, false>);
}

size_t pair_smem(const Geo& g, int TY) { return (size_t)4 * (TY + 2) * g.n[0] * sizeof(float); }

void launch_v_rb_pair(const Geo& g, const LevelPtrs<float>& L, int d, float* out, double inv_re,
                      cudaStream_t s, int TY, int KC) {
  const int bx = ((g.n[0] / 2 + 31) / 32) * 32;
  if (KC < 1) KC = 1;
  dim3 block(bx, TY + 2, 1);
  dim3 grid((g.n[1] + TY - 1) / TY, (g.n[2] + KC - 1) / KC, 1);
  const float ir = (float)(inv_re / (g.h * g.h));
  const size_t sm = pair_smem(g, TY);
  if (g.per[2]) {
    if (d == 0) k_v_rb_pair<0, true><<<grid, block, sm, s>>>(g, L, out, TY, KC, ir);
    else if (d == 1) k_v_rb_pair<1, true><<<grid, block, sm, s>>>(g, L, out, TY, KC, ir);
    else k_v_rb_pair<2, true><<<grid, block, sm, s>>>(g, L, out, TY, KC, ir);
  } else {
    if (d == 0) k_v_rb_pair<0, false><<<grid, block, sm, s>>>(g, L, out, TY, KC, ir);
    else if (d == 1) k_v_rb_pair<1, false><<<grid, block, sm, s>>>(g, L, out, TY, KC, ir);
    else k_v_rb_pair<2, false><<<grid, block, sm, s>>>(g, L, out, TY, KC, ir);
  }
}

const void* p_pair_kernel(bool perz) {
  return perz ? (const void*)k_p_rb_pair<true> : (const void*)k_p_rb_pair<false>;
}

void launch_p_rb_pair(const Geo& g, const LevelPtrs<float>& L, float* out, cudaStream_t s, int TY,
                      int KC) {
  const int bx = ((g.n[0] / 2 + 31) / 32) * 32;
  if (KC < 1) KC = 1;
  dim3 block(bx, TY + 2, 1);
  dim3 grid((g.n[1] + TY - 1) / TY, (g.n[2] + KC - 1) / KC, 1);
  const float h2 = (float)(g.h * g.h);
  const size_t sm = pair_smem(g, TY);
  if (g.per[2]) k_p_rb_pair<true><<<grid, block, sm, s>>>(g, L, out, TY, KC, h2);
  else k_p_rb_pair<false><<<grid, block, sm, s>>>(g, L, out, TY, KC, h2);
}

void launch_b_ppair(const BArgs& A, bool perz, int TY, int KC, int bx, size_t smem,
                    cudaStream_t s) {
  if (A.n <= 0) return;
  const dim3 block(bx, TY + 2, 1);
  if (perz) kb_ppair<true><<<A.n, block, smem, s>>>(A, TY, KC);
  else kb_ppair<false><<<A.n, block, smem, s>>>(A, TY, KC);
}

// Chunk planes giving `waves` full waves of resident pair-sweep blocks (kind
// d: 0..2 viscous, 3 pressure); 0 where the occupancy cannot be had.
int pair_fill_kc(const Geo& g, int d, int TY, int waves) {
  if (!pair_eligible(3, g, TY)) return 0;
  const void* fn = d == 3 ? p_pair_kernel(g.per[2] != 0) : pair_kernel(d, g.per[2] != 0);
  const int bx = ((g.n[0] / 2 + 31) / 32) * 32;
  int bps = 0, dev = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, bx * (TY + 2), pair_smem(g, TY)) !=
          cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const long long tiles = (g.n[1] + TY - 1) / TY;
  long long chunks = (long long)waves * nsm * bps / tiles;
  if (chunks < 1) return 0;
  int KC = (int)((g.n[2] + chunks - 1) / chunks);
  return KC < 2 ? 2 : KC;
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
  for (int K = 0; K < 4; ++K)
    for (int NP = 1; NP <= 2; ++NP)
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(b_sweep_kernel(K, NP),
                                 cudaFuncAttributePreferredSharedMemoryCarveout, 50);
  // the pair sweeps keep most of the unified storage as L1: their row loads
  // are reused by neighbouring rows and by the next plane
  for (int d = 0; d < 3; ++d)
    for (bool perz : {false, true})
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(pair_kernel(d, perz), cudaFuncAttributePreferredSharedMemoryCarveout,
                                 25);
  const void* bp[10] = {(const void*)kb_pair<0, false>, (const void*)kb_pair<1, false>,
                        (const void*)kb_pair<2, false>, (const void*)kb_pair<0, true>,
                        (const void*)kb_pair<1, true>,  (const void*)kb_pair<2, true>,
                        (const void*)k_p_rb_pair<false>, (const void*)k_p_rb_pair<true>,
                        (const void*)kb_ppair<false>,   (const void*)kb_ppair<true>};
  for (const void* f : bp)
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 25);
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

const void* b_sweep_kernel(int K, int NP) {
  if (NP == 2)
    return K == 0 ? (const void*)kb_sweep<0, 2>
                  : K == 1 ? (const void*)kb_sweep<1, 2>
                           : K == 2 ? (const void*)kb_sweep<2, 2> : (const void*)kb_sweep<3, 2>;
  return K == 0 ? (const void*)kb_sweep<0, 1>
                : K == 1 ? (const void*)kb_sweep<1, 1>
                         : K == 2 ? (const void*)kb_sweep<2, 1> : (const void*)kb_sweep<3, 1>;
}

size_t b_sweep_smem(int NP, int TY, int W) {
  return (size_t)(NP + 2) * (TY + 2) * W * sizeof(float);
}

void launch_b_sweep(const BArgs& A, int K, int TY, int KC, int NP, int bx, size_t smem, int grid,
                    cudaStream_t s) {
  if (A.n <= 0) return;
  const dim3 block(bx, TY + 2, 1);
  void* args[] = {(void*)&A, (void*)&TY, (void*)&KC};
  cudaLaunchKernel(b_sweep_kernel(K, NP == 2 ? 2 : 1), dim3(grid), block, args, smem, s);
}

void launch_b_pair(const BArgs& A, int d, bool perz, int TY, int KC, int bx, size_t smem,
                   cudaStream_t s) {
  if (A.n <= 0) return;
  const dim3 block(bx, TY + 2, 1);
  if (perz) {
    if (d == 0) kb_pair<0, true><<<A.n, block, smem, s>>>(A, TY, KC);
    else if (d == 1) kb_pair<1, true><<<A.n, block, smem, s>>>(A, TY, KC);
    else kb_pair<2, true><<<A.n, block, smem, s>>>(A, TY, KC);
  } else {
    if (d == 0) kb_pair<0, false><<<A.n, block, smem, s>>>(A, TY, KC);
    else if (d == 1) kb_pair<1, false><<<A.n, block, smem, s>>>(A, TY, KC);
    else kb_pair<2, false><<<A.n, block, smem, s>>>(A, TY, KC);
  }
}

void launch_b_copy_back(const BArgs& A, int K, int grid, cudaStream_t s) {
  if (A.n <= 0) return;
  if (K == 0) kb_copy_back<0><<<grid, 256, 0, s>>>(A);
  else if (K == 1) kb_copy_back<1><<<grid, 256, 0, s>>>(A);
  else if (K == 2) kb_copy_back<2><<<grid, 256, 0, s>>>(A);
  else kb_copy_back<3><<<grid, 256, 0, s>>>(A);
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
