// Point updates of the one-pass red-black sweeps (Sec. 3.5), shared by the
// sweep kernels (smooth.cu) and the coarse-level cluster kernel (stencil.cu).
// COH = true reads every array the sweeps write (the iterates and right-hand
// sides) through L2 (ld.global.cg): a kernel that updates them in place and
// reads them back after a cluster barrier must not take them from the
// read-only cache. The arithmetic does not depend on COH.
#pragma once

#include "common.cuh"

namespace bf {
namespace {

template <bool COH, typename T>
__device__ __forceinline__ T ldm(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return *p;
}

// edge array of the (d, e) pair: xy 0, xz 1, yz 2
__host__ __device__ constexpr int pt_edge(int d, int e) {
  return (d < e ? d : e) + (d < e ? e : d) - 1;
}

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

// Pressure: the update from the iterate's current neighbours (the red
// points' old black neighbours, or the black points' new red ones). Neighbours
// are summed axis 0, 1, 2, lower then upper, as in the two-kernel sweep.
template <int D, typename T, bool COH = false>
__device__ __forceinline__ T p_red(const LevelPtrs<T>& L, const Pt& q, T h2) {
  T num = T(0), dg = T(0);
#pragma unroll
  for (int a = 0; a < D; ++a) {
    const T* __restrict__ b = L.beta[a];
    if (!q.wm[a]) {
      T bb = b[q.F];
      if constexpr (sizeof(T) == 4) px_acc(num, dg, bb, ldm<COH>(L.p + q.F + q.om[a]));
      else {
        num += bb * ldm<COH>(L.p + q.F + q.om[a]);
        dg += bb;
      }
    }
    if (!q.wp[a]) {
      T bb = b[q.F + q.op[a]];
      if constexpr (sizeof(T) == 4) px_acc(num, dg, bb, ldm<COH>(L.p + q.F + q.op[a]));
      else {
        num += bb * ldm<COH>(L.p + q.F + q.op[a]);
        dg += bb;
      }
    }
  }
  if constexpr (sizeof(T) == 4) return px_final(num, dg, h2, ldm<COH>(L.pf + q.F));
  else return (num - h2 * ldm<COH>(L.pf + q.F)) / dg;
}

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

template <int D, int d, typename T, bool COH = false>
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
    const T* __restrict__ me = L.mue[pt_edge(d, e)];
    const int Ep = F + q.op[e];
    T mep = me[Ep], mem = me[F];
    if constexpr (kIdg<T>)
      v.cross = vx_cross(v.cross, mep, ldm<COH>(ue + Ep), ldm<COH>(ue + Ep + od_m), mem,
                         ldm<COH>(ue + F), ldm<COH>(ue + F + od_m));
    else
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

template <int D, int d, typename T, bool COH = false>
__device__ __forceinline__ T v_red(const LevelPtrs<T>& L, const Pt& q, T ir) {
  VC<D, d, T> v;
  v_coef<D, d, T, COH>(L, q, ir, v);
  const T* __restrict__ ud = L.u[d];
  if constexpr (kIdg<T>) {
    float off = vx_off(v.cross, v.cdp, ldm<COH>(ud + q.F + q.op[d]), v.cdm,
                       ldm<COH>(ud + q.F + q.om[d]));
    int k = 0;
#pragma unroll
    for (int e = 0; e < D; ++e) {
      if (e == d) continue;
      if (!q.wp[e]) off = vx_acc(off, v.cep[k], ldm<COH>(ud + q.F + q.op[e]));
      if (!q.wm[e]) off = vx_acc(off, v.cem[k], ldm<COH>(ud + q.F + q.om[e]));
      ++k;
    }
    return vx_final(ldm<COH>(L.uf[d] + q.F), ir, off, v.diag);
  } else {
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
}

}  // namespace
}  // namespace bf
