// Lagrangian kernels: breakable Hookean springs (Eq. springF, Sec. 3.2),
// binning of nodes into cell tiles, the spreads of force and density
// (Eq. discrForceCouple, Eq. discrDensCouple) and of the viscosity maximum
// (Eq. ViscExp), and the velocity interpolation with the width-h delta
// (Eq. discrVelCouple) fused with the explicit Euler move of the nodes.
//
// Spreading: nodes are counting-sorted by the cell tile that holds them; one
// block per tile accumulates the contributions of its nodes in shared memory
// (the tile plus a halo as wide as the kernel support) and then flushes the
// non-zero entries to the grid with one global atomic each. When the support
// is too wide for the shared region, the block adds to the grid directly.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cmath>
#include <mutex>

#include "common.cuh"

namespace bf {

namespace {

constexpr int kBlock = 256;

// Eq. (PhiPeskin)
__device__ __forceinline__ double phi1(double r) {
  double a = fabs(r);
  if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
  if (a < 2.0) return (5.0 - 2.0 * a - sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) / 8.0;
  return 0.0;
}
// Eq. (PhiCosAlternative)
__device__ __forceinline__ double phi2(double r) {
  double a = fabs(r);
  if (a < 2.0) return 0.25 * (1.0 + cos(CUDART_PI * r / 2.0));
  return 0.0;
}
__device__ __forceinline__ double phi(int kind, double r) { return kind == 1 ? phi1(r) : phi2(r); }

// index of grid point i of a kind (stag: 0 face axis, 1 centre axis) along
// axis a, wrapped on periodic axes; -1 where the point would lie beyond a wall
__device__ __forceinline__ int kind_index(const Geo& g, int stag, int a, int i) {
  int n = g.n[a];
  if (g.per[a]) return ((i % n) + n) % n;
  int hi = stag ? n - 1 : n;
  return (i < 0 || i > hi) ? -1 : i;
}

__device__ __forceinline__ void support(const Geo& g, int stag, double X, double w, int& lo,
                                        int& hi) {
  double q = X / g.h - 0.5 * stag;
  double R = w / g.h;
  lo = (int)floor(q - 2.0 * R) + 1;
  hi = (int)ceil(q + 2.0 * R) - 1;
}

// Visit every point of the grid kind inside the support of width w around X:
// fn(i, j, k unwrapped, global index, prod of phi).
template <int D, typename Fn>
__device__ __forceinline__ void for_support(const Geo& g, const int stag[3], const double* X,
                                            double w, int kind, Fn fn) {
  int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
#pragma unroll
  for (int a = 0; a < D; ++a) support(g, stag[a], X[a], w, lo[a], hi[a]);
  for (int k = lo[2]; k <= hi[2]; ++k) {
    int kk = 0;
    double pz = 1.0;
    if constexpr (D == 3) {
      kk = kind_index(g, stag[2], 2, k);
      if (kk < 0) continue;
      pz = phi(kind, ((k + 0.5 * stag[2]) * g.h - X[2]) / w);
    }
    for (int j = lo[1]; j <= hi[1]; ++j) {
      int jj = kind_index(g, stag[1], 1, j);
      if (jj < 0) continue;
      double py = phi(kind, ((j + 0.5 * stag[1]) * g.h - X[1]) / w);
      for (int i = lo[0]; i <= hi[0]; ++i) {
        int ii = kind_index(g, stag[0], 0, i);
        if (ii < 0) continue;
        double px = phi(kind, ((i + 0.5 * stag[0]) * g.h - X[0]) / w);
        fn(i, j, k, gidx(g, ii, jj, kk), px * py * pz);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Springs: break test on the squared length without fused multiply-adds (so
// the decision matches a plain IEEE evaluation), then the tension
// T = K (|d| - r) pulls both nodes along d (Eq. springF). Each spring stores
// the force on its first node; every node then sums the forces of its
// springs in ascending spring order (a fixed order, so the sums do not depend
// on thread scheduling).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBlock) k_springs(int D, Geo g, NodeSet N, SpringSet S) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= S.m) return;
  double* fq = &S.fvec[3 * q];
  fq[0] = fq[1] = fq[2] = 0.0;
  if (S.broken[q]) return;
  int a = S.ab[2 * q], b = S.ab[2 * q + 1];
  double dv[3] = {0.0, 0.0, 0.0};
  for (int ax = 0; ax < D; ++ax) {
    double v = N.X[3 * (long long)b + ax] - N.X[3 * (long long)a + ax];
    if (g.per[ax]) {
      double Lx = g.n[ax] * g.h;
      if (v > 0.5 * Lx) v -= Lx;
      else if (v < -0.5 * Lx) v += Lx;
    }
    dv[ax] = v;
  }
  double len2 = __dadd_rn(__dmul_rn(dv[0], dv[0]), __dmul_rn(dv[1], dv[1]));
  len2 = __dadd_rn(len2, __dmul_rn(dv[2], dv[2]));
  double thr = __dmul_rn(__dadd_rn(1.0, S.brk[q]), S.rest[q]);
  if (len2 > __dmul_rn(thr, thr)) {
    S.broken[q] = 1;
    int slot = atomicAdd(S.ev_count, 1);
    if (slot < S.m) {
      S.ev_id[slot] = (int)q;
      S.ev_step[slot] = (int)(*S.step);
    }
    return;
  }
  double len = sqrt(len2);
  if (len == 0.0) return;
  double T = S.K[q] * (len - S.rest[q]);
  for (int ax = 0; ax < D; ++ax) fq[ax] = T * dv[ax] / len;
}

__global__ void __launch_bounds__(kBlock) k_node_force(NodeSet N, SpringSet S) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= N.eta) return;
  double F[3] = {0.0, 0.0, 0.0};
  for (int e = S.adj_start[s]; e < S.adj_start[s + 1]; ++e) {
    const int q = S.adj[e] >> 1;
    const bool second = (S.adj[e] & 1) != 0;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      double f = S.fvec[3 * (long long)q + ax];
      F[ax] += second ? -f : f;
    }
  }
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) N.F[3 * s + ax] = F[ax];
}

// ---------------------------------------------------------------------------
// Binning by cell tile (counting sort).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int tile_of(int D, const Geo& g, const TileGeo& tg, const double* X) {
  int t[3] = {0, 0, 0};
  for (int a = 0; a < D; ++a) {
    int c = (int)floor(X[a] / (tg.T[a] * g.h));
    t[a] = c < 0 ? 0 : (c >= tg.nt[a] ? tg.nt[a] - 1 : c);
  }
  return t[0] + tg.nt[0] * (t[1] + tg.nt[1] * t[2]);
}

__global__ void __launch_bounds__(kBlock) k_bin_count(int D, Geo g, TileGeo tg, NodeSet N) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= N.eta) return;
  int t = tile_of(D, g, tg, &N.X[3 * s]);
  N.tile[s] = t;
  atomicAdd(&N.count[t], 1);
}

// exclusive scan of the tile counts in one block
__global__ void __launch_bounds__(1024) k_bin_scan(TileGeo tg, NodeSet N) {
  __shared__ int part[1024];
  int nt = tg.ntiles;
  int per = (nt + blockDim.x - 1) / blockDim.x;
  int b0 = threadIdx.x * per, b1 = min(nt, b0 + per);
  int s = 0;
  for (int t = b0; t < b1; ++t) s += N.count[t];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - s;
  for (int t = b0; t < b1; ++t) {
    N.start[t] = run;
    N.cursor[t] = run;
    run += N.count[t];
  }
  if (threadIdx.x == blockDim.x - 1) N.start[nt] = part[threadIdx.x];
}

__global__ void __launch_bounds__(kBlock) k_bin_scatter(NodeSet N) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= N.eta) return;
  int pos = atomicAdd(&N.cursor[N.tile[s]], 1);
  N.perm[pos] = (int)s;
}

// ---------------------------------------------------------------------------
// Field reset before spreading: the f and rho sums start at zero, mu = mu_f
// everywhere.
// ---------------------------------------------------------------------------
struct FieldPtrs {
  double* frc[3];
  double* rho[3];
  double* muc;
  double* mue[3];
};

__global__ void __launch_bounds__(kBlock) k_reset(int D, Geo g, FieldPtrs P, double rho_f,
                                                  double mu_f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= g.s[0] || j >= g.s[1] || k >= g.s[2]) return;
  long long c = gidx(g, i, j, k);
  (void)rho_f;   // added back when the density sums are converted
  for (int d = 0; d < D; ++d) {
    P.frc[d][c] = 0.0;   // the bit pattern of the fixed-point zero
    P.rho[d][c] = 0.0;
  }
  P.muc[c] = mu_f;
  int ne = D == 3 ? 3 : 1;
  for (int e = 0; e < ne; ++e) P.mue[e][c] = mu_f;
}

// ---------------------------------------------------------------------------
// The width-w delta is a product of 1D factors, so each node evaluates phi
// once per axis and grid stagger (face: coordinate i h, centre: (i+1/2) h) and
// every grid point takes the product of three table entries, in the same
// order (x * y, then * z) as a direct evaluation.
// ---------------------------------------------------------------------------
constexpr int kP = 4;   // points per axis held in a table (support width <= 4 cells)

struct W1 {
  int lo, cnt;
  double w[kP];
};

__device__ __forceinline__ void weights1d(const Geo& g, int stag, int a, double X, double wid,
                                          int kind, W1& o) {
  int lo, hi;
  support(g, stag, X, wid, lo, hi);
  o.lo = lo;
  o.cnt = hi - lo + 1;
#pragma unroll
  for (int q = 0; q < kP; ++q)
    o.w[q] = (q < o.cnt) ? phi(kind, ((lo + q + 0.5 * stag) * g.h - X) / wid) : 0.0;
}

// Visit the points of a grid kind inside the support, with tabulated
// weights: fn(i, j, k unwrapped, global index, prod of phi).
template <int D, typename Fn>
__device__ __forceinline__ void for_table(const Geo& g, const int stag[3], const W1* wx,
                                          const W1* wy, const W1* wz, Fn fn) {
  int kcnt = (D == 3) ? wz->cnt : 1;
  for (int kq = 0; kq < kcnt; ++kq) {
    int k = 0, kk = 0;
    double pz = 1.0;
    if constexpr (D == 3) {
      k = wz->lo + kq;
      kk = kind_index(g, stag[2], 2, k);
      if (kk < 0) continue;
      pz = wz->w[kq];
    }
    for (int jq = 0; jq < wy->cnt; ++jq) {
      int j = wy->lo + jq;
      int jj = kind_index(g, stag[1], 1, j);
      if (jj < 0) continue;
      double py = wy->w[jq];
      for (int iq = 0; iq < wx->cnt; ++iq) {
        int i = wx->lo + iq;
        int ii = kind_index(g, stag[0], 0, i);
        if (ii < 0) continue;
        double px = wx->w[iq];
        fn(i, j, k, gidx(g, ii, jj, kk), px * py * pz);
      }
    }
  }
}

// Per-node visitor: with TAB (support of at most kP points per axis, i.e.
// width <= h) the 1D tables are filled once; otherwise phi is evaluated per
// point.
template <int D, bool TAB>
struct NodeVisit {
  W1 wf[3], wc[3];
  const double* X;
  double wid;
  int kind;
  __device__ __forceinline__ void init(const Geo& g, const double* X_, double w_, int kind_) {
    X = X_;
    wid = w_;
    kind = kind_;
    if constexpr (TAB) {
#pragma unroll
      for (int a = 0; a < D; ++a) {
        weights1d(g, 0, a, X[a], wid, kind, wf[a]);
        weights1d(g, 1, a, X[a], wid, kind, wc[a]);
      }
    }
  }
  template <typename Fn>
  __device__ __forceinline__ void visit(const Geo& g, const int stag[3], Fn fn) {
    if constexpr (TAB)
      for_table<D>(g, stag, stag[0] ? &wc[0] : &wf[0], stag[1] ? &wc[1] : &wf[1],
                   stag[2] ? &wc[2] : &wf[2], fn);
    else
      for_support<D>(g, stag, X, wid, kind, fn);
  }
};

// ---------------------------------------------------------------------------
// Tile spread. Shared region per axis: [t T - H, t T + T + H). Pass 1 holds
// f_d and rho_d of every face grid at once; pass 2 the viscosity maximum of
// the centres and edges.
// ---------------------------------------------------------------------------
struct SpreadK {
  Geo g;
  TileGeo tg;
  NodeSet N;
  SpreadArgs a;
  FieldPtrs P;
  int use_smem;
  int cmax;        // support points per axis at most
  int same_width;  // omega_mu == omega: the viscosity pass reuses table 0
  int R[3];
  int vol;
};

__device__ __forceinline__ unsigned long long dbits(double v) {
  return (unsigned long long)__double_as_longlong(v);
}

// ---------------------------------------------------------------------------
// Per-node 1D weight tables, one thread per (node, width, stagger, axis):
// lo/cnt of the support and phi at its points. Width 0 is omega (force and
// density), width 1 omega_mu (viscosity).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int tab_index(long long s, int wid, int stag, int a) {
  return (int)(((s * 2 + wid) * 2 + stag) * 3 + a);
}

__global__ void __launch_bounds__(kBlock) k_node_tables(int D, Geo g, NodeSet N, double w0,
                                                        double w1, int kind) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= N.eta * 12) return;
  int a = (int)(q % 3);
  int stag = (int)((q / 3) % 2);
  int wid = (int)((q / 6) % 2);
  long long s = q / 12;
  if (a >= D) return;
  double w = wid ? w1 : w0;
  double X = N.X[3 * s + a];
  int lo, hi;
  support(g, stag, X, w, lo, hi);
  int t = tab_index(s, wid, stag, a);
  N.tlo[2 * t] = lo;
  N.tlo[2 * t + 1] = hi - lo + 1;
#pragma unroll
  for (int k = 0; k < kP; ++k)
    N.tw[kP * t + k] = (k <= hi - lo) ? phi(kind, ((lo + k + 0.5 * stag) * g.h - X) / w) : 0.0;
}

// ---------------------------------------------------------------------------
// Tile spread: one block per cell tile, one grid kind at a time. Work items
// are (node, support point) pairs, so dense tiles keep every thread busy;
// contributions meet in shared memory over the tile region [t T - H,
// t T + T + H) and leave with one global atomic per non-zero entry.
// With TAB the weights come from the node tables, otherwise phi is evaluated
// per point (supports wider than the tables).
// ---------------------------------------------------------------------------
constexpr int kSpreadThreads = 512;

template <int D, bool TAB>
__global__ void __launch_bounds__(kSpreadThreads) k_spread(SpreadK A) {
  extern __shared__ double smem[];
  const Geo& g = A.g;
  const int t = blockIdx.x;
  const int s0 = A.N.start[t], s1 = A.N.start[t + 1];
  if (s0 == s1) return;
  const int nn = s1 - s0;
  const int tc[3] = {t % A.tg.nt[0], (t / A.tg.nt[0]) % A.tg.nt[1],
                     t / (A.tg.nt[0] * A.tg.nt[1])};
  int base[3];
  for (int a = 0; a < 3; ++a) base[a] = (a < D) ? tc[a] * A.tg.T[a] - A.tg.H : 0;
  const int vol = A.vol;
  const bool sm = A.use_smem != 0;
  const int kind = A.a.phi_kind;
  const int C = A.cmax;                       // support points per axis at most
  const int slots = (D == 3) ? C * C * C : C * C;
  // index in the tile region, or -1 (global atomic) for a point outside it,
  // which only a node outside the domain can reach
  auto local = [&](int i, int j, int k) -> int {
    int li = i - base[0], lj = j - base[1], lk = D == 3 ? k - base[2] : 0;
    if ((unsigned)li >= (unsigned)A.R[0] || (unsigned)lj >= (unsigned)A.R[1] ||
        (D == 3 && (unsigned)lk >= (unsigned)A.R[2]))
      return -1;
    return li + A.R[0] * (lj + A.R[1] * lk);
  };
  auto flush_index = [&](int q, const int stag[3]) -> long long {
    int li = q % A.R[0];
    int lj = (q / A.R[0]) % A.R[1];
    int lk = q / (A.R[0] * A.R[1]);
    int gi = kind_index(g, stag[0], 0, base[0] + li);
    int gj = kind_index(g, stag[1], 1, base[1] + lj);
    int gk = 0;
    if (D == 3) gk = kind_index(g, stag[2], 2, base[2] + lk);
    if (gi < 0 || gj < 0 || gk < 0) return -1;
    return gidx(g, gi, gj, gk);
  };
  // visit item (node p, slot) of grid kind `stag` at width index wid:
  // fn(local index or -1, global index, prod of phi)
  auto item = [&](int p, int slot, const int stag[3], int wid, double w, auto fn) {
    int sidx = A.N.perm[p];
    const double* X = &A.N.X[3 * (long long)sidx];
    (void)X;
    int off[3] = {slot % C, (slot / C) % C, D == 3 ? slot / (C * C) : 0};
    int idx[3] = {0, 0, 0}, gl[3] = {0, 0, 0};
    double pr[3] = {1.0, 1.0, 1.0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
      int lo, cnt;
      double wt;
      if constexpr (TAB) {
        int ti = tab_index(sidx, wid, stag[a], a);
        lo = A.N.tlo[2 * ti];
        cnt = A.N.tlo[2 * ti + 1];
        if (off[a] >= cnt) return;
        wt = A.N.tw[kP * ti + off[a]];
      } else {
        int hi;
        support(g, stag[a], X[a], w, lo, hi);
        cnt = hi - lo + 1;
        if (off[a] >= cnt) return;
        wt = phi(kind, ((lo + off[a] + 0.5 * stag[a]) * g.h - X[a]) / w);
      }
      idx[a] = lo + off[a];
      gl[a] = kind_index(g, stag[a], a, idx[a]);
      if (gl[a] < 0) return;
      pr[a] = wt;
    }
    fn(sm ? local(idx[0], idx[1], idx[2]) : -1, gidx(g, gl[0], gl[1], gl[2]),
       pr[0] * pr[1] * pr[2]);
  };
  const double winvD =
      1.0 / (D == 3 ? A.a.omega * A.a.omega * A.a.omega : A.a.omega * A.a.omega);
  const double winvDm =
      1.0 / (D == 3 ? A.a.omega_mu * A.a.omega_mu * A.a.omega_mu : A.a.omega_mu * A.a.omega_mu);
  const long long items = (long long)nn * slots;

  // force and density, one face grid at a time, summed as 64-bit fixed-point
  // integers (every contribution rounded once, at the scale of the step's
  // bound on the sums): integer addition is associative, so the result does
  // not depend on the order in which threads and blocks add
  const double sf = A.a.scale[0], sr = A.a.scale[1];
  for (int d = 0; d < D; ++d) {
    int stag[3] = {1, 1, 1};
    stag[d] = 0;
    unsigned long long* accF = reinterpret_cast<unsigned long long*>(smem);
    unsigned long long* accR = accF + vol;
    if (sm) {
      for (int q = threadIdx.x; q < 2 * vol; q += blockDim.x) accF[q] = 0ull;
      __syncthreads();
    }
    unsigned long long* gF = reinterpret_cast<unsigned long long*>(A.P.frc[d]);
    unsigned long long* gR = reinterpret_cast<unsigned long long*>(A.P.rho[d]);
    for (long long it = threadIdx.x; it < items; it += blockDim.x) {
      int p = s0 + (int)(it / slots), slot = (int)(it % slots);
      double Fd = A.N.F[3 * (long long)A.N.perm[p] + d];
      item(p, slot, stag, 0, A.a.omega, [&](int l, long long gi, double w) {
        double wt = winvD * w;
        const unsigned long long cf = (unsigned long long)llrint(Fd * wt * sf);
        const unsigned long long cr = (unsigned long long)llrint(A.a.amp_rho * wt * sr);
        if (l >= 0) {
          if (cf) atomicAdd(&accF[l], cf);
          if (cr) atomicAdd(&accR[l], cr);
        } else {
          if (cf) atomicAdd(&gF[gi], cf);
          if (cr) atomicAdd(&gR[gi], cr);
        }
      });
    }
    if (sm) {
      __syncthreads();
      for (int q = threadIdx.x; q < vol; q += blockDim.x) {
        unsigned long long vf = accF[q], vr = accR[q];
        if (vf == 0ull && vr == 0ull) continue;
        long long gi = flush_index(q, stag);
        if (gi < 0) continue;
        if (vf) atomicAdd(&gF[gi], vf);
        if (vr) atomicAdd(&gR[gi], vr);
      }
      __syncthreads();
    }
  }

  // viscosity maximum, one grid at a time (positive doubles order like their
  // bit patterns, so an unsigned 64-bit max is a floating max)
  unsigned long long* accM = reinterpret_cast<unsigned long long*>(smem);
  const unsigned long long floor_bits = dbits(A.a.mu_out);
  const int nkinds = D == 3 ? 4 : 2;
  for (int kk = 0; kk < nkinds; ++kk) {
    int stag[3] = {1, 1, 1};
    double* target = A.P.muc;
    if (kk > 0) {
      int e = kk - 1;  // 0: xy, 1: xz, 2: yz
      stag[(e == 2) ? 1 : 0] = 0;
      stag[(e == 0) ? 1 : 2] = 0;
      target = A.P.mue[e];
    }
    if (sm) {
      for (int q = threadIdx.x; q < vol; q += blockDim.x) accM[q] = 0ull;
      __syncthreads();
    }
    for (long long it = threadIdx.x; it < items; it += blockDim.x) {
      int p = s0 + (int)(it / slots), slot = (int)(it % slots);
      item(p, slot, stag, A.same_width ? 0 : 1, A.a.omega_mu, [&](int l, long long gi, double w) {
        double cand = A.a.mu_coef * (winvDm * w) + A.a.mu_out;
        if (l >= 0) atomicMax(&accM[l], dbits(cand));
        else atomicMax(reinterpret_cast<unsigned long long*>(&target[gi]), dbits(cand));
      });
    }
    if (sm) {
      __syncthreads();
      for (int q = threadIdx.x; q < vol; q += blockDim.x) {
        unsigned long long v = accM[q];
        if (v <= floor_bits) continue;
        long long gi = flush_index(q, stag);
        if (gi < 0) continue;
        atomicMax(reinterpret_cast<unsigned long long*>(&target[gi]), v);
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// U(s) = sum_x u_d(x) prod phi((x - X)/h) on each component's own grid
// (Eq. discrVelCouple), then X += (dt/sigma) U with the periodic wrap and the
// wall clamp.
// ---------------------------------------------------------------------------
struct Ptr3c {
  const double* a[3];
};

template <int D>
__global__ void __launch_bounds__(kBlock) k_interp_advance(Geo g, NodeSet N, Ptr3c u, int kind,
                                                           double c) {
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= N.eta) return;
  double X[3] = {N.X[3 * s], N.X[3 * s + 1], N.X[3 * s + 2]};
  double U[3] = {0.0, 0.0, 0.0};
  NodeVisit<D, true> nv;   // width h: at most 4 points per axis
  nv.init(g, X, g.h, kind);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    int stag[3] = {1, 1, 1};
    stag[d] = 0;
    const double* __restrict__ ud = u.a[d];
    double v = 0.0;
    nv.visit(g, stag, [&](int, int, int, long long gi, double w) { v += ud[gi] * w; });
    U[d] = v;
  }
  int clamped = 0, bad = 0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    N.U[3 * s + d] = U[d];
    double x = X[d] + c * U[d];
    double Lx = g.n[d] * g.h;
    if (!isfinite(x)) {
      // a run that has blown up: keep the node inside the grid so that every
      // later kernel stays in bounds, and count it
      x = 0.0;
      ++bad;
    } else if (g.per[d]) {
      if (x >= Lx) x -= Lx;
      else if (x < 0.0) x += Lx;
      if (!(x >= 0.0 && x < Lx)) {   // moved by more than one period
        x -= Lx * floor(x / Lx);
        if (!(x >= 0.0 && x < Lx)) x = 0.0;
      }
    } else {
      if (x < 0.0) { x = 0.0; ++clamped; }
      else if (x > Lx) { x = Lx; ++clamped; }
    }
    N.X[3 * s + d] = x;
  }
  if (clamped) atomicAdd(N.clamped, clamped);
  if (bad) atomicAdd(N.nonfinite, bad);
}

__global__ void k_step_increment(long long* step) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step += 1;
}

inline dim3 blk3(int D) { return D == 3 ? dim3(32, 4, 2) : dim3(32, 8, 1); }
inline dim3 grd3(long long nx, long long ny, long long nz, dim3 b) {
  return dim3((unsigned)((nx + b.x - 1) / b.x), (unsigned)((ny + b.y - 1) / b.y),
              (unsigned)((nz + b.z - 1) / b.z));
}

}  // namespace

// ===========================================================================
void launch_springs(int D, const Geo& g, const NodeSet& N, const SpringSet& S, cudaStream_t s) {
  if (N.eta <= 0) return;
  if (S.m <= 0 || S.adj_eta != N.eta) {
    cudaMemsetAsync(N.F, 0, sizeof(double) * 3 * N.eta, s);
    return;
  }
  unsigned nb = (unsigned)((S.m + kBlock - 1) / kBlock);
  k_springs<<<nb, kBlock, 0, s>>>(D, g, N, S);
  k_node_force<<<(unsigned)((N.eta + kBlock - 1) / kBlock), kBlock, 0, s>>>(N, S);
}

void launch_bin(int D, const Geo& g, const TileGeo& tg, const NodeSet& N, cudaStream_t s) {
  cudaMemsetAsync(N.count, 0, sizeof(int) * (tg.ntiles + 1), s);
  if (N.eta > 0) {
    unsigned nb = (unsigned)((N.eta + kBlock - 1) / kBlock);
    k_bin_count<<<nb, kBlock, 0, s>>>(D, g, tg, N);
  }
  k_bin_scan<<<1, 1024, 0, s>>>(tg, N);
  if (N.eta > 0) {
    unsigned nb = (unsigned)((N.eta + kBlock - 1) / kBlock);
    k_bin_scatter<<<nb, kBlock, 0, s>>>(N);
  }
}

void launch_reset_fields(int D, const Geo& g, double* frc[3], double* rho[3], double* muc,
                         double* mue[3], double rho_f, double mu_f, cudaStream_t s) {
  FieldPtrs P;
  for (int d = 0; d < 3; ++d) {
    P.frc[d] = frc[d];
    P.rho[d] = rho[d];
    P.mue[d] = mue[d];
  }
  P.muc = muc;
  dim3 b = blk3(D);
  k_reset<<<grd3(g.s[0], g.s[1], g.s[2], b), b, 0, s>>>(D, g, P, rho_f, mu_f);
}

static void region(int D, const TileGeo& tg, int R[3], int& vol) {
  vol = 1;
  for (int a = 0; a < 3; ++a) {
    R[a] = (a < D) ? tg.T[a] + 2 * tg.H : 1;
    vol *= R[a];
  }
}

// one grid kind at a time: f and rho of one face grid, or one mu grid
size_t spread_smem_bytes(int D, const TileGeo& tg) {
  int R[3], vol;
  region(D, tg, R, vol);
  return (size_t)2 * vol * sizeof(double);
}

size_t spread_smem_limit() { return 200 * 1024; }

bool spread_fits_tables(double omega, double omega_mu, double h) {
  // a width-w support covers fewer than 4 w / h + 1 points per axis: at most 4
  // when w <= h
  double w = omega > omega_mu ? omega : omega_mu;
  return w <= h;
}

namespace {

// Scales of the fixed-point sums: the largest power of two S with
// S * bound < 2^61, where bound >= |any partial sum| (the sum over nodes of
// the largest force component times the delta's peak omega^-D, and eta times
// rho_b d0^D omega^-D). One block sums in a fixed order, so the scales, and
// with them every rounded contribution, are the same in every run.
__global__ void __launch_bounds__(1024) k_spread_scale(NodeSet N, int D, double winvD, double amp,
                                                       double* scale) {
  __shared__ double part[1024];
  double v = 0.0;
  for (long long s = threadIdx.x; s < N.eta; s += blockDim.x) {
    double m = 0.0;
    for (int a = 0; a < D; ++a) m = fmax(m, fabs(N.F[3 * s + a]));
    v += m;
  }
  part[threadIdx.x] = v;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) part[threadIdx.x] += part[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double bound[2] = {part[0] * winvD, (double)N.eta * fabs(amp) * winvD};
    for (int k = 0; k < 2; ++k) {
      int e = 0;
      frexp(bound[k], &e);   // bound < 2^e
      scale[k] = (bound[k] > 0.0 && isfinite(bound[k])) ? ldexp(1.0, 61 - e) : 1.0;
    }
  }
}

__global__ void __launch_bounds__(kBlock) k_spread_finish(int D, Geo g, Ptr3d frc, Ptr3d rho,
                                                          const double* __restrict__ scale,
                                                          double rho_f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  int k = blockIdx.z * blockDim.z + threadIdx.z;
  if (i >= g.s[0] || j >= g.s[1] || k >= g.s[2]) return;
  long long c = gidx(g, i, j, k);
  const double inv_f = 1.0 / scale[0], inv_r = 1.0 / scale[1];   // powers of two: exact
  for (int d = 0; d < D; ++d) {
    long long vf = (long long)__double_as_longlong(frc.a[d][c]);
    long long vr = (long long)__double_as_longlong(rho.a[d][c]);
    frc.a[d][c] = vf ? (double)vf * inv_f : 0.0;
    rho.a[d][c] = rho_f + (vr ? (double)vr * inv_r : 0.0);
  }
}

}  // namespace

void launch_spread_finish(int D, const Geo& g, const SpreadArgs& a, double* frc[3], double* rho[3],
                          cudaStream_t s) {
  Ptr3d F, R;
  for (int d = 0; d < 3; ++d) {
    F.a[d] = frc[d];
    R.a[d] = rho[d];
  }
  dim3 b = blk3(D);
  k_spread_finish<<<grd3(g.s[0], g.s[1], g.s[2], b), b, 0, s>>>(D, g, F, R, a.scale, a.rho_f);
}

void launch_spread(int D, const Geo& g, const TileGeo& tg, const NodeSet& N, const SpreadArgs& a,
                   double* frc[3], double* rho[3], double* muc, double* mue[3], cudaStream_t s) {
  if (N.eta <= 0) return;
  {
    const double w = a.omega;
    k_spread_scale<<<1, 1024, 0, s>>>(N, D, 1.0 / (D == 3 ? w * w * w : w * w), a.amp_rho, a.scale);
  }
  SpreadK A;
  A.g = g;
  A.tg = tg;
  A.N = N;
  A.a = a;
  for (int d = 0; d < 3; ++d) {
    A.P.frc[d] = frc[d];
    A.P.rho[d] = rho[d];
    A.P.mue[d] = mue[d];
  }
  A.P.muc = muc;
  region(D, tg, A.R, A.vol);
  size_t smem = spread_smem_bytes(D, tg);
  A.use_smem = smem <= spread_smem_limit() ? 1 : 0;
  if (!A.use_smem) smem = 0;
  bool tab = spread_fits_tables(a.omega, a.omega_mu, g.h);
  double Rw = (a.omega > a.omega_mu ? a.omega : a.omega_mu) / g.h;
  A.cmax = (int)std::floor(4.0 * Rw) + 1;
  if (tab && A.cmax > kP) A.cmax = kP;
  A.same_width = a.omega == a.omega_mu;
  if (tab) {
    long long q = N.eta * 12;
    k_node_tables<<<(unsigned)((q + kBlock - 1) / kBlock), kBlock, 0, s>>>(
        D, g, N, a.omega, a.omega_mu, a.phi_kind);
  }
  if (D == 3) {
    if (tab) k_spread<3, true><<<tg.ntiles, kSpreadThreads, smem, s>>>(A);
    else k_spread<3, false><<<tg.ntiles, kSpreadThreads, smem, s>>>(A);
  } else {
    if (tab) k_spread<2, true><<<tg.ntiles, kSpreadThreads, smem, s>>>(A);
    else k_spread<2, false><<<tg.ntiles, kSpreadThreads, smem, s>>>(A);
  }
}

// The limit is a property of the kernel, shared by every context of the
// process: it only ever grows, so that a context needing less never lowers it
// below what another context's captured launches use.
cudaError_t spread_set_smem(int D, size_t bytes) {
  static std::mutex mu;
  static size_t granted[4] = {0, 0, 0, 0};
  std::lock_guard<std::mutex> lock(mu);
  if (bytes <= granted[D]) return cudaSuccess;
  cudaError_t e;
  if (D == 3) {
    e = cudaFuncSetAttribute(k_spread<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_spread<3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  } else {
    e = cudaFuncSetAttribute(k_spread<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_spread<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  }
  if (e == cudaSuccess) granted[D] = bytes;
  return e;
}

void launch_interp_advance(int D, const Geo& g, const NodeSet& N, double* const uvel[3],
                           int phi_kind, double dt_over_sigma, cudaStream_t s) {
  if (N.eta <= 0) return;
  Ptr3c u;
  for (int d = 0; d < 3; ++d) u.a[d] = uvel[d];
  unsigned nb = (unsigned)((N.eta + kBlock - 1) / kBlock);
  if (D == 3) k_interp_advance<3><<<nb, kBlock, 0, s>>>(g, N, u, phi_kind, dt_over_sigma);
  else k_interp_advance<2><<<nb, kBlock, 0, s>>>(g, N, u, phi_kind, dt_over_sigma);
}

void launch_step_increment(long long* step, cudaStream_t s) {
  k_step_increment<<<1, 32, 0, s>>>(step);
}

}  // namespace bf
