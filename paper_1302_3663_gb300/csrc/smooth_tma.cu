// Red-black Gauss-Seidel sweeps (Sec. 3.5) with their inputs staged in
// shared memory by the Tensor Memory Accelerator: an alternative 3D FP32
// smoother of the mixed-precision V-cycles, and the autotuner that chooses,
// per level shape and sweep kind, between it and the one-pass sweep of
// smooth.cu (and the one-pass sweep's tile shape).
//
// The arithmetic of every point update is that of the one-pass sweep (FP32
// viscous updates multiply by the precomputed inverse diagonal); only the
// data movement differs. A
// block owns a strip of x (64 columns or whole rows), TY rows of y and a
// chunk of planes along z. For every plane one elected thread issues one
// tiled TMA copy per input array (a box of TY + 4 rows and the strip plus
// four halo columns each side) into a window of plane slots, up to three
// planes ahead of the computation; completion is tracked by
// transaction-count mbarriers. Each phase computes the red values of plane k
// (on the block's rows and columns plus one ring row / column each side,
// from old black values) into a four-plane ring and, independently, the black
// values of plane k - 2 from the ring; one barrier separates phases. The
// sweep is out of place.
//
// Blocks are persistent: block b takes the work items (strip, row tile,
// plane chunk) b, b + G, b + 2G, ..., so the items in flight at any moment are
// neighbours and share their halo rows through L2.
//
// Every wait on an mbarrier is bounded (2 s of the global timer by default;
// a context may set a shorter limit, 0 testing each barrier once without
// waiting). A block whose wait runs out raises the error word, drains its own
// copies in flight from the first one it has not seen complete (bounded by
// the default limit, whatever the context's) and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "common.cuh"

namespace bf {

namespace {

constexpr int kNB = 8;                  // mbarriers (planes in flight <= PD + 1 <= 4)
constexpr int kMaxPD = 3;               // prefetch distance in planes, at most
constexpr int kRing = 4;                // ring planes of red values: k-3 .. k
constexpr int kTmaThreads = 1024;       // threads per block at most
constexpr unsigned long long kWaitNs = kTmaWaitNs;   // the drain's limit
constexpr size_t kSmemMax = 225 * 1024;   // dynamic, leaving room for the static words

// Staged arrays. Viscous component d (kinds 0, 1, 2): old u_d, rhs_d, the
// inverse diagonal of component d, mu_c, the two edge viscosities of d and the
// two other components (axes e1 < e2). Pressure (kind 3): old p, rhs, beta_x, beta_y, beta_z.
__host__ __device__ constexpr int n_staged(int K) { return K == 3 ? 5 : 8; }

// Plane slots: the planes a block still reads at iteration k (k-2 .. k+1:
// the red plane k with its neighbours and the black plane k-2 with its
// neighbours; k-3 as well for the z component, whose stencil reaches one
// plane below the point) plus the PD planes in flight.
__host__ __device__ constexpr int win(int K, int PD) { return (K == 2 ? 5 : 4) + PD; }
__host__ __device__ constexpr int total_slots(int K, int PD) { return win(K, PD) * n_staged(K); }

struct TmaArgs {
  CUtensorMap map[8];
  Geo g;
  float* out;
  int* err;
  int TY, KC, nrt, ns, items;
  int SW, BW, RW;        // strip columns, box columns (SW + 8), ring row floats
  int PD;                // planes issued ahead of the red plane's last need
  int tile;              // floats between array tiles (multiple of 32)
  unsigned box_bytes;    // bytes of one box: (TY + 4) rows of BW floats
  float c;               // viscous: inv_re / h^2; pressure: h^2
  unsigned long long wait_ns;   // limit of each main-loop wait (0: test once)
};

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map,
                                            unsigned long long* b, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(smem_addr(b)), "r"(x), "r"(y), "r"(z)
      : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait for the completion of sequence number s (barrier s % kNB,
// phase parity (s / kNB) & 1); limit 0 tests the barrier once
__device__ __forceinline__ bool wait_seq(unsigned long long* bar, unsigned s,
                                         unsigned long long limit_ns) {
  unsigned long long* b = &bar[s % kNB];
  unsigned par = (s / kNB) & 1u;
  if (limit_ns == 0) return mbar_test_wait(b, par);
  if (mbar_try_wait(b, par)) return true;
  unsigned long long t0 = global_ns();
  while (!mbar_try_wait(b, par))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}

__device__ __forceinline__ int wrapi(int i, int n) { return ((i % n) + n) % n; }

__host__ __device__ constexpr int edge_id(int d, int e) {
  return (d < e ? d : e) + (d < e ? e : d) - 1;
}

// ------------------------------------------------------------------ kernel
// Shared memory: W plane slots, each holding one tile per staged array
// (tile = TY + 4 rows of BW = SW + 8 floats: the strip's columns with four
// halo columns each side); then the three-plane ring of red values (TY + 2
// rows of RW floats, column c holding x = xs - 1 + c); then the mbarriers.
// Plane p of a chunk lives in slot (p - pbase) % W.
template <int K>
__global__ void __launch_bounds__(kTmaThreads) k_rb_tma(const __grid_constant__ TmaArgs A) {
  constexpr int NS = n_staged(K);
  const int PD = A.PD, W = win(K, PD);
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ int abort_flag;
  const Geo& g = A.g;
  const int TY = A.TY, BW = A.BW, RW = A.RW, SW = A.SW, tile = A.tile;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const bool per0 = g.per[0] != 0, per2 = g.per[2] != 0;
  const long long st1 = g.st[1], st2 = g.st[2];
  float* tiles = reinterpret_cast<float*>(sm);
  float* ring = tiles + (size_t)W * NS * tile;
  const int ringplane = (TY + 2) * RW;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(ring + kRing * ringplane);
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int q = tid; q < kRing * ringplane; q += nthr) ring[q] = 0.f;
  if (tid == 0) {
    abort_flag = 0;
    for (int b = 0; b < kNB; ++b) mbar_init(&bar[b], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const float c = A.c;
  // this thread's red item (row r of TY + 2, pair q of SW / 2 + 2, the first
  // one left of the strip) and black item (row r of TY, pair q of SW / 2)
  const int rpairs = SW / 2 + 2, bpairs = SW / 2;
  const bool has_red = tid < (TY + 2) * rpairs, has_blk = tid < TY * bpairs;
  const int r_red = tid / rpairs, q_red = tid - r_red * rpairs;
  const int r_blk = tid / bpairs, q_blk = tid - r_blk * bpairs;
  unsigned seq = 0, waited = 0;   // planes issued / waited for by this block

  for (int item = blockIdx.x; item < A.items; item += gridDim.x) {
    const int strip = item % A.ns, rest = item / A.ns;
    const int t = rest % A.nrt, ch = rest / A.nrt;
    const int xs = strip * SW, j0 = t * TY, k0 = ch * A.KC, k1 = min(k0 + A.KC, n2);
    const int pbase = k0 - 2;   // plane in slot 0 at the start of the chunk
    const unsigned sbase = seq;
    auto plane_tiles = [&](int p) -> float* {
      return tiles + (size_t)((p - pbase) % W) * NS * tile;
    };
    auto issue = [&](int p) {   // one thread: plane p of every staged array
      unsigned long long* b = &bar[(sbase + (unsigned)(p - pbase)) % kNB];
      fence_proxy_async();
      mbar_expect_tx(b, (unsigned)NS * A.box_bytes);
      int z = per2 ? wrapi(p, n2) : p;
      float* dst = plane_tiles(p);
#pragma unroll
      for (int a = 0; a < NS; ++a)
        tma_load_3d(dst + a * tile, &A.map[a], b, xs - 4, j0 - 2, z);
    };
    const int last0 = min(pbase + 1 + PD, k1 + 1);
    if (tid == 0)
      for (int p = pbase; p <= last0; ++p) issue(p);
    seq += (unsigned)(last0 - pbase + 1);

    // One point update. P0 (Pm, Pp) are the tiles of the point's plane (and
    // of the planes below and above), o its offset in a tile, dxp / dxm the
    // offsets of its x neighbours; BLACK reads the iterate's neighbours from
    // the ring (planes Rm, R0, Rp; offset ro; x neighbours at ro + rxp /
    // ro + rxm), red from the staged old values. INTERIOR: no neighbour lies
    // beyond a wall or across a periodic seam, so every flag is false and
    // every x offset is +-1 (the same arithmetic with the branches removed).
    auto update = [&](auto black_tag, auto interior_tag, const float* Pm, const float* P0,
                      const float* Pp, int o, int dxp, int dxm, const float* Rm,
                      const float* R0, const float* Rp, int ro, int rxp, int rxm,
                      const bool* wmv, const bool* wpv) -> float {
      constexpr bool BLACK = decltype(black_tag)::value;
      constexpr bool INTERIOR = decltype(interior_tag)::value;
      auto wm = [&](int a) -> bool {
        if constexpr (INTERIOR) return false;
        else return wmv[a];
      };
      auto wp = [&](int a) -> bool {
        if constexpr (INTERIOR) return false;
        else return wpv[a];
      };
      const int xp = INTERIOR ? 1 : dxp, xm = INTERIOR ? -1 : dxm;
      const int rp = INTERIOR ? 1 : rxp, rm = INTERIOR ? -1 : rxm;
      auto nb = [&](int ax, int side) -> float {   // neighbour of the iterate (array 0)
        if constexpr (BLACK) {
          if (ax == 0) return R0[ro + (side > 0 ? rp : rm)];
          if (ax == 1) return R0[ro + side * RW];
          return (side > 0 ? Rp : Rm)[ro];
        } else {
          if (ax == 0) return P0[o + (side > 0 ? xp : xm)];
          if (ax == 1) return P0[o + side * BW];
          return (side > 0 ? Pp : Pm)[o];
        }
      };
      // staged array a at the point shifted by s1 along ax1 and s2 along ax2
      auto sh = [&](int a, int ax1, int s1, int ax2, int s2) -> float {
        const float* P = P0;
        int off = o + a * tile;
        if (s1 != 0) {
          if (ax1 == 0) off += s1 > 0 ? xp : xm;
          else if (ax1 == 1) off += s1 * BW;
          else P = s1 > 0 ? Pp : Pm;
        }
        if (s2 != 0) {
          if (ax2 == 0) off += s2 > 0 ? xp : xm;
          else if (ax2 == 1) off += s2 * BW;
          else P = s2 > 0 ? Pp : Pm;
        }
        return P[off];
      };
      auto at = [&](int a) -> float { return P0[o + a * tile]; };
      if constexpr (K == 3) {
        float num = 0.f, dg = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (!wm(a)) px_acc(num, dg, at(2 + a), nb(a, -1));
          if (!wp(a)) px_acc(num, dg, sh(2 + a, a, +1, 0, 0), nb(a, +1));
        }
        return px_final(num, dg, c, at(1));
      } else {
        constexpr int d = K;
        constexpr int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
        float mcp = at(3), mcm = sh(3, d, -1, 0, 0);
        float cdp = 2.f * mcp, cdm = 2.f * mcm;
        float cross = 0.f;
        float cep[2], cem[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int e = q == 0 ? e1 : e2;
          const int me = 4 + q, ue = 6 + q;
          float mep = sh(me, e, +1, 0, 0), mem = at(me);
          cross = vx_cross(cross, mep, sh(ue, e, +1, 0, 0), sh(ue, e, +1, d, -1), mem, at(ue),
                           sh(ue, d, -1, 0, 0));
          cep[q] = mep;
          cem[q] = mem;
        }
        float off = vx_off(cross, cdp, nb(d, +1), cdm, nb(d, -1));
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int e = q == 0 ? e1 : e2;
          if (!wp(e)) off = vx_acc(off, cep[q], nb(e, +1));
          if (!wm(e)) off = vx_acc(off, cem[q], nb(e, -1));
        }
        return vx_final(at(1), c, off, at(2));   // slot 2: 1 / diagonal
      }
    };
    auto on_wall_face = [&](int i, int j, int kw) -> bool {   // fixed zero face of u_d
      if constexpr (K == 0) return !per0 && i == 0;
      else if constexpr (K == 1) return j == 0;
      else if constexpr (K == 2) return !per2 && kw == 0;
      return false;
    };
    // the point update with the flags and offsets of (i, j, kw)
    auto point = [&](auto black_tag, const float* Pm, const float* P0, const float* Pp,
                     const float* Rm, const float* R0, const float* Rp, int i, int j, int kw,
                     int o, int ro) -> float {
      const bool xin = i > 0 && i < n0 - 1;
      const bool zin = per2 || (kw > 0 && kw < n2 - 1);
      if (xin && j > 0 && j < n1 - 1 && zin)
        return update(black_tag, std::integral_constant<bool, true>{}, Pm, P0, Pp, o, 1, -1, Rm,
                      R0, Rp, ro, 1, -1, nullptr, nullptr);
      const bool wmv[3] = {!per0 && i == 0, j == 0, !per2 && kw == 0};
      const bool wpv[3] = {!per0 && i == n0 - 1, j == n1 - 1, !per2 && kw == n2 - 1};
      const int dxp = (i == n0 - 1 && per0) ? -(n0 - 1) : 1;
      const int dxm = (i == 0 && per0) ? (n0 - 1) : -1;
      const int rxp = (i == n0 - 1 && per0) ? -(n0 - 1) : 1;
      const int rxm = (i == 0 && per0) ? (n0 - 1) : -1;
      return update(black_tag, std::integral_constant<bool, false>{}, Pm, P0, Pp, o, dxp, dxm,
                    Rm, R0, Rp, ro, rxp, rxm, wmv, wpv);
    };

    // One phase per plane: the red values of plane k and the black values of
    // plane k - 2 (whose red neighbours, planes k - 3 .. k - 1, are complete)
    // are independent, so each thread runs both updates between two barriers.
    // Tile slots of the planes k - 3 .. k + 1, ring slots of k - 3 .. k and the
    // wrapped index of plane k advance by one plane per iteration.
    int sM3 = W - 2, sM2 = W - 1, sM1 = 0, s0 = 1, sP1 = 2;
    int rM3 = 2, rM2 = 3, rM1 = 0, r0 = 1;
    int kw = per2 ? wrapi(k0 - 1, n2) : k0 - 1;
    const int j_red = j0 - 1 + r_red, j_blk = j0 + r_blk;
    const bool row_red = has_red && j_red >= 0 && j_red < n1;
    const int i0_red = xs - 2 + 2 * q_red, i0_blk = xs + 2 * q_blk;
    const bool row_blk = has_blk && j_blk < n1 && i0_blk < n0;
    const size_t plane_floats = (size_t)NS * tile;
    for (int k = k0 - 1; k <= k1 + 1; ++k) {
      if (k + 1 + PD <= k1 + 1) {
        if (tid == 0) issue(k + 1 + PD);
        ++seq;
      }
      bool ok = true;
      const unsigned need = sbase + (unsigned)(min(k + 1, k1 + 1) - pbase);
      while (waited <= need) {   // `waited` stops at the first copy not seen complete
        if (!wait_seq(bar, waited, A.wait_ns)) {
          ok = false;
          break;
        }
        ++waited;
      }
      if (!ok) {
        abort_flag = 1;
        atomicExch(A.err, 1);
      }
      // red values of plane k on the rows j0 - 1 .. j0 + TY and the columns
      // xs - 1 .. xs + SW; zeros where the point does not exist
      if (has_red && k <= k1) {
        const bool planevalid = per2 || (k >= 0 && k < n2);
        float* row = ring + r0 * ringplane + r_red * RW;
        if (!(planevalid && row_red)) {
          if (i0_red >= xs - 1) row[i0_red - xs + 1] = 0.f;
          if (i0_red + 1 <= xs + SW) row[i0_red - xs + 2] = 0.f;
        } else {
          const int i = i0_red + ((j_red + kw) & 1);
          if (i >= xs - 1 && i <= xs + SW) {
            float v = 0.f;
            if (i >= 0 && i < n0 && !on_wall_face(i, j_red, kw))
              v = point(std::integral_constant<bool, false>{}, tiles + sM1 * plane_floats,
                        tiles + s0 * plane_floats, tiles + sP1 * plane_floats, nullptr, nullptr,
                        nullptr, i, j_red, kw, (r_red + 1) * BW + (i - xs + 4), 0);
            row[i - xs + 1] = v;
          }
        }
      }
      // black values of plane k - 2 on the block's rows and columns; both
      // colours out
      const int kb = k - 2;
      if (kb >= k0 && row_blk) {
        const int par = (j_blk + kb) & 1;
        const int ir = i0_blk + par, ib = i0_blk + (par ^ 1);
        float* o = A.out + st1 * j_blk + st2 * kb;
        const float* RB = ring + rM2 * ringplane;
        const int rrow = (r_blk + 1) * RW;
        if (ir < n0) o[ir] = RB[rrow + ir - xs + 1];
        if (ib < n0) {
          float v = 0.f;
          if (!on_wall_face(ib, j_blk, kb))
            v = point(std::integral_constant<bool, true>{}, tiles + sM3 * plane_floats,
                      tiles + sM2 * plane_floats, tiles + sM1 * plane_floats,
                      ring + rM3 * ringplane, RB, ring + rM1 * ringplane, ib, j_blk, kb,
                      (r_blk + 2) * BW + (ib - xs + 4), rrow + ib - xs + 1);
          o[ib] = v;
        }
      }
      __syncthreads();
      if (abort_flag) break;
      sM3 = sM2;
      sM2 = sM1;
      sM1 = s0;
      s0 = sP1;
      sP1 = (sP1 + 1 == W) ? 0 : sP1 + 1;
      rM3 = rM2;
      rM2 = rM1;
      rM1 = r0;
      r0 = (r0 + 1 == kRing) ? 0 : r0 + 1;
      kw = (per2 && kw + 1 == n2) ? 0 : kw + 1;
    }
    if (abort_flag) break;
  }
  if (abort_flag && tid == 0) {
    // drain the copies still in flight into this block's shared memory, from
    // the first one this thread has not seen complete
    while (waited < seq) {
      wait_seq(bar, waited, kWaitNs / 2);
      ++waited;
    }
  }
}

// ------------------------------------------------------------------ host
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// Tensor maps are pure host descriptors: cached by (address, geometry, rows).
using MapKey = std::tuple<const void*, long long, int, int, int, int>;
std::mutex g_map_mu;
std::map<MapKey, CUtensorMap> g_maps;

bool make_map(const Geo& g, const float* base, int TY, int BW, CUtensorMap* out) {
  MapKey key{base, g.st[1], g.s[1], g.s[2], TY, BW};
  std::lock_guard<std::mutex> lock(g_map_mu);
  auto it = g_maps.find(key);
  if (it != g_maps.end()) {
    *out = it->second;
    return true;
  }
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)g.st[1], (cuuint64_t)g.s[1], (cuuint64_t)g.s[2]};
  cuuint64_t strides[2] = {(cuuint64_t)g.st[1] * 4, (cuuint64_t)g.st[2] * 4};
  cuuint32_t box[3] = {(cuuint32_t)BW, (cuuint32_t)(TY + 4), 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUtensorMap m;
  CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return false;
  if (g_maps.size() > 65536) g_maps.clear();
  g_maps.emplace(key, m);
  *out = m;
  return true;
}

// strip geometry: SW columns per strip (a multiple of 4; a whole row when
// SW >= n0), boxes of BW = SW + 8 columns, ring rows of RW floats
int full_strip(const Geo& g) { return (g.n[0] + 3) / 4 * 4; }
int box_cols(int SW) { return SW + 8; }
int ring_cols(int SW) { return SW + 4; }

int tile_of(int TY, int SW) {   // floats, rounded to 128 bytes
  int f = (TY + 4) * box_cols(SW);
  return (f + 31) / 32 * 32;
}

size_t smem_of(int K, int TY, int PD, int SW) {
  return (size_t)total_slots(K, PD) * tile_of(TY, SW) * 4 +
         (size_t)kRing * (TY + 2) * ring_cols(SW) * 4 + kNB * 8;
}

int threads_of(int TY, int SW) {
  int red = (TY + 2) * (SW / 2 + 2), blk = TY * (SW / 2);
  int t = red > blk ? red : blk;
  return (t + 31) / 32 * 32;
}

// a plan the kernel can run: one item per thread, boxes within TMA limits,
// shared memory within the limit, strips only where x has walls
bool plan_fits(int K, const Geo& g, int TY, int PD, int SW) {
  if (TY < 1 || TY + 4 > 256 || box_cols(SW) > 256 || SW % 4) return false;
  if (SW < g.n[0] && g.per[0]) return false;
  if (threads_of(TY, SW) > kTmaThreads) return false;
  return smem_of(K, TY, PD, SW) <= kSmemMax;
}

const void* kernel_of(int K) {
  switch (K) {
    case 0: return (const void*)k_rb_tma<0>;
    case 1: return (const void*)k_rb_tma<1>;
    case 2: return (const void*)k_rb_tma<2>;
    default: return (const void*)k_rb_tma<3>;
  }
}

struct Plan {
  int TY = 4, KC = 16, PD = 1, SW = 0, grid = 0;
  bool tma = false;    // the TMA sweep timed faster than the one-pass global-memory sweep
  int rTY = 0, rKC = 0, rNP = 1;   // fastest rows / chunk planes / planes per phase of the one-pass sweep
  int rBX = 0;                     // and threads per row (0: one per point pair, up to 128)
  int rK = 0;                      // which one-pass sweep: 0 the ring sweep, 1 the pair sweep
};

using PlanKey = std::tuple<int, int, int, int, int, long long, int>;
std::mutex g_plan_mu;
std::map<PlanKey, Plan> g_plans;

PlanKey plan_key(int K, const Geo& g) {
  return PlanKey{K, g.n[0], g.n[1], g.n[2], g.per[0] + 2 * g.per[1] + 4 * g.per[2], g.st[1], 0};
}

int sm_count() {
  static int n = 0;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      n = 152;
    }
  });
  return n;
}

// Fill the launch arguments for kind K with tile height TY and chunk KC.
bool fill_args(int K, const Geo& g, const LevelPtrs<float>& L, float* out, int* err,
               double coef, int TY, int KC, int PD, int SW, TmaArgs& A) {
  if (SW >= g.n[0]) SW = full_strip(g);
  std::memset(&A, 0, sizeof(A));
  const float* src[8] = {nullptr};
  if (K == 3) {
    src[0] = L.p;
    src[1] = L.pf;
    for (int a = 0; a < 3; ++a) src[2 + a] = L.beta[a];
  } else {
    const int d = K, e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
    src[0] = L.u[d];
    src[1] = L.uf[d];
    src[2] = L.idg[d];
    src[3] = L.muc;
    src[4] = L.mue[edge_id(d, e1)];
    src[5] = L.mue[edge_id(d, e2)];
    src[6] = L.u[e1];
    src[7] = L.u[e2];
  }
  for (int a = 0; a < n_staged(K); ++a)
    if (!src[a] || !make_map(g, src[a], TY, box_cols(SW), &A.map[a])) return false;
  A.g = g;
  A.out = out;
  A.err = err;
  A.TY = TY;
  A.KC = KC;
  A.PD = PD;
  A.nrt = (g.n[1] + TY - 1) / TY;
  A.ns = (g.n[0] + SW - 1) / SW;
  A.items = A.ns * A.nrt * ((g.n[2] + KC - 1) / KC);
  A.SW = SW;
  A.BW = box_cols(SW);
  A.RW = ring_cols(SW);
  A.tile = tile_of(TY, SW);
  A.box_bytes = (unsigned)((TY + 4) * A.BW * 4);
  A.c = (float)coef;
  A.wait_ns = kWaitNs;
  return true;
}

cudaError_t launch_args(int K, const TmaArgs& A, int grid, cudaStream_t s) {
  size_t smem = smem_of(K, A.TY, A.PD, A.SW);
  dim3 blk(threads_of(A.TY, A.SW));
  switch (K) {
    case 0: k_rb_tma<0><<<grid, blk, smem, s>>>(A); break;
    case 1: k_rb_tma<1><<<grid, blk, smem, s>>>(A); break;
    case 2: k_rb_tma<2><<<grid, blk, smem, s>>>(A); break;
    default: k_rb_tma<3><<<grid, blk, smem, s>>>(A); break;
  }
  return cudaGetLastError();
}

int resident_grid(int K, int TY, int PD, int SW, int items) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_of(K), threads_of(TY, SW),
                                                    smem_of(K, TY, PD, SW)) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  if (per_sm < 1) per_sm = 1;
  int grid = sm_count() * per_sm;
  return grid < items ? grid : items;
}

}  // namespace

bool tma_eligible(int D, const Geo& g) {
  if (D != 3 || g.per[1]) return false;
  if (g.n[0] < 8 || g.n[1] < 2 || g.n[2] < 2) return false;
  if ((long long)g.n[0] * g.n[1] * g.n[2] < 32768) return false;
  const int SW = g.per[0] ? full_strip(g) : (g.n[0] > 64 ? 64 : full_strip(g));
  for (int K = 0; K < 4; ++K)
    if (!plan_fits(K, g, 2, 1, SW)) return false;
  return encode_fn() != nullptr;
}

cudaError_t tma_set_smem() {
  cudaError_t e = cudaSuccess;
  for (int K = 0; K < 4 && e == cudaSuccess; ++K)
    e = cudaFuncSetAttribute(kernel_of(K), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemMax);
  return e;
}

// Time the one-pass global-memory sweep and the TMA sweep's candidate tile
// heights, prefetch distances, chunk lengths and grids on the level's own
// arrays (both sweeps are out of place, so only `out` is written) and keep
// the fastest per level shape and kind. Call outside stream capture.
cudaError_t tma_autotune(int D, const Geo& g, const LevelPtrs<float>& L, int K, float* out,
                         int* err, double coef, cudaStream_t s) {
  if (!tma_eligible(D, g)) return cudaSuccess;
  PlanKey key = plan_key(K, g);
  {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    if (g_plans.count(key)) return cudaSuccess;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cudaGetLastError();
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cudaGetLastError();
  }
  Plan best;
  float best_ms = 1e30f;
  cudaError_t status = cudaSuccess;
  // per-launch time of a candidate: the better of two rounds of four launches
  auto per_launch_ms = [&](auto&& launch) -> float {
    float t = 1e30f;
    for (int round = 0; round < 2 && status == cudaSuccess; ++round) {
      cudaEventRecord(e0, s);
      for (int r = 0; r < 4; ++r) launch();
      cudaEventRecord(e1, s);
      status = cudaEventSynchronize(e1);
      if (status != cudaSuccess) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms / 4 < t) t = ms / 4;
    }
    return t;
  };
  // the one-pass sweep that reads global memory: tile rows and chunk planes
  const int npairs = (g.n[0] + 1) / 2;
  const int bx = npairs >= 128 ? 128 : (npairs + 31) / 32 * 32;
  // shapes are searched on levels of at least 2^16 cells (the 32 x 32 x 64
  // level and up, where a sweep lasts 5-15 us and the pair sweep beats the
  // built-in ring shape); on smaller ones a launch lasts a few microseconds and
  // the timing cannot tell the candidates apart
  const bool search = (long long)g.n[0] * g.n[1] * g.n[2] >= (1 << 16);
  // bring the clocks up before the first candidate is timed
  for (int r = 0; r < 10; ++r) {
    if (K == 3) launch_p_rb_fused<float>(D, g, L, out, s);
    else launch_v_rb_fused<float>(D, g, L, K, out, coef * g.h * g.h, s);
  }
  // (rows, threads per row): one thread per point pair on up to 8 rows, or
  // 32 threads per row (several pairs each) on taller tiles, where the ring
  // rows recomputed by neighbouring blocks are a smaller share
  const int shapes[8][2] = {{0, 0}, {2, 0}, {4, 0}, {6, 0}, {8, 0}, {8, 32}, {12, 32}, {16, 32}};
  for (int rNP : {1, 2}) {
  for (const auto& shp : shapes) {
    const int rTY = shp[0], rBX = shp[1];
    if ((rTY == 0) == search) continue;
    if (rBX > 0 && rBX >= bx) continue;
    if (rTY > g.n[1] || (rBX > 0 ? rBX : bx) * (rTY + 2) > 1024) continue;
    // fixed chunk sizes, and the sizes that fill one or two waves of resident
    // blocks exactly
    int kcs_ring[5] = {8, 16, 32, 0, 0};
    if (search && rTY > 0) {
      kcs_ring[3] = ring_fill_kc(D, K, g, rTY, rNP, rBX, 1);
      kcs_ring[4] = ring_fill_kc(D, K, g, rTY, rNP, rBX, 2);
    }
    for (int ci = 0; ci < 5; ++ci) {
      const int rKC = kcs_ring[ci];
      if (rKC <= 0) continue;
      bool seen = false;
      for (int cj = 0; cj < ci; ++cj) seen = seen || kcs_ring[cj] == rKC;
      if (seen) continue;
      if (!search && rKC != 8) continue;
      if (search && rKC > g.n[2] && rKC != 8) continue;
      auto ring = [&]() {
        if (K == 3) launch_p_rb_fused<float>(D, g, L, out, s, rTY, rKC, rNP, rBX);
        else launch_v_rb_fused<float>(D, g, L, K, out, coef * g.h * g.h, s, rTY, rKC, rNP, rBX);
      };
      ring();
      float ms = per_launch_ms(ring);
      if (status != cudaSuccess) break;
      if (ms < best_ms) {
        best_ms = ms;
        best.rTY = rTY;
        best.rKC = search ? rKC : 0;
        best.rNP = rNP;
        best.rBX = rBX;
        best.rK = 0;
      }
    }
    if (status != cudaSuccess) break;
  }
  if (status != cudaSuccess) break;
  }
  // the pair sweep (viscous components and pressure): tile rows and chunk planes
  if (search && status == cudaSuccess) {
    for (int pTY : {2, 4, 6, 8, 10, 14}) {
      if (!pair_eligible(D, g, pTY)) continue;
      int kcs_pair[5] = {8, 16, 32, pair_fill_kc(g, K, pTY, 1), pair_fill_kc(g, K, pTY, 2)};
      for (int ci = 0; ci < 5; ++ci) {
        const int pKC = kcs_pair[ci];
        if (pKC <= 0 || pKC > g.n[2]) continue;
        bool seen = false;
        for (int cj = 0; cj < ci; ++cj) seen = seen || kcs_pair[cj] == pKC;
        if (seen) continue;
        auto pr = [&]() {
          if (K == 3) launch_p_rb_pair(g, L, out, s, pTY, pKC);
          else launch_v_rb_pair(g, L, K, out, coef * g.h * g.h, s, pTY, pKC);
        };
        pr();
        float ms = per_launch_ms(pr);
        if (status != cudaSuccess) break;
        if (ms < best_ms) {
          best_ms = ms;
          best.rTY = pTY;
          best.rKC = pKC;
          best.rNP = 1;
          best.rBX = 0;
          best.rK = 1;
        }
      }
      if (status != cudaSuccess) break;
    }
  }
  const int tys[] = {2, 4, 6, 8};
  const int kcs[] = {16, 32, 64};
  const int sws[] = {64, full_strip(g)};
  for (int SW : sws) {
  if (SW == 64 && g.n[0] <= 64) continue;
  for (int TY : tys) {
    if (TY > g.n[1]) continue;
    for (int PD = 1; PD <= kMaxPD; ++PD) {
    if (!plan_fits(K, g, TY, PD, SW)) continue;
    for (int KC : kcs) {
      if (KC > g.n[2] && KC != kcs[0]) continue;
      TmaArgs A;
      if (!fill_args(K, g, L, out, err, coef, TY, KC, PD, SW, A)) continue;
      int grid = resident_grid(K, TY, PD, A.SW, A.items);
      status = launch_args(K, A, grid, s);
      if (status != cudaSuccess) break;
      float ms = per_launch_ms([&]() { launch_args(K, A, grid, s); });
      if (status != cudaSuccess) break;
      if (ms < best_ms) {
        best_ms = ms;
        best.tma = true;
        best.TY = TY;
        best.KC = KC;
        best.PD = PD;
        best.SW = A.SW;
        best.grid = grid;
      }
    }
    if (status != cudaSuccess) break;
    }
    if (status != cudaSuccess) break;
  }
  if (status != cudaSuccess) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != cudaSuccess) return status;
  {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    g_plans[key] = best;
  }
  return cudaSuccess;
}

// One sweep: out = the red-black update of the old iterate in L (kind 3:
// pressure, else viscous component K). Uses the tuned plan of the level shape,
// or a default one before tuning.
cudaError_t launch_rb_tma(int D, const Geo& g, const LevelPtrs<float>& L, int K, float* out,
                          int* err, double coef, cudaStream_t s, unsigned long long wait_ns) {
  Plan pl;
  {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    auto it = g_plans.find(plan_key(K, g));
    if (it != g_plans.end()) pl = it->second;
  }
  if (pl.SW <= 0) pl.SW = (g.per[0] || g.n[0] <= 64) ? full_strip(g) : 64;
  if (pl.TY > g.n[1]) pl.TY = g.n[1];
  while (pl.TY > 2 && !plan_fits(K, g, pl.TY, pl.PD, pl.SW)) --pl.TY;
  TmaArgs A;
  if (!fill_args(K, g, L, out, err, coef, pl.TY, pl.KC, pl.PD, pl.SW, A))
    return cudaErrorInvalidValue;
  A.wait_ns = wait_ns;
  int grid = pl.grid > 0 ? pl.grid : resident_grid(K, pl.TY, pl.PD, A.SW, A.items);
  return launch_args(K, A, grid, s);
}

bool tma_set_plan(int K, const Geo& g, const int in[5]) {
  Plan pl;
  pl.tma = true;
  pl.TY = in[0];
  pl.KC = in[1];
  pl.PD = in[2];
  pl.SW = in[3] >= g.n[0] ? full_strip(g) : in[3];
  pl.grid = in[4];
  if (pl.KC < 1 || pl.PD < 1 || pl.PD > kMaxPD || pl.grid < 0 || !plan_fits(K, g, pl.TY, pl.PD, pl.SW))
    return false;
  std::lock_guard<std::mutex> lock(g_plan_mu);
  auto it = g_plans.find(plan_key(K, g));
  if (it != g_plans.end()) {
    pl.rTY = it->second.rTY;
    pl.rKC = it->second.rKC;
    pl.rNP = it->second.rNP;
    pl.rBX = it->second.rBX;
    pl.rK = it->second.rK;
  }
  g_plans[plan_key(K, g)] = pl;
  return true;
}

// Pin the one-pass sweep (not the TMA one) with shape {TY, KC, NP, BX, kernel}
// for the level shape of g, process-wide (kernel 1, the pair sweep, takes
// TY > 0, KC > 0, NP 1 and BX 0).
bool ring_set_shape(int K, const Geo& g, const int in[5]) {
  if (in[0] < 0 || in[1] < 0 || (in[2] != 1 && in[2] != 2) || in[3] < 0 || in[3] > 128 ||
      in[3] % 32 != 0 || (in[4] != 0 && in[4] != 1))
    return false;
  if (in[4] == 1 && (in[0] < 1 || in[1] < 1 || in[2] != 1 || in[3] != 0 ||
                     !pair_eligible(3, g, in[0])))
    return false;
  std::lock_guard<std::mutex> lock(g_plan_mu);
  Plan pl;
  auto it = g_plans.find(plan_key(K, g));
  if (it != g_plans.end()) pl = it->second;
  pl.tma = false;
  pl.rTY = in[0];
  pl.rKC = in[1];
  pl.rNP = in[2];
  pl.rBX = in[3];
  pl.rK = in[4];
  g_plans[plan_key(K, g)] = pl;
  return true;
}

bool ring_shape_of(int K, const Geo& g, int* TY, int* KC, int* NP, int* BX, int* KERN) {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  auto it = g_plans.find(plan_key(K, g));
  if (it == g_plans.end()) return false;
  *TY = it->second.rTY;
  *KC = it->second.rKC;
  *NP = it->second.rNP;
  *BX = it->second.rBX;
  if (KERN) *KERN = it->second.rK;
  return true;
}

bool tma_chosen(int K, const Geo& g) {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  auto it = g_plans.find(plan_key(K, g));
  return it != g_plans.end() && it->second.tma;
}

bool tma_plan_of(int K, const Geo& g, int out[5]) {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  auto it = g_plans.find(plan_key(K, g));
  if (it == g_plans.end() || !it->second.tma) return false;
  out[0] = it->second.TY;
  out[1] = it->second.KC;
  out[2] = it->second.PD;
  out[3] = it->second.SW;
  out[4] = it->second.grid;
  return true;
}

}  // namespace bf
