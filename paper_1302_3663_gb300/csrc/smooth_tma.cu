// Red-black Gauss-Seidel sweeps (Sec. 3.5) with their inputs staged in
// shared memory by the Tensor Memory Accelerator: the 3D FP32 smoother of the
// mixed-precision V-cycles.
//
// The arithmetic of every point update is that of the two-kernel sweep in
// stencil.cu and of the ring-fused sweep in smooth.cu; only the data movement
// differs. A block owns TY full x rows of the y axis and walks a chunk of
// planes along z. For every plane one elected thread issues one tiled TMA copy
// per input array (a box of TY + 4 rows of one plane: two halo rows on each
// side) into a window of plane slots, two planes ahead of the computation;
// completion is tracked by transaction-count mbarriers. Red values of a plane
// (on the block's rows plus one ring row each side) depend only on old black
// values and go to a three-plane ring; the black values of the plane before
// then read their red neighbours from the ring. The sweep is out of place.
//
// Blocks are persistent: block b takes the work items (row tile, plane chunk)
// b, b + G, b + 2G, ..., so the items in flight at any moment are neighbours
// and share their halo rows through L2. Tile height, chunk length and grid
// size come from a timing autotuner run once per level shape.
//
// Every wait on an mbarrier is bounded (2 s of the global timer); a block
// whose wait runs out raises the error word, drains its own copies in flight
// (again bounded) and returns.
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
constexpr int kTmaThreads = 512;        // threads per block at most
constexpr unsigned long long kWaitNs = 2000000000ull;
constexpr size_t kSmemMax = 225 * 1024;   // dynamic, leaving room for the static words

// Staged arrays. Viscous component d (kinds 0, 1, 2): old u_d, rhs_d, m_d,
// mu_c, the two edge viscosities of d and the two other components (axes e1 <
// e2). Pressure (kind 3): old p, rhs, beta_x, beta_y, beta_z.
__host__ __device__ constexpr int n_staged(int K) { return K == 3 ? 5 : 8; }

// Plane slots: the planes a block still reads (k-1 .. k+1 around the red
// plane k; k-2 as well for the z component, whose stencil reaches one plane
// below the point) plus the PD planes in flight.
__host__ __device__ constexpr int win(int K, int PD) { return (K == 2 ? 4 : 3) + PD; }
__host__ __device__ constexpr int total_slots(int K, int PD) { return win(K, PD) * n_staged(K); }

struct TmaArgs {
  CUtensorMap map[8];
  Geo g;
  float* out;
  int* err;
  int TY, KC, nrt, items, pitch;
  int PD;                // planes issued ahead of the red plane's last need
  int tile;              // floats between array tiles (multiple of 32)
  unsigned box_bytes;    // bytes of one box: (TY + 4) rows of pitch floats
  float c;               // viscous: inv_re / h^2; pressure: h^2
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
// phase parity (s / kNB) & 1)
__device__ __forceinline__ bool wait_seq(unsigned long long* bar, unsigned s,
                                         unsigned long long limit_ns) {
  unsigned long long* b = &bar[s % kNB];
  unsigned par = (s / kNB) & 1u;
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
// (tile = TY + 4 rows of pitch floats); then the three-plane ring; then the
// mbarriers. Plane p of a chunk lives in slot (p - pbase) % W.
template <int K>
__global__ void __launch_bounds__(kTmaThreads) k_rb_tma(const __grid_constant__ TmaArgs A) {
  constexpr int NS = n_staged(K);
  const int PD = A.PD, W = win(K, PD);
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ int abort_flag;
  const Geo& g = A.g;
  const int TY = A.TY, pitch = A.pitch, tile = A.tile;
  const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
  const bool per0 = g.per[0] != 0, per2 = g.per[2] != 0;
  const long long st1 = g.st[1], st2 = g.st[2];
  float* tiles = reinterpret_cast<float*>(sm);
  float* ring = tiles + (size_t)W * NS * tile;
  const int ringplane = (TY + 2) * pitch;
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(ring + 3 * ringplane);
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int q = tid; q < 3 * ringplane; q += nthr) ring[q] = 0.f;
  if (tid == 0) {
    abort_flag = 0;
    for (int b = 0; b < kNB; ++b) mbar_init(&bar[b], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int npairs = (n0 + 1) / 2;
  const float c = A.c;
  unsigned seq = 0, waited = 0;   // planes issued / waited for by this block

  for (int item = blockIdx.x; item < A.items; item += gridDim.x) {
    const int t = item % A.nrt, ch = item / A.nrt;
    const int j0 = t * TY, k0 = ch * A.KC, k1 = min(k0 + A.KC, n2);
    const int pbase = k0 - 2;   // plane in slot 0 at the start of the chunk
    const unsigned sbase = seq;
    auto plane_tiles = [&](int p) -> float* { return tiles + (size_t)((p - pbase) % W) * NS * tile; };
    auto ring_plane = [&](int p) -> float* { return ring + ((p - pbase) % 3) * ringplane; };
    if (tid == 0) {
      for (int p = pbase; p <= min(pbase + 1 + PD, k1 + 1); ++p) {
        unsigned long long* b = &bar[(sbase + (unsigned)(p - pbase)) % kNB];
        mbar_expect_tx(b, (unsigned)NS * A.box_bytes);
        int z = per2 ? wrapi(p, n2) : p;
        float* dst = plane_tiles(p);
#pragma unroll
        for (int a = 0; a < NS; ++a) tma_load_3d(dst + a * tile, &A.map[a], b, 0, j0 - 2, z);
      }
    }
    seq += (unsigned)(min(pbase + 1 + PD, k1 + 1) - pbase + 1);

    // One point update of the plane whose tiles are P0 (neighbours Pm, Pp)
    // at tile offset o; x neighbours at o + dxp / o + dxm. BLACK takes the
    // u_d (or p) neighbours from the ring (planes Rm, R0, Rp at ring offset
    // ro, x neighbours at ro + rxp / ro + rxm), red from the staged old
    // values. Same operation order as the two-kernel sweep.
    auto update = [&](auto black_tag, const float* Pm, const float* P0, const float* Pp, int o,
                      int dxp, int dxm, const float* Rm, const float* R0, const float* Rp,
                      int ro, int rxp, int rxm, const bool* wm, const bool* wp) -> float {
      constexpr bool BLACK = decltype(black_tag)::value;
      // neighbour of the iterate (array 0) along axis ax, side +-1
      auto nb = [&](int ax, int side) -> float {
        if constexpr (BLACK) {
          if (ax == 0) return R0[ro + (side > 0 ? rxp : rxm)];
          if (ax == 1) return R0[ro + side * pitch];
          return (side > 0 ? Rp : Rm)[ro];
        } else {
          if (ax == 0) return P0[o + (side > 0 ? dxp : dxm)];
          if (ax == 1) return P0[o + side * pitch];
          return (side > 0 ? Pp : Pm)[o];
        }
      };
      // staged array a at the point shifted by s1 along ax1 and s2 along ax2
      auto sh = [&](int a, int ax1, int s1, int ax2, int s2) -> float {
        const float* P = P0;
        int off = o + a * tile;
        if (s1 != 0) {
          if (ax1 == 0) off += s1 > 0 ? dxp : dxm;
          else if (ax1 == 1) off += s1 * pitch;
          else P = s1 > 0 ? Pp : Pm;
        }
        if (s2 != 0) {
          if (ax2 == 0) off += s2 > 0 ? dxp : dxm;
          else if (ax2 == 1) off += s2 * pitch;
          else P = s2 > 0 ? Pp : Pm;
        }
        return P[off];
      };
      auto at = [&](int a) -> float { return P0[o + a * tile]; };
      if constexpr (K == 3) {
        float num = 0.f, dg = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (!wm[a]) {
            float bb = at(2 + a);
            num += bb * nb(a, -1);
            dg += bb;
          }
          if (!wp[a]) {
            float bb = sh(2 + a, a, +1, 0, 0);
            num += bb * nb(a, +1);
            dg += bb;
          }
        }
        return (num - c * at(1)) / dg;
      } else {
        constexpr int d = K;
        constexpr int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;
        float mcp = at(3), mcm = sh(3, d, -1, 0, 0);
        float cdp = 2.f * mcp, cdm = 2.f * mcm;
        float dgV = 2.f * (mcp + mcm);
        float cross = 0.f;
        float cep[2], cem[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int e = q == 0 ? e1 : e2;
          const int me = 4 + q, ue = 6 + q;
          float mep = sh(me, e, +1, 0, 0), mem = at(me);
          cross += mep * (sh(ue, e, +1, 0, 0) - sh(ue, e, +1, d, -1)) -
                   mem * (at(ue) - sh(ue, d, -1, 0, 0));
          cep[q] = mep;
          cem[q] = mem;
          dgV += (wp[e] ? 2.f : 1.f) * mep + (wm[e] ? 2.f : 1.f) * mem;
        }
        float diag = at(2) + c * dgV;
        float off = cross + cdp * nb(d, +1) + cdm * nb(d, -1);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int e = q == 0 ? e1 : e2;
          if (!wp[e]) off += cep[q] * nb(e, +1);
          if (!wm[e]) off += cem[q] * nb(e, -1);
        }
        return (at(1) + c * off) / diag;
      }
    };
    auto on_wall_face = [&](int i, int j, int kw) -> bool {   // fixed zero face of u_d
      if constexpr (K == 0) return !per0 && i == 0;
      else if constexpr (K == 1) return j == 0;
      else if constexpr (K == 2) return !per2 && kw == 0;
      return false;
    };
    // tile offsets of the x neighbours (periodic wrap; beyond a wall: the
    // stored wall face or an unused slot)
    auto xdeltas = [&](int i, int& dxp, int& dxm) {
      dxp = (i == n0 - 1 && per0) ? -(n0 - 1) : 1;
      dxm = (i == 0 && per0) ? (n0 - 1) : -1;
    };
    auto rdeltas = [&](int i, int& rxp, int& rxm) {   // as the ring-fused sweep wraps
      rxp = (i == n0 - 1 && per0) ? -(n0 - 1) : 1;
      rxm = (i == 0) ? (n0 - 1) : -1;
    };

    for (int k = k0 - 1; k <= k1; ++k) {
      if (k + 1 + PD <= k1 + 1) {
        if (tid == 0) {
          const int p = k + 1 + PD;
          unsigned long long* b = &bar[(sbase + (unsigned)(p - pbase)) % kNB];
          fence_proxy_async();
          mbar_expect_tx(b, (unsigned)NS * A.box_bytes);
          int z = per2 ? wrapi(p, n2) : p;
          float* dst = plane_tiles(p);
#pragma unroll
          for (int a = 0; a < NS; ++a) tma_load_3d(dst + a * tile, &A.map[a], b, 0, j0 - 2, z);
        }
        ++seq;
      }
      bool ok = true;
      const unsigned need = sbase + (unsigned)(k + 1 - pbase);   // plane k + 1
      while (waited <= need) {
        ok = ok && wait_seq(bar, waited, kWaitNs);
        ++waited;
      }
      if (!ok) {
        abort_flag = 1;
        atomicExch(A.err, 1);
      }
      // red values of plane k on the rows j0 - 1 .. j0 + TY
      {
        const bool planevalid = per2 || (k >= 0 && k < n2);
        const int kw = per2 ? wrapi(k, n2) : k;
        const float* Pm = plane_tiles(k - 1);
        const float* P0 = plane_tiles(k);
        const float* Pp = plane_tiles(k + 1);
        float* R0 = ring_plane(k);
        for (int q = tid; q < (TY + 2) * npairs; q += nthr) {
          const int r = q / npairs, ip = q - r * npairs;
          const int j = j0 - 1 + r;
          float* row = R0 + r * pitch;
          if (!(planevalid && j >= 0 && j < n1)) {
            row[2 * ip] = 0.f;
            if (2 * ip + 1 < n0) row[2 * ip + 1] = 0.f;
            continue;
          }
          const int i = 2 * ip + ((j + kw) & 1);
          if (i >= n0) continue;
          float v = 0.f;
          if (!on_wall_face(i, j, kw)) {
            const bool wm[3] = {!per0 && i == 0, j == 0, !per2 && kw == 0};
            const bool wp[3] = {!per0 && i == n0 - 1, j == n1 - 1, !per2 && kw == n2 - 1};
            int dxp, dxm;
            xdeltas(i, dxp, dxm);
            v = update(std::integral_constant<bool, false>{}, Pm, P0, Pp, (r + 1) * pitch + i,
                       dxp, dxm, nullptr, nullptr, nullptr, 0, 0, 0, wm, wp);
          }
          row[i] = v;
        }
      }
      __syncthreads();
      if (abort_flag) break;
      // black values of plane k - 1 on the block's own rows; both colours out
      const int kb = k - 1;
      if (kb >= k0) {
        const float* Pm = plane_tiles(kb - 1);
        const float* P0 = plane_tiles(kb);
        const float* Pp = plane_tiles(kb + 1);
        const float* Rm = ring_plane(kb - 1);
        const float* R0 = ring_plane(kb);
        const float* Rp = ring_plane(kb + 1);
        for (int q = tid; q < TY * npairs; q += nthr) {
          const int r = q / npairs, ip = q - r * npairs;
          const int j = j0 + r;
          if (j >= n1) continue;
          const int par = (j + kb) & 1;
          const int ir = 2 * ip + par, ib = 2 * ip + (par ^ 1);
          float* o = A.out + st1 * j + st2 * kb;
          const int rrow = (r + 1) * pitch;
          if (ir < n0) o[ir] = R0[rrow + ir];
          if (ib < n0) {
            float v = 0.f;
            if (!on_wall_face(ib, j, kb)) {
              const bool wm[3] = {!per0 && ib == 0, j == 0, !per2 && kb == 0};
              const bool wp[3] = {!per0 && ib == n0 - 1, j == n1 - 1, !per2 && kb == n2 - 1};
              int dxp, dxm, rxp, rxm;
              xdeltas(ib, dxp, dxm);
              rdeltas(ib, rxp, rxm);
              v = update(std::integral_constant<bool, true>{}, Pm, P0, Pp, (r + 2) * pitch + ib,
                         dxp, dxm, Rm, R0, Rp, rrow + ib, rxp, rxm, wm, wp);
            }
            o[ib] = v;
          }
        }
      }
      __syncthreads();
    }
    if (abort_flag) break;
  }
  if (abort_flag && tid == 0) {
    // drain the copies still in flight into this block's shared memory
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
using MapKey = std::tuple<const void*, long long, int, int, int>;
std::mutex g_map_mu;
std::map<MapKey, CUtensorMap> g_maps;

bool make_map(const Geo& g, const float* base, int TY, CUtensorMap* out) {
  MapKey key{base, g.st[1], g.s[1], g.s[2], TY};
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
  cuuint32_t box[3] = {(cuuint32_t)g.st[1], (cuuint32_t)(TY + 4), 1};
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

int tile_of(const Geo& g, int TY) {   // floats, rounded to 128 bytes
  int f = (int)((TY + 4) * g.st[1]);
  return (f + 31) / 32 * 32;
}

size_t smem_of(int K, const Geo& g, int TY, int PD) {
  return (size_t)total_slots(K, PD) * tile_of(g, TY) * 4 + (size_t)3 * (TY + 2) * g.st[1] * 4 +
         kNB * 8;
}

int threads_of(const Geo& g, int TY) {
  int npairs = (g.n[0] + 1) / 2;
  int t = (TY + 2) * npairs;
  if (t > kTmaThreads) t = kTmaThreads;
  return (t + 31) / 32 * 32;
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
  int TY = 4, KC = 16, PD = 1, grid = 0;
  bool tma = false;    // the TMA sweep timed faster than the one-pass global-memory sweep
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
               double coef, int TY, int KC, int PD, TmaArgs& A) {
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
    src[2] = L.m[d];
    src[3] = L.muc;
    src[4] = L.mue[edge_id(d, e1)];
    src[5] = L.mue[edge_id(d, e2)];
    src[6] = L.u[e1];
    src[7] = L.u[e2];
  }
  for (int a = 0; a < n_staged(K); ++a)
    if (!src[a] || !make_map(g, src[a], TY, &A.map[a])) return false;
  A.g = g;
  A.out = out;
  A.err = err;
  A.TY = TY;
  A.KC = KC;
  A.PD = PD;
  A.nrt = (g.n[1] + TY - 1) / TY;
  A.items = A.nrt * ((g.n[2] + KC - 1) / KC);
  A.pitch = (int)g.st[1];
  A.tile = tile_of(g, TY);
  A.box_bytes = (unsigned)((TY + 4) * g.st[1] * 4);
  A.c = (float)coef;
  return true;
}

cudaError_t launch_args(int K, const Geo& g, const TmaArgs& A, int grid, cudaStream_t s) {
  size_t smem = smem_of(K, g, A.TY, A.PD);
  dim3 blk(threads_of(g, A.TY));
  switch (K) {
    case 0: k_rb_tma<0><<<grid, blk, smem, s>>>(A); break;
    case 1: k_rb_tma<1><<<grid, blk, smem, s>>>(A); break;
    case 2: k_rb_tma<2><<<grid, blk, smem, s>>>(A); break;
    default: k_rb_tma<3><<<grid, blk, smem, s>>>(A); break;
  }
  return cudaGetLastError();
}

int resident_grid(int K, const Geo& g, int TY, int PD, int items) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel_of(K), threads_of(g, TY),
                                                    smem_of(K, g, TY, PD)) != cudaSuccess) {
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
  if (g.st[1] > 256 || g.n[0] < 8 || g.n[1] < 2 || g.n[2] < 2) return false;
  if ((long long)g.n[0] * g.n[1] * g.n[2] < 32768) return false;
  for (int K = 0; K < 4; ++K)
    if (smem_of(K, g, 2, 1) > kSmemMax) return false;
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
  // the one-pass sweep that reads global memory is the first candidate
  {
    auto ring = [&]() {
      if (K == 3) launch_p_rb_fused<float>(D, g, L, out, s);
      else launch_v_rb_fused<float>(D, g, L, K, out, coef * g.h * g.h, s);
    };
    ring();
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3; ++r) ring();
    cudaEventRecord(e1, s);
    status = cudaEventSynchronize(e1);
    if (status == cudaSuccess) cudaEventElapsedTime(&best_ms, e0, e1);
  }
  const int tys[] = {2, 4, 6, 8};
  const int kcs[] = {16, 32, 64};
  for (int TY : tys) {
    if (TY > g.n[1]) continue;
    for (int PD = 1; PD <= kMaxPD; ++PD) {
    if (smem_of(K, g, TY, PD) > kSmemMax) continue;
    for (int KC : kcs) {
      if (KC > g.n[2] && KC != kcs[0]) continue;
      TmaArgs A;
      if (!fill_args(K, g, L, out, err, coef, TY, KC, PD, A)) continue;
      int grid = resident_grid(K, g, TY, PD, A.items);
      status = launch_args(K, g, A, grid, s);
      if (status != cudaSuccess) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < 3; ++r) launch_args(K, g, A, grid, s);
      cudaEventRecord(e1, s);
      status = cudaEventSynchronize(e1);
      if (status != cudaSuccess) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best.tma = true;
        best.TY = TY;
        best.KC = KC;
        best.PD = PD;
        best.grid = grid;
      }
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
                          int* err, double coef, cudaStream_t s) {
  Plan pl;
  {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    auto it = g_plans.find(plan_key(K, g));
    if (it != g_plans.end()) pl = it->second;
  }
  if (pl.TY > g.n[1]) pl.TY = g.n[1];
  while (pl.TY > 2 && smem_of(K, g, pl.TY, pl.PD) > kSmemMax) --pl.TY;
  TmaArgs A;
  if (!fill_args(K, g, L, out, err, coef, pl.TY, pl.KC, pl.PD, A)) return cudaErrorInvalidValue;
  int grid = pl.grid > 0 ? pl.grid : resident_grid(K, g, pl.TY, pl.PD, A.items);
  return launch_args(K, g, A, grid, s);
}

bool tma_chosen(int K, const Geo& g) {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  auto it = g_plans.find(plan_key(K, g));
  return it != g_plans.end() && it->second.tma;
}

bool tma_plan_of(int K, const Geo& g, int out[4]) {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  auto it = g_plans.find(plan_key(K, g));
  if (it == g_plans.end() || !it->second.tma) return false;
  out[0] = it->second.TY;
  out[1] = it->second.KC;
  out[2] = it->second.PD;
  out[3] = it->second.grid;
  return true;
}

}  // namespace bf
