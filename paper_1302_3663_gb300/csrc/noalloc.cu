// bfibm_divergence_noalloc: the divergence stage without any device
// allocation.
//
// Some callers cannot let a library call cudaMalloc: applications whose
// device memory is owned by another allocator (a framework's caching pool
// that has already reserved the device), services with a fixed memory budget
// that must not fail with an out-of-memory error after start-up, and
// latency-critical loops that cannot afford cudaMalloc/cudaFree, which may
// synchronise the whole device. This entry point takes the caller's input and
// output buffers and keeps its only scratch (one partial sum per block of the
// mean reduction) in a fixed file-scope device array that every GPU loading
// the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/bfibm.h"
#include "common.cuh"

namespace {

constexpr int kNaBlock = 256;               // cells per block, one partial each
constexpr int kNaMaxBlocks = 65536;         // scratch: 65536 partials + 1 total
constexpr long long kNaMaxCells = (long long)kNaBlock * kNaMaxBlocks;   // 2^24 cells
constexpr int kNaMaxDevices = 64;

// 512 KB + 8 B per device: partial sums of the blocks, then the mean
static __device__ __align__(256) double g_noalloc_scratch[kNaMaxBlocks + 1];

std::mutex g_na_mutex;
double* g_na_ptr[kNaMaxDevices] = {nullptr};

// the device address of the scratch array on the current device, looked up
// once per device
cudaError_t scratch_on_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_ptr[dev] = p;
  }
  *out = g_na_ptr[dev];
  return cudaSuccess;
}

struct DenseGeo {
  int n[3], s[3], per[3];
  long long sy, sz;   // dense strides
  double h;
};

__device__ __forceinline__ long long dnext(const DenseGeo& g, int a, int ci) {
  long long st = a == 0 ? 1 : (a == 1 ? g.sy : g.sz);
  return (g.per[a] && ci == g.n[a] - 1) ? -(long long)(g.n[a] - 1) * st : st;
}

struct U3 {
  const double* a[3];
};

// b = scale * D.u at every cell; one partial sum of b per block
template <int D>
__global__ void __launch_bounds__(kNaBlock) k_div_na(DenseGeo g, U3 u, double* __restrict__ b,
                                                     double scale, double* __restrict__ partial) {
  __shared__ double sh[kNaBlock / 32];
  long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  long long q = blockIdx.x * (long long)kNaBlock + threadIdx.x;
  double v = 0.0;
  if (q < ncell) {
    int i = (int)(q % g.n[0]);
    long long r = q / g.n[0];
    int j = (int)(r % g.n[1]);
    int k = (int)(r / g.n[1]);
    int ci[3] = {i, j, k};
    long long c = i + g.sy * j + g.sz * k;
    double s = 0.0;
#pragma unroll
    for (int a = 0; a < D; ++a) s += (u.a[a][c + dnext(g, a, ci[a])] - u.a[a][c]) / g.h;
    v = scale * s;
    b[c] = v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < kNaBlock / 32 ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
  }
}

// partial[nb] = mean of b, summed in a fixed order by one block
__global__ void __launch_bounds__(1024) k_mean_na(double* partial, int nb, long long ncell) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int q = threadIdx.x; q < nb; q += blockDim.x) v += partial[q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = sh[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) partial[nb] = v / (double)ncell;
  }
}

__global__ void __launch_bounds__(kNaBlock) k_sub_na(DenseGeo g, double* __restrict__ b,
                                                     const double* __restrict__ mean) {
  long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  long long q = blockIdx.x * (long long)kNaBlock + threadIdx.x;
  if (q >= ncell) return;
  int i = (int)(q % g.n[0]);
  long long r = q / g.n[0];
  int j = (int)(r % g.n[1]);
  int k = (int)(r / g.n[1]);
  b[i + g.sy * j + g.sz * k] -= *mean;
}

}  // namespace

extern "C" bfibm_status bfibm_divergence_noalloc(const bfibm_params* p, const double* u0,
                                                 const double* u1, const double* u2, double* b,
                                                 void* stream) {
  if (!p || (p->dim != 2 && p->dim != 3) || !u0 || !u1 || (p->dim == 3 && !u2) || !b)
    return BFIBM_EINVAL;
  if (!(p->h > 0.0) || !(p->dt > 0.0) || !(p->sigma > 0.0) || !(p->euler > 0.0))
    return BFIBM_EINVAL;
  if (p->open_flow) return BFIBM_EINVAL;   // the open duct's divergence keeps its mean
  int D = p->dim;
  DenseGeo g;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = (a < D) ? p->n[a] : 1;
    g.per[a] = (a < D) ? (p->periodic[a] != 0) : 1;
    if (g.n[a] < 1 || (a < D && g.n[a] < 2)) return BFIBM_EINVAL;
    g.s[a] = (a < D && !g.per[a]) ? g.n[a] + 1 : g.n[a];
  }
  g.sy = g.s[0];
  g.sz = (long long)g.s[0] * g.s[1];
  g.h = p->h;
  long long ncell = (long long)g.n[0] * g.n[1] * g.n[2];
  if (ncell > kNaMaxCells) return BFIBM_EINVAL;   // larger than the fixed scratch
  double* scratch = nullptr;
  if (scratch_on_current_device(&scratch) != cudaSuccess) {
    cudaGetLastError();
    return BFIBM_ECUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int nb = (int)((ncell + kNaBlock - 1) / kNaBlock);
  U3 u{{u0, u1, D == 3 ? u2 : u1}};
  double scale = p->sigma / p->euler / p->dt;
  if (D == 3) k_div_na<3><<<nb, kNaBlock, 0, s>>>(g, u, b, scale, scratch);
  else k_div_na<2><<<nb, kNaBlock, 0, s>>>(g, u, b, scale, scratch);
  k_mean_na<<<1, 1024, 0, s>>>(scratch, nb, ncell);
  k_sub_na<<<nb, kNaBlock, 0, s>>>(g, b, scratch + nb);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BFIBM_OK : BFIBM_ECUDA;
}
