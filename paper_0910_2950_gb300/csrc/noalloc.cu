// Allocation-free action sums: fg_action_sums_noalloc (declared in
// include/fg_lattice.h).
//
// This is a variant of the per-site energy kernel of gauge.cu for callers
// that must not have the library allocate device memory.  It reads the gauge
// field and momenta straight from the caller's device arrays in the
// canonical FP64 layout and keeps its per-block partial sums in a fixed
// file-scope device array instead of a buffer owned by a handle.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/fg_lattice.h"
#include "fg_common.cuh"

namespace {

using fg::M3;

constexpr int kThreads = 256;
constexpr long long kMaxSites = FG_NOALLOC_MAX_SITES;
constexpr int kMaxBlocks = (int)(kMaxSites / kThreads);

// Two partial sums (S_G, T) per block of the first kernel: 2 x 65536 doubles
// = 1 MiB, resident on every device that loads the library.
static __device__ __align__(256) double g_noalloc_partials[2 * kMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_partials_addr[kMaxDevices] = {nullptr};

__device__ __forceinline__ M3<double> load_canon(const double* __restrict__ links, int lex, int mu) {
  M3<double> m;
  const double* p = links + ((size_t)lex * 4 + mu) * 18;
#pragma unroll
  for (int k = 0; k < 9; ++k) m.e[k / 3][k % 3] = fg::cx<double>(p[2 * k], p[2 * k + 1]);
  return m;
}

__device__ __forceinline__ int lex_shift(int lex, const int L[4], const int c[4], int mu) {
  const int stride[4] = {1, L[0], L[0] * L[1], L[0] * L[1] * L[2]};
  int out = lex;
#pragma unroll
  for (int d = 0; d < 4; ++d)
    if (d == mu) out += (c[d] + 1 == L[d]) ? -(L[d] - 1) * stride[d] : stride[d];
  return out;
}

// Per site: T(x) = (1/2) sum_{mu,a} p^2 and S_G(x) = beta sum_{mu<nu} (1 - Re Tr U_{mu nu}(x) / 3);
// one pair of block partial sums per block.
__global__ void __launch_bounds__(kThreads) noalloc_energy_kernel(const double* __restrict__ links,
                                                                  const double* __restrict__ mom, int L0, int L1,
                                                                  int L2, int L3, double beta,
                                                                  double* __restrict__ partials) {
  const int L[4] = {L0, L1, L2, L3};
  const int V = L0 * L1 * L2 * L3;
  const int lex = blockIdx.x * blockDim.x + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (lex < V) {
    int c[4];
    int r = lex;
    c[0] = r % L0; r /= L0;
    c[1] = r % L1; r /= L1;
    c[2] = r % L2; c[3] = r / L2;
    double sg = 0.0;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const M3<double> umu = load_canon(links, lex, mu);
      const int xpmu = lex_shift(lex, L, c, mu);
#pragma unroll
      for (int nu = mu + 1; nu < 4; ++nu) {
        const int xpnu = lex_shift(lex, L, c, nu);
        const M3<double> a = fg::mul(umu, load_canon(links, xpmu, nu));
        const M3<double> b = fg::mul(load_canon(links, lex, nu), load_canon(links, xpnu, mu));
        sg += 1.0 - fg::re_tr_mul_nd(a, b) * (1.0 / 3.0);
      }
    }
    v[0] = beta * sg;
    if (mom != nullptr) {
      double t = 0.0;
      const double* p = mom + (size_t)lex * 32;
#pragma unroll 8
      for (int k = 0; k < 32; ++k) t += p[k] * p[k];
      v[1] = 0.5 * t;
    }
  }
  fg::block_reduce_store<2>(v, partials, gridDim.x);
}

// out[k] = sum over blocks of partials[k][b], k = 0 (S_G), 1 (T), in a fixed order.
__global__ void __launch_bounds__(1024) noalloc_reduce_kernel(const double* __restrict__ partials, int nblocks,
                                                               double* __restrict__ out) {
  __shared__ double sh[32];
  for (int k = 0; k < 2; ++k) {
    double x = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) x += partials[(size_t)k * nblocks + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
      x = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) out[k] = x;
    }
    __syncthreads();
  }
}

// Device address of g_noalloc_partials on the current device.  In host code
// the symbol itself is only a stand-in for the device array, so kernels must
// be given this address instead.  It is looked up again on every call made
// outside stream capture (a device reset reloads the module and may move
// the array); during a capture the address cached by an earlier call on the
// device is used.
fg_status partials_address(cudaStream_t st, double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return FG_ECUDA;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    cudaGetLastError();
    return FG_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_partials_addr[dev] == nullptr || cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return FG_ECUDA;
    }
    g_partials_addr[dev] = (double*)p;
  }
  *out = g_partials_addr[dev];
  return FG_OK;
}

}  // namespace

extern "C" fg_status fg_action_sums_noalloc(const double* dev_links, const double* dev_momenta, const int dims[4],
                                            double beta, double* dev_out, void* cuda_stream) {
  if (!dev_links || !dev_out || !dims) return FG_EINVAL;
  long long V = 1;
  for (int i = 0; i < 4; ++i) {
    if (dims[i] < 2 || (dims[i] & 1)) return FG_EINVAL;
    V *= dims[i];
    // checked after every factor: V <= 2^24 before the next multiply, so the
    // product cannot overflow
    if (V > kMaxSites) return FG_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* partials = nullptr;
  fg_status s = partials_address(st, &partials);
  if (s != FG_OK) return s;
  const int nb = (int)((V + kThreads - 1) / kThreads);
  noalloc_energy_kernel<<<nb, kThreads, 0, st>>>(dev_links, dev_momenta, dims[0], dims[1], dims[2], dims[3], beta,
                                                 partials);
  if (cudaGetLastError() != cudaSuccess) return FG_ECUDA;
  noalloc_reduce_kernel<<<1, 1024, 0, st>>>(partials, nb, dev_out);
  if (cudaGetLastError() != cudaSuccess) return FG_ECUDA;
  return FG_OK;
}
