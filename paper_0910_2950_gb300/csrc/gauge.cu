// Pure-gauge kernels of the force-gradient HMC step (sm_103a).
//
//  * gauge_force_kernel: Wilson staple force F^a = (beta/6) Im Tr(lambda^a U A)
//    (the S-hat vector field of section 3), fused with what the integrator does
//    next on the same link: store it, kick the momentum, kick then drift the
//    link, or displace the link along the force for the force-gradient step
//    of Table 1 (U' = exp(-i dt^2/24 F) U).
//  * drift_kernel: the exact T-hat flow U <- exp(i c P) U (section 2).
//  * energy_kernel: per-site T(x) + S_G(x), in double-float for FP32 fields
//    and FP64 for FP64 fields, block partial sums for the dH of section 5
//    (summed as site-by-site differences).
//  * refresh_momenta_kernel: unit-Gaussian momenta from a counter-based RNG.
//
// One thread per link; a block is 64 consecutive checkerboard sites x 4
// directions, so the four links of a site and their staples share L1/L2 lines.
#include <type_traits>

#include "fg_common.cuh"
#include "fg_kernels.h"
#include "gauge_device.cuh"

namespace fg {

static Geom to_dev(const GeomH& h) {
  Geom g;
  for (int i = 0; i < 4; ++i) g.L[i] = h.L[i];
  g.Lxh = h.Lxh; g.Vh = h.Vh; g.V = h.V;
  g.dLxh = make_fastdiv((uint32_t)h.Lxh);
  g.dLy = make_fastdiv((uint32_t)h.L[1]);
  g.dLz = make_fastdiv((uint32_t)h.L[2]);
  return g;
}

constexpr int kSitesPerBlock = 64;


template <typename R, int NC, int MODE>
__global__ void __launch_bounds__(256, (kForceMinBlocks<R, NC>)) gauge_force_kernel(Gauge<R, NC> U, Mom<R> P, Mom<R> F,
                                                          Mom<R> FF, Gauge<R, NC> Ubase,
                                                          Gauge<R, NC> Uout, Geom g, R beta6,
                                                          R ckick, R cdrift, R cdisp, int reunit, R ffw) {
  if constexpr (kForceSharedT<R, NC>) {
    __shared__ float2 tsh[6][9][64];   // 64 sites: both parities x 32 half-sites (link_site)
    int s;
    const bool ok = link_site(g, s);
    force_link_shared<NC, MODE, 64>(tsh, ok, s, U, P, F, FF, Ubase, Uout, g, beta6, ckick, cdrift, cdisp, reunit,
                                    ffw);
  } else {
    int s;
    if (!link_site(g, s)) return;
    int c[4], par;
    cb_coords(g, s, c, par);
    force_link<R, NC, MODE>(U, P, F, FF, Ubase, Uout, g, c, s, (int)threadIdx.y, beta6, ckick, cdrift, cdisp,
                            reunit, ffw);
  }
}

template <typename R, int NC>
__global__ void __launch_bounds__(256) drift_kernel(Gauge<R, NC> Uin, Mom<R> P, Gauge<R, NC> Uout,
                                                    int V, R c, int reunit) {
  const int s = blockIdx.x * kSitesPerBlock + threadIdx.x;
  const int mu = threadIdx.y;
  if (s >= V) return;
  drift_link(Uin, P, Uout, s, mu, c, reunit);
}

template <typename R, int NC>
__global__ void __launch_bounds__(256) unit_links_kernel(Gauge<R, NC> U, int V) {
  const int s = blockIdx.x * kSitesPerBlock + threadIdx.x;
  const int mu = threadIdx.y;
  if (s >= V) return;
  M3<R> u;
  identity(u);
  U.store(mu, s, u);
}

// Haar-random SU(3) link from 12 Gaussians (Philox counter (4 lex + mu, draw,
// stream 5, word)): Gram-Schmidt of two complex Gaussian rows gives the first
// two rows of a Haar U(3) matrix, which fix the SU(3) matrix with the third
// row (row1 x row2)^*; SU(3) is in one-to-one correspondence with such row
// pairs, so the result is Haar on SU(3).
template <typename R, int NC>
__global__ void __launch_bounds__(256) random_links_kernel(Gauge<R, NC> U, Geom g, uint32_t k0, uint32_t k1,
                                                           uint32_t draw) {
  const int s = blockIdx.x * kSitesPerBlock + threadIdx.x;
  const int mu = threadIdx.y;
  if (s >= g.V) return;
  int c[4], par;
  cb_coords(g, s, c, par);
  const uint32_t lex = (uint32_t)(c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3])));
  R z[12];
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    uint32_t ctr[4] = {lex * 4u + (uint32_t)mu, draw, 5u, (uint32_t)q};
    Philox::rounds(ctr, k0, k1);
    box_muller<R>(ctr[0], ctr[1], z[4 * q + 0], z[4 * q + 1]);
    box_muller<R>(ctr[2], ctr[3], z[4 * q + 2], z[4 * q + 3]);
  }
  M3<R> u;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    u.e[0][j] = cx<R>(z[2 * j], z[2 * j + 1]);
    u.e[1][j] = cx<R>(z[6 + 2 * j], z[6 + 2 * j + 1]);
  }
  reunitarize(u);
  U.store(mu, s, u);
}

template <typename R, int NC>
__global__ void __launch_bounds__(256) reunitarize_kernel(Gauge<R, NC> U, int V) {
  const int s = blockIdx.x * kSitesPerBlock + threadIdx.x;
  const int mu = threadIdx.y;
  if (s >= V) return;
  M3<R> u = U.load(mu, s);
  reunitarize(u);
  U.store(mu, s, u);
}

constexpr int kEnergyThreads = 256;

// Per-site energies, one thread per site (blocks of 128 half-sites of both
// parities), block partial sums in the per-site value type A (double-float
// for FP32 fields: GB300's FP64 unit made the FP64 block tree and per-site
// arithmetic most of this kernel's time).
template <typename R>
using EnergyAcc =
    typename std::conditional<std::is_same<R, float>::value || std::is_same<R, DF>::value, DF, double>::type;

template <typename R, int NC>
__global__ void __launch_bounds__(kEnergyThreads, (std::is_same<R, float>::value ? 2 : 1))
    energy_kernel(Gauge<R, NC> U, Mom<R> P, Geom g, EnergyAcc<R> beta6, EnergyAcc<R> beta3, int mode,
                  EnergyAcc<R>* __restrict__ h0, double* __restrict__ partial,
                  const EnergyAcc<R>* __restrict__ sg_in, EnergyAcc<R>* __restrict__ sg_out) {
  using A = EnergyAcc<R>;
  int s;
  A v[3] = {A(0), A(0), A(0)};  // S_G, T, dh
  if (pair_site<kEnergyThreads / 2>(g, s)) site_energy(U, P, g, s, beta6, beta3, mode, h0, v, sg_in, sg_out);
  if constexpr (std::is_same<A, DF>::value) block_reduce_store_df<3>(v, partial, gridDim.x);
  else block_reduce_store<3>(v, partial, gridDim.x);
}

__global__ void __launch_bounds__(1024) reduce_kernel(const double* __restrict__ partial, int nblocks,
                                                      int nv, double* __restrict__ out,
                                                      int accumulate) {
  __shared__ double sh[32];
  for (int k = 0; k < nv; ++k) {
    double x = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) x += partial[(size_t)k * nblocks + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
      x = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) out[k] = accumulate ? out[k] + x : x;
    }
    __syncthreads();
  }
}

template <typename R>
__global__ void __launch_bounds__(256) refresh_momenta_kernel(Mom<R> P, Geom g, uint32_t k0,
                                                              uint32_t k1, uint32_t draw) {
  const int s = blockIdx.x * kSitesPerBlock + threadIdx.x;
  const int mu = threadIdx.y;
  if (s >= g.V) return;
  refresh_link(P, g, s, mu, k0, k1, draw, 0u);
}

template <typename R, int NC>
__global__ void gauge_to_device_kernel(const double* __restrict__ canon, Gauge<R, NC> U, Geom g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // (lex, mu)
  if (i >= 4 * g.V) return;
  const int lex = i >> 2, mu = i & 3;
  int c[4];
  int r = lex;
  c[0] = r % g.L[0]; r /= g.L[0];
  c[1] = r % g.L[1]; r /= g.L[1];
  c[2] = r % g.L[2]; c[3] = r / g.L[2];
  const int s = cb_index(g, c);
  M3<R> m;
  const double* src = canon + (size_t)i * 18;
#pragma unroll
  for (int k = 0; k < 9; ++k) m.e[k / 3][k % 3] = cx<R>(R(src[2 * k]), R(src[2 * k + 1]));
  U.store(mu, s, m);
}

template <typename R, int NC>
__global__ void gauge_to_canon_kernel(Gauge<R, NC> U, double* __restrict__ canon, Geom g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * g.V) return;
  const int lex = i >> 2, mu = i & 3;
  int c[4];
  int r = lex;
  c[0] = r % g.L[0]; r /= g.L[0];
  c[1] = r % g.L[1]; r /= g.L[1];
  c[2] = r % g.L[2]; c[3] = r / g.L[2];
  const M3<R> m = U.load(mu, cb_index(g, c));
  double* dst = canon + (size_t)i * 18;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    dst[2 * k] = double(m.e[k / 3][k % 3].re);
    dst[2 * k + 1] = double(m.e[k / 3][k % 3].im);
  }
}

template <typename R, typename T>
__global__ void mom_to_device_kernel(const T* __restrict__ canon, Mom<R> P, Geom g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * g.V) return;
  const int lex = i >> 2, mu = i & 3;
  int c[4];
  int r = lex;
  c[0] = r % g.L[0]; r /= g.L[0];
  c[1] = r % g.L[1]; r /= g.L[1];
  c[2] = r % g.L[2]; c[3] = r / g.L[2];
  R p[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) p[k] = R(canon[(size_t)i * 8 + k]);
  P.store(mu, cb_index(g, c), p);
}

template <typename R>
__global__ void mom_to_canon_kernel(Mom<R> P, double* __restrict__ canon, Geom g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 4 * g.V) return;
  const int lex = i >> 2, mu = i & 3;
  int c[4];
  int r = lex;
  c[0] = r % g.L[0]; r /= g.L[0];
  c[1] = r % g.L[1]; r /= g.L[1];
  c[2] = r % g.L[2]; c[3] = r / g.L[2];
  R p[8];
  P.load(mu, cb_index(g, c), p);
#pragma unroll
  for (int k = 0; k < 8; ++k) canon[(size_t)i * 8 + k] = double(p[k]);
}

// ---------------------------------------------------------------------------
// Launchers.
template <typename R, int NC>
static Gauge<R, NC> gauge_of(const void* p, int V) {
  Gauge<R, NC> u;
  u.p = const_cast<void*>(p);
  u.V = V;
  return u;
}
template <typename R>
static Mom<R> mom_of(const void* p, int V) {
  Mom<R> m;
  m.p = const_cast<void*>(p);
  m.V = V;
  return m;
}

static inline dim3 link_grid(int V) { return dim3((V + kSitesPerBlock - 1) / kSitesPerBlock); }
static inline dim3 pair_grid(int V) { return dim3((V / 2 + 31) / 32); }
static inline dim3 link_block() { return dim3(kSitesPerBlock, 4); }

template <typename R, int NC>
cudaError_t launch_gauge_force(const GeomH& gh, int mode, const ForceArgs& a, cudaStream_t st) {
  if constexpr (kForceSharedT<R, NC> && FG_FORCE_CARVEOUT > 0) {
    // keep the L1 share of the unified L1/shared storage as large as the
    // staple-product slots allow: the kernel's neighbour loads live in L1.
    // A preference only (once per process, thread-safe static initialisation);
    // a refusal leaves the driver's choice and is not an error.
    static const bool carved = [] {
      const cudaFuncAttribute a = cudaFuncAttributePreferredSharedMemoryCarveout;
      cudaFuncSetAttribute(gauge_force_kernel<R, NC, FM_STORE>, a, FG_FORCE_CARVEOUT);
      cudaFuncSetAttribute(gauge_force_kernel<R, NC, FM_KICK>, a, FG_FORCE_CARVEOUT);
      cudaFuncSetAttribute(gauge_force_kernel<R, NC, FM_KICK_DRIFT>, a, FG_FORCE_CARVEOUT);
      cudaFuncSetAttribute(gauge_force_kernel<R, NC, FM_DISPLACE>, a, FG_FORCE_CARVEOUT);
      cudaGetLastError();
      return true;
    }();
    (void)carved;
  }
  const Geom g = to_dev(gh);
  const int V = g.V;
  auto U = gauge_of<R, NC>(a.U, V);
  auto P = mom_of<R>(a.P, V);
  auto F = mom_of<R>(a.F, V);
  auto FF = mom_of<R>(a.FF, V);
  auto Ub = gauge_of<R, NC>(a.Ubase, V);
  auto Uo = gauge_of<R, NC>(a.Uout, V);
  const R b6 = R(a.beta / 6.0);
  const R ffw = R(a.ffw == 0.0 ? 1.0 : a.ffw);
  switch (mode) {
    case FM_STORE:
      gauge_force_kernel<R, NC, FM_STORE><<<pair_grid(V), link_block(), 0, st>>>(
          U, P, F, FF, Ub, Uo, g, b6, R(a.ckick), R(a.cdrift), R(a.cdisp), a.reunit, ffw);
      break;
    case FM_KICK:
      gauge_force_kernel<R, NC, FM_KICK><<<pair_grid(V), link_block(), 0, st>>>(
          U, P, F, FF, Ub, Uo, g, b6, R(a.ckick), R(a.cdrift), R(a.cdisp), a.reunit, ffw);
      break;
    case FM_KICK_DRIFT:
      gauge_force_kernel<R, NC, FM_KICK_DRIFT><<<pair_grid(V), link_block(), 0, st>>>(
          U, P, F, FF, Ub, Uo, g, b6, R(a.ckick), R(a.cdrift), R(a.cdisp), a.reunit, ffw);
      break;
    case FM_DISPLACE:
      gauge_force_kernel<R, NC, FM_DISPLACE><<<pair_grid(V), link_block(), 0, st>>>(
          U, P, F, FF, Ub, Uo, g, b6, R(a.ckick), R(a.cdrift), R(a.cdisp), a.reunit, ffw);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename R, int NC>
cudaError_t launch_drift(const GeomH& gh, const void* Uin, const void* P, void* Uout, double c,
                         int reunit, cudaStream_t st) {
  drift_kernel<R, NC><<<link_grid(gh.V), link_block(), 0, st>>>(
      gauge_of<R, NC>(Uin, gh.V), mom_of<R>(P, gh.V), gauge_of<R, NC>(Uout, gh.V), gh.V, R(c), reunit);
  return cudaGetLastError();
}

template <typename R, int NC>
cudaError_t launch_unit_links(const GeomH& gh, void* U, cudaStream_t st) {
  unit_links_kernel<R, NC><<<link_grid(gh.V), link_block(), 0, st>>>(gauge_of<R, NC>(U, gh.V), gh.V);
  return cudaGetLastError();
}

template <typename R, int NC>
cudaError_t launch_random_links(const GeomH& gh, void* U, uint64_t seed, uint32_t draw, cudaStream_t st) {
  random_links_kernel<R, NC><<<link_grid(gh.V), link_block(), 0, st>>>(gauge_of<R, NC>(U, gh.V), to_dev(gh),
                                                                       (uint32_t)seed, (uint32_t)(seed >> 32), draw);
  return cudaGetLastError();
}

template <typename R, int NC>
cudaError_t launch_reunitarize(const GeomH& gh, void* U, cudaStream_t st) {
  reunitarize_kernel<R, NC><<<link_grid(gh.V), link_block(), 0, st>>>(gauge_of<R, NC>(U, gh.V), gh.V);
  return cudaGetLastError();
}

template <typename R, int NC>
cudaError_t launch_energy(const GeomH& gh, const void* U, const void* P, double beta, int mode,
                          double* h0, double* partial, int* nblocks, cudaStream_t st, const double* sg_in,
                          double* sg_out) {
  const int nb = (gh.Vh + kEnergyThreads / 2 - 1) / (kEnergyThreads / 2);
  *nblocks = nb;
  // the per-site arrays are 8 bytes a site: doubles, or double-floats for FP32 fields
  using A = EnergyAcc<R>;
  static_assert(sizeof(A) == sizeof(double), "per-site slot size");
  energy_kernel<R, NC><<<nb, kEnergyThreads, 0, st>>>(
      gauge_of<R, NC>(U, gh.V), mom_of<R>(P, gh.V), to_dev(gh), A(6.0 * beta), A(beta / 3.0), mode,
      reinterpret_cast<A*>(h0), partial, reinterpret_cast<const A*>(sg_in), reinterpret_cast<A*>(sg_out));
  return cudaGetLastError();
}

cudaError_t launch_reduce(const double* partial, int nblocks, int nv, double* out, int accumulate,
                          cudaStream_t st) {
  reduce_kernel<<<1, 1024, 0, st>>>(partial, nblocks, nv, out, accumulate);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_refresh_momenta(const GeomH& gh, void* P, uint64_t seed, uint32_t draw,
                                   cudaStream_t st) {
  refresh_momenta_kernel<R><<<link_grid(gh.V), link_block(), 0, st>>>(
      mom_of<R>(P, gh.V), to_dev(gh), (uint32_t)seed, (uint32_t)(seed >> 32), draw);
  return cudaGetLastError();
}

template <typename R, int NC>
cudaError_t launch_gauge_to_device(const GeomH& gh, const double* canon, void* U, cudaStream_t st) {
  gauge_to_device_kernel<R, NC><<<(4 * gh.V + 255) / 256, 256, 0, st>>>(canon, gauge_of<R, NC>(U, gh.V),
                                                                       to_dev(gh));
  return cudaGetLastError();
}
template <typename R, int NC>
cudaError_t launch_gauge_to_canon(const GeomH& gh, const void* U, double* canon, cudaStream_t st) {
  gauge_to_canon_kernel<R, NC><<<(4 * gh.V + 255) / 256, 256, 0, st>>>(gauge_of<R, NC>(U, gh.V), canon,
                                                                      to_dev(gh));
  return cudaGetLastError();
}
template <typename R>
cudaError_t launch_mom_to_device(const GeomH& gh, const double* canon, void* P, cudaStream_t st) {
  mom_to_device_kernel<R, double><<<(4 * gh.V + 255) / 256, 256, 0, st>>>(canon, mom_of<R>(P, gh.V), to_dev(gh));
  return cudaGetLastError();
}
template <typename R>
cudaError_t launch_mom_to_canon(const GeomH& gh, const void* P, double* canon, cudaStream_t st) {
  mom_to_canon_kernel<R><<<(4 * gh.V + 255) / 256, 256, 0, st>>>(mom_of<R>(P, gh.V), canon, to_dev(gh));
  return cudaGetLastError();
}

// P -= c FF (kick with a force computed elsewhere: the pseudofermion force of
// a two-level integrator's outer kicks).
template <typename R>
__global__ void __launch_bounds__(256) kick_ff_kernel(Mom<R> P, Mom<R> FF, int V, R c) {
  const int s = blockIdx.x * kSitesPerBlock + threadIdx.x;
  const int mu = threadIdx.y;
  if (s >= V) return;
  R p[8], f[8];
  P.load(mu, s, p);
  FF.load(mu, s, f);
#pragma unroll
  for (int k = 0; k < 8; ++k) p[k] = fma(-c, f[k], p[k]);
  P.store(mu, s, p);
}
template <typename R>
cudaError_t launch_kick_ff(const GeomH& gh, void* P, const void* FF, double c, cudaStream_t st) {
  kick_ff_kernel<R><<<link_grid(gh.V), link_block(), 0, st>>>(mom_of<R>(P, gh.V), mom_of<R>(FF, gh.V), gh.V,
                                                              R(c));
  return cudaGetLastError();
}
template cudaError_t launch_kick_ff<double>(const GeomH&, void*, const void*, double, cudaStream_t);
template cudaError_t launch_kick_ff<float>(const GeomH&, void*, const void*, double, cudaStream_t);
template cudaError_t launch_kick_ff<DF>(const GeomH&, void*, const void*, double, cudaStream_t);

#define FG_INST_RNC(R, NC)                                                                          \
  template cudaError_t launch_gauge_force<R, NC>(const GeomH&, int, const ForceArgs&, cudaStream_t); \
  template cudaError_t launch_drift<R, NC>(const GeomH&, const void*, const void*, void*, double,   \
                                           int, cudaStream_t);                                      \
  template cudaError_t launch_reunitarize<R, NC>(const GeomH&, void*, cudaStream_t);                \
  template cudaError_t launch_unit_links<R, NC>(const GeomH&, void*, cudaStream_t);                 \
  template cudaError_t launch_random_links<R, NC>(const GeomH&, void*, uint64_t, uint32_t, cudaStream_t); \
  template cudaError_t launch_energy<R, NC>(const GeomH&, const void*, const void*, double, int,    \
                                            double*, double*, int*, cudaStream_t, const double*,    \
                                            double*);                                               \
  template cudaError_t launch_gauge_to_device<R, NC>(const GeomH&, const double*, void*,            \
                                                     cudaStream_t);                                 \
  template cudaError_t launch_gauge_to_canon<R, NC>(const GeomH&, const void*, double*, cudaStream_t);

FG_INST_RNC(double, 9)
FG_INST_RNC(double, 6)
FG_INST_RNC(float, 9)
FG_INST_RNC(float, 6)
FG_INST_RNC(DF, 9)
FG_INST_RNC(DF, 6)

template cudaError_t launch_refresh_momenta<double>(const GeomH&, void*, uint64_t, uint32_t, cudaStream_t);
template cudaError_t launch_refresh_momenta<float>(const GeomH&, void*, uint64_t, uint32_t, cudaStream_t);
template cudaError_t launch_refresh_momenta<DF>(const GeomH&, void*, uint64_t, uint32_t, cudaStream_t);
template cudaError_t launch_mom_to_device<double>(const GeomH&, const double*, void*, cudaStream_t);
template cudaError_t launch_mom_to_device<float>(const GeomH&, const double*, void*, cudaStream_t);
template cudaError_t launch_mom_to_device<DF>(const GeomH&, const double*, void*, cudaStream_t);
template <typename R>
cudaError_t launch_mom_to_device_f32(const GeomH& gh, const float* canon, void* P, cudaStream_t st) {
  mom_to_device_kernel<R, float><<<(4 * gh.V + 255) / 256, 256, 0, st>>>(canon, mom_of<R>(P, gh.V), to_dev(gh));
  return cudaGetLastError();
}
template cudaError_t launch_mom_to_device_f32<double>(const GeomH&, const float*, void*, cudaStream_t);
template cudaError_t launch_mom_to_device_f32<float>(const GeomH&, const float*, void*, cudaStream_t);
template cudaError_t launch_mom_to_device_f32<DF>(const GeomH&, const float*, void*, cudaStream_t);
template cudaError_t launch_mom_to_canon<double>(const GeomH&, const void*, double*, cudaStream_t);
template cudaError_t launch_mom_to_canon<float>(const GeomH&, const void*, double*, cudaStream_t);
template cudaError_t launch_mom_to_canon<DF>(const GeomH&, const void*, double*, cudaStream_t);

// FP32 FMA throughput probe: eight independent FMA chains per thread, 16
// FMAs of each per loop trip, one store per thread so nothing is dropped.
// a <- a b + c with b = 1 - 1e-4 and c = 1e-4 stays near 1 (no overflow or
// subnormals).
__global__ void __launch_bounds__(256) fma_rate_kernel(float* __restrict__ out, int iters, float b, float c) {
  float a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 0.5f + 0.01f * float(k) + 1e-6f * float(threadIdx.x);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t launch_fma_rate(float* out, int blocks, int iters, cudaStream_t st) {
  fma_rate_kernel<<<blocks, 256, 0, st>>>(out, iters, 1.0f - 1e-4f, 1e-4f);
  return cudaGetLastError();
}

}  // namespace fg
