// Host-side launchers of the device kernels (implemented in gauge.cu and
// fermion.cu, used by the runtime in fg_lattice.cu).  Every launcher enqueues
// on `st` and returns the cudaError_t of the launch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fg {

struct GeomH {
  int L[4];
  int Lxh, Vh, V;
};

// Fused gauge-force kernel modes.
enum ForceMode {
  FM_STORE = 0,       // F_out = F(U) (+ FF)
  FM_KICK = 1,        // P -= ckick F(U)
  FM_KICK_DRIFT = 2,  // P -= ckick F(U); U_out = exp(i cdrift P) U_base
  FM_DISPLACE = 3     // U_out = exp(-i cdisp F(U)) U
};

struct ForceArgs {
  const void* U;       // links at which the force is evaluated
  void* P;             // momenta
  void* F;             // force out (FM_STORE)
  const void* FF;      // extra force added to the gauge force (fermions) or nullptr
  const void* Ubase;   // drift base links (FM_KICK_DRIFT); may equal U
  void* Uout;          // output links (FM_KICK_DRIFT, FM_DISPLACE)
  double beta;
  double ckick, cdrift, cdisp;
  double ffw;          // weight of FF relative to the gauge force (0 is treated as 1)
  int reunit;
};

template <typename R, int NC>
cudaError_t launch_gauge_force(const GeomH& g, int mode, const ForceArgs& a, cudaStream_t st);

// P -= c FF on every link (a kick with an externally computed force).
template <typename R>
cudaError_t launch_kick_ff(const GeomH& g, void* P, const void* FF, double c, cudaStream_t st);

// Closed-form force gradient (forcegrad.cu): dU = i F U on every link
// (dU stored with NC = 9); G = derivative of the gauge force along dU, plus
// FFt if not null; P -= c (F - shift G).
template <typename R, int NC>
cudaError_t launch_tangent_links(const GeomH& g, const void* U, const void* F, void* dU, cudaStream_t st);
template <typename R, int NC>
cudaError_t launch_force_tangent(const GeomH& g, const void* U, const void* dU, void* G, const void* FFt,
                                 double beta, cudaStream_t st);
template <typename R>
cudaError_t launch_kick_fg(const GeomH& g, void* P, const void* F, const void* G, double c, double shift,
                           cudaStream_t st);

// U_out = exp(i c P) U_in on every link (U_out may equal U_in).
template <typename R, int NC>
cudaError_t launch_drift(const GeomH& g, const void* Uin, const void* P, void* Uout, double c,
                         int reunit, cudaStream_t st);

// Every link = identity (cold start).
template <typename R, int NC>
cudaError_t launch_unit_links(const GeomH& g, void* U, cudaStream_t st);
// FP32 FMA throughput probe: `blocks` blocks of 256 threads, each running
// 8 chains x 16 x iters FMAs; out holds blocks x 256 floats.
cudaError_t launch_fma_rate(float* out, int blocks, int iters, cudaStream_t st);

// Haar-random SU(3) links (device hot start).
template <typename R, int NC>
cudaError_t launch_random_links(const GeomH& g, void* U, uint64_t seed, uint32_t draw, cudaStream_t st);

template <typename R, int NC>
cudaError_t launch_reunitarize(const GeomH& g, void* U, cudaStream_t st);

// Per-site energy h(x) = T(x) + S_G(x) (T = 0 if P is null).  mode 0: also
// store h0[x] = h(x); mode 1: also sum h(x) - h0[x]; mode 2: sums only.  Writes per-block partial sums of
// (S_G, T, dh) into partial[3][nblocks]; returns nblocks in *nblocks.
// sg_in (optional): per-site S_G of these links stored earlier, used instead
// of the plaquettes; sg_out (optional): per-site S_G stored for later.
template <typename R, int NC>
cudaError_t launch_energy(const GeomH& g, const void* U, const void* P, double beta, int mode,
                          double* h0, double* partial, int* nblocks, cudaStream_t st,
                          const double* sg_in = nullptr, double* sg_out = nullptr);

// out[k] += sum_b partial[k][b] for k < nv (fixed order, one block).  If
// `accumulate` is 0 the sums overwrite out[k].
cudaError_t launch_reduce(const double* partial, int nblocks, int nv, double* out, int accumulate,
                          cudaStream_t st);

// Unit-Gaussian momenta from Philox-4x32-10 keyed by seed, counter (link, draw).
template <typename R>
cudaError_t launch_refresh_momenta(const GeomH& g, void* P, uint64_t seed, uint32_t draw,
                                   cudaStream_t st);

// Layout conversion between the canonical FP64 host order and device SoA.
template <typename R, int NC>
cudaError_t launch_gauge_to_device(const GeomH& g, const double* canon, void* U, cudaStream_t st);
template <typename R, int NC>
cudaError_t launch_gauge_to_canon(const GeomH& g, const void* U, double* canon, cudaStream_t st);
template <typename R>
cudaError_t launch_mom_to_device(const GeomH& g, const double* canon, void* P, cudaStream_t st);
// The same from canonical FP32 momenta.
template <typename R>
cudaError_t launch_mom_to_device_f32(const GeomH& g, const float* canon, void* P, cudaStream_t st);
template <typename R>
cudaError_t launch_mom_to_canon(const GeomH& g, const void* P, double* canon, cudaStream_t st);

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC11), usable on host and device.
struct Philox {
  static inline __host__ __device__ void mulhilo(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
  }
  static inline __host__ __device__ void rounds(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; ++r) {
      uint32_t hi0, lo0, hi1, lo1;
      mulhilo(0xD2511F53u, c[0], hi0, lo0);
      mulhilo(0xCD9E8D57u, c[2], hi1, lo1);
      const uint32_t n0 = hi1 ^ c[1] ^ k0;
      const uint32_t n2 = hi0 ^ c[3] ^ k1;
      c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
  }
};

}  // namespace fg
