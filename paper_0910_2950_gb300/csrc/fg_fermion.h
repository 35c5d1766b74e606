// Launchers of the Wilson-fermion kernels (fermion.cu).  Spinor fields are
// one parity, Vec2[12][Vh] (spin-major), in the precision named by the
// template argument; `n` for vector kernels is 12 * Vh complex entries.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fg_kernels.h"

namespace fg {

// Device-side CG scalars.  rr[] is double-buffered by iteration parity so that
// a kernel can read the previous iteration's value while block 0 publishes
// the new one.
struct CgDev {
  double rr[2];
  double bb;
  double tol2bb;
  double alpha;
  int done;
  int iter;     // last completed iteration (written by xpay's block 0)
  int k_axpy;   // iteration in progress (written by axpy's block 0)
  int restart;  // set by a reliable update whose true residual left the recursion far behind
};

int vec_blocks(int n);
int dslash_blocks(int Vh);

// out = b D in (mode 0); out = x + b D in (mode 1); mode 2 also writes block
// partials of Re <pdot, out>.  D hops from parity 1-out_par to out_par;
// dag = 1 applies g5 D g5.  Links stored as RL with NC complex entries,
// spinors and arithmetic in RS.  If `done` is non-null and *done != 0 the
// kernel returns at once (converged CG).
template <typename RL, int NC, typename RS>
cudaError_t launch_dslash(const GeomH& g, void* out, const void* in, const void* x, const void* pdot,
                          const void* U, int out_par, int dag, int mode, double b, double* partial,
                          const int* done, cudaStream_t st);

// Pseudofermion force (8 Gell-Mann components per link) into FF (momentum
// layout, precision RL); accumulate != 0 adds to FF.
template <typename RL, int NC, typename RS>
cudaError_t launch_fermion_force(const GeomH& g, const void* U, const void* Xe, const void* Xo, const void* Ye,
                                 const void* Yo, void* FF, double kappa2, int accumulate, cudaStream_t st);

template <typename R>
cudaError_t launch_cg_axpy(void* x, void* r, const void* p, const void* ap, const double* pap_part, int npap,
                           CgDev* cgd, double* rr_part, int n, cudaStream_t st);
// hist[k] receives |r_k|^2 for k <= maxiter and *iter_out the iteration k.
template <typename R>
cudaError_t launch_cg_xpay(void* p, const void* r, const double* rr_part, int nrr, CgDev* cgd, double* hist,
                           int* iter_out, int maxiter, int n, cudaStream_t st);
template <typename RI>
cudaError_t launch_ru_accumulate(void* x64, void* xs, int n, cudaStream_t st);
template <typename RI>
cudaError_t launch_ru_residual(const void* b64, const void* ax64, void* r64, void* rs, double* part, int n,
                               cudaStream_t st);
cudaError_t launch_ru_publish(const double* part, int n, CgDev* cgd, double* true_rr, cudaStream_t st);
// p = r when the last reliable update asked for a restart (cgd->restart).
template <typename R>
cudaError_t launch_cg_restart(void* p, const void* r, const CgDev* cgd, int n, cudaStream_t st);
cudaError_t launch_cg_init(const double* part, int n, CgDev* cgd, double tol2, double* bb_out, cudaStream_t st);
// dst = (RO) src, with block partials of |src|^2 if part != nullptr.
template <typename RO, typename RI>
cudaError_t launch_convert(void* dst, const void* src, double* part, int n, cudaStream_t st);
// Block partials of Re <a, b> for FP64 vectors.
cudaError_t launch_dot64(const void* a, const void* b, double* part, int n, cudaStream_t st);
template <typename R>
cudaError_t launch_gaussian_spinor(void* chi, int Vh, uint64_t seed, uint32_t draw, cudaStream_t st);
template <typename R>
cudaError_t launch_spinor_to_device(const double* canon, void* f, int Vh, cudaStream_t st);
template <typename R>
cudaError_t launch_spinor_to_canon(const void* f, double* canon, int Vh, cudaStream_t st);

}  // namespace fg
