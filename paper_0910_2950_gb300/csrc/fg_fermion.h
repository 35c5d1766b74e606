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
  double pap;       // <p, Ap> of the iteration in progress (grand total of the Dslash partials)
  double rr_next;   // |r|^2 after the iteration in progress (grand total of the axpy partials)
  double beta;      // folded iteration: beta of the update in progress
  unsigned ticket[2];  // blocks finished, for the two grand totals; the last block resets it to 0
  // half-precision inner vectors hold r / sigma and p / sigma; sigma^2 is
  // reset at every reliable update to |r|^2 / n, and rho rescales p then
  double sigma2;
  double rho;
};

int vec_blocks(int n);
int dslash_blocks(int Vh);

// RS = DF (df64.cuh) evaluates the hop in double-float arithmetic on FP32
// links (instantiated for RL = float; the solver uses modes 0 and 1).
// out = b D in (mode 0); out = x + b D in (mode 1); mode 2 (CG only) also
// sums Re <pdot, out> into cgd->pap through the block partials `partial`.
// D hops from parity 1-out_par to out_par; dag = 1 applies g5 D g5.  Links
// stored as RL with NC complex entries, spinors and arithmetic in RS.  If
// `cgd` is non-null and cgd->done != 0 the kernel returns at once (converged
// CG).
template <typename RL, int NC, typename RS>
cudaError_t launch_dslash(const GeomH& g, void* out, const void* in, const void* x, const void* pdot,
                          const void* U, int out_par, int dag, int mode, double b, double* partial,
                          CgDev* cgd, cudaStream_t st);

// 16-bit formats of the inner solver's links and vectors (argument s16).
enum { S16_HALF = 0, S16_BF16 = 1 };

// 16-bit copy (format s16) of FP32 links (NC entries per link) for the inner
// Dslash.
template <int NC>
cudaError_t launch_links_to_half(int s16, const GeomH& g, const void* U32, void* U16, cudaStream_t st);

// Pseudofermion force (8 Gell-Mann components per link) into FF (momentum
// layout, precision RL); accumulate != 0 adds to FF.
template <typename RL, int NC, typename RS>
cudaError_t launch_fermion_force(const GeomH& g, const void* U, const void* Xe, const void* Xo, const void* Ye,
                                 const void* Yo, void* FF, double kappa2, int accumulate, cudaStream_t st);

// x += alpha p, r -= alpha Ap with alpha = rr / cgd->pap; |r|^2 into
// cgd->rr_next through the block partials rr_part.
template <typename R>
cudaError_t launch_cg_axpy(void* x, void* r, const void* p, const void* ap, CgDev* cgd, double* rr_part, int n,
                           cudaStream_t st);
// p = r + beta p with beta = cgd->rr_next / rr; hist[k] receives |r_k|^2 for
// k <= maxiter and *iter_out the iteration k.
template <typename R>
cudaError_t launch_cg_xpay(void* p, const void* r, CgDev* cgd, double* hist, int* iter_out, int maxiter, int n,
                           cudaStream_t st);
template <typename RI>
cudaError_t launch_ru_accumulate(void* x64, void* xs, int n, cudaStream_t st);
template <typename RI>
cudaError_t launch_ru_residual(const void* b64, const void* ax64, void* r64, void* rs, double* part, int n,
                               cudaStream_t st);
// Double-float reliable update for the FP32 solver (vectors of float4 =
// one complex double-float, x_s and r_s float2): x += x_s, x_s = 0;
// r_s = (float)(b - Ax) with partials of |r_s|^2; conversions to and from FP64.
cudaError_t launch_ru_accumulate_df(void* xdf, void* xs, int n, cudaStream_t st);
cudaError_t launch_ru_residual_df(const void* bdf, const void* axdf, void* rs, double* part, int n,
                                  cudaStream_t st);
cudaError_t launch_df_from_double(void* dst, const void* src, int n, cudaStream_t st);
cudaError_t launch_df_to_double(void* dst, const void* src, int n, cudaStream_t st);
// ---- 16-bit inner vectors (r, p, Ap and the Dslash temporaries as pairs of
// IEEE half (s16 = S16_HALF) or bfloat16 (S16_BF16) reals, scaled by
// 1/sigma; the solution increment x_s stays FP32)
// Dslash with 16-bit links and spinors of format s16, FP32 arithmetic.
template <int NC>
cudaError_t launch_dslash_h16(int s16, const GeomH& g, void* out, const void* in, const void* x, const void* pdot,
                              const void* U, int out_par, int dag, int mode, double b, double* partial,
                              CgDev* cgd, cudaStream_t st);
cudaError_t launch_cg_axpy_h16(int s16, void* xs, void* r, const void* p, const void* ap, CgDev* cgd,
                               double* rr_part, int n, cudaStream_t st);
cudaError_t launch_cg_xpay_h16(int s16, void* p, const void* r, CgDev* cgd, double* hist, int* iter_out,
                               int maxiter, int n, cudaStream_t st);
// Start of a solve: bb from the partials of |b|^2, sigma^2 = bb / n, rr = n, tol2bb, done.
cudaError_t launch_cg_init_h16(const double* part, int nparts, CgDev* cgd, double tol2, double* bb_out, int n,
                               cudaStream_t st);
// rs = b / sigma (b FP64).
cudaError_t launch_scale_to_h16(int s16, void* rs, const void* b64, const CgDev* cgd, int n, cudaStream_t st);
// dst (FP64) = sigma src (16-bit vector in scaled units).
cudaError_t launch_h16_to_double_scaled(int s16, void* dst64, const void* src16, const CgDev* cgd, int n,
                                        cudaStream_t st);
// x (double-float) += sigma x_s; x_s = 0.
cudaError_t launch_ru_accumulate_df_scaled(void* xdf, void* xs, const CgDev* cgd, int n, cudaStream_t st);
// r = b - Ax written over Ax (double-float), partials of |r|^2.
cudaError_t launch_ru_residual_df_keep(const void* bdf, void* axdf, double* part, int n, cudaStream_t st);
// r = b - Ax written to r64 (FP64), partials of |r|^2.
cudaError_t launch_ru_residual64_keep(const void* b64, const void* ax64, void* r64, double* part, int n,
                                      cudaStream_t st);
// Publish a true residual for the 16-bit solver: rr, restart, new
// sigma^2 and rho, rr[iter&1] in the new scaling, done.
cudaError_t launch_ru_publish_h16(const double* part, int nparts, CgDev* cgd, double* true_rr, int n,
                                  cudaStream_t st);
// rs = r / sigma (r double-float or FP64); p = restart ? rs : rho p.
cudaError_t launch_ru_rescale_df_h16(int s16, const void* rdf, void* rs, void* p, const CgDev* cgd, int n,
                                     cudaStream_t st);
cudaError_t launch_ru_rescale64_h16(int s16, const void* r64, void* rs, void* p, const CgDev* cgd, int n,
                                    cudaStream_t st);

// Publish a reliable update's true residual: rr, restart (true residual more
// than twice the iterated one), and with final != 0 done (rr <= tol2bb).
cudaError_t launch_ru_publish(const double* part, int n, CgDev* cgd, double* true_rr, int final, cudaStream_t st);
// p = r when the last reliable update asked for a restart (cgd->restart).
template <typename R>
cudaError_t launch_cg_restart(void* p, const void* r, const CgDev* cgd, int n, cudaStream_t st);
cudaError_t launch_cg_init(const double* part, int n, CgDev* cgd, double tol2, double* bb_out, cudaStream_t st);
// Start of a solve from an initial guess x0: |b|^2 from part_b, |b - M x0|^2
// from part_r (n partials each); rr = |b - M x0|^2, tolerance tol2 |b|^2.
cudaError_t launch_cg_init_guess(const double* part_b, const double* part_r, int n, CgDev* cgd, double tol2,
                                 double* bb_out, double* rr0_out, cudaStream_t st);

// ---- folded CG iteration (FP32 / FP64 inner vectors, links R with NC entries)
// Ap = te - k2 D_eo^dagger to on the even sites; grand totals of <p, Ap>,
// Re <r, Ap>, |Ap|^2 through `partial` (3 x dslash_blocks(Vh) entries); the
// last block sets cgd->alpha = rr / <p, Ap> and
// cgd->beta = (rr - 2 alpha Re <r, Ap> + alpha^2 |Ap|^2) / rr, rr = cgd->rr[iter & 1].
template <typename R, int NC>
cudaError_t launch_cg_apdot(const GeomH& g, void* ap, const void* to, const void* te, const void* p, const void* r,
                            const void* U, double k2, double* partial, CgDev* cgd, cudaStream_t st);
// x += alpha p; r2 = r - alpha Ap; p2 = r2 + beta p (even sites) and
// to = D_oe p2 (odd sites); |r2|^2 published as iteration iter + 1 (rr[],
// hist, *iter_out, done).  r, p and r2, p2 are different buffers.
template <typename R, int NC>
cudaError_t launch_cg_fold(const GeomH& g, void* to, void* x, const void* r, const void* ap, const void* p,
                           void* r2, void* p2, const void* U, double* partial, CgDev* cgd, double* hist,
                           int* iter_out, int maxiter, cudaStream_t st);
// dst = (RO) src, with block partials of |src|^2 if part != nullptr.
template <typename RO, typename RI>
cudaError_t launch_convert(void* dst, const void* src, double* part, int n, cudaStream_t st);
// out = a x + b y (y may be null) on n complex entries, arithmetic in FP64.
template <typename RO, typename RX, typename RY>
cudaError_t launch_lincomb(void* out, double a, const void* x, double b, const void* y, int n, cudaStream_t st);
// Block partials of Re <a, b> for FP64 vectors.
cudaError_t launch_dot64(const void* a, const void* b, double* part, int n, cudaStream_t st);
template <typename R>
cudaError_t launch_gaussian_spinor(void* chi, int Vh, uint64_t seed, uint32_t draw, cudaStream_t st);
template <typename R>
cudaError_t launch_spinor_to_device(const double* canon, void* f, int Vh, cudaStream_t st);
template <typename R>
cudaError_t launch_spinor_to_canon(const void* f, double* canon, int Vh, cudaStream_t st);

}  // namespace fg
