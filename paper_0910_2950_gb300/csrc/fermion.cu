// Wilson fermion kernels (sm_103a): even-odd hopping term, CG vector
// updates, the pseudofermion force and the Gaussian heat bath.
//
// Section 4 of the paper writes the pseudofermion force as
// e_i(S) = -X^dagger e_i(M) X with X = M^{-1} phi; with M = Mhat^dagger Mhat
// and Mhat = 1 - kappa^2 D_eo D_oe this becomes, per link U_mu(x),
//   F^a = -kappa^2 Im Tr(lambda^a W),  W = U M1 - M2 U^dagger,
//   M1 = sum_s Xt(x+mu)_s ((1 - g_mu) Yt(x))_s^dagger,
//   M2 = sum_s Xt(x)_s ((1 + g_mu) Yt(x+mu))_s^dagger,
// with Xt = (X_e, D_oe X_e) and Yt = (Y_e, g5 D_oe g5 Y_e), Y_e = Mhat X_e.
// The rank-2 spin projectors reduce each of M1, M2 to two colour outer
// products of half spinors.
//
// Gamma matrices (DeGrand-Rossi): g_mu = [[0, A_mu], [A_mu^dagger, 0]] in 2x2
// spin blocks with A_x = [[0, i], [i, 0]], A_y = [[0, -1], [1, 0]],
// A_z = diag(i, -i), A_t = 1, so g5 = diag(1, 1, -1, -1) and
// (1 - s g_mu) psi = (h, -s A_mu^dagger h) with h = psi_up - s A_mu psi_down.
#include <type_traits>

#include "fermion_device.cuh"
#include "fg_kernels.h"

namespace fg {

constexpr int kDslashThreads = 128;

// out = b D in (MODE 0), out = x + b D in (MODE 1), and MODE 2 also writes the
// block partial sum of Re <pdot, out>.  `in` has parity 1 - out_par.
// Resident blocks asked of the register allocator.  The FP32 hop is bound by
// memory latency: six blocks of 128 (80 registers, 24 warps per SM) beat the
// unconstrained five (90 registers) by 8% at 16^3 x 32 and 24^3 x 48.  The
// double-float hop is latency-bound in arithmetic, so it is held to 128
// registers for four blocks per SM.
#ifndef FG_DSLASH_MIN_BLOCKS
#define FG_DSLASH_MIN_BLOCKS 6
#endif
template <typename RS> struct DslashMinBlocks { static constexpr int value = 1; };
template <> struct DslashMinBlocks<float> { static constexpr int value = FG_DSLASH_MIN_BLOCKS; };
#ifndef FG_DSLASH_DF_MIN_BLOCKS
#define FG_DSLASH_DF_MIN_BLOCKS 4
#endif
template <> struct DslashMinBlocks<DF> { static constexpr int value = FG_DSLASH_DF_MIN_BLOCKS; };

template <typename RL, int NC, typename RS, int DAG, int MODE, typename ST = RS>
__global__ void __launch_bounds__(kDslashThreads, DslashMinBlocks<RS>::value) dslash_kernel(
    typename Vec2<ST>::T* __restrict__ out, const typename Vec2<ST>::T* __restrict__ in,
    const typename Vec2<ST>::T* __restrict__ x, const typename Vec2<ST>::T* __restrict__ pdot,
    Gauge<RL, NC> U, Geom g, int out_par, RS b, double* __restrict__ partial, CgDev* __restrict__ cgd) {
  if (cgd != nullptr && cgd->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  RS dot = RS(0);  // one site's 24 terms in the spinor precision (GB300's FP64 unit is slow)
  if (i < g.Vh) {
    const int s = out_par * g.Vh + i;
    int c[4], par;
    cb_coords(g, s, c, par);
    const int in_off = (1 - out_par) * g.Vh;
    Spinor<RS> acc;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) acc.s[k][cc] = cx<RS>(0, 0);
    Hops<DAG, RL, NC, RS, ST>::run(acc, in, U, g, c, s, in_off);
    Spinor<RS> o;
    if (MODE == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) o.s[k][cc] = b * acc.s[k][cc];
    } else {
      const Spinor<RS> xv = load_spinor<RS, ST>(x, i, g.Vh);
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) o.s[k][cc] = xv.s[k][cc] + b * acc.s[k][cc];
      if (MODE == 2) {
        const Spinor<RS> pv = load_spinor<RS, ST>(pdot, i, g.Vh);
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int cc = 0; cc < 3; ++cc)
            dot += pv.s[k][cc].re * o.s[k][cc].re + pv.s[k][cc].im * o.s[k][cc].im;
      }
    }
    store_spinor<RS, ST>(out, i, g.Vh, o);
  }
  if (MODE == 2) block_reduce_total(double(dot), partial, &cgd->ticket[0], &cgd->pap);
}

// --------------------------------------------------------------------------- folded CG
// One CG iteration on Mhat^dagger Mhat in four launches, the vector updates
// carried by the two Dslash launches that end the operator:
//   B  t_e = p - k2 D_eo t_o                 (dslash_kernel, mode 1)
//   C  t_o = D_oe^dagger t_e                  (dslash_kernel, mode 0)
//   D  Ap = t_e - k2 D_eo^dagger t_o, grand totals of <p, Ap>, Re <r, Ap>
//      and |Ap|^2; the last block sets alpha = rr / <p, Ap> and
//      beta = rr' / rr with rr' = |r - alpha Ap|^2 expanded as
//      rr - 2 alpha Re <r, Ap> + alpha^2 |Ap|^2          (cg_apdot_kernel)
//   A  x += alpha p, r' = r - alpha Ap, p' = r' + beta p at the even sites
//      and t_o = D_oe p' at the odd ones, p' of the neighbours formed on the
//      fly from r, Ap and p; the grand total |r'|^2 is the iteration's
//      residual, published with the iteration count    (cg_fold_kernel)
// r' and p' go to the other buffer of a pair (the neighbours' r and p are
// still being read).  Only beta uses the expanded rr'; alpha of the next
// iteration and the convergence test use the summed |r'|^2.

// Block partials of NV values; the last block to finish (ticket) sums each
// in block order into tot[] (fixed for a fixed launch) and resets the
// ticket.  Returns true in that block.
template <int NV>
__device__ __forceinline__ bool block_reduce_last(double v[NV], double* __restrict__ partial,
                                                  unsigned* __restrict__ ticket, double tot[NV]) {
  block_reduce_store<NV>(v, partial, gridDim.x);
  __shared__ int last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  __shared__ double sh[NV][32];
  const int n = gridDim.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) x += __ldcg(partial + (size_t)k * n + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[k][warp] = x;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double t = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t += sh[k][w];
    tot[k] = t;
  }
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// D: Ap = te + b D^dagger_eo to at the even sites, with the three dot products.
template <typename R, int NC>
__global__ void __launch_bounds__(kDslashThreads, DslashMinBlocks<R>::value) cg_apdot_kernel(
    typename Vec2<R>::T* __restrict__ ap, const typename Vec2<R>::T* __restrict__ to,
    const typename Vec2<R>::T* __restrict__ te, const typename Vec2<R>::T* __restrict__ p,
    const typename Vec2<R>::T* __restrict__ r, Gauge<R, NC> U, Geom g, R b, double* __restrict__ partial,
    CgDev* __restrict__ cgd) {
  if (cgd->done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  R pa = R(0), ra = R(0), aa = R(0);  // one site's 24 terms each, in R
  if (i < g.Vh) {
    int c[4], par;
    cb_coords(g, i, c, par);
    Spinor<R> acc;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) acc.s[k][cc] = cx<R>(0, 0);
    hops_src<1, R, NC, R>(acc, FieldSrc<R, R>{to}, U, g, c, i, g.Vh);
    const Spinor<R> tv = load_spinor<R>(te, i, g.Vh);
    const Spinor<R> pv = load_spinor<R>(p, i, g.Vh);
    const Spinor<R> rv = load_spinor<R>(r, i, g.Vh);
    Spinor<R> o;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        o.s[k][cc] = tv.s[k][cc] + b * acc.s[k][cc];
        pa += pv.s[k][cc].re * o.s[k][cc].re + pv.s[k][cc].im * o.s[k][cc].im;
        ra += rv.s[k][cc].re * o.s[k][cc].re + rv.s[k][cc].im * o.s[k][cc].im;
        aa += o.s[k][cc].re * o.s[k][cc].re + o.s[k][cc].im * o.s[k][cc].im;
      }
    store_spinor<R>(ap, i, g.Vh, o);
  }
  double v[3] = {double(pa), double(ra), double(aa)}, tot[3];
  if (block_reduce_last<3>(v, partial, &cgd->ticket[0], tot) && threadIdx.x == 0) {
    const double rr = cgd->rr[cgd->iter & 1];
    const double alpha = tot[0] > 0.0 ? rr / tot[0] : 0.0;
    const double rrn = rr - 2.0 * alpha * tot[1] + alpha * alpha * tot[2];
    cgd->pap = tot[0];
    cgd->alpha = alpha;
    cgd->beta = (rr > 0.0 && rrn > 0.0) ? rrn / rr : 0.0;
  }
}

// A: the vector updates of the iteration and t_o = D_oe p'.
template <typename R, int NC>
__global__ void __launch_bounds__(kDslashThreads, DslashMinBlocks<R>::value) cg_fold_kernel(
    typename Vec2<R>::T* __restrict__ to, typename Vec2<R>::T* __restrict__ x,
    const typename Vec2<R>::T* __restrict__ r, const typename Vec2<R>::T* __restrict__ ap,
    const typename Vec2<R>::T* __restrict__ p, typename Vec2<R>::T* __restrict__ r2,
    typename Vec2<R>::T* __restrict__ p2, Gauge<R, NC> U, Geom g, double* __restrict__ partial,
    CgDev* __restrict__ cgd, double* __restrict__ hist, int* __restrict__ iter_out, int maxiter) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (cgd->done) {
    // no iteration after convergence, but the host has already taken r2, p2
    // as the current buffers (a certification that finds the FP64 residual
    // still too large continues from them): move r and p there
    if (i < g.Vh) {
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const size_t j = (size_t)q * g.Vh + i;
        Cx<R> a0, a1;
        Quad<R>::load(r, j, a0, a1);
        Quad<R>::store(r2, j, a0, a1);
        Quad<R>::load(p, j, a0, a1);
        Quad<R>::store(p2, j, a0, a1);
      }
    }
    return;
  }
  const FoldSrc<R> src{r, ap, p, R(cgd->alpha), R(cgd->beta)};
  R acc = R(0);
  if (i < g.Vh) {
    // the even site i: x, r', p'
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const size_t j = (size_t)q * g.Vh + i;
      Cx<R> x0, x1, r0, r1, a0, a1, p0, p1;
      Quad<R>::load(x, j, x0, x1);
      Quad<R>::load(r, j, r0, r1);
      Quad<R>::load(ap, j, a0, a1);
      Quad<R>::load(p, j, p0, p1);
      x0 = cx<R>(fma(src.alpha, p0.re, x0.re), fma(src.alpha, p0.im, x0.im));
      x1 = cx<R>(fma(src.alpha, p1.re, x1.re), fma(src.alpha, p1.im, x1.im));
      const Cx<R> q0 = src.fold_entry(r0, a0, p0), q1 = src.fold_entry(r1, a1, p1);
      r0 = cx<R>(fma(-src.alpha, a0.re, r0.re), fma(-src.alpha, a0.im, r0.im));
      r1 = cx<R>(fma(-src.alpha, a1.re, r1.re), fma(-src.alpha, a1.im, r1.im));
      Quad<R>::store(x, j, x0, x1);
      Quad<R>::store(r2, j, r0, r1);
      Quad<R>::store(p2, j, q0, q1);
      acc = fma(r0.re, r0.re, acc);
      acc = fma(r0.im, r0.im, acc);
      acc = fma(r1.re, r1.re, acc);
      acc = fma(r1.im, r1.im, acc);
    }
    // the odd site Vh + i: D_oe p'
    const int s = g.Vh + i;
    int c[4], par;
    cb_coords(g, s, c, par);
    Spinor<R> o;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) o.s[k][cc] = cx<R>(0, 0);
    hops_src<0, R, NC, R>(o, src, U, g, c, s, 0);
    store_spinor<R>(to, i, g.Vh, o);
  }
  double v[1] = {double(acc)}, tot[1];
  if (block_reduce_last<1>(v, partial, &cgd->ticket[1], tot) && threadIdx.x == 0) {
    const int k = cgd->iter + 1;
    const double rr = tot[0];
    cgd->rr[k & 1] = rr;
    if (k <= maxiter) hist[k] = rr;
    cgd->iter = k;
    *iter_out = k;
    if (rr <= cgd->tol2bb) cgd->done = 1;
  }
}

// --------------------------------------------------------------------------- force
template <int MU, typename RL, int NC, typename RS>
__device__ __forceinline__ void fermion_force_link(
    const Gauge<RL, NC>& U, const typename Vec2<RS>::T* __restrict__ Xe, const typename Vec2<RS>::T* __restrict__ Xo,
    const typename Vec2<RS>::T* __restrict__ Ye, const typename Vec2<RS>::T* __restrict__ Yo,
    const Mom<RL>& FF, const Geom& g, const int c[4], int s, int par, RL kappa2, int accumulate) {
  const int sn = cb_neighbor(g, c, MU, +1);
  const int i = s - par * g.Vh, in = sn - (1 - par) * g.Vh;
  const Spinor<RS> x0 = load_spinor<RS>(par ? Xo : Xe, i, g.Vh);
  const Spinor<RS> y0 = load_spinor<RS>(par ? Yo : Ye, i, g.Vh);
  const Spinor<RS> x1 = load_spinor<RS>(par ? Xe : Xo, in, g.Vh);
  const Spinor<RS> y1 = load_spinor<RS>(par ? Ye : Yo, in, g.Vh);
  Cx<RS> hx[2][3], hy[2][3], gx[2][3], gy[2][3];
  project<MU, 1>(x1, hx);
  project<MU, 1>(y0, hy);
  project<MU, -1>(x0, gx);
  project<MU, -1>(y1, gy);
  M3<RS> m1, m2;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      Cx<RS> s1 = cx<RS>(0, 0), s2 = cx<RS>(0, 0);
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        cmac_jc(s1, hx[k][a], hy[k][b]);
        cmac_jc(s2, gx[k][a], gy[k][b]);
      }
      m1.e[a][b] = s1;
      m2.e[a][b] = s2;
    }
  const M3<RS> u = convert<RS>(U.load(MU, s));
  M3<RS> w = mul(u, m1);
  const M3<RS> t = mul_nd(m2, u);
  const RS sign = (MU == 3 && c[3] == g.L[3] - 1) ? RS(-1) : RS(1);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) w.e[a][b] = sign * (w.e[a][b] - t.e[a][b]);
  RS f[8];
  im_tr_gellmann(w, f);
  RL out[8];
  if (accumulate) FF.load(MU, s, out);
#pragma unroll
  for (int k = 0; k < 8; ++k) out[k] = (accumulate ? out[k] : RL(0)) - kappa2 * RL(f[k]);
  FF.store(MU, s, out);
}

// Resident blocks of 256 asked of the register allocator (tuning macro).
#ifndef FG_FFORCE_MIN_BLOCKS
#define FG_FFORCE_MIN_BLOCKS 1
#endif
template <typename RL, int NC, typename RS>
__global__ void __launch_bounds__(256, FG_FFORCE_MIN_BLOCKS) fermion_force_kernel(
    Gauge<RL, NC> U, const typename Vec2<RS>::T* __restrict__ Xe, const typename Vec2<RS>::T* __restrict__ Xo,
    const typename Vec2<RS>::T* __restrict__ Ye, const typename Vec2<RS>::T* __restrict__ Yo,
    Mom<RL> FF, Geom g, RL kappa2, int accumulate) {
  int s;
  if (!link_site(g, s)) return;
  int c[4], par;
  cb_coords(g, s, c, par);
  switch (threadIdx.y) {
    case 0: fermion_force_link<0, RL, NC, RS>(U, Xe, Xo, Ye, Yo, FF, g, c, s, par, kappa2, accumulate); break;
    case 1: fermion_force_link<1, RL, NC, RS>(U, Xe, Xo, Ye, Yo, FF, g, c, s, par, kappa2, accumulate); break;
    case 2: fermion_force_link<2, RL, NC, RS>(U, Xe, Xo, Ye, Yo, FF, g, c, s, par, kappa2, accumulate); break;
    default: fermion_force_link<3, RL, NC, RS>(U, Xe, Xo, Ye, Yo, FF, g, c, s, par, kappa2, accumulate); break;
  }
}

// --------------------------------------------------------------------------- CG vectors
constexpr int kVecThreads = 256;

// Sum of `n` partials in a fixed order, computed by every block (so each block
// derives the same scalar without another launch).
__device__ __forceinline__ double block_sum_partials(const double* __restrict__ part, int n) {
  __shared__ double sh[32];
  double x = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) x += part[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    sh[0] = t;
  }
  __syncthreads();
  const double r = sh[0];
  __syncthreads();
  return r;
}

// Iteration k = iter + 1 (iter was published by the previous iteration's
// xpay kernel): alpha = rr[(k-1)&1] / pAp; x += alpha p; r -= alpha Ap;
// |r|^2 into cgd->rr_next.  Block 0 passes k on to xpay through k_axpy.
// The kernels take no iteration argument, so a batch of iterations can be
// captured once in a CUDA graph and replayed.
template <typename R>
__global__ void __launch_bounds__(kVecThreads) cg_axpy_kernel(
    typename Vec2<R>::T* __restrict__ x, typename Vec2<R>::T* __restrict__ r,
    const typename Vec2<R>::T* __restrict__ p, const typename Vec2<R>::T* __restrict__ ap,
    CgDev* __restrict__ cgd, double* __restrict__ rr_part, int n) {
  if (cgd->done) return;
  const int k = cgd->iter + 1;
  const double pap = cgd->pap;
  const double rr = cgd->rr[(k - 1) & 1];
  const double alpha = pap > 0.0 ? rr / pap : 0.0;
  const R a = R(alpha);
  R acc = R(0);  // a thread's few entries in R; blocks and the total in FP64
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    typename Vec2<R>::T xv = x[i], rv = r[i];
    const typename Vec2<R>::T pv = p[i], av = ap[i];
    xv.x = fma(a, pv.x, xv.x); xv.y = fma(a, pv.y, xv.y);
    rv.x = fma(-a, av.x, rv.x); rv.y = fma(-a, av.y, rv.y);
    x[i] = xv;
    r[i] = rv;
    acc = fma(rv.x, rv.x, acc);
    acc = fma(rv.y, rv.y, acc);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cgd->alpha = alpha;
    cgd->k_axpy = k;
  }
  block_reduce_total(double(acc), rr_part, &cgd->ticket[1], &cgd->rr_next);
}

// rr_new = cgd->rr_next; done if rr_new <= tol2 bb; beta = rr_new / rr_old;
// p = r + beta p (also on the converging iteration, so that a reliable update
// that finds the true residual still too large can simply continue).
// Block 0 publishes rr[k&1], the history entry, iter = k (also to the host
// through iter_out) and `done`; no block of this kernel reads those.
template <typename R>
__global__ void __launch_bounds__(kVecThreads) cg_xpay_kernel(
    typename Vec2<R>::T* __restrict__ p, const typename Vec2<R>::T* __restrict__ r,
    CgDev* __restrict__ cgd, double* __restrict__ hist, int* __restrict__ iter_out, int maxiter, int n) {
  if (cgd->done) return;
  const int k = cgd->k_axpy;
  const double rr_new = cgd->rr_next;
  const double rr_old = cgd->rr[(k - 1) & 1];
  const bool conv = rr_new <= cgd->tol2bb;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cgd->rr[k & 1] = rr_new;
    if (k <= maxiter) hist[k] = rr_new;
    cgd->iter = k;
    *iter_out = k;
    if (conv) cgd->done = 1;
  }
  const R beta = R(rr_old > 0.0 ? rr_new / rr_old : 0.0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    typename Vec2<R>::T pv = p[i];
    const typename Vec2<R>::T rv = r[i];
    pv.x = fma(beta, pv.x, rv.x);
    pv.y = fma(beta, pv.y, rv.y);
    p[i] = pv;
  }
}

// Reliable update, first half: x64 += x_s; x_s = 0.
template <typename RI>
__global__ void __launch_bounds__(kVecThreads) ru_accumulate_kernel(double2* __restrict__ x,
                                                                    typename Vec2<RI>::T* __restrict__ xs, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const typename Vec2<RI>::T v = xs[i];
    double2 a = x[i];
    a.x += double(v.x);
    a.y += double(v.y);
    x[i] = a;
    typename Vec2<RI>::T z;
    z.x = RI(0); z.y = RI(0);
    xs[i] = z;
  }
}

// Reliable update, second half: r64 = b - Ax; r_s = (RI) r64; partial |r64|^2.
template <typename RI>
__global__ void __launch_bounds__(kVecThreads) ru_residual_kernel(const double2* __restrict__ b,
                                                                  const double2* __restrict__ ax,
                                                                  double2* __restrict__ r,
                                                                  typename Vec2<RI>::T* __restrict__ rs,
                                                                  double* __restrict__ part, int n) {
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double2 bv = b[i], av = ax[i];
    double2 rv;
    rv.x = bv.x - av.x;
    rv.y = bv.y - av.y;
    r[i] = rv;
    typename Vec2<RI>::T s;
    s.x = RI(rv.x);
    s.y = RI(rv.y);
    rs[i] = s;
    acc += rv.x * rv.x + rv.y * rv.y;
  }
  double v[1] = {acc};
  block_reduce_store<1>(v, part, gridDim.x);
}

// Double-float reliable update (FP32 inner solver), first half:
// x += x_s in double-float; x_s = 0.
__global__ void __launch_bounds__(kVecThreads) ru_accumulate_df_kernel(float4* __restrict__ x,
                                                                       float2* __restrict__ xs, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 v = xs[i];
    float4 a = x[i];
    const DF re = df_add_f(DF(a.x, a.y), v.x), im = df_add_f(DF(a.z, a.w), v.y);
    x[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
    xs[i] = make_float2(0.0f, 0.0f);
  }
}

// Second half: r = b - Ax in double-float, r_s = (float) r, |r|^2 from the
// rounded r_s (a thread's entries in FP32, blocks in FP64).
__global__ void __launch_bounds__(kVecThreads) ru_residual_df_kernel(const float4* __restrict__ b,
                                                                     const float4* __restrict__ ax,
                                                                     float2* __restrict__ rs,
                                                                     double* __restrict__ part, int n) {
  float acc = 0.0f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 bv = b[i], av = ax[i];
    const DF re = DF(bv.x, bv.y) - DF(av.x, av.y), im = DF(bv.z, bv.w) - DF(av.z, av.w);
    rs[i] = make_float2(re.hi, im.hi);
    acc = fmaf(re.hi, re.hi, acc);
    acc = fmaf(im.hi, im.hi, acc);
  }
  double v[1] = {double(acc)};
  block_reduce_store<1>(v, part, gridDim.x);
}

// FP64 <-> double-float vectors (n complex entries).
__global__ void __launch_bounds__(kVecThreads) df_from_double_kernel(float4* __restrict__ dst,
                                                                     const double2* __restrict__ src, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double2 v = src[i];
    const DF re(v.x), im(v.y);
    dst[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
  }
}
__global__ void __launch_bounds__(kVecThreads) df_to_double_kernel(double2* __restrict__ dst,
                                                                   const float4* __restrict__ src, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 v = src[i];
    dst[i] = make_double2(double(DF(v.x, v.y)), double(DF(v.z, v.w)));
  }
}

// ---------------------------------------------------------------------------
// 16-bit inner vectors (S = Half16 or BF16).  The solver iterates on
// r / sigma: CG is invariant under a common scale of r and p, and keeping
// |r / sigma|^2 = n after every reliable update keeps the entries O(1), far
// from the ends of the half range.  Scalars (rr, pAp, alpha, beta) are in the scaled units;
// the history and the convergence test use rr sigma^2.
template <typename S>
__global__ void __launch_bounds__(kVecThreads) cg_axpy_h16_kernel(float2* __restrict__ x,
                                                                  typename Conv16<S>::T2* __restrict__ r,
                                                                  const typename Conv16<S>::T2* __restrict__ p,
                                                                  const typename Conv16<S>::T2* __restrict__ ap,
                                                                  CgDev* __restrict__ cgd, double* __restrict__ rr_part,
                                                                  int n) {
  if (cgd->done) return;
  const int k = cgd->iter + 1;
  const double pap = cgd->pap;
  const double rr = cgd->rr[(k - 1) & 1];
  const double alpha = pap > 0.0 ? rr / pap : 0.0;
  const float a = float(alpha);
  float acc = 0.0f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float2 xv = x[i];
    float2 rv = Conv16<S>::f2(r[i]);
    const float2 pv = Conv16<S>::f2(p[i]), av = Conv16<S>::f2(ap[i]);
    xv.x = fmaf(a, pv.x, xv.x); xv.y = fmaf(a, pv.y, xv.y);
    rv.x = fmaf(-a, av.x, rv.x); rv.y = fmaf(-a, av.y, rv.y);
    x[i] = xv;
    const typename Conv16<S>::T2 rh = Conv16<S>::of(rv);
    r[i] = rh;
    const float2 rq = Conv16<S>::f2(rh);   // |r|^2 of the stored residual
    acc = fmaf(rq.x, rq.x, acc);
    acc = fmaf(rq.y, rq.y, acc);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cgd->alpha = alpha;
    cgd->k_axpy = k;
  }
  block_reduce_total(double(acc), rr_part, &cgd->ticket[1], &cgd->rr_next);
}

template <typename S>
__global__ void __launch_bounds__(kVecThreads) cg_xpay_h16_kernel(typename Conv16<S>::T2* __restrict__ p,
                                                                  const typename Conv16<S>::T2* __restrict__ r,
                                                                  CgDev* __restrict__ cgd, double* __restrict__ hist,
                                                                  int* __restrict__ iter_out, int maxiter, int n) {
  if (cgd->done) return;
  const int k = cgd->k_axpy;
  const double rr_new = cgd->rr_next;
  const double rr_old = cgd->rr[(k - 1) & 1];
  const double rr_true = rr_new * cgd->sigma2;
  const bool conv = rr_true <= cgd->tol2bb;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cgd->rr[k & 1] = rr_new;
    if (k <= maxiter) hist[k] = rr_true;
    cgd->iter = k;
    *iter_out = k;
    if (conv) cgd->done = 1;
  }
  const float beta = float(rr_old > 0.0 ? rr_new / rr_old : 0.0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float2 pv = Conv16<S>::f2(p[i]);
    const float2 rv = Conv16<S>::f2(r[i]);
    pv.x = fmaf(beta, pv.x, rv.x);
    pv.y = fmaf(beta, pv.y, rv.y);
    p[i] = Conv16<S>::of(pv);
  }
}

__global__ void cg_init_h16_kernel(const double* __restrict__ part, int nparts, CgDev* __restrict__ cgd, double tol2,
                                   double* __restrict__ bb_out, int n) {
  const double bb = block_sum_partials(part, nparts);
  if (threadIdx.x == 0) {
    const double s2 = bb > 0.0 ? bb / n : 1.0;
    cgd->bb = bb;
    cgd->tol2bb = tol2 * bb;
    cgd->sigma2 = s2;
    cgd->rho = 1.0;
    cgd->rr[0] = cgd->rr[1] = bb / s2;
    cgd->done = bb == 0.0 ? 1 : 0;
    cgd->iter = 0;
    cgd->k_axpy = 0;
    cgd->restart = 0;
    *bb_out = bb;
  }
}

template <typename S>
__global__ void __launch_bounds__(kVecThreads) scale_to_h16_kernel(typename Conv16<S>::T2* __restrict__ rs,
                                                                   const double2* __restrict__ b,
                                                                   const CgDev* __restrict__ cgd, int n) {
  const double inv = 1.0 / sqrt(cgd->sigma2);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double2 v = b[i];
    rs[i] = Conv16<S>::of(make_float2(float(v.x * inv), float(v.y * inv)));
  }
}

// dst (FP64) = sigma src (16-bit inner vector in scaled units).
template <typename S>
__global__ void __launch_bounds__(kVecThreads) h16_to_double_scaled_kernel(double2* __restrict__ dst,
                                                                          const typename Conv16<S>::T2* __restrict__ src,
                                                                          const CgDev* __restrict__ cgd, int n) {
  const double sg = sqrt(cgd->sigma2);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 v = Conv16<S>::f2(src[i]);
    dst[i] = make_double2(sg * (double)v.x, sg * (double)v.y);
  }
}

__global__ void __launch_bounds__(kVecThreads) ru_accumulate_df_scaled_kernel(float4* __restrict__ x,
                                                                              float2* __restrict__ xs,
                                                                              const CgDev* __restrict__ cgd,
                                                                              int n) {
  const float sg = float(sqrt(cgd->sigma2));
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float2 v = xs[i];
    const float4 a = x[i];
    const DF re = df_add_f(DF(a.x, a.y), sg * v.x), im = df_add_f(DF(a.z, a.w), sg * v.y);
    x[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
    xs[i] = make_float2(0.0f, 0.0f);
  }
}

__global__ void __launch_bounds__(kVecThreads) ru_residual_df_keep_kernel(const float4* __restrict__ b,
                                                                          float4* __restrict__ ax,
                                                                          double* __restrict__ part, int n) {
  float acc = 0.0f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 bv = b[i], av = ax[i];
    const DF re = DF(bv.x, bv.y) - DF(av.x, av.y), im = DF(bv.z, bv.w) - DF(av.z, av.w);
    ax[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
    acc = fmaf(re.hi, re.hi, acc);
    acc = fmaf(im.hi, im.hi, acc);
  }
  double v[1] = {double(acc)};
  block_reduce_store<1>(v, part, gridDim.x);
}

__global__ void __launch_bounds__(kVecThreads) ru_residual64_keep_kernel(const double2* __restrict__ b,
                                                                         const double2* __restrict__ ax,
                                                                         double2* __restrict__ r,
                                                                         double* __restrict__ part, int n) {
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double2 bv = b[i], av = ax[i];
    const double2 rv = make_double2(bv.x - av.x, bv.y - av.y);
    r[i] = rv;
    acc += rv.x * rv.x + rv.y * rv.y;
  }
  double v[1] = {acc};
  block_reduce_store<1>(v, part, gridDim.x);
}

__global__ void ru_publish_h16_kernel(const double* __restrict__ part, int nparts, CgDev* __restrict__ cgd,
                                      double* __restrict__ true_rr, int n) {
  const double rr = block_sum_partials(part, nparts);
  if (threadIdx.x == 0) {
    const double rr_iter = cgd->rr[cgd->iter & 1] * cgd->sigma2;
    const double s2 = rr > 0.0 ? rr / n : cgd->sigma2;
    cgd->restart = (rr > 2.0 * rr_iter) ? 1 : 0;
    cgd->rho = sqrt(cgd->sigma2 / s2);
    cgd->sigma2 = s2;
    cgd->rr[cgd->iter & 1] = rr / s2;
    cgd->done = rr <= cgd->tol2bb ? 1 : 0;
    *true_rr = rr;
  }
}

template <typename S, typename RV>
__global__ void __launch_bounds__(kVecThreads) ru_rescale_h16_kernel(const RV* __restrict__ r,
                                                                     typename Conv16<S>::T2* __restrict__ rs,
                                                                     typename Conv16<S>::T2* __restrict__ p,
                                                                     const CgDev* __restrict__ cgd, int n) {
  const double inv = 1.0 / sqrt(cgd->sigma2);
  const float rho = float(cgd->rho);
  const bool restart = cgd->restart != 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double re, im;
    if constexpr (std::is_same<RV, float4>::value) {   // double-float residual
      const float4 v = ((const float4*)r)[i];
      re = double(DF(v.x, v.y));
      im = double(DF(v.z, v.w));
    } else {
      const double2 v = ((const double2*)r)[i];
      re = v.x;
      im = v.y;
    }
    const typename Conv16<S>::T2 h = Conv16<S>::of(make_float2(float(re * inv), float(im * inv)));
    rs[i] = h;
    if (restart) {
      p[i] = h;
    } else {
      const float2 pv = Conv16<S>::f2(p[i]);
      p[i] = Conv16<S>::of(make_float2(rho * pv.x, rho * pv.y));
    }
  }
}

// Publishes a reliable-update residual after iteration k = iter:
// rr[k&1] = |r|^2, done = rr <= tol2 bb.  The search direction is kept (the
// usual reliable update) while the true |r|^2 is within a factor 2 of the
// recursive one it replaces; beyond that the recursion has drifted too far
// for p to match r, and `restart` asks cg_restart_kernel to set p = r.
__global__ void ru_publish_kernel(const double* __restrict__ part, int n, CgDev* __restrict__ cgd,
                                  double* __restrict__ true_rr, int final) {
  const double rr = block_sum_partials(part, n);
  if (threadIdx.x == 0) {
    const double rr_iter = cgd->rr[cgd->iter & 1];
    cgd->restart = (rr > 2.0 * rr_iter) ? 1 : 0;
    cgd->rr[cgd->iter & 1] = rr;
    // only the certifying update ends the solve; after an intermediate one
    // the next iteration publishes the residual, which the host watches
    cgd->done = (final && rr <= cgd->tol2bb) ? 1 : 0;
    *true_rr = rr;
  }
}

// p = r_s after a reliable update that asked for a restart.
template <typename R>
__global__ void __launch_bounds__(kVecThreads) cg_restart_kernel(typename Vec2<R>::T* __restrict__ p,
                                                                 const typename Vec2<R>::T* __restrict__ r,
                                                                 const CgDev* __restrict__ cgd, int n) {
  if (!cgd->restart) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = r[i];
}

// Start of a solve: bb = |b|^2 from partials, rr = bb, done = (bb == 0).
__global__ void cg_init_kernel(const double* __restrict__ part, int n, CgDev* __restrict__ cgd, double tol2,
                               double* __restrict__ bb_out) {
  const double bb = block_sum_partials(part, n);
  if (threadIdx.x == 0) {
    cgd->bb = bb;
    cgd->tol2bb = tol2 * bb;
    cgd->rr[0] = cgd->rr[1] = bb;
    cgd->done = bb == 0.0 ? 1 : 0;
    cgd->iter = 0;
    cgd->k_axpy = 0;
    cgd->restart = 0;
    *bb_out = bb;
  }
}

// Start of a solve from an initial guess: bb = |b|^2 and rr = |b - M x0|^2
// from their partials; the tolerance stays relative to |b|.
__global__ void cg_init_guess_kernel(const double* __restrict__ part_b, const double* __restrict__ part_r, int n,
                                     CgDev* __restrict__ cgd, double tol2, double* __restrict__ bb_out,
                                     double* __restrict__ rr0_out) {
  const double bb = block_sum_partials(part_b, n);
  const double rr = block_sum_partials(part_r, n);
  if (threadIdx.x == 0) {
    cgd->bb = bb;
    cgd->tol2bb = tol2 * bb;
    cgd->rr[0] = cgd->rr[1] = rr;
    cgd->done = (bb == 0.0 || rr <= tol2 * bb) ? 1 : 0;
    cgd->iter = 0;
    cgd->k_axpy = 0;
    cgd->restart = 0;
    *bb_out = bb;
    *rr0_out = rr;
  }
}

// dst = (RO) src; optional partial |src|^2.
template <typename RO, typename RI>
__global__ void __launch_bounds__(kVecThreads) convert_kernel(typename Vec2<RO>::T* __restrict__ dst,
                                                              const typename Vec2<RI>::T* __restrict__ src,
                                                              double* __restrict__ part, int n) {
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const typename Vec2<RI>::T v = src[i];
    typename Vec2<RO>::T o;
    o.x = RO(v.x);
    o.y = RO(v.y);
    dst[i] = o;
    acc += double(v.x) * v.x + double(v.y) * v.y;
  }
  if (part != nullptr) {
    double v[1] = {acc};
    block_reduce_store<1>(v, part, gridDim.x);
  }
}

__global__ void __launch_bounds__(kVecThreads) dot64_kernel(const double2* __restrict__ a,
                                                             const double2* __restrict__ b,
                                                             double* __restrict__ part, int n) {
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double2 x = a[i], y = b[i];
    acc += x.x * y.x + x.y * y.y;
  }
  double v[1] = {acc};
  block_reduce_store<1>(v, part, gridDim.x);
}

// Complex Gaussian spinor with density exp(-|chi|^2): re, im ~ N(0, 1/2).
template <typename R>
__global__ void __launch_bounds__(256) gaussian_spinor_kernel(typename Vec2<R>::T* __restrict__ chi, int Vh,
                                                              uint32_t k0, uint32_t k1, uint32_t draw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Vh) return;
  const double inv_sqrt2 = 0.70710678118654752440;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    uint32_t ctr[4] = {(uint32_t)i, draw, 1u /* stream: pseudofermion */, (uint32_t)q};
    Philox::rounds(ctr, k0, k1);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const double u1 = ((double)ctr[2 * h] + 1.0) * 2.3283064365386963e-10;
      const double u2 = (double)ctr[2 * h + 1] * 2.3283064365386963e-10;
      const double rad = sqrt(-2.0 * log(u1)) * inv_sqrt2;
      double sn, cs;
      sincospi(2.0 * u2, &sn, &cs);
      typename Vec2<R>::T v;
      v.x = R(rad * cs);
      v.y = R(rad * sn);
      chi[(size_t)(2 * q + h) * Vh + i] = v;
    }
  }
}

// canonical [Vh][12] complex <-> device pair-major (entry k of site i at
// pair k / 2, slot k % 2: flat complex index ((k / 2) * Vh + i) * 2 + k % 2)
template <typename R>
__global__ void spinor_to_device_kernel(const double* __restrict__ canon, typename Vec2<R>::T* __restrict__ f, int Vh) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 12 * Vh) return;
  const int i = t / 12, k = t % 12;
  typename Vec2<R>::T v;
  v.x = R(canon[(size_t)t * 2]);
  v.y = R(canon[(size_t)t * 2 + 1]);
  f[((size_t)(k >> 1) * Vh + i) * 2 + (k & 1)] = v;
}

template <typename R>
__global__ void spinor_to_canon_kernel(const typename Vec2<R>::T* __restrict__ f, double* __restrict__ canon, int Vh) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 12 * Vh) return;
  const int i = t / 12, k = t % 12;
  const typename Vec2<R>::T v = f[((size_t)(k >> 1) * Vh + i) * 2 + (k & 1)];
  canon[(size_t)t * 2] = v.x;
  canon[(size_t)t * 2 + 1] = v.y;
}

// ============================================================================ launchers
template <typename R> static typename Vec2<R>::T* v2(void* p) { return (typename Vec2<R>::T*)p; }
template <typename R> static const typename Vec2<R>::T* cv2(const void* p) { return (const typename Vec2<R>::T*)p; }

int vec_blocks(int n) {
  int b = (n + kVecThreads - 1) / kVecThreads;
  return b > 152 * 8 ? 152 * 8 : b;
}
int dslash_blocks(int Vh) { return (Vh + kDslashThreads - 1) / kDslashThreads; }

template <typename RL, int NC, typename RS>
cudaError_t launch_dslash(const GeomH& gh, void* out, const void* in, const void* x, const void* pdot,
                          const void* U, int out_par, int dag, int mode, double b, double* partial,
                          CgDev* cgd, cudaStream_t st) {
  Gauge<RL, NC> u;
  u.p = const_cast<void*>(U);
  u.V = gh.V;
  const Geom g = to_devg(gh);
  const int nb = dslash_blocks(gh.Vh);
#define FG_DS(D, M)                                                                                     \
  dslash_kernel<RL, NC, RS, D, M><<<nb, kDslashThreads, 0, st>>>(v2<RS>(out), cv2<RS>(in), cv2<RS>(x),   \
                                                                 cv2<RS>(pdot), u, g, out_par, RS(b),   \
                                                                 partial, cgd)
  if (dag) {
    if (mode == 0) FG_DS(1, 0); else if (mode == 1) FG_DS(1, 1); else FG_DS(1, 2);
  } else {
    if (mode == 0) FG_DS(0, 0); else if (mode == 1) FG_DS(0, 1); else FG_DS(0, 2);
  }
#undef FG_DS
  return cudaGetLastError();
}

template <typename RL, int NC, typename RS>
cudaError_t launch_fermion_force(const GeomH& gh, const void* U, const void* Xe, const void* Xo, const void* Ye,
                                 const void* Yo, void* FF, double kappa2, int accumulate, cudaStream_t st) {
  Gauge<RL, NC> u;
  u.p = const_cast<void*>(U);
  u.V = gh.V;
  Mom<RL> f;
  f.p = FF;
  f.V = gh.V;
  fermion_force_kernel<RL, NC, RS><<<(gh.Vh + 31) / 32, dim3(64, 4), 0, st>>>(
      u, cv2<RS>(Xe), cv2<RS>(Xo), cv2<RS>(Ye), cv2<RS>(Yo), f, to_devg(gh), RL(kappa2), accumulate);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_cg_axpy(void* x, void* r, const void* p, const void* ap, CgDev* cgd, double* rr_part, int n,
                           cudaStream_t st) {
  cg_axpy_kernel<R><<<vec_blocks(n), kVecThreads, 0, st>>>(v2<R>(x), v2<R>(r), cv2<R>(p), cv2<R>(ap), cgd,
                                                           rr_part, n);
  return cudaGetLastError();
}
template <typename R>
cudaError_t launch_cg_xpay(void* p, const void* r, CgDev* cgd, double* hist, int* iter_out, int maxiter, int n,
                           cudaStream_t st) {
  cg_xpay_kernel<R><<<vec_blocks(n), kVecThreads, 0, st>>>(v2<R>(p), cv2<R>(r), cgd, hist, iter_out, maxiter, n);
  return cudaGetLastError();
}
template <typename R, int NC>
cudaError_t launch_cg_apdot(const GeomH& gh, void* ap, const void* to, const void* te, const void* p, const void* r,
                            const void* U, double k2, double* partial, CgDev* cgd, cudaStream_t st) {
  Gauge<R, NC> u;
  u.p = const_cast<void*>(U);
  u.V = gh.V;
  cg_apdot_kernel<R, NC><<<dslash_blocks(gh.Vh), kDslashThreads, 0, st>>>(
      v2<R>(ap), cv2<R>(to), cv2<R>(te), cv2<R>(p), cv2<R>(r), u, to_devg(gh), R(-k2), partial, cgd);
  return cudaGetLastError();
}
template <typename R, int NC>
cudaError_t launch_cg_fold(const GeomH& gh, void* to, void* x, const void* r, const void* ap, const void* p,
                           void* r2, void* p2, const void* U, double* partial, CgDev* cgd, double* hist,
                           int* iter_out, int maxiter, cudaStream_t st) {
  Gauge<R, NC> u;
  u.p = const_cast<void*>(U);
  u.V = gh.V;
  cg_fold_kernel<R, NC><<<dslash_blocks(gh.Vh), kDslashThreads, 0, st>>>(
      v2<R>(to), v2<R>(x), cv2<R>(r), cv2<R>(ap), cv2<R>(p), v2<R>(r2), v2<R>(p2), u, to_devg(gh), partial, cgd,
      hist, iter_out, maxiter);
  return cudaGetLastError();
}
template <typename RI>
cudaError_t launch_ru_accumulate(void* x64, void* xs, int n, cudaStream_t st) {
  ru_accumulate_kernel<RI><<<vec_blocks(n), kVecThreads, 0, st>>>((double2*)x64, v2<RI>(xs), n);
  return cudaGetLastError();
}
template <typename RI>
cudaError_t launch_ru_residual(const void* b64, const void* ax64, void* r64, void* rs, double* part, int n,
                               cudaStream_t st) {
  ru_residual_kernel<RI><<<vec_blocks(n), kVecThreads, 0, st>>>((const double2*)b64, (const double2*)ax64,
                                                                (double2*)r64, v2<RI>(rs), part, n);
  return cudaGetLastError();
}
cudaError_t launch_ru_publish(const double* part, int n, CgDev* cgd, double* true_rr, int final, cudaStream_t st) {
  ru_publish_kernel<<<1, 1024, 0, st>>>(part, n, cgd, true_rr, final);
  return cudaGetLastError();
}
template <typename R>
cudaError_t launch_cg_restart(void* p, const void* r, const CgDev* cgd, int n, cudaStream_t st) {
  cg_restart_kernel<R><<<vec_blocks(n), kVecThreads, 0, st>>>(v2<R>(p), cv2<R>(r), cgd, n);
  return cudaGetLastError();
}
cudaError_t launch_cg_init(const double* part, int n, CgDev* cgd, double tol2, double* bb_out, cudaStream_t st) {
  cg_init_kernel<<<1, 1024, 0, st>>>(part, n, cgd, tol2, bb_out);
  return cudaGetLastError();
}
cudaError_t launch_cg_init_guess(const double* part_b, const double* part_r, int n, CgDev* cgd, double tol2,
                                 double* bb_out, double* rr0_out, cudaStream_t st) {
  cg_init_guess_kernel<<<1, 1024, 0, st>>>(part_b, part_r, n, cgd, tol2, bb_out, rr0_out);
  return cudaGetLastError();
}
template <typename RO, typename RI>
cudaError_t launch_convert(void* dst, const void* src, double* part, int n, cudaStream_t st) {
  convert_kernel<RO, RI><<<vec_blocks(n), kVecThreads, 0, st>>>(v2<RO>(dst), cv2<RI>(src), part, n);
  return cudaGetLastError();
}
cudaError_t launch_ru_accumulate_df(void* xdf, void* xs, int n, cudaStream_t st) {
  ru_accumulate_df_kernel<<<vec_blocks(n), kVecThreads, 0, st>>>((float4*)xdf, (float2*)xs, n);
  return cudaGetLastError();
}
cudaError_t launch_ru_residual_df(const void* bdf, const void* axdf, void* rs, double* part, int n,
                                  cudaStream_t st) {
  ru_residual_df_kernel<<<vec_blocks(n), kVecThreads, 0, st>>>((const float4*)bdf, (const float4*)axdf,
                                                                (float2*)rs, part, n);
  return cudaGetLastError();
}
cudaError_t launch_df_from_double(void* dst, const void* src, int n, cudaStream_t st) {
  df_from_double_kernel<<<vec_blocks(n), kVecThreads, 0, st>>>((float4*)dst, (const double2*)src, n);
  return cudaGetLastError();
}
cudaError_t launch_df_to_double(void* dst, const void* src, int n, cudaStream_t st) {
  df_to_double_kernel<<<vec_blocks(n), kVecThreads, 0, st>>>((double2*)dst, (const float4*)src, n);
  return cudaGetLastError();
}
template <typename S, int NC>
static cudaError_t dslash16(const GeomH& gh, void* out, const void* in, const void* x, const void* pdot,
                            const void* U, int out_par, int dag, int mode, double b, double* partial, CgDev* cgd,
                            cudaStream_t st) {
  typedef typename Conv16<S>::T2 T2;
  Gauge<S, NC> u;
  u.p = const_cast<void*>(U);
  u.V = gh.V;
  const Geom g = to_devg(gh);
  const int nb = dslash_blocks(gh.Vh);
#define FG_DH(D, M)                                                                                            \
  dslash_kernel<S, NC, float, D, M, S><<<nb, kDslashThreads, 0, st>>>(                                        \
      (T2*)out, (const T2*)in, (const T2*)x, (const T2*)pdot, u, g, out_par, float(b), partial, cgd)
  if (dag) {
    if (mode == 0) FG_DH(1, 0); else if (mode == 1) FG_DH(1, 1); else FG_DH(1, 2);
  } else {
    if (mode == 0) FG_DH(0, 0); else if (mode == 1) FG_DH(0, 1); else FG_DH(0, 2);
  }
#undef FG_DH
  return cudaGetLastError();
}
template <int NC>
cudaError_t launch_dslash_h16(int s16, const GeomH& gh, void* out, const void* in, const void* x, const void* pdot,
                              const void* U, int out_par, int dag, int mode, double b, double* partial,
                              CgDev* cgd, cudaStream_t st) {
  return s16 == S16_BF16
             ? dslash16<BF16, NC>(gh, out, in, x, pdot, U, out_par, dag, mode, b, partial, cgd, st)
             : dslash16<Half16, NC>(gh, out, in, x, pdot, U, out_par, dag, mode, b, partial, cgd, st);
}
template cudaError_t launch_dslash_h16<9>(int, const GeomH&, void*, const void*, const void*, const void*,
                                          const void*, int, int, int, double, double*, CgDev*, cudaStream_t);
template cudaError_t launch_dslash_h16<6>(int, const GeomH&, void*, const void*, const void*, const void*,
                                          const void*, int, int, int, double, double*, CgDev*, cudaStream_t);
// Runs KERNEL<S> with the arguments that follow for the 16-bit format s16.
#define FG_S16(KERNEL, GRID, ...)                                                                              \
  do {                                                                                                         \
    if (s16 == S16_BF16) {                                                                                     \
      typedef Conv16<BF16>::T2 T2;                                                                             \
      KERNEL<BF16><<<GRID, kVecThreads, 0, st>>>(__VA_ARGS__);                                                 \
    } else {                                                                                                   \
      typedef Conv16<Half16>::T2 T2;                                                                           \
      KERNEL<Half16><<<GRID, kVecThreads, 0, st>>>(__VA_ARGS__);                                               \
    }                                                                                                          \
  } while (0)
cudaError_t launch_cg_axpy_h16(int s16, void* xs, void* r, const void* p, const void* ap, CgDev* cgd,
                               double* rr_part, int n, cudaStream_t st) {
  FG_S16(cg_axpy_h16_kernel, vec_blocks(n), (float2*)xs, (T2*)r, (const T2*)p, (const T2*)ap, cgd, rr_part, n);
  return cudaGetLastError();
}
cudaError_t launch_cg_xpay_h16(int s16, void* p, const void* r, CgDev* cgd, double* hist, int* iter_out,
                               int maxiter, int n, cudaStream_t st) {
  FG_S16(cg_xpay_h16_kernel, vec_blocks(n), (T2*)p, (const T2*)r, cgd, hist, iter_out, maxiter, n);
  return cudaGetLastError();
}
cudaError_t launch_cg_init_h16(const double* part, int nparts, CgDev* cgd, double tol2, double* bb_out, int n,
                               cudaStream_t st) {
  cg_init_h16_kernel<<<1, 256, 0, st>>>(part, nparts, cgd, tol2, bb_out, n);
  return cudaGetLastError();
}
cudaError_t launch_scale_to_h16(int s16, void* rs, const void* b64, const CgDev* cgd, int n, cudaStream_t st) {
  FG_S16(scale_to_h16_kernel, vec_blocks(n), (T2*)rs, (const double2*)b64, cgd, n);
  return cudaGetLastError();
}
cudaError_t launch_h16_to_double_scaled(int s16, void* dst64, const void* src16, const CgDev* cgd, int n,
                                        cudaStream_t st) {
  FG_S16(h16_to_double_scaled_kernel, vec_blocks(n), (double2*)dst64, (const T2*)src16, cgd, n);
  return cudaGetLastError();
}
cudaError_t launch_ru_accumulate_df_scaled(void* xdf, void* xs, const CgDev* cgd, int n, cudaStream_t st) {
  ru_accumulate_df_scaled_kernel<<<vec_blocks(n), kVecThreads, 0, st>>>((float4*)xdf, (float2*)xs, cgd, n);
  return cudaGetLastError();
}
cudaError_t launch_ru_residual_df_keep(const void* bdf, void* axdf, double* part, int n, cudaStream_t st) {
  ru_residual_df_keep_kernel<<<vec_blocks(n), kVecThreads, 0, st>>>((const float4*)bdf, (float4*)axdf, part, n);
  return cudaGetLastError();
}
cudaError_t launch_ru_residual64_keep(const void* b64, const void* ax64, void* r64, double* part, int n,
                                      cudaStream_t st) {
  ru_residual64_keep_kernel<<<vec_blocks(n), kVecThreads, 0, st>>>((const double2*)b64, (const double2*)ax64,
                                                                   (double2*)r64, part, n);
  return cudaGetLastError();
}
cudaError_t launch_ru_publish_h16(const double* part, int nparts, CgDev* cgd, double* true_rr, int n,
                                  cudaStream_t st) {
  ru_publish_h16_kernel<<<1, 256, 0, st>>>(part, nparts, cgd, true_rr, n);
  return cudaGetLastError();
}
cudaError_t launch_ru_rescale_df_h16(int s16, const void* rdf, void* rs, void* p, const CgDev* cgd, int n,
                                     cudaStream_t st) {
  if (s16 == S16_BF16)
    ru_rescale_h16_kernel<BF16, float4><<<vec_blocks(n), kVecThreads, 0, st>>>(
        (const float4*)rdf, (Conv16<BF16>::T2*)rs, (Conv16<BF16>::T2*)p, cgd, n);
  else
    ru_rescale_h16_kernel<Half16, float4><<<vec_blocks(n), kVecThreads, 0, st>>>(
        (const float4*)rdf, (Conv16<Half16>::T2*)rs, (Conv16<Half16>::T2*)p, cgd, n);
  return cudaGetLastError();
}
cudaError_t launch_ru_rescale64_h16(int s16, const void* r64, void* rs, void* p, const CgDev* cgd, int n,
                                    cudaStream_t st) {
  if (s16 == S16_BF16)
    ru_rescale_h16_kernel<BF16, double2><<<vec_blocks(n), kVecThreads, 0, st>>>(
        (const double2*)r64, (Conv16<BF16>::T2*)rs, (Conv16<BF16>::T2*)p, cgd, n);
  else
    ru_rescale_h16_kernel<Half16, double2><<<vec_blocks(n), kVecThreads, 0, st>>>(
        (const double2*)r64, (Conv16<Half16>::T2*)rs, (Conv16<Half16>::T2*)p, cgd, n);
  return cudaGetLastError();
}
#undef FG_S16
cudaError_t launch_dot64(const void* a, const void* b, double* part, int n, cudaStream_t st) {
  dot64_kernel<<<vec_blocks(n), kVecThreads, 0, st>>>((const double2*)a, (const double2*)b, part, n);
  return cudaGetLastError();
}
template <typename R>
cudaError_t launch_gaussian_spinor(void* chi, int Vh, uint64_t seed, uint32_t draw, cudaStream_t st) {
  gaussian_spinor_kernel<R><<<(Vh + 255) / 256, 256, 0, st>>>(v2<R>(chi), Vh, (uint32_t)seed,
                                                             (uint32_t)(seed >> 32), draw);
  return cudaGetLastError();
}
template <typename R>
cudaError_t launch_spinor_to_device(const double* canon, void* f, int Vh, cudaStream_t st) {
  spinor_to_device_kernel<R><<<(12 * Vh + 255) / 256, 256, 0, st>>>(canon, v2<R>(f), Vh);
  return cudaGetLastError();
}
template <typename R>
cudaError_t launch_spinor_to_canon(const void* f, double* canon, int Vh, cudaStream_t st) {
  spinor_to_canon_kernel<R><<<(12 * Vh + 255) / 256, 256, 0, st>>>(cv2<R>(f), canon, Vh);
  return cudaGetLastError();
}

#define FG_INST_F(RL, NC, RS)                                                                                  \
  template cudaError_t launch_dslash<RL, NC, RS>(const GeomH&, void*, const void*, const void*, const void*,  \
                                                 const void*, int, int, int, double, double*, CgDev*,        \
                                                 cudaStream_t);                                               \
  template cudaError_t launch_fermion_force<RL, NC, RS>(const GeomH&, const void*, const void*, const void*,  \
                                                        const void*, const void*, void*, double, int,         \
                                                        cudaStream_t);
FG_INST_F(double, 9, double)
FG_INST_F(double, 6, double)
FG_INST_F(float, 9, float)
FG_INST_F(float, 6, float)
FG_INST_F(float, 9, double)
FG_INST_F(float, 6, double)
template cudaError_t launch_dslash<Half16, 9, float>(const GeomH&, void*, const void*, const void*,
                                                     const void*, const void*, int, int, int, double, double*,
                                                     CgDev*, cudaStream_t);
template cudaError_t launch_dslash<Half16, 6, float>(const GeomH&, void*, const void*, const void*,
                                                     const void*, const void*, int, int, int, double, double*,
                                                     CgDev*, cudaStream_t);

template <typename S, int NC>
__global__ void __launch_bounds__(256) links_to_half_kernel(Gauge<float, NC> in, Gauge<S, NC> out, int V) {
  const int s = blockIdx.x * 64 + threadIdx.x;
  const int mu = threadIdx.y;
  if (s >= V) return;
  out.store(mu, s, in.load(mu, s));
}
template <int NC>
cudaError_t launch_links_to_half(int s16, const GeomH& gh, const void* U32, void* U16, cudaStream_t st) {
  Gauge<float, NC> a;
  a.p = const_cast<void*>(U32);
  a.V = gh.V;
  if (s16 == S16_BF16) {
    Gauge<BF16, NC> b;
    b.p = U16;
    b.V = gh.V;
    links_to_half_kernel<BF16, NC><<<(gh.V + 63) / 64, dim3(64, 4), 0, st>>>(a, b, gh.V);
  } else {
    Gauge<Half16, NC> b;
    b.p = U16;
    b.V = gh.V;
    links_to_half_kernel<Half16, NC><<<(gh.V + 63) / 64, dim3(64, 4), 0, st>>>(a, b, gh.V);
  }
  return cudaGetLastError();
}
template cudaError_t launch_links_to_half<9>(int, const GeomH&, const void*, void*, cudaStream_t);
template cudaError_t launch_links_to_half<6>(int, const GeomH&, const void*, void*, cudaStream_t);

template cudaError_t launch_dslash<float, 9, DF>(const GeomH&, void*, const void*, const void*, const void*,
                                                 const void*, int, int, int, double, double*, CgDev*, cudaStream_t);
template cudaError_t launch_dslash<float, 6, DF>(const GeomH&, void*, const void*, const void*, const void*,
                                                 const void*, int, int, int, double, double*, CgDev*, cudaStream_t);

template cudaError_t launch_cg_axpy<double>(void*, void*, const void*, const void*, CgDev*, double*, int,
                                            cudaStream_t);
template cudaError_t launch_cg_axpy<float>(void*, void*, const void*, const void*, CgDev*, double*, int,
                                           cudaStream_t);
template cudaError_t launch_cg_xpay<double>(void*, const void*, CgDev*, double*, int*, int, int, cudaStream_t);
template cudaError_t launch_cg_xpay<float>(void*, const void*, CgDev*, double*, int*, int, int, cudaStream_t);
#define FG_INST_FOLD(R, NC)                                                                                    \
  template cudaError_t launch_cg_apdot<R, NC>(const GeomH&, void*, const void*, const void*, const void*,      \
                                              const void*, const void*, double, double*, CgDev*, cudaStream_t); \
  template cudaError_t launch_cg_fold<R, NC>(const GeomH&, void*, void*, const void*, const void*, const void*, \
                                             void*, void*, const void*, double*, CgDev*, double*, int*, int,    \
                                             cudaStream_t);
FG_INST_FOLD(float, 9)
FG_INST_FOLD(float, 6)
FG_INST_FOLD(double, 9)
FG_INST_FOLD(double, 6)
#undef FG_INST_FOLD
template cudaError_t launch_cg_restart<double>(void*, const void*, const CgDev*, int, cudaStream_t);
template cudaError_t launch_cg_restart<float>(void*, const void*, const CgDev*, int, cudaStream_t);
template cudaError_t launch_ru_accumulate<double>(void*, void*, int, cudaStream_t);
template cudaError_t launch_ru_accumulate<float>(void*, void*, int, cudaStream_t);
template cudaError_t launch_ru_residual<double>(const void*, const void*, void*, void*, double*, int, cudaStream_t);
template cudaError_t launch_ru_residual<float>(const void*, const void*, void*, void*, double*, int, cudaStream_t);
template cudaError_t launch_convert<double, double>(void*, const void*, double*, int, cudaStream_t);
template cudaError_t launch_convert<float, double>(void*, const void*, double*, int, cudaStream_t);
template cudaError_t launch_convert<double, float>(void*, const void*, double*, int, cudaStream_t);
template cudaError_t launch_convert<float, float>(void*, const void*, double*, int, cudaStream_t);
template cudaError_t launch_gaussian_spinor<double>(void*, int, uint64_t, uint32_t, cudaStream_t);
template cudaError_t launch_gaussian_spinor<float>(void*, int, uint64_t, uint32_t, cudaStream_t);
template cudaError_t launch_spinor_to_device<double>(const double*, void*, int, cudaStream_t);
template cudaError_t launch_spinor_to_device<float>(const double*, void*, int, cudaStream_t);
template cudaError_t launch_spinor_to_canon<double>(const void*, double*, int, cudaStream_t);
template cudaError_t launch_spinor_to_canon<float>(const void*, double*, int, cudaStream_t);

}  // namespace fg
