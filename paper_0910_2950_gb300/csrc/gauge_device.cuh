// Per-link and per-site device functions of the pure-gauge step, shared by
// the single-lattice kernels (gauge.cu) and the multi-chain kernels
// (batch.cu), so that a chain in a batch runs the same arithmetic.
#pragma once

#include "df64.cuh"
#include "fg_common.cuh"
#include "fg_kernels.h"

namespace fg {

// Tuning knobs of the gauge-force kernel: minimum resident blocks of 256
// threads per SM (register cap) and whether the loop over the three staple
// directions is unrolled.
#ifndef FG_FORCE_MIN_BLOCKS
#define FG_FORCE_MIN_BLOCKS 2
#endif
#ifndef FG_FORCE_UNROLL_NU
#define FG_FORCE_UNROLL_NU 0
#endif

// Sum of the six staples that close a plaquette with U_mu(x).  Neighbour
// indices are formed with selects, so mu and nu may be run-time values
// without the coordinate array going to local memory; one copy of the body
// keeps the kernel small enough for the instruction cache.
// Changes dp, dm of the half index lex/2 when coordinate nu of c moves by
// +1 and -1 (periodic); the parity flips.  Only that coordinate moves, so the change
// is (v>>1) - (c>>1) in x and (v - c) times the half stride of nu otherwise,
// and the changes of two steps in different directions add.
__device__ __forceinline__ void cb_half_steps(const Geom& g, const int c[4], int nu, int& dp, int& dm) {
  const int cn = sel4(c, nu);
  const int ln = nu == 0 ? g.L[0] : (nu == 1 ? g.L[1] : (nu == 2 ? g.L[2] : g.L[3]));
  const int vp = cn + 1 == ln ? 0 : cn + 1;
  const int vm = cn == 0 ? ln - 1 : cn - 1;
  if (nu == 0) {
    dp = (vp >> 1) - (cn >> 1);
    dm = (vm >> 1) - (cn >> 1);
  } else {
    const int hs = nu == 1 ? g.Lxh : (nu == 2 ? g.Lxh * g.L[1] : g.Lxh * g.L[1] * g.L[2]);
    dp = (vp - cn) * hs;
    dm = (vm - cn) * hs;
  }
}

template <typename R, int NC>
__device__ __forceinline__ M3<R> staple_sum(const Gauge<R, NC>& U, const Geom& g, const int c[4], int s, int mu) {
  M3<R> a;
  zero(a);
  // neighbours as half-index steps from s: x + mu, x +- nu flip the parity,
  // x + mu - nu keeps it
  const int par = s >= g.Vh;
  const int other = s + (par ? -g.Vh : g.Vh);
  int dmu, dmu_m;
  cb_half_steps(g, c, mu, dmu, dmu_m);
  (void)dmu_m;
  const int s_pmu = other + dmu;
#if FG_FORCE_UNROLL_NU
#pragma unroll
#else
#pragma unroll 1
#endif
  for (int k = 1; k < 4; ++k) {
    const int nu = (mu + k) & 3;
    int dp, dm;
    cb_half_steps(g, c, nu, dp, dm);
    {
      // upper: U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
      const M3<R> t = mul_nd(U.load(nu, s_pmu), U.load(mu, other + dp));
      mac_nd(a, t, U.load(nu, s));
    }
    {
      // lower: U_nu(x+mu-nu)^dag U_mu(x-nu)^dag U_nu(x-nu) = (U_mu(x-nu) U_nu(x+mu-nu))^dag U_nu(x-nu)
      const int s_mnu = other + dm;
      const M3<R> t = mul(U.load(mu, s_mnu), U.load(nu, s + dm + dmu));
      mac_dn(a, t, U.load(nu, s_mnu));
    }
  }
  return a;
}

template <typename R, int NC, int MODE>
__device__ __forceinline__ void force_link(const Gauge<R, NC>& U, const Mom<R>& P, const Mom<R>& F,
                                           const Mom<R>& FF, const Gauge<R, NC>& Ubase,
                                           const Gauge<R, NC>& Uout, const Geom& g, const int c[4], int s,
                                           int mu, R beta6, R ckick, R cdrift, R cdisp, int reunit,
                                           R ffw = R(1)) {
  const M3<R> a = staple_sum(U, g, c, s, mu);
  const M3<R> ul = U.load(mu, s);
  const M3<R> omega = mul(ul, a);
  R f[8];
  im_tr_gellmann(omega, f);
#pragma unroll
  for (int k = 0; k < 8; ++k) f[k] *= beta6;
  if (FF.p != nullptr) {
    R ff[8];
    FF.load(mu, s, ff);
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] = fma(ffw, ff[k], f[k]);
  }
  if (MODE == FM_STORE) {
    F.store(mu, s, f);
  } else if (MODE == FM_KICK || MODE == FM_KICK_DRIFT) {
    R p[8];
    P.load(mu, s, p);
#pragma unroll
    for (int k = 0; k < 8; ++k) p[k] = fma(-ckick, f[k], p[k]);
    P.store(mu, s, p);
    if (MODE == FM_KICK_DRIFT) {
#pragma unroll
      for (int k = 0; k < 8; ++k) p[k] *= cdrift;
      const M3<R> e = expi_herm(alg_to_mat(p));
      const M3<R> ub = (Ubase.p == U.p) ? ul : Ubase.load(mu, s);
      M3<R> un = mul(e, ub);
      if (reunit) reunitarize(un);
      Uout.store(mu, s, un);
    }
  } else {  // FM_DISPLACE
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] *= -cdisp;
    const M3<R> e = expi_herm(alg_to_mat(f));
    M3<R> un = mul(e, ul);
    if (reunit) reunitarize(un);
    Uout.store(mu, s, un);
  }
}

// U_out(s, mu) = exp(i c P) U_in(s, mu), the exact T-hat flow of section 2.
template <typename R, int NC>
__device__ __forceinline__ void drift_link(const Gauge<R, NC>& Uin, const Mom<R>& P, const Gauge<R, NC>& Uout,
                                           int s, int mu, R c, int reunit) {
  R p[8];
  P.load(mu, s, p);
#pragma unroll
  for (int k = 0; k < 8; ++k) p[k] *= c;
  const M3<R> e = expi_herm(alg_to_mat(p));
  M3<R> un = mul(e, Uin.load(mu, s));
  if (reunit) reunitarize(un);
  Uout.store(mu, s, un);
}

// Per-site energy h(x) = T(x) + S_G(x) in FP64 (T = 0 if P is null): v[0] = S_G(x),
// v[1] = T(x); mode 0 stores h0[s] = h(x), mode 1 sets v[2] = h(x) - h0[s].
// If sg_in is given, S_G(x) is read from it instead of recomputed (the links
// have not changed since it was stored); if sg_out is given, S_G(x) is stored.
template <typename R, int NC>
__device__ __forceinline__ void site_energy(const Gauge<R, NC>& U, const Mom<R>& P, const Geom& g, int s,
                                            double beta, int mode, double* __restrict__ h0, double v[3],
                                            const double* __restrict__ sg_in = nullptr,
                                            double* __restrict__ sg_out = nullptr) {
  int c[4], par;
  cb_coords(g, s, c, par);
  // Sums of FP32 terms are taken in double-float (each p^2 split exactly by
  // an FMA, each plaquette trace added with two_sum): as accurate as FP64
  // sums to ~1e-14 relative, without GB300's slow FP64 unit; FP64 fields
  // keep FP64 sums.
  constexpr bool kDF = sizeof(R) == sizeof(float);
  double t = 0.0;
  if (P.p != nullptr) {
    DF tdf(0.0f);
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
      R p[8];
      P.load(mu, s, p);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if constexpr (kDF) {
          const float sq = __fmul_rn(p[k], p[k]);
          tdf = tdf + DF(sq, __fmaf_rn(p[k], p[k], -sq));
        } else {
          t += double(p[k]) * double(p[k]);
        }
      }
    }
    if constexpr (kDF) t = double(tdf);
    t *= 0.5;
  }
  double sg = 0.0;
  if (sg_in != nullptr) {
    sg = sg_in[s];
  } else {
    DF trdf(0.0f);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const M3<R> umu = U.load(mu, s);
#pragma unroll
      for (int nu = mu + 1; nu < 4; ++nu) {
        const M3<R> a = mul(umu, U.load(nu, cb_neighbor(g, c, mu, +1)));
        const M3<R> b = mul(U.load(nu, s), U.load(mu, cb_neighbor(g, c, nu, +1)));
        if constexpr (kDF) trdf = trdf + DF(float(re_tr_mul_nd(a, b)));
        else sg += 1.0 - double(re_tr_mul_nd(a, b)) * (1.0 / 3.0);
      }
    }
    if constexpr (kDF) sg = 6.0 - double(trdf) * (1.0 / 3.0);
    sg *= beta;
  }
  if (sg_out != nullptr) sg_out[s] = sg;
  v[0] = sg;
  v[1] = t;
  const double h = sg + t;
  if (mode == 0) h0[s] = h;
  else if (mode == 1) v[2] = h - h0[s];
}

// Box-Muller on two 32-bit uniforms, u1 in (0, 1], u2 in [0, 1), evaluated
// in the precision of the momenta (GB300's FP64 unit is slow, and FP32
// momenta cannot hold more than an FP32 draw).
template <typename R>
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, R& z0, R& z1) {
  const R u1 = (R(a) + R(1)) * R(2.3283064365386963e-10);
  const R u2 = R(b) * R(2.3283064365386963e-10);
  const R r = sqrt(R(-2) * log(u1));
  R sn, cs;
  sincospi(R(2) * u2, &sn, &cs);
  z0 = r * cs;
  z1 = r * sn;
}

// Unit-Gaussian momenta of link (s, mu): two Philox-4x32-10 draws with
// counter (4 lex + mu, draw, stream, half); stream 0 = one lattice,
// stream 3 + chain for the chains of a batch.
template <typename R>
__device__ __forceinline__ void refresh_link(const Mom<R>& P, const Geom& g, int s, int mu, uint32_t k0, uint32_t k1,
                                             uint32_t draw, uint32_t stream) {
  int c[4], par;
  cb_coords(g, s, c, par);
  const uint32_t lex = (uint32_t)(c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3])));
  R p[8];
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    uint32_t ctr[4] = {lex * 4u + (uint32_t)mu, draw, stream, (uint32_t)half};
    Philox::rounds(ctr, k0, k1);
    box_muller<R>(ctr[0], ctr[1], p[4 * half + 0], p[4 * half + 1]);
    box_muller<R>(ctr[2], ctr[3], p[4 * half + 2], p[4 * half + 3]);
  }
  P.store(mu, s, p);
}

}  // namespace fg
