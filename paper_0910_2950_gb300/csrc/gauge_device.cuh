// Per-link and per-site device functions of the pure-gauge step, shared by
// the single-lattice kernels (gauge.cu) and the multi-chain kernels
// (batch.cu), so that a chain in a batch runs the same arithmetic.
#pragma once

#include <type_traits>

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

// Product of two special unitary matrices (a link and a link, or exp(iA)
// and a link): the anchored products for double-float links.
template <typename R>
__device__ __forceinline__ M3<R> link_mul(const M3<R>& a, const M3<R>& b) {
  if constexpr (std::is_same<R, DF>::value) return su3_mul(a, b);
  else return mul(a, b);
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
    if constexpr (std::is_same<R, DF>::value) {
      // Double-float: every staple is a product of links, hence unitary, so
      // the anchored products (df64.cuh) apply.  Both staples of the plane
      // are written as X Y^dag Z with run-time daggers,
      //   upper  U_nu(x+mu)          U_mu(x+nu)^dag U_nu(x)^dag,
      //   lower  U_nu(x+mu-nu)^dag   U_mu(x-nu)^dag U_nu(x-nu),
      // and the two products of each run through one loop body: unrolled,
      // the double-float code of four products per plane overflowed the
      // instruction cache (most issue stalls were instruction fetch).
      const int s_mnu = other + dm;
#pragma unroll 1
      for (int up = 1; up >= 0; --up) {
        M3<DF> l = dagger_if(U.load(nu, up ? s_pmu : s + dm + dmu), !up);
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {
          // Y^dag = U_mu(x+nu)^dag or U_mu(x-nu)^dag, then Z
          const int sr = q ? (up ? s : s_mnu) : (up ? other + dp : s_mnu);
          l = su3_mul(l, dagger_if(U.load(q ? nu : mu, sr), q ? up != 0 : true));
        }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) a.e[i][j] = a.e[i][j] + l.e[i][j];
      }
    } else {
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
  }
  return a;
}

// Everything after the staple sum a of U_mu(x): the force, then what MODE
// does with it on this link.
template <typename R, int NC, int MODE>
__device__ __forceinline__ void force_finish(const Gauge<R, NC>& U, const Mom<R>& P, const Mom<R>& F,
                                             const Mom<R>& FF, const Gauge<R, NC>& Ubase,
                                             const Gauge<R, NC>& Uout, int s, int mu, const M3<R>& a, R beta6,
                                             R ckick, R cdrift, R cdisp, int reunit, R ffw) {
  const M3<R> ul = U.load(mu, s);
  R f[8];
  if constexpr (std::is_same<R, DF>::value) {
    // a is a sum of six unitary staples, so a / 8 has columns of norm <= 3/4
    // and U (a / 8) is within the anchored products' bounds; scaling by a
    // power of two is exact
    M3<DF> a8;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
        a8.e[i][j] = cx<DF>(DF(a.e[i][j].re.hi * 0.125f, a.e[i][j].re.lo * 0.125f),
                            DF(a.e[i][j].im.hi * 0.125f, a.e[i][j].im.lo * 0.125f));
    im_tr_gellmann(su3_mul(ul, a8), f);
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] = (f[k] * 8.0f) * beta6;
  } else {
    const M3<R> omega = mul(ul, a);
    im_tr_gellmann(omega, f);
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] *= beta6;
  }
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
      M3<R> un = link_mul(e, ub);
      if (reunit) reunitarize(un);
      Uout.store(mu, s, un);
    }
  } else {  // FM_DISPLACE
    // The displaced links only serve one force evaluation and are then
    // dropped, so they are not re-projected.  (FP32 exp(i A) U comes out
    // short of unitary by ~7e-9 of |U|^2 on average, but re-projecting the
    // displaced FP32 links as the drifted ones are raised the FP32 dH error
    // of a 24^4 trajectory from 2.5e-2 to 3.4e-2: the projection's own
    // rounding is not of random sign either.)
    (void)reunit;
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] *= -cdisp;
    const M3<R> e = expi_herm(alg_to_mat(f));
    Uout.store(mu, s, link_mul(e, ul));
  }
}

template <typename R, int NC, int MODE>
__device__ __forceinline__ void force_link(const Gauge<R, NC>& U, const Mom<R>& P, const Mom<R>& F,
                                           const Mom<R>& FF, const Gauge<R, NC>& Ubase,
                                           const Gauge<R, NC>& Uout, const Geom& g, const int c[4], int s,
                                           int mu, R beta6, R ckick, R cdrift, R cdisp, int reunit,
                                           R ffw = R(1)) {
  const M3<R> a = staple_sum(U, g, c, s, mu);
  force_finish<R, NC, MODE>(U, P, F, FF, Ubase, Uout, s, mu, a, beta6, ckick, cdrift, cdisp, reunit, ffw);
}

// Whether the FP32 12-real force kernels share the upper-staple products of
// a plane between its two links through shared memory (below).  With 12-real
// links every load rebuilds a row, and the two loads a shared product saves
// pay for the barrier and the shared memory: 418 vs 437 us per launch at
// 32^4.  With 18-real links the same change executed 8% fewer instructions
// but ran 2% slower (426 vs 416 us; the slots take L1 capacity from the
// neighbour loads and the barrier stalls), and the FP64 kernels would need
// 55 KB of slots per block; those compute every staple in full.
#ifndef FG_FORCE_SHARED_T
#define FG_FORCE_SHARED_T 1
#endif
// Resident blocks per SM of the sharing kernel (its register cap) and its
// preferred shared-memory carveout in percent of the SM's maximum (44%: the
// 100 KB configuration, room for three blocks of 64 sites).
#ifndef FG_FORCE_SHARED_MIN_BLOCKS
#define FG_FORCE_SHARED_MIN_BLOCKS 3
#endif
#ifndef FG_FORCE_CARVEOUT
#define FG_FORCE_CARVEOUT 44
#endif

// Upper staples of the plane (mu, nu) at x, for its two links: with
// T_{mu,nu} = U_nu(x+mu) U_mu(x+nu)^dag, the upper staple of U_mu(x) is
// T U_nu(x)^dag and that of U_nu(x) is U_mu(x+nu) U_nu(x+mu)^dag U_mu(x)^dag
// = T^dag U_mu(x)^dag = (U_mu(x) T)^dag.  The four direction threads of a
// site are in one block: thread mu computes T_{mu,mu+1} and, for mu < 2,
// T_{mu,mu+2} (6 products per site, 1 or 2 per thread), keeps its own term
// and leaves T in shared memory; after a barrier the other thread of each
// plane reads it.  A site's four links then take 46 3x3 products instead of
// 52 and two fewer link loads per shared plane.  Slots: T_{mu,mu+1} in mu,
// T_{mu,mu+2} in 4 + mu; entries as (re, im) pairs, site-minor.
// The block is NS sites (threadIdx.x) x 4 directions (threadIdx.y); tsh has
// room for the six slots of its NS sites.  Every thread of the block must
// call this (it holds a barrier); ok = false threads only take part in the
// barrier.  The caller separates two calls on the same tsh by a barrier.
template <typename R, int NC>
constexpr bool kForceSharedT = FG_FORCE_SHARED_T && std::is_same<R, float>::value && NC == 6;
#ifndef FG_FORCE_DF_MIN_BLOCKS
#define FG_FORCE_DF_MIN_BLOCKS 2
#endif
// Double-float links need about twice the registers of FP32 ones.  With the
// exponential in a launch of its own the force launch fits two blocks of
// 256 threads per SM (128 registers a thread): 2-3% faster than one block
// with up to 255 registers (32^4 trajectory 34.7 against 35.5 ms, 64-chain
// batch 39.7 against 40.5 ms).
template <typename R, int NC>
constexpr int kForceMinBlocks = std::is_same<R, DF>::value
                                    ? FG_FORCE_DF_MIN_BLOCKS
                                    : (kForceSharedT<R, NC> ? FG_FORCE_SHARED_MIN_BLOCKS : FG_FORCE_MIN_BLOCKS);

template <int NC, int MODE, int NS>
__device__ __forceinline__ void force_link_shared(float2 (*tsh)[9][NS], bool ok, int s, const Gauge<float, NC>& U,
                                                  const Mom<float>& P, const Mom<float>& F, const Mom<float>& FF,
                                                  const Gauge<float, NC>& Ubase, const Gauge<float, NC>& Uout,
                                                  const Geom& g, float beta6, float ckick, float cdrift,
                                                  float cdisp, int reunit, float ffw) {
  const int x = threadIdx.x;
  const int mu = threadIdx.y;
  M3<float> a;
  zero(a);
  int c[4], par;
  if (ok) {
    cb_coords(g, s, c, par);
    const int other = s + (par ? -g.Vh : g.Vh);
    int dmu, dmu_m;
    cb_half_steps(g, c, mu, dmu, dmu_m);
    (void)dmu_m;
    const int s_pmu = other + dmu;
#pragma unroll 1
    for (int k = 1; k < 4; ++k) {
      const int nu = (mu + k) & 3;
      int dp, dm;
      cb_half_steps(g, c, nu, dp, dm);
      if (k == 1 || (k == 2 && mu < 2)) {
        const M3<float> t = mul_nd(U.load(nu, s_pmu), U.load(mu, other + dp));
        const int slot = k == 1 ? mu : 4 + mu;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) tsh[slot][3 * i + j][x] = make_float2(t.e[i][j].re, t.e[i][j].im);
        mac_nd(a, t, U.load(nu, s));
      }
      {
        // lower: (U_mu(x-nu) U_nu(x+mu-nu))^dag U_nu(x-nu)
        const int s_mnu = other + dm;
        const M3<float> t = mul(U.load(mu, s_mnu), U.load(nu, s + dm + dmu));
        mac_dn(a, t, U.load(nu, s_mnu));
      }
    }
  }
  __syncthreads();
  if (!ok) return;
  // planes whose T the other thread left: p = mu - 1 (slot p) and, for
  // mu >= 2, p = mu - 2 (slot 4 + p); add (U_p(x) T_{p,mu})^dag
#pragma unroll 1
  for (int r = 0; r < 2; ++r) {
    if (r == 1 && mu < 2) break;
    const int p = r == 0 ? ((mu + 3) & 3) : mu - 2;
    const int slot = r == 0 ? p : 4 + p;
    M3<float> t;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const float2 v = tsh[slot][3 * i + j][x];
        t.e[i][j] = cx<float>(v.x, v.y);
      }
    const M3<float> up = U.load(p, s);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        // a_ij += conj((U_p T)_ji)
        Cx<float> acc = conj(a.e[i][j]);
        cmac(acc, up.e[j][0], t.e[0][i]);
        cmac(acc, up.e[j][1], t.e[1][i]);
        cmac(acc, up.e[j][2], t.e[2][i]);
        a.e[i][j] = conj(acc);
      }
  }
  force_finish<float, NC, MODE>(U, P, F, FF, Ubase, Uout, s, mu, a, beta6, ckick, cdrift, cdisp, reunit, ffw);
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
  M3<R> un = link_mul(e, Uin.load(mu, s));
  if (reunit) reunitarize(un);
  Uout.store(mu, s, un);
}

// Per-site energy h(x) = T(x) + S_G(x) (T = 0 if P is null), with
// S_G(x) = sum_{mu<nu} beta (1 - Re Tr P_mu,nu(x) / 3) = beta6 - beta3 sum Re Tr
// (beta6 = 6 beta, beta3 = beta / 3): v[0] = S_G(x), v[1] = T(x); mode 0
// stores h0[s] = h(x), mode 1 sets v[2] = h(x) - h0[s].  If sg_in is given,
// S_G(x) is read from it instead of recomputed (the links have not changed
// since it was stored); if sg_out is given, S_G(x) is stored.  A is the type
// of the per-site values: double, or DF for FP32 and double-float fields,
// which keeps FP64 arithmetic (1/64 of the FP32 rate on GB300) out of the
// kernel.  Sums of FP32 terms are double-float in either case (each p^2
// split exactly by an FMA, each plaquette trace added with two_sum);
// double-float fields compute and sum in double-float, FP64 fields in FP64.
template <typename A> __device__ __forceinline__ A acc_of(DF x);
template <> __device__ __forceinline__ DF acc_of<DF>(DF x) { return x; }
template <> __device__ __forceinline__ double acc_of<double>(DF x) { return double(x); }

template <typename R, int NC, typename A>
__device__ __forceinline__ void site_energy(const Gauge<R, NC>& U, const Mom<R>& P, const Geom& g, int s,
                                            A beta6, A beta3, int mode, A* __restrict__ h0, A v[3],
                                            const A* __restrict__ sg_in = nullptr, A* __restrict__ sg_out = nullptr) {
  constexpr bool kDF = std::is_same<R, float>::value;
  constexpr bool kDD = std::is_same<R, DF>::value;
  static_assert(kDF || kDD || std::is_same<A, double>::value, "FP64 fields keep FP64 per-site values");
  A t = A(0);
  if (P.p != nullptr) {
    DF tdf(0.0f);
    double t64 = 0.0;
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
      R p[8];
      P.load(mu, s, p);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if constexpr (kDF) {
          const float sq = __fmul_rn(p[k], p[k]);
          tdf = tdf + DF(sq, __fmaf_rn(p[k], p[k], -sq));
        } else if constexpr (kDD) {
          tdf = fma(p[k], p[k], tdf);
        } else {
          t64 += double(p[k]) * double(p[k]);
        }
      }
    }
    if constexpr (kDF || kDD) t = acc_of<A>(tdf) * A(0.5f);
    else t = A(0.5 * t64);
  }
  A sg;
  if (sg_in != nullptr) {
    sg = sg_in[s];
  } else {
    int c[4], par;
    cb_coords(g, s, c, par);
    // x + mu as a half-index step from s (see staple_sum)
    const int other = s + (par ? -g.Vh : g.Vh);
    int dp[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      int dm;
      cb_half_steps(g, c, mu, dp[mu], dm);
      (void)dm;
    }
    DF trdf(0.0f);
    double tr64 = 0.0;
    if constexpr (kDD) {
      // double-float links: the plaquette's two products by the anchored
      // products, one copy of the code for the six planes (x, y, z, t as
      // mu, nu with mu < nu; the planes' half-index steps by selects)
#pragma unroll 1
      for (int pl = 0; pl < 6; ++pl) {
        const int mu = pl < 3 ? 0 : (pl < 5 ? 1 : 2);
        const int nu = pl < 3 ? pl + 1 : (pl < 5 ? pl - 1 : 3);
        const int dmu = sel4(dp, mu), dnu = sel4(dp, nu);
        M3<DF> pr[2];
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {
          // U_mu(x) U_nu(x+mu), then U_nu(x) U_mu(x+nu)
          const M3<DF> l = U.load(q ? nu : mu, s);
          const M3<DF> r = U.load(q ? mu : nu, other + (q ? dnu : dmu));
          const M3<DF> m = su3_mul(l, r);
          if (q) pr[1] = m;
          else pr[0] = m;
        }
        trdf = trdf + re_tr_mul_nd(pr[0], pr[1]);
      }
    } else {
#pragma unroll
      for (int mu = 0; mu < 4; ++mu) {
        const M3<R> umu = U.load(mu, s);
#pragma unroll
        for (int nu = mu + 1; nu < 4; ++nu) {
          const M3<R> a = mul(umu, U.load(nu, other + dp[mu]));
          const M3<R> b = mul(U.load(nu, s), U.load(mu, other + dp[nu]));
          if constexpr (kDF) trdf = trdf + DF(float(re_tr_mul_nd(a, b)));
          else tr64 += double(re_tr_mul_nd(a, b));
        }
      }
    }
    if constexpr (kDF || kDD) sg = beta6 - beta3 * acc_of<A>(trdf);
    else sg = beta6 - beta3 * A(tr64);
  }
  if (sg_out != nullptr) sg_out[s] = sg;
  v[0] = sg;
  v[1] = t;
  const A h = sg + t;
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

// Double-float fields take FP32 draws: the Gaussian deviates need no more
// than FP32 resolution, and every later use of them (kinetic term, MD) is
// exact to double-float rounding for whatever value was drawn.
template <>
__device__ __forceinline__ void box_muller<DF>(uint32_t a, uint32_t b, DF& z0, DF& z1) {
  float x0, x1;
  box_muller<float>(a, b, x0, x1);
  z0 = DF(x0);
  z1 = DF(x1);
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
