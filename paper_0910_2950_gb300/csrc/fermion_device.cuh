// Device building blocks of the Wilson hopping term (section 4's even-odd
// operator Mhat = 1 - kappa^2 D_eo D_oe): spinor storage access, the spin
// projections of (1 -+ g_mu), the colour products and the four-direction
// hop sum, in FP32, FP64, double-float and half-precision storage.
#pragma once
#include "df64.cuh"
#include "fg_common.cuh"
#include "fg_fermion.h"

namespace fg {

static inline Geom to_devg(const GeomH& h) {
  Geom g;
  for (int i = 0; i < 4; ++i) g.L[i] = h.L[i];
  g.Lxh = h.Lxh; g.Vh = h.Vh; g.V = h.V;
  g.dLxh = make_fastdiv((uint32_t)h.Lxh);
  g.dLy = make_fastdiv((uint32_t)h.L[1]);
  g.dLz = make_fastdiv((uint32_t)h.L[2]);
  return g;
}

template <typename R> struct Spinor {
  Cx<R> s[4][3];
};

// Spinor entry k = spin * 3 + colour sits in pair k / 2, slot k % 2.  ST is
// the storage type (the arithmetic type R, or Half16 for R = float).
template <typename R, typename ST = R>
__device__ __forceinline__ Spinor<R> load_spinor(const typename Vec2<ST>::T* __restrict__ f, int i, int Vh) {
  Spinor<R> x;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    Cx<R> a, b;
    Quad<ST>::load(f, (size_t)q * Vh + i, a, b);
    x.s[(2 * q) / 3][(2 * q) % 3] = a;
    x.s[(2 * q + 1) / 3][(2 * q + 1) % 3] = b;
  }
  return x;
}
template <typename R, typename ST = R>
__device__ __forceinline__ void store_spinor(typename Vec2<ST>::T* __restrict__ f, int i, int Vh,
                                             const Spinor<R>& x) {
#pragma unroll
  for (int q = 0; q < 6; ++q)
    Quad<ST>::store(f, (size_t)q * Vh + i, x.s[(2 * q) / 3][(2 * q) % 3], x.s[(2 * q + 1) / 3][(2 * q + 1) % 3]);
}

template <typename RO, typename RI>
__device__ __forceinline__ M3<RO> convert(const M3<RI>& m) {
  M3<RO> o;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) o.e[i][j] = cx<RO>(RO(m.e[i][j].re), RO(m.e[i][j].im));
  return o;
}

// h_k = psi_k - S (A_mu psi_down)_k, k = 0, 1
template <int MU, int S, typename R>
__device__ __forceinline__ void project(const Spinor<R>& p, Cx<R> h[2][3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Cx<R> a0, a1;  // (A_mu psi_down)_0, _1
    if (MU == 0) { a0 = times_i(p.s[3][c]); a1 = times_i(p.s[2][c]); }
    if (MU == 1) { a0 = cx<R>(-p.s[3][c].re, -p.s[3][c].im); a1 = p.s[2][c]; }
    if (MU == 2) { a0 = times_i(p.s[2][c]); a1 = cx<R>(p.s[3][c].im, -p.s[3][c].re); }
    if (MU == 3) { a0 = p.s[2][c]; a1 = p.s[3][c]; }
    if (S > 0) { h[0][c] = p.s[0][c] - a0; h[1][c] = p.s[1][c] - a1; }
    else { h[0][c] = p.s[0][c] + a0; h[1][c] = p.s[1][c] + a1; }
  }
}

// (b0, b1) = A_mu^dagger (w0, w1)
template <int MU, typename R>
__device__ __forceinline__ void adag_mu(const Cx<R>& w0, const Cx<R>& w1, Cx<R>& b0, Cx<R>& b1) {
  if (MU == 0) { b0 = cx<R>(w1.im, -w1.re); b1 = cx<R>(w0.im, -w0.re); }
  if (MU == 1) { b0 = w1; b1 = cx<R>(-w0.re, -w0.im); }
  if (MU == 2) { b0 = cx<R>(w0.im, -w0.re); b1 = times_i(w1); }
  if (MU == 3) { b0 = w0; b1 = w1; }
}

// acc_up += sign * w, acc_down += sign * (-S) A_mu^dagger w
template <int MU, int S, typename R>
__device__ __forceinline__ void reconstruct_add(Spinor<R>& acc, const Cx<R> w[2][3], R sign) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Cx<R> b0, b1;
    adag_mu<MU>(w[0][c], w[1][c], b0, b1);
    const R sd = (S > 0) ? -sign : sign;
    acc.s[0][c] = acc.s[0][c] + sign * w[0][c];
    acc.s[1][c] = acc.s[1][c] + sign * w[1][c];
    acc.s[2][c] = acc.s[2][c] + sd * b0;
    acc.s[3][c] = acc.s[3][c] + sd * b1;
  }
}

// w = U h (ADJ = 0) or U^dagger h (ADJ = 1), for both half-spinor rows
template <int ADJ, typename R>
__device__ __forceinline__ void mat_half(const M3<R>& u, const Cx<R> h[2][3], Cx<R> w[2][3]) {
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Cx<R> s = cx<R>(0, 0);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (ADJ) cmac_cj(s, u.e[b][a], h[k][b]);
        else cmac(s, u.e[a][b], h[k][b]);
      }
      w[k][a] = s;
    }
}

// Double-float versions of the two inner steps.  The links are FP32, so a
// product of a double-float half-spinor entry h and a link entry u is the
// exact pair (fl(h.hi u), its error) plus h.lo u; the six products of each
// output component are summed with two_sum on the high parts and the error
// terms collected in FP32 (a compensated dot product, Ogita, Rump and
// Oishi 2005), normalised once at the end.
struct DfAcc {
  float s, c;
};
__device__ __forceinline__ void dfacc_add(DfAcc& a, DF h, float u) {
  const float p = __fmul_rn(h.hi, u);
  float e = __fmaf_rn(h.hi, u, -p);
  e = __fmaf_rn(h.lo, u, e);
  const DF t = df_two_sum(a.s, p);
  a.s = t.hi;
  a.c = __fadd_rn(a.c, __fadd_rn(t.lo, e));
}
template <int ADJ>
__device__ __forceinline__ void mat_half(const M3<DF>& u, const Cx<DF> h[2][3], Cx<DF> w[2][3]) {
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      DfAcc re = {0.0f, 0.0f}, im = {0.0f, 0.0f};
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        // u_ab h_b, or conj(u_ba) h_b
        const float ur = ADJ ? u.e[b][a].re.hi : u.e[a][b].re.hi;
        const float ui = ADJ ? -u.e[b][a].im.hi : u.e[a][b].im.hi;
        dfacc_add(re, h[k][b].re, ur);
        dfacc_add(re, h[k][b].im, -ui);
        dfacc_add(im, h[k][b].im, ur);
        dfacc_add(im, h[k][b].re, ui);
      }
      w[k][a] = cx<DF>(df_fast_two_sum(re.s, re.c), df_fast_two_sum(im.s, im.c));
    }
}
// The same reconstruction with sign = +-1 applied exactly (no double-float product).
__device__ __forceinline__ Cx<DF> df_scale_sign(const Cx<DF>& w, float sg) {
  return cx<DF>(DF(sg * w.re.hi, sg * w.re.lo), DF(sg * w.im.hi, sg * w.im.lo));
}
template <int MU, int S>
__device__ __forceinline__ void reconstruct_add(Spinor<DF>& acc, const Cx<DF> w[2][3], DF sign) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Cx<DF> w0 = df_scale_sign(w[0][c], sign.hi), w1 = df_scale_sign(w[1][c], sign.hi);
    Cx<DF> b0, b1;
    adag_mu<MU>(w0, w1, b0, b1);
    acc.s[0][c] = acc.s[0][c] + w0;
    acc.s[1][c] = acc.s[1][c] + w1;
    if (S > 0) {
      acc.s[2][c] = acc.s[2][c] - b0;
      acc.s[3][c] = acc.s[3][c] - b1;
    } else {
      acc.s[2][c] = acc.s[2][c] + b0;
      acc.s[3][c] = acc.s[3][c] + b1;
    }
  }
}

// ---- runtime-direction hop (double-float): one loop body for all eight
// hops keeps the long double-float code within the instruction cache.
// The spin structure of each direction is a choice of component and a unit
// factor in {1, i, -1, -i}, taken with selects.
__device__ __forceinline__ Cx<DF> unit_mul(const Cx<DF>& x, bool is_i, bool neg) {
  const float sg = neg ? -1.0f : 1.0f;
  const DF re = is_i ? -x.im : x.re;
  const DF im = is_i ? x.re : x.im;
  return cx<DF>(DF(sg * re.hi, sg * re.lo), DF(sg * im.hi, sg * im.lo));
}
__device__ __forceinline__ Cx<DF> pick(bool first, const Cx<DF>& a, const Cx<DF>& b) {
  return cx<DF>(first ? a.re : b.re, first ? a.im : b.im);
}
// h_k = psi_k - S (A_mu psi_down)_k: (A_mu psi_down)_0 = c0 psi_j0,
// (A_mu psi_down)_1 = c1 psi_(5-j0); j0 = 3 for mu = x, y and 2 for z, t;
// c0, c1 = (i, i), (-1, 1), (i, -i), (1, 1).
__device__ __forceinline__ void project_rt(int mu, int S, const Spinor<DF>& p, Cx<DF> h[2][3]) {
  const bool j3 = mu < 2, is_i = mu == 0 || mu == 2;
  const bool n0 = (mu == 1) != (S > 0), n1 = (mu == 2) != (S > 0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    h[0][c] = p.s[0][c] + unit_mul(pick(j3, p.s[3][c], p.s[2][c]), is_i, n0);
    h[1][c] = p.s[1][c] + unit_mul(pick(j3, p.s[2][c], p.s[3][c]), is_i, n1);
  }
}
// acc_up += sign w; acc_down += sign (-S) A_mu^dagger w with
// (A_mu^dagger w)_0 = d0 w_k0, (A_mu^dagger w)_1 = d1 w_(1-k0); k0 = 1 for
// mu = x, y and 0 for z, t; d0, d1 = (-i, -i), (1, -1), (-i, i), (1, 1).
__device__ __forceinline__ void reconstruct_rt(int mu, int S, float sign, const Cx<DF> w[2][3], Spinor<DF>& acc) {
  const bool k1 = mu < 2, is_i = mu == 0 || mu == 2;
  // w0, w1 carry `sign`; unit_mul applies d and the factor -S
  const bool n0 = is_i != (S > 0), n1 = (mu < 2) != (S > 0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Cx<DF> w0 = df_scale_sign(w[0][c], sign), w1 = df_scale_sign(w[1][c], sign);
    acc.s[0][c] = acc.s[0][c] + w0;
    acc.s[1][c] = acc.s[1][c] + w1;
    acc.s[2][c] = acc.s[2][c] + unit_mul(pick(k1, w1, w0), is_i, n0);
    acc.s[3][c] = acc.s[3][c] + unit_mul(pick(k1, w0, w1), is_i, n1);
  }
}
// w = U h (adj = false) or U^dagger h, FP32 link, compensated double-float sums
__device__ __forceinline__ void mat_half_rt(const M3<float>& u, bool adj, const Cx<DF> h[2][3], Cx<DF> w[2][3]) {
  float ur[3][3], ui[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      ur[a][b] = adj ? u.e[b][a].re : u.e[a][b].re;
      ui[a][b] = adj ? -u.e[b][a].im : u.e[a][b].im;
    }
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      DfAcc re = {0.0f, 0.0f}, im = {0.0f, 0.0f};
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        dfacc_add(re, h[k][b].re, ur[a][b]);
        dfacc_add(re, h[k][b].im, -ui[a][b]);
        dfacc_add(im, h[k][b].im, ur[a][b]);
        dfacc_add(im, h[k][b].re, ui[a][b]);
      }
      w[k][a] = cx<DF>(df_fast_two_sum(re.s, re.c), df_fast_two_sum(im.s, im.c));
    }
}
template <int DAG, int NC>
__device__ __forceinline__ void hops_rt(Spinor<DF>& acc, const float4* __restrict__ in, const Gauge<float, NC>& U,
                                        const Geom& g, const int c[4], int s, int in_off) {
  constexpr int SF = DAG ? -1 : 1;  // forward hop: (1 - g_mu), (1 + g_mu) for the dagger
#pragma unroll 1
  for (int hd = 0; hd < 8; ++hd) {
    const int mu = hd >> 1;
    const bool fwd = (hd & 1) == 0;
    const int sn = cb_neighbor_rt(g, c, mu, fwd ? 1 : -1);
    const Spinor<DF> p = load_spinor<DF>(in, sn - in_off, g.Vh);
    const int S = fwd ? SF : -SF;
    Cx<DF> h[2][3], w[2][3];
    project_rt(mu, S, p, h);
    const M3<float> u = U.load(mu, fwd ? s : sn);
    mat_half_rt(u, !fwd, h, w);
    const bool anti = mu == 3 && (fwd ? c[3] == g.L[3] - 1 : c[3] == 0);
    reconstruct_rt(mu, S, anti ? -1.0f : 1.0f, w, acc);
  }
}
template <int DAG, typename RL, int NC, typename RS, typename ST = RS>
struct Hops {
  static __device__ __forceinline__ void run(Spinor<RS>& acc, const typename Vec2<ST>::T* __restrict__ in,
                                             const Gauge<RL, NC>& U, const Geom& g, const int c[4], int s,
                                             int in_off);
};

// Where a hop reads its input spinor: a stored field, or (FoldSrc) the
// conjugate-gradient direction of the next iteration formed on the fly.
template <typename RS, typename ST>
struct FieldSrc {
  const typename Vec2<ST>::T* __restrict__ f;
  __device__ __forceinline__ Spinor<RS> operator()(int i, int Vh) const { return load_spinor<RS, ST>(f, i, Vh); }
};
// p' = (r - alpha Ap) + beta p entry by entry, with the same two roundings
// (fma) as the owner thread that stores r' and p', so every thread sees the
// same p' bits.
template <typename R>
struct FoldSrc {
  const typename Vec2<R>::T* __restrict__ r;
  const typename Vec2<R>::T* __restrict__ ap;
  const typename Vec2<R>::T* __restrict__ p;
  R alpha, beta;
  __device__ __forceinline__ Spinor<R> operator()(int i, int Vh) const {
    Spinor<R> x;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      Cx<R> r0, r1, a0, a1, p0, p1;
      Quad<R>::load(r, (size_t)q * Vh + i, r0, r1);
      Quad<R>::load(ap, (size_t)q * Vh + i, a0, a1);
      Quad<R>::load(p, (size_t)q * Vh + i, p0, p1);
      x.s[(2 * q) / 3][(2 * q) % 3] = fold_entry(r0, a0, p0);
      x.s[(2 * q + 1) / 3][(2 * q + 1) % 3] = fold_entry(r1, a1, p1);
    }
    return x;
  }
  __device__ __forceinline__ Cx<R> fold_entry(const Cx<R>& rv, const Cx<R>& av, const Cx<R>& pv) const {
    const R rre = fma(-alpha, av.re, rv.re), rim = fma(-alpha, av.im, rv.im);
    return cx<R>(fma(beta, pv.re, rre), fma(beta, pv.im, rim));
  }
};

template <int MU, int DAG, typename RL, int NC, typename RS, class Src>
__device__ __forceinline__ void hop_dir_src(Spinor<RS>& acc, const Src& src, const Gauge<RL, NC>& U,
                                            const Geom& g, const int c[4], int s, int in_off) {
  constexpr int SF = DAG ? -1 : 1;   // forward hop: (1 - g_mu), (1 + g_mu) for the dagger
  constexpr int SB = -SF;
  {
    const int sn = cb_neighbor(g, c, MU, +1);
    const Spinor<RS> p = src(sn - in_off, g.Vh);
    Cx<RS> h[2][3], w[2][3];
    project<MU, SF>(p, h);
    const M3<RS> u = convert<RS>(U.load(MU, s));
    mat_half<0>(u, h, w);
    const RS sign = (MU == 3 && c[3] == g.L[3] - 1) ? RS(-1) : RS(1);
    reconstruct_add<MU, SF>(acc, w, sign);
  }
  {
    const int sn = cb_neighbor(g, c, MU, -1);
    const Spinor<RS> p = src(sn - in_off, g.Vh);
    Cx<RS> h[2][3], w[2][3];
    project<MU, SB>(p, h);
    const M3<RS> u = convert<RS>(U.load(MU, sn));
    mat_half<1>(u, h, w);
    const RS sign = (MU == 3 && c[3] == 0) ? RS(-1) : RS(1);
    reconstruct_add<MU, SB>(acc, w, sign);
  }
}
template <int DAG, typename RL, int NC, typename RS, class Src>
__device__ __forceinline__ void hops_src(Spinor<RS>& acc, const Src& src, const Gauge<RL, NC>& U, const Geom& g,
                                         const int c[4], int s, int in_off) {
  hop_dir_src<0, DAG, RL, NC, RS>(acc, src, U, g, c, s, in_off);
  hop_dir_src<1, DAG, RL, NC, RS>(acc, src, U, g, c, s, in_off);
  hop_dir_src<2, DAG, RL, NC, RS>(acc, src, U, g, c, s, in_off);
  hop_dir_src<3, DAG, RL, NC, RS>(acc, src, U, g, c, s, in_off);
}

template <int DAG, typename RL, int NC, typename RS, typename ST>
__device__ __forceinline__ void Hops<DAG, RL, NC, RS, ST>::run(Spinor<RS>& acc,
                                                               const typename Vec2<ST>::T* __restrict__ in,
                                                               const Gauge<RL, NC>& U, const Geom& g,
                                                               const int c[4], int s, int in_off) {
  hops_src<DAG, RL, NC, RS>(acc, FieldSrc<RS, ST>{in}, U, g, c, s, in_off);
}
template <int DAG, int NC>
struct Hops<DAG, float, NC, DF, DF> {
  static __device__ __forceinline__ void run(Spinor<DF>& acc, const float4* __restrict__ in,
                                             const Gauge<float, NC>& U, const Geom& g, const int c[4], int s,
                                             int in_off) {
    hops_rt<DAG, NC>(acc, in, U, g, c, s, in_off);
  }
};

}  // namespace fg
