// Shared device definitions for the force-gradient HMC kernels (sm_103a).
//
// Device layout of every field (structure of arrays, checkerboard order):
//   site index s = parity * Vh + lex / 2, parity = (x+y+z+t) & 1, Vh = V / 2,
//   so each parity half is contiguous and a warp of consecutive s touches
//   consecutive addresses for every component.  Complex entries are stored
//   in pairs (2 complex = 16 bytes in FP32, 32 bytes in FP64):
//   gauge   Pair[4 mu][NC/2][V] (+ Cplx[4 mu][V] for the 9th entry when NC = 9)
//           NC = 9 complex entries (18 reals) or 6 (12 reals: rows 0-1, row 2
//           rebuilt as (row0 x row1)^*)
//   momenta Pair[4 mu][2][V]    Gell-Mann coefficients (p0..p3), (p4..p7)
//   spinor  Pair[6][Vh]         entries spin * 3 + colour, two per pair, one parity
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fg {

template <typename R> struct Vec2;
template <> struct Vec2<double> { typedef double2 T; };
template <> struct Vec2<float> { typedef float2 T; };

template <typename R> struct Cx {
  R re, im;
};

template <typename R> __host__ __device__ __forceinline__ Cx<R> cx(R re, R im) {
  Cx<R> c; c.re = re; c.im = im; return c;
}
template <typename R> __device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) { return cx(a.re + b.re, a.im + b.im); }
template <typename R> __device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) { return cx(a.re - b.re, a.im - b.im); }
template <typename R> __device__ __forceinline__ Cx<R> operator*(Cx<R> a, Cx<R> b) {
  return cx(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R> __device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a) { return cx(s * a.re, s * a.im); }
template <typename R> __device__ __forceinline__ Cx<R> conj(Cx<R> a) { return cx(a.re, -a.im); }
// a * i
template <typename R> __device__ __forceinline__ Cx<R> times_i(Cx<R> a) { return cx(-a.im, a.re); }
// acc += a * b
template <typename R> __device__ __forceinline__ void cmac(Cx<R>& acc, Cx<R> a, Cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im); acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R> __device__ __forceinline__ void cmac_cj(Cx<R>& acc, Cx<R> a, Cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im); acc.im = fma(-a.im, b.re, acc.im);
}
// acc += a * conj(b)
template <typename R> __device__ __forceinline__ void cmac_jc(Cx<R>& acc, Cx<R> a, Cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.im, b.re, acc.im); acc.im = fma(-a.re, b.im, acc.im);
}
// acc += conj(a) * conj(b)
template <typename R> __device__ __forceinline__ void cmac_cc(Cx<R>& acc, Cx<R> a, Cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(-a.re, b.im, acc.im); acc.im = fma(-a.im, b.re, acc.im);
}

template <typename R> struct M3 {
  Cx<R> e[3][3];
};

template <typename R> __device__ __forceinline__ void zero(M3<R>& m) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) m.e[i][j] = cx<R>(0, 0);
}
template <typename R> __device__ __forceinline__ void identity(M3<R>& m) {
  zero(m);
  m.e[0][0].re = m.e[1][1].re = m.e[2][2].re = R(1);
}

// c = a * b
template <typename R> __device__ __forceinline__ M3<R> mul(const M3<R>& a, const M3<R>& b) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<R> s = a.e[i][0] * b.e[0][j];
      cmac(s, a.e[i][1], b.e[1][j]);
      cmac(s, a.e[i][2], b.e[2][j]);
      c.e[i][j] = s;
    }
  return c;
}
// c = a * b^dagger
template <typename R> __device__ __forceinline__ M3<R> mul_nd(const M3<R>& a, const M3<R>& b) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<R> s = cx<R>(0, 0);
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac_jc(s, a.e[i][k], b.e[j][k]);
      c.e[i][j] = s;
    }
  return c;
}
// c = a^dagger * b
template <typename R> __device__ __forceinline__ M3<R> mul_dn(const M3<R>& a, const M3<R>& b) {
  M3<R> c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<R> s = cx<R>(0, 0);
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac_cj(s, a.e[k][i], b.e[k][j]);
      c.e[i][j] = s;
    }
  return c;
}
// acc += a * b^dagger
template <typename R> __device__ __forceinline__ void mac_nd(M3<R>& acc, const M3<R>& a, const M3<R>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac_jc(acc.e[i][j], a.e[i][k], b.e[j][k]);
}
// acc += a^dagger * b
template <typename R> __device__ __forceinline__ void mac_dn(M3<R>& acc, const M3<R>& a, const M3<R>& b) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) cmac_cj(acc.e[i][j], a.e[k][i], b.e[k][j]);
}

// Re Tr(a * b)
template <typename R> __device__ __forceinline__ R re_tr_mul(const M3<R>& a, const M3<R>& b) {
  R s = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) s += a.e[i][k].re * b.e[k][i].re - a.e[i][k].im * b.e[k][i].im;
  return s;
}
// Re Tr(a * b^dagger) = sum Re(a_ik conj(b_ik))
template <typename R> __device__ __forceinline__ R re_tr_mul_nd(const M3<R>& a, const M3<R>& b) {
  R s = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) s += a.e[i][k].re * b.e[i][k].re + a.e[i][k].im * b.e[i][k].im;
  return s;
}

// Im Tr(lambda^a W) for the eight Gell-Mann matrices (written out from their
// entries: lambda^1 = sigma_x on rows 0-1, lambda^2 = sigma_y on rows 0-1, ...).
template <typename R> __device__ __forceinline__ void im_tr_gellmann(const M3<R>& w, R out[8]) {
  const R inv_sqrt3 = R(0.57735026918962576451);
  out[0] = w.e[0][1].im + w.e[1][0].im;
  out[1] = w.e[0][1].re - w.e[1][0].re;
  out[2] = w.e[0][0].im - w.e[1][1].im;
  out[3] = w.e[0][2].im + w.e[2][0].im;
  out[4] = w.e[0][2].re - w.e[2][0].re;
  out[5] = w.e[1][2].im + w.e[2][1].im;
  out[6] = w.e[1][2].re - w.e[2][1].re;
  out[7] = (w.e[0][0].im + w.e[1][1].im - R(2) * w.e[2][2].im) * inv_sqrt3;
}

// Hermitian traceless Q = sum_a p^a lambda^a / 2.
template <typename R> __device__ __forceinline__ M3<R> alg_to_mat(const R p[8]) {
  const R s3 = R(0.57735026918962576451);
  M3<R> q;
  q.e[0][0] = cx<R>(R(0.5) * (p[2] + s3 * p[7]), 0);
  q.e[1][1] = cx<R>(R(0.5) * (-p[2] + s3 * p[7]), 0);
  q.e[2][2] = cx<R>(-s3 * p[7], 0);
  q.e[0][1] = cx<R>(R(0.5) * p[0], R(-0.5) * p[1]);
  q.e[1][0] = cx<R>(R(0.5) * p[0], R(0.5) * p[1]);
  q.e[0][2] = cx<R>(R(0.5) * p[3], R(-0.5) * p[4]);
  q.e[2][0] = cx<R>(R(0.5) * p[3], R(0.5) * p[4]);
  q.e[1][2] = cx<R>(R(0.5) * p[5], R(-0.5) * p[6]);
  q.e[2][1] = cx<R>(R(0.5) * p[5], R(0.5) * p[6]);
  return q;
}

template <typename R> struct ExpSmall;
template <> struct ExpSmall<double> { static constexpr double c1_min = 1e-24; };
template <> struct ExpSmall<float> { static constexpr float c1_min = 1e-12f; };

// exp(i A) for Hermitian traceless A by the Cayley-Hamilton closed form of
// Morningstar and Peardon (Phys. Rev. D 69 (2004) 054501, section III):
// exp(iA) = f0 + f1 A + f2 A^2 with f_j from c0 = det A and c1 = Tr A^2 / 2;
// negative c0 is mapped to positive through f_j(-c0) = (-1)^j conj(f_j(c0)).
// A^2 for Hermitian A: real diagonal entries sum_k |a_ik|^2, the lower
// triangle the conjugate of the upper one (half the products of mul).
template <typename R> __device__ __forceinline__ M3<R> herm_sq(const M3<R>& a) {
  M3<R> s;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    R d = R(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) d = fma(a.e[i][k].re, a.e[i][k].re, fma(a.e[i][k].im, a.e[i][k].im, d));
    s.e[i][i] = cx<R>(d, R(0));
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = i + 1; j < 3; ++j) {
      Cx<R> c = a.e[i][0] * a.e[0][j];
      cmac(c, a.e[i][1], a.e[1][j]);
      cmac(c, a.e[i][2], a.e[2][j]);
      s.e[i][j] = c;
      s.e[j][i] = conj(c);
    }
  return s;
}

// The coefficients f0, f1, f2 of exp(i A) = f0 + f1 A + f2 A^2 from
// c0 = det A and c1 = Tr A^2 / 2 (scalar part of the closed form).
template <typename R>
__device__ __forceinline__ void expi_coeffs(R c0, R c1, Cx<R>& f0, Cx<R>& f1, Cx<R>& f2) {
  if (c1 < ExpSmall<R>::c1_min) {
    // |A| ~ sqrt(c1): exp(iA) = 1 + iA - A^2/2 + O(|A|^3)
    f0 = cx<R>(1, 0); f1 = cx<R>(0, 1); f2 = cx<R>(R(-0.5), 0);
  } else {
    const bool neg = c0 < R(0);
    const R c0a = neg ? -c0 : c0;
    const R r = sqrt(c1 * R(1.0 / 3.0));
    const R c0max = R(2) * r * r * r;
    R ratio = c0a / c0max;
    ratio = ratio > R(1) ? R(1) : ratio;
    const R theta = acos(ratio);
    R st, ct;
    sincos(theta * R(1.0 / 3.0), &st, &ct);
    const R u = r * ct;
    const R w = sqrt(c1) * st;
    const R u2 = u * u, w2 = w * w;
    R su, cu, sw, cw;
    sincos(u, &su, &cu);
    sincos(w, &sw, &cw);
    R xi0;
    if (fabs(w) < R(0.05)) xi0 = R(1) - w2 * R(1.0 / 6.0) * (R(1) - w2 * R(0.05) * (R(1) - w2 * R(1.0 / 42.0)));
    else xi0 = sw / w;
    // double-angle identities for 2u (a few ulp, as a third sincos would give)
    const R s2u = R(2) * su * cu;
    const R c2u = (cu - su) * (cu + su);
    const Cx<R> e2 = cx<R>(c2u, s2u);
    const Cx<R> em = cx<R>(cu, -su);
    const Cx<R> h0 = (u2 - w2) * e2 + em * cx<R>(R(8) * u2 * cw, R(2) * u * (R(3) * u2 + w2) * xi0);
    const Cx<R> h1 = (R(2) * u) * e2 - em * cx<R>(R(2) * u * cw, -(R(3) * u2 - w2) * xi0);
    const Cx<R> h2 = e2 - em * cx<R>(cw, R(3) * u * xi0);
    const R inv = R(1) / (R(9) * u2 - w2);
    f0 = inv * h0; f1 = inv * h1; f2 = inv * h2;
    if (neg) { f0 = conj(f0); f1 = cx<R>(-f1.re, f1.im); f2 = conj(f2); }
  }
}

// Requires A exactly Hermitian (as alg_to_mat builds it).
template <typename R> __device__ __forceinline__ M3<R> expi_herm(const M3<R>& a) {
  M3<R> a2 = herm_sq(a);
  R c0 = re_tr_mul(a, a2) * R(1.0 / 3.0);
  R c1 = R(0.5) * (a2.e[0][0].re + a2.e[1][1].re + a2.e[2][2].re);
  Cx<R> f0, f1, f2;
  expi_coeffs(c0, c1, f0, f1, f2);
  M3<R> e;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<R> s = f1 * a.e[i][j];
      cmac(s, f2, a2.e[i][j]);
      if (i == j) s = s + f0;
      e.e[i][j] = s;
    }
  return e;
}

// Rebuild row 2 of a special unitary matrix from rows 0 and 1: row2 = (row0 x row1)^*.
template <typename R> __device__ __forceinline__ void rebuild_row2(M3<R>& u) {
  u.e[2][0] = conj(u.e[0][1] * u.e[1][2] - u.e[0][2] * u.e[1][1]);
  u.e[2][1] = conj(u.e[0][2] * u.e[1][0] - u.e[0][0] * u.e[1][2]);
  u.e[2][2] = conj(u.e[0][0] * u.e[1][1] - u.e[0][1] * u.e[1][0]);
}

// Scale a row of squared norm 1 + d to unit norm.  The factor is applied as
// x += c x with c = (1 + d)^(-1/2) - 1, not as x *= (1 + c): a factor that
// close to 1 would be rounded on the grid around 1.0, which is twice as
// coarse above 1 as below, so rows slightly too long would survive more often
// than rows slightly too short and every link would drift the same way
// (the Wilson action would move coherently, by an amount proportional to the
// volume, in each trajectory).
template <typename R> __device__ __forceinline__ void normalize_row(Cx<R> row[3]) {
  R d = R(-1);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    d = fma(row[j].re, row[j].re, d);
    d = fma(row[j].im, row[j].im, d);
  }
  // (1 + d)^(-1/2) - 1 = -d/2 + 3 d^2 / 8 - 5 d^3 / 16 + ...
  const R c = fabs(d) < R(1e-3) ? d * (R(-0.5) + d * (R(0.375) - d * R(0.3125))) : R(1) / sqrt(R(1) + d) - R(1);
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    row[j].re = fma(c, row[j].re, row[j].re);
    row[j].im = fma(c, row[j].im, row[j].im);
  }
}

// Gram-Schmidt of rows 0-1 in the link's own precision, then row 2 from the
// cross product.
template <typename R> __device__ __forceinline__ void reunitarize(M3<R>& u) {
  normalize_row(u.e[0]);
  Cx<R> pr = cx<R>(0, 0);  // <row0, row1>
#pragma unroll
  for (int j = 0; j < 3; ++j) cmac_cj(pr, u.e[0][j], u.e[1][j]);
#pragma unroll
  for (int j = 0; j < 3; ++j) u.e[1][j] = u.e[1][j] - pr * u.e[0][j];
  normalize_row(u.e[1]);
  rebuild_row2(u);
}

// ---------------------------------------------------------------------------
// Exact division of a 32-bit n by a run-time constant d >= 1 without the
// integer-divide sequence: q = floor(c n / 2^64) with c = floor((2^64-1)/d) + 1
// (Lemire, Kaser and Kurz, "Faster remainder by direct computation", 2019);
// d = 1 is special-cased because c would overflow.
struct FastDiv {
  uint32_t d;
  unsigned long long c;
};
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.c = d > 1 ? (~0ULL) / d + 1 : 0ULL;
  return f;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
  return f.d == 1 ? n : (uint32_t)__umul64hi(f.c, (unsigned long long)n);
}

// ---------------------------------------------------------------------------
// Lattice geometry in checkerboard order.
struct Geom {
  int L[4];     // Lx, Ly, Lz, Lt
  int Lxh;      // Lx / 2
  int Vh;       // V / 2
  int V;
  FastDiv dLxh, dLy, dLz;
};

__device__ __forceinline__ void cb_coords(const Geom& g, int s, int c[4], int& par) {
  par = s >= g.Vh;
  const uint32_t i = (uint32_t)(s - par * g.Vh);
  const uint32_t q1 = fdiv(i, g.dLxh);
  const uint32_t xh = i - q1 * (uint32_t)g.Lxh;
  const uint32_t q2 = fdiv(q1, g.dLy);
  c[1] = (int)(q1 - q2 * (uint32_t)g.L[1]);
  const uint32_t q3 = fdiv(q2, g.dLz);
  c[2] = (int)(q2 - q3 * (uint32_t)g.L[2]);
  c[3] = (int)q3;
  c[0] = 2 * (int)xh + ((c[1] + c[2] + c[3] + par) & 1);
}

__device__ __forceinline__ int cb_index(const Geom& g, const int c[4]) {
  const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
  const int lex = c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
  return par * g.Vh + (lex >> 1);
}

// Index of the neighbour x + d * mu-hat (d = +1 or -1), periodic.  Call with
// compile-time mu (unrolled loops or template arguments) so that the
// coordinate array stays in registers.
__device__ __forceinline__ int cb_neighbor(const Geom& g, const int c[4], int mu, int d) {
  int n[4] = {c[0], c[1], c[2], c[3]};
  int v = n[mu] + d;
  v = v < 0 ? v + g.L[mu] : (v >= g.L[mu] ? v - g.L[mu] : v);
  n[mu] = v;
  return cb_index(g, n);
}
// The same with a run-time direction, by selects instead of an indexed
// coordinate array (which the compiler would place in local memory).
__device__ __forceinline__ int sel4(const int v[4], int i) {
  return i == 0 ? v[0] : (i == 1 ? v[1] : (i == 2 ? v[2] : v[3]));
}
__device__ __forceinline__ int cb_neighbor_rt(const Geom& g, const int c[4], int mu, int d) {
  int n[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    int v = c[k] + (k == mu ? d : 0);
    v = v < 0 ? v + g.L[k] : (v >= g.L[k] ? v - g.L[k] : v);
    n[k] = v;
  }
  return cb_index(g, n);
}

// Site of a link thread: a block of (64, 4) threads covers half-site indices
// [32 b, 32 b + 32) in both parities (warp 0 even, warp 1 odd) and all four
// directions, so the +-x neighbours of its sites are its own sites and both
// parity halves of a field are swept together (L1 and L2 reuse).  Launch
// with (V/2 + 31) / 32 blocks.
__device__ __forceinline__ bool link_site(const Geom& g, int& s) {
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  if (i >= g.Vh) return false;
  s = (threadIdx.x >> 5) * g.Vh + i;
  return true;
}
// The same for one thread per site and blocks of 2 * H threads: half-site
// indices [H b, H b + H) of both parities.  Launch with (V/2 + H - 1) / H blocks.
template <int H>
__device__ __forceinline__ bool pair_site(const Geom& g, int& s) {
  const int i = blockIdx.x * H + (threadIdx.x % H);
  if (i >= g.Vh) return false;
  s = (threadIdx.x / H) * g.Vh + i;
  return true;
}

// ---------------------------------------------------------------------------
// Field access.  Fields are stored "pair-major": complex entries are grouped
// in pairs, and pair q of every site is contiguous, so that one thread moves
// a pair with one 16-byte access in FP32 (float4) or two adjacent 16-byte
// accesses in FP64.  The flat order of a field is therefore the same in both
// precisions (pair, site, entry), which lets vector kernels convert and
// combine fields element by element.
template <typename R> struct Quad;
template <> struct Quad<float> {
  // one complex entry (the ninth link entry, stored apart from the pairs)
  static __device__ __forceinline__ Cx<float> load1(const void* base, size_t idx) {
    const float2 v = __ldg((const float2*)base + idx);
    return cx<float>(v.x, v.y);
  }
  static __device__ __forceinline__ void store1(void* base, size_t idx, Cx<float> a) {
    ((float2*)base)[idx] = make_float2(a.re, a.im);
  }
  static __device__ __forceinline__ void load(const void* base, size_t idx, Cx<float>& a, Cx<float>& b) {
    const float4 v = __ldg((const float4*)base + idx);
    a = cx<float>(v.x, v.y);
    b = cx<float>(v.z, v.w);
  }
  static __device__ __forceinline__ void load_cg(const void* base, size_t idx, Cx<float>& a, Cx<float>& b) {
    const float4 v = ((const float4*)base)[idx];
    a = cx<float>(v.x, v.y);
    b = cx<float>(v.z, v.w);
  }
  static __device__ __forceinline__ void store(void* base, size_t idx, Cx<float> a, Cx<float> b) {
    ((float4*)base)[idx] = make_float4(a.re, a.im, b.re, b.im);
  }
};
template <> struct Quad<double> {
  static __device__ __forceinline__ Cx<double> load1(const void* base, size_t idx) {
    const double2 v = __ldg((const double2*)base + idx);
    return cx<double>(v.x, v.y);
  }
  static __device__ __forceinline__ void store1(void* base, size_t idx, Cx<double> a) {
    ((double2*)base)[idx] = make_double2(a.re, a.im);
  }
  static __device__ __forceinline__ void load(const void* base, size_t idx, Cx<double>& a, Cx<double>& b) {
    const double2* p = (const double2*)base + 2 * idx;
    const double2 u = __ldg(p), v = __ldg(p + 1);
    a = cx<double>(u.x, u.y);
    b = cx<double>(v.x, v.y);
  }
  static __device__ __forceinline__ void load_cg(const void* base, size_t idx, Cx<double>& a, Cx<double>& b) {
    const double2* p = (const double2*)base + 2 * idx;
    const double2 u = p[0], v = p[1];
    a = cx<double>(u.x, u.y);
    b = cx<double>(v.x, v.y);
  }
  static __device__ __forceinline__ void store(void* base, size_t idx, Cx<double> a, Cx<double> b) {
    double2* p = (double2*)base + 2 * idx;
    p[0] = make_double2(a.re, a.im);
    p[1] = make_double2(b.re, b.im);
  }
};

// 16-bit storage with FP32 arithmetic for the inner solver: links and, with
// a per-solve-cycle scale, its spinor vectors.  A complex number is one pair
// of 16-bit reals (32 bits), a pair of entries 8 bytes.  Two formats:
//  * Half16: IEEE binary16, 11 significant bits (unit roundoff 2^-11);
//  * BF16: bfloat16, the exponent range of FP32 with 8 significant bits
//    (unit roundoff 2^-8).
struct Half16 {};
struct BF16 {};
template <> struct Vec2<Half16> { typedef __half2 T; };
template <> struct Vec2<BF16> { typedef __nv_bfloat162 T; };
// conversions of one complex number (or any pair of reals) to and from the
// 32-bit pair, round to nearest even
template <typename S> struct Conv16;
template <> struct Conv16<Half16> {
  typedef __half2 T2;
  static __device__ __forceinline__ float2 f2(T2 h) { return __half22float2(h); }
  static __device__ __forceinline__ T2 of(float2 v) { return __float22half2_rn(v); }
};
template <> struct Conv16<BF16> {
  typedef __nv_bfloat162 T2;
  static __device__ __forceinline__ float2 f2(T2 h) { return __bfloat1622float2(h); }
  static __device__ __forceinline__ T2 of(float2 v) { return __float22bfloat162_rn(v); }
};
template <typename S> __device__ __forceinline__ Cx<float> w16_to_cx(unsigned int w) {
  const float2 f = Conv16<S>::f2(*reinterpret_cast<const typename Conv16<S>::T2*>(&w));
  return cx<float>(f.x, f.y);
}
template <typename S> __device__ __forceinline__ unsigned int cx_to_w16(const Cx<float>& c) {
  const typename Conv16<S>::T2 h = Conv16<S>::of(make_float2(c.re, c.im));
  return *reinterpret_cast<const unsigned int*>(&h);
}
template <typename S> struct Quad16 {
  static __device__ __forceinline__ void load(const void* base, size_t idx, Cx<float>& a, Cx<float>& b) {
    const uint2 v = __ldg((const uint2*)base + idx);
    a = w16_to_cx<S>(v.x);
    b = w16_to_cx<S>(v.y);
  }
  static __device__ __forceinline__ void load_cg(const void* base, size_t idx, Cx<float>& a, Cx<float>& b) {
    const uint2 v = ((const uint2*)base)[idx];
    a = w16_to_cx<S>(v.x);
    b = w16_to_cx<S>(v.y);
  }
  static __device__ __forceinline__ void store(void* base, size_t idx, Cx<float> a, Cx<float> b) {
    ((uint2*)base)[idx] = make_uint2(cx_to_w16<S>(a), cx_to_w16<S>(b));
  }
};
template <> struct Quad<Half16> : Quad16<Half16> {};
template <> struct Quad<BF16> : Quad16<BF16> {};

// Links: NP = NC / 2 pairs per link in [mu][pair][site] order, then, for
// NC = 9, the ninth entry of every link in [mu][site] order.
template <typename R, int NC> struct Gauge {
  typedef typename Vec2<R>::T C2;
  static constexpr int NP = NC / 2;
  void* __restrict__ p;
  int V;
  // Element indices in 32 bits (the largest is 4 NP V + V, and the handles
  // reject lattices where that would overflow), widened once per access.
  __device__ __forceinline__ unsigned idx(int mu, int q, int s) const {
    return ((unsigned)mu * NP + (unsigned)q) * (unsigned)V + (unsigned)s;
  }
  __device__ __forceinline__ M3<R> load(int mu, int s) const {
    M3<R> m;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      Cx<R> a, b;
      Quad<R>::load(p, (size_t)idx(mu, q, s), a, b);
      m.e[(2 * q) / 3][(2 * q) % 3] = a;
      m.e[(2 * q + 1) / 3][(2 * q + 1) % 3] = b;
    }
    if (NC == 9) {
      const void* tail = (const char*)p + (size_t)4 * NP * V * 4 * sizeof(R);
      m.e[2][2] = Quad<R>::load1(tail, (size_t)((unsigned)mu * (unsigned)V + (unsigned)s));
    } else {
      rebuild_row2(m);
    }
    return m;
  }
  __device__ __forceinline__ void store(int mu, int s, const M3<R>& m) const {
#pragma unroll
    for (int q = 0; q < NP; ++q)
      Quad<R>::store(p, (size_t)idx(mu, q, s), m.e[(2 * q) / 3][(2 * q) % 3],
                     m.e[(2 * q + 1) / 3][(2 * q + 1) % 3]);
    if (NC == 9) {
      void* tail = (char*)p + (size_t)4 * NP * V * 4 * sizeof(R);
      Quad<R>::store1(tail, (size_t)((unsigned)mu * (unsigned)V + (unsigned)s), m.e[2][2]);
    }
  }
};

// Links stored in a 16-bit format (Half16 or BF16) for the inner Dslash of
// the solver (entries of an SU(3) matrix lie in [-1, 1], so neither format
// needs a scale).  Same layout as Gauge<float, NC> with two bytes per real:
// a pair of entries is 8 bytes, the NC = 9 tail 4 bytes.  Loads return FP32
// matrices.
template <typename S, int NC> struct Gauge16 {
  static constexpr int NP = NC / 2;
  void* __restrict__ p;
  int V;
  static __device__ __forceinline__ Cx<float> cx_of(unsigned int w) { return w16_to_cx<S>(w); }
  static __device__ __forceinline__ unsigned int word_of(const Cx<float>& c) { return cx_to_w16<S>(c); }
  __device__ __forceinline__ M3<float> load(int mu, int s) const {
    M3<float> m;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const uint2 v = __ldg((const uint2*)p + (size_t)(((unsigned)mu * NP + (unsigned)q) * (unsigned)V + (unsigned)s));
      m.e[(2 * q) / 3][(2 * q) % 3] = cx_of(v.x);
      m.e[(2 * q + 1) / 3][(2 * q + 1) % 3] = cx_of(v.y);
    }
    if (NC == 9) {
      const unsigned int* tail = (const unsigned int*)((const char*)p + (size_t)4 * NP * V * 8);
      m.e[2][2] = cx_of(__ldg(tail + (size_t)((unsigned)mu * (unsigned)V + (unsigned)s)));
    } else {
      rebuild_row2(m);
    }
    return m;
  }
  __device__ __forceinline__ void store(int mu, int s, const M3<float>& m) const {
#pragma unroll
    for (int q = 0; q < NP; ++q)
      ((uint2*)p)[(size_t)(((unsigned)mu * NP + (unsigned)q) * (unsigned)V + (unsigned)s)] =
          make_uint2(word_of(m.e[(2 * q) / 3][(2 * q) % 3]), word_of(m.e[(2 * q + 1) / 3][(2 * q + 1) % 3]));
    if (NC == 9) {
      unsigned int* tail = (unsigned int*)((char*)p + (size_t)4 * NP * V * 8);
      tail[(size_t)((unsigned)mu * (unsigned)V + (unsigned)s)] = word_of(m.e[2][2]);
    }
  }
};
template <int NC> struct Gauge<Half16, NC> : Gauge16<Half16, NC> {};
template <int NC> struct Gauge<BF16, NC> : Gauge16<BF16, NC> {};

// Momenta and forces: the 8 Gell-Mann coefficients of a link as two pairs of
// (re, im)-like slots, [mu][pair][site].
template <typename R> struct Mom {
  void* __restrict__ p;
  int V;
  __device__ __forceinline__ unsigned idx(int mu, int q, int s) const {
    return ((unsigned)mu * 2u + (unsigned)q) * (unsigned)V + (unsigned)s;
  }
  __device__ __forceinline__ void load(int mu, int s, R out[8]) const {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      Cx<R> a, b;
      Quad<R>::load_cg(p, (size_t)idx(mu, q, s), a, b);
      out[4 * q] = a.re; out[4 * q + 1] = a.im; out[4 * q + 2] = b.re; out[4 * q + 3] = b.im;
    }
  }
  __device__ __forceinline__ void store(int mu, int s, const R in[8]) const {
#pragma unroll
    for (int q = 0; q < 2; ++q)
      Quad<R>::store(p, (size_t)idx(mu, q, s), cx<R>(in[4 * q], in[4 * q + 1]),
                     cx<R>(in[4 * q + 2], in[4 * q + 3]));
  }
};

// ---------------------------------------------------------------------------
// Deterministic block reduction of NV doubles (fixed tree for a fixed launch).
template <int NV>
__device__ __forceinline__ void block_reduce_store(double v[NV], double* __restrict__ partial,
                                                   int nblocks_stride) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[k][warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double x = lane < nwarps ? sh[k][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) partial[(size_t)k * nblocks_stride + blockIdx.x] = x;
    }
  }
}

// block_reduce_store<1> followed by a grand total: the last block to finish
// (counted on *ticket, which it resets to 0 for the next launch) sums the
// partials in block order and writes *total, so the sum is deterministic and
// the next kernel reads one scalar.  Every block of the launch must call it.
__device__ __forceinline__ void block_reduce_total(double v, double* __restrict__ partial,
                                                   unsigned* __restrict__ ticket, double* __restrict__ total) {
  double vv[1] = {v};
  block_reduce_store<1>(vv, partial, gridDim.x);
  __shared__ int last;
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // each thread's partials in block order; four loads in flight at a time
  double x = 0.0;
  const int n = gridDim.x, bd = blockDim.x;
  int i = threadIdx.x;
  for (; i + 3 * bd < n; i += 4 * bd) {
    const double a = __ldcg(partial + i), b = __ldcg(partial + i + bd);
    const double c = __ldcg(partial + i + 2 * bd), d = __ldcg(partial + i + 3 * bd);
    x += a;
    x += b;
    x += c;
    x += d;
  }
  for (; i < n; i += bd) x += __ldcg(partial + i);
  __shared__ double sh[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t += sh[w];
    *total = t;
    *ticket = 0u;
  }
}

}  // namespace fg
