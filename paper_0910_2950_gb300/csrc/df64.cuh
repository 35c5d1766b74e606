// Double-float numbers: a value is the unevaluated sum hi + lo of two floats
// with |lo| <= ulp(hi) / 2, about 48 significant bits (relative rounding
// ~3.6e-15).  GB300 issues FP32 FMAs at about 64 times its FP64 rate, so
// vector work that needs more than FP32 but tolerates ~1e-14 relative error
// (the Dslash of a CG reliable update) runs faster on the FP32 pipes in this
// form than in FP64.
//
// Error-free transformations used:
//   two_sum       Knuth, TAOCP vol. 2, sec. 4.2.2: s + e == a + b exactly;
//   fast_two_sum  Dekker (1971), valid when |a| >= |b| or a == 0;
//   product       a * b == p + e exactly with p = fl(a b), e = fma(a, b, -p).
// Addition is the "sloppy" double-float sum (one two_sum of the high parts,
// the low parts added in FP32): its error is bounded by ~2^-47 of the larger
// operand, which is the scale that matters for residuals.  These routines
// must not be compiled with reassociation (no fast-math); nvcc's FMA
// contraction is harmless here because every product is written out.
#pragma once

#include <cuda_runtime.h>

#include "fg_common.cuh"

namespace fg {

struct DF {
  float hi, lo;
  DF() = default;
  __host__ __device__ __forceinline__ constexpr DF(float h) : hi(h), lo(0.0f) {}
  __host__ __device__ __forceinline__ constexpr DF(int h) : hi((float)h), lo(0.0f) {}
  // Nearest double-float to a double (host or device; FP64 arithmetic, which
  // the compiler folds away for a literal argument).
  __host__ __device__ __forceinline__ constexpr explicit DF(double d)
      : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ __forceinline__ constexpr DF(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return DF(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return DF(s, e);
}

__device__ __forceinline__ DF operator+(DF a, DF b) {
  const DF s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF& operator+=(DF& a, DF b) { return a = a + b; }
__device__ __forceinline__ DF operator-(DF a) { return DF(-a.hi, -a.lo); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }
// Products keep the lo * lo term: it is ~2^-48 of the result, but for a
// square it is never negative, so dropping it (the usual "sloppy" product)
// biases every x * x low by ~6e-16 on average; in the exponential of the
// link update that made each drift shrink |U|^2 by ~4e-15, which moved the
// dH of a 32^4 trajectory by ~7e-7.
__device__ __forceinline__ DF operator*(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.lo, b.lo, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// a * b + c with one normalisation.  Generic code calls fma, sqrt, fabs and
// sincos unqualified; the using-declarations keep the float and double
// overloads visible next to the double-float ones declared here (otherwise
// those would hide them, and a float argument would convert to DF).
using ::fma;
using ::sqrt;
using ::fabs;
using ::sincos;
__device__ __forceinline__ DF fma(DF a, DF b, DF c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  const DF s = df_two_sum(p, c.hi);
  e = __fmaf_rn(a.lo, b.lo, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  e = __fadd_rn(e, __fadd_rn(s.lo, c.lo));
  return df_fast_two_sum(s.hi, e);
}
// a + f for a float f (CG solution updates)
__device__ __forceinline__ DF df_add_f(DF a, float f) {
  const DF s = df_two_sum(a.hi, f);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ DF& operator-=(DF& a, DF b) { return a = a - b; }
__device__ __forceinline__ DF& operator*=(DF& a, DF b) { return a = a * b; }
// a * f for a float f
__device__ __forceinline__ DF operator*(DF a, float f) {
  const float p = __fmul_rn(a.hi, f);
  float e = __fmaf_rn(a.hi, f, -p);
  e = __fmaf_rn(a.lo, f, e);
  return df_fast_two_sum(p, e);
}
// Quotient by two correction steps: q1 = a.hi / b.hi, q2 = r1.hi / b.hi
// with the remainder r1 = a - q1 b, q3 = r2.hi / b.hi with r2 = r1 - q2 b.
// One step is accurate to ~2^-47 but not unbiased: dividing r1 (which
// contains -q1 b.lo) by b.hi instead of b leaves -q (b.lo / b.hi)^2, never
// positive, so 1/x came out low by 6.5e-16 on average and every exp(iA)
// (its coefficients divide by 9u^2 - w^2) shrank the links.  The second
// step's own error is ~2^-72.
__device__ __forceinline__ DF operator/(DF a, DF b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const DF r1 = a - b * q1;
  const float q2 = __fdiv_rn(r1.hi, b.hi);
  const DF r2 = r1 - b * q2;
  const DF q = df_fast_two_sum(q1, q2);
  return df_add_f(q, __fdiv_rn(r2.hi, b.hi));
}
// Ordering of normalised double-floats (|lo| <= ulp(hi) / 2).
__device__ __forceinline__ bool operator<(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(DF a, DF b) { return b < a; }
__device__ __forceinline__ DF fabs(DF a) { return (a.hi < 0.0f || (a.hi == 0.0f && a.lo < 0.0f)) ? -a : a; }
// Square root: s = sqrt(a.hi) in FP32, then a Newton step on s^2 = a with
// the residual a - s^2 formed exactly (s^2 = p + e by the FMA product, and
// a.hi - p is exact by Sterbenz's lemma), then a second one in double-float.
// One step leaves an error of one sign (a Newton step for sqrt always lands
// above the root, here by ~2^-49 relative); the second removes it.
__device__ __forceinline__ DF sqrt(DF a) {
  if (!(a.hi > 0.0f)) return DF(0.0f);
  const float s = __fsqrt_rn(a.hi);
  const float p = __fmul_rn(s, s);
  const float e = __fmaf_rn(s, s, -p);
  const float d = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), e), a.lo);
  const DF y = df_fast_two_sum(s, __fdiv_rn(d, __fadd_rn(s, s)));
  const DF r = a - y * y;
  return y + DF(__fdiv_rn(r.hi, __fadd_rn(y.hi, y.hi)));
}

// sin and cos of a double-float argument.  Arguments beyond pi/4 are first
// reduced by n pi/2 (Cody and Waite's additive reduction, with pi/2 split
// into three floats; the first two products are formed exactly), then the
// Taylor series run on y / 2^k, |y / 2^k| <= 1/8, followed by k double-angle
// steps (sin 2y = 2 sin y cos y, cos 2y = 1 - 2 sin^2 y), and the quadrant
// n mod 4 permutes the result.  The series stop at y^11 and y^10: the first
// omitted terms are below 3e-20 of the result.  A truncation error has one
// sign, so it must stay far below the rounding: stopping one term earlier
// (cos short by up to 2.6e-16) made every exp(iA) shrink the links by
// ~1e-15, and over 16 drifts of 4.2 M links that moved S by ~1e-6 on 32^4.
// Each doubling at most doubles the absolute rounding error and k <= 3
// after the reduction, so the error stays near 3e-14 plus the 2^-48 |x| that
// the argument itself carries.  Arguments here are rotation angles of link
// updates, usually below 1.
__device__ __forceinline__ void sincos(DF x, DF* s, DF* c) {
  int quadrant = 0;
  if (fabsf(x.hi) > 0.785398163f) {
    const float n = rintf(__fmul_rn(x.hi, 0.636619772f));  // round(2 x / pi)
    constexpr float p1 = 1.57079637050628662109375f, p2 = -4.37113882867379300296306610107421875e-8f,
                    p3 = -1.71512451000588190e-15f;         // p1 + p2 + p3 = pi/2 to ~1e-23
    const float q1 = __fmul_rn(n, p1), q2 = __fmul_rn(n, p2);
    x = x - DF(q1, __fmaf_rn(n, p1, -q1));
    x = x - DF(q2, __fmaf_rn(n, p2, -q2));
    x = x - DF(__fmul_rn(n, p3));
    quadrant = (int)n & 3;
  }
  // k = max(0, e + 3) with |x.hi| = m 2^e, m in [0.5, 1)
  const int e = (int)((__float_as_uint(x.hi) >> 23) & 0xffu) - 126;
  const int k = e + 3 > 0 ? (e + 3 < 60 ? e + 3 : 60) : 0;
  const float sc = __uint_as_float((uint32_t)(127 - k) << 23);  // 2^-k, exact scaling
  const DF y(__fmul_rn(x.hi, sc), __fmul_rn(x.lo, sc));
  const DF z = y * y;
  constexpr DF s3(-1.0 / 6.0), s5(1.0 / 120.0), s7(-1.0 / 5040.0), s9(1.0 / 362880.0), s11(-1.0 / 39916800.0);
  constexpr DF c4(1.0 / 24.0), c6(-1.0 / 720.0), c8(1.0 / 40320.0), c10(-1.0 / 3628800.0);
  DF ps = fma(z, s11, s9);
  ps = fma(z, ps, s7);
  ps = fma(z, ps, s5);
  ps = fma(z, ps, s3);
  DF sn = fma(y * z, ps, y);
  DF pc = fma(z, c10, c8);
  pc = fma(z, pc, c6);
  pc = fma(z, pc, c4);
  DF cs = fma(z * z, pc, DF(1.0f) - z * 0.5f);
  for (int i = 0; i < k; ++i) {
    const DF s2 = sn * sn;
    sn = (sn * cs) * 2.0f;
    cs = DF(1.0f) - s2 * 2.0f;
  }
  // sin(y + n pi/2), cos(y + n pi/2)
  const DF ms = -sn, mc = -cs;
  *s = quadrant == 0 ? sn : (quadrant == 1 ? cs : (quadrant == 2 ? ms : mc));
  *c = quadrant == 0 ? cs : (quadrant == 1 ? ms : (quadrant == 2 ? mc : sn));
}

// Storage: one complex double-float is a float4 (re.hi, re.lo, im.hi, im.lo),
// the same 16 bytes as a complex double; a pair of entries is two float4.
template <> struct Vec2<DF> { typedef float4 T; };
template <> struct Quad<DF> {
  static __device__ __forceinline__ Cx<DF> c(float4 v) { return cx<DF>(DF(v.x, v.y), DF(v.z, v.w)); }
  static __device__ __forceinline__ Cx<DF> load1(const void* base, size_t idx) {
    return c(__ldg((const float4*)base + idx));
  }
  static __device__ __forceinline__ void store1(void* base, size_t idx, Cx<DF> a) {
    ((float4*)base)[idx] = make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo);
  }
  static __device__ __forceinline__ void load(const void* base, size_t idx, Cx<DF>& a, Cx<DF>& b) {
    const float4* p = (const float4*)base + 2 * idx;
    a = c(__ldg(p));
    b = c(__ldg(p + 1));
  }
  static __device__ __forceinline__ void load_cg(const void* base, size_t idx, Cx<DF>& a, Cx<DF>& b) {
    const float4* p = (const float4*)base + 2 * idx;
    a = c(p[0]);
    b = c(p[1]);
  }
  static __device__ __forceinline__ void store(void* base, size_t idx, Cx<DF> a, Cx<DF> b) {
    float4* p = (float4*)base + 2 * idx;
    p[0] = make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo);
    p[1] = make_float4(b.re.hi, b.re.lo, b.im.hi, b.im.lo);
  }
};

// block_reduce_store (fg_common.cuh) for double-float values (fixed tree, FP32 arithmetic only); the
// partials are stored as doubles.
template <int NV>
__device__ __forceinline__ void block_reduce_store_df(DF v[NV], double* __restrict__ partial,
                                                      int nblocks_stride) {
  __shared__ DF shd[NV][32];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    DF x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      x = x + DF(__shfl_down_sync(0xffffffffu, x.hi, o), __shfl_down_sync(0xffffffffu, x.lo, o));
    if (lane == 0) shd[k][warp] = x;
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      DF x = lane < nwarps ? shd[k][lane] : DF(0.0f);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        x = x + DF(__shfl_down_sync(0xffffffffu, x.hi, o), __shfl_down_sync(0xffffffffu, x.lo, o));
      if (lane == 0) partial[(size_t)k * nblocks_stride + blockIdx.x] = double(x);
    }
  }
}

// exp(i A) for Hermitian traceless A in double-float: the closed form of
// Morningstar and Peardon (Phys. Rev. D 69 (2004) 054501, section III),
// exp(iA) = f0 + f1 A + f2 A^2, as in the generic expi_herm, with the
// scalars computed to double-float accuracy on the FP32 pipes:
//   * 2u, the largest eigenvalue of A for c0 = det A >= 0 (negative c0 is
//     mapped through f_j(-c0) = (-1)^j conj(f_j(c0))), is a simple root of the
//     characteristic polynomial lambda^3 - c1 lambda - c0 separated from the
//     others by at least sqrt(c1); it starts from the FP32 angle formula and
//     takes two Newton steps in double-float (1e-7 -> 1e-14 -> rounding);
//   * w^2 = c1 - 3 u^2 (the eigenvalues are 2u and -u +- w, and
//     c1 = Tr A^2 / 2 = 3 u^2 + w^2), so cos w and sin(w)/w, the only
//     functions of w that enter, are even in w and need no angle;
//   * sin and cos by the double-float series above.
// Below c1 = 1e-12 (|A| < 1.5e-6) the exponential series to A^4 is used, with
// A^3 = c1 A + c0 and A^4 = c1 A^2 + c0 A (Cayley-Hamilton); the omitted
// terms are below |A|^5 / 120 < 1e-31.
template <>
__device__ __forceinline__ M3<DF> expi_herm<DF>(const M3<DF>& a) {
  const M3<DF> a2 = herm_sq(a);
  const DF c1 = (a2.e[0][0].re + a2.e[1][1].re + a2.e[2][2].re) * 0.5f;
  constexpr DF third(1.0 / 3.0), sixth(1.0 / 6.0), c24(1.0 / 24.0);
  const DF c0 = re_tr_mul(a, a2) * third;
  Cx<DF> f0, f1, f2;
  if (c1.hi < 1e-12f) {
    f0 = cx<DF>(DF(1.0f), -(c0 * sixth));
    f1 = cx<DF>(c0 * c24, DF(1.0f) - c1 * sixth);
    f2 = cx<DF>(DF(-0.5f) + c1 * c24, DF(0.0f));
  } else {
    const bool neg = c0.hi < 0.0f;
    const DF c0a = neg ? -c0 : c0;
    // FP32 seed: u = r cos(theta / 3), r = sqrt(c1 / 3), cos theta = c0 / (2 r^3)
    const float r32 = sqrtf(c1.hi * (1.0f / 3.0f));
    const float ratio = fminf(c0a.hi / (2.0f * r32 * r32 * r32), 1.0f);
    DF lam(2.0f * r32 * cosf(acosf(ratio) * (1.0f / 3.0f)));
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const DF l2 = lam * lam;
      const DF pv = (l2 - c1) * lam - c0a;
      const DF dp = l2 * 3.0f - c1;
      // the correction is ~1e-7 of lam or less: FP32 accuracy suffices
      lam = lam - DF(__fdiv_rn(pv.hi, dp.hi));
    }
    const DF u = lam * 0.5f;
    const DF u2 = u * u;
    DF w2 = c1 - u2 * 3.0f;
    if (w2.hi < 0.0f) w2 = DF(0.0f);
    const DF w = sqrt(w2);
    // sin and cos of u and of w through one copy of the series code (two
    // inlined copies cost instruction-cache misses in the force kernel)
    DF su, cu, sw, cw;
#pragma unroll 1
    for (int i = 0; i < 2; ++i) {
      DF sv, cv;
      sincos(i ? w : u, &sv, &cv);
      if (i) {
        sw = sv;
        cw = cv;
      } else {
        su = sv;
        cu = cv;
      }
    }
    DF xi0;
    if (w2.hi < 0.0025f) {
      // |w| < 0.05: sin(w)/w from its series in w^2 (first omitted term
      // below 3e-21), not from a quotient of small numbers
      constexpr DF x2(-1.0 / 6.0), x4(1.0 / 120.0), x6(-1.0 / 5040.0), x8(1.0 / 362880.0);
      DF q = fma(w2, x8, x6);
      q = fma(w2, q, x4);
      q = fma(w2, q, x2);
      xi0 = fma(w2, q, DF(1.0f));
    } else {
      xi0 = sw / w;
    }
    const DF s2u = (su * cu) * 2.0f;
    const DF c2u = (cu - su) * (cu + su);
    const Cx<DF> e2 = cx<DF>(c2u, s2u);
    const Cx<DF> em = cx<DF>(cu, -su);
    const DF u2x3 = u2 * 3.0f;
    const Cx<DF> h0 = cx<DF>(u2 - w2, DF(0.0f)) * e2 +
                      em * cx<DF>(u2 * cw * 8.0f, (u * (u2x3 + w2) * xi0) * 2.0f);
    const Cx<DF> h1 = cx<DF>(u * 2.0f, DF(0.0f)) * e2 - em * cx<DF>((u * cw) * 2.0f, -((u2x3 - w2) * xi0));
    const Cx<DF> h2 = e2 - em * cx<DF>(cw, (u * xi0) * 3.0f);
    const DF inv = DF(1.0f) / (u2 * 9.0f - w2);
    f0 = inv * h0;
    f1 = inv * h1;
    f2 = inv * h2;
    if (neg) {
      f0 = conj(f0);
      f1 = cx<DF>(-f1.re, f1.im);
      f2 = conj(f2);
    }
  }
  M3<DF> e;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<DF> s = f1 * a.e[i][j];
      cmac(s, f2, a2.e[i][j]);
      if (i == j) s = s + f0;
      e.e[i][j] = s;
    }
  return e;
}


// ---------------------------------------------------------------------------
// Products of SU(3) matrices in double-float with an anchored accumulator.
// For unitary a and b every partial sum of the real or imaginary part of an
// entry of a b lies in [-1, 1] (each term is bounded by |a_ik| |b_kj| and
// those sum to at most |row i of a| |column j of b| = 1, Cauchy-Schwarz), so
// t = 3 + (partial sum) stays in [2, 4], where the FP32 grid is 2^-22.  A
// term x_h y_h enters t by one FMA; its rounding error
// rho = t_old + x_h y_h - t_new (|rho| <= 2^-23) is recovered by a second FMA,
// fma(x_h, y_h, t_old - t_new), whose operand t_old - t_new is exact
// (Sterbenz's lemma) and whose result is within 2^-24 |rho| <= 2^-47 of rho;
// the low parts enter as x_h y_l + x_l y_h in FP32.  The value is
// (t - 3) + lo, t - 3 being exact, normalised by two_sum: six FP32
// operations per term instead of the fifteen of a double-float FMA, at the
// same ~2^-47 accuracy.  Callers guarantee unitary factors (the links of a
// staple and products of them); other inputs lose accuracy gracefully as t
// leaves [2, 4].
struct Anchored {
  float t, lo;
  __device__ __forceinline__ Anchored() : t(3.0f), lo(0.0f) {}
  // += x y
  __device__ __forceinline__ void add(DF x, DF y) {
    const float t0 = t;
    t = __fmaf_rn(x.hi, y.hi, t0);
    lo = __fadd_rn(lo, __fmaf_rn(x.hi, y.hi, __fsub_rn(t0, t)));
    lo = __fmaf_rn(x.hi, y.lo, lo);
    lo = __fmaf_rn(x.lo, y.hi, lo);
  }
  // -= x y
  __device__ __forceinline__ void sub(DF x, DF y) { add(-x, y); }
  __device__ __forceinline__ DF value() const { return df_two_sum(__fsub_rn(t, 3.0f), lo); }
};

// m^dagger if d, else m (run-time choice by selects, so that one code path
// serves both).
__device__ __forceinline__ M3<DF> dagger_if(const M3<DF>& m, bool d) {
  M3<DF> r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const Cx<DF> v = d ? m.e[j][i] : m.e[i][j];
      r.e[i][j] = cx<DF>(v.re, d ? -v.im : v.im);
    }
  return r;
}

// a b, a b^dagger and a^dagger b for unitary double-float matrices.
__device__ __forceinline__ M3<DF> su3_mul(const M3<DF>& a, const M3<DF>& b) {
  M3<DF> c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Anchored re, im;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        re.add(a.e[i][k].re, b.e[k][j].re);
        re.sub(a.e[i][k].im, b.e[k][j].im);
        im.add(a.e[i][k].re, b.e[k][j].im);
        im.add(a.e[i][k].im, b.e[k][j].re);
      }
      c.e[i][j] = cx<DF>(re.value(), im.value());
    }
  return c;
}
__device__ __forceinline__ M3<DF> su3_mul_nd(const M3<DF>& a, const M3<DF>& b) {
  M3<DF> c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Anchored re, im;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        re.add(a.e[i][k].re, b.e[j][k].re);
        re.add(a.e[i][k].im, b.e[j][k].im);
        im.add(a.e[i][k].im, b.e[j][k].re);
        im.sub(a.e[i][k].re, b.e[j][k].im);
      }
      c.e[i][j] = cx<DF>(re.value(), im.value());
    }
  return c;
}
__device__ __forceinline__ M3<DF> su3_mul_dn(const M3<DF>& a, const M3<DF>& b) {
  M3<DF> c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Anchored re, im;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        re.add(a.e[k][i].re, b.e[k][j].re);
        re.add(a.e[k][i].im, b.e[k][j].im);
        im.add(a.e[k][i].re, b.e[k][j].im);
        im.sub(a.e[k][i].im, b.e[k][j].re);
      }
      c.e[i][j] = cx<DF>(re.value(), im.value());
    }
  return c;
}


}  // namespace fg
