// Shared device definitions for the force-gradient HMC kernels (sm_103a).
//
// Device layout of every field (structure of arrays, checkerboard order):
//   site index s = parity * Vh + lex / 2, parity = (x+y+z+t) & 1, Vh = V / 2,
//   so each parity half is contiguous and a warp of consecutive s touches
//   consecutive addresses for every component.
//   gauge   Cplx2[4 mu][NC][V]   NC = 9 complex entries (18 reals) or 6 (12 reals:
//                                rows 0-1, row 2 rebuilt as (row0 x row1)^*)
//   momenta Cplx2[4 mu][4][V]    Gell-Mann coefficient pairs (p0,p1) .. (p6,p7)
//   spinor  Cplx2[12][Vh]        spin-major (spin * 3 + colour), one parity
// where Cplx2 is float2 or double2 (re, im).
#pragma once

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
template <typename R> __device__ __forceinline__ M3<R> expi_herm(const M3<R>& a) {
  M3<R> a2 = mul(a, a);
  R c0 = re_tr_mul(a, a2) * R(1.0 / 3.0);
  R c1 = R(0.5) * (a2.e[0][0].re + a2.e[1][1].re + a2.e[2][2].re);
  Cx<R> f0, f1, f2;
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
    R xi0;
    if (fabs(w) < R(0.05)) xi0 = R(1) - w2 * R(1.0 / 6.0) * (R(1) - w2 * R(0.05) * (R(1) - w2 * R(1.0 / 42.0)));
    else xi0 = sin(w) / w;
    R s2u, c2u, su, cu, sw, cw;
    sincos(R(2) * u, &s2u, &c2u);
    sincos(u, &su, &cu);
    sincos(w, &sw, &cw);
    (void)sw;
    const Cx<R> e2 = cx<R>(c2u, s2u);
    const Cx<R> em = cx<R>(cu, -su);
    const Cx<R> h0 = (u2 - w2) * e2 + em * cx<R>(R(8) * u2 * cw, R(2) * u * (R(3) * u2 + w2) * xi0);
    const Cx<R> h1 = (R(2) * u) * e2 - em * cx<R>(R(2) * u * cw, -(R(3) * u2 - w2) * xi0);
    const Cx<R> h2 = e2 - em * cx<R>(cw, R(3) * u * xi0);
    const R inv = R(1) / (R(9) * u2 - w2);
    f0 = inv * h0; f1 = inv * h1; f2 = inv * h2;
    if (neg) { f0 = conj(f0); f1 = cx<R>(-f1.re, f1.im); f2 = conj(f2); }
  }
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

// Gram-Schmidt of rows 0-1 (norms in FP64), then row 2 from the cross product.
template <typename R> __device__ __forceinline__ void reunitarize(M3<R>& u) {
  double n0 = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j) n0 += double(u.e[0][j].re) * u.e[0][j].re + double(u.e[0][j].im) * u.e[0][j].im;
  const double in0 = rsqrt(n0);
#pragma unroll
  for (int j = 0; j < 3; ++j) u.e[0][j] = cx<R>(R(u.e[0][j].re * in0), R(u.e[0][j].im * in0));
  double pr = 0, pi = 0;  // <row0, row1>
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    pr += double(u.e[0][j].re) * u.e[1][j].re + double(u.e[0][j].im) * u.e[1][j].im;
    pi += double(u.e[0][j].re) * u.e[1][j].im - double(u.e[0][j].im) * u.e[1][j].re;
  }
  double r1[3][2];
  double n1 = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    r1[j][0] = u.e[1][j].re - (pr * u.e[0][j].re - pi * u.e[0][j].im);
    r1[j][1] = u.e[1][j].im - (pr * u.e[0][j].im + pi * u.e[0][j].re);
    n1 += r1[j][0] * r1[j][0] + r1[j][1] * r1[j][1];
  }
  const double in1 = rsqrt(n1);
#pragma unroll
  for (int j = 0; j < 3; ++j) u.e[1][j] = cx<R>(R(r1[j][0] * in1), R(r1[j][1] * in1));
  rebuild_row2(u);
}

// ---------------------------------------------------------------------------
// Lattice geometry in checkerboard order.
struct Geom {
  int L[4];     // Lx, Ly, Lz, Lt
  int Lxh;      // Lx / 2
  int Vh;       // V / 2
  int V;
};

__device__ __forceinline__ void cb_coords(const Geom& g, int s, int c[4], int& par) {
  par = s >= g.Vh;
  int i = s - par * g.Vh;
  const int xh = i % g.Lxh;
  i /= g.Lxh;
  c[1] = i % g.L[1];
  i /= g.L[1];
  c[2] = i % g.L[2];
  c[3] = i / g.L[2];
  c[0] = 2 * xh + ((c[1] + c[2] + c[3] + par) & 1);
}

__device__ __forceinline__ int cb_index(const Geom& g, const int c[4]) {
  const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
  const int lex = c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
  return par * g.Vh + (lex >> 1);
}

// Index of the neighbour x + d * mu-hat (d = +1 or -1), periodic.
__device__ __forceinline__ int cb_neighbor(const Geom& g, const int c[4], int mu, int d) {
  int n[4] = {c[0], c[1], c[2], c[3]};
  int v = n[mu] + d;
  v = v < 0 ? v + g.L[mu] : (v >= g.L[mu] ? v - g.L[mu] : v);
  n[mu] = v;
  return cb_index(g, n);
}
// x + d1 * mu1-hat + d2 * mu2-hat
__device__ __forceinline__ int cb_neighbor2(const Geom& g, const int c[4], int mu1, int d1, int mu2, int d2) {
  int n[4] = {c[0], c[1], c[2], c[3]};
  int v = n[mu1] + d1;
  n[mu1] = v < 0 ? v + g.L[mu1] : (v >= g.L[mu1] ? v - g.L[mu1] : v);
  v = n[mu2] + d2;
  n[mu2] = v < 0 ? v + g.L[mu2] : (v >= g.L[mu2] ? v - g.L[mu2] : v);
  return cb_index(g, n);
}

// ---------------------------------------------------------------------------
// Field access.
template <typename R, int NC> struct Gauge {
  typedef typename Vec2<R>::T C2;
  C2* __restrict__ p;
  int V;
  __device__ __forceinline__ M3<R> load(int mu, int s) const {
    M3<R> m;
    const C2* b = p + (size_t)mu * NC * V + s;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const C2 v = __ldg(b + (size_t)k * V);
      m.e[k / 3][k % 3] = cx<R>(v.x, v.y);
    }
    if (NC == 6) rebuild_row2(m);
    return m;
  }
  __device__ __forceinline__ void store(int mu, int s, const M3<R>& m) const {
    C2* b = p + (size_t)mu * NC * V + s;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      C2 v; v.x = m.e[k / 3][k % 3].re; v.y = m.e[k / 3][k % 3].im;
      b[(size_t)k * V] = v;
    }
  }
};

template <typename R> struct Mom {
  typedef typename Vec2<R>::T C2;
  C2* __restrict__ p;
  int V;
  __device__ __forceinline__ void load(int mu, int s, R out[8]) const {
    const C2* b = p + (size_t)mu * 4 * V + s;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const C2 v = b[(size_t)k * V];
      out[2 * k] = v.x; out[2 * k + 1] = v.y;
    }
  }
  __device__ __forceinline__ void store(int mu, int s, const R in[8]) const {
    C2* b = p + (size_t)mu * 4 * V + s;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      C2 v; v.x = in[2 * k]; v.y = in[2 * k + 1];
      b[(size_t)k * V] = v;
    }
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

}  // namespace fg
