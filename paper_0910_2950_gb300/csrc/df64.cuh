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
  __host__ __device__ __forceinline__ DF(float h) : hi(h), lo(0.0f) {}
  __host__ __device__ __forceinline__ DF(int h) : hi((float)h), lo(0.0f) {}
  // Nearest double-float to a double (host or device; uses FP64 arithmetic).
  __host__ __device__ __forceinline__ explicit DF(double d) {
    hi = (float)d;
    lo = (float)(d - (double)hi);
  }
  __host__ __device__ __forceinline__ DF(float h, float l) : hi(h), lo(l) {}
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
__device__ __forceinline__ DF operator*(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// a * b + c with one normalisation.  The generic complex helpers call fma
// unqualified; the using-declaration keeps the float and double overloads
// visible next to this one.
using ::fma;
__device__ __forceinline__ DF fma(DF a, DF b, DF c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  const DF s = df_two_sum(p, c.hi);
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

// Storage: one complex double-float is a float4 (re.hi, re.lo, im.hi, im.lo),
// the same 16 bytes as a complex double; a pair of entries is two float4.
template <> struct Vec2<DF> { typedef float4 T; };
template <> struct Quad<DF> {
  static __device__ __forceinline__ Cx<DF> c(float4 v) { return cx<DF>(DF(v.x, v.y), DF(v.z, v.w)); }
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

}  // namespace fg
