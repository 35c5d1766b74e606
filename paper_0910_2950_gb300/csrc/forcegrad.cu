// Closed-form force gradient (section 4): the derivative of the force along
// the vector field e^j(S) e_j, i.e. along the link tangent dU = i F U where F
// is the force itself (F = sum_a F^a lambda^a / 2).  The force-gradient kick
// of Table 1 then uses F - (dt^2/24) G exactly, instead of the force at
// displaced links.
//
//  * tangent_links_kernel: dU = i F U for every link (a general 3x3 matrix,
//    stored with all nine entries).
//  * force_tangent_kernel: the gauge part of G by the product rule through
//    the staples, G^a = (beta/6) Im Tr(lambda^a (dU_mu A_mu + U_mu dA_mu)),
//    plus an optional pseudofermion part computed elsewhere.
//  * kick_fg_kernel: P -= c (F - shift G).
//  * lincomb_kernel: out = a x + b y on spinor vectors (the pseudofermion part
//    of G is assembled from Dslash applications on U and on dU, see
//    backend.cu).
#include <cuda_runtime.h>

#include "fg_common.cuh"
#include "fg_fermion.h"
#include "fg_kernels.h"
#include "gauge_device.cuh"

namespace fg {

namespace {

Geom to_devg(const GeomH& h) {
  Geom g;
  for (int i = 0; i < 4; ++i) g.L[i] = h.L[i];
  g.Lxh = h.Lxh; g.Vh = h.Vh; g.V = h.V;
  g.dLxh = make_fastdiv((uint32_t)h.Lxh);
  g.dLy = make_fastdiv((uint32_t)h.L[1]);
  g.dLz = make_fastdiv((uint32_t)h.L[2]);
  return g;
}

constexpr int kSites = 64;
inline dim3 grid_of(int V) { return dim3((V + kSites - 1) / kSites); }
inline dim3 block_of() { return dim3(kSites, 4); }

template <typename R, int NC>
Gauge<R, NC> gauge_at(const void* p, int V) {
  Gauge<R, NC> u;
  u.p = const_cast<void*>(p);
  u.V = V;
  return u;
}
template <typename R>
Mom<R> mom_at(const void* p, int V) {
  Mom<R> m;
  m.p = const_cast<void*>(p);
  m.V = V;
  return m;
}

}  // namespace

template <typename R, int NC>
__global__ void __launch_bounds__(256) tangent_links_kernel(Gauge<R, NC> U, Mom<R> F, Gauge<R, 9> dU, int V) {
  const int s = blockIdx.x * kSites + threadIdx.x;
  const int mu = threadIdx.y;
  if (s >= V) return;
  R f[8];
  F.load(mu, s, f);
  const M3<R> fu = mul(alg_to_mat(f), U.load(mu, s));
  M3<R> d;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) d.e[i][j] = times_i(fu.e[i][j]);
  dU.store(mu, s, d);
}

// Staple sum A_mu(x) and its derivative dA_mu(x) along dU, term by term:
// upper (A B^dag) C^dag with A = U_nu(x+mu), B = U_mu(x+nu), C = U_nu(x);
// lower (P Q)^dag R with P = U_mu(x-nu), Q = U_nu(x+mu-nu), R = U_nu(x-nu).
template <typename R, int NC>
__device__ __forceinline__ void staple_sum_tangent(const Gauge<R, NC>& U, const Gauge<R, 9>& dU, const Geom& g,
                                                   const int c[4], int s, int mu, M3<R>& a, M3<R>& da) {
  zero(a);
  zero(da);
  // neighbours as half-index steps from s (see staple_sum)
  const int par = s >= g.Vh;
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
    {
      const int s_pnu = other + dp;
      const M3<R> A = U.load(nu, s_pmu), B = U.load(mu, s_pnu);
      const M3<R> dA = dU.load(nu, s_pmu), dB = dU.load(mu, s_pnu);
      const M3<R> t = mul_nd(A, B);
      M3<R> dt = mul_nd(dA, B);
      mac_nd(dt, A, dB);
      const M3<R> C = U.load(nu, s), dC = dU.load(nu, s);
      mac_nd(a, t, C);
      mac_nd(da, dt, C);
      mac_nd(da, t, dC);
    }
    {
      const int s_mnu = other + dm;
      const int s_pm = s + dm + dmu;
      const M3<R> P = U.load(mu, s_mnu), Q = U.load(nu, s_pm);
      const M3<R> dP = dU.load(mu, s_mnu), dQ = dU.load(nu, s_pm);
      const M3<R> t = mul(P, Q);
      M3<R> dt = mul(dP, Q);
      const M3<R> pdq = mul(P, dQ);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) dt.e[i][j] = dt.e[i][j] + pdq.e[i][j];
      const M3<R> Rm = U.load(nu, s_mnu), dR = dU.load(nu, s_mnu);
      mac_dn(a, t, Rm);
      mac_dn(da, dt, Rm);
      mac_dn(da, t, dR);
    }
  }
}

template <typename R, int NC>
__global__ void __launch_bounds__(256) force_tangent_kernel(Gauge<R, NC> U, Gauge<R, 9> dU, Mom<R> G, Mom<R> FFt,
                                                            Geom g, R beta6) {
  const int s = blockIdx.x * kSites + threadIdx.x;
  const int mu = threadIdx.y;
  if (s >= g.V) return;
  int c[4], par;
  cb_coords(g, s, c, par);
  M3<R> a, da;
  staple_sum_tangent(U, dU, g, c, s, mu, a, da);
  M3<R> w = mul(dU.load(mu, s), a);
  const M3<R> uda = mul(U.load(mu, s), da);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) w.e[i][j] = w.e[i][j] + uda.e[i][j];
  R f[8];
  im_tr_gellmann(w, f);
#pragma unroll
  for (int k = 0; k < 8; ++k) f[k] *= beta6;
  if (FFt.p != nullptr) {
    R ff[8];
    FFt.load(mu, s, ff);
#pragma unroll
    for (int k = 0; k < 8; ++k) f[k] += ff[k];
  }
  G.store(mu, s, f);
}

template <typename R>
__global__ void __launch_bounds__(256) kick_fg_kernel(Mom<R> P, Mom<R> F, Mom<R> G, int V, R c, R shift) {
  const int s = blockIdx.x * kSites + threadIdx.x;
  const int mu = threadIdx.y;
  if (s >= V) return;
  R p[8], f[8], gg[8];
  P.load(mu, s, p);
  F.load(mu, s, f);
  G.load(mu, s, gg);
#pragma unroll
  for (int k = 0; k < 8; ++k) p[k] = fma(-c, fma(-shift, gg[k], f[k]), p[k]);
  P.store(mu, s, p);
}

template <typename RO, typename RX, typename RY>
__global__ void __launch_bounds__(256) lincomb_kernel(typename Vec2<RO>::T* __restrict__ out, double a,
                                                     const typename Vec2<RX>::T* __restrict__ x, double b,
                                                     const typename Vec2<RY>::T* __restrict__ y, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const typename Vec2<RX>::T xv = x[i];
    double re = a * double(xv.x), im = a * double(xv.y);
    if (y != nullptr) {
      const typename Vec2<RY>::T yv = y[i];
      re += b * double(yv.x);
      im += b * double(yv.y);
    }
    typename Vec2<RO>::T o;
    o.x = RO(re);
    o.y = RO(im);
    out[i] = o;
  }
}

// ---------------------------------------------------------------------------
template <typename R, int NC>
cudaError_t launch_tangent_links(const GeomH& g, const void* U, const void* F, void* dU, cudaStream_t st) {
  tangent_links_kernel<R, NC><<<grid_of(g.V), block_of(), 0, st>>>(gauge_at<R, NC>(U, g.V), mom_at<R>(F, g.V),
                                                                    gauge_at<R, 9>(dU, g.V), g.V);
  return cudaGetLastError();
}
template <typename R, int NC>
cudaError_t launch_force_tangent(const GeomH& g, const void* U, const void* dU, void* G, const void* FFt,
                                 double beta, cudaStream_t st) {
  force_tangent_kernel<R, NC><<<grid_of(g.V), block_of(), 0, st>>>(
      gauge_at<R, NC>(U, g.V), gauge_at<R, 9>(dU, g.V), mom_at<R>(G, g.V), mom_at<R>(FFt, g.V), to_devg(g),
      R(beta / 6.0));
  return cudaGetLastError();
}
template <typename R>
cudaError_t launch_kick_fg(const GeomH& g, void* P, const void* F, const void* G, double c, double shift,
                           cudaStream_t st) {
  kick_fg_kernel<R><<<grid_of(g.V), block_of(), 0, st>>>(mom_at<R>(P, g.V), mom_at<R>(F, g.V), mom_at<R>(G, g.V),
                                                         g.V, R(c), R(shift));
  return cudaGetLastError();
}
template <typename RO, typename RX, typename RY>
cudaError_t launch_lincomb(void* out, double a, const void* x, double b, const void* y, int n, cudaStream_t st) {
  const int blocks = (n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8;
  lincomb_kernel<RO, RX, RY><<<blocks, 256, 0, st>>>((typename Vec2<RO>::T*)out, a,
                                                      (const typename Vec2<RX>::T*)x, b,
                                                      (const typename Vec2<RY>::T*)y, n);
  return cudaGetLastError();
}

#define FG_INST_TG(R, NC)                                                                                   \
  template cudaError_t launch_tangent_links<R, NC>(const GeomH&, const void*, const void*, void*, cudaStream_t); \
  template cudaError_t launch_force_tangent<R, NC>(const GeomH&, const void*, const void*, void*, const void*, \
                                                   double, cudaStream_t);
FG_INST_TG(double, 9)
FG_INST_TG(double, 6)
FG_INST_TG(float, 9)
FG_INST_TG(float, 6)
FG_INST_TG(DF, 9)
FG_INST_TG(DF, 6)
template cudaError_t launch_kick_fg<DF>(const GeomH&, void*, const void*, const void*, double, double, cudaStream_t);
template cudaError_t launch_kick_fg<double>(const GeomH&, void*, const void*, const void*, double, double,
                                            cudaStream_t);
template cudaError_t launch_kick_fg<float>(const GeomH&, void*, const void*, const void*, double, double,
                                           cudaStream_t);
template cudaError_t launch_lincomb<double, double, double>(void*, double, const void*, double, const void*, int,
                                                            cudaStream_t);
template cudaError_t launch_lincomb<float, float, float>(void*, double, const void*, double, const void*, int,
                                                         cudaStream_t);
template cudaError_t launch_lincomb<double, float, float>(void*, double, const void*, double, const void*, int,
                                                          cudaStream_t);
template cudaError_t launch_lincomb<float, double, double>(void*, double, const void*, double, const void*, int,
                                                           cudaStream_t);

}  // namespace fg
