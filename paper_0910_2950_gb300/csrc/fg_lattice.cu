// Host runtime behind the C ABI of include/fg_lattice.h.
//
// A handle owns the device fields of one lattice in checkerboard SoA order
// (see fg_common.cuh), one CUDA stream, and a small pinned host buffer for
// the scalars that cross back to the host (dH and the action sums).  The
// integrator sequencer turns one MD step of Table 1 / section 3 into a list
// of kicks (P), drifts (Q) and force-gradient kicks (G), merges adjacent
// kicks and adjacent drifts of neighbouring steps, and launches it as fused
// kernels: a kick followed by a drift is one launch (force, kick, drift of
// the same link, written to a second link buffer); a force-gradient kick is
// one launch that displaces the links along the force and one that kicks
// with the force at the displaced links (then drifts, if a drift follows).
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "../../include/fg_lattice.h"
#include "fg_kernels.h"
#include "fg_runtime.h"
#include "host_wait.h"

namespace fg {

const char* kKernelClasses[] = {"gauge_force", "drift", "energy", "reduce", "momenta",
                                "dslash", "cg_blas", "fermion_force", "convert", "dslash_fp64",
                                "dslash_df"};

// ---------------------------------------------------------------------------
// Integrator sequences (Table 1 and section 3).
std::vector<Op> step_ops(int integ, double alpha) {
  std::vector<Op> v;
  switch (integ) {
    case FG_LEAPFROG:
      v = {{'P', 0.5, 0}, {'Q', 1.0, 0}, {'P', 0.5, 0}};
      break;
    case FG_QPQ:
      v = {{'Q', 0.5, 0}, {'P', 1.0, 0}, {'Q', 0.5, 0}};
      break;
    case FG_OMELYAN:
      v = {{'P', alpha, 0}, {'Q', 0.5, 0}, {'P', 1.0 - 2.0 * alpha, 0}, {'Q', 0.5, 0}, {'P', alpha, 0}};
      break;
    case FG_FORCE_GRADIENT:
      // middle: exp((48 dt S-hat - dt^3 {S,{S,T}}-hat)/72) -> kick 2/3 with the force
      // evaluated at links displaced by 2 (1/72) / (2/3) dt^2 = dt^2/24 along the force
      v = {{'P', 1.0 / 6.0, 0}, {'Q', 0.5, 0}, {'G', 2.0 / 3.0, 1.0 / 24.0}, {'Q', 0.5, 0},
           {'P', 1.0 / 6.0, 0}};
      break;
    case FG_FORCE_GRADIENT_ANALYTIC:
      // the same step with G in closed form: kick with F - (dt^2/24) G
      v = {{'P', 1.0 / 6.0, 0}, {'Q', 0.5, 0}, {'A', 2.0 / 3.0, 1.0 / 24.0}, {'Q', 0.5, 0},
           {'P', 1.0 / 6.0, 0}};
      break;
    case FG_CAMPOSTRINI: {
      const double w1 = 1.0 / (2.0 - std::cbrt(2.0));
      const double w0 = 1.0 - 2.0 * w1;
      v = {{'Q', w1 / 2, 0}, {'P', w1, 0}, {'Q', (w1 + w0) / 2, 0}, {'P', w0, 0},
           {'Q', (w1 + w0) / 2, 0}, {'P', w1, 0}, {'Q', w1 / 2, 0}};
      break;
    }
    default:
      break;
  }
  return v;
}

std::vector<Op> trajectory_ops(int integ, double alpha, int nsteps, bool merge) {
  std::vector<Op> out;
  const std::vector<Op> one = step_ops(integ, alpha);
  for (int n = 0; n < nsteps; ++n) {
    for (const Op& o : one) {
      if (merge && !out.empty() && out.back().kind == o.kind && (o.kind == 'P' || o.kind == 'Q')) {
        out.back().c += o.c;
      } else {
        out.push_back(o);
      }
    }
  }
  return out;
}

std::vector<Op> nested_trajectory_ops(int outer, int inner, double alpha, int n_inner, double dt, int nsteps) {
  std::vector<Op> out;
  auto kick = [&](double cg, double cf) {
    if (!out.empty() && out.back().kind == 'K') {
      out.back().c += cg;
      out.back().d += cf;
    } else {
      out.push_back({'K', cg, cf});
    }
  };
  auto drift = [&](double c) {
    if (!out.empty() && out.back().kind == 'Q') out.back().c += c;
    else out.push_back({'Q', c, 0});
  };
  const std::vector<Op> o_ops = step_ops(outer, alpha), i_ops = step_ops(inner, alpha);
  for (int n = 0; n < nsteps; ++n) {
    for (const Op& o : o_ops) {
      if (o.kind == 'P') {
        kick(0.0, o.c * dt);
      } else if (o.kind == 'G' || o.kind == 'A') {
        out.push_back({o.kind == 'G' ? 'f' : 'a', o.c * dt, o.d * dt * dt});
      } else {
        const double h = o.c * dt / n_inner;
        for (int k = 0; k < n_inner; ++k)
          for (const Op& i : i_ops) {
            if (i.kind == 'P') kick(i.c * h, 0.0);
            else if (i.kind == 'Q') drift(i.c * h);
            else out.push_back({i.kind == 'G' ? 'g' : 'h', i.c * h, i.d * h * h});
          }
      }
    }
  }
  return out;
}

int count_forces(const std::vector<Op>& ops) {
  int n = 0;
  for (const Op& o : ops)
    n += (o.kind == 'P' || o.kind == 'K') ? 1 : ((o.kind == 'Q') ? 0 : 2);
  return n;
}

// ---------------------------------------------------------------------------
// Kernel timing with CUDA events.
static cudaEvent_t pool_event(Timer& t) {
  if (t.used == t.pool.size()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    t.pool.push_back(e);
  }
  return t.pool[t.used++];
}
void Timer::begin(int cls, cudaStream_t st) {
  if (!on) return;
  Rec r;
  r.cls = cls;
  r.a = pool_event(*this);
  r.b = pool_event(*this);
  if (!r.a || !r.b) return;
  cudaEventRecord(r.a, st);
  recs.push_back(r);
}
void Timer::end(cudaStream_t st) {
  if (!on || recs.empty()) return;
  cudaEventRecord(recs.back().b, st);
}
void Timer::reset() {
  recs.clear();
  used = 0;
}
Timer::~Timer() {
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}
bool Timer::total(int cls, double* ms, long long* n) {
  double t = 0;
  long long c = 0;
  for (Rec& r : recs) {
    if (r.cls != cls) continue;
    float x = 0;
    if (cudaEventElapsedTime(&x, r.a, r.b) != cudaSuccess) return false;
    t += x;
    ++c;
  }
  *ms = t;
  *n = c;
  return true;
}

}  // namespace fg

using namespace fg;

// ---------------------------------------------------------------------------
// Bounded host waits (polling in host_wait.h).
namespace fg {
namespace {
double steady_seconds() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
void pause_us(double us) { std::this_thread::sleep_for(std::chrono::duration<double, std::micro>(us)); }
template <class QueryFn, class SyncFn>
fg_status wait_bounded(QueryFn query, SyncFn sync, double limit_s, std::string* why) {
  cudaError_t e = cudaSuccess;
  if (!(limit_s > 0.0)) {
    e = sync();
  } else {
    const WaitResult w = wait_limited(
        [&] {
          e = query();
          if (e == cudaErrorNotReady) {
            cudaGetLastError();   // not an error: clear it
            return 1;
          }
          return e == cudaSuccess ? 0 : 2;
        },
        steady_seconds, pause_us, limit_s);
    if (w == WAIT_TIMEOUT) {
      *why = "a host wait exceeded its limit of " + std::to_string(limit_s) + " s (work left queued)";
      return FG_ETIMEOUT;
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    *why = cudaGetErrorString(e);
    return FG_ECUDA;
  }
  return FG_OK;
}
}  // namespace

fg_status host_wait_stream(cudaStream_t st, double limit_s, std::string* why) {
  return wait_bounded([&] { return cudaStreamQuery(st); }, [&] { return cudaStreamSynchronize(st); }, limit_s, why);
}
fg_status host_wait_event(cudaEvent_t ev, double limit_s, std::string* why) {
  return wait_bounded([&] { return cudaEventQuery(ev); }, [&] { return cudaEventSynchronize(ev); }, limit_s, why);
}
}  // namespace fg

// ---------------------------------------------------------------------------
// C ABI.
#define FG_CHECK_HANDLE(h) \
  do {                     \
    if (!(h)) return FG_EINVAL; \
  } while (0)

extern "C" {

fg_status fg_params_default(fg_params* p) {
  if (!p) return FG_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->dims[0] = p->dims[1] = p->dims[2] = p->dims[3] = 4;
  p->beta = 6.0;
  p->kappa = 0.0;
  p->alpha = 0.1932;
  p->precision = FG_FP64;
  p->link_reals = 18;
  p->reunitarize = -1;
  p->cg_tol = 1e-10;
  p->cg_tol_action = 1e-12;
  p->cg_maxiter = 20000;
  p->cg_delta = 0.01;
  p->seed = 1;
  p->cuda_stream = nullptr;
  return FG_OK;
}

fg_status fg_fp32_fma_rate(double* tflops_out) {
  if (!tflops_out) return FG_EINVAL;
  *tflops_out = 0.0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    return FG_ECUDA;
  }
  const int blocks = 8 * sms, iters = 512;
  float* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  fg_status rc = FG_ECUDA;
  float best = 0.0f;
  if (cudaMalloc(&out, (size_t)blocks * 256 * sizeof(float)) != cudaSuccess ||
      cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    goto done;
  if (fg::launch_fma_rate(out, blocks, iters, st) != cudaSuccess) goto done;  // warm-up
  for (int k = 0; k < 5; ++k) {
    float ms = 0.0f;
    if (cudaEventRecord(e0, st) != cudaSuccess || fg::launch_fma_rate(out, blocks, iters, st) != cudaSuccess ||
        cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
      goto done;
    if (ms > 0.0f && (best == 0.0f || ms < best)) best = ms;
  }
  if (best > 0.0f) {
    const double flop = 2.0 * 8.0 * 16.0 * (double)iters * (double)blocks * 256.0;
    *tflops_out = flop / ((double)best * 1e-3) / 1e12;
    rc = FG_OK;
  }
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  if (out) cudaFree(out);
  if (rc != FG_OK) cudaGetLastError();
  return rc;
}

fg_status fg_lattice_create(const fg_params* p, fg_lattice** out) {
  if (!out) return FG_EINVAL;
  *out = nullptr;
  if (!p) return FG_EINVAL;
  for (int i = 0; i < 4; ++i)
    if (p->dims[i] < 2 || (p->dims[i] & 1)) return FG_EINVAL;
  const long long V = (long long)p->dims[0] * p->dims[1] * p->dims[2] * p->dims[3];
  if (V > (1LL << 28)) return FG_EINVAL;  // 32-bit element indices of links and momenta: 16 V - 1 < 2^32
  if (p->precision != FG_FP64 && p->precision != FG_FP32 && p->precision != FG_FP32_FP16CG &&
      p->precision != FG_DF64 && p->precision != FG_FP32_AUTOCG && p->precision != FG_FP32_BF16CG)
    return FG_EINVAL;
  if (p->precision == FG_DF64 && p->kappa != 0.0) return FG_EINVAL;  // double-float handles are pure gauge
  if (p->link_reals != 18 && p->link_reals != 12) return FG_EINVAL;
  if (!(p->beta >= 0.0) || !(p->kappa >= 0.0) || !(p->cg_tol > 0.0) || !(p->cg_tol_action > 0.0) ||
      p->cg_maxiter < 1 || !(p->cg_delta > 0.0 && p->cg_delta < 1.0))
    return FG_EINVAL;
  fg_lattice* h = new (std::nothrow) fg_lattice();
  if (!h) return FG_ENOMEM;
  h->prm = *p;
  if (h->prm.reunitarize < 0)
    h->prm.reunitarize =
        (p->precision == FG_FP32 || p->precision == FG_FP32_FP16CG || p->precision == FG_FP32_AUTOCG ||
         p->precision == FG_FP32_BF16CG)
            ? 1
            : 0;
  if (!(h->prm.alpha > 0.0)) h->prm.alpha = 0.1932;
  fg_status s = lattice_init(h);
  if (s != FG_OK) {
    delete h;
    return s;
  }
  *out = h;
  return FG_OK;
}

void fg_lattice_destroy(fg_lattice* h) {
  if (!h) return;
  delete h;
}

const char* fg_last_error(const fg_lattice* h) { return h ? h->err.c_str() : "null handle"; }

fg_status fg_set_gauge(fg_lattice* h, const double* x) {
  FG_CHECK_HANDLE(h);
  if (!x) return h->fail(FG_EINVAL, "null gauge pointer");
  return h->be->set_gauge(x);
}
fg_status fg_get_gauge(fg_lattice* h, double* x) {
  FG_CHECK_HANDLE(h);
  if (!x) return h->fail(FG_EINVAL, "null gauge pointer");
  return h->be->get_gauge(x);
}
fg_status fg_set_momenta(fg_lattice* h, const double* x) {
  FG_CHECK_HANDLE(h);
  if (!x) return h->fail(FG_EINVAL, "null momenta pointer");
  return h->be->set_momenta(x);
}
fg_status fg_get_momenta(fg_lattice* h, double* x) {
  FG_CHECK_HANDLE(h);
  if (!x) return h->fail(FG_EINVAL, "null momenta pointer");
  return h->be->get_momenta(x);
}
fg_status fg_refresh_momenta(fg_lattice* h) {
  FG_CHECK_HANDLE(h);
  return h->be->refresh_momenta();
}
fg_status fg_set_pseudofermion(fg_lattice* h, const double* chi) {
  FG_CHECK_HANDLE(h);
  if (!chi) return h->fail(FG_EINVAL, "null chi pointer");
  if (h->prm.kappa == 0.0) return h->fail(FG_ESTATE, "pure-gauge handle has no pseudofermion");
  return h->be->set_pseudofermion(chi);
}
fg_status fg_refresh_pseudofermion(fg_lattice* h) {
  FG_CHECK_HANDLE(h);
  if (h->prm.kappa == 0.0) return h->fail(FG_ESTATE, "pure-gauge handle has no pseudofermion");
  return h->be->refresh_pseudofermion();
}
fg_status fg_force(fg_lattice* h, double* f) {
  FG_CHECK_HANDLE(h);
  if (!f) return h->fail(FG_EINVAL, "null force pointer");
  return h->be->force(f);
}
fg_status fg_action(fg_lattice* h, double* sg, double* sf, double* t) {
  FG_CHECK_HANDLE(h);
  return h->be->action(sg, sf, t);
}
fg_status fg_plaquette(fg_lattice* h, double* plaq) {
  FG_CHECK_HANDLE(h);
  if (!plaq) return h->fail(FG_EINVAL, "null pointer");
  double sg = 0;
  fg_status s = h->be->gauge_action(&sg);
  if (s != FG_OK) return s;
  const double nplaq = 6.0 * h->g.V;
  *plaq = (h->prm.beta > 0) ? 1.0 - sg / (h->prm.beta * nplaq) : 0.0;
  if (h->prm.beta == 0) return h->fail(FG_EINVAL, "plaquette needs beta > 0");
  return FG_OK;
}
fg_status fg_md_step(fg_lattice* h, fg_integrator integ, double dt) {
  FG_CHECK_HANDLE(h);
  if ((int)integ < 0 || (int)integ > 5 || !std::isfinite(dt)) return h->fail(FG_EINVAL, "bad integrator or dt");
  return h->be->md_step((int)integ, dt);
}
fg_status fg_fg_step(fg_lattice* h, double dt) { return fg_md_step(h, FG_FORCE_GRADIENT, dt); }

fg_status fg_trajectory(fg_lattice* h, fg_integrator integ, double dt, double tau, int refresh,
                        double u_accept, fg_traj_result* out) {
  FG_CHECK_HANDLE(h);
  if ((int)integ < 0 || (int)integ > 5) return h->fail(FG_EINVAL, "bad integrator");
  if (!(dt > 0.0) || !(tau > 0.0)) return h->fail(FG_EINVAL, "dt and tau must be positive");
  const double ns = tau / dt;
  const int n = (int)std::llround(ns);
  if (n < 1 || std::fabs(n * dt - tau) > 1e-9 * tau) return h->fail(FG_EINVAL, "tau must be a multiple of dt");
  if (u_accept >= 1.0) return h->fail(FG_EINVAL, "u_accept must be < 1");
  fg_traj_result r;
  std::memset(&r, 0, sizeof(r));
  fg_status s = h->be->trajectory((int)integ, dt, n, refresh, u_accept, &r);
  if (out) *out = r;
  return s;
}
fg_status fg_trajectory_nested(fg_lattice* h, fg_integrator outer, fg_integrator inner, int n_inner, double dt,
                               double tau, int refresh, double u_accept, fg_traj_result* out) {
  FG_CHECK_HANDLE(h);
  if ((int)outer < 0 || (int)outer > 5 || (int)inner < 0 || (int)inner > 5)
    return h->fail(FG_EINVAL, "bad integrator");
  if (n_inner < 1) return h->fail(FG_EINVAL, "n_inner must be >= 1");
  if (!(dt > 0.0) || !(tau > 0.0)) return h->fail(FG_EINVAL, "dt and tau must be positive");
  const int n = (int)std::llround(tau / dt);
  if (n < 1 || std::fabs(n * dt - tau) > 1e-9 * tau) return h->fail(FG_EINVAL, "tau must be a multiple of dt");
  if (u_accept >= 1.0) return h->fail(FG_EINVAL, "u_accept must be < 1");
  fg_traj_result r;
  std::memset(&r, 0, sizeof(r));
  fg_status s = h->be->trajectory_nested((int)outer, (int)inner, n_inner, dt, n, refresh, u_accept, &r);
  if (out) *out = r;
  return s;
}
static fg_status host_momenta_trajectories(fg_lattice* h, fg_integrator integ, double dt, double tau, int n,
                                           const void* const* host_p8, int f32, const double* u_accept,
                                           fg_traj_result* out) {
  if ((int)integ < 0 || (int)integ > 5) return h->fail(FG_EINVAL, "bad integrator");
  if (!(dt > 0.0) || !(tau > 0.0)) return h->fail(FG_EINVAL, "dt and tau must be positive");
  const int ns = (int)std::llround(tau / dt);
  if (ns < 1 || std::fabs(ns * dt - tau) > 1e-9 * tau) return h->fail(FG_EINVAL, "tau must be a multiple of dt");
  if (n < 0) return h->fail(FG_EINVAL, "n must be >= 0");
  if (n > 0 && !host_p8) return h->fail(FG_EINVAL, "null momenta array");
  for (int k = 0; k < n; ++k) {
    if (!host_p8[k]) return h->fail(FG_EINVAL, "null momenta pointer");
    if (u_accept && !(u_accept[k] < 1.0)) return h->fail(FG_EINVAL, "u_accept must be < 1");
  }
  return h->be->trajectories_host_momenta((int)integ, dt, ns, n, host_p8, f32, u_accept, out);
}
fg_status fg_trajectories_host_momenta(fg_lattice* h, fg_integrator integ, double dt, double tau, int n,
                                       const double* const* host_p8, const double* u_accept,
                                       fg_traj_result* out) {
  FG_CHECK_HANDLE(h);
  return host_momenta_trajectories(h, integ, dt, tau, n, reinterpret_cast<const void* const*>(host_p8), 0,
                                   u_accept, out);
}
fg_status fg_trajectories_host_momenta_f32(fg_lattice* h, fg_integrator integ, double dt, double tau, int n,
                                           const float* const* host_p8, const double* u_accept,
                                           fg_traj_result* out) {
  FG_CHECK_HANDLE(h);
  return host_momenta_trajectories(h, integ, dt, tau, n, reinterpret_cast<const void* const*>(host_p8), 1,
                                   u_accept, out);
}
fg_status fg_apply_mhat(fg_lattice* h, const double* in, double* out, int dagger) {
  FG_CHECK_HANDLE(h);
  if (!in || !out) return h->fail(FG_EINVAL, "null spinor pointer");
  if (h->prm.kappa == 0.0) return h->fail(FG_ESTATE, "pure-gauge handle has no fermions");
  return h->be->apply_mhat(in, out, dagger);
}
fg_status fg_apply_mhat_inner(fg_lattice* h, const double* in, double* out, int dagger) {
  FG_CHECK_HANDLE(h);
  if (!in || !out) return h->fail(FG_EINVAL, "null spinor pointer");
  if (h->prm.kappa == 0.0) return h->fail(FG_ESTATE, "pure-gauge handle has no fermions");
  return h->be->apply_mhat_inner(in, out, dagger);
}
fg_status fg_cg_solve(fg_lattice* h, const double* b, double* x, fg_cg_result* res) {
  FG_CHECK_HANDLE(h);
  if (!b || !x) return h->fail(FG_EINVAL, "null spinor pointer");
  if (h->prm.kappa == 0.0) return h->fail(FG_ESTATE, "pure-gauge handle has no fermions");
  fg_cg_result r;
  std::memset(&r, 0, sizeof(r));
  fg_status s = h->be->cg_solve(b, x, &r);
  if (res) *res = r;
  return s;
}
fg_status fg_random_gauge(fg_lattice* h) {
  FG_CHECK_HANDLE(h);
  return h->be->random_gauge();
}
fg_status fg_set_rng_position(fg_lattice* h, unsigned long long pos) {
  FG_CHECK_HANDLE(h);
  return h->be->set_rng_position(pos);
}
fg_status fg_reunitarize(fg_lattice* h) {
  FG_CHECK_HANDLE(h);
  return h->be->reunitarize_all();
}
fg_status fg_timing_enable(fg_lattice* h, int on) {
  FG_CHECK_HANDLE(h);
  h->timer.on = on != 0;
  return FG_OK;
}
fg_status fg_timing_reset(fg_lattice* h) {
  FG_CHECK_HANDLE(h);
  std::string why;
  const fg_status s = host_wait_stream(h->st, h->wait_limit_s, &why);
  if (s != FG_OK) return h->fail(s, why);
  h->timer.reset();
  return FG_OK;
}
fg_status fg_kernel_time(fg_lattice* h, const char* cls, double* ms, long long* n) {
  FG_CHECK_HANDLE(h);
  if (!cls || !ms || !n) return h->fail(FG_EINVAL, "null argument");
  int id = -1;
  for (int i = 0; i < kNumKernelClasses; ++i)
    if (std::strcmp(cls, kKernelClasses[i]) == 0) id = i;
  if (id < 0) return h->fail(FG_EINVAL, "unknown kernel class");
  std::string why;
  const fg_status s = host_wait_stream(h->st, h->wait_limit_s, &why);
  if (s != FG_OK) return h->fail(s, why);
  if (!h->timer.total(id, ms, n)) return h->fail(FG_ECUDA, "event timing failed");
  return FG_OK;
}
long long fg_launch_count(const fg_lattice* h) { return h ? h->launches : -1; }
fg_status fg_sync(fg_lattice* h) {
  FG_CHECK_HANDLE(h);
  std::string why;
  const fg_status s = host_wait_stream(h->st, h->wait_limit_s, &why);
  if (s != FG_OK) return h->fail(s, why);
  return FG_OK;
}
fg_status fg_set_wait_limit(fg_lattice* h, double seconds) {
  FG_CHECK_HANDLE(h);
  if (!(seconds >= 0.0)) return h->fail(FG_EINVAL, "wait limit must be >= 0");
  h->wait_limit_s = seconds;
  return FG_OK;
}
unsigned long long fg_device_bytes(const fg_lattice* h) { return h ? h->dev_bytes : 0ULL; }

}  // extern "C"
