// Host runtime types shared by the C ABI (fg_lattice.cu) and the backends.
#pragma once

#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/fg_lattice.h"
#include "fg_kernels.h"

namespace fg {

// One sub-step of an integrator: 'P' kick exp(c dt S-hat), 'Q' drift
// exp(c dt T-hat), 'G' force-gradient kick with coefficient c and the force
// taken at links displaced by d dt^2 along the force.
// One operation of an integrator sequence, with coefficients in units of dt
// (c dt, d dt^2) when the list is run with a step size:
//   'P' kick with the total force, c;      'Q' drift, c;
//   'G' force-gradient kick on the total force (kick c, displacement d).
// Two-level (nested) lists carry absolute coefficients and also use
//   'K' kick with c times the gauge force plus d times the pseudofermion force;
//   'g' force-gradient kick on the gauge force alone;
//   'f' force-gradient kick on the pseudofermion force alone.
// 'A', 'a', 'h' are the closed-form versions of 'G', 'f', 'g' (the kick uses
// F - d G with G the derivative of the force along i F U, instead of the
// force at links displaced by d along the force).
struct Op {
  char kind;
  double c;
  double d;
};

std::vector<Op> step_ops(int integ, double alpha);
std::vector<Op> trajectory_ops(int integ, double alpha, int nsteps, bool merge);
// nsteps outer steps of `outer` (step dt) on the pseudofermion action whose
// drifts are n_inner steps of `inner` on the gauge action; absolute
// coefficients, adjacent kicks and drifts merged.
std::vector<Op> nested_trajectory_ops(int outer, int inner, double alpha, int n_inner, double dt, int nsteps);
int count_forces(const std::vector<Op>& ops);

enum KernelClass {
  KC_GAUGE_FORCE = 0, KC_DRIFT, KC_ENERGY, KC_REDUCE, KC_MOMENTA,
  KC_DSLASH, KC_CG_BLAS, KC_FERMION_FORCE, KC_CONVERT, KC_DSLASH64, KC_DSLASH_DF
};
constexpr int kNumKernelClasses = 11;
extern const char* kKernelClasses[];

// Per-launch CUDA-event timing.  Events come from a pool that grows on
// demand and is reused after reset(), so timing adds two event records per
// launch and no event creation in steady state.
struct Timer {
  struct Rec {
    int cls;
    cudaEvent_t a, b;
  };
  bool on = false;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  void begin(int cls, cudaStream_t st);
  void end(cudaStream_t st);
  void reset();
  bool total(int cls, double* ms, long long* n);
  ~Timer();
};

struct IBackend {
  virtual ~IBackend() {}
  virtual fg_status set_gauge(const double* host) = 0;
  virtual fg_status get_gauge(double* host) = 0;
  virtual fg_status set_momenta(const double* host) = 0;
  virtual fg_status get_momenta(double* host) = 0;
  virtual fg_status refresh_momenta() = 0;
  virtual fg_status set_pseudofermion(const double* chi) = 0;
  virtual fg_status refresh_pseudofermion() = 0;
  virtual fg_status force(double* host_f8) = 0;
  virtual fg_status gauge_action(double* sg) = 0;
  virtual fg_status action(double* sg, double* sf, double* t) = 0;
  virtual fg_status md_step(int integ, double dt) = 0;
  virtual fg_status trajectory(int integ, double dt, int nsteps, int refresh, double u_accept,
                               fg_traj_result* r) = 0;
  virtual fg_status trajectory_nested(int outer, int inner, int n_inner, double dt, int nsteps, int refresh,
                                      double u_accept, fg_traj_result* r) = 0;
  // host_p8[k]: n canonical momentum arrays, FP64 (f32 = 0) or FP32 (f32 = 1)
  virtual fg_status trajectories_host_momenta(int integ, double dt, int nsteps, int n, const void* const* host_p8,
                                              int f32, const double* u_accept, fg_traj_result* out) = 0;
  virtual fg_status apply_mhat(const double* in, double* out, int dagger) = 0;
  virtual fg_status apply_mhat_inner(const double* in, double* out, int dagger) = 0;
  virtual fg_status cg_solve(const double* b, double* x, fg_cg_result* r) = 0;
  virtual fg_status reunitarize_all() = 0;
  virtual fg_status random_gauge() = 0;
  virtual fg_status set_rng_position(unsigned long long pos) = 0;
};

}  // namespace fg

struct fg_lattice {
  fg_params prm;
  fg::GeomH g;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::string err;
  std::unique_ptr<fg::IBackend> be;
  fg::Timer timer;
  long long launches = 0;
  unsigned long long dev_bytes = 0;
  unsigned long long accept_draws = 0;
  double wait_limit_s = 0.0;   // limit on host waits (0: none), fg_set_wait_limit
  fg_status fail(fg_status s, const std::string& m) {
    err = m;
    return s;
  }
  ~fg_lattice();
};

namespace fg {
// Creates the stream and the backend for h->prm (defined in backend.cu).
fg_status lattice_init(fg_lattice* h);
// Host waits for a stream or an event, bounded by limit_s seconds (0 or
// less: unbounded): FG_OK, FG_ETIMEOUT (work left queued) or FG_ECUDA, with
// a description in *why (defined in fg_lattice.cu).
fg_status host_wait_stream(cudaStream_t st, double limit_s, std::string* why);
fg_status host_wait_event(cudaEvent_t ev, double limit_s, std::string* why);
}  // namespace fg
