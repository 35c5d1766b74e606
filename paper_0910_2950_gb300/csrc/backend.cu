// Backend<R, NC>: device fields of one lattice in precision R with NC complex
// entries stored per link, and the host-side sequencing of the kernels:
// the integrator executor (fused force kernels), the HMC trajectory with its
// FP64 dH, and for Nf = 2 Wilson fermions the CG driver, the pseudofermion
// heat bath and the pseudofermion force.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "df64.cuh"
#include "fg_common.cuh"
#include "fg_fermion.h"

#ifdef FG_CG_TRACE
#include <cstdio>
#define CG_TRACE(...) std::fprintf(stderr, __VA_ARGS__)
#else
#define CG_TRACE(...) ((void)0)
#endif
#include "fg_kernels.h"
#include "fg_runtime.h"

namespace fg {

// Host-visible scalars written by kernels (pinned, mapped memory).
struct Mapped {
  double bb;
  double true_rr;
  int dev_iter;     // last completed CG iteration (device numbering)
  int pad_i;
  double rr0;       // |b - M x0|^2 at the start of a solve from an initial guess
  double pad[4];
  double hist[1];   // residual history, one entry per CG iteration (allocated longer)
};

template <typename R, int NC>
class Backend final : public IBackend {
 public:
  typedef typename Vec2<R>::T C2;

  explicit Backend(fg_lattice* h) : h_(h), g_(h->g), st_(h->st), ferm_(h->prm.kappa > 0.0) {}

  ~Backend() override {
    for (void* p : allocs_) cudaFree(p);
    if (host_out_) cudaFreeHost(host_out_);
    if (mapped_) cudaFreeHost(mapped_);
    for (int i = 0; i < 2; ++i) {
      if (ev_[i]) cudaEventDestroy(ev_[i]);
      if (ev_copied_[i]) cudaEventDestroy(ev_copied_[i]);
      if (ev_read_[i]) cudaEventDestroy(ev_read_[i]);
    }
    if (cs_) cudaStreamDestroy(cs_);
    for (const CgGraph& c : cg_graphs_) cudaGraphExecDestroy(c.exec);
  }

  fg_status init() {
    const size_t V = (size_t)g_.V;
    const size_t mom_bytes = (size_t)4 * 4 * V * sizeof(C2);
    fg_status s;
    for (int b = 0; b < 3; ++b)
      if ((s = alloc(&buf_[b], gauge_bytes())) != FG_OK) return s;
    U_ = buf_[0];
    if ((s = alloc(&P_, mom_bytes)) != FG_OK) return s;
    if ((s = alloc(&F_, mom_bytes)) != FG_OK) return s;
    if ((s = alloc((void**)&h0_, V * sizeof(double))) != FG_OK) return s;
    for (int k = 0; k < 2; ++k)
      if ((s = alloc((void**)&sgc_[k], V * sizeof(double))) != FG_OK) return s;
    const size_t nb = (V + 255) / 256 + 1;
    if ((s = alloc((void**)&partial_, 4 * nb * sizeof(double))) != FG_OK) return s;
    if ((s = alloc((void**)&dout_, 32 * sizeof(double))) != FG_OK) return s;
    if (cudaMallocHost((void**)&host_out_, 32 * sizeof(double)) != cudaSuccess) {
      host_out_ = nullptr;
      return h_->fail(FG_ENOMEM, "pinned host allocation failed");
    }
    if (cudaMemsetAsync(P_, 0, mom_bytes, st_) != cudaSuccess) return cuda_fail("memset");
    if (ferm_ && (s = init_fermions()) != FG_OK) return s;
    s = run(KC_CONVERT, [&] { return launch_unit_links<R, NC>(g_, U_, st_); });
    if (s != FG_OK) return s;
    return sync();
  }

  // ---------------------------------------------------------------- I/O
  fg_status set_gauge(const double* host) override {
    const size_t n = (size_t)4 * g_.V * 18;
    fg_status s = ensure_canon(n);
    if (s != FG_OK) return s;
    if (cudaMemcpyAsync(canon_, host, n * sizeof(double), cudaMemcpyHostToDevice, st_) != cudaSuccess)
      return cuda_fail("gauge upload");
    s = run(KC_CONVERT, [&] { return launch_gauge_to_device<R, NC>(g_, canon_, U_, st_); });
    if (s != FG_OK) return s;
    sf0_valid_ = false;
    sgc_valid_ = false;
    return sync();
  }
  fg_status get_gauge(double* host) override {
    const size_t n = (size_t)4 * g_.V * 18;
    fg_status s = ensure_canon(n);
    if (s != FG_OK) return s;
    s = run(KC_CONVERT, [&] { return launch_gauge_to_canon<R, NC>(g_, U_, canon_, st_); });
    if (s != FG_OK) return s;
    if (cudaMemcpyAsync(host, canon_, n * sizeof(double), cudaMemcpyDeviceToHost, st_) != cudaSuccess)
      return cuda_fail("gauge download");
    return sync();
  }
  fg_status set_momenta(const double* host) override {
    const size_t n = (size_t)4 * g_.V * 8;
    fg_status s = ensure_canon(n);
    if (s != FG_OK) return s;
    if (cudaMemcpyAsync(canon_, host, n * sizeof(double), cudaMemcpyHostToDevice, st_) != cudaSuccess)
      return cuda_fail("momenta upload");
    s = run(KC_CONVERT, [&] { return launch_mom_to_device<R>(g_, canon_, P_, st_); });
    if (s != FG_OK) return s;
    return sync();
  }
  fg_status get_momenta(double* host) override { return download_mom(P_, host); }

  // n trajectories from host momenta: the upload of trajectory k+1's momenta
  // (into the other half of the canonical staging buffer, on a copy stream)
  // overlaps trajectory k on st_.  Each half is rewritten only after the
  // conversion that read it two trajectories earlier has run.
  fg_status trajectories_host_momenta(int integ, double dt, int nsteps, int n, const void* const* hp, int f32,
                                      const double* u, fg_traj_result* out) override {
    if (n <= 0) return FG_OK;
    const size_t nd = (size_t)4 * g_.V * 8;
    fg_status s = ensure_canon(2 * nd);
    if (s != FG_OK) return s;
    if ((s = ensure_copy_stream()) != FG_OK) return s;
    double* const stage[2] = {canon_, canon_ + nd};
    const size_t bytes = nd * (f32 ? sizeof(float) : sizeof(double));
    auto upload = [&](int j) -> fg_status {
      const int b = j & 1;
      if (j >= 2 && cudaStreamWaitEvent(cs_, ev_read_[b], 0) != cudaSuccess) return cuda_fail("stream wait");
      if (cudaMemcpyAsync(stage[b], hp[j], bytes, cudaMemcpyHostToDevice, cs_) != cudaSuccess)
        return cuda_fail("momenta upload");
      if (cudaEventRecord(ev_copied_[b], cs_) != cudaSuccess) return cuda_fail("event record");
      return FG_OK;
    };
    s = upload(0);
    for (int k = 0; s == FG_OK && k < n; ++k) {
      if (k + 1 < n && (s = upload(k + 1)) != FG_OK) break;
      const int b = k & 1;
      if (cudaStreamWaitEvent(st_, ev_copied_[b], 0) != cudaSuccess) {
        s = cuda_fail("stream wait");
        break;
      }
      s = run(KC_CONVERT, [&] {
        return f32 ? launch_mom_to_device_f32<R>(g_, reinterpret_cast<const float*>(stage[b]), P_, st_)
                   : launch_mom_to_device<R>(g_, stage[b], P_, st_);
      });
      if (s != FG_OK) break;
      if (cudaEventRecord(ev_read_[b], st_) != cudaSuccess) {
        s = cuda_fail("event record");
        break;
      }
      fg_traj_result r;
      std::memset(&r, 0, sizeof(r));
      s = trajectory(integ, dt, nsteps, 0, u ? u[k] : -1.0, &r);
      if (out) out[k] = r;
    }
    // no copy may read the caller's memory after the call returns
    const cudaError_t e = cudaStreamSynchronize(cs_);
    if (s == FG_OK && e != cudaSuccess) s = h_->fail(FG_ECUDA, cudaGetErrorString(e));
    return s;
  }

  fg_status refresh_momenta() override {
    const uint32_t d = draw_++;
    return run(KC_MOMENTA, [&] { return launch_refresh_momenta<R>(g_, P_, h_->prm.seed, d, st_); });
  }

  // ---------------------------------------------------------------- fermions (ABI)
  fg_status set_pseudofermion(const double* chi) override {
    if constexpr (!kFerm) {
      return no_fermions();
    } else {
      fg_status s = upload_spinor(chi, chi64_);
      if (s != FG_OK) return s;
      if ((s = heatbath_from_chi()) != FG_OK) return s;
      return sync();
    }
  }
  fg_status refresh_pseudofermion() override {
    if constexpr (!kFerm) {
      return no_fermions();
    } else {
      const uint32_t d = pf_draw_++;
      fg_status s = run(KC_MOMENTA, [&] { return launch_gaussian_spinor<double>(chi64_, g_.Vh, h_->prm.seed, d, st_); });
      if (s != FG_OK) return s;
      return heatbath_from_chi();
    }
  }
  fg_status apply_mhat(const double* in, double* out, int dagger) override {
    if constexpr (!kFerm) {
      return no_fermions();
    } else {
      fg_status s = upload_spinor(in, b64_);
      if (s != FG_OK) return s;
      if ((s = apply_mhat64(ax64_, b64_, U_, dagger)) != FG_OK) return s;
      return download_spinor(ax64_, out);
    }
  }
  // Mhat (or Mhat^dagger) by the inner solver's operator: the Dslash launches
  // of a CG iteration on vectors in the inner precision (FP32, or half
  // precision scaled by sigma with sigma^2 = |in|^2 / n on the half-precision
  // copy of the links), the input rounded to that precision and the output
  // widened to FP64.  FP64 handles iterate in FP64: apply_mhat.
  fg_status apply_mhat_inner(const double* in, double* out, int dagger) override {
    if constexpr (!kFerm) {
      return no_fermions();
    } else {
      if (!kMixed) return apply_mhat(in, out, dagger);
      const int n = nvec();
      const double k2 = h_->prm.kappa * h_->prm.kappa;
      fg_status s = upload_spinor(in, b64_);
      if (s != FG_OK) return s;
      const void* Uin = U_;
      if (half_links_) {
        const int nbv = vec_blocks(n);
        double* bbp = &mapped_->bb;
        if ((s = run(KC_CG_BLAS, [&] { return launch_dot64(b64_, b64_, part_rr_, n, st_); })) != FG_OK) return s;
        if ((s = run(KC_REDUCE, [&] { return launch_cg_init_h16(part_rr_, nbv, cgd_, 0.0, bbp, n, st_); })) != FG_OK)
          return s;
        if ((s = run(KC_CG_BLAS, [&] { return launch_scale_to_h16(s16_, rs_, b64_, cgd_, n, st_); })) != FG_OK) return s;
        if ((s = run(KC_CONVERT, [&] { return launch_links_to_half<NC>(s16_, g_, U_, U16_, st_); })) != FG_OK) return s;
        Uin = U16_;
      } else {
        if ((s = run(KC_CG_BLAS, [&] { return launch_convert<R, double>(rs_, b64_, nullptr, n, st_); })) != FG_OK)
          return s;
      }
      if ((s = run(KC_DSLASH, [&] {
             return inner_dslash(to_, rs_, nullptr, nullptr, Uin, 1, dagger, 0, 1.0, nullptr, false);
           })) != FG_OK)
        return s;
      if ((s = run(KC_DSLASH, [&] { return inner_dslash(te_, to_, rs_, nullptr, Uin, 0, dagger, 1, -k2, nullptr, false); })) !=
          FG_OK)
        return s;
      if (half_links_) s = run(KC_CONVERT, [&] { return launch_h16_to_double_scaled(s16_, ax64_, te_, cgd_, n, st_); });
      else s = run(KC_CONVERT, [&] { return launch_convert<double, R>(ax64_, te_, nullptr, n, st_); });
      if (s != FG_OK) return s;
      return download_spinor(ax64_, out);
    }
  }
  fg_status cg_solve(const double* b, double* x, fg_cg_result* r) override {
    if constexpr (!kFerm) {
      return no_fermions();
    } else {
      fg_status s = upload_spinor(b, b64_);
      if (s != FG_OK) return s;
      CgStats cs;
      s = cg(U_, b64_, h_->prm.cg_tol, &cs);
      r->iterations = cs.iters;
      r->reliable_updates = cs.nru;
      r->true_residual = cs.true_res;
      if (s != FG_OK) return s;
      return download_spinor(x64_, x);
    }
  }

  // ---------------------------------------------------------------- observables
  fg_status force(double* host_f8) override {
    ForceArgs a = force_args(U_);
    a.F = F_;
    fg_status s = force_launch(FM_STORE, a);
    if (s != FG_OK) return s;
    return download_mom(F_, host_f8);
  }

  fg_status gauge_action(double* sg) override {
    fg_status s = energy(2, nullptr, 0);
    if (s != FG_OK) return s;
    if ((s = fetch(3)) != FG_OK) return s;
    *sg = host_out_[0];
    return FG_OK;
  }

  fg_status action(double* sg, double* sf, double* t) override {
    fg_status s = energy(2, P_, 0);
    if (s != FG_OK) return s;
    if ((s = fetch(3)) != FG_OK) return s;
    if (sg) *sg = host_out_[0];
    if (t) *t = host_out_[1];
    double f = 0.0;
    if (ferm_ && sf) {
      if ((s = fermion_action(U_, &f)) != FG_OK) return s;
    }
    if (sf) *sf = f;
    return FG_OK;
  }

  fg_status reunitarize_all() override {
    fg_status s = run(KC_DRIFT, [&] { return launch_reunitarize<R, NC>(g_, U_, st_); });
    if (s != FG_OK) return s;
    sf0_valid_ = false;
    sgc_valid_ = false;
    return sync();
  }

  fg_status random_gauge() override {
    const uint32_t d = hot_draw_++;
    fg_status s = run(KC_CONVERT, [&] { return launch_random_links<R, NC>(g_, U_, h_->prm.seed, d, st_); });
    if (s != FG_OK) return s;
    sf0_valid_ = false;
    sgc_valid_ = false;
    return sync();
  }
  fg_status set_rng_position(unsigned long long pos) override {
    draw_ = (uint32_t)pos;
    pf_draw_ = (uint32_t)pos;
    h_->accept_draws = pos;
    return FG_OK;
  }

  // ---------------------------------------------------------------- MD
  fg_status md_step(int integ, double dt) override {
    std::vector<Op> ops = trajectory_ops(integ, h_->prm.alpha, 1, false);
    fg_status s = execute(ops, dt, nullptr);
    if (s != FG_OK) return s;
    sf0_valid_ = false;
    sgc_valid_ = false;
    return sync();
  }

  fg_status trajectory(int integ, double dt, int nsteps, int refresh, double u_accept,
                       fg_traj_result* r) override {
    return run_trajectory(trajectory_ops(integ, h_->prm.alpha, nsteps, true), dt, nsteps, refresh, u_accept, r);
  }

  fg_status trajectory_nested(int outer, int inner, int n_inner, double dt, int nsteps, int refresh,
                              double u_accept, fg_traj_result* r) override {
    return run_trajectory(nested_trajectory_ops(outer, inner, h_->prm.alpha, n_inner, dt, nsteps), 1.0, nsteps,
                          refresh, u_accept, r);
  }

  // Refresh, H at the start, the op list (coefficients times dt), H at the
  // end, Metropolis.
  fg_status run_trajectory(const std::vector<Op>& ops, double dt, int nsteps, int refresh, double u_accept,
                           fg_traj_result* r) {
    guess_ok_ = false;  // every trajectory starts its solves from zero
    fg_status s;
    solves_ = 0;
    cg_iters_ = 0;
    if (refresh) {
      if ((s = refresh_momenta()) != FG_OK) return s;
      if (ferm_ && (s = refresh_pseudofermion()) != FG_OK) return s;
    }
    double sf0 = 0.0;
    if (ferm_) {
      if (!sf0_valid_) {
        if ((s = fermion_action(U_, &sf0_)) != FG_OK) return s;
        sf0_valid_ = true;
      }
      sf0 = sf0_;
    }
    // H at the start: per-site energies kept for the site-by-site dH sum.
    // The per-site gauge action of these links was stored at the end of the
    // previous trajectory unless the links changed since; then only the
    // kinetic term is new.
    if ((s = energy(0, P_, 0, sgc_valid_ ? sgc_[sgc_cur_] : nullptr, sgc_valid_ ? nullptr : sgc_[sgc_cur_])) !=
        FG_OK)
      return s;
    // The start field is never written during the trajectory (see execute),
    // so a rejection only has to point back at it.
    void* const start = U_;
    // until the trajectory completes, the stored per-site action and S_F may
    // not match the current links (an error below leaves them moved)
    sgc_valid_ = false;
    sf0_valid_ = false;
    if ((s = execute(ops, dt, start)) != FG_OK) return s;
    if ((s = energy(1, P_, 3, nullptr, sgc_[1 - sgc_cur_])) != FG_OK) return s;
    if ((s = fetch(6)) != FG_OK) return s;
    double o[6];
    std::memcpy(o, host_out_, sizeof(o));
    double sf1 = 0.0;
    if (ferm_ && (s = fermion_action(U_, &sf1)) != FG_OK) return s;
    r->S_gauge0 = o[0];
    r->T0 = o[1];
    r->S_gauge1 = o[3];
    r->T1 = o[4];
    r->S_ferm0 = sf0;
    r->S_ferm1 = sf1;
    r->dH = o[5] + (sf1 - sf0);
    r->H0 = r->S_gauge0 + r->T0 + r->S_ferm0;
    r->H1 = r->S_gauge1 + r->T1 + r->S_ferm1;
    r->n_steps = nsteps;
    r->n_force = count_forces(ops);
    r->n_solves = solves_;
    r->cg_iters = cg_iters_;
    const double u = (u_accept < 0.0) ? host_uniform() : u_accept;
    r->accepted = std::isfinite(r->dH) && (r->dH <= 0.0 || u < std::exp(-r->dH));
    // the stored per-site gauge action follows the links kept
    if (r->accepted) sgc_cur_ = 1 - sgc_cur_;
    sgc_valid_ = true;
    if (!r->accepted) {
      U_ = start;
      sf0_ = sf0;             // phi unchanged and the links are back: S_F is S_F0 again
      sf0_valid_ = ferm_;
    } else {
      sf0_ = sf1;
      sf0_valid_ = ferm_;
    }
    return FG_OK;
  }

 private:
  struct CgStats {
    int iters = 0;
    int nru = 0;
    double true_res = 0.0;
  };

  fg_lattice* h_;
  GeomH g_;
  cudaStream_t st_;
  bool ferm_;
  std::vector<void*> allocs_;
  void* buf_[3] = {nullptr, nullptr, nullptr};   // link buffers; U_ is one of them
  void* U_ = nullptr;
  void* P_ = nullptr;
  void* F_ = nullptr;
  double* h0_ = nullptr;
  // per-site gauge action of the current links (sgc_[sgc_cur_]) and of the
  // end of the running trajectory (the other one); valid while only
  // trajectories have moved the links
  double* sgc_[2] = {nullptr, nullptr};
  int sgc_cur_ = 0;
  bool sgc_valid_ = false;
  double* partial_ = nullptr;
  double* dout_ = nullptr;
  double* canon_ = nullptr;
  size_t canon_n_ = 0;
  double* host_out_ = nullptr;
  uint32_t draw_ = 0;
  uint32_t pf_draw_ = 0;
  uint32_t hot_draw_ = 0;
  // fermions
  void *chi64_ = nullptr, *phi64_ = nullptr, *b64_ = nullptr, *x64_ = nullptr, *r64_ = nullptr;
  void *ax64_ = nullptr, *te64_ = nullptr, *to64_ = nullptr;
  // closed-form force gradient: tangent links (NC = 9), force, gradient and
  // pseudofermion-gradient momenta-layout fields, derivative spinors and
  // temporaries (allocated at the first analytic FG step)
  void *dU_ = nullptr, *Fa_ = nullptr, *G_ = nullptr, *FFt_ = nullptr;
  void *dXe_ = nullptr, *dXo_ = nullptr, *dYe_ = nullptr, *dYo_ = nullptr;
  void *Te1_ = nullptr, *Te2_ = nullptr, *To1_ = nullptr, *To2_ = nullptr;
  // double-float solution and source of the FP32 solver's reliable updates
  // (its Dslash temporaries reuse ax64_, te64_, to64_, which have the same size)
  void *xdf_ = nullptr, *bdf_ = nullptr;
  static constexpr bool kMixed = sizeof(R) < sizeof(double);
  // Double-float handles are pure gauge (fg_lattice_create rejects kappa > 0):
  // their fermion entry points are not compiled.
  static constexpr bool kFerm = !std::is_same<R, DF>::value;
  fg_status no_fermions() {
    return h_->fail(FG_ESTATE, "fermions need FG_FP64, FG_FP32, FG_FP32_FP16CG, FG_FP32_AUTOCG or FG_FP32_BF16CG");
  }
  // inner CG Dslash on a 16-bit copy of the links: IEEE half for
  // FG_FP32_FP16CG (and FG_FP32_AUTOCG above the L2 size), bfloat16 for
  // FG_FP32_BF16CG
  void* U16_ = nullptr;
  const bool half_links_ = kMixed && (h_->prm.precision == FG_FP32_FP16CG || h_->prm.precision == FG_FP32_BF16CG ||
                                      (h_->prm.precision == FG_FP32_AUTOCG && inner_exceeds_l2()));
  const int s16_ = h_->prm.precision == FG_FP32_BF16CG ? S16_BF16 : S16_HALF;
  // The FP32 inner solver's working set (links and six half-lattice spinor
  // vectors) against the GPU's L2 cache.
  bool inner_exceeds_l2() const {
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
      cudaGetLastError();
      return true;
    }
    const double bytes = (double)g_.V * (4.0 * NC * 8.0 + 6.0 * 48.0);
    return bytes > (double)l2;
  }
  // The same working set in this handle's precision (links and six
  // half-lattice vectors of R).
  bool solver_exceeds_l2() const {
    int dev = 0, l2 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
      cudaGetLastError();
      return true;
    }
    const double bytes = (double)g_.V * (4.0 * NC * 2.0 + 6.0 * 12.0) * (double)sizeof(R);
    return bytes > (double)l2;
  }
  void *xs_ = nullptr, *rs_ = nullptr, *p_ = nullptr, *ap_ = nullptr, *te_ = nullptr, *to_ = nullptr;
  // the folded iteration writes r' and p' to the other buffer of a pair;
  // rs_ and p_ always name the current ones
  void *rs2_ = nullptr, *p2_ = nullptr;
  // Folded CG iterations (four launches, vector updates inside the Dslash
  // launches) or six (four Dslash, axpy, xpay) for FP32 and FP64 inner
  // vectors.  The folded form forms p' at each of a site's eight neighbours,
  // reading r, Ap and p per hop, to save two streaming vector passes and two
  // launches.  While the solver's links and vectors fit in L2 the extra hop
  // reads hit L2 and the saved launches count (served 8^3 x 16 and
  // 12^3 x 24 chains; 16^3 x 32 FP32 within run-to-run spread: 8.9 against
  // 9.0 and 8.1 against 7.5 ms per solve on two fields); beyond L2 they
  // cost DRAM bandwidth (FP32 25.7 against 17.9 ms at 20^3 x 40, 38.8
  // against 34.2 at 24^3 x 48; FP64 at 16^3 x 32 61.7 against 56.6).
  // Default: folded when the fields fit in L2; FG_CG_FOLD=1 or 0 in the
  // environment forces either form.  The 16-bit solvers always take six
  // launches.
  const bool fold_ = [this] {
    const char* e = std::getenv("FG_CG_FOLD");
    if (e && e[0] == '1') return true;
    if (e && e[0] == '0') return false;
    return !solver_exceeds_l2();
  }() && !half_links_;
  void *Xe_ = nullptr, *Xo_ = nullptr, *Ye_ = nullptr, *Yo_ = nullptr, *FF_ = nullptr;
  CgDev* cgd_ = nullptr;
  double* part_pap_ = nullptr;
  double* part_rr_ = nullptr;
  double* part_b_ = nullptr;   // partials of |b|^2 for a solve from an initial guess
  // Chronological initial guess: within a trajectory every pseudofermion
  // solve has the same source phi at nearby links (a force-gradient
  // displacement moves them by dt^2/24 F), so a solve starts from the
  // previous solution instead of zero.  x64_ holds it while guess_ok_; the
  // guess is dropped at the start of every trajectory and whenever phi
  // changes, so a trajectory's result depends only on its own inputs.
  // FG_CG_GUESS=0 in the environment turns it off.
  bool guess_ok_ = false;
  const bool use_guess_ = [] {
    const char* e = std::getenv("FG_CG_GUESS");
    return !(e && e[0] == '0');
  }();
  Mapped* mapped_ = nullptr;
  cudaEvent_t ev_[2] = {nullptr, nullptr};
  // copy stream and its events for trajectories_host_momenta
  cudaStream_t cs_ = nullptr;
  cudaEvent_t ev_copied_[2] = {nullptr, nullptr};
  cudaEvent_t ev_read_[2] = {nullptr, nullptr};
  double sf0_ = 0.0;
  bool sf0_valid_ = false;
  int solves_ = 0;
  long long cg_iters_ = 0;

  size_t gauge_bytes() const { return (size_t)4 * NC * g_.V * sizeof(C2); }
  int nvec() const { return 12 * g_.Vh; }

  fg_status alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return h_->fail(FG_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    allocs_.push_back(*p);
    h_->dev_bytes += bytes;
    return FG_OK;
  }
  fg_status ensure_canon(size_t n) {
    if (canon_n_ >= n) return FG_OK;
    const size_t want = std::max(n, (size_t)4 * g_.V * 18);
    fg_status s = alloc((void**)&canon_, want * sizeof(double));
    if (s != FG_OK) return s;
    canon_n_ = want;
    return FG_OK;
  }
  fg_status ensure_copy_stream() {
    if (cs_) return FG_OK;
    if (cudaStreamCreateWithFlags(&cs_, cudaStreamNonBlocking) != cudaSuccess) {
      cs_ = nullptr;
      return cuda_fail("copy stream");
    }
    for (int i = 0; i < 2; ++i)
      if (cudaEventCreateWithFlags(&ev_copied_[i], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&ev_read_[i], cudaEventDisableTiming) != cudaSuccess)
        return cuda_fail("event");
    return FG_OK;
  }
  fg_status cuda_fail(const char* what) {
    cudaError_t e = cudaGetLastError();
    return h_->fail(FG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
  fg_status sync() {
    std::string why;
    const fg_status s = host_wait_stream(st_, h_->wait_limit_s, &why);
    if (s != FG_OK) return h_->fail(s, why);
    return FG_OK;
  }

  template <class Fn>
  fg_status run(int cls, Fn&& fn) {
    h_->timer.begin(cls, st_);
    cudaError_t e = fn();
    h_->timer.end(st_);
    ++h_->launches;
    if (e != cudaSuccess) return h_->fail(FG_ECUDA, std::string(kKernelClasses[cls]) + ": " + cudaGetErrorString(e));
    return FG_OK;
  }

  fg_status download_mom(const void* src, double* host) {
    const size_t n = (size_t)4 * g_.V * 8;
    fg_status s = ensure_canon(n);
    if (s != FG_OK) return s;
    s = run(KC_CONVERT, [&] { return launch_mom_to_canon<R>(g_, src, canon_, st_); });
    if (s != FG_OK) return s;
    if (cudaMemcpyAsync(host, canon_, n * sizeof(double), cudaMemcpyDeviceToHost, st_) != cudaSuccess)
      return cuda_fail("momenta download");
    return sync();
  }

  // energy kernel + fixed-order reduction into dout_[off .. off+2]
  fg_status energy(int mode, const void* P, int off, const double* sg_in = nullptr, double* sg_out = nullptr) {
    int nb = 0;
    fg_status s = run(KC_ENERGY, [&] {
      return launch_energy<R, NC>(g_, U_, P, h_->prm.beta, mode, h0_, partial_, &nb, st_, sg_in, sg_out);
    });
    if (s != FG_OK) return s;
    return run(KC_REDUCE, [&] { return launch_reduce(partial_, nb, 3, dout_ + off, 0, st_); });
  }
  fg_status fetch(int n) {
    if (cudaMemcpyAsync(host_out_, dout_, n * sizeof(double), cudaMemcpyDeviceToHost, st_) != cudaSuccess)
      return cuda_fail("result download");
    return sync();
  }

  ForceArgs force_args(const void* Uf) {
    ForceArgs a;
    std::memset(&a, 0, sizeof(a));
    a.U = Uf;
    a.P = P_;
    a.Ubase = Uf;
    a.beta = h_->prm.beta;
    a.reunit = h_->prm.reunitarize;
    return a;
  }

  // Total force at a.U: the pseudofermion part (CG solve + force kernel) goes
  // into FF_, which the fused gauge-force kernel adds before it kicks, drifts,
  // displaces or stores.
  fg_status force_launch(int mode, ForceArgs a) {
    if (ferm_) {
      fg_status s = fermion_force(a.U, h_->prm.cg_tol);
      if (s != FG_OK) return s;
      a.FF = FF_;
    }
    return gauge_launch(mode, a);
  }
  // The fused gauge-force kernel with whatever a.FF holds (no solve).  With
  // split_exp_ (the default for double-float) the exponential of a
  // kick-and-drift or a displacement runs in a launch of its own after the
  // force (the same arithmetic, the same bits): the staple products and the
  // double-float exponential together overflow the instruction cache, and
  // the split takes 16-21% off a double-float trajectory, while FP32 runs 9%
  // faster fused.  FG_SPLIT_EXP=0 / =1 in the environment turns the split
  // off / on for any precision.
  const bool split_exp_ = [] {
    const char* e = std::getenv("FG_SPLIT_EXP");
    return e ? e[0] == '1' : std::is_same<R, DF>::value;
  }();
  fg_status gauge_launch(int mode, const ForceArgs& a) {
    if (split_exp_ && (mode == FM_KICK_DRIFT || mode == FM_DISPLACE)) {
      ForceArgs f = a;
      fg_status s;
      if (mode == FM_KICK_DRIFT) {
        if ((s = run(KC_GAUGE_FORCE, [&] { return launch_gauge_force<R, NC>(g_, FM_KICK, f, st_); })) != FG_OK)
          return s;
        return run(KC_DRIFT, [&] {
          return launch_drift<R, NC>(g_, a.Ubase, P_, a.Uout, a.cdrift, a.reunit, st_);
        });
      }
      f.F = F_;
      if ((s = run(KC_GAUGE_FORCE, [&] { return launch_gauge_force<R, NC>(g_, FM_STORE, f, st_); })) != FG_OK)
        return s;
      return run(KC_DRIFT, [&] { return launch_drift<R, NC>(g_, a.U, F_, a.Uout, -a.cdisp, 0, st_); });
    }
    return run(KC_GAUGE_FORCE, [&] { return launch_gauge_force<R, NC>(g_, mode, a, st_); });
  }

  fg_status ensure_fg_buffers() {
    if (dU_ != nullptr) return FG_OK;
    fg_status s;
    const size_t mom_bytes = (size_t)4 * 4 * g_.V * sizeof(C2);
    // NC = 9 layout: four pairs and a tail entry per link, 36 complex per site
    if ((s = alloc(&dU_, (size_t)4 * 9 * g_.V * sizeof(C2))) != FG_OK) return s;
    void** m[] = {&Fa_, &G_, &FFt_};
    for (void** q : m)
      if ((s = alloc(q, mom_bytes)) != FG_OK) return s;
    if (ferm_) {
      void** v[] = {&dXe_, &dXo_, &dYe_, &dYo_, &Te1_, &Te2_, &To1_, &To2_};
      for (void** q : v)
        if ((s = alloc(q, (size_t)nvec() * sizeof(C2))) != FG_OK) return s;
    }
    return FG_OK;
  }

  // Derivative of the pseudofermion force along the tangent links dU_ into
  // FFt_ (section 4).  Needs the state of the fermion_force(U) call just
  // before it: X_e (Xe_, and x64_), X_o = D_oe X_e, Y_e = Mhat X_e,
  // Y_o = D_oe^dag Y_e.  With X = calM^{-1} phi its derivative is
  // -calM^{-1} F(calM) X (one more solve); X~ = (X_e, X_o) and
  // Y~ = (Y_e, Y_o) move with it and with the links, and the force's
  // bilinear form is differentiated in each argument in turn.
  fg_status fermion_force_tangent(const void* U, double tol) {
    if constexpr (!kFerm) {
      return no_fermions();
    } else {
      const int n = nvec();
      const double k2 = h_->prm.kappa * h_->prm.kappa;
      fg_status s;
      auto ds = [&](void* out, const void* in, const void* x, const void* links, bool tangent, int out_par, int dag,
                    int mode, double b) {
        return run(KC_DSLASH, [&] {
          return tangent ? launch_dslash<R, 9, R>(g_, out, in, x, nullptr, links, out_par, dag, mode, b, nullptr,
                                                  nullptr, st_)
                         : launch_dslash<R, NC, R>(g_, out, in, x, nullptr, links, out_par, dag, mode, b, nullptr,
                                                   nullptr, st_);
        });
      };
      auto lc = [&](auto launch) { return run(KC_CG_BLAS, launch); };
      // dMhat X_e = -k2 (dD_eo X_o + D_eo dD_oe X_e)
      if ((s = ds(To1_, Xe_, nullptr, dU_, true, 1, 0, 0, 1.0)) != FG_OK) return s;
      if ((s = ds(Te1_, Xo_, nullptr, dU_, true, 0, 0, 0, -k2)) != FG_OK) return s;
      if ((s = ds(dYe_, To1_, Te1_, U, false, 0, 0, 1, -k2)) != FG_OK) return s;
      // dMhat^dag Y_e = -k2 (dD^dag_eo Y_o + D^dag_eo dD^dag_oe Y_e); dD^dag_oe Y_e kept in dYo_
      if ((s = ds(dYo_, Ye_, nullptr, dU_, true, 1, 1, 0, 1.0)) != FG_OK) return s;
      if ((s = ds(Te1_, Yo_, nullptr, dU_, true, 0, 1, 0, -k2)) != FG_OK) return s;
      if ((s = ds(Te2_, dYo_, Te1_, U, false, 0, 1, 1, -k2)) != FG_OK) return s;
      // Mhat^dag (dMhat X_e)
      if ((s = ds(To2_, dYe_, nullptr, U, false, 1, 1, 0, 1.0)) != FG_OK) return s;
      if ((s = ds(Te1_, To2_, dYe_, U, false, 0, 1, 1, -k2)) != FG_OK) return s;
      // F(calM) X = dMhat^dag Y_e + Mhat^dag dMhat X_e, in FP64, and the solve
      if ((s = lc([&] { return launch_lincomb<double, R, R>(b64_, 1.0, Te1_, 1.0, Te2_, n, st_); })) != FG_OK) return s;
      CgStats cs;
      if ((s = cg(U, b64_, tol, &cs)) != FG_OK) return s;
      // dX_e = -calM^{-1} F(calM) X; dX_o = dD_oe X_e + D_oe dX_e
      if ((s = lc([&] { return launch_lincomb<R, double, double>(dXe_, -1.0, x64_, 0.0, nullptr, n, st_); })) != FG_OK)
        return s;
      if ((s = ds(To2_, dXe_, nullptr, U, false, 1, 0, 0, 1.0)) != FG_OK) return s;
      if ((s = lc([&] { return launch_lincomb<R, R, R>(dXo_, 1.0, To1_, 1.0, To2_, n, st_); })) != FG_OK) return s;
      // dY_e = dMhat X_e + Mhat dX_e; dY_o = dD^dag_oe Y_e + D^dag_oe dY_e
      if ((s = ds(Te1_, To2_, dXe_, U, false, 0, 0, 1, -k2)) != FG_OK) return s;
      if ((s = lc([&] { return launch_lincomb<R, R, R>(dYe_, 1.0, dYe_, 1.0, Te1_, n, st_); })) != FG_OK) return s;
      if ((s = ds(dYo_, dYe_, dYo_, U, false, 1, 1, 1, 1.0)) != FG_OK) return s;
      // the bilinear force form with the links, X~ and Y~ moved in turn
      auto ff = [&](const void* links, bool tangent, const void* xe, const void* xo, const void* ye, const void* yo,
                    int acc) {
        return run(KC_FERMION_FORCE, [&] {
          return tangent ? launch_fermion_force<R, 9, R>(g_, links, xe, xo, ye, yo, FFt_, k2, acc, st_)
                         : launch_fermion_force<R, NC, R>(g_, links, xe, xo, ye, yo, FFt_, k2, acc, st_);
        });
      };
      if ((s = ff(dU_, true, Xe_, Xo_, Ye_, Yo_, 0)) != FG_OK) return s;
      if ((s = ff(U, false, dXe_, dXo_, Ye_, Yo_, 1)) != FG_OK) return s;
      return ff(U, false, Xe_, Xo_, dYe_, dYo_, 1);
    }
  }

  // Closed-form force-gradient kick P -= c (F - shift G), G the derivative of
  // the force along i F U; the force is the gauge part, the pseudofermion
  // part, or both.
  fg_status analytic_fg_kick(double c, double shift, bool gauge, bool ferm) {
    fg_status s;
    if ((s = ensure_fg_buffers()) != FG_OK) return s;
    ferm = ferm && ferm_;
    if (!gauge && !ferm) return FG_OK;
    if (ferm && (s = fermion_force(U_, h_->prm.cg_tol)) != FG_OK) return s;
    const void* F = FF_;
    if (gauge) {
      ForceArgs a = force_args(U_);
      a.F = Fa_;
      a.FF = ferm ? FF_ : nullptr;
      if ((s = gauge_launch(FM_STORE, a)) != FG_OK) return s;
      F = Fa_;
    }
    const void* Ucur = U_;
    if ((s = run(KC_GAUGE_FORCE, [&] { return launch_tangent_links<R, NC>(g_, Ucur, F, dU_, st_); })) != FG_OK)
      return s;
    if (ferm && (s = fermion_force_tangent(U_, h_->prm.cg_tol)) != FG_OK) return s;
    const void* G = FFt_;
    if (gauge) {
      const void* fft = ferm ? FFt_ : nullptr;
      if ((s = run(KC_GAUGE_FORCE, [&] {
             return launch_force_tangent<R, NC>(g_, Ucur, dU_, G_, fft, h_->prm.beta, st_);
           })) != FG_OK)
        return s;
      G = G_;
    }
    return run(KC_MOMENTA, [&] { return launch_kick_fg<R>(g_, P_, F, G, c, shift, st_); });
  }

  // One of the three link buffers that is neither the current field nor the
  // protected one.
  void* free_buffer(const void* protect) const { return buffer_not(U_, protect); }
  void* buffer_not(const void* a, const void* b) const {
    for (void* c : buf_)
      if (c != a && c != b) return c;
    return nullptr;
  }

  // Runs a merged op list with fused kernels (see the file header of
  // fg_lattice.cu).  The links rotate through three buffers; the buffer
  // `protect` (the trajectory's start field, or null) is never written.
  fg_status execute(const std::vector<Op>& ops, double dt, const void* protect) {
    fg_status s;
    const size_t n = ops.size();
    for (size_t i = 0; i < n;) {
      const Op& o = ops[i];
      const bool next_q = (i + 1 < n) && ops[i + 1].kind == 'Q';
      if (o.kind == 'P') {
        ForceArgs a = force_args(U_);
        a.ckick = o.c * dt;
        if (next_q) {
          void* out = free_buffer(protect);
          a.cdrift = ops[i + 1].c * dt;
          a.Ubase = U_;
          a.Uout = out;
          if ((s = force_launch(FM_KICK_DRIFT, a)) != FG_OK) return s;
          U_ = out;
          i += 2;
        } else {
          if ((s = force_launch(FM_KICK, a)) != FG_OK) return s;
          i += 1;
        }
      } else if (o.kind == 'K') {
        // c dt times the gauge force plus d dt times the pseudofermion force
        const double cg = o.c * dt, cf = ferm_ ? o.d * dt : 0.0;
        if (cf != 0.0 && (s = fermion_force(U_, h_->prm.cg_tol)) != FG_OK) return s;
        if (cg == 0.0) {
          if (cf != 0.0 && (s = run(KC_MOMENTA, [&] { return launch_kick_ff<R>(g_, P_, FF_, cf, st_); })) != FG_OK)
            return s;
          i += 1;
          continue;
        }
        ForceArgs a = force_args(U_);
        a.ckick = cg;
        a.FF = (cf != 0.0) ? FF_ : nullptr;
        a.ffw = cf / cg;
        if (next_q) {
          void* out = free_buffer(protect);
          a.cdrift = ops[i + 1].c * dt;
          a.Ubase = U_;
          a.Uout = out;
          if ((s = gauge_launch(FM_KICK_DRIFT, a)) != FG_OK) return s;
          U_ = out;
          i += 2;
        } else {
          if ((s = gauge_launch(FM_KICK, a)) != FG_OK) return s;
          i += 1;
        }
      } else if (o.kind == 'f') {
        // force-gradient kick on the pseudofermion force alone: displace along
        // it (a drift with FF in place of P), evaluate it there, kick
        if (!ferm_) {
          i += 1;
          continue;
        }
        if ((s = fermion_force(U_, h_->prm.cg_tol)) != FG_OK) return s;
        void* disp = free_buffer(protect);
        const double cdisp = o.d * dt * dt;
        const void* in = U_;
        if ((s = run(KC_DRIFT, [&] {
               return launch_drift<R, NC>(g_, in, FF_, disp, -cdisp, h_->prm.reunitarize, st_);
             })) != FG_OK)
          return s;
        if ((s = fermion_force(disp, h_->prm.cg_tol)) != FG_OK) return s;
        const double ck = o.c * dt;
        if ((s = run(KC_MOMENTA, [&] { return launch_kick_ff<R>(g_, P_, FF_, ck, st_); })) != FG_OK) return s;
        i += 1;
      } else if (o.kind == 'g') {
        // force-gradient kick on the gauge force alone
        void* disp = free_buffer(protect);
        ForceArgs d = force_args(U_);
        d.cdisp = o.d * dt * dt;
        d.Uout = disp;
        if ((s = gauge_launch(FM_DISPLACE, d)) != FG_OK) return s;
        ForceArgs a = force_args(disp);
        a.ckick = o.c * dt;
        if (next_q) {
          void* out = (U_ == protect) ? buffer_not(protect, disp) : U_;
          a.cdrift = ops[i + 1].c * dt;
          a.Ubase = U_;
          a.Uout = out;
          s = gauge_launch(FM_KICK_DRIFT, a);
          U_ = out;
          i += 2;
        } else {
          s = gauge_launch(FM_KICK, a);
          i += 1;
        }
        if (s != FG_OK) return s;
      } else if (o.kind == 'A' || o.kind == 'a' || o.kind == 'h') {
        // closed-form force-gradient kick: total ('A'), pseudofermion ('a')
        // or gauge ('h') force
        if ((s = analytic_fg_kick(o.c * dt, o.d * dt * dt, o.kind != 'a', o.kind != 'h')) != FG_OK) return s;
        i += 1;
      } else if (o.kind == 'Q') {
        void* out = (U_ == protect) ? free_buffer(protect) : U_;
        const void* in = U_;
        s = run(KC_DRIFT, [&] {
          return launch_drift<R, NC>(g_, in, P_, out, o.c * dt, h_->prm.reunitarize, st_);
        });
        if (s != FG_OK) return s;
        U_ = out;
        i += 1;
      } else {  // 'G': displace along the force, then kick with the force there
        void* disp = free_buffer(protect);
        ForceArgs d = force_args(U_);
        d.cdisp = o.d * dt * dt;
        d.Uout = disp;
        if ((s = force_launch(FM_DISPLACE, d)) != FG_OK) return s;
        ForceArgs a = force_args(disp);
        a.ckick = o.c * dt;
        if (next_q) {
          // the drift after the FG kick moves the current links; write it
          // in place unless they are the protected start field
          void* out = (U_ == protect) ? buffer_not(protect, disp) : U_;
          a.cdrift = ops[i + 1].c * dt;
          a.Ubase = U_;
          a.Uout = out;
          s = force_launch(FM_KICK_DRIFT, a);
          U_ = out;
          i += 2;
        } else {
          s = force_launch(FM_KICK, a);
          i += 1;
        }
        if (s != FG_OK) return s;
      }
    }
    return FG_OK;
  }

  double host_uniform() {
    uint32_t c[4] = {(uint32_t)h_->accept_draws, (uint32_t)(h_->accept_draws >> 32), 2u, 0u};
    ++h_->accept_draws;
    Philox::rounds(c, (uint32_t)h_->prm.seed, (uint32_t)(h_->prm.seed >> 32));
    const uint64_t bits = ((uint64_t)c[0] << 21) ^ ((uint64_t)c[1] >> 11);
    return (double)(bits & ((1ULL << 53) - 1)) * (1.0 / 9007199254740992.0);
  }

  // ---------------------------------------------------------------- fermion internals
  fg_status init_fermions() {
    if constexpr (!kFerm) {
      return no_fermions();
    } else {
      const size_t n = (size_t)nvec();
      const size_t b64 = n * sizeof(double2), bR = n * sizeof(C2);
      fg_status s;
      void** d64[] = {&chi64_, &phi64_, &b64_, &x64_, &r64_, &ax64_, &te64_, &to64_};
      for (void** p : d64)
        if ((s = alloc(p, b64)) != FG_OK) return s;
      if (kMixed) {
        if ((s = alloc(&xdf_, b64)) != FG_OK) return s;
        if ((s = alloc(&bdf_, b64)) != FG_OK) return s;
      }
      // two bytes per real, NC complex entries per link
      if (half_links_ && (s = alloc(&U16_, (size_t)4 * NC * g_.V * 4)) != FG_OK) return s;
      void** dR[] = {&xs_, &rs_, &p_, &ap_, &te_, &to_, &Xe_, &Xo_, &Ye_, &Yo_};
      for (void** p : dR)
        if ((s = alloc(p, bR)) != FG_OK) return s;
      if (fold_ && ((s = alloc(&rs2_, bR)) != FG_OK || (s = alloc(&p2_, bR)) != FG_OK)) return s;
      if ((s = alloc(&FF_, (size_t)4 * 4 * g_.V * sizeof(C2))) != FG_OK) return s;
      if ((s = alloc((void**)&cgd_, sizeof(CgDev))) != FG_OK) return s;
      if (cudaMemsetAsync(cgd_, 0, sizeof(CgDev), st_) != cudaSuccess) return cuda_fail("cg state init");
      if ((s = alloc((void**)&part_pap_, (3 * dslash_blocks(g_.Vh) + 1) * sizeof(double))) != FG_OK) return s;
      if ((s = alloc((void**)&part_rr_, (vec_blocks(nvec()) + 1) * sizeof(double))) != FG_OK) return s;
      if ((s = alloc((void**)&part_b_, (vec_blocks(nvec()) + 1) * sizeof(double))) != FG_OK) return s;
      const size_t mbytes = sizeof(Mapped) + (size_t)(h_->prm.cg_maxiter + 8) * sizeof(double);
      if (cudaHostAlloc((void**)&mapped_, mbytes, cudaHostAllocMapped) != cudaSuccess) {
        mapped_ = nullptr;
        return h_->fail(FG_ENOMEM, "mapped host allocation failed");
      }
      std::memset(mapped_, 0, mbytes);
      for (int i = 0; i < 2; ++i)
        if (cudaEventCreateWithFlags(&ev_[i], cudaEventDisableTiming) != cudaSuccess) return cuda_fail("event");
      if (cudaMemsetAsync(chi64_, 0, b64, st_) != cudaSuccess || cudaMemsetAsync(phi64_, 0, b64, st_) != cudaSuccess)
        return cuda_fail("memset");
      return FG_OK;
    }
  }

  fg_status upload_spinor(const double* host, void* dst64) {
    const size_t nd = (size_t)nvec() * 2;
    fg_status s = ensure_canon(nd);
    if (s != FG_OK) return s;
    if (cudaMemcpyAsync(canon_, host, nd * sizeof(double), cudaMemcpyHostToDevice, st_) != cudaSuccess)
      return cuda_fail("spinor upload");
    return run(KC_CONVERT, [&] { return launch_spinor_to_device<double>(canon_, dst64, g_.Vh, st_); });
  }
  fg_status download_spinor(const void* src64, double* host) {
    const size_t nd = (size_t)nvec() * 2;
    fg_status s = ensure_canon(nd);
    if (s != FG_OK) return s;
    s = run(KC_CONVERT, [&] { return launch_spinor_to_canon<double>(src64, canon_, g_.Vh, st_); });
    if (s != FG_OK) return s;
    if (cudaMemcpyAsync(host, canon_, nd * sizeof(double), cudaMemcpyDeviceToHost, st_) != cudaSuccess)
      return cuda_fail("spinor download");
    return sync();
  }

  // FP64 arithmetic on the stored links: out = Mhat in, or Mhat^dagger in.
  fg_status apply_mhat64(void* out, const void* in, const void* U, int dag) {
    const double k2 = h_->prm.kappa * h_->prm.kappa;
    fg_status s = run(KC_DSLASH64, [&] {
      return launch_dslash<R, NC, double>(g_, to64_, in, nullptr, nullptr, U, 1, dag, 0, 1.0, nullptr, nullptr, st_);
    });
    if (s != FG_OK) return s;
    return run(KC_DSLASH64, [&] {
      return launch_dslash<R, NC, double>(g_, out, to64_, in, nullptr, U, 0, dag, 1, -k2, nullptr, nullptr, st_);
    });
  }
  fg_status apply_mdagm64(void* out, const void* in, const void* U) {
    fg_status s = apply_mhat64(te64_, in, U, 0);
    if (s != FG_OK) return s;
    return apply_mhat64(out, te64_, U, 1);
  }

  // The same in double-float arithmetic on double-float vectors (FP32 links only).
  fg_status apply_mhat_df(void* out, const void* in, const void* U, int dag) {
    if constexpr (kMixed) {
      const double k2 = h_->prm.kappa * h_->prm.kappa;
      fg_status s = run(KC_DSLASH_DF, [&] {
        return launch_dslash<R, NC, DF>(g_, to64_, in, nullptr, nullptr, U, 1, dag, 0, 1.0, nullptr, nullptr, st_);
      });
      if (s != FG_OK) return s;
      return run(KC_DSLASH_DF, [&] {
        return launch_dslash<R, NC, DF>(g_, out, to64_, in, nullptr, U, 0, dag, 1, -k2, nullptr, nullptr, st_);
      });
    } else {
      return h_->fail(FG_ESTATE, "double-float Dslash needs FP32 links");
    }
  }
  fg_status apply_mdagm_df(void* out, const void* in, const void* U) {
    fg_status s = apply_mhat_df(te64_, in, U, 0);
    if (s != FG_OK) return s;
    return apply_mhat_df(out, te64_, U, 1);
  }

  // phi = Mhat^dagger chi at the current links; S_F at the heat bath = |chi|^2.
  fg_status heatbath_from_chi() {
    guess_ok_ = false;  // a new phi
    fg_status s = apply_mhat64(phi64_, chi64_, U_, 1);
    if (s != FG_OK) return s;
    if ((s = run(KC_CG_BLAS, [&] { return launch_dot64(chi64_, chi64_, part_rr_, nvec(), st_); })) != FG_OK) return s;
    const int nb = vec_blocks(nvec());
    if ((s = run(KC_REDUCE, [&] { return launch_reduce(part_rr_, nb, 1, dout_ + 8, 0, st_); })) != FG_OK) return s;
    if (cudaMemcpyAsync(host_out_ + 8, dout_ + 8, sizeof(double), cudaMemcpyDeviceToHost, st_) != cudaSuccess)
      return cuda_fail("download");
    if ((s = sync()) != FG_OK) return s;
    sf0_ = host_out_[8];
    sf0_valid_ = true;
    return FG_OK;
  }

  // S_F = phi^dagger (Mhat^dagger Mhat)^{-1} phi at links U (section 4's action).
  fg_status fermion_action(const void* U, double* sf) {
    if constexpr (!kFerm) {
      return no_fermions();
    } else {
      CgStats cs;
      fg_status s = cg(U, phi64_, h_->prm.cg_tol_action, &cs);
      if (s != FG_OK) return s;
      if ((s = run(KC_CG_BLAS, [&] { return launch_dot64(phi64_, x64_, part_rr_, nvec(), st_); })) != FG_OK) return s;
      const int nb = vec_blocks(nvec());
      if ((s = run(KC_REDUCE, [&] { return launch_reduce(part_rr_, nb, 1, dout_ + 9, 0, st_); })) != FG_OK) return s;
      if (cudaMemcpyAsync(host_out_ + 9, dout_ + 9, sizeof(double), cudaMemcpyDeviceToHost, st_) != cudaSuccess)
        return cuda_fail("download");
      if ((s = sync()) != FG_OK) return s;
      *sf = host_out_[9];
      return FG_OK;
    }
  }

  // Pseudofermion force at links U into FF_ (section 4: e_i(S) = -X^dagger e_i(M) X).
  fg_status fermion_force(const void* U, double tol) {
    if constexpr (!kFerm) {
      return no_fermions();
    } else {
      CgStats cs;
      fg_status s = cg(U, phi64_, tol, &cs);
      if (s != FG_OK) return s;
      const int n = nvec();
      const double k2 = h_->prm.kappa * h_->prm.kappa;
      if ((s = run(KC_CG_BLAS, [&] { return launch_convert<R, double>(Xe_, x64_, nullptr, n, st_); })) != FG_OK) return s;
      // X_o = D_oe X_e; Y_e = X_e - kappa^2 D_eo X_o; Y_o = g5 D_oe g5 Y_e
      if ((s = run(KC_DSLASH, [&] {
             return launch_dslash<R, NC, R>(g_, Xo_, Xe_, nullptr, nullptr, U, 1, 0, 0, 1.0, nullptr, nullptr, st_);
           })) != FG_OK) return s;
      if ((s = run(KC_DSLASH, [&] {
             return launch_dslash<R, NC, R>(g_, Ye_, Xo_, Xe_, nullptr, U, 0, 0, 1, -k2, nullptr, nullptr, st_);
           })) != FG_OK) return s;
      if ((s = run(KC_DSLASH, [&] {
             return launch_dslash<R, NC, R>(g_, Yo_, Ye_, nullptr, nullptr, U, 1, 1, 0, 1.0, nullptr, nullptr, st_);
           })) != FG_OK) return s;
      return run(KC_FERMION_FORCE, [&] {
        return launch_fermion_force<R, NC, R>(g_, U, Xe_, Xo_, Ye_, Yo_, FF_, k2, 0, st_);
      });
    }
  }

  // Dslash of the inner iterations: on the FP32 links, or with a 16-bit
  // inner solver on the links' 16-bit copy (then U is that copy) and 16-bit
  // spinors.
  // `solver` = false: outside a solve (no early return on the solver's
  // converged flag).
  cudaError_t inner_dslash(void* out, const void* in, const void* x, const void* pdot, const void* U, int out_par,
                           int dag, int mode, double b, double* partial, bool solver = true) {
    CgDev* const cgd = solver ? cgd_ : nullptr;
    if constexpr (kMixed) {
      if (half_links_)
        return launch_dslash_h16<NC>(s16_, g_, out, in, x, pdot, U, out_par, dag, mode, b, partial, cgd, st_);
    }
    return launch_dslash<R, NC, R>(g_, out, in, x, pdot, U, out_par, dag, mode, b, partial, cgd, st_);
  }

  // Folded iteration, launches D and A (B and C are plain Dslash launches).
  // A swaps the current and other buffers of r and p.
  cudaError_t fold_apdot(const void* U) {
    if constexpr (kMixed || std::is_same<R, double>::value) {
      const double k2 = h_->prm.kappa * h_->prm.kappa;
      return launch_cg_apdot<R, NC>(g_, ap_, to_, te_, p_, rs_, U, k2, part_pap_, cgd_, st_);
    } else {
      return cudaErrorNotSupported;
    }
  }
  cudaError_t fold_update(const void* U) {
    if constexpr (kMixed || std::is_same<R, double>::value) {
      const cudaError_t e = launch_cg_fold<R, NC>(g_, to_, xs_, rs_, ap_, p_, rs2_, p2_, U, part_rr_, cgd_,
                                                  mapped_->hist, &mapped_->dev_iter, h_->prm.cg_maxiter, st_);
      std::swap(rs_, rs2_);
      std::swap(p_, p2_);
      return e;
    } else {
      return cudaErrorNotSupported;
    }
  }
  // t_o = D_oe p, which the folded iteration expects on entry (after the
  // setup and after every reliable update, which may replace p).
  fg_status fold_prime(const void* U) {
    return run(KC_DSLASH, [&] { return inner_dslash(to_, p_, nullptr, nullptr, U, 1, 0, 0, 1.0, nullptr); });
  }

  // One CG iteration in the inner precision R: 4 Dslash + 2 vector kernels,
  // which all return at once after convergence (cgd_->done).  Raw launches,
  // usable inside stream capture.
  cudaError_t cg_iteration_raw(const void* U) {
    const double k2 = h_->prm.kappa * h_->prm.kappa;
    const int n = nvec();
    cudaError_t e;
    if (fold_) {
      if ((e = inner_dslash(te_, to_, p_, nullptr, U, 0, 0, 1, -k2, nullptr)) != cudaSuccess) return e;
      if ((e = inner_dslash(to_, te_, nullptr, nullptr, U, 1, 1, 0, 1.0, nullptr)) != cudaSuccess) return e;
      if ((e = fold_apdot(U)) != cudaSuccess) return e;
      return fold_update(U);
    }
    if ((e = inner_dslash(to_, p_, nullptr, nullptr, U, 1, 0, 0, 1.0, nullptr)) != cudaSuccess) return e;
    if ((e = inner_dslash(te_, to_, p_, nullptr, U, 0, 0, 1, -k2, nullptr)) != cudaSuccess) return e;
    if ((e = inner_dslash(to_, te_, nullptr, nullptr, U, 1, 1, 0, 1.0, nullptr)) != cudaSuccess) return e;
    if ((e = inner_dslash(ap_, to_, te_, p_, U, 0, 1, 2, -k2, part_pap_)) != cudaSuccess) return e;
    if (half_links_) {
      if ((e = launch_cg_axpy_h16(s16_, xs_, rs_, p_, ap_, cgd_, part_rr_, n, st_)) != cudaSuccess) return e;
      return launch_cg_xpay_h16(s16_, p_, rs_, cgd_, mapped_->hist, &mapped_->dev_iter, h_->prm.cg_maxiter, n, st_);
    }
    if ((e = launch_cg_axpy<R>(xs_, rs_, p_, ap_, cgd_, part_rr_, n, st_)) !=
        cudaSuccess)
      return e;
    return launch_cg_xpay<R>(p_, rs_, cgd_, mapped_->hist, &mapped_->dev_iter,
                             h_->prm.cg_maxiter, n, st_);
  }

  // The same through run(), so that per-kernel timing and launch counting see
  // each kernel (used when timing is on or a graph is not available).
  fg_status cg_iteration(const void* U) {
    const double k2 = h_->prm.kappa * h_->prm.kappa;
    const int n = nvec();
    fg_status s;
    if (fold_) {
      if ((s = run(KC_DSLASH, [&] { return inner_dslash(te_, to_, p_, nullptr, U, 0, 0, 1, -k2, nullptr); })) !=
          FG_OK)
        return s;
      if ((s = run(KC_DSLASH, [&] { return inner_dslash(to_, te_, nullptr, nullptr, U, 1, 1, 0, 1.0, nullptr); })) !=
          FG_OK)
        return s;
      if ((s = run(KC_DSLASH, [&] { return fold_apdot(U); })) != FG_OK) return s;
      return run(KC_DSLASH, [&] { return fold_update(U); });
    }
    if ((s = run(KC_DSLASH, [&] { return inner_dslash(to_, p_, nullptr, nullptr, U, 1, 0, 0, 1.0, nullptr); })) !=
        FG_OK)
      return s;
    if ((s = run(KC_DSLASH, [&] { return inner_dslash(te_, to_, p_, nullptr, U, 0, 0, 1, -k2, nullptr); })) != FG_OK)
      return s;
    if ((s = run(KC_DSLASH, [&] { return inner_dslash(to_, te_, nullptr, nullptr, U, 1, 1, 0, 1.0, nullptr); })) !=
        FG_OK)
      return s;
    if ((s = run(KC_DSLASH, [&] { return inner_dslash(ap_, to_, te_, p_, U, 0, 1, 2, -k2, part_pap_); })) != FG_OK)
      return s;
    if (half_links_) {
      if ((s = run(KC_CG_BLAS, [&] { return launch_cg_axpy_h16(s16_, xs_, rs_, p_, ap_, cgd_, part_rr_, n, st_); })) !=
          FG_OK)
        return s;
      return run(KC_CG_BLAS, [&] {
        return launch_cg_xpay_h16(s16_, p_, rs_, cgd_, mapped_->hist, &mapped_->dev_iter, h_->prm.cg_maxiter, n, st_);
      });
    }
    if ((s = run(KC_CG_BLAS, [&] {
           return launch_cg_axpy<R>(xs_, rs_, p_, ap_, cgd_, part_rr_, n, st_);
         })) != FG_OK) return s;
    return run(KC_CG_BLAS, [&] {
      return launch_cg_xpay<R>(p_, rs_, cgd_, mapped_->hist, &mapped_->dev_iter,
                               h_->prm.cg_maxiter, n, st_);
    });
  }

  // A CUDA graph of n iterations (n = 2, 4 or 8) on links U, captured on first
  // use and cached per link buffer and n (the links are the only argument
  // that changes between solves).  Null if capture is not possible.
  static constexpr int kCgBatch = 8;
  struct CgGraph {
    const void* U;
    int n;
    const void* r;  // the current r buffer at capture (the folded iteration alternates two)
    cudaGraphExec_t exec;
  };
  std::vector<CgGraph> cg_graphs_;
  bool cg_graphs_broken_ = false;
  // FG_CG_GRAPHS=0 in the environment turns the graph batches off (tuning).
  const bool use_cg_graphs_ = [] {
    const char* e = std::getenv("FG_CG_GRAPHS");
    return !(e && e[0] == '0');
  }();

  cudaGraphExec_t cg_graph(const void* U, int n) {
    for (const CgGraph& c : cg_graphs_)
      if (c.U == U && c.n == n && c.r == rs_) return c.exec;
    const void* r_at_capture = rs_;
    if (cg_graphs_broken_) return nullptr;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      cg_graphs_broken_ = true;
      return nullptr;
    }
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cg_iteration_raw(U);
    cudaError_t e2 = cudaStreamEndCapture(st_, &graph);
    if (rs_ != r_at_capture) {  // a capture that stopped after an odd number of folded iterations
      std::swap(rs_, rs2_);
      std::swap(p_, p2_);
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && e2 == cudaSuccess && graph != nullptr &&
        cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
      cg_graphs_.push_back({U, n, r_at_capture, exec});
    } else {
      cudaGetLastError();
      exec = nullptr;
      cg_graphs_broken_ = true;
    }
    if (graph) cudaGraphDestroy(graph);
    return exec;
  }

  // Queue n iterations: one graph launch when n is 2, 4 or 8 and timing is
  // off, single launches otherwise.
  fg_status cg_batch(const void* U, int n) {
    if ((n == 2 || n == 4 || n == 8) && !h_->timer.on && use_cg_graphs_) {
      cudaGraphExec_t g = cg_graph(U, n);
      if (g != nullptr) {
        if (cudaGraphLaunch(g, st_) != cudaSuccess) return cuda_fail("cg graph launch");
        // an even number of folded iterations leaves rs_ and p_ where they were
        h_->launches += (fold_ ? 4 : 6) * n;
        return FG_OK;
      }
    }
    for (int i = 0; i < n; ++i) {
      fg_status s = cg_iteration(U);
      if (s != FG_OK) return s;
    }
    return FG_OK;
  }

  // Reliable update after the last queued iteration: x += x_s, r = b - M x,
  // r_s = r, rr = |r|^2 (also published to the host).  The FP64 solver keeps
  // x in FP64.  The FP32 solver keeps x in double-float and evaluates the
  // intermediate updates' M x in double-float arithmetic (GB300's FP64 rate
  // is 1/64 of its FP32 rate); the final update, which certifies
  // convergence, converts x to FP64 and applies M in FP64.
  fg_status reliable_update(const void* U, const void* b64, bool final) {
    const int n = nvec();
    fg_status s;
    if (half_links_) return reliable_update_h16(U, b64, final);
    if (kMixed) {
      if ((s = run(KC_CG_BLAS, [&] { return launch_ru_accumulate_df(xdf_, xs_, n, st_); })) != FG_OK) return s;
      if (!final) {
        if ((s = apply_mdagm_df(ax64_, xdf_, U)) != FG_OK) return s;
        if ((s = run(KC_CG_BLAS, [&] { return launch_ru_residual_df(bdf_, ax64_, rs_, part_rr_, n, st_); })) !=
            FG_OK)
          return s;
      } else {
        if ((s = run(KC_CG_BLAS, [&] { return launch_df_to_double(x64_, xdf_, n, st_); })) != FG_OK) return s;
      }
    } else {
      if ((s = run(KC_CG_BLAS, [&] { return launch_ru_accumulate<R>(x64_, xs_, n, st_); })) != FG_OK) return s;
    }
    if (!kMixed || final) {
      if ((s = apply_mdagm64(ax64_, x64_, U)) != FG_OK) return s;
      if ((s = run(KC_CG_BLAS, [&] { return launch_ru_residual<R>(b64, ax64_, r64_, rs_, part_rr_, n, st_); })) !=
          FG_OK)
        return s;
    }
    double* tr = &mapped_->true_rr;
    if ((s = run(KC_REDUCE, [&] { return launch_ru_publish(part_rr_, vec_blocks(n), cgd_, tr, final ? 1 : 0, st_); })) !=
        FG_OK)
      return s;
    return run(KC_CG_BLAS, [&] { return launch_cg_restart<R>(p_, rs_, cgd_, n, st_); });
  }

  // The same for half-precision inner vectors: x += sigma x_s; the true
  // residual is kept in double-float (or FP64 for the certifying update),
  // sigma is reset from it, and r_s = r / sigma, p = rho p (or r_s).
  fg_status reliable_update_h16(const void* U, const void* b64, bool final) {
    const int n = nvec();
    const int nbv = vec_blocks(n);
    double* tr = &mapped_->true_rr;
    fg_status s;
    if ((s = run(KC_CG_BLAS, [&] { return launch_ru_accumulate_df_scaled(xdf_, xs_, cgd_, n, st_); })) != FG_OK)
      return s;
    if (!final) {
      if ((s = apply_mdagm_df(ax64_, xdf_, U)) != FG_OK) return s;
      if ((s = run(KC_CG_BLAS, [&] { return launch_ru_residual_df_keep(bdf_, ax64_, part_rr_, n, st_); })) != FG_OK)
        return s;
      if ((s = run(KC_REDUCE, [&] { return launch_ru_publish_h16(part_rr_, nbv, cgd_, tr, n, st_); })) != FG_OK)
        return s;
      return run(KC_CG_BLAS, [&] { return launch_ru_rescale_df_h16(s16_, ax64_, rs_, p_, cgd_, n, st_); });
    }
    if ((s = run(KC_CG_BLAS, [&] { return launch_df_to_double(x64_, xdf_, n, st_); })) != FG_OK) return s;
    if ((s = apply_mdagm64(ax64_, x64_, U)) != FG_OK) return s;
    if ((s = run(KC_CG_BLAS, [&] { return launch_ru_residual64_keep(b64, ax64_, r64_, part_rr_, n, st_); })) != FG_OK)
      return s;
    if ((s = run(KC_REDUCE, [&] { return launch_ru_publish_h16(part_rr_, nbv, cgd_, tr, n, st_); })) != FG_OK)
      return s;
    return run(KC_CG_BLAS, [&] { return launch_ru_rescale64_h16(s16_, r64_, rs_, p_, cgd_, n, st_); });
  }

  // Conjugate gradient on Mhat^dagger Mhat x = b (b FP64 on the device), x0 = 0,
  // to |b - M x| <= tol |b| in FP64; solution in x64_.
  //
  // The iterations run in precision R with device-side scalars; the host
  // never waits for the iteration it has just queued: after queueing
  // iteration k it waits for iteration k-1 and reads its residual from mapped
  // memory.  For R = float, a reliable update (FP64 true residual, Sleijpen
  // and van der Vorst) is queued whenever the iterated residual has fallen by
  // cg_delta since the last one; convergence is always confirmed by an FP64
  // true residual.
  fg_status cg(const void* U, const void* b64, double tol, CgStats* st) {
    const int n = nvec();
    const int nbv = vec_blocks(n);
    const bool mixed = sizeof(R) < sizeof(double);
    // with half-precision links the inner operator is off by ~5e-4, and the
    // recursion stalls long before the residual has fallen by 0.01: update
    // at least every factor 0.1
    const double delta = half_links_ ? std::max(h_->prm.cg_delta, 0.1) : h_->prm.cg_delta;
    const double delta2 = delta * delta;
    fg_status s;
    ++solves_;
    // a solve for phi after one for the same phi starts from its solution
    const bool guess = use_guess_ && guess_ok_ && b64 == phi64_ && !half_links_;
    guess_ok_ = false;  // until this solve succeeds
    if ((!guess && cudaMemsetAsync(x64_, 0, (size_t)n * sizeof(double2), st_) != cudaSuccess) ||
        cudaMemsetAsync(xs_, 0, (size_t)n * sizeof(C2), st_) != cudaSuccess ||
        (!guess && cudaMemcpyAsync(r64_, b64, (size_t)n * sizeof(double2), cudaMemcpyDeviceToDevice, st_) !=
                       cudaSuccess))
      return cuda_fail("cg setup");
    if (kMixed && ((!guess && cudaMemsetAsync(xdf_, 0, (size_t)n * sizeof(double2), st_) != cudaSuccess) ||
                   run(KC_CG_BLAS, [&] { return launch_df_from_double(bdf_, b64, n, st_); }) != FG_OK))
      return cuda_fail("cg setup");
    double* bbp = &mapped_->bb;
    if (guess) {
      // r = b - M x0: in double-float for the FP32 solver (x0 held as x_df),
      // in FP64 for the FP64 one; r_s = (R) r and the partials of |r|^2
      if (kMixed) {
        if ((s = run(KC_CG_BLAS, [&] { return launch_df_from_double(xdf_, x64_, n, st_); })) != FG_OK) return s;
        if ((s = apply_mdagm_df(ax64_, xdf_, U)) != FG_OK) return s;
        if ((s = run(KC_CG_BLAS, [&] { return launch_ru_residual_df(bdf_, ax64_, rs_, part_rr_, n, st_); })) !=
            FG_OK)
          return s;
      } else {
        if ((s = apply_mdagm64(ax64_, x64_, U)) != FG_OK) return s;
        if ((s = run(KC_CG_BLAS, [&] { return launch_ru_residual<R>(b64, ax64_, r64_, rs_, part_rr_, n, st_); })) !=
            FG_OK)
          return s;
      }
      if ((s = run(KC_CG_BLAS, [&] { return launch_dot64(b64, b64, part_b_, n, st_); })) != FG_OK) return s;
      if ((s = run(KC_REDUCE, [&] {
             return launch_cg_init_guess(part_b_, part_rr_, nbv, cgd_, tol * tol, bbp, &mapped_->rr0, st_);
           })) != FG_OK)
        return s;
      if (cudaMemcpyAsync(p_, rs_, (size_t)n * sizeof(C2), cudaMemcpyDeviceToDevice, st_) != cudaSuccess)
        return cuda_fail("cg setup");
    } else if (half_links_) {
      // half-precision inner vectors: r_s = b / sigma with sigma^2 = |b|^2 / n
      if ((s = run(KC_CG_BLAS, [&] { return launch_dot64(b64, b64, part_rr_, n, st_); })) != FG_OK) return s;
      if ((s = run(KC_REDUCE, [&] { return launch_cg_init_h16(part_rr_, nbv, cgd_, tol * tol, bbp, n, st_); })) !=
          FG_OK)
        return s;
      if ((s = run(KC_CG_BLAS, [&] { return launch_scale_to_h16(s16_, rs_, b64, cgd_, n, st_); })) != FG_OK) return s;
      if (cudaMemcpyAsync(p_, rs_, (size_t)n * sizeof(__half2), cudaMemcpyDeviceToDevice, st_) != cudaSuccess)
        return cuda_fail("cg setup");
    } else {
      if ((s = run(KC_CG_BLAS, [&] { return launch_convert<R, double>(rs_, b64, part_rr_, n, st_); })) != FG_OK)
        return s;
      if ((s = run(KC_REDUCE, [&] { return launch_cg_init(part_rr_, nbv, cgd_, tol * tol, bbp, st_); })) != FG_OK)
        return s;
      if (cudaMemcpyAsync(p_, rs_, (size_t)n * sizeof(C2), cudaMemcpyDeviceToDevice, st_) != cudaSuccess)
        return cuda_fail("cg setup");
    }
    // the inner iterations' links: the FP32 field, or its half-precision copy
    const void* Uin = U;
    if (half_links_) {
      if ((s = run(KC_CONVERT, [&] { return launch_links_to_half<NC>(s16_, g_, U, U16_, st_); })) != FG_OK) return s;
      Uin = U16_;
    }
    if (fold_ && (s = fold_prime(Uin)) != FG_OK) return s;
    st->iters = 0;
    st->nru = 0;
    st->true_res = 0.0;
    // |b|^2 reaches the host through mapped memory; it is read at the first
    // check, which comes after the setup kernels, so the setup needs no sync.
    double bb = -1.0, tol2bb = 0.0;
    auto know_bb = [&]() {
      if (bb < 0.0) {
        bb = mapped_->bb;
        tol2bb = tol * tol * bb;
      }
    };
    double maxrr = 0.0;
    double rate = -1.0;  // observed per-iteration factor of |r|^2
    const int maxiter = h_->prm.cg_maxiter;
    int queued = 0;      // iterations queued so far (including ones that return at once)
    int checked = 0;     // device iterations whose residual the host has read
    int iters = 0;
    int pending = -1;    // event slot of the batch queued before the last one
    mapped_->dev_iter = 0;
    for (;;) {
      bool converged = false;
      while (!converged) {
        if (queued >= maxiter) {
          if ((s = sync()) != FG_OK) return s;
          know_bb();
          if (bb == 0.0) return FG_OK;
          const int upto = mapped_->dev_iter;
          for (int j = checked + 1; j <= upto; ++j)
            if (mapped_->hist[j] <= tol2bb) { converged = true; iters = j; break; }
          if (!converged) {
            cg_iters_ += upto;
            st->iters = upto;
            return h_->fail(FG_ENOCONV, "CG did not converge in " + std::to_string(maxiter) + " iterations");
          }
          break;
        }
        // batch size: small enough that a reliable update decided on the
        // last checked batch still lands within about half a factor delta^2
        // of residual reduction (fast-converging systems get short batches)
        int nb = kCgBatch;
        if (mixed && rate > 0.0 && rate < 1.0) {
          const double per_delta = std::log(delta2) / std::log(rate);
          nb = per_delta >= 16.0 ? 8 : (per_delta >= 8.0 ? 4 : (per_delta >= 4.0 ? 2 : 1));
        }
        nb = std::min(nb, maxiter - queued);
        if ((s = cg_batch(Uin, nb)) != FG_OK) return s;
        queued += nb;
        const int slot = (pending + 1) & 1;
        if (cudaEventRecord(ev_[slot], st_) != cudaSuccess) return cuda_fail("event");
        if (pending >= 0) {
          // wait for the batch before this one; the GPU keeps working on this one
          std::string why;
          if ((s = host_wait_event(ev_[pending], h_->wait_limit_s, &why)) != FG_OK) return h_->fail(s, why);
          if (bb < 0.0) {
            know_bb();
            maxrr = guess ? mapped_->rr0 : bb;
            if (bb == 0.0) {            // b = 0: x = 0, nothing to iterate
              if ((s = sync()) != FG_OK) return s;
              return FG_OK;
            }
            if (guess && maxrr <= tol2bb) {  // the guess already meets the tolerance
              converged = true;
              iters = 0;
              pending = slot;
              break;
            }
          }
          const int upto = *(volatile int*)&mapped_->dev_iter;
          const int first = checked + 1;
          double first_rr = -1.0, last = -1.0;
          for (int j = first; j <= upto; ++j) {
            const double rr = mapped_->hist[j];
            CG_TRACE("cg it %d rr/bb %.3e (queued %d)\n", j, rr / bb, queued);
            if (!(rr == rr)) return h_->fail(FG_ENOCONV, "CG residual is NaN");
            if (first_rr < 0.0) first_rr = rr;
            last = rr;
            if (rr <= tol2bb) { converged = true; iters = j; break; }
          }
          checked = std::max(checked, upto);
          if (!converged && mixed && last > 0.0) {
            // extrapolate the residual to the last queued iteration with the
            // convergence rate just seen, so the update is not late
            double predicted = last;
            if (first_rr > 0.0 && upto > first && last < first_rr) {
              rate = std::pow(last / first_rr, 1.0 / (upto - first));
              predicted = last * std::pow(rate, queued - upto);
            }
            if (predicted < delta2 * maxrr) {
              CG_TRACE("cg reliable update after queued %d (last %.3e predicted %.3e)\n", queued, last / bb,
                       predicted / bb);
              if ((s = reliable_update(U, b64, false)) != FG_OK) return s;
              if (fold_ && (s = fold_prime(Uin)) != FG_OK) return s;
              ++st->nru;
              maxrr = predicted;
            }
          }
        }
        pending = slot;
      }
      if ((s = reliable_update(U, b64, true)) != FG_OK) return s;
      ++st->nru;
      if (fold_ && (s = fold_prime(Uin)) != FG_OK) return s;
      if ((s = sync()) != FG_OK) return s;
      const double trr = mapped_->true_rr;
      st->true_res = std::sqrt(trr / bb);
      CG_TRACE("cg final check: iters %d true rr/bb %.3e tol2 %.3e\n", iters, trr / bb, tol * tol);
      if (trr <= tol2bb) break;
      // The FP64 residual is not yet below tol: the reliable update has put
      // it into r and cleared `done`; continue from there.
      maxrr = trr;
      checked = mapped_->dev_iter;
      queued = checked;  // the iterations queued past convergence returned at once
      pending = -1;
    }
    st->iters = iters;
    cg_iters_ += iters;
    guess_ok_ = b64 == phi64_;
    return FG_OK;
  }
};

fg_status lattice_init(fg_lattice* h) {
  const fg_params& p = h->prm;
  h->g.L[0] = p.dims[0];
  h->g.L[1] = p.dims[1];
  h->g.L[2] = p.dims[2];
  h->g.L[3] = p.dims[3];
  h->g.V = p.dims[0] * p.dims[1] * p.dims[2] * p.dims[3];
  h->g.Vh = h->g.V / 2;
  h->g.Lxh = p.dims[0] / 2;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return h->fail(FG_ECUDA, "no CUDA device");
  }
  if (p.cuda_stream) {
    h->st = (cudaStream_t)p.cuda_stream;
    h->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking) != cudaSuccess)
      return h->fail(FG_ECUDA, "stream creation failed");
    h->own_stream = true;
  }
  fg_status s = FG_OK;
  if (p.precision == FG_FP64 && p.link_reals == 18) {
    auto* b = new (std::nothrow) Backend<double, 9>(h);
    if (!b) return FG_ENOMEM;
    h->be.reset(b);
    s = b->init();
  } else if (p.precision == FG_FP64) {
    auto* b = new (std::nothrow) Backend<double, 6>(h);
    if (!b) return FG_ENOMEM;
    h->be.reset(b);
    s = b->init();
  } else if (p.precision == FG_DF64 && p.link_reals == 18) {
    auto* b = new (std::nothrow) Backend<DF, 9>(h);
    if (!b) return FG_ENOMEM;
    h->be.reset(b);
    s = b->init();
  } else if (p.precision == FG_DF64) {
    auto* b = new (std::nothrow) Backend<DF, 6>(h);
    if (!b) return FG_ENOMEM;
    h->be.reset(b);
    s = b->init();
  } else if (p.link_reals == 18) {
    auto* b = new (std::nothrow) Backend<float, 9>(h);
    if (!b) return FG_ENOMEM;
    h->be.reset(b);
    s = b->init();
  } else {
    auto* b = new (std::nothrow) Backend<float, 6>(h);
    if (!b) return FG_ENOMEM;
    h->be.reset(b);
    s = b->init();
  }
  return s;
}

}  // namespace fg

fg_lattice::~fg_lattice() {
  if (st) cudaStreamSynchronize(st);
  timer.reset();
  be.reset();
  if (own_stream && st) cudaStreamDestroy(st);
}
