// Backend<R, NC>: device fields of one lattice in precision R with NC complex
// entries stored per link, and the host-side sequencing of the kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <algorithm>
#include <utility>
#include <vector>

#include "fg_common.cuh"
#include "fg_kernels.h"
#include "fg_runtime.h"

namespace fg {

template <typename R, int NC>
class Backend final : public IBackend {
 public:
  typedef typename Vec2<R>::T C2;

  explicit Backend(fg_lattice* h) : h_(h), g_(h->g), st_(h->st) {}

  ~Backend() override {
    for (void* p : allocs_) cudaFree(p);
    if (host_out_) cudaFreeHost(host_out_);
  }

  fg_status init() {
    const size_t V = (size_t)g_.V;
    const size_t gauge_bytes = (size_t)4 * NC * V * sizeof(C2);
    const size_t mom_bytes = (size_t)4 * 4 * V * sizeof(C2);
    fg_status s;
    if ((s = alloc(&U_, gauge_bytes)) != FG_OK) return s;
    if ((s = alloc(&Ualt_, gauge_bytes)) != FG_OK) return s;
    if ((s = alloc(&Ubak_, gauge_bytes)) != FG_OK) return s;
    if ((s = alloc(&P_, mom_bytes)) != FG_OK) return s;
    if ((s = alloc(&F_, mom_bytes)) != FG_OK) return s;
    if ((s = alloc((void**)&h0_, V * sizeof(double))) != FG_OK) return s;
    const size_t nb = (V + 255) / 256 + 1;
    if ((s = alloc((void**)&partial_, 4 * nb * sizeof(double))) != FG_OK) return s;
    if ((s = alloc((void**)&dout_, 32 * sizeof(double))) != FG_OK) return s;
    if (cudaMallocHost((void**)&host_out_, 32 * sizeof(double)) != cudaSuccess) {
      host_out_ = nullptr;
      return h_->fail(FG_ENOMEM, "pinned host allocation failed");
    }
    if (cudaMemsetAsync(P_, 0, mom_bytes, st_) != cudaSuccess) return cuda_fail("memset");
    // cold start: unit links
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

  fg_status refresh_momenta() override {
    const uint32_t d = draw_++;
    return run(KC_MOMENTA, [&] { return launch_refresh_momenta<R>(g_, P_, h_->prm.seed, d, st_); });
  }

  fg_status set_pseudofermion(const double*) override { return no_fermions(); }
  fg_status refresh_pseudofermion() override { return no_fermions(); }
  fg_status apply_mhat(const double*, double*, int) override { return no_fermions(); }
  fg_status cg_solve(const double*, double*, fg_cg_result*) override { return no_fermions(); }

  fg_status force(double* host_f8) override {
    ForceArgs a = force_args(U_);
    a.F = F_;
    fg_status s = run(KC_GAUGE_FORCE, [&] { return launch_gauge_force<R, NC>(g_, FM_STORE, a, st_); });
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
    if (sf) *sf = 0.0;
    return FG_OK;
  }

  fg_status reunitarize_all() override {
    fg_status s = run(KC_DRIFT, [&] { return launch_reunitarize<R, NC>(g_, U_, st_); });
    if (s != FG_OK) return s;
    return sync();
  }

  // ---------------------------------------------------------------- MD
  fg_status md_step(int integ, double dt) override {
    std::vector<Op> ops = trajectory_ops(integ, h_->prm.alpha, 1, false);
    fg_status s = execute(ops, dt);
    if (s != FG_OK) return s;
    return sync();
  }

  fg_status trajectory(int integ, double dt, int nsteps, int refresh, double u_accept,
                       fg_traj_result* r) override {
    fg_status s;
    if (refresh) {
      if ((s = refresh_momenta()) != FG_OK) return s;
    }
    // H at the start: per-site energies kept for the site-by-site dH sum
    if ((s = energy(0, P_, 0)) != FG_OK) return s;
    if (cudaMemcpyAsync(Ubak_, U_, gauge_bytes(), cudaMemcpyDeviceToDevice, st_) != cudaSuccess)
      return cuda_fail("backup copy");
    std::vector<Op> ops = trajectory_ops(integ, h_->prm.alpha, nsteps, true);
    if ((s = execute(ops, dt)) != FG_OK) return s;
    if ((s = energy(1, P_, 3)) != FG_OK) return s;
    if ((s = fetch(6)) != FG_OK) return s;
    const double* o = host_out_;
    r->S_gauge0 = o[0];
    r->T0 = o[1];
    r->S_gauge1 = o[3];
    r->T1 = o[4];
    r->dH = o[5];
    r->S_ferm0 = r->S_ferm1 = 0.0;
    r->H0 = r->S_gauge0 + r->T0 + r->S_ferm0;
    r->H1 = r->S_gauge1 + r->T1 + r->S_ferm1;
    r->n_steps = nsteps;
    r->n_force = count_forces(ops);
    r->n_solves = 0;
    r->cg_iters = 0;
    const double u = (u_accept < 0.0) ? host_uniform() : u_accept;
    r->accepted = std::isfinite(r->dH) && (r->dH <= 0.0 || u < std::exp(-r->dH));
    if (!r->accepted) {
      if (cudaMemcpyAsync(U_, Ubak_, gauge_bytes(), cudaMemcpyDeviceToDevice, st_) != cudaSuccess)
        return cuda_fail("restore copy");
      if ((s = sync()) != FG_OK) return s;
    }
    return FG_OK;
  }

 private:
  fg_lattice* h_;
  GeomH g_;
  cudaStream_t st_;
  std::vector<void*> allocs_;
  void* U_ = nullptr;
  void* Ualt_ = nullptr;
  void* Ubak_ = nullptr;
  void* P_ = nullptr;
  void* F_ = nullptr;
  double* h0_ = nullptr;
  double* partial_ = nullptr;
  double* dout_ = nullptr;
  double* canon_ = nullptr;
  size_t canon_n_ = 0;
  double* host_out_ = nullptr;
  uint32_t draw_ = 0;

  size_t gauge_bytes() const { return (size_t)4 * NC * g_.V * sizeof(C2); }

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
  fg_status cuda_fail(const char* what) {
    cudaError_t e = cudaGetLastError();
    return h_->fail(FG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
  fg_status sync() {
    cudaError_t e = cudaStreamSynchronize(st_);
    if (e != cudaSuccess) return h_->fail(FG_ECUDA, cudaGetErrorString(e));
    return FG_OK;
  }
  fg_status no_fermions() { return h_->fail(FG_ESTATE, "fermion path not available in this build"); }

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
  fg_status energy(int mode, const void* P, int off) {
    int nb = 0;
    fg_status s = run(KC_ENERGY, [&] {
      return launch_energy<R, NC>(g_, U_, P, h_->prm.beta, mode, h0_, partial_, &nb, st_);
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
    a.F = nullptr;
    a.FF = nullptr;
    a.Ubase = Uf;
    a.Uout = nullptr;
    a.beta = h_->prm.beta;
    a.reunit = h_->prm.reunitarize;
    return a;
  }

  // Runs a merged op list with fused kernels (see the file header of fg_lattice.cu).
  fg_status execute(const std::vector<Op>& ops, double dt) {
    fg_status s;
    const size_t n = ops.size();
    for (size_t i = 0; i < n;) {
      const Op& o = ops[i];
      const bool next_q = (i + 1 < n) && ops[i + 1].kind == 'Q';
      if (o.kind == 'P') {
        ForceArgs a = force_args(U_);
        a.ckick = o.c * dt;
        if (next_q) {
          a.cdrift = ops[i + 1].c * dt;
          a.Ubase = U_;
          a.Uout = Ualt_;
          s = run(KC_GAUGE_FORCE, [&] { return launch_gauge_force<R, NC>(g_, FM_KICK_DRIFT, a, st_); });
          if (s != FG_OK) return s;
          std::swap(U_, Ualt_);
          i += 2;
        } else {
          s = run(KC_GAUGE_FORCE, [&] { return launch_gauge_force<R, NC>(g_, FM_KICK, a, st_); });
          if (s != FG_OK) return s;
          i += 1;
        }
      } else if (o.kind == 'Q') {
        s = run(KC_DRIFT, [&] {
          return launch_drift<R, NC>(g_, U_, P_, U_, o.c * dt, h_->prm.reunitarize, st_);
        });
        if (s != FG_OK) return s;
        i += 1;
      } else {  // 'G'
        ForceArgs d = force_args(U_);
        d.cdisp = o.d * dt * dt;
        d.Uout = Ualt_;
        s = run(KC_GAUGE_FORCE, [&] { return launch_gauge_force<R, NC>(g_, FM_DISPLACE, d, st_); });
        if (s != FG_OK) return s;
        ForceArgs a = force_args(Ualt_);
        a.ckick = o.c * dt;
        if (next_q) {
          a.cdrift = ops[i + 1].c * dt;
          a.Ubase = U_;
          a.Uout = U_;
          s = run(KC_GAUGE_FORCE, [&] { return launch_gauge_force<R, NC>(g_, FM_KICK_DRIFT, a, st_); });
          i += 2;
        } else {
          s = run(KC_GAUGE_FORCE, [&] { return launch_gauge_force<R, NC>(g_, FM_KICK, a, st_); });
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
