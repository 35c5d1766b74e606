// Many independent pure-gauge HMC chains of different volumes and couplings,
// advanced together (fg_batch_* in include/fg_lattice.h).
//
// All chains share one integrator and step size, so every MD sub-step of
// Table 1 (a kick, a drift, a force-gradient displacement) is one launch over
// the links of all chains, instead of one launch per chain.  The chains'
// fields are concatenated in each device buffer, each chain keeping the
// single-lattice layout (fg_common.cuh) at its own offset; a tile list
// assigns blocks of H half-sites (both parities, four directions) to chains,
// and the kernels walk it with a grid-stride loop over a grid sized to fill
// the GPU once (a persistent launch).  Per-link arithmetic is the same code
// as for one lattice (gauge_device.cuh), so a chain gives the same links alone
// and in a batch.  The dH of every chain is summed in FP64 per chain and the
// Metropolis step runs on the device, so a whole trajectory of all chains is
// one CUDA graph: refresh, start energies, the fused force launches, end
// energies, accept/reject, restore of rejected chains.  The tile size H is
// chosen by timing the force kernel at the first trajectory (autotuning).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/fg_lattice.h"
#include "fg_common.cuh"
#include "fg_kernels.h"
#include "fg_runtime.h"
#include "gauge_device.cuh"

namespace fg {

struct ChainDesc {
  Geom g;
  long long goff;  // byte offset of the chain's links in a link buffer
  long long moff;  // byte offset of its momenta
  long long soff;  // offset of its sites in per-site arrays
  double beta;
  int tile0, ntiles;
};

struct Tile {
  int chain;
  int i0;  // first half-site index of the tile
};

// Per-chain results, FP64: S_G and T at start and end, dH, accepted.
constexpr int kChainOut = 8;

// Site of thread threadIdx.x in tile t (H half-sites, both parities).
template <int H>
__device__ __forceinline__ bool tile_site(const Tile& t, const Geom& g, int& s) {
  const int i = t.i0 + (int)(threadIdx.x % H);
  if (i >= g.Vh) return false;
  s = (int)(threadIdx.x / H) * g.Vh + i;
  return true;
}

template <int H> struct TileBounds;
template <> struct TileBounds<16> { static constexpr int min_blocks = 4; };
template <> struct TileBounds<32> { static constexpr int min_blocks = 2; };
template <> struct TileBounds<64> { static constexpr int min_blocks = 1; };
// Register cap of the force kernel: 128 per thread for FP32 and FP64 links;
// double-float links get up to 255 (as in the single-lattice kernel).
template <typename R, int H>
constexpr int kBatchMinBlocks =
    std::is_same<R, DF>::value ? (H == 16 ? 2 * FG_FORCE_DF_MIN_BLOCKS : FG_FORCE_DF_MIN_BLOCKS) : TileBounds<H>::min_blocks;

// Double-float links: a block barrier after each tile keeps the warps of an
// SM on the same tile.  Left to drift apart, some warps run the staple
// products while others run the exponential, and the two long code paths
// together overflow the instruction cache: a 64-chain FG trajectory took
// 80 ms without the barrier and 45 ms with it.  FG_BATCH_TILE_SYNC (tuning
// macro): 0 no barrier, 1 double-float only, 2 also FP32.
#ifndef FG_BATCH_TILE_SYNC
#define FG_BATCH_TILE_SYNC 1
#endif
template <typename R>
constexpr bool kTileSync =
    (std::is_same<R, DF>::value && FG_BATCH_TILE_SYNC >= 1) || (std::is_same<R, float>::value && FG_BATCH_TILE_SYNC >= 2);

template <typename R, int NC, int MODE, int H>
__global__ void __launch_bounds__(8 * H, (kBatchMinBlocks<R, H>))
    batch_force_kernel(const Tile* __restrict__ tiles, int ntiles, const ChainDesc* __restrict__ chains,
                       char* U, char* P, char* F, char* Ubase, char* Uout, double ckick, double cdrift, double cdisp,
                       int reunit) {
  for (int b = blockIdx.x; b < ntiles; b += gridDim.x) {
    const Tile t = tiles[b];
    const ChainDesc& cd = chains[t.chain];
    const Geom g = cd.g;
    int s;
    const bool ok = tile_site<H>(t, g, s);
    if (!kForceSharedT<R, NC> && !kTileSync<R> && !ok) continue;
    Gauge<R, NC> u, ub, uo;
    u.p = U + cd.goff; u.V = g.V;
    ub.p = Ubase ? Ubase + cd.goff : nullptr; ub.V = g.V;
    uo.p = Uout ? Uout + cd.goff : nullptr; uo.V = g.V;
    Mom<R> p, f, ff;
    p.p = P ? P + cd.moff : nullptr; p.V = g.V;
    f.p = F ? F + cd.moff : nullptr; f.V = g.V;
    ff.p = nullptr; ff.V = g.V;
    if constexpr (kForceSharedT<R, NC>) {
      // the same staple arithmetic as the single-lattice kernel; the whole
      // block takes the barriers (uniform tile loop)
      extern __shared__ float2 batch_tsh[];
      force_link_shared<NC, MODE, 2 * H>(reinterpret_cast<float2(*)[9][2 * H]>(batch_tsh), ok, s, u, p, f, ff, ub,
                                         uo, g, R(cd.beta / 6.0), R(ckick), R(cdrift), R(cdisp), reunit, R(1));
      __syncthreads();   // the next tile rewrites the slots
    } else {
      if (ok) {
        int c[4], par;
        cb_coords(g, s, c, par);
        force_link<R, NC, MODE>(u, p, f, ff, ub, uo, g, c, s, (int)threadIdx.y, R(cd.beta / 6.0), R(ckick),
                                R(cdrift), R(cdisp), reunit);
      }
      if constexpr (kTileSync<R>) __syncthreads();  // every thread of the block runs the same tiles
    }
  }
}

// Dynamic shared memory of batch_force_kernel with H half-sites per tile.
template <typename R, int NC, int H>
constexpr size_t batch_force_smem() {
  return kForceSharedT<R, NC> ? (size_t)6 * 9 * 2 * H * sizeof(float2) : 0;
}

template <typename R, int NC, int H>
__global__ void __launch_bounds__(8 * H) batch_drift_kernel(const Tile* __restrict__ tiles, int ntiles,
                                                            const ChainDesc* __restrict__ chains, char* Uin,
                                                            char* P, char* Uout, double c, int reunit) {
  for (int b = blockIdx.x; b < ntiles; b += gridDim.x) {
    const Tile t = tiles[b];
    const ChainDesc& cd = chains[t.chain];
    int s;
    if (!tile_site<H>(t, cd.g, s)) continue;
    Gauge<R, NC> ui, uo;
    ui.p = Uin + cd.goff; ui.V = cd.g.V;
    uo.p = Uout + cd.goff; uo.V = cd.g.V;
    Mom<R> p;
    p.p = P + cd.moff; p.V = cd.g.V;
    drift_link(ui, p, uo, s, (int)threadIdx.y, R(c), reunit);
  }
}

template <typename R, int H>
__global__ void __launch_bounds__(8 * H) batch_refresh_kernel(const Tile* __restrict__ tiles, int ntiles,
                                                              const ChainDesc* __restrict__ chains, char* P,
                                                              uint32_t k0, uint32_t k1,
                                                              const uint32_t* __restrict__ counters) {
  const uint32_t draw = counters[0];
  for (int b = blockIdx.x; b < ntiles; b += gridDim.x) {
    const Tile t = tiles[b];
    const ChainDesc& cd = chains[t.chain];
    int s;
    if (!tile_site<H>(t, cd.g, s)) continue;
    Mom<R> p;
    p.p = P + cd.moff; p.V = cd.g.V;
    refresh_link(p, cd.g, s, (int)threadIdx.y, k0, k1, draw, 3u + (uint32_t)t.chain);
  }
}

// Per-site energies; one (S_G, T, dh) partial per tile, partial[k][tile].
template <typename R, int NC, int H>
__global__ void __launch_bounds__(2 * H) batch_energy_kernel(const Tile* __restrict__ tiles, int ntiles,
                                                             const ChainDesc* __restrict__ chains, char* U, char* P,
                                                             int mode, double* __restrict__ h0,
                                                             double* __restrict__ partial) {
  for (int b = blockIdx.x; b < ntiles; b += gridDim.x) {
    const Tile t = tiles[b];
    const ChainDesc& cd = chains[t.chain];
    double v[3] = {0.0, 0.0, 0.0};
    int s;
    if (tile_site<H>(t, cd.g, s)) {
      Gauge<R, NC> u;
      u.p = U + cd.goff; u.V = cd.g.V;
      Mom<R> p;
      p.p = P ? P + cd.moff : nullptr; p.V = cd.g.V;
      site_energy(u, p, cd.g, s, 6.0 * cd.beta, cd.beta / 3.0, mode, h0 + cd.soff, v);
    }
    // one partial per tile (a block may handle several tiles)
    __shared__ double sh[3][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double x = v[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) sh[k][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      double x = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += sh[threadIdx.x][w];
      partial[(size_t)threadIdx.x * ntiles + b] = x;
    }
    __syncthreads();
  }
}

// out[chain][off + k] = sum over the chain's tiles of partial[k][tile], fixed order.
__global__ void __launch_bounds__(256) batch_chain_reduce_kernel(const ChainDesc* __restrict__ chains,
                                                                 const double* __restrict__ partial, int ntiles,
                                                                 double* __restrict__ out, int off) {
  const ChainDesc& cd = chains[blockIdx.x];
  __shared__ double sh[8];
  for (int k = 0; k < 3; ++k) {
    double x = 0.0;
    for (int i = threadIdx.x; i < cd.ntiles; i += blockDim.x) x += partial[(size_t)k * ntiles + cd.tile0 + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
      out[(size_t)blockIdx.x * kChainOut + off + k] = t;
    }
    __syncthreads();
  }
}

// Metropolis per chain on the device: accept iff dH <= 0 or u < exp(-dH),
// u from Philox (chain, accept draw, stream 4); mode 1 accepts every finite
// dH.  Results also go to mapped host memory.
__global__ void batch_accept_kernel(int n, double* __restrict__ out, int* __restrict__ accepted, uint32_t k0,
                                    uint32_t k1, const uint32_t* __restrict__ counters, int mode,
                                    double* __restrict__ host_out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double* o = out + (size_t)c * kChainOut;
  const double dh = o[5];
  uint32_t ctr[4] = {(uint32_t)c, counters[1], 4u, 0u};
  Philox::rounds(ctr, k0, k1);
  const uint64_t bits = ((uint64_t)ctr[0] << 21) ^ ((uint64_t)ctr[1] >> 11);
  const double u = (double)(bits & ((1ULL << 53) - 1)) * (1.0 / 9007199254740992.0);
  const bool finite = isfinite(dh);
  const int acc = finite && (mode == 1 || dh <= 0.0 || u < exp(-dh));
  accepted[c] = acc;
  o[6] = acc;
  for (int k = 0; k < kChainOut; ++k) host_out[(size_t)c * kChainOut + k] = o[k];
}

// Rejected chains: copy their start links over the current ones.
template <typename R, int NC, int H>
__global__ void __launch_bounds__(8 * H) batch_restore_kernel(const Tile* __restrict__ tiles, int ntiles,
                                                              const ChainDesc* __restrict__ chains,
                                                              const int* __restrict__ accepted, char* Ustart,
                                                              char* Ucur) {
  for (int b = blockIdx.x; b < ntiles; b += gridDim.x) {
    const Tile t = tiles[b];
    if (accepted[t.chain]) continue;
    const ChainDesc& cd = chains[t.chain];
    int s;
    if (!tile_site<H>(t, cd.g, s)) continue;
    Gauge<R, NC> us, uc;
    us.p = Ustart + cd.goff; us.V = cd.g.V;
    uc.p = Ucur + cd.goff; uc.V = cd.g.V;
    uc.store((int)threadIdx.y, s, us.load((int)threadIdx.y, s));
  }
}

__global__ void batch_advance_kernel(uint32_t* counters, int refreshed) {
  if (refreshed) counters[0] += 1;
  counters[1] += 1;
}

}  // namespace fg

// ============================================================================ host side
using namespace fg;

namespace fg {

struct IBatch {
  virtual ~IBatch() {}
  virtual fg_status set_gauge(int chain, const double* host) = 0;
  virtual fg_status get_gauge(int chain, double* host) = 0;
  virtual fg_status set_momenta(int chain, const double* host) = 0;
  virtual fg_status get_momenta(int chain, double* host) = 0;
  virtual fg_status trajectory(int integ, double dt, int nsteps, int refresh, int accept_mode,
                               fg_traj_result* out) = 0;
  virtual int tile() const = 0;
};

}  // namespace fg

struct fg_batch {
  fg_batch_params prm;
  std::vector<int> dims;
  std::vector<double> beta;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::string err;
  long long launches = 0;
  double wait_limit_s = 0.0;   // limit on host waits (0: none), fg_batch_set_wait_limit
  std::unique_ptr<fg::IBatch> impl;
  fg_status fail(fg_status s, const std::string& m) {
    err = m;
    return s;
  }
  ~fg_batch() {
    if (st) cudaStreamSynchronize(st);
    impl.reset();
    if (own_stream && st) cudaStreamDestroy(st);
  }
};

namespace fg {

static Geom geom_of(const int* d) {
  Geom g;
  for (int i = 0; i < 4; ++i) g.L[i] = d[i];
  g.V = d[0] * d[1] * d[2] * d[3];
  g.Vh = g.V / 2;
  g.Lxh = d[0] / 2;
  g.dLxh = make_fastdiv((uint32_t)g.Lxh);
  g.dLy = make_fastdiv((uint32_t)d[1]);
  g.dLz = make_fastdiv((uint32_t)d[2]);
  return g;
}

template <typename R, int NC>
class Batch final : public IBatch {
 public:
  typedef typename Vec2<R>::T C2;
  // Tile sizes compiled for this precision: 16, 32 and 64 half-sites, or 16
  // and 32 for double-float links (their force kernel is several times the
  // size of the FP32 one; fg_batch_create rejects tile 64 for them).
  static constexpr int kTileSizes = std::is_same<R, DF>::value ? 2 : 3;
  explicit Batch(fg_batch* b) : b_(b), st_(b->st) {}
  ~Batch() override {
    for (auto& g : graphs_) cudaGraphExecDestroy(g.exec);
    for (void* p : allocs_) cudaFree(p);
    if (host_out_) cudaFreeHost(host_out_);
  }

  fg_status init() {
    // 64-half-site tiles of the FP32 force kernel use more than the default
    // 48 KB of dynamic shared memory
    if constexpr (batch_force_smem<R, NC, 64>() > 48 * 1024) {
      const int bytes = (int)batch_force_smem<R, NC, 64>();
      if (cudaFuncSetAttribute(batch_force_kernel<R, NC, FM_STORE, 64>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess ||
          cudaFuncSetAttribute(batch_force_kernel<R, NC, FM_KICK, 64>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess ||
          cudaFuncSetAttribute(batch_force_kernel<R, NC, FM_KICK_DRIFT, 64>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess ||
          cudaFuncSetAttribute(batch_force_kernel<R, NC, FM_DISPLACE, 64>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess)
        return cuda_fail("force kernel shared-memory attribute");
    }
    const int n = b_->prm.nchains;
    std::vector<ChainDesc> cds(n);
    long long goff = 0, moff = 0, soff = 0;
    for (int c = 0; c < n; ++c) {
      ChainDesc& cd = cds[c];
      cd.g = geom_of(&b_->dims[4 * c]);
      cd.beta = b_->beta[c];
      cd.goff = goff;
      cd.moff = moff;
      cd.soff = soff;
      goff += align256((long long)4 * NC * cd.g.V * sizeof(C2));
      moff += align256((long long)4 * 4 * cd.g.V * sizeof(C2));
      soff += cd.g.V;
    }
    gauge_bytes_ = goff;
    mom_bytes_ = moff;
    sites_ = soff;
    cds_ = cds;
    fg_status s;
    for (int k = 0; k < 3; ++k)
      if ((s = alloc(&buf_[k], gauge_bytes_)) != FG_OK) return s;
    cur_ = 0;
    if ((s = alloc(&P_, mom_bytes_)) != FG_OK) return s;
    if ((s = alloc(&F_, mom_bytes_)) != FG_OK) return s;
    if ((s = alloc((void**)&h0_, sites_ * sizeof(double))) != FG_OK) return s;
    if ((s = alloc((void**)&d_out_, (size_t)n * kChainOut * sizeof(double))) != FG_OK) return s;
    if ((s = alloc((void**)&d_acc_, (size_t)n * sizeof(int))) != FG_OK) return s;
    if ((s = alloc((void**)&d_counters_, 4 * sizeof(uint32_t))) != FG_OK) return s;
    if (cudaHostAlloc((void**)&host_out_, (size_t)n * kChainOut * sizeof(double), cudaHostAllocMapped) !=
        cudaSuccess) {
      host_out_ = nullptr;
      return b_->fail(FG_ENOMEM, "pinned host allocation failed");
    }
    if (cudaMemsetAsync(d_counters_, 0, 4 * sizeof(uint32_t), st_) != cudaSuccess ||
        cudaMemsetAsync(P_, 0, mom_bytes_, st_) != cudaSuccess)
      return cuda_fail("memset");
    // tile lists for H = 16, 32, 64
    for (int hi = 0; hi < 3; ++hi) {
      const int H = 16 << hi;
      std::vector<Tile> tl;
      std::vector<ChainDesc> cdh = cds;
      for (int c = 0; c < n; ++c) {
        cdh[c].tile0 = (int)tl.size();
        for (int i0 = 0; i0 < cds[c].g.Vh; i0 += H) tl.push_back(Tile{c, i0});
        cdh[c].ntiles = (int)tl.size() - cdh[c].tile0;
      }
      ntiles_[hi] = (int)tl.size();
      if ((s = alloc((void**)&d_tiles_[hi], tl.size() * sizeof(Tile))) != FG_OK) return s;
      if ((s = alloc((void**)&d_chains_h_[hi], n * sizeof(ChainDesc))) != FG_OK) return s;
      if (cudaMemcpyAsync(d_tiles_[hi], tl.data(), tl.size() * sizeof(Tile), cudaMemcpyHostToDevice, st_) !=
              cudaSuccess ||
          cudaMemcpyAsync(d_chains_h_[hi], cdh.data(), n * sizeof(ChainDesc), cudaMemcpyHostToDevice, st_) !=
              cudaSuccess)
        return cuda_fail("descriptor upload");
      if ((s = alloc((void**)&d_partial_[hi], (size_t)3 * tl.size() * sizeof(double))) != FG_OK) return s;
    }
    if (b_->prm.tile == 16) hsel_ = 0;
    else if (b_->prm.tile == 32) hsel_ = 1;
    else if (b_->prm.tile == 64) hsel_ = 2;
    else hsel_ = -1;  // autotune at the first trajectory
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    sms_ = sms > 0 ? sms : 152;
    // cold start
    for (int c = 0; c < n; ++c) {
      GeomH gh = geomh(c);
      if ((s = lrun([&] { return launch_unit_links<R, NC>(gh, (char*)buf_[cur_] + cds_[c].goff, st_); })) != FG_OK)
        return s;
    }
    return sync();
  }

  int tile() const override { return hsel_ < 0 ? 0 : (16 << hsel_); }

  fg_status set_gauge(int c, const double* host) override {
    const size_t n = (size_t)4 * cds_[c].g.V * 18;
    fg_status s = ensure_canon(n);
    if (s != FG_OK) return s;
    if (cudaMemcpyAsync(canon_, host, n * sizeof(double), cudaMemcpyHostToDevice, st_) != cudaSuccess)
      return cuda_fail("gauge upload");
    GeomH gh = geomh(c);
    if ((s = lrun([&] { return launch_gauge_to_device<R, NC>(gh, canon_, (char*)buf_[cur_] + cds_[c].goff, st_); })) !=
        FG_OK)
      return s;
    return sync();
  }
  fg_status get_gauge(int c, double* host) override {
    const size_t n = (size_t)4 * cds_[c].g.V * 18;
    fg_status s = ensure_canon(n);
    if (s != FG_OK) return s;
    GeomH gh = geomh(c);
    if ((s = lrun([&] { return launch_gauge_to_canon<R, NC>(gh, (char*)buf_[cur_] + cds_[c].goff, canon_, st_); })) !=
        FG_OK)
      return s;
    if (cudaMemcpyAsync(host, canon_, n * sizeof(double), cudaMemcpyDeviceToHost, st_) != cudaSuccess)
      return cuda_fail("gauge download");
    return sync();
  }
  fg_status set_momenta(int c, const double* host) override {
    const size_t n = (size_t)4 * cds_[c].g.V * 8;
    fg_status s = ensure_canon(n);
    if (s != FG_OK) return s;
    if (cudaMemcpyAsync(canon_, host, n * sizeof(double), cudaMemcpyHostToDevice, st_) != cudaSuccess)
      return cuda_fail("momenta upload");
    GeomH gh = geomh(c);
    if ((s = lrun([&] { return launch_mom_to_device<R>(gh, canon_, (char*)P_ + cds_[c].moff, st_); })) != FG_OK)
      return s;
    return sync();
  }
  fg_status get_momenta(int c, double* host) override {
    const size_t n = (size_t)4 * cds_[c].g.V * 8;
    fg_status s = ensure_canon(n);
    if (s != FG_OK) return s;
    GeomH gh = geomh(c);
    if ((s = lrun([&] { return launch_mom_to_canon<R>(gh, (char*)P_ + cds_[c].moff, canon_, st_); })) != FG_OK)
      return s;
    if (cudaMemcpyAsync(host, canon_, n * sizeof(double), cudaMemcpyDeviceToHost, st_) != cudaSuccess)
      return cuda_fail("momenta download");
    return sync();
  }

  fg_status trajectory(int integ, double dt, int nsteps, int refresh, int accept_mode,
                       fg_traj_result* out) override {
    fg_status s;
    if (hsel_ < 0 && (s = autotune()) != FG_OK) return s;
    const int start = cur_;
    std::vector<Op> ops = trajectory_ops(integ, b_->prm.alpha, nsteps, true);
    int final_buf = start;
    if (b_->prm.use_graphs) {
      cudaGraphExec_t g = nullptr;
      for (auto& e : graphs_)
        if (e.start == start && e.integ == integ && e.dt == dt && e.nsteps == nsteps && e.refresh == refresh &&
            e.accept == accept_mode && e.hsel == hsel_) {
          g = e.exec;
          final_buf = e.final_buf;
        }
      if (g == nullptr) {
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
          return cuda_fail("begin capture");
        long long before = b_->launches;
        fg_status es = enqueue_trajectory(ops, dt, refresh, accept_mode, start, &final_buf);
        cudaError_t ce = cudaStreamEndCapture(st_, &graph);
        if (es != FG_OK) {
          if (graph) cudaGraphDestroy(graph);
          return es;
        }
        if (ce != cudaSuccess || cudaGraphInstantiate(&g, graph, 0) != cudaSuccess) {
          if (graph) cudaGraphDestroy(graph);
          return cuda_fail("graph instantiate");
        }
        cudaGraphDestroy(graph);
        const long long per = b_->launches - before;
        b_->launches = before;
        graphs_.push_back(GraphEntry{start, integ, dt, nsteps, refresh, accept_mode, hsel_, final_buf, g, per});
      }
      long long per = 0;
      for (auto& e : graphs_)
        if (e.exec == g) per = e.kernels;
      if (cudaGraphLaunch(g, st_) != cudaSuccess) return cuda_fail("graph launch");
      b_->launches += per;
    } else {
      if ((s = enqueue_trajectory(ops, dt, refresh, accept_mode, start, &final_buf)) != FG_OK) return s;
    }
    if ((s = sync()) != FG_OK) return s;
    cur_ = final_buf;
    if (out) {
      const int n = b_->prm.nchains;
      const int nforce = count_forces(ops);
      for (int c = 0; c < n; ++c) {
        const double* o = host_out_ + (size_t)c * kChainOut;
        fg_traj_result& r = out[c];
        std::memset(&r, 0, sizeof(r));
        r.S_gauge0 = o[0];
        r.T0 = o[1];
        r.S_gauge1 = o[3];
        r.T1 = o[4];
        r.dH = o[5];
        r.H0 = o[0] + o[1];
        r.H1 = o[3] + o[4];
        r.accepted = o[6] != 0.0;
        r.n_steps = nsteps;
        r.n_force = nforce;
      }
    }
    return FG_OK;
  }

 private:
  struct GraphEntry {
    int start, integ;
    double dt;
    int nsteps, refresh, accept, hsel, final_buf;
    cudaGraphExec_t exec;
    long long kernels;
  };

  fg_batch* b_;
  cudaStream_t st_;
  std::vector<void*> allocs_;
  std::vector<ChainDesc> cds_;
  long long gauge_bytes_ = 0, mom_bytes_ = 0, sites_ = 0;
  void* buf_[3] = {nullptr, nullptr, nullptr};
  int cur_ = 0;
  void* P_ = nullptr;
  void* F_ = nullptr;
  double* h0_ = nullptr;
  ChainDesc* d_chains_h_[3] = {nullptr, nullptr, nullptr};
  Tile* d_tiles_[3] = {nullptr, nullptr, nullptr};
  int ntiles_[3] = {0, 0, 0};
  double* d_partial_[3] = {nullptr, nullptr, nullptr};
  double* d_out_ = nullptr;
  int* d_acc_ = nullptr;
  uint32_t* d_counters_ = nullptr;
  double* host_out_ = nullptr;
  double* canon_ = nullptr;
  size_t canon_n_ = 0;
  int hsel_ = 1;
  int sms_ = 152;
  std::vector<GraphEntry> graphs_;

  static long long align256(long long x) { return (x + 255) & ~255LL; }
  GeomH geomh(int c) const {
    GeomH h;
    for (int i = 0; i < 4; ++i) h.L[i] = cds_[c].g.L[i];
    h.V = cds_[c].g.V;
    h.Vh = cds_[c].g.Vh;
    h.Lxh = cds_[c].g.Lxh;
    return h;
  }
  fg_status alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return b_->fail(FG_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    allocs_.push_back(*p);
    return FG_OK;
  }
  fg_status ensure_canon(size_t n) {
    if (canon_n_ >= n) return FG_OK;
    fg_status s = alloc((void**)&canon_, n * sizeof(double));
    if (s != FG_OK) return s;
    canon_n_ = n;
    return FG_OK;
  }
  fg_status cuda_fail(const char* what) {
    cudaError_t e = cudaGetLastError();
    return b_->fail(FG_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  }
  fg_status sync() {
    std::string why;
    const fg_status s = host_wait_stream(st_, b_->wait_limit_s, &why);
    if (s != FG_OK) return b_->fail(s, why);
    return FG_OK;
  }
  template <class Fn>
  fg_status lrun(Fn&& fn) {
    cudaError_t e = fn();
    ++b_->launches;
    if (e != cudaSuccess) return b_->fail(FG_ECUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    return FG_OK;
  }

  // grid of a persistent launch: enough blocks to fill every SM once
  int grid(int ntiles, int blocks_per_sm) const { return std::max(1, std::min(ntiles, sms_ * blocks_per_sm)); }

  template <int H>
  fg_status force_h(int hi, int mode, void* U, void* Ubase, void* Uout, void* F, double ckick, double cdrift,
                    double cdisp) {
    const int nt = ntiles_[hi];
    const dim3 blk(2 * H, 4);
    const int gr = grid(nt, kBatchMinBlocks<R, H>);
    const int reunit = b_->prm.reunitarize;
    char* Pp = (char*)P_;
    return lrun([&] {
      const size_t sm = batch_force_smem<R, NC, H>();
      const Tile* tl = d_tiles_[hi];
      const ChainDesc* cds = d_chains_h_[hi];
      switch (mode) {
        case FM_STORE:
          batch_force_kernel<R, NC, FM_STORE, H><<<gr, blk, sm, st_>>>(tl, nt, cds, (char*)U, Pp, (char*)F,
                                                                      (char*)Ubase, (char*)Uout, ckick, cdrift,
                                                                      cdisp, reunit);
          break;
        case FM_KICK:
          batch_force_kernel<R, NC, FM_KICK, H><<<gr, blk, sm, st_>>>(tl, nt, cds, (char*)U, Pp, (char*)F,
                                                                     (char*)Ubase, (char*)Uout, ckick, cdrift,
                                                                     cdisp, reunit);
          break;
        case FM_KICK_DRIFT:
          batch_force_kernel<R, NC, FM_KICK_DRIFT, H><<<gr, blk, sm, st_>>>(tl, nt, cds, (char*)U, Pp, (char*)F,
                                                                           (char*)Ubase, (char*)Uout, ckick,
                                                                           cdrift, cdisp, reunit);
          break;
        default:
          batch_force_kernel<R, NC, FM_DISPLACE, H><<<gr, blk, sm, st_>>>(tl, nt, cds, (char*)U, Pp, (char*)F,
                                                                         (char*)Ubase, (char*)Uout, ckick, cdrift,
                                                                         cdisp, reunit);
          break;
      }
      return cudaGetLastError();
    });
  }
  // Double-float: the exponential of a kick-and-drift or a displacement runs
  // in a launch of its own after the force (the same arithmetic, the same
  // bits); the two long code paths in one launch overflow the instruction
  // cache.  FG_SPLIT_EXP=0 / =1 in the environment turns the split off / on
  // for any precision.
  const bool split_exp_ = [] {
    const char* e = std::getenv("FG_SPLIT_EXP");
    return e ? e[0] == '1' : std::is_same<R, DF>::value;
  }();
  fg_status force(int mode, void* U, void* Ubase, void* Uout, double ckick, double cdrift, double cdisp) {
    if (split_exp_ && mode == FM_KICK_DRIFT) {
      fg_status s = force_tiles(FM_KICK, U, nullptr, nullptr, ckick, 0, 0);
      if (s != FG_OK) return s;
      return drift(Ubase, Uout, cdrift);
    }
    if (split_exp_ && mode == FM_DISPLACE) {
      fg_status s = force_tiles(FM_STORE, U, nullptr, nullptr, 0, 0, 0);
      if (s != FG_OK) return s;
      return drift(U, Uout, -cdisp, F_, 0);
    }
    return force_tiles(mode, U, Ubase, Uout, ckick, cdrift, cdisp);
  }
  fg_status force_tiles(int mode, void* U, void* Ubase, void* Uout, double ckick, double cdrift, double cdisp) {
    switch (hsel_) {
      case 0: return force_h<16>(0, mode, U, Ubase, Uout, F_, ckick, cdrift, cdisp);
      case 2:
        if constexpr (kTileSizes > 2) return force_h<64>(2, mode, U, Ubase, Uout, F_, ckick, cdrift, cdisp);
        [[fallthrough]];
      default: return force_h<32>(1, mode, U, Ubase, Uout, F_, ckick, cdrift, cdisp);
    }
  }
  // Uout = exp(i c G) Uin for the generator G (the momenta, or the force
  // buffer for a displacement); reunit < 0: the handle's setting.
  template <int H>
  fg_status drift_h(int hi, void* Uin, void* Uout, double c, void* G, int reunit) {
    const int nt = ntiles_[hi];
    return lrun([&] {
      batch_drift_kernel<R, NC, H><<<grid(nt, 2), dim3(2 * H, 4), 0, st_>>>(d_tiles_[hi], nt, d_chains_h_[hi],
                                                                            (char*)Uin, (char*)G, (char*)Uout, c,
                                                                            reunit);
      return cudaGetLastError();
    });
  }
  fg_status drift(void* Uin, void* Uout, double c, void* G = nullptr, int reunit = -1) {
    if (G == nullptr) G = P_;
    if (reunit < 0) reunit = b_->prm.reunitarize;
    switch (hsel_) {
      case 0: return drift_h<16>(0, Uin, Uout, c, G, reunit);
      case 2:
        if constexpr (kTileSizes > 2) return drift_h<64>(2, Uin, Uout, c, G, reunit);
        [[fallthrough]];
      default: return drift_h<32>(1, Uin, Uout, c, G, reunit);
    }
  }
  template <int H>
  fg_status misc_h(int hi, int what, void* U, int mode, int refreshed, int accept_mode, void* Ustart, void* Ucur,
                   int off) {
    const int nt = ntiles_[hi];
    const uint32_t k0 = (uint32_t)b_->prm.seed, k1 = (uint32_t)(b_->prm.seed >> 32);
    const int n = b_->prm.nchains;
    return lrun([&] {
      switch (what) {
        case 0:
          batch_refresh_kernel<R, H><<<grid(nt, 4), dim3(2 * H, 4), 0, st_>>>(d_tiles_[hi], nt, d_chains_h_[hi],
                                                                              (char*)P_, k0, k1, d_counters_);
          break;
        case 1:
          batch_energy_kernel<R, NC, H><<<grid(nt, 8), 2 * H, 0, st_>>>(d_tiles_[hi], nt, d_chains_h_[hi], (char*)U,
                                                                        (char*)P_, mode, h0_, d_partial_[hi]);
          break;
        case 2:
          batch_chain_reduce_kernel<<<n, 256, 0, st_>>>(d_chains_h_[hi], d_partial_[hi], nt, d_out_, off);
          break;
        case 3:
          batch_accept_kernel<<<(n + 127) / 128, 128, 0, st_>>>(n, d_out_, d_acc_, k0, k1, d_counters_, accept_mode,
                                                                host_out_);
          break;
        case 4:
          batch_restore_kernel<R, NC, H><<<grid(nt, 4), dim3(2 * H, 4), 0, st_>>>(d_tiles_[hi], nt, d_chains_h_[hi],
                                                                                  d_acc_, (char*)Ustart, (char*)Ucur);
          break;
        default:
          batch_advance_kernel<<<1, 1, 0, st_>>>(d_counters_, refreshed);
          break;
      }
      return cudaGetLastError();
    });
  }
  fg_status misc(int what, void* U = nullptr, int mode = 0, int refreshed = 0, int accept_mode = 0,
                 void* Ustart = nullptr, void* Ucur = nullptr, int off = 0) {
    switch (hsel_) {
      case 0: return misc_h<16>(0, what, U, mode, refreshed, accept_mode, Ustart, Ucur, off);
      case 2:
        if constexpr (kTileSizes > 2) return misc_h<64>(2, what, U, mode, refreshed, accept_mode, Ustart, Ucur, off);
        [[fallthrough]];
      default: return misc_h<32>(1, what, U, mode, refreshed, accept_mode, Ustart, Ucur, off);
    }
  }

  int free_buffer(int cur, int protect) const {
    for (int k = 0; k < 3; ++k)
      if (k != cur && k != protect) return k;
    return -1;
  }
  int buffer_not(int a, int b) const {
    for (int k = 0; k < 3; ++k)
      if (k != a && k != b) return k;
    return -1;
  }

  // The whole trajectory of all chains, stream-ordered (captured into a graph
  // when graphs are on).  Same buffer rotation as the single-lattice executor.
  fg_status enqueue_trajectory(const std::vector<Op>& ops, double dt, int refresh, int accept_mode, int start,
                               int* final_buf) {
    fg_status s;
    if (refresh && (s = misc(0)) != FG_OK) return s;
    if ((s = misc(1, buf_[start], 0)) != FG_OK) return s;
    if ((s = misc(2, nullptr, 0, 0, 0, nullptr, nullptr, 0)) != FG_OK) return s;
    int cur = start;
    const int protect = start;
    const size_t n = ops.size();
    for (size_t i = 0; i < n;) {
      const Op& o = ops[i];
      const bool next_q = (i + 1 < n) && ops[i + 1].kind == 'Q';
      if (o.kind == 'P') {
        if (next_q) {
          const int out = free_buffer(cur, protect);
          if ((s = force(FM_KICK_DRIFT, buf_[cur], buf_[cur], buf_[out], o.c * dt, ops[i + 1].c * dt, 0)) != FG_OK)
            return s;
          cur = out;
          i += 2;
        } else {
          if ((s = force(FM_KICK, buf_[cur], nullptr, nullptr, o.c * dt, 0, 0)) != FG_OK) return s;
          i += 1;
        }
      } else if (o.kind == 'Q') {
        const int out = (cur == protect) ? free_buffer(cur, protect) : cur;
        if ((s = drift(buf_[cur], buf_[out], o.c * dt)) != FG_OK) return s;
        cur = out;
        i += 1;
      } else {
        const int disp = free_buffer(cur, protect);
        if ((s = force(FM_DISPLACE, buf_[cur], nullptr, buf_[disp], 0, 0, o.d * dt * dt)) != FG_OK) return s;
        if (next_q) {
          const int out = (cur == protect) ? buffer_not(protect, disp) : cur;
          if ((s = force(FM_KICK_DRIFT, buf_[disp], buf_[cur], buf_[out], o.c * dt, ops[i + 1].c * dt, 0)) != FG_OK)
            return s;
          cur = out;
          i += 2;
        } else {
          if ((s = force(FM_KICK, buf_[disp], nullptr, nullptr, o.c * dt, 0, 0)) != FG_OK) return s;
          i += 1;
        }
      }
    }
    if ((s = misc(1, buf_[cur], 1)) != FG_OK) return s;
    if ((s = misc(2, nullptr, 0, 0, 0, nullptr, nullptr, 3)) != FG_OK) return s;
    if ((s = misc(3, nullptr, 0, 0, accept_mode)) != FG_OK) return s;
    if (cur != start && (s = misc(4, nullptr, 0, 0, 0, buf_[start], buf_[cur])) != FG_OK) return s;
    if ((s = misc(5, nullptr, 0, refresh)) != FG_OK) return s;
    *final_buf = cur;
    return FG_OK;
  }

  // Times the force kernel (store mode, all chains) for every tile size and
  // keeps the fastest.
  fg_status autotune() {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return cuda_fail("event");
    float best = 1e30f;
    int best_h = 1;
    for (int hi = 0; hi < kTileSizes; ++hi) {
      hsel_ = hi;
      float tmin = 1e30f;
      for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(a, st_);
        // a displacement into a scratch buffer: the force and the exponential,
        // as in the kick-and-drift and displace launches that dominate a
        // trajectory (the exponential's code decides the tile for double-float)
        fg_status s = force(FM_DISPLACE, buf_[cur_], nullptr, buf_[(cur_ + 1) % 3], 0, 0, 0.01);
        if (s != FG_OK) {
          cudaEventDestroy(a);
          cudaEventDestroy(b);
          return s;
        }
        cudaEventRecord(b, st_);
        std::string why;
        if ((s = host_wait_event(b, b_->wait_limit_s, &why)) != FG_OK) {
          cudaEventDestroy(a);
          cudaEventDestroy(b);
          return b_->fail(s, why);
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0) tmin = std::min(tmin, ms);  // first repetition warms up
      }
      if (tmin < best) {
        best = tmin;
        best_h = hi;
      }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    hsel_ = best_h;
    return FG_OK;
  }
};

}  // namespace fg

extern "C" {

fg_status fg_batch_params_default(fg_batch_params* p) {
  if (!p) return FG_EINVAL;
  std::memset(p, 0, sizeof(*p));
  p->precision = FG_FP32;
  p->link_reals = 18;
  p->reunitarize = -1;
  p->alpha = 0.1932;
  p->tile = 0;
  p->use_graphs = 1;
  p->seed = 1;
  return FG_OK;
}

fg_status fg_batch_create(const fg_batch_params* p, fg_batch** out) {
  if (!out) return FG_EINVAL;
  *out = nullptr;
  if (!p || p->nchains < 1 || !p->dims || !p->beta) return FG_EINVAL;
  if (p->precision != FG_FP64 && p->precision != FG_FP32 && p->precision != FG_DF64) return FG_EINVAL;
  if (p->link_reals != 18 && p->link_reals != 12) return FG_EINVAL;
  if (p->tile != 0 && p->tile != 16 && p->tile != 32 && p->tile != 64) return FG_EINVAL;
  // double-float chains: 18-real links and tiles of 16 or 32 half-sites
  if (p->precision == FG_DF64 && (p->link_reals != 18 || p->tile == 64)) return FG_EINVAL;
  long long total = 0;
  for (int c = 0; c < p->nchains; ++c) {
    long long V = 1;
    for (int i = 0; i < 4; ++i) {
      const int d = p->dims[4 * c + i];
      if (d < 2 || (d & 1)) return FG_EINVAL;
      V *= d;
    }
    if (V > (1LL << 28)) return FG_EINVAL;  // 32-bit element indices, as for one lattice
    if (!(p->beta[c] >= 0.0)) return FG_EINVAL;
    total += V;
  }
  if (total > (1LL << 28)) return FG_EINVAL;
  fg_batch* b = new (std::nothrow) fg_batch();
  if (!b) return FG_ENOMEM;
  b->prm = *p;
  b->dims.assign(p->dims, p->dims + 4 * p->nchains);
  b->beta.assign(p->beta, p->beta + p->nchains);
  b->prm.dims = nullptr;
  b->prm.beta = nullptr;
  if (b->prm.reunitarize < 0) b->prm.reunitarize = (p->precision == FG_FP32) ? 1 : 0;
  if (!(b->prm.alpha > 0.0)) b->prm.alpha = 0.1932;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    delete b;
    return FG_ECUDA;
  }
  if (p->cuda_stream) {
    b->st = (cudaStream_t)p->cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return FG_ECUDA;
    }
    b->own_stream = true;
  }
  fg_status s;
  if (p->precision == FG_FP64 && p->link_reals == 18) {
    auto* x = new (std::nothrow) Batch<double, 9>(b);
    b->impl.reset(x);
    s = x ? x->init() : FG_ENOMEM;
  } else if (p->precision == FG_FP64) {
    auto* x = new (std::nothrow) Batch<double, 6>(b);
    b->impl.reset(x);
    s = x ? x->init() : FG_ENOMEM;
  } else if (p->precision == FG_DF64) {
    auto* x = new (std::nothrow) Batch<DF, 9>(b);
    b->impl.reset(x);
    s = x ? x->init() : FG_ENOMEM;
  } else if (p->link_reals == 18) {
    auto* x = new (std::nothrow) Batch<float, 9>(b);
    b->impl.reset(x);
    s = x ? x->init() : FG_ENOMEM;
  } else {
    auto* x = new (std::nothrow) Batch<float, 6>(b);
    b->impl.reset(x);
    s = x ? x->init() : FG_ENOMEM;
  }
  if (s != FG_OK) {
    delete b;
    return s;
  }
  *out = b;
  return FG_OK;
}

void fg_batch_destroy(fg_batch* b) { delete b; }

const char* fg_batch_last_error(const fg_batch* b) { return b ? b->err.c_str() : "null handle"; }

static bool chain_ok(const fg_batch* b, int c) { return b && c >= 0 && c < b->prm.nchains; }

fg_status fg_batch_set_gauge(fg_batch* b, int chain, const double* x) {
  if (!chain_ok(b, chain) || !x) return FG_EINVAL;
  return b->impl->set_gauge(chain, x);
}
fg_status fg_batch_get_gauge(fg_batch* b, int chain, double* x) {
  if (!chain_ok(b, chain) || !x) return FG_EINVAL;
  return b->impl->get_gauge(chain, x);
}
fg_status fg_batch_set_momenta(fg_batch* b, int chain, const double* x) {
  if (!chain_ok(b, chain) || !x) return FG_EINVAL;
  return b->impl->set_momenta(chain, x);
}
fg_status fg_batch_get_momenta(fg_batch* b, int chain, double* x) {
  if (!chain_ok(b, chain) || !x) return FG_EINVAL;
  return b->impl->get_momenta(chain, x);
}
fg_status fg_batch_trajectory(fg_batch* b, fg_integrator integ, double dt, double tau, int refresh,
                              int accept_mode, fg_traj_result* out) {
  if (!b) return FG_EINVAL;
  if ((int)integ < 0 || (int)integ > 4 || !(dt > 0.0) || !(tau > 0.0) || accept_mode < 0 || accept_mode > 1)
    return b->fail(FG_EINVAL, "bad integrator, dt, tau or accept mode");
  const int n = (int)std::llround(tau / dt);
  if (n < 1 || std::fabs(n * dt - tau) > 1e-9 * tau) return b->fail(FG_EINVAL, "tau must be a multiple of dt");
  return b->impl->trajectory((int)integ, dt, n, refresh, accept_mode, out);
}
fg_status fg_batch_tile(const fg_batch* b, int* tile) {
  if (!b || !tile) return FG_EINVAL;
  *tile = b->impl->tile();
  return FG_OK;
}
long long fg_batch_launch_count(const fg_batch* b) { return b ? b->launches : -1; }
fg_status fg_batch_set_wait_limit(fg_batch* b, double seconds) {
  if (!b) return FG_EINVAL;
  if (!(seconds >= 0.0)) return b->fail(FG_EINVAL, "wait limit must be >= 0");
  b->wait_limit_s = seconds;
  return FG_OK;
}

}  // extern "C"
