"""Benchmark: force-gradient HMC trajectories per second on one GB300 per rank.

Workload (one "step" = one HMC trajectory): pure-gauge SU(3) Wilson action on
a 32^4 lattice at beta = 6.0, force-gradient PQPQP integrator of Table 1 with
dt = 0.25 and tau = 1 (4 MD steps, 13 force evaluations, 8 link drifts),
FP32 links, momenta and forces with FP64 dH sums, 18-real links.  The chain
starts from a seeded hot start thermalised by 10 force-gradient trajectories
(dt = 1/8, always accepted) and 150 untimed Metropolis FG trajectories at
dt = 1/8; W warm-up trajectories follow, then K timed trajectories.

A second, smaller measurement covers the Nf=2 Wilson-fermion path (16^3 x 32,
beta = 5.6, kappa = 0.158, pure-gauge thermalised start): mixed-precision CG
solves to 1e-10 with the even-odd Dslash timed per launch against HBM.

Output: one JSON line (rank 0).  `value` is trajectories per second over all
ranks with the fields resident in HBM; `e2e` is the same metric through the
C ABI with host buffers (each trajectory's momenta uploaded from pinned host
memory while the previous trajectory runs, its result read back; beside it
the same without the overlap, and with the gauge field also uploaded and
read back every trajectory); `roofline` reports the gauge-force kernel against
the FP32 FMA peak; `cpu_baseline` times the FP64 CPU oracle on a 16^4 sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_0910_2950_gb300 import inputs  # noqa: E402

BETA = 6.0
DT = 0.25
TAU = 1.0
L_BENCH = 32
THERM_TRAJ = 10
EQUIL_TRAJ = 150
METRIC = "FG-HMC trajectories/s at fixed acceptance"
UNIT = "trajectories/s"
# FP32 peak of the FMA pipes: 152 SMs x 128 lanes x 2 flop x 2070 MHz (maximum SM clock).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2070e6 / 1e12
# FP64 is nominal (1.25 TFLOP/s for the whole GPU).
FP64_PEAK_TFLOPS = 1.25

# Algorithmic work per link of the fused gauge-force kernel, by mode, with
# 198 flop per 3x3 complex product and 18 per accumulation: the staple sum is
# 6 x (2 x 198 + 18) = 2484; the FP32 12-real kernel shares the upper-staple
# product T of a plane between its two links (per site 6 T products and 12
# accumulated products instead of 12 and 12), 3 x 414 + (6 x 198 + 12 x 216) / 4
# = 2187; then U*A 198, projection and scale 24, kick 16; exp(i c P)
# (Cayley-Hamilton with the Hermitian square) 322 and U <- E U 198; FP32
# re-unitarisation 100 after a drift (the displaced links of the FG step are
# not re-projected).  Rebuilding the third row of 12-real links is not counted.
FLOP_STAPLES = {("fp32", 18): 2484, ("fp32", 12): 2187, ("fp64", 18): 2484, ("fp64", 12): 2484}
FLOP_FORCE_REST = 198 + 24
FLOP_KICK = 16
FLOP_EXP_MUL = 322 + 198
FLOP_REUNIT = 100


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lattice", type=int, default=L_BENCH)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--integrator", default="fg")
    ap.add_argument("--dt", type=float, default=DT)
    ap.add_argument("--link-reals", type=int, default=18)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-full", action="store_true",
                    help="also time 3 oracle forces and whole oracle trajectories at the benchmark lattice (minutes)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fermion", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-compare", action="store_true")
    ap.add_argument("--fermion-dims", default="16,16,16,32")
    ap.add_argument("--compare-steps", type=int, default=20)
    return ap.parse_args()


def hbm_peak():
    """Measured copy bandwidth of the GB300s (GB/s), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def reduce_max(x: float, world: int, device) -> float:
    """Maximum of x over all ranks (the slowest rank's time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, max_seconds: float) -> float:
    """Units processed by all ranks divided by the slowest rank's time."""
    return world * units_per_rank / max_seconds


def rank_seeds(rank: int) -> dict:
    """Independent chains per rank: distinct start fields and RNG streams."""
    return {"hot_start": 1 + rank, "device_rng": 1000 + rank, "e2e_momenta": 77 + rank}


# ----------------------------------------------------------------------------- oracle legs
def oracle_unit_times(seed: int = 3):
    """The oracle's per-unit costs on one host core (seconds): a gauge force
    evaluation on 16^4, and on 8^3 x 16 with kappa = 0.158 a full-lattice
    hop (the Dslash of both parities), one CG iteration (Mhat^dag Mhat and
    the vector updates) and a pseudofermion force from a given solution."""
    from oracle import fermion as fe, gauge
    out = {}
    u = inputs.hot_start((16,) * 4, seed)
    t0 = time.perf_counter()
    gauge.gauge_force(u, BETA)
    out["gauge_force_16^4_s"] = time.perf_counter() - t0
    dims = (8, 8, 8, 16)
    u = inputs.hot_start(dims, seed)
    x = inputs.unpack_even(inputs.gaussian_spinor_even(dims, seed), dims)
    t0 = time.perf_counter()
    fe.hop(u, x)
    out["hop_8^3x16_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, iters = fe.cg(u, 0.158, x, tol=1e-6)
    out["cg_iteration_8^3x16_s"] = (time.perf_counter() - t0) / max(iters, 1)
    t0 = time.perf_counter()
    fe.fermion_force(u, 0.158, x, x=x)
    out["fermion_force_8^3x16_s"] = time.perf_counter() - t0
    return out


def cpu_cores_used():
    return 1  # numpy batched 3x3 products and eigh run on one thread


def cpu_model():
    """The host CPU's model name and logical core count."""
    name = None
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    name = ln.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if name is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
            for ln in out.splitlines():
                if ln.startswith("Model name"):
                    name = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"model": name or "unknown", "logical_cores": os.cpu_count()}


def _single_thread_env():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def _oracle_traj_worker(job):
    """One oracle trajectory (separate process): returns its wall seconds."""
    _single_thread_env()
    sys.path.insert(0, ROOT)
    from oracle import integrators as it
    L, integ, dt, seed = job
    dims = (L,) * 4
    u = inputs.hot_start(dims, seed)
    p = inputs.gaussian_momenta(dims, seed)
    t0 = time.perf_counter()
    it.trajectory(it.GaugeSystem(BETA), it.Integrator(integ), u, p, dt, TAU)
    return time.perf_counter() - t0


class _OraclePool:
    """Processes for independent oracle chains, started with spawn (never
    forked from a process that may hold a CUDA context); a worker that dies
    raises instead of hanging the pool."""

    def __init__(self, n):
        import concurrent.futures as cf
        import multiprocessing as mp
        self._ex = cf.ProcessPoolExecutor(max_workers=n, mp_context=mp.get_context("spawn"))

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self._ex.shutdown(wait=True)
        return False

    def map(self, fn, jobs):
        return list(self._ex.map(fn, jobs))


def oracle_pool(n):
    return _OraclePool(n)


def oracle_units_at(L, seed=7):
    """Measured single-thread oracle costs at L^4 (seconds): one gauge force,
    one exponential drift of every link and one Wilson action."""
    from oracle import gauge, integrators as it
    dims = (L,) * 4
    # the oracle's cost does not depend on the link values: a cold start
    # saves drawing 4 V Haar matrices
    u = inputs.cold_start(dims)
    p = inputs.gaussian_momenta(dims, seed)
    out = {}
    t0 = time.perf_counter()
    gauge.gauge_force(u, BETA)
    out["force_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    it.drift(u, p, 0.1)
    out["drift_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    gauge.wilson_action(u, BETA)
    out["action_s"] = time.perf_counter() - t0
    return out


def fg_trajectory_units(dt):
    """Forces, exponentials (drifts and FG displacements) and actions of one
    FG trajectory of length TAU as the oracle runs it (no merged kicks)."""
    n = int(round(TAU / dt))
    return {"force": 4 * n, "exp": 3 * n, "action": 2}


def cpu_baseline_measurement(args, pool_procs=None):
    """The oracle on the host's cores, bounded to ~a minute: (a) one force,
    one drift and one action measured at the benchmark's lattice on one
    thread, composed into the FG trajectory's unit counts; (b) independent
    FG trajectories on a 8^4 sample, one per process across all cores,
    measured, with their volume-scaled rate at the benchmark lattice
    labelled as scaled."""
    units = oracle_units_at(args.lattice)
    cnt = fg_trajectory_units(args.dt)
    traj_s = cnt["force"] * units["force_s"] + cnt["exp"] * units["drift_s"] + cnt["action"] * units["action_s"]
    nproc = pool_procs or os.cpu_count() or 1
    sample_l = 8
    with oracle_pool(nproc) as pool:
        pool.map(_oracle_traj_worker, [(4, args.integrator, args.dt, 1)] * nproc)   # import warm-up
        t0 = time.perf_counter()
        per = pool.map(_oracle_traj_worker, [(sample_l, args.integrator, args.dt, 50 + k) for k in range(nproc)])
        wall = time.perf_counter() - t0
    all_core_rate = nproc / wall
    scale = (sample_l / args.lattice) ** 4
    return {"value": 1.0 / traj_s, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one gauge force ({units['force_s']:.1f} s), one exponential drift ({units['drift_s']:.1f} s) "
                      f"and one Wilson action ({units['action_s']:.1f} s) measured at {args.lattice}^4 on one "
                      f"thread, composed into an FG trajectory (dt={args.dt}): {cnt['force']} forces, "
                      f"{cnt['exp']} exponentials, {cnt['action']} actions = {traj_s:.0f} s",
            "unit_times_s": units, "cpu": cpu_model(),
            "all_cores": {"processes": nproc, "sample": f"{nproc} independent FG trajectories (dt={args.dt}) on "
                                                        f"{sample_l}^4, one per process, measured",
                          "trajectories_per_s_measured": all_core_rate, "wall_s": wall,
                          "mean_trajectory_s": float(np.mean(per)),
                          "scaled_to_benchmark_lattice": all_core_rate * scale,
                          "scaling_note": f"x ({sample_l}/{args.lattice})^4: oracle work per trajectory is "
                                          "linear in the volume"},
            "unit_times": oracle_unit_times()}


def cpu_full_measurement(args):
    """Section 8(d)'s full oracle timing at the benchmark lattice (minutes):
    three force evaluations and one whole FG trajectory on one thread, and
    one trajectory per process on every core at once."""
    from oracle import gauge, integrators as it
    dims = (args.lattice,) * 4
    u = inputs.hot_start(dims, 3)
    forces = []
    for _ in range(3):
        t0 = time.perf_counter()
        gauge.gauge_force(u, BETA)
        forces.append(time.perf_counter() - t0)
    one = _oracle_traj_worker((args.lattice, args.integrator, args.dt, 5))
    nproc = os.cpu_count() or 1
    with oracle_pool(nproc) as pool:
        t0 = time.perf_counter()
        per = pool.map(_oracle_traj_worker, [(args.lattice, args.integrator, args.dt, 60 + k) for k in range(nproc)])
        wall = time.perf_counter() - t0
    return {"lattice": args.lattice, "cpu": cpu_model(), "force_s": forces, "trajectory_s_one_thread": one,
            "trajectories_per_s_one_thread": 1.0 / one,
            "all_cores": {"processes": nproc, "wall_s": wall, "trajectory_s": per,
                          "trajectories_per_s": nproc / wall}}


def run_reference(args):
    """The oracle as the reference arm: each step runs one FG trajectory on
    an 8^4 sample in every host core at once (independent chains, one per
    process); ms_per_step is that step's measured wall time.  `value` is the
    measured sample rate scaled to the benchmark lattice by the volume ratio
    (labelled in `scaled_from`); the measured rate is reported beside it."""
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    sample_l = 8
    nproc = os.cpu_count() or 1
    walls = []
    t_run = time.perf_counter()
    with oracle_pool(nproc) as pool:
        for k in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            pool.map(_oracle_traj_worker, [(sample_l, args.integrator, args.dt, 100 + k * nproc + j)
                                           for j in range(nproc)])
            w = time.perf_counter() - t0
            if k >= args.warmup:
                walls.append(w)
    run_s = time.perf_counter() - t_run
    step_s = float(np.mean(walls))
    measured = nproc / step_s
    scale = (sample_l / args.lattice) ** 4
    value = measured * scale
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * step_s, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "scaled_from": {"sample_lattice": [sample_l] * 4, "trajectories_per_s_measured": measured,
                        "factor": scale, "note": f"value = measured sample rate x ({sample_l}/{args.lattice})^4 "
                                                 "(oracle work per trajectory is linear in the volume)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nproc, "kind": "oracle", "cpu": cpu_model(),
                         "sample": f"each step: {nproc} independent FG trajectories (dt={args.dt}, tau={TAU}) on "
                                   f"{sample_l}^4, one per process on {nproc} host cores"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "run_s": run_s,
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(args):
    L = args.lattice
    return {
        "workload": f"pure-gauge SU(3) Wilson {L}^4, beta={BETA}, {args.integrator} integrator "
                    f"tau={TAU} dt={args.dt}, {args.precision} links/forces, FP64 dH sums, "
                    f"{args.link_reals}-real links, hot start + {THERM_TRAJ} thermalising trajectories "
                    f"(dt=1/8, always accepted) + {EQUIL_TRAJ} untimed Metropolis FG trajectories at dt=1/8",
        "lattice": [L] * 4, "beta": BETA, "integrator": args.integrator, "dt": args.dt, "tau": TAU,
        "precision": args.precision, "link_reals": args.link_reals,
        "l2": f"inputs larger than L2: gauge field "
              f"{4 * L**4 * args.link_reals * (4 if args.precision == 'fp32' else 8) / 1e6:.0f} MB",
        "parallelism": "replicas (one independent chain per GPU)",
    }


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- our arm
# Dslash algorithmic bytes per output site (FP32, 18-real links): 8 neighbour
# spinors (96 B) + 8 links (72 B) read, one spinor (96 B) written.
# dram__bytes_read + write of the fused force kernel per link, FP32 18-real,
# averaged over an FG trajectory's launch mix (ncu capture at 28^4)
FORCE_TRAFFIC_BYTES_PER_LINK = 203   # re-measure after a kernel change (None: not reported)
DSLASH_BYTES_FP32_18 = 8 * 96 + 8 * 72 + 96
# Compulsory bytes per output site of the four Dslash-class launches of a
# folded CG iteration (each of the 4V links is read once per half-lattice
# hop, every input and output spinor once): 8 * 72 + 96 + 96 each, plus the
# x term of t_e = p - k2 D t_o (96), the te, p, r reads of the launch that
# also sums <p,Ap>, Re<r,Ap>, |Ap|^2 (3 x 96), and the launch that updates
# the vectors: x, r, Ap, p read and x, r', p' written, one of the reads
# counted above as its input (6 x 96): (4 * 768 + 96 + 288 + 576) / 4 =
# 1008 B on average.
DSLASH_BYTES_CG_AVG = (4 * (8 * 72 + 96 + 96) + 96 + 3 * 96 + 6 * 96) // 4
# The same for the six-launch iteration (four Dslash launches, then axpy and
# xpay): t_o = D p, t_e = p - k2 D t_o (+96, the p read), t_o = D^dag t_e,
# Ap = t_e - k2 D^dag t_o with <p, Ap> (+2 x 96): (4 * 768 + 96 + 192) / 4.
DSLASH_BYTES_CG_SIX = (4 * (8 * 72 + 96 + 96) + 96 + 2 * 96) // 4
DSLASH_FLOP = 1320


def torch_sync():
    import torch
    torch.cuda.synchronize()


def fermion_measurement(fg, stream, rank, hbm_peak, dims=(16, 16, 16, 32)):
    """CG on the Nf=2 workload (16^3 x 32 by default); returns a dict for the JSON line."""
    dims = tuple(dims)
    gauge = fg.Lattice(dims, 5.6, precision="fp32", seed=300 + rank, stream=stream)
    gauge.set_gauge(inputs.hot_start(dims, 3 + rank))
    for _ in range(10):
        gauge.trajectory("fg", 0.125, TAU, refresh=True, u_accept=0.0)
    for _ in range(40):
        gauge.trajectory("fg", 0.25, TAU, refresh=True, u_accept=-1.0)
    u = gauge.get_gauge()
    plaq = gauge.plaquette()
    gauge.close()
    lat = fg.Lattice(dims, 5.6, kappa=0.158, precision="fp32", cg_tol=1e-10, seed=400 + rank,
                     stream=stream)
    lat.set_gauge(u)
    vh = inputs.volume(dims) // 2
    solves = 2
    bs = [inputs.gaussian_spinor_even(dims, 5 + k + rank) for k in range(solves + 2)]   # host RNG outside timing
    lat.cg_solve(bs[0])                    # warm-up (captures the iteration graphs for these links)
    iters, ru, res = 0, 0, 0.0
    t0 = time.perf_counter()
    for k in range(solves):
        _, info = lat.cg_solve(bs[1 + k])
        iters += info["iterations"]
        ru += info["reliable_updates"]
        res = max(res, info["true_residual"])
    wall = time.perf_counter() - t0
    # a second pass with per-launch CUDA-event timing (graphs off) for the
    # per-kernel breakdown and the Dslash roofline
    lat.timing(True)
    lat.timing_reset()
    _, info = lat.cg_solve(bs[-1])
    cls = {c: lat.kernel_time(c) for c in ("dslash", "dslash_df", "dslash_fp64", "cg_blas", "reduce", "convert")}
    lat.timing(False)
    # the library folds the vector updates into the Dslash launches on small
    # lattices only; the six-launch form runs two vector kernels per iteration
    folded = cls["cg_blas"][1] < info["iterations"]
    # the same solves with the other iteration form forced
    prev_fold = os.environ.get("FG_CG_FOLD")
    os.environ["FG_CG_FOLD"] = "0" if folded else "1"
    try:
        with fg.Lattice(dims, 5.6, kappa=0.158, precision="fp32", cg_tol=1e-10, seed=400 + rank,
                        stream=stream) as lalt:
            lalt.set_gauge(u)
            lalt.cg_solve(bs[0])
            t0 = time.perf_counter()
            its_alt = sum(lalt.cg_solve(bs[1 + k])[1]["iterations"] for k in range(solves))
            wall_alt = time.perf_counter() - t0
            lalt.timing(True)
            lalt.timing_reset()
            lalt.cg_solve(bs[-1])
            cls_alt = {c: lalt.kernel_time(c)[0] for c in ("dslash", "dslash_df", "dslash_fp64", "cg_blas", "reduce",
                                                           "convert")}
            lalt.timing(False)
    finally:
        if prev_fold is None:
            del os.environ["FG_CG_FOLD"]
        else:
            os.environ["FG_CG_FOLD"] = prev_fold
    other_form = {"iteration": "six launches" if folded else "folded (four launches)",
                  "ms_per_solve": 1000 * wall_alt / solves, "cg_iterations_per_solve": its_alt / solves,
                  "cg_blas_ms_share": cls_alt["cg_blas"] / max(sum(cls_alt.values()), 1e-9)}
    # pseudofermion force kernel: compulsory bytes per link = U (72) + F^a out
    # (32) + a quarter of the site's Xt and Yt spinors (2 x 96 / 4).  Each
    # force() solves for X first, so the kernel reads links and spinors the
    # solve has just left in L2 when they fit there (16^3 x 32: 80 MB); the
    # HBM figure is taken at 24^3 x 48 (405 MB), where they do not.
    def ff_kernel(l, n=5):
        l.force()
        l.timing(True)
        l.timing_reset()
        for _ in range(n):
            l.force()
        ms, cnt = l.kernel_time("fermion_force")
        l.timing(False)
        return ms / 1000.0 / max(cnt, 1), cnt

    lat.set_pseudofermion(inputs.gaussian_spinor_even(dims, 20 + rank))
    ffk_s, ffk_n = ff_kernel(lat)
    big = (24, 24, 24, 48)
    with fg.Lattice(big, 5.6, kappa=0.158, precision="fp32", cg_tol=1e-8, seed=450 + rank, stream=stream) as lb:
        lb.random_gauge()
        lb.refresh_pseudofermion()
        ffb_s, ffb_n = ff_kernel(lb)
    vhb = inputs.volume(big) // 2
    ff_roof = {"bound": "hbm", "lattice": "24^3x48 (fields > L2)", "bytes_per_link": 152,
               "links_per_launch": 4 * 2 * vhb, "avg_launch_us": ffb_s * 1e6, "launches": ffb_n,
               "achieved": 152 * 4 * 2 * vhb / ffb_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
               "l2_resident": {"lattice": "x".join(map(str, dims)), "avg_launch_us": ffk_s * 1e6,
                               "launches": ffk_n, "bytes_per_s_over_hbm_peak":
                                   152 * 4 * 2 * vh / ffk_s / 1e9 / hbm_peak}}
    ff_roof["frac"] = ff_roof["achieved"] / hbm_peak
    # FG trajectories on the total force (tau = 1, dt = 0.1 and 0.05) from one
    # start (links, momenta, chi), and the FP64 path's dH for dt = 0.1
    chi = inputs.gaussian_spinor_even(dims, 21 + rank)
    p0 = inputs.gaussian_momenta(dims, 22 + rank)
    trajs = {}
    for integ, dt in (("fg", 0.1), ("fg", 0.05), ("fg_analytic", 0.1), ("omelyan", 0.1), ("omelyan", 0.05)):
        lat.set_gauge(u)
        lat.set_momenta(p0)
        lat.set_pseudofermion(chi)
        torch_sync()
        t0 = time.perf_counter()
        r = lat.trajectory(integ, dt, TAU, refresh=False, u_accept=0.0)
        ms = 1000 * (time.perf_counter() - t0)
        trajs[f"{integ}_dt_{dt}"] = {"dH": r["dH"], "ms": ms, "forces": r["n_force"], "solves": r["n_solves"],
                                     "cg_iterations": r["cg_iters"]}
    # two-level integrators: outer step on S_F at twice the step, gauge inside
    for outer, inner, m, dt in (("fg", "fg", 1, 0.2), ("fg", "fg", 2, 0.2), ("fg", "omelyan", 2, 0.2),
                                ("fg", "omelyan", 4, 0.2), ("omelyan", "omelyan", 4, 0.1)):
        lat.set_gauge(u)
        lat.set_momenta(p0)
        lat.set_pseudofermion(chi)
        torch_sync()
        t0 = time.perf_counter()
        r = lat.trajectory_nested(outer, inner, m, dt, TAU, refresh=False, u_accept=0.0)
        ms = 1000 * (time.perf_counter() - t0)
        trajs[f"nested_{outer}_over_{m}x{inner}_dt_{dt}"] = {"dH": r["dH"], "ms": ms, "solves": r["n_solves"],
                                                            "cg_iterations": r["cg_iters"]}
    # the same solves and one FG trajectory with the half-precision inner solver
    half = {}
    lat16 = fg.Lattice(dims, 5.6, kappa=0.158, precision="fp32_fp16cg", cg_tol=1e-10, seed=400 + rank,
                       stream=stream)
    lat16.set_gauge(u)
    lat16.cg_solve(bs[0])
    its16, ru16, res16 = 0, 0, 0.0
    t0 = time.perf_counter()
    for k in range(solves):
        _, info = lat16.cg_solve(bs[1 + k])
        its16 += info["iterations"]
        ru16 += info["reliable_updates"]
        res16 = max(res16, info["true_residual"])
    half["ms_per_solve"] = 1000 * (time.perf_counter() - t0) / solves
    half["cg_iterations_per_solve"] = its16 / solves
    half["reliable_updates_per_solve"] = ru16 / solves
    half["true_residual_max"] = res16
    lat16.timing(True)
    lat16.timing_reset()
    lat16.cg_solve(bs[-1])
    half["device_ms_per_solve_by_class"] = {c: lat16.kernel_time(c)[0]
                                            for c in ("dslash", "dslash_df", "dslash_fp64", "cg_blas", "convert")}
    d16_ms, d16_n = lat16.kernel_time("dslash")
    half["dslash_avg_launch_us"] = 1000.0 * d16_ms / max(d16_n, 1)
    lat16.timing(False)
    lat16.set_gauge(u)
    lat16.set_momenta(p0)
    lat16.set_pseudofermion(chi)
    torch_sync()
    t0 = time.perf_counter()
    r = lat16.trajectory("fg", 0.1, TAU, refresh=False, u_accept=0.0)
    half["fg_dt_0.1"] = {"dH": r["dH"], "ms": 1000 * (time.perf_counter() - t0), "solves": r["n_solves"],
                         "cg_iterations": r["cg_iters"]}
    lat16.close()
    lat64 = fg.Lattice(dims, 5.6, kappa=0.158, precision="fp64", cg_tol=1e-10, seed=400 + rank, stream=stream)
    lat64.set_gauge(u)
    lat64.set_momenta(p0)
    lat64.set_pseudofermion(chi)
    t0 = time.perf_counter()
    r64 = lat64.trajectory("fg", 0.1, TAU, refresh=False, u_accept=0.0)
    ms64 = 1000 * (time.perf_counter() - t0)
    lat64.close()
    trajs["fp64_fg_dt_0.1"] = {"dH": r64["dH"], "ms": ms64, "solves": r64["n_solves"],
                               "cg_iterations": r64["cg_iters"]}
    trajs["dH_error_fp32_vs_fp64_dt_0.1"] = abs(trajs["fg_dt_0.1"]["dH"] - r64["dH"])
    lat.close()
    inner16 = inner_precision_measurement(fg, stream, rank, u, dims)
    ds_ms, ds_n = cls["dslash"]
    avg = ds_ms / 1000.0 / max(ds_n, 1)
    dslash_bytes = DSLASH_BYTES_CG_AVG if folded else DSLASH_BYTES_CG_SIX
    achieved = dslash_bytes * vh / avg / 1e9
    return {
        "workload": f"Nf=2 Wilson {dims[0]}^3x{dims[3]}, beta=5.6, kappa=0.158, even-odd CG on Mhat^dag Mhat "
                    "to 1e-10 (FP32 inner, FP64 reliable updates), gauge field: hot start + 50 FG trajectories",
        "plaquette": plaq, "cg_iterations_per_solve": iters / solves, "reliable_updates_per_solve": ru / solves,
        "true_residual_max": res,
        "ms_per_solve": 1000 * wall / solves,
        "ms_per_solve_note": "wall clock of fg_cg_solve, including the pageable host copies of b and x",
        "us_per_cg_iteration": 1e6 * wall / max(iters, 1),
        "device_ms_per_solve_by_class": {c: v[0] for c, v in cls.items()},
        "launches_per_solve_by_class": {c: v[1] for c, v in cls.items()},
        "dslash_roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                            "frac": achieved / hbm_peak, "traffic": None,
                            "bytes_per_site": dslash_bytes,
                            "bytes_per_site_no_cache_reuse": DSLASH_BYTES_FP32_18,
                            "sites_per_launch": vh, "avg_launch_us": avg * 1e6, "launches": ds_n,
                            "gflops": DSLASH_FLOP * vh / avg / 1e9},
        "cg_blas_ms_share": cls["cg_blas"][0] / max(sum(v[0] for v in cls.values()), 1e-9),
        "cg_iteration": "folded (four launches)" if folded else "six launches (four Dslash, axpy, xpay)",
        "cg_other_iteration_form": other_form,
        "fermion_force_roofline": ff_roof,
        "trajectories": trajs,
        "half_precision_cg": half,
        "inner_precision_16bit": inner16,
        "trajectories_note": "one FG trajectory per entry from the same links, momenta and chi; FP32 "
                             "links/forces with the mixed solver vs the FP64 path; ms is wall clock",
    }


def inner_precision_measurement(fg, stream, rank, u_small, dims_small, solves=3):
    """The inner solver's storage format at the two Nf=2 sizes (16^3 x 32,
    whose fields fit in L2, with the thermalised links of the Nf=2
    measurement; 24^3 x 48, which does not, from a device hot start and 20
    FG trajectories): FP32, IEEE half and bfloat16 links and vectors (the
    16-bit ones with reliable updates at least every factor 0.1 of residual,
    bfloat16 also every 0.3), solves to 1e-10 at kappa 0.158.  Device time
    is the sum of the solver's kernels over one timed solve (single
    launches); wall time includes the pageable copies of b and x."""
    big = (24, 24, 24, 48)
    th = fg.Lattice(big, 5.6, precision="fp32", seed=480 + rank, stream=stream)
    th.random_gauge()
    for _ in range(10):
        th.trajectory("fg", 0.125, TAU, refresh=True, u_accept=0.0)
    for _ in range(10):
        th.trajectory("fg", 0.25, TAU, refresh=True, u_accept=-1.0)
    u_big = th.get_gauge()
    th.close()
    out = {}
    for dims, u in ((tuple(dims_small), u_small), (big, u_big)):
        bs = [inputs.gaussian_spinor_even(dims, 70 + k + rank) for k in range(solves + 2)]
        res = {}
        for prec, delta in (("fp32", 0.01), ("fp32_fp16cg", 0.1), ("fp32_bf16cg", 0.1), ("fp32_bf16cg", 0.3)):
            try:
                res[f"{prec}_delta_{delta}"] = _time_inner_solves(fg, stream, rank, dims, u, bs, prec, delta, solves)
            except fg.FgError as e:     # a 16-bit solver that does not reach the tolerance is a result too
                res[f"{prec}_delta_{delta}"] = {"error": str(e)}
        out["x".join(map(str, dims))] = res
    return out


def _time_inner_solves(fg, stream, rank, dims, u, bs, prec, delta, solves):
    """Solves of the inner-precision comparison on one handle (see above)."""
    with fg.Lattice(dims, 5.6, kappa=0.158, precision=prec, cg_tol=1e-10, cg_delta=delta, seed=490 + rank,
                    stream=stream) as l:
        l.set_gauge(u)
        l.cg_solve(bs[0])
        it = ru = 0
        rmax = 0.0
        t0 = time.perf_counter()
        for k in range(solves):
            _, info = l.cg_solve(bs[1 + k])
            it += info["iterations"]
            ru += info["reliable_updates"]
            rmax = max(rmax, info["true_residual"])
        wall_ms = 1000 * (time.perf_counter() - t0) / solves
        l.timing(True)
        l.timing_reset()
        l.cg_solve(bs[-1])
        dev_ms = sum(l.kernel_time(c)[0] for c in ("dslash", "dslash_df", "dslash_fp64", "cg_blas",
                                                   "reduce", "convert"))
        l.timing(False)
    return {"device_ms_per_solve": dev_ms, "wall_ms_per_solve": wall_ms,
            "cg_iterations_per_solve": it / solves,
            "reliable_updates_per_solve": ru / solves, "true_residual_max": rmax}


def precision_measurement(fg, stream, rank, L=16, n_time=5):
    """FP64 vs FP32 links/forces and 18- vs 12-real storage on 16^4 (beta 6):
    dH of one FG (dt 0.25) and one Omelyan (dt 0.125) trajectory from the same
    thermalised links and momenta, the error against FP64, trajectories/s and
    the force kernel's algorithmic GB/s."""
    import torch
    dims = (L,) * 4
    base = fg.Lattice(dims, BETA, precision="fp64", seed=500 + rank, stream=stream)
    base.set_gauge(inputs.hot_start(dims, 11 + rank))
    for _ in range(THERM_TRAJ):
        base.trajectory("fg", 0.125, TAU, refresh=True, u_accept=0.0)
    u = base.get_gauge()
    base.close()
    p0 = inputs.gaussian_momenta(dims, 13 + rank)
    out, ref = {}, {}
    for name, prec, reals in (("fp64_18", "fp64", 18), ("df64_18", "df64", 18), ("fp32_18", "fp32", 18),
                              ("fp32_12", "fp32", 12)):
        lat = fg.Lattice(dims, BETA, precision=prec, link_reals=reals, seed=600 + rank, stream=stream)
        row = {}
        for integ, dt in (("fg", 0.25), ("omelyan", 0.125)):
            lat.set_gauge(u)
            lat.set_momenta(p0)
            r = lat.trajectory(integ, dt, TAU, refresh=False, u_accept=0.0)
            row[f"dH_{integ}_dt_{dt}"] = r["dH"]
            if prec == "fp64":
                ref[integ] = r["dH"]
            else:
                row[f"dH_error_vs_fp64_{integ}"] = abs(r["dH"] - ref[integ])
        lat.set_gauge(u)
        lat.trajectory("fg", 0.25, TAU, refresh=True, u_accept=0.0)
        st = torch.cuda.ExternalStream(stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(n_time):
            lat.trajectory("fg", 0.25, TAU, refresh=True, u_accept=0.0)
        e1.record(st)
        torch.cuda.synchronize()
        row["fg_trajectories_per_s"] = n_time / (e0.elapsed_time(e1) / 1000.0)
        lat.timing(True)
        lat.timing_reset()
        lat.trajectory("fg", 0.25, TAU, refresh=True, u_accept=0.0)
        f_ms, f_n = lat.kernel_time("gauge_force")
        lat.timing(False)
        lat.close()
        esize = 4 if prec == "fp32" else 8
        link_bytes = reals * esize + 2 * 8 * esize
        row["force_avg_launch_us"] = 1000.0 * f_ms / max(f_n, 1)
        row["force_algorithmic_gbs"] = link_bytes * 4 * L ** 4 / (f_ms / 1000.0 / max(f_n, 1)) / 1e9
        row["force_bytes_per_link"] = link_bytes
        out[name] = row
    out["workload"] = (f"pure-gauge {L}^4, beta={BETA}, hot start + {THERM_TRAJ} FP64 FG trajectories; one "
                       "trajectory per integrator from the same links and momenta")
    out["error_vs_volume"] = error_vs_volume(fg, stream, rank)
    return out


def error_vs_volume(fg, stream, rank, sizes=(4, 8, 12, 16, 24, 32)):
    """|dH - dH_fp64| of one FG trajectory (dt 1/8, tau 1) for double-float
    and FP32 fields against the FP64 path (itself pinned to the oracle), per
    volume, from the same links (hot start + 3 FP32 FG trajectories) and
    momenta."""
    rows = {}
    for L in sizes:
        dims = (L,) * 4
        th = fg.Lattice(dims, BETA, precision="fp32", seed=40 + rank, stream=stream)
        th.set_gauge(inputs.hot_start(dims, 41 + rank))
        for _ in range(3):
            th.trajectory("fg", 0.125, TAU, refresh=True, u_accept=0.0)
        u = th.get_gauge()
        th.close()
        p = inputs.gaussian_momenta(dims, 42 + rank)
        dh = {}
        for prec in ("fp64", "df64", "fp32"):
            lat = fg.Lattice(dims, BETA, precision=prec, seed=43, stream=stream)
            lat.set_gauge(u)
            lat.set_momenta(p)
            dh[prec] = lat.trajectory("fg", 0.125, TAU, refresh=False, u_accept=0.0)["dH"]
            lat.close()
        rows[f"{L}^4"] = {"dH_fp64": dh["fp64"], "df64_error": abs(dh["df64"] - dh["fp64"]),
                          "fp32_error": abs(dh["fp32"] - dh["fp64"])}
    return {"workload": f"FG dt=1/8 tau=1, beta={BETA}, hot start + 3 FP32 FG trajectories, one trajectory "
                        "per precision from the same links and momenta; errors against the FP64 path",
            "by_volume": rows}


def batched_measurement(fg, stream, rank, n_traj=6, n_oracle=6):
    """64 independent chains, volumes drawn from {4,6,8,10,12}^4 and beta from
    U[5.7, 6.2] (seed 4), FG tau=1 dt=1/8: the batches (one launch per MD
    sub-step for all chains, one CUDA graph per trajectory, autotuned tiles)
    in double-float and in FP32, against the plain FP64 one-chain-per-launch
    path on the same configurations.  Reports accepted trajectories per
    second and <exp(-dH)>, and each batch's dH error on every chain: one
    trajectory from the same links and uploaded momenta against the FP64
    path, and against the FP64 oracle on the n_oracle smallest chains."""
    import torch
    rng = inputs.make_rng(4 + 1000 * rank)
    extents = rng.choice([4, 6, 8, 10, 12], size=64)
    betas = rng.uniform(5.7, 6.2, size=64)
    dims_list = [(int(L),) * 4 for L in extents]
    sites = int(sum(L ** 4 for L in extents))
    # thermalised starts from the FP32 batch
    bat = fg.Batch(dims_list, betas, precision="fp32", tile=0, use_graphs=True, seed=500 + rank, stream=stream)
    for k, d in enumerate(dims_list):
        bat.set_gauge(k, inputs.hot_start(d, 700 + k + 1000 * rank))
    for _ in range(20):
        bat.trajectory("fg", 0.125, 1.0, refresh=True, always_accept=True)
    for _ in range(20):
        bat.trajectory("fg", 0.125, 1.0, refresh=True, always_accept=False)
    starts = [bat.get_gauge(k) for k in range(64)]
    bat.close()
    moms = [inputs.gaussian_momenta(d, 800 + k + 1000 * rank) for k, d in enumerate(dims_list)]

    def stats(res, secs):
        flat = [r for sweep in res for r in sweep]
        acc = sum(r["accepted"] for r in flat)
        e = np.array([np.exp(-r["dH"]) for r in flat])
        return {"accepted_traj_per_s": acc / secs, "traj_per_s": len(flat) / secs,
                "acceptance": acc / len(flat), "mean_exp_minus_dH": float(e.mean()),
                "mean_exp_minus_dH_err": float(e.std(ddof=1) / np.sqrt(len(e)))}

    # one chain per launch, FP64: the precision reference and the speed baseline
    lats = []
    for k, d in enumerate(dims_list):
        lat = fg.Lattice(d, float(betas[k]), precision="fp64", seed=900 + k + 1000 * rank, stream=stream)
        lats.append(lat)
    dh64 = []
    for k, lat in enumerate(lats):
        lat.set_gauge(starts[k])
        lat.set_momenta(moms[k])
        dh64.append(lat.trajectory("fg", 0.125, 1.0, refresh=False, u_accept=0.0)["dH"])
        lat.set_gauge(starts[k])
    dh64 = np.array(dh64)
    for lat in lats:      # warm-up
        lat.trajectory("fg", 0.125, 1.0, refresh=True, u_accept=-1.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res_s = [[lat.trajectory("fg", 0.125, 1.0, refresh=True, u_accept=-1.0) for lat in lats]
             for _ in range(n_traj)]
    ts = time.perf_counter() - t0
    for lat in lats:
        lat.close()
    s1 = stats(res_s, ts)

    # the FP64 oracle on the smallest chains (same links and momenta)
    from oracle import integrators as it
    small = sorted(range(64), key=lambda k: (extents[k], k))[:n_oracle]
    dh_or = {}
    for k in small:
        _, _, h0, h1 = it.trajectory(it.GaugeSystem(float(betas[k])), it.Integrator("fg"), starts[k], moms[k],
                                     0.125, 1.0)
        dh_or[k] = h1 - h0
    out = {"workload": "64 pure-gauge chains, L^4 with L drawn from {4,6,8,10,12} and beta from U[5.7,6.2] "
                       "(seed 4), FG tau=1 dt=1/8", "sites_total": sites,
           "one_chain_per_launch_fp64": s1, "trajectories_timed_per_chain": n_traj,
           "fp64_path_vs_oracle_max_abs_dH_error": float(max(abs(dh64[k] - dh_or[k]) for k in small)),
           "oracle_chains": [int(extents[k]) for k in small]}
    for prec in ("df64", "fp32"):
        bat = fg.Batch(dims_list, betas, precision=prec, tile=0, use_graphs=True, seed=500 + rank, stream=stream)
        for k in range(64):
            bat.set_gauge(k, starts[k])
            bat.set_momenta(k, moms[k])
        r0 = bat.trajectory("fg", 0.125, 1.0, refresh=False, always_accept=False)
        dh = np.array([r["dH"] for r in r0])
        for k in range(64):
            bat.set_gauge(k, starts[k])
        for _ in range(2):   # autotune, graph capture, warm-up
            bat.trajectory("fg", 0.125, 1.0, refresh=True, always_accept=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res_b = [bat.trajectory("fg", 0.125, 1.0, refresh=True, always_accept=False) for _ in range(n_traj)]
        tb = time.perf_counter() - t0
        b = stats(res_b, tb)
        b["tile"] = bat.tile()
        bat.close()
        err = np.abs(dh - dh64)
        b["dH_error_vs_fp64_path"] = {"max": float(err.max()), "median": float(np.median(err)),
                                      "max_by_L": {str(L): float(err[extents == L].max()) for L in (4, 6, 8, 10, 12)
                                                   if (extents == L).any()}}
        b["dH_error_vs_oracle_max"] = float(max(abs(dh[k] - dh_or[k]) for k in small))
        b["meets_1e-6"] = bool(err.max() <= 1e-6 and b["dH_error_vs_oracle_max"] <= 1e-6)
        b["speedup_accepted_per_s_vs_fp64_one_chain"] = b["accepted_traj_per_s"] / s1["accepted_traj_per_s"]
        out[f"batched_{prec}_graphs"] = b
    return out


def fixed_acceptance_comparison(lat, torch, n_stat=200, n_tune=30, target=0.75):
    """FG against Omelyan at matched acceptance on the running chain (section
    5 compares integrators at equal acceptance, Fig. 2 at 75%): for each
    integrator the fewest steps per unit trajectory whose acceptance over
    n_tune trajectories reaches the target (else the most steps tried),
    then n_stat trajectories there.  Reports acceptance and <exp(-dH)> with
    their standard errors, accepted trajectories/s and force evaluations per
    accepted trajectory (the paper's cost model counts force/solve
    evaluations), and the FG / Omelyan ratio of accepted trajectories/s with
    its error from the two acceptances."""
    out = {}
    order = {"fg": 4, "omelyan": 2}
    dh75 = 4.0 * erfcinv(target) ** 2            # <dH> at which erfc(sqrt(<dH>) / 2) = target
    for integ, steps in (("fg", (5, 6, 7, 8, 10)), ("omelyan", (20, 24, 28, 32, 36, 40))):
        chosen, tune = steps[-1], {}
        for n in steps:
            rs = [lat.trajectory(integ, 1.0 / n, TAU, refresh=True, u_accept=-1.0) for _ in range(n_tune)]
            a = float(np.mean([r["accepted"] for r in rs]))
            tune[str(n)] = a
            if a >= target:
                chosen = n
                break
        dt = 1.0 / chosen
        torch.cuda.synchronize()
        c0 = time.perf_counter()
        rs = [lat.trajectory(integ, dt, TAU, refresh=True, u_accept=-1.0) for _ in range(n_stat)]
        torch.cuda.synchronize()
        secs = time.perf_counter() - c0
        acc = np.array([r["accepted"] for r in rs], dtype=float)
        dh = np.array([r["dH"] for r in rs])
        e = np.exp(-dh)
        a = float(acc.mean())
        a_err = float(np.sqrt(max(a * (1 - a), 1e-12) / len(rs)))
        # the steps per unit trajectory that would give the target acceptance,
        # from <dH> ~ dt^(2 p) for an integrator of order p
        mdh = float(dh.mean())
        n75 = chosen * (max(mdh, 1e-12) / dh75) ** (1.0 / (2 * order[integ]))
        forces75 = (3 if integ == "fg" else 2) * n75 + 1
        out[integ] = {"md_steps": chosen, "dt": dt, "forces_per_trajectory": rs[0]["n_force"],
                      "mean_dH": mdh, "mean_dH_err": float(dh.std(ddof=1) / np.sqrt(len(dh))),
                      "model_md_steps_at_target": n75,
                      "model_forces_per_accepted_at_target": forces75 / target,
                      "trajectories": len(rs), "acceptance": a, "acceptance_err": a_err,
                      "mean_exp_minus_dH": float(e.mean()), "mean_exp_minus_dH_err": float(e.std(ddof=1) / np.sqrt(len(e))),
                      "trajectories_per_s": len(rs) / secs, "accepted_per_s": a * len(rs) / secs,
                      "accepted_per_s_err": a_err * len(rs) / secs,
                      "forces_per_accepted_trajectory": rs[0]["n_force"] / max(a, 1e-12),
                      "tuning_acceptance": tune}
    f, o = out["fg"], out["omelyan"]
    ratio = f["accepted_per_s"] / o["accepted_per_s"]
    rel = np.hypot(f["acceptance_err"] / f["acceptance"], o["acceptance_err"] / o["acceptance"])
    out["fg_over_omelyan_accepted_per_s"] = {"ratio": ratio, "err": float(ratio * rel)}
    cost = o["forces_per_accepted_trajectory"] / f["forces_per_accepted_trajectory"]
    out["omelyan_over_fg_forces_per_accepted"] = {"ratio": cost, "err": float(cost * rel)}
    out["model_omelyan_over_fg_forces_per_accepted_at_target"] = {
        "ratio": o["model_forces_per_accepted_at_target"] / f["model_forces_per_accepted_at_target"],
        "model": "acceptance = erfc(sqrt(<dH>) / 2) and <dH> ~ dt^(2 p) (p = 4 for FG, 2 for Omelyan), from each "
                 "integrator's measured <dH>; forces per trajectory 3 n + 1 (FG) and 2 n + 1 (Omelyan) at the "
                 "step count n that gives the target acceptance (section 5's cost model counts force "
                 "evaluations, Fig. 2 compares at 75% acceptance)"}
    out["target_acceptance"] = target
    return out


def erfcinv(y):
    """Inverse complementary error function (scipy)."""
    from scipy.special import erfcinv as _e
    return float(_e(y))


def headline_precision_check(fg, lat, stream, args, seed=91):
    """dH of one trajectory of the benchmark chain's configuration (its
    current links, fresh momenta) in its own precision, in double-float and
    in FP64 (the FP64 path is pinned to the oracle): the error against FP64.
    The chain's links are put back afterwards."""
    u = lat.get_gauge()
    p = inputs.gaussian_momenta(lat.dims, seed)
    dh = {}
    for prec in dict.fromkeys((args.precision, "df64", "fp64")):
        if prec == args.precision:
            x = lat
        else:
            x = fg.Lattice(lat.dims, BETA, precision=prec, link_reals=18, seed=92, stream=stream)
        x.set_gauge(u)
        x.set_momenta(p)
        dh[prec] = x.trajectory(args.integrator, args.dt, TAU, refresh=False, u_accept=0.0)["dH"]
        if x is not lat:
            x.close()
    lat.set_gauge(u)
    return {"dH_fp64": dh["fp64"],
            "dH_error_vs_fp64": {k: abs(v - dh["fp64"]) for k, v in dh.items() if k != "fp64"},
            "note": "one trajectory from the benchmark chain's links after the timed region, momenta seed "
                    f"{seed}; each precision from the same links and momenta"}


def serving_measurement(duration_s=4.0, rate_hz=200.0, slots=8, budget_gb=24.0):
    """Poisson stream of trajectory requests (seed 5) over 32 resident chains
    (70% pure gauge at 8^4..24^4, 30% Nf=2 Wilson at 8^3x16 / 12^3x24),
    Omelyan or FG with dt 1/8 or 1/12, FP32, admission by HBM footprint."""
    from paper_0910_2950_gb300 import serve
    chains = serve.served_chain_mix(32, seed=5)
    reqs = serve.poisson_stream(rate_hz, duration_s, chains, seed=5)
    srv = serve.TrajectoryServer(slots=slots, hbm_budget_bytes=int(budget_gb * (1 << 30)))
    res, wall, busy = srv.serve(reqs, realtime=True)
    lat = np.array([r.latency for r in res])
    nf2 = np.array([chains[r.chain].kappa > 0 for r in res])
    out = {
        "workload": f"Poisson {rate_hz:g} requests/s for {duration_s:g} s over 32 chains (70% pure gauge L^4, "
                    "L in {8,12,16,24}, beta in [5.7,6.2]; 30% Nf=2 Wilson 8^3x16 / 12^3x24, kappa in "
                    "[0.155,0.159]); Omelyan or FG, dt 1/8 or 1/12, FP32; chains resident on device",
        "requests": len(res), "slots": slots, "hbm_budget_gb": budget_gb,
        "trajectories_per_s": len(res) / wall, "wall_s": wall, "utilisation": busy / wall,
        "latency_ms": {"p50": 1000 * float(np.percentile(lat, 50)), "p99": 1000 * float(np.percentile(lat, 99)),
                       "max": 1000 * float(lat.max())},
        "latency_ms_pure_gauge_p50_p99": [1000 * float(np.percentile(lat[~nf2], q)) for q in (50, 99)]
        if (~nf2).any() else None,
        "latency_ms_nf2_p50_p99": [1000 * float(np.percentile(lat[nf2], q)) for q in (50, 99)] if nf2.any() else None,
        "acceptance": float(np.mean([r.accepted for r in res])),
        "evictions": srv.evictions, "peak_resident_gb": srv.peak_resident_bytes / (1 << 30),
        "offered_load_stable": bool(wall < duration_s * 1.5),
    }
    srv.close()
    return out


def run_ours(args):
    rank, world, local = dist_info()
    import torch
    import torch.distributed as dist

    cpu = None
    if rank == 0 and world >= 1 and not args.no_cpu_baseline:
        # oracle first, before this process touches the GPU (its process pool is spawned)
        cpu = cpu_baseline_measurement(args)
        if args.cpu_full:
            cpu["full_8d"] = cpu_full_measurement(args)

    if world > 1:
        dist.init_process_group("nccl", rank=rank, world_size=world)
    torch.cuda.set_device(local)
    from paper_0910_2950_gb300 import build, fg
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    fg.load()

    L = args.lattice
    dims = (L,) * 4
    stream = torch.cuda.Stream()
    seeds = rank_seeds(rank)
    lat = fg.Lattice(dims, BETA, precision=args.precision, link_reals=args.link_reals,
                     seed=seeds["device_rng"], stream=stream.cuda_stream)
    u0 = inputs.hot_start(dims, seeds["hot_start"])
    lat.set_gauge(u0)
    del u0
    for _ in range(THERM_TRAJ):
        lat.trajectory("fg", 0.125, TAU, refresh=True, u_accept=0.0)
    # equilibrate with Metropolis at dt = 1/8 (untimed)
    for _ in range(EQUIL_TRAJ):
        lat.trajectory("fg", 0.125, TAU, refresh=True, u_accept=-1.0)
    for _ in range(args.warmup):
        lat.trajectory(args.integrator, args.dt, TAU, refresh=True, u_accept=-1.0)

    clocks = ClockSampler(local)
    lat.timing(True)
    lat.timing_reset()
    lat.timing(True)
    n_launch0 = lat.launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    results = []
    for _ in range(args.steps):
        results.append(lat.trajectory(args.integrator, args.dt, TAU, refresh=True, u_accept=-1.0))
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    launches = lat.launch_count() - n_launch0
    force_ms, force_n = lat.kernel_time("gauge_force")
    lat.timing(False)

    max_ms = reduce_max(elapsed_ms, world, "cuda")
    value = whole_job_rate(args.steps, world, max_ms / 1000.0)

    acc = float(np.mean([r["accepted"] for r in results]))
    emdh = float(np.mean([np.exp(-r["dH"]) for r in results]))
    n_force = results[0]["n_force"]
    nsteps = results[0]["n_steps"]

    # ---------------------------------------------------------------- roofline (gauge force)
    links = 4 * lat.V
    reunit = 1 if args.precision == "fp32" else 0
    FLOP_FORCE = FLOP_STAPLES[(args.precision, args.link_reals)] + FLOP_FORCE_REST
    # per FG trajectory: n (kick+drift) + n displacements + n (FG kick + drift) + 1 final kick
    if args.integrator in ("fg", "force_gradient"):
        per_traj = nsteps * (FLOP_FORCE + FLOP_KICK + FLOP_EXP_MUL + reunit * FLOP_REUNIT)   # P Q
        per_traj += nsteps * (FLOP_FORCE + FLOP_EXP_MUL)                                     # G displace
        per_traj += nsteps * (FLOP_FORCE + FLOP_KICK + FLOP_EXP_MUL + reunit * FLOP_REUNIT)  # G kick + Q
        per_traj += FLOP_FORCE + FLOP_KICK                                                  # final P
    else:
        per_traj = n_force * (FLOP_FORCE + FLOP_KICK + FLOP_EXP_MUL)
    flops_per_launch = per_traj * links / n_force
    avg_launch_s = force_ms / 1000.0 / max(force_n, 1)
    achieved = flops_per_launch / avg_launch_s / 1e12
    esize = 4 if args.precision == "fp32" else 8
    bytes_per_launch = links * (args.link_reals * esize + 2 * 8 * esize)
    # FP32 FMA peak from this GPU's SM count and the maximum SM clock sampled
    # during the timed region (the unit counts: 128 FP32 lanes per SM, 2 flop
    # per FMA); the constant for 152 SMs at 2070 MHz if either is missing
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    sm_max_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    fp32_peak = sm_count * 128 * 2 * sm_max_mhz * 1e6 / 1e12 if sm_count else FP32_PEAK_TFLOPS
    peak = fp32_peak if args.precision == "fp32" else FP64_PEAK_TFLOPS * fp32_peak / FP32_PEAK_TFLOPS
    # DRAM bytes per link of the FP32 18-real FG mix from one ncu capture of
    # the force kernel at 28^4 (its summary is kept with the profiles),
    # scaled to this lattice
    traffic = (FORCE_TRAFFIC_BYTES_PER_LINK * links
               if FORCE_TRAFFIC_BYTES_PER_LINK is not None
               and (args.precision, args.link_reals, args.integrator) == ("fp32", 18, "fg") else None)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic,
            "traffic_note": "bytes per launch: 203 B/link measured by ncu at 28^4, scaled by links" if traffic
            else None,
            "peak_derivation": f"{sm_count} SMs x 128 FP32 lanes x 2 flop x {sm_max_mhz:g} MHz (maximum SM clock "
                               "sampled by nvidia-smi during the timed region); FP64 at 1/64 of it",
            "kernel": "gauge_force (fused staple force + kick/drift/displace)",
            "launches": force_n, "avg_launch_us": avg_launch_s * 1e6,
            "algorithmic_gbs": bytes_per_launch / avg_launch_s / 1e9,
            "share_of_step": force_ms / elapsed_ms}
    # cross-check of the derived peak: the FP32 FMA rate independent FMA
    # chains reach on this GPU now (after the timed region)
    try:
        fma = fg.fp32_fma_rate()
    except fg.FgError:
        fma = None
    roof["measured_fp32_fma_tflops"] = fma
    roof["frac_of_measured_fma"] = (achieved / fma if fma and args.precision == "fp32" else None)

    # ---------------------------------------------------------------- dH error of the headline precision
    headline_dh = headline_precision_check(fg, lat, stream.cuda_stream, args) if not args.no_compare else None

    # ---------------------------------------------------------------- FG vs Omelyan
    # Section 5 compares integrators at equal acceptance; on this chain: FG at
    # the configured dt and at dt/2, Omelyan at the configured 0.125 and 1/16,
    # then both tuned to ~75% acceptance with statistics.
    comparison = None
    if not args.no_compare:
        comparison = {}
        for name, integ, dt in [("fg_dt_0.25", "fg", 0.25), ("fg_dt_0.125", "fg", 0.125),
                                ("fg_analytic_dt_0.25", "fg_analytic", 0.25),
                                ("fg_analytic_dt_0.125", "fg_analytic", 0.125),
                                ("omelyan_dt_0.125", "omelyan", 0.125), ("omelyan_dt_0.0625", "omelyan", 0.0625)]:
            for _ in range(2):
                lat.trajectory(integ, dt, TAU, refresh=True, u_accept=-1.0)
            torch.cuda.synchronize()
            c0 = time.perf_counter()
            rs = [lat.trajectory(integ, dt, TAU, refresh=True, u_accept=-1.0) for _ in range(args.compare_steps)]
            torch.cuda.synchronize()
            secs = time.perf_counter() - c0
            a_cmp = float(np.mean([r["accepted"] for r in rs]))
            comparison[name] = {"dt": dt, "forces_per_trajectory": rs[0]["n_force"], "acceptance": a_cmp,
                                "mean_dH": float(np.mean([r["dH"] for r in rs])),
                                "trajectories_per_s": len(rs) / secs, "accepted_per_s": a_cmp * len(rs) / secs}
        comparison["fixed_acceptance"] = fixed_acceptance_comparison(lat, torch)

    # ---------------------------------------------------------------- e2e through host buffers
    e2e = None
    if not args.no_e2e:
        ncanon_u = lat.V * 4 * 18
        ncanon_p = lat.V * 4 * 8
        hu = torch.empty(ncanon_u, dtype=torch.float64, pin_memory=True).numpy()
        # an FP32 chain takes its momenta as FP32 (the precision it holds them
        # in): half the bytes of the FP64 canonical arrays
        pdt = torch.float32 if args.precision == "fp32" else torch.float64
        p_bytes = 4 if args.precision == "fp32" else 8
        hp = torch.empty(ncanon_p, dtype=pdt, pin_memory=True).numpy()
        hu[:] = lat.get_gauge().view(np.float64).ravel()
        rng = inputs.make_rng(seeds["e2e_momenta"])
        hp[:] = rng.standard_normal(ncanon_p)
        hp2 = torch.empty(ncanon_p, dtype=pdt, pin_memory=True).numpy()
        hp2[:] = rng.standard_normal(ncanon_p)
        moms = [hp if k % 2 == 0 else hp2 for k in range(args.steps)]
        # fg_set_momenta takes canonical FP64: the sequential and stateless
        # forms get pinned FP64 copies of the same momenta (no per-step host
        # conversion inside their timed regions)
        if pdt == torch.float64:
            moms64 = moms
        else:
            hp64 = torch.empty(ncanon_p, dtype=torch.float64, pin_memory=True).numpy()
            hp64b = torch.empty(ncanon_p, dtype=torch.float64, pin_memory=True).numpy()
            hp64[:] = hp
            hp64b[:] = hp2
            moms64 = [hp64 if k % 2 == 0 else hp64b for k in range(args.steps)]
        lat.set_gauge(hu)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        # (a) the chain stays on the device (as an HMC user runs it): each
        # trajectory's input, the momenta, comes from pinned host memory (two
        # buffers in turn) and its result (dH, H, accept) goes back; one
        # fg_trajectories_host_momenta call, which uploads the next momenta
        # while the current trajectory runs
        t0 = time.perf_counter()
        lat.trajectories_host_momenta(args.integrator, args.dt, TAU, moms)
        torch.cuda.synchronize()
        e2e_s = reduce_max(time.perf_counter() - t0, world, "cuda")
        # (a') the same with one fg_set_momenta + fg_trajectory pair per
        # trajectory: upload and MD in sequence
        lat.set_gauge(hu)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            lat.set_momenta(moms64[k])
            r = lat.trajectory(args.integrator, args.dt, TAU, refresh=False, u_accept=-1.0)
        torch.cuda.synchronize()
        e2e_seq = reduce_max(time.perf_counter() - t0, world, "cuda")
        # (b) stateless: the whole gauge field goes up and comes back as well
        lat.set_gauge(hu)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            lat.set_gauge(hu)
            lat.set_momenta(moms64[0])
            r = lat.trajectory(args.integrator, args.dt, TAU, refresh=False, u_accept=-1.0)
            lat.get_gauge(out=hu)
        torch.cuda.synchronize()
        e2e_sl = reduce_max(time.perf_counter() - t0, world, "cuda")
        e2e = {"value": whole_job_rate(args.steps, world, e2e_s), "unit": UNIT,
               "h2d_bytes_per_step": ncanon_p * p_bytes,
               "d2h_bytes_per_step": 6 * 8,
               "note": "per trajectory through fg_trajectories_host_momenta(_f32): momenta uploaded from pinned "
                       "host memory (canonical, in the chain's precision: FP32 for an FP32 chain) on a copy "
                       "stream while the previous trajectory runs, trajectory run on the device-resident chain, "
                       "result (dH, H0, H1 sums, accept) read back after each trajectory",
               "sequential": {"value": whole_job_rate(args.steps, world, e2e_seq), "unit": UNIT,
                              "h2d_bytes_per_step": ncanon_p * 8, "d2h_bytes_per_step": 6 * 8,
                              "note": "fg_set_momenta (canonical FP64 from pinned memory) then fg_trajectory "
                                      "per trajectory: upload, conversion and MD in sequence"},
               "stateless": {"value": whole_job_rate(args.steps, world, e2e_sl), "unit": UNIT,
                             "h2d_bytes_per_step": (ncanon_u + ncanon_p) * 8,
                             "d2h_bytes_per_step": ncanon_u * 8 + 6 * 8,
                             "note": "the gauge field (canonical FP64) also uploaded and read back every "
                                     "trajectory"}}

    ferm = None
    if not args.no_fermion:
        ferm = fermion_measurement(fg, stream.cuda_stream, rank, hbm_peak(),
                                   tuple(int(x) for x in args.fermion_dims.split(",")))
    precision = None
    if not args.no_compare:
        precision = precision_measurement(fg, stream.cuda_stream, rank)
    batched = None
    if not args.no_batch:
        batched = batched_measurement(fg, stream.cuda_stream, rank)
    served = None
    if not args.no_serve:
        served = serving_measurement()
        # the same stream at a rate the GPU sustains (80% of the capacity just measured)
        stable = 0.8 * served["trajectories_per_s"]
        served["at_sustainable_rate"] = serving_measurement(rate_hz=stable)

    if rank == 0:
        cfg = workload_config(args)
        cfg.update({"acceptance": acc, "mean_exp_minus_dH": emdh,
                    "dH": [round(r["dH"], 6) for r in results[:8]],
                    "forces_per_trajectory": n_force, "md_steps": nsteps,
                    "plaquette": lat.plaquette(), "dH_precision_check": headline_dh})
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
                "config": cfg, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "fermion": ferm,
                "batched_chains": batched, "serving": served, "integrator_comparison": comparison,
                "precision_comparison": precision,
                "gpu_launches": launches, "clocks": clk}
        print(json.dumps(line), flush=True)
    lat.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
