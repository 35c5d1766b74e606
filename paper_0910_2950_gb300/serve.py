"""Continuous-batching HMC trajectory server.

Requests ask for one trajectory of a chain (lattice extents, beta, kappa for
Nf = 2 Wilson fermions or 0 for pure gauge, integrator, dt, tau).  Chains
stay resident on the device between requests; a chain's first request
starts it from a Haar-random (hot) gauge field drawn on the device.

Scheduling: requests are admitted in arrival order as soon as (a) a slot is
free, (b) no earlier request of the same chain is still running and (c) the
chain's device footprint fits the HBM budget - a new chain is created only
when the resident chains plus it stay within the budget, evicting idle
chains (least recently used; their links are kept on the host and restored
on their next request) if needed.  Each admitted request runs on its own
slot thread and its chain's own CUDA stream, so requests that arrive while
others are on the GPU overlap with them on the device.

Determinism: before each trajectory the chain's random streams are set to
the chain's trajectory index (fg_set_rng_position), so a chain gives the same
result whatever ran before, beside or between its requests, and whether or
not it was evicted: alone and in the mix.

The server does no lattice arithmetic itself; every step runs in the CUDA
library through ``paper_0910_2950_gb300.fg``.
"""

from __future__ import annotations

import collections
import concurrent.futures as cf
import threading
import time
from dataclasses import dataclass

import numpy as np

from . import fg as _fg

INTEGRATOR_NAMES = ("leapfrog", "omelyan", "fg", "campostrini", "qpq")


@dataclass(frozen=True)
class ChainSpec:
    """What defines a chain: its lattice and action (fixed for its lifetime)."""
    dims: tuple
    beta: float
    kappa: float = 0.0
    seed: int = 1


@dataclass
class Request:
    rid: int
    chain: int
    spec: ChainSpec
    integrator: str = "fg"
    dt: float = 0.125
    tau: float = 1.0
    arrival: float = 0.0          # seconds after the start of the stream
    # Optional inputs supplied by the client (host arrays in the library's
    # canonical layouts): `links` replace the chain's links before the
    # trajectory; `momenta` replace the device momentum refresh, and then
    # `chi` (Nf = 2 chains) sets the pseudofermion heat bath (without it the
    # chain keeps its current pseudofermion); `u_accept` in [0, 1) is the
    # Metropolis uniform, < 0 the chain's own random stream.
    links: object = None
    momenta: object = None
    chi: object = None
    u_accept: float = -1.0


@dataclass
class Result:
    rid: int
    chain: int
    traj_index: int
    dH: float
    accepted: int
    plaquette: float
    n_force: int
    n_solves: int
    cg_iters: int
    arrival: float
    start: float
    end: float

    @property
    def latency(self):
        return self.end - self.arrival


def footprint_bytes(spec: ChainSpec, precision: str = "fp32", link_reals: int = 18,
                    l2_bytes: int = 126 << 20) -> int:
    """Device bytes a chain holds, from the library's allocation plan: three
    link buffers, momenta and force, per-site energies and the stored per-site
    gauge actions, block partials and
    result scalars, the FP64 host-layout staging buffer, and for fermions 8
    FP64 and 10 working half-lattice spinors (plus 2 double-float ones for the
    FP32 solver's reliable updates, and the second r and p buffers of the
    folded CG iteration, which the library runs while the solver's links
    and six vectors fit in L2 and never with 16-bit inner vectors), the
    pseudofermion force, the CG scalars and the Dslash (three values) and
    vector block partials (two arrays of the latter).  4 KiB are added for allocator
    rounding of the small buffers.  (The closed-form force gradient's
    buffers are not included: the server does not offer that integrator.)
    `l2_bytes` is the GPU's L2 size, which decides FG_FP32_AUTOCG's inner
    precision and the CG iteration form."""
    v = int(np.prod(spec.dims))
    r = 8 if precision in ("fp64", "df64") else 4     # bytes per real (double-float: two floats)
    gauge = 4 * v * link_reals * r
    mom = 4 * v * 8 * r
    total = 3 * gauge + 2 * mom + 3 * 8 * v + 4 * 8 * ((v + 255) // 256 + 1) + 32 * 8 + 4 * v * 18 * 8
    if spec.kappa > 0:
        vh = v // 2
        nvec = 12 * vh
        n64 = 8 + (2 if precision != "fp64" else 0)
        dslash_blocks = (vh + 127) // 128
        vec_blocks = min((nvec + 255) // 256, 152 * 8)
        half = precision in ("fp32_fp16cg", "fp32_bf16cg") or (
            precision == "fp32_autocg" and v * (4 * (link_reals // 2) * 8 + 6 * 48) > l2_bytes)
        # the fold buffers are left out only well beyond L2, so that the
        # estimate stays an upper bound whatever L2 size the library sees
        folded = not half and v * (4 * (link_reals // 2) * 2 + 6 * 12) * r <= 1.25 * l2_bytes
        n_inner = 12 if folded else 10
        total += n64 * nvec * 16 + n_inner * nvec * 2 * r + mom + 128 + 8 * (3 * dslash_blocks + 2 * vec_blocks + 3)
        if half:
            total += 4 * v * link_reals * 2      # 16-bit links of the inner solver
    return total + 4096


class _Chain:
    def __init__(self, spec):
        self.spec = spec
        self.lat = None            # resident handle, or None
        self.host_links = None     # links kept on the host while evicted
        self.busy = False
        self.traj_index = 0
        self.last_used = 0.0
        self.bytes = 0


class TrajectoryServer:
    """Continuous-batching server over resident chains (see the module doc)."""

    def __init__(self, slots: int = 4, hbm_budget_bytes: int = 8 << 30, precision: str = "fp32",
                 cg_tol: float = 1e-10, clock=time.perf_counter, lattice_factory=None, cg_tol_action: float = 1e-12):
        if slots < 1:
            raise ValueError("slots must be >= 1")
        self.slots = slots
        self.budget = int(hbm_budget_bytes)
        self.precision = precision
        self.cg_tol = cg_tol
        self.cg_tol_action = cg_tol_action
        self.clock = clock
        self.lattice_factory = lattice_factory or (
            lambda spec: _fg.Lattice(spec.dims, spec.beta, kappa=spec.kappa, precision=self.precision,
                                     cg_tol=self.cg_tol, cg_tol_action=self.cg_tol_action, seed=spec.seed))
        self.chains = {}
        self.resident_bytes = 0
        self.evictions = 0
        self.peak_resident_bytes = 0
        self._lock = threading.Lock()
        self._pool = cf.ThreadPoolExecutor(max_workers=slots)

    # -- chain residency ------------------------------------------------
    def _make_resident(self, ch: _Chain):
        lat = self.lattice_factory(ch.spec)
        if ch.host_links is None:
            lat.random_gauge()
        else:
            lat.set_gauge(ch.host_links)
            ch.host_links = None
        ch.lat = lat

    def _evict(self, ch: _Chain):
        ch.host_links = ch.lat.get_gauge()
        ch.lat.close()
        ch.lat = None
        self.resident_bytes -= ch.bytes
        ch.bytes = 0
        self.evictions += 1

    def _admit(self, req: Request) -> bool:
        """Reserve the chain for req if it can run now (called under the lock)."""
        ch = self.chains.get(req.chain)
        if ch is None:
            ch = self.chains[req.chain] = _Chain(req.spec)
        elif ch.spec != req.spec:
            raise ValueError(f"chain {req.chain} was created with another lattice or action")
        if ch.busy:
            return False
        if ch.lat is None and ch.bytes == 0:
            need = footprint_bytes(req.spec, self.precision)
            if need > self.budget:
                raise ValueError(f"chain {req.chain} alone exceeds the HBM budget")
            if self.resident_bytes + need > self.budget:
                idle = sorted((c for c in self.chains.values() if c.lat is not None and not c.busy),
                              key=lambda c: c.last_used)
                for c in idle:
                    if self.resident_bytes + need <= self.budget:
                        break
                    self._evict(c)
                if self.resident_bytes + need > self.budget:
                    return False
            ch.bytes = need
            self.resident_bytes += need
            self.peak_resident_bytes = max(self.peak_resident_bytes, self.resident_bytes)
        ch.busy = True
        return True

    # -- one request ----------------------------------------------------
    def _run(self, req: Request, t0: float) -> Result:
        ch = self.chains[req.chain]
        start = self.clock() - t0
        if ch.lat is None:
            self._make_resident(ch)
        lat = ch.lat
        k = ch.traj_index
        lat.set_rng_position(k)
        if req.links is not None:
            lat.set_gauge(req.links)
        refresh = req.momenta is None
        if not refresh:
            lat.set_momenta(req.momenta)
            if req.chi is not None:
                lat.set_pseudofermion(req.chi)
        r = lat.trajectory(req.integrator, req.dt, req.tau, refresh=refresh, u_accept=req.u_accept)
        plaq = lat.plaquette()
        end = self.clock() - t0
        with self._lock:
            ch.traj_index += 1
            ch.busy = False
            ch.last_used = end
        return Result(req.rid, req.chain, k, r["dH"], r["accepted"], plaq, r["n_force"], r["n_solves"],
                      r["cg_iters"], req.arrival, start, end)

    # -- a stream of requests ---------------------------------------------
    def serve(self, requests, realtime: bool = True):
        """Process requests (sorted by arrival time).  With realtime, a request
        is not admitted before its arrival time; otherwise all are queued at
        once.  Returns (results in request order, wall seconds, busy seconds)."""
        reqs = sorted(requests, key=lambda r: (r.arrival, r.rid))
        pending = collections.deque()
        running = {}
        results = {}
        i = 0
        t0 = self.clock()
        busy_since, busy = None, 0.0
        while i < len(reqs) or pending or running:
            now = self.clock() - t0
            while i < len(reqs) and (not realtime or reqs[i].arrival <= now):
                pending.append(reqs[i])
                i += 1
            # admit in arrival order; a request blocked by its chain or by memory
            # does not hold back the ones behind it (continuous batching)
            with self._lock:
                kept = collections.deque()
                held = set()          # chains with an earlier request still waiting
                while pending:
                    req = pending.popleft()
                    if req.chain not in held and len(running) < self.slots and self._admit(req):
                        running[self._pool.submit(self._run, req, t0)] = req
                    else:
                        held.add(req.chain)
                        kept.append(req)
                pending = kept
            if running and busy_since is None:
                busy_since = self.clock() - t0
            if not running and busy_since is not None:
                busy += (self.clock() - t0) - busy_since
                busy_since = None
            if not running and not pending and i < len(reqs) and realtime:
                time.sleep(max(0.0, reqs[i].arrival - (self.clock() - t0)))
                continue
            timeout = None
            if i < len(reqs) and realtime:
                timeout = max(0.0, reqs[i].arrival - (self.clock() - t0))
            if running:
                done, _ = cf.wait(list(running), timeout=timeout, return_when=cf.FIRST_COMPLETED)
                for f in done:
                    req = running.pop(f)
                    results[req.rid] = f.result()
        wall = self.clock() - t0
        if busy_since is not None:
            busy += wall - busy_since
        return [results[r.rid] for r in sorted(requests, key=lambda r: r.rid)], wall, busy

    def final_links(self, chain: int):
        ch = self.chains[chain]
        return ch.lat.get_gauge() if ch.lat is not None else ch.host_links

    def close(self):
        self._pool.shutdown(wait=True)
        for ch in self.chains.values():
            if ch.lat is not None:
                ch.lat.close()
                ch.lat = None


def poisson_stream(rate_hz: float, duration_s: float, chains, seed: int = 5, integrators=("omelyan", "fg"),
                   dts=(1 / 8, 1 / 12)):
    """Poisson arrivals at rate_hz for duration_s over the given chain specs
    (dict id -> ChainSpec); each request picks a chain, an integrator and a
    step size uniformly."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t, out, rid = 0.0, [], 0
    ids = sorted(chains)
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        c = ids[int(rng.integers(len(ids)))]
        out.append(Request(rid, c, chains[c], integrators[int(rng.integers(len(integrators)))],
                           float(dts[int(rng.integers(len(dts)))]), 1.0, t))
        rid += 1
    return out


def served_chain_mix(n_chains: int = 32, seed: int = 5):
    """Chains of the served workload: 70% pure gauge at 8^4, 12^4, 16^4 or 24^4
    with beta in [5.7, 6.2]; 30% Nf=2 Wilson at 8^3x16 or 12^3x24 with kappa in
    [0.155, 0.159] (beta 5.6)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    chains = {}
    for c in range(n_chains):
        if rng.random() < 0.7:
            L = int(rng.choice([8, 12, 16, 24]))
            chains[c] = ChainSpec((L, L, L, L), float(rng.uniform(5.7, 6.2)), 0.0, 100 + c)
        else:
            d = [(8, 8, 8, 16), (12, 12, 12, 24)][int(rng.integers(2))]
            chains[c] = ChainSpec(d, 5.6, float(rng.uniform(0.155, 0.159)), 100 + c)
    return chains
