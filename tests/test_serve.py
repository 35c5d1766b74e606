"""Scheduler logic of the trajectory server, on CPU with a stand-in lattice.

The stand-in records when each chain runs and returns a result that depends
only on (chain, trajectory index), like the real library with its random
streams set to the trajectory index; the GPU version of the same checks is
in test_gpu_serve.py.
"""

import threading
import time

import numpy as np
import pytest

from paper_0910_2950_gb300 import serve


class FakeLattice:
    live = 0
    max_live = 0
    running = 0
    max_running = 0
    lock = threading.Lock()
    log = []

    def __init__(self, spec):
        self.spec = spec
        self.links = None
        self.pos = None
        with FakeLattice.lock:
            FakeLattice.live += 1
            FakeLattice.max_live = max(FakeLattice.max_live, FakeLattice.live)

    def random_gauge(self):
        self.links = np.full(4, float(self.spec.seed))

    def set_gauge(self, u):
        self.links = np.array(u)

    def get_gauge(self):
        return self.links.copy()

    def set_rng_position(self, k):
        self.pos = k

    def trajectory(self, integ, dt, tau, refresh=True, u_accept=-1.0):
        with FakeLattice.lock:
            FakeLattice.running += 1
            FakeLattice.max_running = max(FakeLattice.max_running, FakeLattice.running)
            FakeLattice.log.append((self.spec.seed, self.pos))
        time.sleep(0.002)
        self.links = self.links * 1.0001 + self.pos
        with FakeLattice.lock:
            FakeLattice.running -= 1
        return {"dH": float(self.spec.seed * 1000 + self.pos), "accepted": 1, "n_force": 13, "n_solves": 0,
                "cg_iters": 0}

    def plaquette(self):
        return float(self.links.sum())

    def close(self):
        with FakeLattice.lock:
            FakeLattice.live -= 1


def _reset():
    FakeLattice.live = FakeLattice.max_live = FakeLattice.running = FakeLattice.max_running = 0
    FakeLattice.log = []


def _chains(n=6):
    return {c: serve.ChainSpec((4, 4, 4, 4) if c % 2 else (8, 8, 8, 8), 6.0, 0.0, 100 + c) for c in range(n)}


def _requests(chains, n=60, seed=1):
    rng = np.random.default_rng(seed)
    return [serve.Request(i, c, chains[c]) for i, c in enumerate(rng.integers(len(chains), size=n).tolist())]


def test_results_are_the_same_alone_and_in_the_mix():
    chains = _chains()
    reqs = _requests(chains)
    _reset()
    s1 = serve.TrajectoryServer(slots=1, lattice_factory=FakeLattice)
    seq, _, _ = s1.serve(reqs, realtime=False)
    links1 = {c: s1.final_links(c) for c in chains if c in s1.chains}
    s1.close()
    _reset()
    s4 = serve.TrajectoryServer(slots=4, lattice_factory=FakeLattice)
    mix, _, _ = s4.serve(reqs, realtime=False)
    links4 = {c: s4.final_links(c) for c in chains if c in s4.chains}
    s4.close()
    assert FakeLattice.max_running > 1            # requests really overlapped
    assert [(r.chain, r.traj_index, r.dH) for r in seq] == [(r.chain, r.traj_index, r.dH) for r in mix]
    for c in links1:
        assert np.array_equal(links1[c], links4[c])


def test_chain_order_slots_and_budget_with_eviction():
    chains = _chains()
    reqs = _requests(chains, n=80, seed=2)
    big = serve.footprint_bytes(chains[0])
    small = serve.footprint_bytes(chains[1])
    budget = big + 2 * small                    # fewer than all chains fit at once
    _reset()
    srv = serve.TrajectoryServer(slots=3, hbm_budget_bytes=budget, lattice_factory=FakeLattice)
    res, _, _ = srv.serve(reqs, realtime=False)
    assert srv.evictions > 0
    assert srv.peak_resident_bytes <= budget
    assert FakeLattice.max_running <= 3
    # per chain, trajectories run in request order with consecutive indices
    seen = {}
    for r in sorted(res, key=lambda r: r.rid):
        assert r.traj_index == seen.get(r.chain, 0)
        seen[r.chain] = r.traj_index + 1
    # the results equal an unconstrained sequential run: eviction keeps the state
    _reset()
    ref = serve.TrajectoryServer(slots=1, lattice_factory=FakeLattice)
    res1, _, _ = ref.serve(reqs, realtime=False)
    assert [r.dH for r in res] == [r.dH for r in res1]
    for c in chains:
        if c in ref.chains:
            assert np.array_equal(srv.final_links(c), ref.final_links(c))
    srv.close()
    ref.close()


def test_realtime_arrivals_and_latency_bookkeeping():
    chains = _chains(3)
    reqs = serve.poisson_stream(400.0, 0.1, chains, seed=3)
    assert len(reqs) > 10
    assert all(a.arrival <= b.arrival for a, b in zip(reqs, reqs[1:]))
    _reset()
    srv = serve.TrajectoryServer(slots=2, lattice_factory=FakeLattice)
    res, wall, busy = srv.serve(reqs, realtime=True)
    srv.close()
    for r in res:
        assert r.start >= r.arrival - 1e-9 and r.end >= r.start and r.latency > 0
    assert 0 < busy <= wall + 1e-9


def test_chain_that_cannot_fit_is_refused():
    spec = serve.ChainSpec((24, 24, 24, 24), 6.0)
    srv = serve.TrajectoryServer(slots=1, hbm_budget_bytes=1 << 20, lattice_factory=FakeLattice)
    with pytest.raises(ValueError):
        srv.serve([serve.Request(0, 0, spec)], realtime=False)
    srv.close()


def test_served_mix_matches_the_workload():
    chains = serve.served_chain_mix(200, seed=5)
    nf2 = [c for c in chains.values() if c.kappa > 0]
    assert 0.2 < len(nf2) / len(chains) < 0.4
    assert all(0.155 <= c.kappa <= 0.159 and c.dims in [(8, 8, 8, 16), (12, 12, 12, 24)] for c in nf2)
    pg = [c for c in chains.values() if c.kappa == 0]
    assert all(5.7 <= c.beta <= 6.2 and c.dims[0] in (8, 12, 16, 24) for c in pg)


def test_footprint_follows_the_cg_iteration_form():
    """The folded CG iteration's second r and p buffers are counted while
    the solver's links and six half-lattice vectors fit in L2 (with a margin,
    so the estimate stays an upper bound), and never for 16-bit inner
    vectors: beyond L2 the estimate drops exactly those two vectors."""
    spec = serve.ChainSpec((24, 24, 24, 48), 5.6, 0.158, 1)
    nvec = 12 * int(np.prod(spec.dims)) // 2           # complex entries of one even-site vector
    for precision, r in (("fp32", 4), ("fp64", 8)):
        in_l2 = serve.footprint_bytes(spec, precision, l2_bytes=1 << 40)
        beyond = serve.footprint_bytes(spec, precision, l2_bytes=1 << 20)
        assert in_l2 - beyond == 2 * nvec * 2 * r
    for precision in ("fp32_fp16cg", "fp32_bf16cg"):
        assert serve.footprint_bytes(spec, precision, l2_bytes=1 << 40) == \
            serve.footprint_bytes(spec, precision, l2_bytes=1 << 20)
    # pure gauge chains have no solver
    pg = serve.ChainSpec((16, 16, 16, 16), 6.0, 0.0, 2)
    assert serve.footprint_bytes(pg, "fp32", l2_bytes=1 << 40) == serve.footprint_bytes(pg, "fp32", l2_bytes=1 << 20)
