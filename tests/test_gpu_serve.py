"""Trajectory server on the GPU: each result is the same alone and in the mix,
and the served trajectories agree with the oracle on client-supplied inputs.

The same requests run (a) one at a time, (b) four at a time overlapping on
the device, and (c) three at a time under an HBM budget that forces chains
to be evicted to the host and restored.  A chain's computation runs on its
own stream with its random streams set to its trajectory index, so every
pure-gauge request's dH and acceptance and every pure-gauge chain's final
links agree bit for bit.  The FP32 solver of an Nf=2 chain places its
reliable updates where the host's extrapolation of the residual (read as
the GPU runs ahead) says, so its results agree within the solver's
tolerance: dH within 1e-3, the FP32 path's bar against FP64.
"""

import numpy as np
import pytest

from oracle import fermion as fe, integrators as it
from paper_0910_2950_gb300 import inputs, serve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fgmod():
    from paper_0910_2950_gb300 import build, fg
    build.build()
    fg.load()
    return fg


def _workload():
    chains = {
        0: serve.ChainSpec((4, 4, 4, 4), 6.0, 0.0, 11),
        1: serve.ChainSpec((6, 6, 6, 6), 5.8, 0.0, 12),
        2: serve.ChainSpec((4, 4, 2, 6), 6.1, 0.0, 13),
        3: serve.ChainSpec((4, 4, 4, 8), 5.6, 0.13, 14),
    }
    rng = np.random.default_rng(7)
    reqs = []
    for i in range(24):
        c = int(rng.integers(4))
        reqs.append(serve.Request(i, c, chains[c], ["omelyan", "fg"][int(rng.integers(2))],
                                  [1 / 8, 1 / 12][int(rng.integers(2))]))
    return chains, reqs


def _run(slots, budget):
    chains, reqs = _workload()
    srv = serve.TrajectoryServer(slots=slots, hbm_budget_bytes=budget)
    res, wall, busy = srv.serve(reqs, realtime=False)
    links = {c: srv.final_links(c) for c in chains}
    ev = srv.evictions
    srv.close()
    return res, links, ev


def test_alone_and_in_the_mix_gpu(fgmod):
    seq, l1, _ = _run(1, 8 << 30)
    mix, l4, _ = _run(4, 8 << 30)
    chains, _ = _workload()
    tight = serve.footprint_bytes(chains[1]) + serve.footprint_bytes(chains[3]) + 4096
    ev_res, l3, ev = _run(3, tight)
    assert ev > 0
    for a, b, c in zip(seq, mix, ev_res):
        assert (a.chain, a.traj_index) == (b.chain, b.traj_index) == (c.chain, c.traj_index)
        if chains[a.chain].kappa > 0:
            assert abs(a.dH - b.dH) <= 1e-3 and abs(a.dH - c.dH) <= 1e-3, (a.dH, b.dH, c.dH)
        else:
            assert a.dH == b.dH == c.dH
        assert a.accepted == b.accepted == c.accepted
        assert np.isfinite(a.dH)
    for k in l1:
        if chains[k].kappa > 0:
            assert np.max(np.abs(l1[k] - l4[k])) < 1e-3 and np.max(np.abs(l1[k] - l3[k])) < 1e-3
        else:
            assert np.array_equal(l1[k], l4[k]) and np.array_equal(l1[k], l3[k])
    # fermion requests did CG solves; pure-gauge ones did not
    assert all((r.n_solves > 0) == (r.chain == 3) for r in seq)


ORACLE_CHAINS = {
    0: serve.ChainSpec((4, 4, 4, 4), 6.0, 0.0, 21),
    1: serve.ChainSpec((4, 4, 2, 6), 5.8, 0.0, 22),
    2: serve.ChainSpec((4, 4, 2, 4), 5.6, 0.13, 23),
}


def _oracle_workload():
    """Requests with client-supplied inputs: each chain's first request brings
    its start links, every request its momenta (and chi for the Nf = 2
    chain); the Metropolis uniform 0 accepts every finite dH."""
    rng = np.random.default_rng(9)
    reqs, first = [], set()
    for i in range(12):
        c = int(rng.integers(3))
        spec = ORACLE_CHAINS[c]
        links = inputs.hot_start(spec.dims, spec.seed) if c not in first else None
        first.add(c)
        chi = inputs.gaussian_spinor_even(spec.dims, 300 + i) if spec.kappa > 0 else None
        reqs.append(serve.Request(i, c, spec, ["omelyan", "fg", "leapfrog"][int(rng.integers(3))],
                                  [1 / 4, 1 / 8][int(rng.integers(2))], links=links,
                                  momenta=inputs.gaussian_momenta(spec.dims, 200 + i), chi=chi, u_accept=0.0))
    return reqs


def _oracle_results(reqs):
    """The oracle's trajectories, each chain's requests in order."""
    links, out = {}, {}
    for r in sorted(reqs, key=lambda r: r.rid):
        spec = r.spec
        u = r.links if r.links is not None else links[r.chain]
        if spec.kappa > 0:
            phi = fe.heatbath_phi(u, spec.kappa, inputs.unpack_even(r.chi, spec.dims))
            system = fe.FermionSystem(spec.beta, spec.kappa, phi, tol=1e-13)
        else:
            system = it.GaugeSystem(spec.beta)
        u1, _, h0, h1 = it.trajectory(system, it.Integrator(r.integrator), u, r.momenta, r.dt, r.tau)
        out[r.rid] = (h1 - h0, h0)
        links[r.chain] = u1
    return out, links


def test_served_results_match_the_oracle(fgmod):
    """Served requests (FP64) against the oracle on the same inputs, one slot
    at a time and four at a time, and under a budget that evicts chains to
    the host: every dH within the FP64 tolerances (1e-12 |H| for pure gauge,
    1e-6 absolute) and every chain's final links within 1e-10."""
    reqs = _oracle_workload()
    ref, ref_links = _oracle_results(reqs)
    tight = max(serve.footprint_bytes(s, "fp64") for s in ORACLE_CHAINS.values()) * 2 + 4096
    runs = []
    for slots, budget in ((1, 8 << 30), (4, 8 << 30), (2, tight)):
        srv = serve.TrajectoryServer(slots=slots, hbm_budget_bytes=budget, precision="fp64", cg_tol=1e-13,
                                     cg_tol_action=1e-13)
        res, _, _ = srv.serve(reqs, realtime=False)
        links = {c: srv.final_links(c) for c in ORACLE_CHAINS}
        runs.append((res, links, srv.evictions))
        srv.close()
    assert runs[2][2] > 0
    for res, links, _ in runs:
        for r in res:
            dh_o, h0_o = ref[r.rid]
            tol = 1e-6 if ORACLE_CHAINS[r.chain].kappa > 0 else min(1e-6, 1e-12 * abs(h0_o))
            assert abs(r.dH - dh_o) <= tol, (r.rid, r.chain, r.dH, dh_o)
            assert r.accepted == 1
        for c, u in links.items():
            assert float(np.max(np.abs(u - ref_links[c]))) < 1e-10, c
    # alone and in the mix: the same bits
    for a, b in zip(runs[0][0], runs[1][0]):
        assert a.dH == b.dH
    for c in ORACLE_CHAINS:
        assert np.array_equal(runs[0][1][c], runs[1][1][c])


@pytest.mark.parametrize("spec", [serve.ChainSpec((8, 8, 8, 8), 6.0, 0.0, 1),
                                  serve.ChainSpec((8, 8, 8, 16), 5.6, 0.157, 2),
                                  serve.ChainSpec((6, 6, 6, 12), 5.6, 0.155, 3)])
@pytest.mark.parametrize("precision", ["fp32", "fp32_fp16cg", "fp32_bf16cg", "fp64"])
def test_footprint_bounds_the_library_allocation(fgmod, spec, precision):
    """Admission by HBM footprint is only safe if the estimate is an upper
    bound of what a chain's handle holds after a trajectory (all lazy
    buffers allocated), and it should not waste much of the budget."""
    with fgmod.Lattice(spec.dims, spec.beta, kappa=spec.kappa, precision=precision, seed=spec.seed) as lat:
        lat.random_gauge()
        lat.trajectory("fg", 0.25, 1.0, refresh=True, u_accept=0.0)
        lat.get_gauge()
        held = lat.device_bytes()
    est = serve.footprint_bytes(spec, precision)
    assert held <= est <= 1.15 * held, (held, est)
