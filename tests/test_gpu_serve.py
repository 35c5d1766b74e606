"""Trajectory server on the GPU: each result is the same alone and in the mix.

The same requests run (a) one at a time, (b) four at a time overlapping on
the device, and (c) three at a time under an HBM budget that forces chains
to be evicted to the host and restored.  Every request's dH and acceptance
and every chain's final links agree bit for bit: a chain's computation runs
on its own stream with its random streams set to its trajectory index.
"""

import numpy as np
import pytest

from paper_0910_2950_gb300 import serve

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
        assert a.dH == b.dH == c.dH
        assert a.accepted == b.accepted == c.accepted
        assert np.isfinite(a.dH)
    for k in l1:
        assert np.array_equal(l1[k], l4[k]) and np.array_equal(l1[k], l3[k])
    # fermion requests did CG solves; pure-gauge ones did not
    assert all((r.n_solves > 0) == (r.chain == 3) for r in seq)


@pytest.mark.parametrize("spec", [serve.ChainSpec((8, 8, 8, 8), 6.0, 0.0, 1),
                                  serve.ChainSpec((8, 8, 8, 16), 5.6, 0.157, 2),
                                  serve.ChainSpec((6, 6, 6, 12), 5.6, 0.155, 3)])
@pytest.mark.parametrize("precision", ["fp32", "fp32_fp16cg", "fp64"])
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
