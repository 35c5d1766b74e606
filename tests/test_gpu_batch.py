"""Batches of independent chains (fg_batch) against the oracle and against
single-lattice handles ("same alone and in the mix")."""

import numpy as np
import pytest

from oracle import integrators as it
from paper_0910_2950_gb300 import inputs

pytestmark = pytest.mark.gpu

CHAINS = [((4, 4, 4, 4), 6.0), ((2, 4, 2, 6), 5.7), ((6, 4, 2, 4), 6.2), ((4, 2, 4, 2), 5.9)]


@pytest.fixture(scope="module")
def fgmod():
    from paper_0910_2950_gb300 import build, fg
    build.build()
    fg.load()
    return fg


def _inputs(k, dims):
    return inputs.hot_start(dims, 40 + k), inputs.gaussian_momenta(dims, 60 + k)


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("integ", ["fg", "omelyan", "qpq"])
def test_batch_fp64_matches_oracle(fgmod, integ):
    dims_list = [d for d, _ in CHAINS]
    betas = [b for _, b in CHAINS]
    with fgmod.Batch(dims_list, betas, precision="fp64", tile=32) as bat:
        for k, dims in enumerate(dims_list):
            u, p = _inputs(k, dims)
            bat.set_gauge(k, u)
            bat.set_momenta(k, p)
        res = bat.trajectory(integ, 0.125, 1.0, refresh=False, always_accept=True)
        for k, (dims, beta) in enumerate(CHAINS):
            u, p = _inputs(k, dims)
            u1, p1, h0, h1 = it.trajectory(it.GaugeSystem(beta), it.Integrator(integ), u, p, 0.125, 1.0)
            assert res[k]["accepted"] == 1
            assert abs(res[k]["dH"] - (h1 - h0)) <= min(1e-6, 1e-12 * abs(h0)), (k, res[k]["dH"], h1 - h0)
            assert _rel(bat.get_gauge(k), u1) < 1e-12
            assert _rel(bat.get_momenta(k), p1) < 1e-11


# FP32 12-real runs the kernel that shares the upper-staple products through
# shared memory, in every tile shape
@pytest.mark.parametrize("precision,link_reals,tile", [("fp32", 18, 0), ("fp64", 18, 0), ("fp32", 12, 16),
                                                       ("fp32", 12, 32), ("fp32", 12, 64)])
def test_same_alone_and_in_the_mix(fgmod, precision, link_reals, tile):
    dims_list = [d for d, _ in CHAINS]
    betas = [b for _, b in CHAINS]
    with fgmod.Batch(dims_list, betas, precision=precision, link_reals=link_reals, tile=tile) as bat:
        for k, dims in enumerate(dims_list):
            u, p = _inputs(k, dims)
            bat.set_gauge(k, u)
            bat.set_momenta(k, p)
        res = bat.trajectory("fg", 0.25, 1.0, refresh=False, always_accept=True)
        assert bat.tile() in (16, 32, 64)
        mixed = [bat.get_gauge(k) for k in range(len(CHAINS))]
    for k, (dims, beta) in enumerate(CHAINS):
        u, p = _inputs(k, dims)
        with fgmod.Lattice(dims, beta, precision=precision, link_reals=link_reals) as lat:
            lat.set_gauge(u)
            lat.set_momenta(p)
            r = lat.trajectory("fg", 0.25, 1.0, refresh=False, u_accept=0.0)
            alone = lat.get_gauge()
        # identical per-link arithmetic: the links agree bit for bit
        assert np.array_equal(mixed[k], alone), k
        # dH sums the same sites in another order
        assert abs(res[k]["dH"] - r["dH"]) <= 1e-9 * abs(r["H0"])


def test_graphs_tiles_and_metropolis(fgmod):
    dims_list = [(4, 4, 4, 4), (6, 6, 6, 6), (8, 4, 4, 4), (4, 4, 2, 2), (6, 4, 4, 8)]
    betas = [5.7, 5.8, 6.0, 6.1, 6.2]
    starts = [inputs.hot_start(d, 90 + k) for k, d in enumerate(dims_list)]
    outs = {}
    for tile, graphs in [(16, False), (32, True), (64, True)]:
        with fgmod.Batch(dims_list, betas, precision="fp32", tile=tile, use_graphs=graphs, seed=5) as bat:
            for k in range(len(dims_list)):
                bat.set_gauge(k, starts[k])
            res = []
            for _ in range(3):
                res.append(bat.trajectory("fg", 0.125, 1.0, refresh=True, always_accept=False))
            outs[(tile, graphs)] = ([bat.get_gauge(k) for k in range(len(dims_list))], res)
            n0 = bat.launch_count()
            bat.trajectory("fg", 0.125, 1.0)
            # one launch per MD sub-step for all chains, plus refresh/energy/accept bookkeeping
            assert bat.launch_count() - n0 < 40
    ref_links, ref_res = outs[(16, False)]
    for key, (links, res) in outs.items():
        for k in range(len(dims_list)):
            assert np.array_equal(links[k], ref_links[k]), (key, k)
        for a, b in zip(res, ref_res):
            for ra, rb in zip(a, b):
                assert ra["accepted"] == rb["accepted"]
                assert abs(ra["dH"] - rb["dH"]) < 1e-6 * max(1.0, abs(rb["H0"]) * 1e-6)


def test_rejected_chains_are_restored(fgmod):
    """Run forward (always accepted) from hot starts, then back with reversed
    momenta: by reversibility dH is minus the first one, large and positive
    for the chains that lost energy, so Metropolis rejects them and their
    links must be restored bit for bit."""
    dims_list = [(4, 4, 4, 4)] * 4
    with fgmod.Batch(dims_list, [6.0] * 4, precision="fp64", tile=32, seed=3) as bat:
        starts = [inputs.hot_start(d, 7 + k) for k, d in enumerate(dims_list)]
        for k in range(4):
            bat.set_gauge(k, starts[k])
            bat.set_momenta(k, inputs.gaussian_momenta(dims_list[k], 17 + k))
        fwd = bat.trajectory("leapfrog", 0.25, 1.0, refresh=False, always_accept=True)
        mids = [bat.get_gauge(k) for k in range(4)]
        for k in range(4):
            bat.set_momenta(k, -bat.get_momenta(k))
        back = bat.trajectory("leapfrog", 0.25, 1.0, refresh=False, always_accept=False)
        for k in range(4):
            assert abs(back[k]["dH"] + fwd[k]["dH"]) < 1e-8 * abs(fwd[k]["H0"])
            after = bat.get_gauge(k)
            if back[k]["accepted"]:
                assert np.max(np.abs(after - starts[k])) < 1e-10
            else:
                assert np.array_equal(after, mids[k])
        assert sum(1 for r in back if not r["accepted"]) >= 1
