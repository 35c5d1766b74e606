"""GPU parity of the double-float path (FG_DF64) against the FP64 oracle.

Double-float fields hold every real as hi + lo of two floats (~48 bits) and
compute on the FP32 pipes.  Tolerances:
* one MD step, forces, actions: normwise relative 1e-12, the bar the FP64
  path meets (double-float rounding is ~2^-47 = 7e-15 per operation);
* a whole trajectory: |dH_gpu - dH_oracle| <= 1e-6 absolute, the tolerance
  a trajectory's dH is held to in the chosen precision (section 5, Fig. 1
  plots dH), on config 1 (4^4) and on every volume of the batched chains
  (4^4 ... 12^4).
"""

import numpy as np
import pytest

from oracle import gauge, integrators as it, su3
from paper_0910_2950_gb300 import inputs

pytestmark = pytest.mark.gpu

BETA = 6.0


@pytest.fixture(scope="module")
def fgmod():
    from paper_0910_2950_gb300 import build, fg
    build.build()
    fg.load()
    return fg


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


DIMS_CASES = [(4, 4, 4, 4), (6, 4, 2, 6), (8, 8, 8, 8)]


@pytest.mark.parametrize("dims", DIMS_CASES)
@pytest.mark.parametrize("link_reals", [18, 12])
def test_roundtrip_force_and_action_df64(fgmod, dims, link_reals):
    u = inputs.hot_start(dims, 5)
    p = inputs.gaussian_momenta(dims, 6)
    with fgmod.Lattice(dims, BETA, precision="df64", link_reals=link_reals) as lat:
        lat.set_gauge(u)
        lat.set_momenta(p)
        back, pback = lat.get_gauge(), lat.get_momenta()
        f = lat.force()
        sg, sf, t = lat.action()
    # storage keeps ~48 significant bits of every real
    assert np.max(np.abs(back - u)) < 2e-14
    assert np.max(np.abs(pback - p) / np.maximum(np.abs(p), 1e-300)) < 1e-14
    assert _rel(f, gauge.gauge_force(u, BETA)) < 1e-12
    assert abs(sg - gauge.wilson_action(u, BETA)) <= 1e-12 * abs(sg)
    assert abs(t - gauge.kinetic(p)) <= 1e-12 * abs(t)
    assert sf == 0.0


@pytest.mark.parametrize("name", ["leapfrog", "omelyan", "fg", "campostrini", "qpq", "fg_analytic"])
@pytest.mark.parametrize("link_reals", [18, 12])
def test_one_md_step_df64(fgmod, name, link_reals):
    dims = (6, 4, 2, 6)
    u = inputs.hot_start(dims, 8)
    p = inputs.gaussian_momenta(dims, 9)
    dt = 0.1
    with fgmod.Lattice(dims, BETA, precision="df64", link_reals=link_reals) as lat:
        lat.set_gauge(u)
        lat.set_momenta(p)
        lat.md_step(name, dt)
        ug, pg = lat.get_gauge(), lat.get_momenta()
    uo, po = it.md_step(it.GaugeSystem(BETA), it.Integrator(name), u, p, dt)
    assert _rel(ug, uo) < 1e-12
    assert _rel(pg, po) < 1e-12


def test_large_step_exponential_df64(fgmod):
    """Drifts with rotation angles up to ~3 (dt = 1 on unit-Gaussian momenta
    scaled by 3) exercise the double-angle steps of the sine and cosine."""
    dims = (4, 4, 2, 2)
    u = inputs.hot_start(dims, 21)
    p = 3.0 * inputs.gaussian_momenta(dims, 22)
    with fgmod.Lattice(dims, BETA, precision="df64") as lat:
        lat.set_gauge(u)
        lat.set_momenta(p)
        lat.md_step("qpq", 1.0)
        ug, pg = lat.get_gauge(), lat.get_momenta()
    uo, po = it.md_step(it.GaugeSystem(BETA), it.Integrator("qpq"), u, p, 1.0)
    assert _rel(ug, uo) < 1e-12
    assert _rel(pg, po) < 1e-12
    # exp(iA) = f0 + f1 A + f2 A^2 rounds at ~2^-48 |A|^2 with |A| up to ~6 here
    assert su3.unitarity_defect(ug) < 1e-12


@pytest.fixture(scope="module")
def config1_oracle():
    """Oracle dH for config 1: 4^4 hot start (seed 1), momenta seed 1, tau = 1."""
    dims = (4, 4, 4, 4)
    u = inputs.hot_start(dims, 1)
    p = inputs.gaussian_momenta(dims, 1)
    out = {}
    for name in ("leapfrog", "omelyan", "fg"):
        for dt in (1 / 4, 1 / 8, 1 / 16, 1 / 32):
            u1, p1, h0, h1 = it.trajectory(it.GaugeSystem(BETA), it.Integrator(name), u, p, dt, 1.0)
            out[(name, dt)] = (h1 - h0, h0, u1, p1)
    return dims, u, p, out


@pytest.mark.parametrize("name", ["leapfrog", "omelyan", "fg"])
@pytest.mark.parametrize("link_reals", [18, 12])
def test_config1_trajectory_dh_df64(fgmod, config1_oracle, name, link_reals):
    dims, u, p, ref = config1_oracle
    dhs = []
    with fgmod.Lattice(dims, BETA, precision="df64", link_reals=link_reals) as lat:
        for dt in (1 / 4, 1 / 8, 1 / 16, 1 / 32):
            lat.set_gauge(u)
            lat.set_momenta(p)
            r = lat.trajectory(name, dt, 1.0, refresh=False, u_accept=0.0)
            dh_o, h0_o, u1_o, p1_o = ref[(name, dt)]
            assert abs(r["H0"] - h0_o) <= 1e-12 * abs(h0_o)
            assert abs(r["dH"] - dh_o) <= 1e-6, (name, dt, r["dH"], dh_o)
            assert _rel(lat.get_gauge(), u1_o) < 1e-11
            assert _rel(lat.get_momenta(), p1_o) < 1e-11
            dhs.append(abs(r["dH"]))
    slope = np.polyfit(np.log([1 / 4, 1 / 8, 1 / 16, 1 / 32]), np.log(dhs), 1)[0]
    assert (3.6 < slope < 4.5) if name == "fg" else (1.7 < slope < 2.3), slope


# the volumes of the batched chains (4^4 ... 12^4), couplings in [5.7, 6.2]
BATCH = [((4, 4, 4, 4), 5.7), ((6, 6, 6, 6), 6.2), ((8, 8, 8, 8), 5.9), ((10, 10, 10, 10), 6.0),
         ((12, 12, 12, 12), 5.8)]


@pytest.fixture(scope="module")
def batch_oracle():
    out = []
    for k, (dims, beta) in enumerate(BATCH):
        u = inputs.hot_start(dims, 200 + k)
        p = inputs.gaussian_momenta(dims, 300 + k)
        u1, p1, h0, h1 = it.trajectory(it.GaugeSystem(beta), it.Integrator("fg"), u, p, 1 / 8, 1.0)
        out.append((u, p, h1 - h0, h0, u1))
    return out


@pytest.mark.parametrize("tile", [16, 32])
def test_batch_df64_dh_matches_oracle(fgmod, batch_oracle, tile):
    dims_list = [d for d, _ in BATCH]
    betas = [b for _, b in BATCH]
    with fgmod.Batch(dims_list, betas, precision="df64", tile=tile) as bat:
        for k, (u, p, _, _, _) in enumerate(batch_oracle):
            bat.set_gauge(k, u)
            bat.set_momenta(k, p)
        res = bat.trajectory("fg", 1 / 8, 1.0, refresh=False, always_accept=True)
        links = [bat.get_gauge(k) for k in range(len(BATCH))]
    for k, (u, p, dh_o, h0_o, u1_o) in enumerate(batch_oracle):
        assert res[k]["accepted"] == 1
        assert abs(res[k]["H0"] - h0_o) <= 1e-12 * abs(h0_o)
        assert abs(res[k]["dH"] - dh_o) <= 1e-6, (BATCH[k], res[k]["dH"], dh_o)
        assert _rel(links[k], u1_o) < 1e-11


def test_batch_df64_same_alone_and_in_the_mix(fgmod, batch_oracle):
    dims_list = [d for d, _ in BATCH[:3]]
    betas = [b for _, b in BATCH[:3]]
    with fgmod.Batch(dims_list, betas, precision="df64", tile=0) as bat:
        for k in range(3):
            u, p = batch_oracle[k][:2]
            bat.set_gauge(k, u)
            bat.set_momenta(k, p)
        res = bat.trajectory("fg", 0.25, 1.0, refresh=False, always_accept=True)
        assert bat.tile() in (16, 32)
        mixed = [bat.get_gauge(k) for k in range(3)]
    for k, (dims, beta) in enumerate(BATCH[:3]):
        u, p = batch_oracle[k][:2]
        with fgmod.Lattice(dims, beta, precision="df64") as lat:
            lat.set_gauge(u)
            lat.set_momenta(p)
            r = lat.trajectory("fg", 0.25, 1.0, refresh=False, u_accept=0.0)
            alone = lat.get_gauge()
        assert np.array_equal(mixed[k], alone), k
        assert abs(res[k]["dH"] - r["dH"]) <= 1e-9


def test_single_lattice_df64_12x4_matches_oracle(fgmod, batch_oracle):
    dims, beta = BATCH[4]
    u, p, dh_o, h0_o, u1_o = batch_oracle[4]
    with fgmod.Lattice(dims, beta, precision="df64") as lat:
        lat.set_gauge(u)
        lat.set_momenta(p)
        r = lat.trajectory("fg", 1 / 8, 1.0, refresh=False, u_accept=0.0)
        ug = lat.get_gauge()
    assert abs(r["dH"] - dh_o) <= 1e-6, (r["dH"], dh_o)
    assert _rel(ug, u1_o) < 1e-11


def test_df64_device_draws(fgmod):
    """Momentum refresh and hot start on the device for double-float fields:
    Gaussian statistics, and Haar links special unitary to double-float
    rounding."""
    dims = (8, 8, 8, 8)
    with fgmod.Lattice(dims, BETA, precision="df64", seed=77) as lat:
        lat.refresh_momenta()
        p = lat.get_momenta()
        lat.random_gauge()
        ug = lat.get_gauge()
    v = inputs.volume(dims)
    assert abs(p.mean()) < 5 / np.sqrt(p.size)
    assert abs(p.var() - 1) < 5 * np.sqrt(2 / p.size)
    assert abs(0.5 * np.sum(p * p) / (16 * v) - 1) < 5 * np.sqrt(2 / p.size)
    # Gram-Schmidt of Gaussian rows in double-float: ~2e-13 at worst over 2^16 links
    assert su3.unitarity_defect(ug) < 1e-12
    assert np.max(np.abs(np.linalg.det(ug) - 1)) < 1e-12
    assert abs(gauge.mean_plaquette(ug)) < 0.02


def test_df64_dh_against_fp64_16x4(fgmod):
    """16^4, FG dt = 0.25 from a hot start: the double-float dH against the
    GPU FP64 path (itself pinned to the oracle at 1e-12 per step)."""
    dims = (16, 16, 16, 16)
    u = inputs.hot_start(dims, 31)
    p = inputs.gaussian_momenta(dims, 32)
    out = {}
    for prec in ("fp64", "df64"):
        with fgmod.Lattice(dims, BETA, precision=prec) as lat:
            lat.set_gauge(u)
            lat.set_momenta(p)
            out[prec] = lat.trajectory("fg", 0.25, 1.0, refresh=False, u_accept=0.0)
    assert abs(out["df64"]["dH"] - out["fp64"]["dH"]) <= 1e-6, (out["df64"]["dH"], out["fp64"]["dH"])
