"""GPU parity of the pure-gauge path against the FP64 oracle, through the C ABI.

Tolerances:
* FP64 path: normwise relative 1e-12 for forces, links and momenta after one
  MD step; |dH_gpu - dH_oracle| <= 1e-12 (|S| + |T|) and <= 1e-6 absolute for
  a whole trajectory.
* FP32 path: see the individual tests; bounds follow from FP32 rounding
  (unit roundoff 6e-8) of O(10) terms per link.
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
def test_gauge_roundtrip_fp64(fgmod, dims, link_reals):
    u = inputs.hot_start(dims, 3)
    with fgmod.Lattice(dims, BETA, precision="fp64", link_reals=link_reals) as lat:
        lat.set_gauge(u)
        back = lat.get_gauge()
    tol = 0.0 if link_reals == 18 else 1e-14
    assert np.max(np.abs(back - u)) <= tol


@pytest.mark.parametrize("dims", DIMS_CASES)
@pytest.mark.parametrize("link_reals", [18, 12])
def test_force_fp64(fgmod, dims, link_reals):
    u = inputs.hot_start(dims, 5)
    with fgmod.Lattice(dims, BETA, precision="fp64", link_reals=link_reals) as lat:
        lat.set_gauge(u)
        f = lat.force()
    ref = gauge.gauge_force(u, BETA)
    assert _rel(f, ref) < 1e-12


@pytest.mark.parametrize("link_reals", [18, 12])
def test_force_fp32(fgmod, link_reals):
    dims = (6, 4, 2, 6)
    u = inputs.hot_start(dims, 5)
    with fgmod.Lattice(dims, BETA, precision="fp32", link_reals=link_reals) as lat:
        lat.set_gauge(u)
        f = lat.force()
    ref = gauge.gauge_force(u, BETA)
    assert _rel(f, ref) < 2e-6


@pytest.mark.parametrize("dims", DIMS_CASES)
def test_action_and_plaquette_fp64(fgmod, dims):
    u = inputs.hot_start(dims, 6)
    p = inputs.gaussian_momenta(dims, 7)
    with fgmod.Lattice(dims, BETA) as lat:
        lat.set_gauge(u)
        lat.set_momenta(p)
        sg, sf, t = lat.action()
        plaq = lat.plaquette()
    assert abs(sg - gauge.wilson_action(u, BETA)) <= 1e-12 * abs(sg)
    assert abs(t - gauge.kinetic(p)) <= 1e-12 * abs(t)
    assert sf == 0.0
    assert abs(plaq - gauge.mean_plaquette(u)) < 1e-13


def test_cold_start_and_momenta_roundtrip(fgmod):
    dims = (4, 4, 2, 6)
    p = inputs.gaussian_momenta(dims, 2)
    with fgmod.Lattice(dims, BETA) as lat:
        assert np.array_equal(lat.get_gauge(), inputs.cold_start(dims))
        assert lat.plaquette() == 1.0
        assert np.max(np.abs(lat.force())) == 0.0
        lat.set_momenta(p)
        assert np.array_equal(lat.get_momenta(), p)


@pytest.mark.parametrize("name", ["leapfrog", "omelyan", "fg", "campostrini", "qpq"])
@pytest.mark.parametrize("link_reals", [18, 12])
def test_one_md_step_fp64(fgmod, name, link_reals):
    dims = (6, 4, 2, 6)
    u = inputs.hot_start(dims, 8)
    p = inputs.gaussian_momenta(dims, 9)
    dt = 0.1
    with fgmod.Lattice(dims, BETA, link_reals=link_reals) as lat:
        lat.set_gauge(u)
        lat.set_momenta(p)
        lat.md_step(name, dt)
        ug, pg = lat.get_gauge(), lat.get_momenta()
    uo, po = it.md_step(it.GaugeSystem(BETA), it.Integrator(name), u, p, dt)
    assert _rel(ug, uo) < 1e-12
    assert _rel(pg, po) < 1e-12


def test_fg_step_entry_point(fgmod):
    dims = (4, 4, 4, 4)
    u = inputs.hot_start(dims, 10)
    p = inputs.gaussian_momenta(dims, 11)
    with fgmod.Lattice(dims, BETA) as lat:
        lat.set_gauge(u)
        lat.set_momenta(p)
        lat.fg_step(0.2)
        ug, pg = lat.get_gauge(), lat.get_momenta()
    uo, po = it.md_step(it.GaugeSystem(BETA), it.Integrator("fg"), u, p, 0.2)
    assert _rel(ug, uo) < 1e-12 and _rel(pg, po) < 1e-12


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
def test_config1_trajectory_dh_fp64(fgmod, config1_oracle, name):
    dims, u, p, ref = config1_oracle
    dhs = []
    with fgmod.Lattice(dims, BETA) as lat:
        for dt in (1 / 4, 1 / 8, 1 / 16, 1 / 32):
            lat.set_gauge(u)
            lat.set_momenta(p)
            r = lat.trajectory(name, dt, 1.0, refresh=False, u_accept=0.0)
            dh_o, h0_o, u1_o, p1_o = ref[(name, dt)]
            assert abs(r["H0"] - h0_o) <= 1e-12 * abs(h0_o)
            assert abs(r["dH"] - dh_o) <= min(1e-6, 1e-12 * abs(h0_o)), (name, dt, r["dH"], dh_o)
            assert r["accepted"] == 1
            assert r["n_steps"] == round(1 / dt)
            n = r["n_steps"]
            assert r["n_force"] == {"leapfrog": n + 1, "omelyan": 2 * n + 1, "fg": 3 * n + 1}[name]
            assert _rel(lat.get_gauge(), u1_o) < 1e-12
            assert _rel(lat.get_momenta(), p1_o) < 1e-11
            dhs.append(abs(r["dH"]))
    slope = np.polyfit(np.log([1 / 4, 1 / 8, 1 / 16, 1 / 32]), np.log(dhs), 1)[0]
    assert (3.6 < slope < 4.5) if name == "fg" else (1.7 < slope < 2.3), slope


def test_reject_restores_links(fgmod):
    """Run a trajectory, then run back from its end with reversed momenta: by
    reversibility dH is minus the first one (large and positive), so a uniform
    close to 1 rejects and the links must be restored bit for bit."""
    dims = (4, 4, 4, 4)
    u = inputs.hot_start(dims, 1)
    p = inputs.gaussian_momenta(dims, 1)
    with fgmod.Lattice(dims, BETA) as lat:
        lat.set_gauge(u)
        lat.set_momenta(p)
        r1 = lat.trajectory("leapfrog", 0.25, 1.0, refresh=False, u_accept=0.0)
        assert r1["dH"] < -1.0 and r1["accepted"] == 1
        u1 = lat.get_gauge()
        lat.set_momenta(-lat.get_momenta())
        r2 = lat.trajectory("leapfrog", 0.25, 1.0, refresh=False, u_accept=0.999999)
        assert abs(r2["dH"] + r1["dH"]) < 1e-8 * abs(r1["H0"])
        assert r2["accepted"] == 0
        assert np.array_equal(lat.get_gauge(), u1)


def test_device_momentum_refresh_statistics(fgmod):
    dims = (8, 8, 8, 8)
    with fgmod.Lattice(dims, BETA, seed=1234) as lat:
        lat.refresh_momenta()
        p1 = lat.get_momenta()
        lat.refresh_momenta()
        p2 = lat.get_momenta()
    v = inputs.volume(dims)
    for p in (p1, p2):
        assert abs(p.mean()) < 5 / np.sqrt(p.size)
        assert abs(p.var() - 1) < 5 * np.sqrt(2 / p.size)
        assert abs(0.5 * np.sum(p * p) / (16 * v) - 1) < 5 * np.sqrt(2 / p.size)
    assert np.max(np.abs(p1 - p2)) > 1        # the counter advanced
    assert abs(np.corrcoef(p1.ravel(), p2.ravel())[0, 1]) < 5 / np.sqrt(p1.size)


def test_fp32_reunitarized_drift_stays_special_unitary(fgmod):
    dims = (6, 4, 2, 6)
    u = inputs.hot_start(dims, 3)
    p = inputs.gaussian_momenta(dims, 4)
    with fgmod.Lattice(dims, BETA, precision="fp32") as lat:
        lat.set_gauge(u)
        lat.set_momenta(p)
        for _ in range(20):
            lat.md_step("fg", 0.1)
        ug = lat.get_gauge()
    assert su3.unitarity_defect(ug) < 2e-6
    assert np.max(np.abs(np.linalg.det(ug) - 1)) < 5e-6


def test_fp32_trajectory_dh_close_to_fp64(fgmod, config1_oracle):
    dims, u, p, ref = config1_oracle
    with fgmod.Lattice(dims, BETA, precision="fp32") as lat:
        lat.set_gauge(u)
        lat.set_momenta(p)
        r = lat.trajectory("fg", 1 / 8, 1.0, refresh=False, u_accept=0.0)
    dh_o = ref[("fg", 1 / 8)][0]
    # FP32 link arithmetic: each of the ~4V*18 link entries carries ~1e-7
    # relative error, so S (~1e4 here) moves by ~1e-3 at most; dH is a
    # site-by-site FP64 sum of FP32 terms.
    assert abs(r["dH"] - dh_o) < 2e-3, (r["dH"], dh_o)


def test_wait_limit_reports_timeout(fgmod):
    """A host wait limit far below a trajectory's run time: the trajectory
    call returns FG_ETIMEOUT with its work still queued; without the limit
    the queue drains and, with its fields set again, the handle gives the
    same result as a fresh one."""
    dims = (24, 24, 24, 24)
    u = inputs.hot_start(dims, 5)
    p = inputs.gaussian_momenta(dims, 6)
    with fgmod.Lattice(dims, BETA, precision="fp32") as fresh:
        fresh.set_gauge(u)
        fresh.set_momenta(p)
        ref = fresh.trajectory("fg", 0.125, 1.0, refresh=False, u_accept=0.0)
    with fgmod.Lattice(dims, BETA, precision="fp32") as lat:
        lat.set_gauge(u)
        lat.set_momenta(p)
        lat.set_wait_limit(1e-6)
        with pytest.raises(fgmod.FgError) as e:
            lat.trajectory("fg", 0.125, 1.0, refresh=False, u_accept=0.0)
        assert e.value.status == fgmod.FG_ETIMEOUT
        lat.set_wait_limit(0.0)
        lat.sync()
        lat.set_gauge(u)
        lat.set_momenta(p)
        r = lat.trajectory("fg", 0.125, 1.0, refresh=False, u_accept=0.0)
    assert r["dH"] == ref["dH"]
    with pytest.raises(fgmod.FgError):
        lat2 = fgmod.Lattice((4, 4, 4, 4), BETA)
        try:
            lat2.set_wait_limit(-1.0)
        finally:
            lat2.close()


def test_fp32_fma_rate(fgmod):
    """The FMA probe fills the FP32 pipes: between half and all of the
    unit-count rate (SMs x 128 lanes x 2 flop) at 2.2 GHz, above any GB300
    SM clock (2070 MHz at most)."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    ceiling = sms * 128 * 2 * 2.2e9 / 1e12
    rate = fgmod.fp32_fma_rate()
    assert 0.5 * ceiling < rate < ceiling, (rate, ceiling)


def test_timing_and_launch_count(fgmod):
    dims = (4, 4, 4, 4)
    with fgmod.Lattice(dims, BETA) as lat:
        lat.set_gauge(inputs.hot_start(dims, 1))
        lat.timing(True)
        n0 = lat.launch_count()
        lat.trajectory("fg", 0.25, 1.0, refresh=True, u_accept=0.0)
        n1 = lat.launch_count()
        ms, n = lat.kernel_time("gauge_force")
        assert n == 13 and ms > 0
        assert n1 - n0 >= 13 + 1 + 2
        assert lat.device_bytes() > 0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_stored_site_action_matches_recomputation(fgmod, precision):
    """A trajectory takes the per-site gauge action of its start links from
    the end of the previous trajectory (accepted or rejected) unless the links
    changed in between.  A second lattice that re-uploads its links before
    every trajectory (which drops the stored values) must see the same H0
    and dH bit for bit, through accepts and rejects."""
    dims = (6, 4, 4, 6)
    u = inputs.hot_start(dims, 51)
    ps = [inputs.gaussian_momenta(dims, 60 + k) for k in range(6)]
    out = []
    for reupload in (False, True):
        rows = []
        with fgmod.Lattice(dims, BETA, precision=precision) as lat:
            lat.set_gauge(u)
            for k, p in enumerate(ps):
                if reupload:
                    lat.set_gauge(lat.get_gauge())
                lat.set_momenta(p)
                r = lat.trajectory("fg", 0.5, 1.0, refresh=False, u_accept=0.9 if k % 2 else 0.0)
                rows.append((r["H0"], r["dH"], r["accepted"]))
        out.append(rows)
    assert out[0] == out[1]
    assert any(not a for _, _, a in out[0]) and any(a for _, _, a in out[0])


def test_c_example_chain_runs(fgmod, tmp_path):
    """The plain-C example (examples/hmc_chain.c) runs a short FG HMC chain
    through the ABI alone: every dH finite, the plaquette of the evolving
    field in (0, 1)."""
    import os
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pkg = os.path.join(root, "paper_0910_2950_gb300")
    exe = tmp_path / "hmc_chain"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(root, "include"), os.path.join(pkg, "examples", "hmc_chain.c"),
                    "-L", pkg, "-l:libfg_lattice.so", "-Wl,-rpath," + pkg, "-lm", "-o", str(exe)], check=True)
    res = subprocess.run([str(exe), "6", "6"], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr
    lines = [ln.split() for ln in res.stdout.splitlines() if ln.startswith("trajectory")]
    assert len(lines) == 6
    for ln in lines:
        assert np.isfinite(float(ln[3]))
        assert 0.0 < float(ln[9]) < 1.0
    assert res.stdout.splitlines()[-1].startswith("accepted")
