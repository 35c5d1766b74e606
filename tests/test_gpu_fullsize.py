"""Full-size GPU checks in the launch configuration the benchmark times.

* 32^4 pure gauge, FP32, 18-real links (the bench workload): the force at
  sampled links against the per-link oracle, the action and kinetic totals
  against the whole-field oracle, gauge covariance of the force (sampled),
  and reversibility of a force-gradient trajectory (a property at any size).
* 16^4 pure gauge from a thermalised FP64 start: the FP32 path's dH against
  the FP64 path's (itself pinned to the oracle at 1e-12) for FG and leapfrog
  trajectories; a one-signed rounding bias in the link normalisation shows
  up here as an offset proportional to the volume.
* 16^3 x 32 Nf=2 Wilson, kappa = 0.158, FP32 links with mixed-precision CG:
  Mhat against the whole-field oracle, the CG solution's FP64 true residual
  recomputed by the oracle, and the total force against the oracle's force
  evaluated with the GPU's solution.

FP32 tolerances: a link product carries ~1e-7 relative rounding, so forces
(sums of O(10) such products) are compared at 2e-6 relative to the largest
component; totals over 10^6 sites at 1e-6 relative.
"""

import numpy as np
import pytest

from oracle import fermion as fe, gauge, su3
from paper_0910_2950_gb300 import inputs

pytestmark = pytest.mark.gpu

BETA = 6.0


@pytest.fixture(scope="module")
def fgmod():
    from paper_0910_2950_gb300 import build, fg
    build.build()
    fg.load()
    return fg


@pytest.fixture(scope="module")
def hot32():
    dims = (32, 32, 32, 32)
    return dims, inputs.hot_start(dims, 1)


def _sample_links(dims, n, seed):
    rng = inputs.make_rng(seed)
    lt, lz, ly, lx = inputs.site_shape(dims)
    return [((int(rng.integers(lt)), int(rng.integers(lz)), int(rng.integers(ly)), int(rng.integers(lx))),
             int(rng.integers(4))) for _ in range(n)]


def test_force_32x4_fp32_sampled(fgmod, hot32):
    dims, u = hot32
    with fgmod.Lattice(dims, BETA, precision="fp32") as lat:
        lat.set_gauge(u)
        f = lat.force()
        sg, _, _ = lat.action()
    u32 = None
    worst, scale = 0.0, 0.0
    for site, mu in _sample_links(dims, 256, 3):
        # the GPU holds FP32 links: compare with the oracle on the rounded links
        if u32 is None:
            u32 = u.astype(np.complex64).astype(np.complex128)
        ref = gauge.link_force(u32, site, mu, BETA)
        worst = max(worst, float(np.max(np.abs(f[site + (mu,)] - ref))))
        scale = max(scale, float(np.max(np.abs(ref))))
    assert worst < 2e-6 * scale, (worst, scale)
    s_ref = gauge.wilson_action(u32, BETA)
    assert abs(sg - s_ref) < 1e-6 * abs(s_ref)


def test_force_covariance_32x4_fp32_sampled(fgmod, hot32):
    dims, u = hot32
    g = inputs.random_gauge_transform(dims, 7)
    ug = gauge.gauge_transform_links(u, g)
    with fgmod.Lattice(dims, BETA, precision="fp32") as lat:
        lat.set_gauge(u)
        f0 = lat.force()
        lat.set_gauge(ug)
        f1 = lat.force()
    worst, scale = 0.0, 0.0
    for site, mu in _sample_links(dims, 256, 4):
        rot = g[site] @ su3.alg_to_mat(f0[site + (mu,)]) @ su3.dag(g[site])
        new = su3.alg_to_mat(f1[site + (mu,)])
        worst = max(worst, float(np.max(np.abs(rot - new))))
        scale = max(scale, float(np.max(np.abs(new))))
    assert worst < 5e-6 * scale, (worst, scale)


def test_fg_trajectory_reversibility_32x4_fp32(fgmod, hot32):
    dims, u = hot32
    with fgmod.Lattice(dims, BETA, precision="fp32", seed=11) as lat:
        lat.set_gauge(u)
        for _ in range(3):     # move off the hot start so forces are moderate
            lat.trajectory("fg", 0.125, 1.0, refresh=True, u_accept=0.0)
        u0 = lat.get_gauge()
        lat.refresh_momenta()
        p0 = lat.get_momenta()
        sg, _, t = lat.action()
        assert abs(t - 0.5 * np.sum(p0 * p0)) < 1e-6 * t
        r1 = lat.trajectory("fg", 0.25, 1.0, refresh=False, u_accept=0.0)
        lat.set_momenta(-lat.get_momenta())
        r2 = lat.trajectory("fg", 0.25, 1.0, refresh=False, u_accept=0.0)
        u2 = lat.get_gauge()
        p2 = lat.get_momenta()
    # FP32 links and re-unitarisation after every drift: reversible to FP32 rounding
    assert np.max(np.abs(u2 - u0)) < 1e-4
    assert np.max(np.abs(p2 + p0)) < 1e-3
    assert abs(r1["dH"] + r2["dH"]) < 0.05 * max(1.0, abs(r1["dH"]))


@pytest.fixture(scope="module")
def nf2_case():
    dims = (16, 16, 16, 32)
    u = inputs.hot_start(dims, 2)
    return dims, u, u.astype(np.complex64).astype(np.complex128)


@pytest.mark.parametrize("integ,dt", [("fg", 0.25), ("leapfrog", 0.05)])
def test_fp32_dh_against_fp64_16x4(fgmod, integ, dt):
    dims = (16, 16, 16, 16)
    with fgmod.Lattice(dims, BETA, precision="fp64", seed=500) as base:
        base.set_gauge(inputs.hot_start(dims, 11))
        for _ in range(10):
            base.trajectory("fg", 0.125, 1.0, refresh=True, u_accept=0.0)
        u = base.get_gauge()
    p = inputs.gaussian_momenta(dims, 13)
    dh = {}
    for prec in ("fp64", "fp32"):
        with fgmod.Lattice(dims, BETA, precision=prec, seed=600) as lat:
            lat.set_gauge(u)
            lat.set_momenta(p)
            dh[prec] = lat.trajectory(integ, dt, 1.0, refresh=False, u_accept=0.0)["dH"]
    # H ~ 2e6 here; random FP32 rounding of 4.7e6 link and momentum entries per
    # step moves dH by ~1e-3; a coherent half-ulp bias per link moved it by 0.2
    assert abs(dh["fp32"] - dh["fp64"]) < 2e-2, dh


def test_mhat_16x16x16x32_fp32_links(fgmod, nf2_case):
    dims, u, u32 = nf2_case
    psi = inputs.gaussian_spinor_even(dims, 3)
    with fgmod.Lattice(dims, 5.6, kappa=0.158, precision="fp32") as lat:
        lat.set_gauge(u)
        out = lat.apply_mhat(psi)
        outd = lat.apply_mhat(psi, dagger=True)
    full = inputs.unpack_even(psi, dims)
    ref = inputs.pack_even(fe.mhat(u32, 0.158, full), dims)
    refd = inputs.pack_even(fe.mhat_dag(u32, 0.158, full), dims)
    assert np.max(np.abs(out - ref)) < 1e-13 * np.max(np.abs(ref))
    assert np.max(np.abs(outd - refd)) < 1e-13 * np.max(np.abs(refd))


@pytest.mark.parametrize("precision", ["fp32", "fp32_fp16cg", "fp32_bf16cg"])
def test_cg_and_force_16x16x16x32(fgmod, nf2_case, precision):
    dims, u, u32 = nf2_case
    kappa, tol = 0.158, 1e-10
    chi = inputs.gaussian_spinor_even(dims, 4)
    phi = fe.heatbath_phi(u32, kappa, inputs.unpack_even(chi, dims))
    with fgmod.Lattice(dims, 5.6, kappa=kappa, precision=precision, cg_tol=tol) as lat:
        lat.set_gauge(u)
        lat.set_pseudofermion(chi)
        x, info = lat.cg_solve(inputs.pack_even(phi, dims))
        f = lat.force()
    assert info["true_residual"] <= tol
    xf = inputs.unpack_even(x, dims)
    res = phi - fe.mdagm(u32, kappa, xf)
    assert np.linalg.norm(res) <= 1.01 * tol * np.linalg.norm(phi)
    ref = gauge.gauge_force(u32, 5.6) + fe.fermion_force(u32, kappa, phi, x=xf)
    assert np.max(np.abs(f - ref)) < 5e-6 * np.max(np.abs(ref))
