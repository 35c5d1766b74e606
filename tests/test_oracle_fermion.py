"""Pins for oracle.fermion: Clifford algebra, closed forms, brute force, finite differences."""

import numpy as np
import pytest

from oracle import fermion as fe, gauge, integrators as it, su3
from paper_0910_2950_gb300 import inputs

KAPPA = 0.12


def _rand_spinor(dims, seed):
    g = inputs.make_rng(seed)
    sh = inputs.site_shape(dims) + (4, 3)
    return g.standard_normal(sh) + 1j * g.standard_normal(sh)


def _even(dims, seed):
    return _rand_spinor(dims, seed) * inputs.parity_mask(dims)[..., None, None]


def test_gamma_matrices():
    g = fe.GAMMA
    for m in range(4):
        assert np.allclose(g[m], su3.dag(g[m]))
        for n in range(4):
            assert np.allclose(g[m] @ g[n] + g[n] @ g[m], 2 * (m == n) * np.eye(4), atol=0)
    assert np.allclose(fe.GAMMA5, np.diag([1, 1, -1, -1]))   # chiral (DeGrand-Rossi) basis


def test_gamma5_hermiticity():
    dims = (4, 4, 2, 4)
    u = inputs.hot_start(dims, 1)
    a, b = _rand_spinor(dims, 2), _rand_spinor(dims, 3)
    lhs = fe.vdot(a, fe.spin_mul(fe.GAMMA5, fe.hop(u, fe.spin_mul(fe.GAMMA5, b))))
    rhs = fe.vdot(fe.hop(u, a), b)
    assert abs(lhs - rhs) < 1e-11 * abs(rhs)
    ae, be = _even(dims, 4), _even(dims, 5)
    assert abs(fe.vdot(ae, fe.mhat_dag(u, KAPPA, be)) - fe.vdot(fe.mhat(u, KAPPA, ae), be)) < 1e-11 * np.abs(fe.vdot(ae, be)) + 1e-11


def test_free_field_plane_waves():
    """U = 1: M e^{ipx} eta = (1 - 2k sum cos p + 2ik sum gamma sin p) e^{ipx} eta,
    with p_t = (2n+1) pi / Lt for the antiperiodic time direction."""
    dims = (4, 6, 4, 8)
    u = inputs.cold_start(dims)
    lt, lz, ly, lx = inputs.site_shape(dims)
    n = (1, 2, 3, 1)
    p = np.array([2 * np.pi * n[0] / lx, 2 * np.pi * n[1] / ly, 2 * np.pi * n[2] / lz,
                  (2 * n[3] + 1) * np.pi / lt])
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    eta = _rand_spinor((2, 2, 2, 2), 7)[0, 0, 0, 0]
    psi = phase[..., None, None] * eta
    mp = (1 - 2 * KAPPA * np.sum(np.cos(p))) * np.eye(4) + 2j * KAPPA * np.einsum(
        "m,mst->st", np.sin(p), fe.GAMMA)
    assert np.allclose(fe.wilson_m(u, KAPPA, psi), phase[..., None, None] * (mp @ eta), atol=1e-13)


def _dense(op, dims, even_only):
    mask = inputs.parity_mask(dims)
    sh = inputs.site_shape(dims) + (4, 3)
    sel = np.broadcast_to(mask[..., None, None] if even_only else np.ones(inputs.site_shape(dims), bool)[..., None, None], sh)
    idx = np.flatnonzero(sel.reshape(-1))
    mat = np.zeros((idx.size, idx.size), dtype=np.complex128)
    for j, k in enumerate(idx):
        e = np.zeros(int(np.prod(sh)), dtype=np.complex128)
        e[k] = 1.0
        mat[:, j] = op(e.reshape(sh)).reshape(-1)[idx]
    return mat, idx


def test_cg_matches_dense_solve_on_2x2x2x2():
    dims = (2, 2, 2, 2)
    u = inputs.hot_start(dims, 3)
    mat, idx = _dense(lambda v: fe.mdagm(u, KAPPA, v), dims, True)
    assert mat.shape == (96, 96)
    assert np.allclose(mat, su3.dag(mat), atol=1e-13)
    assert np.min(np.linalg.eigvalsh(mat)) > 0
    b = _even(dims, 8)
    x, iters = fe.cg(u, KAPPA, b, tol=1e-13)
    xd = np.linalg.solve(mat, b.reshape(-1)[idx])
    assert np.max(np.abs(x.reshape(-1)[idx] - xd)) < 1e-12 * np.max(np.abs(xd))
    assert iters <= 96 + 20


def test_even_odd_schur_equals_full_solve():
    dims = (2, 2, 2, 4)
    u = inputs.hot_start(dims, 5)
    full, idx = _dense(lambda v: fe.wilson_m(u, KAPPA, v), dims, False)
    eta = _rand_spinor(dims, 9)
    psi = np.linalg.solve(full, eta.reshape(-1)[idx]).reshape(eta.shape)
    mask = inputs.parity_mask(dims)[..., None, None]
    eta_e, eta_o = eta * mask, eta * ~mask
    rhs = eta_e + KAPPA * fe.hop(u, eta_o) * mask        # eta_e + kappa D_eo eta_o
    x, _ = fe.cg(u, KAPPA, fe.mhat_dag(u, KAPPA, rhs), tol=1e-14)
    assert np.max(np.abs(x - psi * mask)) < 1e-11
    psi_o = eta_o + KAPPA * fe.hop(u, x) * ~mask
    assert np.max(np.abs(psi_o - psi * ~mask)) < 1e-11


def test_heatbath_action_equals_chi_norm():
    dims = (4, 4, 4, 4)
    u = inputs.hot_start(dims, 2)
    chi = inputs.unpack_even(inputs.gaussian_spinor_even(dims, 3), dims)
    phi = fe.heatbath_phi(u, KAPPA, chi)
    s = fe.pseudofermion_action(u, KAPPA, phi, tol=1e-12)
    assert abs(s - fe.vdot(chi, chi).real) < 1e-9 * s
    # <chi^dagger chi> = 12 V/2 for density exp(-|chi|^2)
    assert abs(fe.vdot(chi, chi).real / (12 * inputs.volume(dims) / 2) - 1) < 0.05


def test_fermion_force_matches_finite_difference():
    dims = (4, 4, 2, 4)
    u = inputs.hot_start(dims, 6)
    chi = inputs.unpack_even(inputs.gaussian_spinor_even(dims, 4), dims)
    phi = fe.heatbath_phi(u, KAPPA, chi)
    f = fe.fermion_force(u, KAPPA, phi, tol=1e-14)
    rng = inputs.make_rng(12)
    eps = 1e-3
    for _ in range(8):
        site = tuple(int(rng.integers(n)) for n in inputs.site_shape(dims)) + (int(rng.integers(4)),)
        a = int(rng.integers(8))

        def s(e):
            v = u.copy()
            v[site] = su3.expi(su3.GENERATORS[a], e) @ v[site]
            return fe.pseudofermion_action(v, KAPPA, phi, tol=1e-14)
        fd = (8 * (s(eps) - s(-eps)) - (s(2 * eps) - s(-2 * eps))) / (12 * eps)
        assert abs(fd - f[site + (a,)]) <= 1e-8 * max(1.0, abs(fd)), (fd, f[site + (a,)])


def test_fermion_gauge_covariance():
    dims = (4, 4, 2, 4)
    u = inputs.hot_start(dims, 7)
    g = inputs.random_gauge_transform(dims, 8)
    ug = gauge.gauge_transform_links(u, g)
    chi = inputs.unpack_even(inputs.gaussian_spinor_even(dims, 9), dims)
    phi = fe.heatbath_phi(u, KAPPA, chi)
    phig = fe.colour_mul(g, phi)
    assert np.allclose(fe.heatbath_phi(ug, KAPPA, fe.colour_mul(g, chi)), phig, atol=1e-12)
    s0 = fe.pseudofermion_action(u, KAPPA, phi)
    s1 = fe.pseudofermion_action(ug, KAPPA, phig)
    assert abs(s0 - s1) < 1e-9 * s0
    f0 = su3.alg_to_mat(fe.fermion_force(u, KAPPA, phi))
    f1 = su3.alg_to_mat(fe.fermion_force(ug, KAPPA, phig))
    rot = g[..., None, :, :] @ f0 @ su3.dag(g)[..., None, :, :]
    assert np.max(np.abs(rot - f1)) < 1e-9 * np.max(np.abs(f1))


@pytest.mark.slow
def test_fermion_fg_trajectory_is_fourth_order():
    """Force-gradient on gauge + pseudofermion force keeps dH ~ dt^4; Omelyan dt^2."""
    dims = (2, 2, 2, 4)
    u = inputs.hot_start(dims, 2)
    chi = inputs.unpack_even(inputs.gaussian_spinor_even(dims, 3), dims)
    phi = fe.heatbath_phi(u, KAPPA, chi)
    p = inputs.gaussian_momenta(dims, 4)
    dts = [1 / 4, 1 / 8, 1 / 16]
    slopes = {}
    for name in ("omelyan", "fg"):
        dh = []
        for dt in dts:
            system = fe.FermionSystem(5.6, KAPPA, phi, tol=1e-13)
            _, _, h0, h1 = it.trajectory(system, it.Integrator(name), u, p, dt, 1.0)
            dh.append(abs(h1 - h0))
        slopes[name] = np.polyfit(np.log(dts), np.log(dh), 1)[0]
    assert 1.7 < slopes["omelyan"] < 2.4, slopes
    assert 3.5 < slopes["fg"] < 4.6, slopes


def test_fg_step_uses_three_solves_per_step():
    """Section 5: the force-gradient step needs three inversions per step once
    the outer 1/6 kicks of neighbouring steps are merged (four unmerged)."""
    dims = (2, 2, 2, 2)
    u = inputs.hot_start(dims, 2)
    phi = fe.heatbath_phi(u, KAPPA, inputs.unpack_even(inputs.gaussian_spinor_even(dims, 3), dims))
    system = fe.FermionSystem(5.6, KAPPA, phi)
    it.md_step(system, it.Integrator("fg"), u, inputs.gaussian_momenta(dims, 1), 0.1)
    assert system.n_solve == 4
