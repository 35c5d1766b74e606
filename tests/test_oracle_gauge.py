"""Pins for oracle.gauge: closed forms, invariances and finite differences."""

import numpy as np
import pytest

from oracle import gauge, su3
from paper_0910_2950_gb300 import inputs

BETA = 6.0


def _action_difference(u_a, u_b, beta):
    """S(u_a) - S(u_b) summed plaquette by plaquette (no cancellation of totals)."""
    d = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            pa = np.real(su3.trace(gauge.plaquette_field(u_a, mu, nu)))
            pb = np.real(su3.trace(gauge.plaquette_field(u_b, mu, nu)))
            d += np.sum(pb - pa) / 3.0
    return beta * d


def _fd_derivative(u, site_link, a, fn_diff, eps=1e-3):
    """Fourth-order central difference of a scalar along U -> exp(i e T^a) U."""
    def moved(e):
        v = u.copy()
        v[site_link] = su3.expi(su3.GENERATORS[a], e) @ v[site_link]
        return v
    d1 = fn_diff(moved(eps), moved(-eps))
    d2 = fn_diff(moved(2 * eps), moved(-2 * eps))
    return (8 * d1 - d2) / (12 * eps)


def test_cold_start_is_vacuum():
    u = inputs.cold_start((4, 4, 4, 4))
    assert gauge.wilson_action(u, BETA) == 0.0
    assert np.max(np.abs(gauge.gauge_force(u, BETA))) == 0.0
    assert gauge.mean_plaquette(u) == 1.0


def test_single_rotated_link_closed_form():
    """One link diag(e^{i th/2}, e^{-i th/2}, 1) in a cold field.

    It sits in 6 plaquettes with Re Tr = 2 cos(th/2) + 1, so
    S = 4 beta (1 - cos(th/2)) and the force is F^3 = 2 beta sin(th/2), all
    other components zero (dS/d th along lambda^3 / 2).
    """
    dims = (4, 4, 4, 6)
    th = 0.83
    u = inputs.cold_start(dims)
    site = (2, 1, 3, 0, 1)
    u[site] = np.diag([np.exp(0.5j * th), np.exp(-0.5j * th), 1.0])
    assert np.isclose(gauge.wilson_action(u, BETA), 4 * BETA * (1 - np.cos(th / 2)), rtol=1e-13)
    f = gauge.gauge_force(u, BETA)[site]
    expect = np.zeros(8)
    expect[2] = 2 * BETA * np.sin(th / 2)
    assert np.allclose(f, expect, atol=1e-13)


def test_constant_abelian_flux_closed_form():
    """U_x(x) = diag(e^{i phi y}, e^{-i phi y}, 1), phi = 2 pi k / Ly: every (x,y)
    plaquette is diag(e^{-i phi}, e^{i phi}, 1), all others are 1; it is a
    classical solution so the force vanishes."""
    dims = (4, 6, 4, 4)
    phi = 2 * np.pi * 1 / 6
    u = inputs.cold_start(dims)
    y = np.arange(6)[None, None, :, None]
    u[..., 0, 0, 0] = np.exp(1j * phi * y)
    u[..., 0, 1, 1] = np.exp(-1j * phi * y)
    v = inputs.volume(dims)
    expect = BETA * v * (1 - (2 * np.cos(phi) + 1) / 3)
    assert np.isclose(gauge.wilson_action(u, BETA), expect, rtol=1e-13)
    assert np.max(np.abs(gauge.gauge_force(u, BETA))) < 1e-13


def test_haar_links_are_disordered():
    dims = (4, 4, 4, 4)
    u = inputs.hot_start(dims, 1)
    ratio = gauge.wilson_action(u, BETA) / (6 * inputs.volume(dims) * BETA)
    assert abs(ratio - 1.0) < 0.03     # std of the mean plaquette ~ 0.006


def test_force_matches_finite_difference_of_action():
    dims = (4, 4, 4, 4)
    u = inputs.hot_start(dims, 7)
    f = gauge.gauge_force(u, BETA)
    rng = inputs.make_rng(11)
    for _ in range(12):
        t, z, y, x, mu = (int(rng.integers(4)) for _ in range(5))
        a = int(rng.integers(8))
        fd = _fd_derivative(u, (t, z, y, x, mu), a,
                            lambda ua, ub: _action_difference(ua, ub, BETA))
        assert abs(fd - f[t, z, y, x, mu, a]) <= 1e-8 * max(1.0, abs(fd)), (fd, f[t, z, y, x, mu, a])


def test_gauge_invariance_and_force_covariance():
    dims = (4, 4, 4, 4)
    u = inputs.hot_start(dims, 2)
    g = inputs.random_gauge_transform(dims, 9)
    ug = gauge.gauge_transform_links(u, g)
    s0, s1 = gauge.wilson_action(u, BETA), gauge.wilson_action(ug, BETA)
    assert abs(s0 - s1) <= 1e-12 * abs(s0)
    f0 = su3.alg_to_mat(gauge.gauge_force(u, BETA))
    f1 = su3.alg_to_mat(gauge.gauge_force(ug, BETA))
    # F_mu(x) -> g(x) F_mu(x) g(x)^dagger
    rot = g[..., None, :, :] @ f0 @ su3.dag(g)[..., None, :, :]
    assert np.max(np.abs(rot - f1)) < 1e-12


def test_kinetic_term():
    p = inputs.gaussian_momenta((4, 4, 4, 4), 1)
    assert gauge.kinetic(p) == pytest.approx(np.sum(np.real(su3.trace(su3.alg_to_mat(p) @ su3.alg_to_mat(p)))), rel=1e-13)
    # <T> = (8 / 2) * 4V = 16 V for unit-Gaussian momenta
    v = inputs.volume((4, 4, 4, 4))
    assert abs(gauge.kinetic(p) / (16 * v) - 1) < 5 * np.sqrt(2 / (32 * v))


def test_link_force_equals_whole_lattice_force():
    dims = (4, 6, 2, 4)
    u = inputs.hot_start(dims, 12)
    f = gauge.gauge_force(u, BETA)
    for t in range(4):
        for z in range(2):
            for y in range(6):
                for x in range(4):
                    for mu in range(4):
                        assert np.allclose(gauge.link_force(u, (t, z, y, x), mu, BETA), f[t, z, y, x, mu],
                                           rtol=0, atol=1e-13)
