"""Pins for the oracle's closed-form force gradient (section 4): the
derivative of the force along a link tangent, for the gauge and the
pseudofermion force, against Richardson-extrapolated central differences of
the force along exp(i s H) U; and the analytic force-gradient step against the
finite-difference one."""

import numpy as np
import pytest

from oracle import fermion as fe, gauge, integrators as it
from oracle.su3 import alg_to_mat, expi
from paper_0910_2950_gb300 import inputs

BETA, KAPPA = 5.6, 0.12


def _direction(dims, seed):
    g = inputs.make_rng(seed)
    return alg_to_mat(g.standard_normal(inputs.site_shape(dims) + (4, 8)))


def _richardson(force, u, h, eps):
    def d(e):
        return (force(expi(h, e) @ u) - force(expi(h, -e) @ u)) / (2.0 * e)
    return (4.0 * d(eps / 2) - d(eps)) / 3.0


def test_gauge_force_tangent_matches_finite_difference():
    dims = (4, 4, 2, 4)
    u = inputs.hot_start(dims, 3)
    h = _direction(dims, 4)
    t = gauge.gauge_force_tangent(u, 1j * h @ u, BETA)
    ref = _richardson(lambda v: gauge.gauge_force(v, BETA), u, h, 1e-3)
    assert np.max(np.abs(t - ref)) < 1e-9 * np.max(np.abs(ref))


def test_gauge_force_tangent_is_linear_and_vanishes_at_cold_start():
    dims = (2, 2, 2, 4)
    u = inputs.hot_start(dims, 5)
    h1, h2 = _direction(dims, 6), _direction(dims, 7)
    t1 = gauge.gauge_force_tangent(u, 1j * h1 @ u, BETA)
    t2 = gauge.gauge_force_tangent(u, 1j * h2 @ u, BETA)
    t12 = gauge.gauge_force_tangent(u, 1j * (2.0 * h1 - h2) @ u, BETA)
    assert np.max(np.abs(t12 - (2.0 * t1 - t2))) < 1e-12 * np.max(np.abs(t12))
    # from U = 1 along a generator H that is the same on every link, every
    # link is exp(i s H): all plaquettes stay 1, the force stays 0, and so
    # does its derivative
    cold = inputs.cold_start(dims)
    hc = np.broadcast_to(alg_to_mat(np.arange(1, 9, dtype=float) / 8.0), cold.shape).copy()
    t = gauge.gauge_force_tangent(cold, 1j * hc @ cold, BETA)
    assert np.max(np.abs(t)) < 1e-13


def test_fermion_force_tangent_matches_finite_difference():
    dims = (2, 2, 2, 4)
    u = inputs.hot_start(dims, 8)
    chi = inputs.unpack_even(inputs.gaussian_spinor_even(dims, 9), dims)
    phi = fe.heatbath_phi(u, KAPPA, chi)
    h = _direction(dims, 10)
    t = fe.fermion_force_tangent(u, 1j * h @ u, KAPPA, phi, tol=1e-15)
    ref = _richardson(lambda v: fe.fermion_force(v, KAPPA, phi, tol=1e-15), u, h, 1e-3)
    assert np.max(np.abs(t - ref)) < 1e-8 * np.max(np.abs(ref))


def test_mdagm_tangent_matches_finite_difference():
    """F(calM) X of section 4 for one direction: the derivative of the
    operator itself, applied to a fixed vector."""
    dims = (2, 2, 2, 4)
    u = inputs.hot_start(dims, 11)
    x = inputs.unpack_even(inputs.gaussian_spinor_even(dims, 12), dims)
    h = _direction(dims, 13)
    t = fe.mdagm_tangent(u, 1j * h @ u, KAPPA, x)
    ref = _richardson(lambda v: fe.mdagm(v, KAPPA, x), u, h, 1e-3)
    assert np.max(np.abs(t - ref)) < 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("system_kind", ["gauge", "fermion"])
def test_analytic_fg_step_matches_finite_difference_fg_step(system_kind):
    dims = (2, 2, 2, 4)
    u = inputs.hot_start(dims, 14)
    p = inputs.gaussian_momenta(dims, 15)
    if system_kind == "gauge":
        make = lambda: it.GaugeSystem(BETA)          # noqa: E731
    else:
        phi = fe.heatbath_phi(u, KAPPA, inputs.unpack_even(inputs.gaussian_spinor_even(dims, 16), dims))
        make = lambda: fe.FermionSystem(BETA, KAPPA, phi, tol=1e-15)   # noqa: E731
    ua, pa = it.md_step(make(), it.Integrator("fg_analytic"), u, p, 0.2)
    ue, pe = it.md_step(make(), it.Integrator("fg", fg_mode="exact", fd_eps=1e-4), u, p, 0.2)
    ud, pd = it.md_step(make(), it.Integrator("fg"), u, p, 0.2)
    # finite-difference error ~ eps^2 |F'''| dt^3, far below the O(dt^5)
    # difference to the displaced-force surrogate
    err_fd = np.max(np.abs(pa - pe))
    err_disp = np.max(np.abs(pa - pd))
    assert err_fd < 1e-9
    assert err_disp > 100 * err_fd
    assert np.max(np.abs(ua - ue)) < 1e-9


@pytest.mark.slow
def test_analytic_fg_is_fourth_order_with_fermions():
    dims = (2, 2, 2, 4)
    u = inputs.hot_start(dims, 2)
    phi = fe.heatbath_phi(u, KAPPA, inputs.unpack_even(inputs.gaussian_spinor_even(dims, 3), dims))
    p = inputs.gaussian_momenta(dims, 4)
    dts = [1 / 4, 1 / 8, 1 / 16]
    dh = []
    for dt in dts:
        system = fe.FermionSystem(BETA, KAPPA, phi, tol=1e-14)
        _, _, h0, h1 = it.trajectory(system, it.Integrator("fg_analytic"), u, p, dt, 1.0)
        dh.append(abs(h1 - h0))
    slope = np.polyfit(np.log(dts), np.log(dh), 1)[0]
    assert 3.5 < slope < 4.6, (slope, dh)
