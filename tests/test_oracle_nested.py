"""Pins for the oracle's two-level (nested) integrator: reductions to the
one-level integrators, order, reversibility."""

import numpy as np
import pytest

from oracle import fermion as fe, integrators as it
from paper_0910_2950_gb300 import inputs

KAPPA = 0.12


class ZeroSystem:
    """An outer action that is identically zero."""

    def action(self, u):
        return 0.0

    def force(self, u):
        return np.zeros(u.shape[:-2] + (8,))


def _fermion_case(dims, seed=2):
    u = inputs.hot_start(dims, seed)
    chi = inputs.unpack_even(inputs.gaussian_spinor_even(dims, seed + 1), dims)
    phi = fe.heatbath_phi(u, KAPPA, chi)
    p = inputs.gaussian_momenta(dims, seed + 2)
    return u, phi, p


@pytest.mark.parametrize("outer,inner,n_inner", [("leapfrog", "omelyan", 3), ("fg", "leapfrog", 2),
                                                  ("omelyan", "fg", 1)])
def test_zero_outer_action_gives_the_inner_integrator(outer, inner, n_inner):
    """With S_outer = 0 the outer kicks vanish and its drifts, of total length
    dt per step, become n_inner inner steps each: the trajectory is the inner
    integrator's at step (drift weight) x dt / n_inner, operation for operation."""
    dims = (4, 4, 4, 4)
    u = inputs.hot_start(dims, 1)
    p = inputs.gaussian_momenta(dims, 1)
    gs = it.GaugeSystem(6.0)
    dt = 0.25
    u1, p1, _, _ = it.nested_trajectory(gs, ZeroSystem(), gs, it.Integrator(outer), it.Integrator(inner),
                                        n_inner, u, p, dt)
    # every drift of these outer integrators has the same weight
    q = [op[1] for op in it.Integrator(outer).steps if op[0] == "Q"]
    assert len(set(q)) == 1
    u2, p2, _, _ = it.trajectory(gs, it.Integrator(inner), u, p, q[0] * dt / n_inner, 1.0)
    assert np.array_equal(u1, u2) and np.array_equal(p1, p2)


def test_one_level_leapfrog_split_equals_total_force_leapfrog():
    """Outer = inner = leapfrog with one inner step: the fermion and gauge
    half kicks act at the same links, so the step is leapfrog on S_G + S_F."""
    dims = (2, 2, 2, 4)
    u, phi, p = _fermion_case(dims)
    total = fe.FermionSystem(5.6, KAPPA, phi, tol=1e-14)
    outer = fe.PseudofermionPart(KAPPA, phi, tol=1e-14)
    lf = it.Integrator("leapfrog")
    u1, p1, h0, h1 = it.nested_trajectory(total, outer, total.gauge, lf, lf, 1, u, p, 0.25)
    u2, p2, g0, g1 = it.trajectory(total, lf, u, p, 0.25)
    assert np.max(np.abs(u1 - u2)) < 1e-12
    assert np.max(np.abs(p1 - p2)) < 1e-11
    assert abs((h1 - h0) - (g1 - g0)) < 1e-10


@pytest.mark.slow
def test_nested_orders():
    """Outer force-gradient over an inner force-gradient keeps dH ~ dt^4;
    outer Omelyan over inner Omelyan dt^2 (two inner steps per drift).  At
    dt = 1/4 the outer and inner errors of the FG pair nearly cancel on this
    lattice, so the fit starts at 1/8."""
    dims = (2, 2, 2, 4)
    u, phi, p = _fermion_case(dims)
    dts = [1 / 8, 1 / 16, 1 / 32]
    slopes = {}
    for name in ("omelyan", "fg"):
        dh = []
        for dt in dts:
            total = fe.FermionSystem(5.6, KAPPA, phi, tol=1e-14)
            outer = fe.PseudofermionPart(KAPPA, phi, tol=1e-14)
            integ = it.Integrator(name)
            _, _, h0, h1 = it.nested_trajectory(total, outer, total.gauge, integ, integ, 2, u, p, dt)
            dh.append(abs(h1 - h0))
        slopes[name] = np.polyfit(np.log(dts), np.log(dh), 1)[0]
    assert 1.7 < slopes["omelyan"] < 2.4, slopes
    assert 3.5 < slopes["fg"] < 4.6, slopes


def test_nested_trajectory_is_reversible():
    dims = (2, 2, 2, 4)
    u, phi, p = _fermion_case(dims, 5)
    total = fe.FermionSystem(5.6, KAPPA, phi, tol=1e-14)
    outer = fe.PseudofermionPart(KAPPA, phi, tol=1e-14)
    fg, om = it.Integrator("fg"), it.Integrator("omelyan")
    u1, p1, _, _ = it.nested_trajectory(total, outer, total.gauge, fg, om, 2, u, p, 0.25)
    u2, p2, _, _ = it.nested_trajectory(total, outer, total.gauge, fg, om, 2, u1, -p1, 0.25)
    assert np.max(np.abs(u2 - u)) < 1e-11
    assert np.max(np.abs(-p2 - p)) < 1e-10


def test_outer_force_gradient_uses_the_outer_force_only():
    """The outer FG kick displaces along and kicks with the fermion force:
    per outer FG step with merged outer kicks the fermion force is evaluated
    three times (four unmerged) whatever the inner integrator does."""
    dims = (2, 2, 2, 2)
    u, phi, p = _fermion_case(dims)
    total = fe.FermionSystem(5.6, KAPPA, phi)
    outer = fe.PseudofermionPart(KAPPA, phi)
    it.nested_md_step(outer, total.gauge, it.Integrator("fg"), it.Integrator("omelyan"), 3, u, p, 0.1)
    assert outer.n_force == 4
    assert total.gauge.n_force == 2 * 3 * 3   # two drifts x three Omelyan steps x three kicks
