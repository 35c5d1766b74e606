"""Pins for oracle.integrators and oracle.toy1d against Table 1 and section 3."""

import json
import math
import os

import numpy as np
import pytest

from oracle import gauge, integrators as it, su3, toy1d
from paper_0910_2950_gb300 import inputs

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table1.json")))
C4, C2 = 4 ** (1 / 3), 2 ** (1 / 3)


def _num(s):
    return float(eval(str(s), {"__builtins__": {}}, {"sqrt": math.sqrt}))


def _cbrt(t):
    return t[0] * C4 + t[1] * C2 + t[2]


def _golden_steps(entry):
    if "steps_cbrt" in entry:
        return [(k, _cbrt(v) / d) for k, v, d in entry["steps_cbrt"]]
    out = []
    for s in entry["steps"]:
        out.append((s[0],) + tuple(_num(x) for x in s[1:]))
    return out


def _golden_shadow(name, q, p, dt):
    entry = GOLDEN["integrators"][name]
    b = toy1d.brackets(q, p)
    h = toy1d.energy(q, p)
    if entry["shadow_order"] == 2:
        return h + dt ** 2 * sum(_num(c) * b[k] for k, c in entry["shadow"].items())
    den = entry["shadow_denominator"]
    coef = ({k: _cbrt(v) for k, v in entry["shadow_cbrt"].items()} if "shadow_cbrt" in entry
            else {k: _num(v) for k, v in entry["shadow"].items()})
    return h + dt ** 4 / den * sum(c * b[k] for k, c in coef.items())


ORACLE_NAME = {"leapfrog": ("leapfrog", None), "qpq": ("qpq", None),
               "omelyan_sixth": ("omelyan", 1 / 6), "omelyan_sqrt3": ("omelyan", (3 - math.sqrt(3)) / 6),
               "campostrini": ("campostrini", None), "fg": ("fg", None)}


@pytest.mark.parametrize("name", sorted(ORACLE_NAME))
def test_sequences_match_table1(name):
    oname, alpha = ORACLE_NAME[name]
    seq = it.sequence(oname) if alpha is None else it.sequence(oname, alpha)
    gold = _golden_steps(GOLDEN["integrators"][name])
    assert [s[0] for s in seq] == [g[0] for g in gold]
    for s, g in zip(seq, gold):
        assert np.allclose(s[1:], g[1:], rtol=1e-14, atol=1e-15)


def _slope(xs, ys):
    return np.polyfit(np.log(xs), np.log(np.abs(ys)), 1)[0]


@pytest.mark.parametrize("name", sorted(ORACLE_NAME))
def test_toy_shadow_hamiltonian_is_conserved(name):
    """The Table 1 shadow Hamiltonian changes by O(dt^(k+3)) per step while H
    changes by O(dt^(k+1)) (k = the integrator's order)."""
    oname, alpha = ORACLE_NAME[name]
    order = GOLDEN["integrators"][name]["shadow_order"]
    # fourth-order residuals reach double rounding below dt ~ 0.02
    dts = np.array([0.1, 0.05, 0.025, 0.0125]) if order == 2 else np.array([0.16, 0.08, 0.04, 0.02])
    dsh, dh = [], []
    for q0, p0 in [(0.7, -0.4), (-1.1, 0.9)]:
        a, b = [], []
        for dt in dts:
            q, p = toy1d.step(oname, q0, p0, dt, alpha)
            a.append(_golden_shadow(name, q, p, dt) - _golden_shadow(name, q0, p0, dt))
            b.append(toy1d.energy(q, p) - toy1d.energy(q0, p0))
        dsh.append(_slope(dts, a))
        dh.append(_slope(dts, b))
    assert min(dsh) > order + 2.3, dsh
    assert min(dsh) - max(dh) > 1.4, (dsh, dh)
    # the toy's own coded shadow agrees with the golden one
    assert np.isclose(toy1d.shadow(oname, 0.3, 0.2, 0.1, alpha), _golden_shadow(name, 0.3, 0.2, 0.1), rtol=1e-14)


def test_pqpqp_general_shadow_coefficients():
    """Section 3's PQPQP(alpha) shadow for alpha values outside Table 1."""
    g = GOLDEN["pqpqp_general"]
    dts = np.array([0.1, 0.05, 0.025, 0.0125])
    for alpha in [0.1932, 0.3, 0.5]:
        def sh(q, p, dt):
            b = toy1d.brackets(q, p)
            a = alpha
            return toy1d.energy(q, p) + dt ** 2 * (
                eval(g["SST"], {}, {"a": a}) * b["SST"] + eval(g["TST"], {}, {"a": a}) * b["TST"])
        res = []
        for dt in dts:
            q, p = toy1d.step("omelyan", 0.7, -0.4, dt, alpha)
            res.append(sh(q, p, dt) - sh(0.7, -0.4, dt))
        assert _slope(dts, res) > 4.6


def test_toy_fg_sign_is_pinned():
    """A flipped sign of the {S,{S,T}} term degrades FG to second order."""
    dts = np.array([0.1, 0.05, 0.025])

    def traj(dt, sign):
        q, p = 0.7, -0.4
        for _ in range(int(round(1 / dt))):
            p = p - dt / 6 * toy1d.v1(q)
            q = q + dt / 2 * p
            p = p - 2 / 3 * dt * (toy1d.v1(q) - sign * dt * dt / 24 * toy1d.v1(q) * toy1d.v2(q))
            q = q + dt / 2 * p
            p = p - dt / 6 * toy1d.v1(q)
        return toy1d.energy(q, p) - toy1d.energy(0.7, -0.4)
    good = [traj(dt, +1) for dt in dts]
    bad = [traj(dt, -1) for dt in dts]
    assert _slope(dts, good) > 3.6
    assert _slope(dts, bad) < 2.5
    # the oracle's toy step is the good one
    q, p = toy1d.step("fg", 0.7, -0.4, 0.05)
    p2 = -0.4 - 0.05 / 6 * toy1d.v1(0.7)
    assert np.isfinite(q) and np.isfinite(p) and np.isfinite(p2)


DIMS4 = (4, 4, 4, 4)
DTS = [1 / 4, 1 / 8, 1 / 16, 1 / 32]


@pytest.fixture(scope="module")
def hot4():
    return inputs.hot_start(DIMS4, 1)


@pytest.mark.parametrize("name,lo,hi", [("leapfrog", 1.8, 2.2), ("omelyan", 1.8, 2.2), ("fg", 3.7, 4.4)])
def test_lattice_dh_slopes(hot4, name, lo, hi):
    """dH = k dt^n with n = 2 (PQP, PQPQP) and n = 4 (force gradient), section 1."""
    system = it.GaugeSystem(6.0)
    integ = it.Integrator(name)
    rms = []
    for dt in DTS:
        vals = []
        for seed in (1, 2):
            p = inputs.gaussian_momenta(DIMS4, seed)
            _, _, h0, h1 = it.trajectory(system, integ, hot4, p, dt, 1.0)
            vals.append(h1 - h0)
        rms.append(np.sqrt(np.mean(np.square(vals))))
    s = _slope(DTS, rms)
    assert lo < s < hi, (name, s, rms)


def test_fg_counts_three_forces_per_step(hot4):
    system = it.GaugeSystem(6.0)
    p = inputs.gaussian_momenta(DIMS4, 1)
    it.md_step(system, it.Integrator("fg"), hot4, p, 0.1)
    assert system.n_force == 4          # 1/6 kick, F for the displacement, F(U'), 1/6 kick


@pytest.mark.parametrize("name", ["leapfrog", "omelyan", "fg", "campostrini"])
def test_reversibility(hot4, name):
    system = it.GaugeSystem(6.0)
    integ = it.Integrator(name)
    p = inputs.gaussian_momenta(DIMS4, 3)
    u1, p1, _, _ = it.trajectory(system, integ, hot4, p, 1 / 8, 1.0)
    u2, p2, _, _ = it.trajectory(system, integ, u1, -p1, 1 / 8, 1.0)
    assert np.max(np.abs(u2 - hot4)) < 1e-11
    assert np.max(np.abs(p2 + p)) < 1e-10


def _sst_tst(system, u, p, h=1e-4):
    """SST = sum (F^a)^2 (section 4) and TST = -d^2 S(exp(i s P) U)/ds^2 at s = 0.

    dS/ds along the drift equals sum_a F^a(U_s) p^a, so TST is minus its
    central difference.
    """
    f = system.force(u)
    sst = float(np.sum(f * f))
    pm = su3.alg_to_mat(p)
    fp = system.force(su3.expi(pm, h) @ u)
    fm = system.force(su3.expi(pm, -h) @ u)
    tst = -float(np.sum((fp - fm) * p)) / (2 * h)
    return sst, tst


@pytest.mark.parametrize("alpha", [0.1932, 1 / 6, (3 - math.sqrt(3)) / 6, 0.5])
def test_lattice_pqpqp_shadow(hot4, alpha):
    """Section 3: H + dt^2 [(6a^2-6a+1)/12 SST + (1-6a)/24 TST] is conserved to
    O(dt^5) per step on the SU(3) lattice, while H moves at O(dt^3)."""
    system = it.GaugeSystem(6.0)
    integ = it.Integrator("omelyan", alpha=alpha)
    p0 = inputs.gaussian_momenta(DIMS4, 5)
    u0 = hot4
    s0, t0 = _sst_tst(system, u0, p0)
    h0 = system.action(u0) + gauge.kinetic(p0)
    dts = np.array([0.02, 0.01, 0.005])
    dsh, dh = [], []
    for dt in dts:
        u1, p1 = it.md_step(system, integ, u0, p0, dt)
        s1, t1 = _sst_tst(system, u1, p1)
        h1 = system.action(u1) + gauge.kinetic(p1)
        c1, c2 = (6 * alpha ** 2 - 6 * alpha + 1) / 12, (1 - 6 * alpha) / 24
        dh.append(h1 - h0)
        dsh.append((h1 - h0) + dt * dt * (c1 * (s1 - s0) + c2 * (t1 - t0)))
    assert _slope(dts, dh) < 3.6
    assert _slope(dts, dsh) > max(4.4, _slope(dts, dh) + 1.2), (dsh, dh)


def test_displaced_fg_agrees_with_exact_fg(hot4):
    """The displaced-force surrogate differs from the finite-difference force
    gradient by O(dt^5) in one step."""
    system = it.GaugeSystem(6.0)
    p0 = inputs.gaussian_momenta(DIMS4, 6)
    dts = np.array([0.1, 0.05, 0.025])
    diffs = []
    for dt in dts:
        ud, pd = it.md_step(system, it.Integrator("fg"), hot4, p0, dt)
        ue, pe = it.md_step(system, it.Integrator("fg", fg_mode="exact", fd_eps=1e-4), hot4, p0, dt)
        diffs.append(np.max(np.abs(pd - pe)))
    assert 4.6 < _slope(dts, diffs) < 5.4, diffs


def test_metropolis():
    assert it.metropolis(-0.5, 0.999)
    assert it.metropolis(0.1, math.exp(-0.1) - 1e-9)
    assert not it.metropolis(0.1, math.exp(-0.1) + 1e-9)
    assert not it.metropolis(50.0, 1e-20)   # exp(-50) ~ 1.9e-22


@pytest.mark.slow
def test_creutz_equality():
    """<exp(-dH)> = 1 in equilibrium for a reversible, area-preserving integrator."""
    dims = (2, 2, 2, 2)
    system = it.GaugeSystem(2.0)
    integ = it.Integrator("leapfrog")
    rng = inputs.make_rng(99)
    u = inputs.hot_start(dims, 4)
    vals = []
    for k in range(700):
        p = rng.standard_normal(inputs.site_shape(dims) + (4, 8))
        u, dh, _ = it.hmc_trajectory(system, integ, u, p, 0.25, 1.0, rng.random())
        if k >= 100:
            vals.append(math.exp(-dh))
    vals = np.array(vals)
    err = vals.std() / math.sqrt(len(vals)) * 3   # autocorrelation allowance
    assert abs(vals.mean() - 1.0) < 4 * err + 1e-3, (vals.mean(), err)
