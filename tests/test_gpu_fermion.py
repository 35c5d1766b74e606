"""GPU parity of the Wilson-fermion path (Dslash, CG, pseudofermion force,
heat bath, fermion HMC) against the FP64 oracle, through the C ABI.

Tolerances:
* FP64 operator applications: normwise relative 1e-13.
* Solves: the FP64 true residual must meet cg_tol (checked by the library and
  here); solutions agree with the oracle to cg_tol times a condition factor.
* Forces and MD steps use cg_tol = 1e-12 on both sides, so they agree to
  ~1e-10 relative (the difference of two solves at that tolerance).
"""

import numpy as np
import pytest

from oracle import fermion as fe, gauge, integrators as it
from paper_0910_2950_gb300 import inputs

pytestmark = pytest.mark.gpu

BETA, KAPPA = 5.6, 0.12


@pytest.fixture(scope="module")
def fgmod():
    from paper_0910_2950_gb300 import build, fg
    build.build()
    fg.load()
    return fg


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _rand_even(dims, seed):
    g = inputs.make_rng(seed)
    v = inputs.volume(dims)
    return g.standard_normal((v // 2, 4, 3)) + 1j * g.standard_normal((v // 2, 4, 3))


DIMS = [(4, 4, 4, 4), (6, 4, 2, 6), (2, 2, 2, 4), (8, 4, 4, 8)]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("dagger", [False, True])
@pytest.mark.parametrize("link_reals", [18, 12])
def test_apply_mhat_fp64(fgmod, dims, dagger, link_reals):
    u = inputs.hot_start(dims, 2)
    psi = _rand_even(dims, 3)
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, link_reals=link_reals) as lat:
        lat.set_gauge(u)
        out = lat.apply_mhat(psi, dagger=dagger)
    full = inputs.unpack_even(psi, dims)
    ref = (fe.mhat_dag if dagger else fe.mhat)(u, KAPPA, full)
    assert _rel(out, inputs.pack_even(ref, dims)) < 1e-13


def test_apply_mhat_fp32_links_in_fp64_arithmetic(fgmod):
    dims = (6, 4, 2, 6)
    u = inputs.hot_start(dims, 2)
    u32 = u.astype(np.complex64).astype(np.complex128)
    psi = _rand_even(dims, 4)
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, precision="fp32") as lat:
        lat.set_gauge(u)
        out = lat.apply_mhat(psi)
    ref = inputs.pack_even(fe.mhat(u32, KAPPA, inputs.unpack_even(psi, dims)), dims)
    assert _rel(out, ref) < 1e-13


_INNER_CACHE = {}


def _inner_case(dims):
    """Links, an even spinor and the oracle's Mhat / Mhat^dag of it, with the
    links and spinor also rounded to FP32 (what the FP32 inner operator
    receives)."""
    if dims not in _INNER_CACHE:
        u = inputs.hot_start(dims, 31)
        psi = _rand_even(dims, 32)
        u32 = u.astype(np.complex64).astype(np.complex128)
        psi32 = psi.astype(np.complex64).astype(np.complex128)
        full, full32 = inputs.unpack_even(psi, dims), inputs.unpack_even(psi32, dims)
        ref = {d: inputs.pack_even((fe.mhat_dag if d else fe.mhat)(u, KAPPA, full), dims) for d in (0, 1)}
        ref32 = {d: inputs.pack_even((fe.mhat_dag if d else fe.mhat)(u32, KAPPA, full32), dims) for d in (0, 1)}
        _INNER_CACHE[dims] = (u, psi, ref, ref32)
    return _INNER_CACHE[dims]


INNER_DIMS = [(6, 4, 2, 6), (4, 4, 4, 4), (16, 16, 16, 32), (24, 24, 24, 48)]


@pytest.mark.parametrize("dims", INNER_DIMS)
@pytest.mark.parametrize("link_reals", [18, 12])
@pytest.mark.parametrize("dagger", [0, 1])
def test_inner_dslash_fp32_element_by_element(fgmod, dims, link_reals, dagger):
    """The FP32 operator of the inner CG iterations (two Dslash launches in
    FP32 on FP32 spinors) against the oracle's Mhat on the same FP32-rounded
    links and input: only the arithmetic's rounding differs, ~1e-7 per term
    over the ~60 terms of a site (bound 2e-6 of the largest entry)."""
    u, psi, ref, ref32 = _inner_case(dims)
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, precision="fp32", link_reals=link_reals) as lat:
        lat.set_gauge(u)
        out = lat.apply_mhat_inner(psi, dagger=bool(dagger))
    assert _rel(out, ref32[dagger]) < 2e-6
    # and against the exact operator on the unrounded inputs
    assert _rel(out, ref[dagger]) < 5e-6


@pytest.mark.parametrize("dims", INNER_DIMS)
@pytest.mark.parametrize("link_reals", [18, 12])
@pytest.mark.parametrize("dagger", [0, 1])
def test_inner_dslash_half_element_by_element(fgmod, dims, link_reals, dagger):
    """The half-precision inner operator (FG_FP32_FP16CG: half links, half
    spinors scaled to unit rms, FP32 arithmetic) against the oracle: half
    precision keeps 11 significant bits (unit roundoff 4.9e-4) in the links,
    the input and the intermediate vector, bound 5e-3 of the largest entry;
    a defect in a hop would show at O(1)."""
    u, psi, ref, _ = _inner_case(dims)
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, precision="fp32_fp16cg", link_reals=link_reals) as lat:
        lat.set_gauge(u)
        out = lat.apply_mhat_inner(psi, dagger=bool(dagger))
    err = _rel(out, ref[dagger])
    assert 1e-5 < err < 5e-3, err    # half-precision rounding is visible, and bounded


@pytest.mark.parametrize("dims", INNER_DIMS)
@pytest.mark.parametrize("link_reals", [18, 12])
@pytest.mark.parametrize("dagger", [0, 1])
def test_inner_dslash_bf16_element_by_element(fgmod, dims, link_reals, dagger):
    """The bfloat16 inner operator (FG_FP32_BF16CG: bfloat16 links and
    spinors scaled to unit rms, FP32 arithmetic) against the oracle:
    bfloat16 keeps 8 significant bits (unit roundoff 3.9e-3) in the links,
    the input and the intermediate vector, bound 4e-2 of the largest entry
    (the half-precision test's 10 units of roundoff); its error lies above
    the half-precision operator's on the same input, as 3 fewer bits give."""
    u, psi, ref, _ = _inner_case(dims)
    out = {}
    for prec in ("fp32_bf16cg", "fp32_fp16cg"):
        with fgmod.Lattice(dims, BETA, kappa=KAPPA, precision=prec, link_reals=link_reals) as lat:
            lat.set_gauge(u)
            out[prec] = lat.apply_mhat_inner(psi, dagger=bool(dagger))
    err = _rel(out["fp32_bf16cg"], ref[dagger])
    err_half = _rel(out["fp32_fp16cg"], ref[dagger])
    assert 1e-4 < err < 4e-2, err
    assert err > 2 * err_half, (err, err_half)


@pytest.mark.parametrize("dims,same_as", [((16, 16, 16, 32), "fp32"), ((24, 24, 24, 48), "fp32_fp16cg")])
def test_autocg_follows_the_l2_size(fgmod, dims, same_as):
    """FG_FP32_AUTOCG runs the FP32 inner solver while its working set fits
    the L2 cache (16^3 x 32: ~75 MB) and the half-precision one above it
    (24^3 x 48: ~380 MB): the solutions are those of the chosen mode, bit
    for bit."""
    u, psi, _, _ = _inner_case(dims)
    out = {}
    for prec in ("fp32_autocg", same_as):
        with fgmod.Lattice(dims, BETA, kappa=KAPPA, precision=prec) as lat:
            lat.set_gauge(u)
            out[prec] = lat.cg_solve(psi)
    assert np.array_equal(out["fp32_autocg"][0], out[same_as][0])
    assert out["fp32_autocg"][1]["iterations"] == out[same_as][1]["iterations"]


def test_inner_dslash_fp64_is_apply_mhat(fgmod):
    dims = (6, 4, 2, 6)
    u, psi, ref, _ = _inner_case(dims)
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, precision="fp64") as lat:
        lat.set_gauge(u)
        out = lat.apply_mhat_inner(psi)
        assert np.array_equal(out, lat.apply_mhat(psi))
    assert _rel(out, ref[0]) < 1e-13


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_fp16cg", "fp32_bf16cg"])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 6)])
def test_cg_solve(fgmod, precision, dims):
    u = inputs.hot_start(dims, 5)
    b = _rand_even(dims, 6)
    tol = 1e-10
    with fgmod.Lattice(dims, BETA, kappa=0.158, precision=precision, cg_tol=tol) as lat:
        lat.set_gauge(u)
        x, info = lat.cg_solve(b)
    assert info["true_residual"] <= tol
    assert info["iterations"] > 0
    if precision != "fp64":
        assert info["reliable_updates"] >= 1
    uu = u.astype(np.complex64).astype(np.complex128) if precision != "fp64" else u
    full_x = inputs.unpack_even(x, dims)
    res = inputs.unpack_even(b, dims) - fe.mdagm(uu, 0.158, full_x)
    assert np.linalg.norm(res) <= 1.01 * tol * np.linalg.norm(b)
    xo, _ = fe.cg(uu, 0.158, inputs.unpack_even(b, dims), tol=1e-13)
    assert _rel(x, inputs.pack_even(xo, dims)) < 1e-7


def test_fp32_reliable_updates_in_double_float(fgmod):
    """The FP32 solver's intermediate reliable updates apply Mhat^dag Mhat in
    double-float arithmetic; only the update that certifies convergence uses
    the FP64 Dslash, and the certified residual holds against the oracle."""
    dims = (8, 8, 8, 8)
    u = inputs.hot_start(dims, 7)
    b = _rand_even(dims, 9)
    tol = 1e-10
    with fgmod.Lattice(dims, BETA, kappa=0.158, precision="fp32", cg_tol=tol) as lat:
        lat.set_gauge(u)
        lat.timing(True)
        lat.timing_reset()
        x, info = lat.cg_solve(b)
        _, n_df = lat.kernel_time("dslash_df")
        _, n64 = lat.kernel_time("dslash_fp64")
        _, n32 = lat.kernel_time("dslash")
    assert info["reliable_updates"] >= 3
    # one certifying FP64 update: the double-float residuals were right, so the
    # FP64 check confirmed convergence at the first attempt
    assert n64 == 4 and n_df > 0
    assert n_df + n64 == 4 * info["reliable_updates"]
    assert n32 >= 4 * info["iterations"]
    # and the iteration count matches the all-FP64 solver's
    with fgmod.Lattice(dims, BETA, kappa=0.158, precision="fp64", cg_tol=tol) as lat64:
        lat64.set_gauge(u.astype(np.complex64).astype(np.complex128))
        _, info64 = lat64.cg_solve(b)
    assert abs(info["iterations"] - info64["iterations"]) <= 0.1 * info64["iterations"] + 2
    uu = u.astype(np.complex64).astype(np.complex128)
    res = inputs.unpack_even(b, dims) - fe.mdagm(uu, 0.158, inputs.unpack_even(x, dims))
    assert np.linalg.norm(res) <= 1.01 * tol * np.linalg.norm(b)


def test_cg_matches_dense_solve_2x2x2x2(fgmod):
    dims = (2, 2, 2, 2)
    u = inputs.hot_start(dims, 3)
    b = _rand_even(dims, 8)
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, cg_tol=1e-13) as lat:
        lat.set_gauge(u)
        x, info = lat.cg_solve(b)
    # dense M^dagger M on the 96 even-site unknowns, built column by column
    n = 96
    cols = []
    for j in range(n):
        e = np.zeros(n, dtype=np.complex128)
        e[j] = 1
        cols.append(inputs.pack_even(fe.mdagm(u, KAPPA, inputs.unpack_even(e.reshape(8, 4, 3), dims)),
                                     dims).reshape(-1))
    mat = np.array(cols).T
    xd = np.linalg.solve(mat, b.reshape(-1))
    assert _rel(x.reshape(-1), xd) < 1e-11


def test_zero_rhs_and_state_errors(fgmod):
    dims = (4, 4, 4, 4)
    with fgmod.Lattice(dims, BETA, kappa=KAPPA) as lat:
        x, info = lat.cg_solve(np.zeros((128, 4, 3), np.complex128))
        assert np.all(x == 0) and info["iterations"] == 0
    with fgmod.Lattice(dims, BETA) as lat:
        with pytest.raises(fgmod.FgError) as e:
            lat.apply_mhat(np.zeros((128, 4, 3), np.complex128))
        assert e.value.status == fgmod.FG_ESTATE


def test_cg_iteration_cap_reports_enoconv(fgmod):
    dims = (4, 4, 4, 4)
    with fgmod.Lattice(dims, BETA, kappa=0.158, cg_maxiter=3, cg_tol=1e-12) as lat:
        lat.set_gauge(inputs.hot_start(dims, 1))
        with pytest.raises(fgmod.FgError) as e:
            lat.cg_solve(_rand_even(dims, 1))
        assert e.value.status == fgmod.FG_ENOCONV
        # the handle stays usable
        x, info = lat.apply_mhat(_rand_even(dims, 2)), None
        assert np.isfinite(x).all()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_heatbath_action(fgmod, precision):
    dims = (6, 4, 2, 6)
    u = inputs.hot_start(dims, 4)
    chi = inputs.gaussian_spinor_even(dims, 5)
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, precision=precision, cg_tol_action=1e-12) as lat:
        lat.set_gauge(u)
        lat.set_pseudofermion(chi)
        sg, sf, t = lat.action()
    assert abs(sf - np.vdot(chi, chi).real) < 1e-9 * sf
    assert abs(sg - gauge.wilson_action(u, BETA)) < (1e-12 if precision == "fp64" else 1e-5) * sg


@pytest.mark.parametrize("link_reals", [18, 12])
def test_total_force_fp64(fgmod, link_reals):
    dims = (6, 4, 2, 6)
    u = inputs.hot_start(dims, 6)
    chi = inputs.gaussian_spinor_even(dims, 7)
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, cg_tol=1e-13, link_reals=link_reals) as lat:
        lat.set_gauge(u)
        lat.set_pseudofermion(chi)
        f = lat.force()
    phi = fe.heatbath_phi(u, KAPPA, inputs.unpack_even(chi, dims))
    ref = gauge.gauge_force(u, BETA) + fe.fermion_force(u, KAPPA, phi, tol=1e-13)
    assert _rel(f, ref) < 1e-10


def test_fermion_force_fp32(fgmod):
    dims = (6, 4, 2, 6)
    u = inputs.hot_start(dims, 6)
    chi = inputs.gaussian_spinor_even(dims, 7)
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, precision="fp32", cg_tol=1e-10) as lat:
        lat.set_gauge(u)
        lat.set_pseudofermion(chi)
        f = lat.force()
    phi = fe.heatbath_phi(u, KAPPA, inputs.unpack_even(chi, dims))
    ref = gauge.gauge_force(u, BETA) + fe.fermion_force(u, KAPPA, phi, tol=1e-12)
    assert _rel(f, ref) < 5e-6


@pytest.mark.parametrize("name", ["fg", "omelyan", "leapfrog"])
def test_fermion_md_step_fp64(fgmod, name):
    dims = (4, 4, 2, 4)
    u = inputs.hot_start(dims, 8)
    p = inputs.gaussian_momenta(dims, 9)
    chi = inputs.gaussian_spinor_even(dims, 10)
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, cg_tol=1e-13) as lat:
        lat.set_gauge(u)
        lat.set_pseudofermion(chi)
        lat.set_momenta(p)
        lat.md_step(name, 0.1)
        ug, pg = lat.get_gauge(), lat.get_momenta()
    phi = fe.heatbath_phi(u, KAPPA, inputs.unpack_even(chi, dims))
    system = fe.FermionSystem(BETA, KAPPA, phi, tol=1e-13)
    uo, po = it.md_step(system, it.Integrator(name), u, p, 0.1)
    assert _rel(ug, uo) < 1e-11
    assert _rel(pg, po) < 1e-10


@pytest.fixture(scope="module")
def fermion_traj_oracle():
    dims = (4, 4, 2, 4)
    u = inputs.hot_start(dims, 11)
    p = inputs.gaussian_momenta(dims, 12)
    chi = inputs.gaussian_spinor_even(dims, 13)
    phi = fe.heatbath_phi(u, KAPPA, inputs.unpack_even(chi, dims))
    out = {}
    for dt in (0.25, 0.125):
        system = fe.FermionSystem(BETA, KAPPA, phi, tol=1e-13)
        u1, p1, h0, h1 = it.trajectory(system, it.Integrator("fg"), u, p, dt, 1.0)
        out[dt] = (h1 - h0, h0, u1)
    return dims, u, p, chi, out


@pytest.mark.parametrize("dt", [0.25, 0.125])
def test_fermion_fg_trajectory_dh_fp64(fgmod, fermion_traj_oracle, dt):
    dims, u, p, chi, ref = fermion_traj_oracle
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, cg_tol=1e-13, cg_tol_action=1e-13) as lat:
        lat.set_gauge(u)
        lat.set_pseudofermion(chi)
        lat.set_momenta(p)
        r = lat.trajectory("fg", dt, 1.0, refresh=False, u_accept=0.0)
        ug = lat.get_gauge()
    dh_o, h0_o, u1_o = ref[dt]
    assert abs(r["dH"] - dh_o) < 1e-6, (r["dH"], dh_o)
    assert abs(r["H0"] - h0_o) < 1e-9 * abs(h0_o)
    assert _rel(ug, u1_o) < 1e-10
    n = r["n_steps"]
    assert r["n_force"] == 3 * n + 1
    # one solve per force evaluation plus the action solve at the end; S_F at
    # the start is chi^dagger chi from the heat bath
    assert r["n_solves"] == 3 * n + 1 + 1
    assert r["cg_iters"] > 0


@pytest.mark.parametrize("precision", ["fp32", "fp32_fp16cg", "fp32_bf16cg"])
def test_fermion_fg_trajectory_fp32_mixed(fgmod, fermion_traj_oracle, precision):
    dims, u, p, chi, ref = fermion_traj_oracle
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, precision=precision, cg_tol=1e-10,
                       cg_tol_action=1e-12) as lat:
        lat.set_gauge(u)
        lat.set_pseudofermion(chi)
        lat.set_momenta(p)
        r = lat.trajectory("fg", 0.125, 1.0, refresh=False, u_accept=0.0)
    # FP32 links and forces: dH moves by ~1e-7 relative to the O(10^3) terms of H
    assert abs(r["dH"] - ref[0.125][0]) < 5e-4, (r["dH"], ref[0.125][0])


def test_device_pseudofermion_refresh(fgmod):
    dims = (8, 8, 4, 8)
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, seed=77) as lat:
        lat.set_gauge(inputs.hot_start(dims, 1))
        lat.refresh_pseudofermion()
        sg, sf, t = lat.action()
    # S_F = chi^dagger chi ~ 12 V/2 (one unit per complex component)
    v = inputs.volume(dims)
    assert abs(sf / (12 * v / 2) - 1) < 5 * np.sqrt(1 / (12 * v / 2))


# ---------------------------------------------------------------- two-level integrator
NESTED = [("fg", "omelyan", 2), ("omelyan", "fg", 1), ("fg", "fg", 3), ("leapfrog", "qpq", 2)]


@pytest.fixture(scope="module")
def nested_oracle():
    dims = (4, 4, 2, 4)
    u = inputs.hot_start(dims, 21)
    p = inputs.gaussian_momenta(dims, 22)
    chi = inputs.gaussian_spinor_even(dims, 23)
    phi = fe.heatbath_phi(u, KAPPA, inputs.unpack_even(chi, dims))
    out = {}
    for outer, inner, m in NESTED:
        total = fe.FermionSystem(BETA, KAPPA, phi, tol=1e-13)
        outer_sys = fe.PseudofermionPart(KAPPA, phi, tol=1e-13)
        u1, p1, h0, h1 = it.nested_trajectory(total, outer_sys, total.gauge, it.Integrator(outer),
                                              it.Integrator(inner), m, u, p, 0.25, 0.5)
        out[(outer, inner, m)] = (h1 - h0, h0, u1, p1, outer_sys.n_force)
    return dims, u, p, chi, out


@pytest.mark.parametrize("outer,inner,m", NESTED)
def test_nested_trajectory_fp64_matches_oracle(fgmod, nested_oracle, outer, inner, m):
    dims, u, p, chi, ref = nested_oracle
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, cg_tol=1e-13, cg_tol_action=1e-13) as lat:
        lat.set_gauge(u)
        lat.set_pseudofermion(chi)
        lat.set_momenta(p)
        r = lat.trajectory_nested(outer, inner, m, 0.25, 0.5, refresh=False, u_accept=0.0)
        ug = lat.get_gauge()
        pg = lat.get_momenta()
    dh_o, h0_o, u1_o, p1_o, n_outer = ref[(outer, inner, m)]
    assert abs(r["H0"] - h0_o) < 1e-9 * abs(h0_o)
    assert abs(r["dH"] - dh_o) < 1e-6, (r["dH"], dh_o)
    assert _rel(ug, u1_o) < 1e-10
    assert _rel(pg, p1_o) < 1e-9
    # outer kicks of neighbouring steps share one solve; the outer FG kick
    # takes two; plus the action solve at the end
    n_steps = 2
    per_step = {"fg": 3, "omelyan": 2, "leapfrog": 1}[outer]
    assert r["n_solves"] == per_step * n_steps + 1 + 1


def test_nested_pure_gauge_is_the_inner_integrator(fgmod):
    """Without fermions the outer kicks vanish: the nested trajectory is the
    inner integrator's at step (drift weight) x dt / n_inner, op for op."""
    dims = (6, 4, 4, 6)
    u = inputs.hot_start(dims, 3)
    p = inputs.gaussian_momenta(dims, 4)
    res = []
    for nested in (True, False):
        with fgmod.Lattice(dims, 6.0) as lat:
            lat.set_gauge(u)
            lat.set_momenta(p)
            if nested:
                r = lat.trajectory_nested("leapfrog", "omelyan", 3, 0.25, 1.0, refresh=False, u_accept=0.0)
            else:
                r = lat.trajectory("omelyan", 0.25 / 3, 1.0, refresh=False, u_accept=0.0)
            res.append((r["dH"], lat.get_gauge(), lat.get_momenta()))
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][2], res[1][2])


def test_nested_fp32_mixed(fgmod, nested_oracle):
    dims, u, p, chi, ref = nested_oracle
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, precision="fp32", cg_tol=1e-10, cg_tol_action=1e-11) as lat:
        lat.set_gauge(u)
        lat.set_pseudofermion(chi)
        lat.set_momenta(p)
        r = lat.trajectory_nested("fg", "omelyan", 2, 0.25, 0.5, refresh=False, u_accept=0.0)
    assert abs(r["dH"] - ref[("fg", "omelyan", 2)][0]) < 2e-3


# ---------------------------------------------------------------- closed-form force gradient
def test_analytic_fg_step_pure_gauge_fp64_matches_oracle(fgmod):
    dims = (6, 4, 2, 4)
    u = inputs.hot_start(dims, 31)
    p = inputs.gaussian_momenta(dims, 32)
    u1, p1 = it.md_step(it.GaugeSystem(6.0), it.Integrator("fg_analytic"), u, p, 0.2)
    with fgmod.Lattice(dims, 6.0) as lat:
        lat.set_gauge(u)
        lat.set_momenta(p)
        lat.md_step("fg_analytic", 0.2)
        ug, pg = lat.get_gauge(), lat.get_momenta()
    assert _rel(ug, u1) < 1e-12
    assert _rel(pg, p1) < 1e-12
    # and it is not the displaced-force step
    u2, p2 = it.md_step(it.GaugeSystem(6.0), it.Integrator("fg"), u, p, 0.2)
    assert _rel(pg, p2) > 1e-8


@pytest.mark.parametrize("link_reals", [18, 12])
def test_analytic_fg_step_fermions_fp64_matches_oracle(fgmod, link_reals):
    dims = (4, 4, 2, 4)
    u = inputs.hot_start(dims, 33)
    p = inputs.gaussian_momenta(dims, 34)
    chi = inputs.gaussian_spinor_even(dims, 35)
    phi = fe.heatbath_phi(u, KAPPA, inputs.unpack_even(chi, dims))
    system = fe.FermionSystem(BETA, KAPPA, phi, tol=1e-14)
    u1, p1 = it.md_step(system, it.Integrator("fg_analytic"), u, p, 0.2)
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, link_reals=link_reals, cg_tol=1e-13,
                       cg_tol_action=1e-13) as lat:
        lat.set_gauge(u)
        lat.set_pseudofermion(chi)
        lat.set_momenta(p)
        lat.md_step("fg_analytic", 0.2)
        ug, pg = lat.get_gauge(), lat.get_momenta()
    assert _rel(ug, u1) < 1e-10
    assert _rel(pg, p1) < 1e-9


def test_analytic_fg_trajectory_fermions(fgmod):
    dims = (4, 4, 2, 4)
    u = inputs.hot_start(dims, 36)
    p = inputs.gaussian_momenta(dims, 37)
    chi = inputs.gaussian_spinor_even(dims, 38)
    phi = fe.heatbath_phi(u, KAPPA, inputs.unpack_even(chi, dims))
    system = fe.FermionSystem(BETA, KAPPA, phi, tol=1e-13)
    _, _, h0, h1 = it.trajectory(system, it.Integrator("fg_analytic"), u, p, 0.25, 1.0)
    res = {}
    for prec in ("fp64", "fp32"):
        with fgmod.Lattice(dims, BETA, kappa=KAPPA, precision=prec, cg_tol=1e-13 if prec == "fp64" else 1e-10,
                           cg_tol_action=1e-13 if prec == "fp64" else 1e-11) as lat:
            lat.set_gauge(u)
            lat.set_pseudofermion(chi)
            lat.set_momenta(p)
            res[prec] = lat.trajectory("fg_analytic", 0.25, 1.0, refresh=False, u_accept=0.0)
    assert abs(res["fp64"]["dH"] - (h1 - h0)) < 1e-6, (res["fp64"]["dH"], h1 - h0)
    assert abs(res["fp32"]["dH"] - (h1 - h0)) < 2e-3
    # section 4: the closed form costs one extra solve per FG kick, as the
    # displaced force does: 3n + 1 force solves plus the action solve
    n = res["fp64"]["n_steps"]
    assert res["fp64"]["n_solves"] == 3 * n + 1 + 1


@pytest.mark.parametrize("outer,inner", [("fg_analytic", "omelyan"), ("fg", "fg_analytic"),
                                         ("fg_analytic", "fg_analytic")])
def test_nested_analytic_fp64_matches_oracle(fgmod, outer, inner):
    dims = (4, 4, 2, 4)
    u = inputs.hot_start(dims, 41)
    p = inputs.gaussian_momenta(dims, 42)
    chi = inputs.gaussian_spinor_even(dims, 43)
    phi = fe.heatbath_phi(u, KAPPA, inputs.unpack_even(chi, dims))
    total = fe.FermionSystem(BETA, KAPPA, phi, tol=1e-13)
    outer_sys = fe.PseudofermionPart(KAPPA, phi, tol=1e-13)
    u1, p1, h0, h1 = it.nested_trajectory(total, outer_sys, total.gauge, it.Integrator(outer), it.Integrator(inner),
                                          2, u, p, 0.25, 0.5)
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, cg_tol=1e-13, cg_tol_action=1e-13) as lat:
        lat.set_gauge(u)
        lat.set_pseudofermion(chi)
        lat.set_momenta(p)
        r = lat.trajectory_nested(outer, inner, 2, 0.25, 0.5, refresh=False, u_accept=0.0)
        ug = lat.get_gauge()
    assert abs(r["dH"] - (h1 - h0)) < 1e-6
    assert _rel(ug, u1) < 1e-10
