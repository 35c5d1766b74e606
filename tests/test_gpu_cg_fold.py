"""The folded CG iteration (four launches, the vector updates inside the
Dslash launches) against the oracle and against the six-launch iteration.

The solver of section 4's even-odd system Mhat^dagger Mhat x = b forms the
next search direction p' = (r - alpha Ap) + beta p on the fly in the launch
that applies D_oe to it, and takes beta from the expansion
|r - alpha Ap|^2 = rr - 2 alpha Re <r, Ap> + alpha^2 |Ap|^2.  Checked here:
* solutions against the oracle's FP64 CG (normwise relative 1e-7 at cg_tol
  1e-10) and the certified residual against the oracle's operator on the
  links the solver holds, from ragged lattices (one partial block) up;
* iteration counts against the six-launch iteration (within 10% + 2);
* the same bits with CUDA-graph batches and with single launches (timing on),
  and on a repeated solve;
* the launch count: four per iteration, no separate vector kernels.
"""

import numpy as np
import pytest

from oracle import fermion as fe
from paper_0910_2950_gb300 import inputs

pytestmark = pytest.mark.gpu

BETA, KAPPA = 5.6, 0.158


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


def _solve(fgmod, monkeypatch, dims, precision, link_reals, u, b, fold, timing=False, repeat=1, tol=1e-10):
    monkeypatch.setenv("FG_CG_FOLD", fold)
    out = []
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, precision=precision, link_reals=link_reals, cg_tol=tol) as lat:
        lat.set_gauge(u)
        held = lat.get_gauge()  # the links the solver works with (FP32 rounding, 12-real rebuild)
        lat.timing(timing)
        for _ in range(repeat):
            lat.timing_reset()
            x, info = lat.cg_solve(b)
            if timing:
                info["n_dslash"] = lat.kernel_time("dslash")[1]
                info["n_blas"] = lat.kernel_time("cg_blas")[1]
            info["links"] = held
            out.append((x, info))
    return out


@pytest.mark.parametrize("dims", [(6, 4, 2, 6), (4, 4, 4, 4), (8, 8, 8, 8), (8, 8, 8, 16)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("link_reals", [18, 12])
def test_folded_cg_matches_the_oracle(fgmod, monkeypatch, dims, precision, link_reals):
    u = inputs.hot_start(dims, 11)
    b = _rand_even(dims, 12)
    tol = 1e-10
    (x, info), (x2, info2) = _solve(fgmod, monkeypatch, dims, precision, link_reals, u, b, "1", repeat=2)
    assert info["true_residual"] <= tol and info["iterations"] > 0
    # deterministic: a repeated solve gives the same bits
    assert np.array_equal(x, x2) and info["iterations"] == info2["iterations"]
    res = inputs.unpack_even(b, dims) - fe.mdagm(info["links"], KAPPA, inputs.unpack_even(x, dims))
    assert np.linalg.norm(res) <= 1.01 * tol * np.linalg.norm(b)
    if inputs.volume(dims) <= 4096:
        xo, _ = fe.cg(info["links"], KAPPA, inputs.unpack_even(b, dims), tol=1e-13)
        assert _rel(x, inputs.pack_even(xo, dims)) < 1e-7
    # the six-launch iteration on the same system
    [(xs, infs)] = _solve(fgmod, monkeypatch, dims, precision, link_reals, u, b, "0")
    assert abs(info["iterations"] - infs["iterations"]) <= 0.1 * infs["iterations"] + 2
    assert _rel(x, xs) < 1e-7


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_folded_cg_graphs_and_single_launches_agree(fgmod, monkeypatch, precision):
    """CUDA-graph batches of 2, 4 or 8 iterations (timing off) and one launch
    at a time (timing on) run the same kernels in the same order: the same
    bits.  With timing on, every iteration is four Dslash-class launches
    and the vector kernels appear only in the setup and the reliable
    updates."""
    dims = (8, 8, 8, 16)
    u = inputs.hot_start(dims, 13)
    b = _rand_even(dims, 14)
    [(xg, ig)] = _solve(fgmod, monkeypatch, dims, precision, 18, u, b, "1", timing=False)
    [(xt, it)] = _solve(fgmod, monkeypatch, dims, precision, 18, u, b, "1", timing=True)
    assert np.array_equal(xg, xt) and ig["iterations"] == it["iterations"]
    n_iter, n_ru = it["iterations"], it["reliable_updates"]
    # 4 per iteration (the host queues up to two batches of at most 8 past
    # convergence or past an FP32 reliable-update request, which return at
    # once), one t_o = D_oe p after the setup and after each reliable update
    assert 4 * n_iter + 1 + n_ru <= it["n_dslash"] <= 4 * (n_iter + 16 * (n_ru + 1)) + 1 + n_ru
    assert it["n_blas"] <= 4 + 3 * n_ru


def test_folded_cg_larger_lattice(fgmod, monkeypatch):
    """12^3 x 24 in FP32: the folded and six-launch solvers agree, and the
    certified residual holds against the oracle's operator."""
    dims = (12, 12, 12, 24)
    u = inputs.hot_start(dims, 15)
    b = _rand_even(dims, 16)
    tol = 1e-10
    [(xf, inf)] = _solve(fgmod, monkeypatch, dims, "fp32", 18, u, b, "1")
    [(xs, ins)] = _solve(fgmod, monkeypatch, dims, "fp32", 18, u, b, "0")
    assert abs(inf["iterations"] - ins["iterations"]) <= 0.1 * ins["iterations"] + 2
    assert _rel(xf, xs) < 1e-7
    res = inputs.unpack_even(b, dims) - fe.mdagm(inf["links"], KAPPA, inputs.unpack_even(xf, dims))
    assert np.linalg.norm(res) <= 1.01 * tol * np.linalg.norm(b)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_chronological_guess_trajectory(fgmod, monkeypatch, precision):
    """Within a trajectory each pseudofermion solve starts from the previous
    one's solution (same phi, nearby links).  The trajectory's dH agrees
    with solves from zero to the solver tolerance's effect (FP64, cg_tol
    1e-13: 1e-8; with FP32 links and forces the different rounding of the
    solves moves dH by ~1e-4, within the FP32 path's 1e-3 bar against FP64),
    with fewer CG iterations, and
    two runs give the same bits (the guess is dropped at each trajectory's
    start)."""
    dims = (6, 6, 6, 12)
    u = inputs.hot_start(dims, 31)
    p = inputs.gaussian_momenta(dims, 32)
    chi = inputs.gaussian_spinor_even(dims, 33)
    tol = 1e-13 if precision == "fp64" else 1e-10
    out = {}
    for guess in ("1", "0"):
        monkeypatch.setenv("FG_CG_GUESS", guess)
        runs = []
        with fgmod.Lattice(dims, BETA, kappa=KAPPA, precision=precision, cg_tol=tol, cg_tol_action=tol) as lat:
            for _ in range(2):
                lat.set_gauge(u)
                lat.set_momenta(p)
                lat.set_pseudofermion(chi)
                r = lat.trajectory("fg", 0.125, 1.0, refresh=False, u_accept=0.0)
                runs.append((r, lat.get_gauge()))
        assert runs[0][0]["dH"] == runs[1][0]["dH"] and np.array_equal(runs[0][1], runs[1][1])
        out[guess] = runs[0]
    (rg, ug), (r0, u0) = out["1"], out["0"]
    assert rg["n_solves"] == r0["n_solves"]
    assert rg["cg_iters"] < 0.85 * r0["cg_iters"], (rg["cg_iters"], r0["cg_iters"])
    assert abs(rg["dH"] - r0["dH"]) <= (1e-8 if precision == "fp64" else 1e-3), (rg["dH"], r0["dH"])
    assert _rel(ug, u0) < (1e-11 if precision == "fp64" else 1e-4)


@pytest.mark.parametrize("dims,precision,folded", [((16, 16, 16, 32), "fp32", True), ((24, 24, 24, 48), "fp32", False),
                                                   ((16, 16, 16, 32), "fp64", False), ((8, 8, 8, 16), "fp64", True)])
def test_default_form_follows_the_l2_working_set(fgmod, monkeypatch, dims, precision, folded):
    """Without FG_CG_FOLD the library folds the iterations while the
    solver's links and six vectors fit in L2 (FP32 16^3 x 32: 76 MB; FP64
    8^3 x 16: 9 MB) and runs six launches beyond (FP32 24^3 x 48: 382 MB;
    FP64 16^3 x 32: 151 MB): the six-launch form runs two vector kernels per
    iteration, the folded one only in the setup and the reliable updates."""
    monkeypatch.delenv("FG_CG_FOLD", raising=False)
    b = _rand_even(dims, 18)
    with fgmod.Lattice(dims, BETA, kappa=KAPPA, precision=precision, cg_tol=1e-8) as lat:
        lat.random_gauge()
        lat.timing(True)
        _, info = lat.cg_solve(b)
        n_blas = lat.kernel_time("cg_blas")[1]
    assert info["true_residual"] <= 1e-8
    assert (n_blas < info["iterations"]) == folded, (n_blas, info["iterations"])
