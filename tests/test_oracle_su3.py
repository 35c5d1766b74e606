"""Pins for oracle.su3 against textbook facts and library routines."""

import numpy as np
import pytest
import scipy.linalg

from oracle import su3
from paper_0910_2950_gb300 import inputs


def test_gell_mann_textbook_relations():
    lam = su3.GELL_MANN
    gram = np.einsum("aij,bji->ab", lam, lam)
    assert np.allclose(gram, 2 * np.eye(8), atol=1e-15)
    assert np.allclose(lam, su3.dag(lam), atol=0)
    assert np.allclose(su3.trace(lam), 0, atol=1e-15)
    # structure constants f_123 = 1, f_458 = sqrt(3)/2: [T^a, T^b] = i f_abc T^c
    t = su3.GENERATORS
    assert np.allclose(t[0] @ t[1] - t[1] @ t[0], 1j * t[2], atol=1e-15)
    assert np.allclose(t[3] @ t[4] - t[4] @ t[3],
                       1j * (0.5 * t[2] + np.sqrt(3) / 2 * t[7]), atol=1e-15)


def test_algebra_roundtrip_and_kinetic_normalisation():
    p = inputs.make_rng(3).standard_normal((50, 8))
    h = su3.alg_to_mat(p)
    assert np.allclose(h, su3.dag(h), atol=1e-15)
    assert np.allclose(su3.trace(h), 0, atol=1e-14)
    assert np.allclose(su3.mat_to_alg(h), p, atol=1e-14)
    # T = (1/2) sum p^2 = Tr P^2 with lambda/2 normalisation
    assert np.allclose(np.real(su3.trace(h @ h)), 0.5 * np.sum(p * p, axis=-1), atol=1e-13)


def test_expi_matches_scipy_expm():
    g = inputs.make_rng(4)
    for _ in range(20):
        a = g.standard_normal((3, 3)) + 1j * g.standard_normal((3, 3))
        h = a + su3.dag(a)
        c = g.uniform(-2, 2)
        assert np.allclose(su3.expi(h, c), scipy.linalg.expm(1j * c * h), atol=1e-13)


def test_expi_diagonal_closed_form_and_group_properties():
    theta = np.array([0.3, -1.1, 0.8])
    h = np.diag(theta).astype(np.complex128)
    assert np.allclose(su3.expi(h, 0.7), np.diag(np.exp(0.7j * theta)), atol=1e-15)
    p = su3.alg_to_mat(inputs.make_rng(5).standard_normal((100, 8)))
    e = su3.expi(p, 0.9)
    assert su3.unitarity_defect(e) < 1e-14
    assert np.allclose(np.linalg.det(e), 1.0, atol=1e-13)
    assert np.allclose(e @ su3.expi(p, -0.9), np.eye(3), atol=1e-14)


def test_im_tr_gellmann_picks_coefficients():
    for b in range(8):
        expect = np.zeros(8)
        expect[b] = 2.0
        assert np.allclose(su3.im_tr_gellmann(1j * su3.GELL_MANN[b]), expect, atol=1e-15)


@pytest.mark.parametrize("seed", [1, 2])
def test_haar_inputs_are_special_unitary(seed):
    u = inputs.haar_su3(inputs.make_rng(seed), (200,))
    assert su3.unitarity_defect(u) < 1e-14
    assert np.allclose(np.linalg.det(u), 1.0, atol=1e-13)
    # Haar: E[Tr U] = 0 and E[|Tr U|^2] = 1
    tr = su3.trace(u)
    assert abs(np.mean(tr)) < 0.3
    assert abs(np.mean(np.abs(tr) ** 2) - 1.0) < 0.35
