"""SU(3) group and su(3) algebra helpers (oracle; test infrastructure only).

Section 2 of the paper puts the Hamiltonian system on the group manifold:
momenta live in the Lie algebra, P = p_i T^i, and the T-hat flow (drift) is
integrated exactly.  Conventions (the paper leaves them open):

* generators T^a = lambda^a / 2 (Gell-Mann), Tr(T^a T^b) = delta^{ab} / 2;
* momenta are Hermitian traceless P = sum_a p^a lambda^a / 2, so that
  T = (1/2) sum_a (p^a)^2 = Tr P^2;
* left action: a link moves as U -> exp(i eps T^a) U, consistent with the
  left-invariant derivative e_i(U) = -T_i U of section 4 up to the sign of
  the generator.
"""

from __future__ import annotations

import numpy as np

# Gell-Mann matrices lambda^1 .. lambda^8 (standard textbook definition).
GELL_MANN = np.zeros((8, 3, 3), dtype=np.complex128)
GELL_MANN[0][0, 1] = GELL_MANN[0][1, 0] = 1
GELL_MANN[1][0, 1], GELL_MANN[1][1, 0] = -1j, 1j
GELL_MANN[2][0, 0], GELL_MANN[2][1, 1] = 1, -1
GELL_MANN[3][0, 2] = GELL_MANN[3][2, 0] = 1
GELL_MANN[4][0, 2], GELL_MANN[4][2, 0] = -1j, 1j
GELL_MANN[5][1, 2] = GELL_MANN[5][2, 1] = 1
GELL_MANN[6][1, 2], GELL_MANN[6][2, 1] = -1j, 1j
GELL_MANN[7][0, 0] = GELL_MANN[7][1, 1] = 1 / np.sqrt(3)
GELL_MANN[7][2, 2] = -2 / np.sqrt(3)

GENERATORS = GELL_MANN / 2.0  # T^a


def dag(u: np.ndarray) -> np.ndarray:
    """Hermitian conjugate over the last two axes."""
    return np.conj(np.swapaxes(u, -1, -2))


def trace(u: np.ndarray) -> np.ndarray:
    return np.trace(u, axis1=-2, axis2=-1)


def alg_to_mat(p: np.ndarray) -> np.ndarray:
    """P = sum_a p^a lambda^a / 2 for real coefficients ``p[..., 8]``."""
    return np.tensordot(p, GENERATORS, axes=([-1], [0]))


def mat_to_alg(h: np.ndarray) -> np.ndarray:
    """Coefficients p^a = Re Tr(lambda^a H) of a Hermitian traceless H."""
    return np.real(np.einsum("aij,...ji->...a", GELL_MANN, h))


def expi(p_mat: np.ndarray, c: float) -> np.ndarray:
    """exp(i c P) for Hermitian P, by its eigendecomposition.

    This is the exact T-hat flow of section 2 for a time c: with
    P = V diag(w) V^dagger, exp(i c P) = V diag(exp(i c w)) V^dagger.
    """
    w, v = np.linalg.eigh(p_mat)
    return (v * np.exp(1j * c * w)[..., None, :]) @ dag(v)


def im_tr_gellmann(omega: np.ndarray) -> np.ndarray:
    """Im Tr(lambda^a Omega) for a = 1..8, shape ``[..., 8]``."""
    return np.imag(np.einsum("aij,...ji->...a", GELL_MANN, omega))


def unitarity_defect(u: np.ndarray) -> float:
    """max |U^dagger U - 1| over all matrices."""
    eye = np.eye(3)
    return float(np.max(np.abs(dag(u) @ u - eye)))
