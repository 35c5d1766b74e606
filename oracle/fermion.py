"""Wilson fermions, even-odd preconditioning, CG and the pseudofermion force.

Oracle; test infrastructure only.  Section 4 of the paper takes a generic
pseudofermion action S = phi^dagger M^{-1}(U) phi with a Hermitian kernel M
and derives its force e_i(S) = -X^dagger e_i(M) X with X = M^{-1} phi;
section 5 uses Nf = 2 Wilson fermions with "the usual even-odd
preconditioning".  The paper fixes none of the conventions; the oracle uses

* Wilson-Dirac operator M = 1 - kappa D with the hopping term
  (D psi)(x) = sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu)
                       + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu)],
  periodic links, fermion fields antiperiodic in t;
* DeGrand-Rossi (chiral) Euclidean gamma matrices, gamma_5 = g1 g2 g3 g4;
* even-odd Schur complement on the even sites,
  Mhat = 1 - kappa^2 D_eo D_oe, and the Hermitian kernel
  calM = Mhat^dagger Mhat with Mhat^dagger = gamma_5 Mhat gamma_5;
* pseudofermions phi_e = Mhat^dagger chi_e from a complex Gaussian chi_e, so
  S_F = phi^dagger calM^{-1} phi equals chi^dagger chi at the heat bath.

Spinor fields are full-lattice arrays ``complex128[Lt, Lz, Ly, Lx, 4, 3]``;
"even" fields are zero on odd sites.
"""

from __future__ import annotations

import numpy as np

from .gauge import shift
from .su3 import dag, GENERATORS

GAMMA = np.zeros((4, 4, 4), dtype=np.complex128)
# gamma_1 (x)
GAMMA[0][0, 3], GAMMA[0][1, 2], GAMMA[0][2, 1], GAMMA[0][3, 0] = 1j, 1j, -1j, -1j
# gamma_2 (y)
GAMMA[1][0, 3], GAMMA[1][1, 2], GAMMA[1][2, 1], GAMMA[1][3, 0] = -1, 1, 1, -1
# gamma_3 (z)
GAMMA[2][0, 2], GAMMA[2][1, 3], GAMMA[2][2, 0], GAMMA[2][3, 1] = 1j, -1j, -1j, 1j
# gamma_4 (t)
GAMMA[3][0, 2], GAMMA[3][1, 3], GAMMA[3][2, 0], GAMMA[3][3, 1] = 1, 1, 1, 1
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
EYE4 = np.eye(4, dtype=np.complex128)


def spin_mul(g: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply a 4x4 spin matrix to every site of psi."""
    return np.einsum("st,...tc->...sc", g, psi)


def colour_mul(u: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Apply a per-site 3x3 colour matrix to every spin component."""
    return np.einsum("...ij,...sj->...si", u, psi)


def fshift(psi: np.ndarray, mu: int, step: int) -> np.ndarray:
    """psi(x + step*mu-hat) with antiperiodic wrap in t (mu = 3)."""
    out = shift(psi, mu, step)
    if mu == 3:
        out = out.copy()
        if step > 0:
            out[-1] *= -1.0      # x + t-hat wraps for t = Lt - 1
        else:
            out[0] *= -1.0       # x - t-hat wraps for t = 0
    return out


def hop(u: np.ndarray, psi: np.ndarray) -> np.ndarray:
    """Wilson hopping term D psi on the full lattice."""
    out = np.zeros_like(psi)
    for mu in range(4):
        u_mu = u[..., mu, :, :]
        fwd = colour_mul(u_mu, fshift(psi, mu, 1))
        bwd = colour_mul(dag(shift(u_mu, mu, -1)), fshift(psi, mu, -1))
        out += spin_mul(EYE4 - GAMMA[mu], fwd) + spin_mul(EYE4 + GAMMA[mu], bwd)
    return out


def wilson_m(u, kappa, psi):
    """Unpreconditioned M psi = psi - kappa D psi."""
    return psi - kappa * hop(u, psi)


def mhat(u, kappa, psi_e):
    """Mhat psi_e = psi_e - kappa^2 D_eo D_oe psi_e for an even-supported psi_e."""
    return psi_e - kappa * kappa * hop(u, hop(u, psi_e))


def mhat_dag(u, kappa, psi_e):
    """Mhat^dagger = gamma_5 Mhat gamma_5."""
    return spin_mul(GAMMA5, mhat(u, kappa, spin_mul(GAMMA5, psi_e)))


def mdagm(u, kappa, psi_e):
    return mhat_dag(u, kappa, mhat(u, kappa, psi_e))


def vdot(a, b):
    """<a, b> = sum conj(a) b over all components."""
    return complex(np.vdot(a.reshape(-1), b.reshape(-1)))


def cg(u, kappa, b, tol=1e-10, maxiter=10000):
    """Textbook conjugate gradient for calM x = b, x0 = 0.

    Stops when the recursively updated residual satisfies |r| <= tol |b|.
    Returns (x, iterations).
    """
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = vdot(r, r).real
    bnorm = np.sqrt(vdot(b, b).real)
    if bnorm == 0.0:
        return x, 0
    for k in range(1, maxiter + 1):
        ap = mdagm(u, kappa, p)
        alpha = rr / vdot(p, ap).real
        x = x + alpha * p
        r = r - alpha * ap
        rr_new = vdot(r, r).real
        if np.sqrt(rr_new) <= tol * bnorm:
            return x, k
        p = r + (rr_new / rr) * p
        rr = rr_new
    raise RuntimeError("CG did not converge")


def heatbath_phi(u, kappa, chi_e):
    """phi_e = Mhat^dagger chi_e (pseudofermion refresh)."""
    return mhat_dag(u, kappa, chi_e)


def pseudofermion_action(u, kappa, phi_e, tol=1e-12):
    x, _ = cg(u, kappa, phi_e, tol)
    return vdot(phi_e, x).real


def fermion_force(u, kappa, phi_e, tol=1e-12, x=None):
    """F^a_mu(x) = dS_F / d eps^a for S_F = phi^dagger (Mhat^dagger Mhat)^{-1} phi.

    Section 4: e_i(S) = -X^dagger e_i(calM) X with X = calM^{-1} phi.  With
    Y = Mhat X and e_i(Mhat) = -kappa^2 (e_i(D) D + D e_i(D)) this is
    2 kappa^2 Re <Ytilde, e_i(D) Xtilde>, where Xtilde = X_e + D X_e and
    Ytilde = Y_e + D^dagger Y_e (D^dagger = gamma_5 D gamma_5).  The derivative
    of D with respect to U_mu(x) -> exp(i eps T^a) U_mu(x) touches only the
    two hopping terms through that link, written out below for each a.
    """
    if x is None:
        x, _ = cg(u, kappa, phi_e, tol)
    y = mhat(u, kappa, x)
    xt = x + hop(u, x)
    yt = y + spin_mul(GAMMA5, hop(u, spin_mul(GAMMA5, y)))
    return _force_form(u, kappa, xt, yt)


def _force_form(u, kappa, xt, yt):
    """2 kappa^2 Re <Ytilde, e_a(D) Xtilde> per link: real-linear in each of
    the links (U enters each hop term once, as U or U^dagger), Xtilde and
    Ytilde."""
    f = np.empty(u.shape[:5] + (8,))
    for mu in range(4):
        u_mu = u[..., mu, :, :]
        x_fwd = fshift(xt, mu, 1)      # Xtilde(x + mu), with the boundary sign
        y_fwd = fshift(yt, mu, 1)      # Ytilde(x + mu), with the boundary sign
        pm = spin_mul(EYE4 - GAMMA[mu], colour_mul(u_mu, x_fwd))
        for a in range(8):
            ta = GENERATORS[a]
            # forward hop at x: Ytilde(x)^dag (1 - g_mu) (i T^a U) Xtilde(x+mu)
            t1 = np.einsum("...sc,...sc->...", np.conj(yt),
                           1j * np.einsum("ij,...sj->...si", ta, pm))
            # backward hop at x+mu: Ytilde(x+mu)^dag (1 + g_mu) (-i U^dag T^a) Xtilde(x)
            q = colour_mul(-1j * dag(u_mu) @ ta, xt)
            t2 = np.einsum("...sc,...sc->...", np.conj(y_fwd),
                           spin_mul(EYE4 + GAMMA[mu], q))
            f[..., mu, a] = 2.0 * kappa * kappa * np.real(t1 + t2)
    return f


def mhat_tangent(u, du, kappa, psi_e):
    """d/ds Mhat psi_e along U -> U + s dU: -kappa^2 (D(dU) D(U) + D(U) D(dU)) psi_e
    (the hop is linear in the links, its backward terms in U^dagger)."""
    return -kappa * kappa * (hop(du, hop(u, psi_e)) + hop(u, hop(du, psi_e)))


def mhat_dag_tangent(u, du, kappa, psi_e):
    return spin_mul(GAMMA5, mhat_tangent(u, du, kappa, spin_mul(GAMMA5, psi_e)))


def mdagm_tangent(u, du, kappa, x):
    """F(calM) X of section 4 for the direction dU: dMhat^dag Mhat X + Mhat^dag dMhat X."""
    return mhat_dag_tangent(u, du, kappa, mhat(u, kappa, x)) + mhat_dag(u, kappa, mhat_tangent(u, du, kappa, x))


def fermion_force_tangent(u, du, kappa, phi_e, tol=1e-12, x=None):
    """Directional derivative of ``fermion_force`` along the link tangent dU.

    Section 4: with X = calM^{-1} phi, its derivative is Y = -calM^{-1} F(calM) X
    (one more solve); the force -X^dag e_i(calM) X then changes by
    Y^dag e_i(calM) X + X^dag F(e_i(calM)) X + X^dag e_i(calM) Y.  Here the same
    sum is taken through the bilinear form of ``fermion_force``: the links,
    Xtilde and Ytilde each move in turn.  With dU = i F U (F the total force)
    this is the fermion part of the force gradient G.
    """
    if x is None:
        x, _ = cg(u, kappa, phi_e, tol)
    z, _ = cg(u, kappa, mdagm_tangent(u, du, kappa, x), tol)
    dx = -z
    y = mhat(u, kappa, x)
    dy = mhat_tangent(u, du, kappa, x) + mhat(u, kappa, dx)
    xt = x + hop(u, x)
    dxt = dx + hop(du, x) + hop(u, dx)
    yt = y + spin_mul(GAMMA5, hop(u, spin_mul(GAMMA5, y)))
    dyt = (dy + spin_mul(GAMMA5, hop(du, spin_mul(GAMMA5, y)))
           + spin_mul(GAMMA5, hop(u, spin_mul(GAMMA5, dy))))
    return _force_form(du, kappa, xt, yt) + _force_form(u, kappa, dxt, yt) + _force_form(u, kappa, xt, dyt)


class FermionSystem:
    """H = S_G(U) + S_F(U) + T(p) for Nf = 2 Wilson fermions (section 5)."""

    def __init__(self, beta, kappa, phi_e, tol=1e-12):
        from .integrators import GaugeSystem
        self.gauge = GaugeSystem(beta)
        self.kappa = float(kappa)
        self.phi = phi_e
        self.tol = tol
        self.n_force = 0
        self.n_solve = 0

    def action(self, u):
        self.n_solve += 1
        return self.gauge.action(u) + pseudofermion_action(u, self.kappa, self.phi, self.tol)

    def force(self, u):
        self.n_force += 1
        self.n_solve += 1
        return self.gauge.force(u) + fermion_force(u, self.kappa, self.phi, self.tol)

    def force_tangent(self, u, du):
        self.n_solve += 2
        return self.gauge.force_tangent(u, du) + fermion_force_tangent(u, du, self.kappa, self.phi, self.tol)


class PseudofermionPart:
    """S_F alone (the outer action of a two-level integrator)."""

    def __init__(self, kappa, phi_e, tol=1e-12):
        self.kappa = float(kappa)
        self.phi = phi_e
        self.tol = tol
        self.n_force = 0

    def action(self, u):
        return pseudofermion_action(u, self.kappa, self.phi, self.tol)

    def force(self, u):
        self.n_force += 1
        return fermion_force(u, self.kappa, self.phi, self.tol)

    def force_tangent(self, u, du):
        return fermion_force_tangent(u, du, self.kappa, self.phi, self.tol)
