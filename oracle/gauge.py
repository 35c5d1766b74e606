"""Wilson gauge action, staple force and kinetic term (oracle; test infrastructure only).

The paper writes the Hamiltonian as H(q, p) = S(q) + T(p) (section 2) and
calls the S-hat vector field the force (section 3).  It does not state the
gauge action; the oracle uses the unimproved Wilson plaquette action

    S_G = beta * sum_x sum_{mu<nu} (1 - Re Tr U_{mu nu}(x) / 3),
    U_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dagger U_nu(x)^dagger,

periodic in all four directions.  The force is the left derivative
F^a_mu(x) = dS/d eps^a along U_mu(x) -> exp(i eps T^a) U_mu(x), and the
kinetic term is T = (1/2) sum (p^a)^2 over all links and colours.
"""

from __future__ import annotations

import numpy as np

from .su3 import dag, trace, im_tr_gellmann


def shift(f: np.ndarray, mu: int, step: int) -> np.ndarray:
    """f(x + step * mu-hat) with periodic wrap; site axes are (t, z, y, x)."""
    return np.roll(f, -step, axis=3 - mu)


def plaquette_field(u: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """U_{mu nu}(x) on every site."""
    return (u[..., mu, :, :] @ shift(u[..., nu, :, :], mu, 1)
            @ dag(shift(u[..., mu, :, :], nu, 1)) @ dag(u[..., nu, :, :]))


def wilson_action(u: np.ndarray, beta: float) -> float:
    s = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            s += np.sum(1.0 - np.real(trace(plaquette_field(u, mu, nu))) / 3.0)
    return float(beta * s)


def mean_plaquette(u: np.ndarray) -> float:
    """<Re Tr U_p / 3> over the 6V plaquettes."""
    acc = 0.0
    for mu in range(4):
        for nu in range(mu + 1, 4):
            acc += np.mean(np.real(trace(plaquette_field(u, mu, nu)))) / 3.0
    return float(acc / 6.0)


def staple_sum(u: np.ndarray, mu: int) -> np.ndarray:
    """A_mu(x): the six staples closing a plaquette with U_mu(x).

    Upper staple U_nu(x+mu) U_mu(x+nu)^dagger U_nu(x)^dagger and lower staple
    U_nu(x+mu-nu)^dagger U_mu(x-nu)^dagger U_nu(x-nu), for every nu != mu, so
    that Re Tr(U_mu(x) A_mu(x)) is the sum over the plaquettes holding U_mu(x).
    """
    a = np.zeros(u.shape[:4] + (3, 3), dtype=np.complex128)
    for nu in range(4):
        if nu == mu:
            continue
        u_mu = u[..., mu, :, :]
        u_nu = u[..., nu, :, :]
        a += shift(u_nu, mu, 1) @ dag(shift(u_mu, nu, 1)) @ dag(u_nu)
        u_nu_m = shift(u_nu, nu, -1)                 # U_nu(x - nu)
        a += (dag(shift(u_nu_m, mu, 1))              # U_nu(x + mu - nu)^dagger
              @ dag(shift(u_mu, nu, -1))             # U_mu(x - nu)^dagger
              @ u_nu_m)
    return a


def _product_tangent(factors, tangents):
    """d/ds of factors[0] @ factors[1] @ ... with factor k -> factor k + s tangents[k]."""
    out = None
    for k in range(len(factors)):
        term = None
        for j, f in enumerate(factors):
            m = tangents[j] if j == k else f
            term = m if term is None else term @ m
        out = term if out is None else out + term
    return out


def staple_sum_tangent(u: np.ndarray, du: np.ndarray, mu: int) -> np.ndarray:
    """d/ds A_mu(x) along U -> U + s dU (every link moves; daggered links
    move by dU^dagger), term by term from ``staple_sum``."""
    a = np.zeros(u.shape[:4] + (3, 3), dtype=np.complex128)
    for nu in range(4):
        if nu == mu:
            continue
        u_mu, u_nu = u[..., mu, :, :], u[..., nu, :, :]
        d_mu, d_nu = du[..., mu, :, :], du[..., nu, :, :]
        a += _product_tangent([shift(u_nu, mu, 1), dag(shift(u_mu, nu, 1)), dag(u_nu)],
                              [shift(d_nu, mu, 1), dag(shift(d_mu, nu, 1)), dag(d_nu)])
        u_nu_m, d_nu_m = shift(u_nu, nu, -1), shift(d_nu, nu, -1)
        a += _product_tangent([dag(shift(u_nu_m, mu, 1)), dag(shift(u_mu, nu, -1)), u_nu_m],
                              [dag(shift(d_nu_m, mu, 1)), dag(shift(d_mu, nu, -1)), d_nu_m])
    return a


def gauge_force_tangent(u: np.ndarray, du: np.ndarray, beta: float) -> np.ndarray:
    """Directional derivative of ``gauge_force`` along the link tangent dU:
    (beta/6) Im Tr(lambda^a (dU_mu A_mu + U_mu dA_mu)).  With dU = i F U it is
    the force gradient G of section 4 (the derivative of the force along the
    vector field e^j(S) e_j)."""
    f = np.empty(u.shape[:5] + (8,))
    for mu in range(4):
        omega = du[..., mu, :, :] @ staple_sum(u, mu) + u[..., mu, :, :] @ staple_sum_tangent(u, du, mu)
        f[..., mu, :] = (beta / 6.0) * im_tr_gellmann(omega)
    return f


def gauge_force(u: np.ndarray, beta: float) -> np.ndarray:
    """F^a_mu(x) = dS_G/d eps^a = (beta/6) Im Tr(lambda^a U_mu(x) A_mu(x)).

    From d/d eps [-(beta/3) Re Tr(exp(i eps T^a) U A)] at eps = 0
    = (beta/3) Im Tr(T^a U A).  Shape ``[Lt, Lz, Ly, Lx, 4, 8]``.
    """
    f = np.empty(u.shape[:5] + (8,))
    for mu in range(4):
        omega = u[..., mu, :, :] @ staple_sum(u, mu)
        f[..., mu, :] = (beta / 6.0) * im_tr_gellmann(omega)
    return f


def link_force(u: np.ndarray, site, mu: int, beta: float) -> np.ndarray:
    """F^a for the single link U_mu(x) at site = (t, z, y, x): the same staple
    definition as ``gauge_force``, evaluated with explicit neighbour indices
    so that it can be sampled on lattices too large for whole-field numpy."""
    lt, lz, ly, lx = u.shape[:4]
    ext = (lx, ly, lz, lt)

    def at(c, d):                       # c = (x, y, z, t), link U_d(c)
        return u[c[3] % ext[3], c[2] % ext[2], c[1] % ext[1], c[0] % ext[0], d]

    def step(c, d, k):
        c = list(c)
        c[d] += k
        return c

    t, z, y, x = site
    c = [x, y, z, t]
    a = np.zeros((3, 3), dtype=np.complex128)
    for nu in range(4):
        if nu == mu:
            continue
        a += at(step(c, mu, 1), nu) @ dag(at(step(c, nu, 1), mu)) @ dag(at(c, nu))
        cm = step(c, nu, -1)
        a += dag(at(step(cm, mu, 1), nu)) @ dag(at(cm, mu)) @ at(cm, nu)
    return (beta / 6.0) * im_tr_gellmann(at(c, mu) @ a)


def kinetic(p: np.ndarray) -> float:
    """T = (1/2) sum_links sum_a (p^a)^2 = sum_links Tr P^2."""
    return float(0.5 * np.sum(p * p))


def gauge_transform_links(u: np.ndarray, g: np.ndarray) -> np.ndarray:
    """U_mu(x) -> g(x) U_mu(x) g(x+mu)^dagger."""
    out = np.empty_like(u)
    for mu in range(4):
        out[..., mu, :, :] = g @ u[..., mu, :, :] @ dag(shift(g, mu, 1))
    return out
