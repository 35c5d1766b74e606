"""One-dimensional anharmonic oscillator with closed-form Poisson brackets.

Oracle test infrastructure: a flat-space system H = S(q) + T(p) with
S = q^4/4 + q^2/2 and T = p^2/2 on which every bracket of Table 1 has a
closed form, so the shadow Hamiltonians of section 3 can be checked
directly.  With {A, B} = A_q B_p - A_p B_q and V = S:

    {S,T}            = p V'
    {S,{S,T}}        = V'^2                     (section 4: e^i(S) e_i(S))
    {T,{S,T}}        = -p^2 V''
    {S,{S,{S,{S,T}}}} = 0
    {{S,T},{S,{S,T}}} = -2 V'^2 V''
    {{S,T},{T,{S,T}}} = -2 p^2 V''^2 + p^2 V' V'''
    {T,{S,{S,{S,T}}}} = 0
    {T,{T,{S,{S,T}}}} = 2 p^2 (V''^2 + V' V''')
    {T,{T,{T,{S,T}}}} = -p^4 V''''

(derived by hand from the bracket definition).  The flows are exact: a kick
p <- p - c dt V'(q), a drift q <- q + c dt p, and the force-gradient kick of
Table 1 uses the gradient of (2/3) S - (dt^2/72) V'^2.
"""

from __future__ import annotations

import numpy as np

from .integrators import sequence


def v1(q):
    return q ** 3 + q


def v2(q):
    return 3 * q ** 2 + 1


def v3(q):
    return 6 * q


def v4(q):
    return 6.0 + 0 * q


def energy(q, p):
    return q ** 4 / 4 + q ** 2 / 2 + p ** 2 / 2


def brackets(q, p):
    """Dictionary of the Poisson brackets that appear in Table 1."""
    return {
        "SST": v1(q) ** 2,
        "TST": -p ** 2 * v2(q),
        "SSSST": 0.0 * q,
        "STSST": -2 * v1(q) ** 2 * v2(q),
        "STTST": -2 * p ** 2 * v2(q) ** 2 + p ** 2 * v1(q) * v3(q),
        "TSSST": 0.0 * q,
        "TTSST": 2 * p ** 2 * (v2(q) ** 2 + v1(q) * v3(q)),
        "TTTST": -p ** 4 * v4(q),
    }


def step(name, q, p, dt, alpha=None, fg_mode="exact"):
    """One step of the named integrator on the toy (exact sub-flows)."""
    seq = sequence(name) if alpha is None else sequence(name, alpha)
    for op in seq:
        if op[0] == "P":
            p = p - op[1] * dt * v1(q)
        elif op[0] == "Q":
            q = q + op[1] * dt * p
        else:
            c, g = op[1], op[2]
            shift = 2.0 * g / c * dt * dt
            if fg_mode == "exact":
                # gradient of c S - g dt^2 V'^2 is c [V' - (2g/c) dt^2 V' V'']
                f_eff = v1(q) - shift * v1(q) * v2(q)
            else:
                # force at a point displaced along the force
                f_eff = v1(q - shift * v1(q))
            p = p - c * dt * f_eff
    return q, p


def shadow(name, q, p, dt, alpha=None):
    """Truncated shadow Hamiltonian of Table 1 / section 3 for the named integrator."""
    b = brackets(q, p)
    h = energy(q, p)
    if name == "leapfrog":
        return h - dt ** 2 / 24 * (b["SST"] + 2 * b["TST"])
    if name == "qpq":
        return h + dt ** 2 / 24 * (2 * b["SST"] + b["TST"])
    if name == "omelyan":
        a = alpha
        return h + dt ** 2 * ((6 * a * a - 6 * a + 1) / 12 * b["SST"]
                              + (1 - 6 * a) / 24 * b["TST"])
    if name == "fg":
        return h - dt ** 4 / 155520 * (41 * b["SSSST"] + 36 * b["STSST"]
                                        + 72 * b["STTST"] + 84 * b["TSSST"]
                                        + 126 * b["TTSST"] + 54 * b["TTTST"])
    if name == "campostrini":
        c4, c2 = 4 ** (1 / 3), 2 ** (1 / 3)

        def k(a, bb, c):
            return a * c4 + bb * c2 + c
        return h + dt ** 4 / 34560 * (-k(40, 40, 48) * b["SSSST"]
                                      + k(180, 240, 312) * b["STSST"]
                                      + k(60, 80, 104) * b["STTST"]
                                      + k(-20, 0, 8) * b["TSSST"]
                                      + k(0, 20, 32) * b["TTSST"]
                                      + k(0, 5, 8) * b["TTTST"])
    raise ValueError(name)
