"""fg_trajectories_host_momenta: n trajectories whose momenta come from host
memory, with the upload of the next momenta overlapping the running
trajectory.  The links, momenta and results must be exactly those of the
sequential fg_set_momenta + fg_trajectory(refresh = 0) loop on a second
handle with the same parameters (same kernels on the same inputs, so the
comparison is bit-for-bit), including rejected trajectories and accept
uniforms drawn from the handle's host RNG; the first FP64 trajectory is also
checked against the oracle's dH (section 5)."""

import numpy as np
import pytest

from oracle import integrators as it
from paper_0910_2950_gb300 import inputs

pytestmark = pytest.mark.gpu

BETA = 6.0


@pytest.fixture(scope="module")
def fgmod():
    from paper_0910_2950_gb300 import build, fg
    build.build()
    fg.load()
    return fg


def _momenta(dims, n, seed, pinned):
    out = []
    for k in range(n):
        p = inputs.gaussian_momenta(dims, seed + k).reshape(-1)
        if pinned:
            import torch
            buf = torch.empty(p.size, dtype=torch.float64, pin_memory=True).numpy()
            buf[:] = p
            p = buf
        out.append(p)
    return out


def _sequential(lat, integ, dt, moms, us):
    res = []
    for p, u in zip(moms, us):
        lat.set_momenta(p)
        res.append(lat.trajectory(integ, dt, 1.0, refresh=False, u_accept=u))
    return res


@pytest.mark.parametrize("precision,pinned", [("fp32", True), ("fp64", False), ("fp32", False)])
def test_pure_gauge_matches_sequential(fgmod, precision, pinned):
    dims = (8, 8, 8, 8)
    u0 = inputs.hot_start(dims, 21)
    moms = _momenta(dims, 5, 22, pinned)
    # accept always, reject if dH > ~0, accept uniform 0.5, host RNG twice
    us = [0.0, 0.999999999, 0.5, -1.0, -1.0]
    kw = dict(precision=precision, seed=77)
    with fgmod.Lattice(dims, BETA, **kw) as a, fgmod.Lattice(dims, BETA, **kw) as b:
        a.set_gauge(u0)
        b.set_gauge(u0)
        ra = a.trajectories_host_momenta("fg", 0.25, 1.0, moms, u_accept=us)
        rb = _sequential(b, "fg", 0.25, moms, us)
        assert len(ra) == len(rb) == 5
        for x, y in zip(ra, rb):
            assert x == y
        assert np.array_equal(a.get_gauge(), b.get_gauge())
        assert np.array_equal(a.get_momenta(), b.get_momenta())
        # the handle's RNG drew the same uniforms: one more trajectory agrees
        x = a.trajectories_host_momenta("omelyan", 0.125, 1.0, moms[:1])
        y = _sequential(b, "omelyan", 0.125, moms[:1], [-1.0])
        assert x == y
    if precision == "fp64":
        _, _, h0, h1 = it.trajectory(it.GaugeSystem(BETA), it.Integrator("fg"), u0,
                                     moms[0].reshape(inputs.site_shape(dims) + (4, 8)), 0.25, 1.0)
        assert abs(ra[0]["dH"] - (h1 - h0)) < 1e-6


def test_nf2_matches_sequential(fgmod):
    dims = (4, 4, 4, 8)
    kappa = 0.12
    u0 = inputs.hot_start(dims, 31)
    chi = inputs.gaussian_spinor_even(dims, 32)
    moms = _momenta(dims, 3, 33, True)
    us = [0.0, 0.5, -1.0]
    kw = dict(precision="fp32", kappa=kappa, seed=5)
    with fgmod.Lattice(dims, 5.6, **kw) as a, fgmod.Lattice(dims, 5.6, **kw) as b:
        for lat in (a, b):
            lat.set_gauge(u0)
            lat.set_pseudofermion(chi)
        ra = a.trajectories_host_momenta("fg", 0.25, 1.0, moms, u_accept=us)
        rb = _sequential(b, "fg", 0.25, moms, us)
        for x, y in zip(ra, rb):
            assert x == y
        assert np.array_equal(a.get_gauge(), b.get_gauge())


@pytest.mark.parametrize("precision", ["fp32", "df64", "fp64"])
def test_fp32_host_momenta(fgmod, precision):
    """FP32 host momenta (half the upload): the trajectories are those of the
    FP64 host momenta rounded to FP32, bit for bit (every handle widens or
    keeps the FP32 values exactly)."""
    import torch
    dims = (8, 8, 8, 8)
    u0 = inputs.hot_start(dims, 41)
    m64 = [p.astype(np.float32).astype(np.float64) for p in _momenta(dims, 4, 42, False)]
    m32 = []
    for p in m64:
        buf = torch.empty(p.size, dtype=torch.float32, pin_memory=True).numpy()
        buf[:] = p
        m32.append(buf)
    us = [0.0, 0.5, -1.0, -1.0]
    kw = dict(precision=precision, seed=9)
    with fgmod.Lattice(dims, BETA, **kw) as a, fgmod.Lattice(dims, BETA, **kw) as b:
        a.set_gauge(u0)
        b.set_gauge(u0)
        ra = a.trajectories_host_momenta("fg", 0.25, 1.0, m32, u_accept=us)
        rb = b.trajectories_host_momenta("fg", 0.25, 1.0, m64, u_accept=us)
        assert ra == rb
        assert np.array_equal(a.get_gauge(), b.get_gauge())
        assert np.array_equal(a.get_momenta(), b.get_momenta())


def test_arguments(fgmod):
    dims = (4, 4, 4, 4)
    with fgmod.Lattice(dims, BETA, precision="fp32") as lat:
        assert lat.trajectories_host_momenta("fg", 0.25, 1.0, []) == []
        moms = _momenta(dims, 2, 40, False)
        with pytest.raises(fgmod.FgError):
            lat.trajectories_host_momenta("fg", 0.25, 1.0, moms, u_accept=[0.0, 1.0])
        with pytest.raises(fgmod.FgError):
            lat.trajectories_host_momenta("fg", 0.3, 1.0, moms)
        # the handle still works after the refused calls
        r = lat.trajectories_host_momenta("fg", 0.25, 1.0, moms, u_accept=[0.0, 0.0])
        assert len(r) == 2 and all(x["accepted"] for x in r)
