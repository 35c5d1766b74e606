"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This module holds no arithmetic of the integrators: it only draws random
numbers and moves them between array layouts.  Both the oracle and the CUDA
path receive the arrays it produces, so they never have to agree on a random
number generator.

Canonical host layouts (FP64, the ones the C ABI accepts):

* lattice dims are ``(Lx, Ly, Lz, Lt)``; site arrays are shaped
  ``(Lt, Lz, Ly, Lx, ...)`` so that the lexicographic site index is
  ``i = x + Lx*(y + Ly*(z + Lz*t))``;
* gauge field: ``complex128[Lt, Lz, Ly, Lx, 4, 3, 3]`` (direction mu = 0..3
  for x, y, z, t, then row, column);
* momenta: ``float64[Lt, Lz, Ly, Lx, 4, 8]``, the coefficients p^a of
  P = sum_a p^a lambda^a / 2 in the Gell-Mann basis;
* even-parity spinor: ``complex128[V/2, 4, 3]`` (spin, colour), even sites
  ((x+y+z+t) even) in increasing lexicographic order, so the even site with
  lexicographic index i sits at row i // 2 (Lx is even).
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "make_rng", "site_shape", "volume", "haar_su3", "hot_start", "cold_start",
    "gaussian_momenta", "gaussian_spinor_even", "random_gauge_transform",
    "parity_mask", "pack_even", "unpack_even", "check_dims",
]


def check_dims(dims) -> tuple:
    dims = tuple(int(d) for d in dims)
    if len(dims) != 4 or any(d < 2 or d % 2 for d in dims):
        raise ValueError(f"lattice dims must be four even extents >= 2, got {dims}")
    return dims


def make_rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def site_shape(dims) -> tuple:
    lx, ly, lz, lt = check_dims(dims)
    return (lt, lz, ly, lx)


def volume(dims) -> int:
    return int(np.prod(check_dims(dims)))


def haar_su3(rng: np.random.Generator, shape) -> np.ndarray:
    """Haar-distributed SU(3) matrices, ``complex128[*shape, 3, 3]``.

    QR of a complex Gaussian matrix with the phases of R's diagonal moved
    into Q gives Haar U(3) (Mezzadri, Notices AMS 54 (2007) 592); dividing
    by the principal cube root of the determinant maps that onto SU(3) while
    keeping left invariance.
    """
    shape = tuple(shape)
    z = (rng.standard_normal(shape + (3, 3)) +
         1j * rng.standard_normal(shape + (3, 3))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(q)
    return q / (det ** (1.0 / 3.0))[..., None, None]


def hot_start(dims, seed: int) -> np.ndarray:
    """Independent Haar-random links on every (site, direction)."""
    return haar_su3(make_rng(seed), site_shape(dims) + (4,))


def cold_start(dims) -> np.ndarray:
    u = np.zeros(site_shape(dims) + (4, 3, 3), dtype=np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def gaussian_momenta(dims, seed: int) -> np.ndarray:
    """Unit-Gaussian su(3) momenta: 8 independent N(0,1) coefficients per link."""
    return make_rng(seed).standard_normal(site_shape(dims) + (4, 8))


def gaussian_spinor_even(dims, seed: int) -> np.ndarray:
    """Complex Gaussian even-site spinor with density proportional to exp(-|chi|^2).

    Real and imaginary parts are each N(0, 1/2).
    """
    v = volume(dims)
    g = make_rng(seed)
    return (g.standard_normal((v // 2, 4, 3)) +
            1j * g.standard_normal((v // 2, 4, 3))) * np.sqrt(0.5)


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """One Haar-random SU(3) matrix per site, ``complex128[Lt, Lz, Ly, Lx, 3, 3]``."""
    return haar_su3(make_rng(seed), site_shape(dims))


def parity_mask(dims) -> np.ndarray:
    """Boolean ``[Lt, Lz, Ly, Lx]`` array, True on even sites."""
    lt, lz, ly, lx = site_shape(dims)
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly),
                             np.arange(lx), indexing="ij")
    return (x + y + z + t) % 2 == 0


def pack_even(full: np.ndarray, dims) -> np.ndarray:
    """Full-lattice spinor ``[Lt,Lz,Ly,Lx,4,3]`` -> even-site rows ``[V/2,4,3]``."""
    sh = site_shape(dims)
    flat = full.reshape((-1,) + full.shape[len(sh):])
    return np.ascontiguousarray(flat[parity_mask(dims).reshape(-1)])


def unpack_even(packed: np.ndarray, dims) -> np.ndarray:
    """Even-site rows ``[V/2,4,3]`` -> full-lattice spinor, zero on odd sites."""
    sh = site_shape(dims)
    out = np.zeros((int(np.prod(sh)),) + packed.shape[1:], dtype=packed.dtype)
    out[parity_mask(dims).reshape(-1)] = packed
    return out.reshape(sh + packed.shape[1:])
