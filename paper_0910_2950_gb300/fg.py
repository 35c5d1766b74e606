"""ctypes binding of ``libfg_lattice.so`` (C ABI in ``include/fg_lattice.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  The names follow the C ABI (``fg_set_gauge`` -> ``Lattice.set_gauge``
and so on).  Host arrays use the canonical FP64 layouts documented in
``paper_0910_2950_gb300.inputs`` and in the header.  If the library is
missing or cannot be loaded, every entry point raises: there is no CPU
fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
# FG_LATTICE_LIB selects another build of the library (e.g. a tuning variant).
LIB_PATH = os.environ.get("FG_LATTICE_LIB", os.path.join(_PKG, "libfg_lattice.so"))

FG_OK, FG_EINVAL, FG_ENOMEM, FG_ECUDA, FG_ENOCONV, FG_ETIMEOUT, FG_ESTATE = range(7)
STATUS_NAMES = {0: "FG_OK", 1: "FG_EINVAL", 2: "FG_ENOMEM", 3: "FG_ECUDA", 4: "FG_ENOCONV",
                5: "FG_ETIMEOUT", 6: "FG_ESTATE"}
INTEGRATORS = {"leapfrog": 0, "omelyan": 1, "fg": 2, "force_gradient": 2, "campostrini": 3, "qpq": 4,
               "fg_analytic": 5}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp32_fp16cg": 2, "df64": 3, "fp32_autocg": 4, "fp32_bf16cg": 5}

# Every function the header declares, with its ctypes signature.
_vp, _dp, _i, _d = C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_double


class FgParams(C.Structure):
    _fields_ = [("dims", C.c_int * 4), ("beta", C.c_double), ("kappa", C.c_double),
                ("alpha", C.c_double), ("precision", C.c_int), ("link_reals", C.c_int),
                ("reunitarize", C.c_int), ("cg_tol", C.c_double), ("cg_tol_action", C.c_double),
                ("cg_maxiter", C.c_int), ("cg_delta", C.c_double), ("seed", C.c_ulonglong),
                ("cuda_stream", C.c_void_p)]


class FgTrajResult(C.Structure):
    _fields_ = [("dH", C.c_double), ("H0", C.c_double), ("H1", C.c_double),
                ("S_gauge0", C.c_double), ("S_gauge1", C.c_double),
                ("S_ferm0", C.c_double), ("S_ferm1", C.c_double),
                ("T0", C.c_double), ("T1", C.c_double), ("accepted", C.c_int),
                ("n_steps", C.c_int), ("n_force", C.c_int), ("n_solves", C.c_int),
                ("cg_iters", C.c_longlong)]


class FgCgResult(C.Structure):
    _fields_ = [("iterations", C.c_int), ("reliable_updates", C.c_int),
                ("true_residual", C.c_double)]


class FgBatchParams(C.Structure):
    _fields_ = [("nchains", C.c_int), ("dims", C.POINTER(C.c_int)), ("beta", C.POINTER(C.c_double)),
                ("precision", C.c_int), ("link_reals", C.c_int), ("reunitarize", C.c_int),
                ("alpha", C.c_double), ("tile", C.c_int), ("use_graphs", C.c_int),
                ("seed", C.c_ulonglong), ("cuda_stream", C.c_void_p)]


SIGNATURES = {
    "fg_params_default": (_i, [C.POINTER(FgParams)]),
    "fg_fp32_fma_rate": (_i, [C.POINTER(C.c_double)]),
    "fg_lattice_create": (_i, [C.POINTER(FgParams), C.POINTER(_vp)]),
    "fg_lattice_destroy": (None, [_vp]),
    "fg_last_error": (C.c_char_p, [_vp]),
    "fg_set_gauge": (_i, [_vp, _dp]),
    "fg_get_gauge": (_i, [_vp, _dp]),
    "fg_set_momenta": (_i, [_vp, _dp]),
    "fg_get_momenta": (_i, [_vp, _dp]),
    "fg_refresh_momenta": (_i, [_vp]),
    "fg_set_pseudofermion": (_i, [_vp, _dp]),
    "fg_refresh_pseudofermion": (_i, [_vp]),
    "fg_force": (_i, [_vp, _dp]),
    "fg_action": (_i, [_vp, _dp, _dp, _dp]),
    "fg_plaquette": (_i, [_vp, _dp]),
    "fg_md_step": (_i, [_vp, _i, _d]),
    "fg_fg_step": (_i, [_vp, _d]),
    "fg_trajectory": (_i, [_vp, _i, _d, _d, _i, _d, C.POINTER(FgTrajResult)]),
    "fg_apply_mhat": (_i, [_vp, _dp, _dp, _i]),
    "fg_apply_mhat_inner": (_i, [_vp, _dp, _dp, _i]),
    "fg_cg_solve": (_i, [_vp, _dp, _dp, C.POINTER(FgCgResult)]),
    "fg_reunitarize": (_i, [_vp]),
    "fg_random_gauge": (_i, [_vp]),
    "fg_set_rng_position": (_i, [_vp, C.c_ulonglong]),
    "fg_timing_enable": (_i, [_vp, _i]),
    "fg_timing_reset": (_i, [_vp]),
    "fg_kernel_time": (_i, [_vp, C.c_char_p, _dp, C.POINTER(C.c_longlong)]),
    "fg_trajectory_nested": (_i, [_vp, _i, _i, _i, _d, _d, _i, _d, C.POINTER(FgTrajResult)]),
    "fg_trajectories_host_momenta_f32": (_i, [_vp, _i, _d, _d, _i, C.POINTER(C.POINTER(C.c_float)), _dp,
                                              C.POINTER(FgTrajResult)]),
    "fg_trajectories_host_momenta": (_i, [_vp, _i, _d, _d, _i, C.POINTER(_dp), _dp,
                                         C.POINTER(FgTrajResult)]),
    "fg_launch_count": (C.c_longlong, [_vp]),
    "fg_sync": (_i, [_vp]),
    "fg_set_wait_limit": (_i, [_vp, _d]),
    "fg_device_bytes": (C.c_ulonglong, [_vp]),
    "fg_action_sums_noalloc": (_i, [_vp, _vp, C.POINTER(C.c_int), _d, _vp, _vp]),
    "fg_batch_params_default": (_i, [C.POINTER(FgBatchParams)]),
    "fg_batch_create": (_i, [C.POINTER(FgBatchParams), C.POINTER(_vp)]),
    "fg_batch_destroy": (None, [_vp]),
    "fg_batch_last_error": (C.c_char_p, [_vp]),
    "fg_batch_set_gauge": (_i, [_vp, _i, _dp]),
    "fg_batch_get_gauge": (_i, [_vp, _i, _dp]),
    "fg_batch_set_momenta": (_i, [_vp, _i, _dp]),
    "fg_batch_get_momenta": (_i, [_vp, _i, _dp]),
    "fg_batch_trajectory": (_i, [_vp, _i, _d, _d, _i, _i, C.POINTER(FgTrajResult)]),
    "fg_batch_tile": (_i, [_vp, C.POINTER(_i)]),
    "fg_batch_launch_count": (C.c_longlong, [_vp]),
    "fg_batch_set_wait_limit": (_i, [_vp, _d]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libfg_lattice.so and attach signatures; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_0910_2950_gb300.build`")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class FgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def fp32_fma_rate() -> float:
    """The current device's measured FP32 FMA throughput in TFLOP/s
    (fg_fp32_fma_rate: independent FMA chains filling every SM)."""
    lib = load()
    v = C.c_double()
    st = lib.fg_fp32_fma_rate(C.byref(v))
    if st != FG_OK:
        raise FgError(st, "fg_fp32_fma_rate failed")
    return v.value


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a, shape):
    a = np.ascontiguousarray(a)
    if a.dtype == np.complex128:
        a = a.view(np.float64)
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != int(np.prod(shape)):
        raise ValueError(f"expected {int(np.prod(shape))} doubles, got {a.size}")
    return a


def _out(out, n):
    if out is None:
        return np.empty(n, dtype=np.float64)
    a = out.view(np.float64) if out.dtype == np.complex128 else out
    if a.dtype != np.float64 or not a.flags.c_contiguous or a.size != n:
        raise ValueError(f"out must be a contiguous float64 buffer of {n} doubles")
    return a.reshape(-1)


class Lattice:
    """One lattice handle (``fg_lattice*``)."""

    def __init__(self, dims, beta=6.0, kappa=0.0, precision="fp64", link_reals=18, alpha=0.1932,
                 cg_tol=1e-10, cg_tol_action=1e-12, cg_maxiter=20000, cg_delta=0.01, seed=1,
                 reunitarize=None, stream=None):
        lib = load()
        p = FgParams()
        _check(lib.fg_params_default(C.byref(p)), None)
        for i, d in enumerate(dims):
            p.dims[i] = int(d)
        p.beta, p.kappa, p.alpha = float(beta), float(kappa), float(alpha)
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p.link_reals = int(link_reals)
        p.cg_tol, p.cg_tol_action, p.cg_maxiter, p.cg_delta = cg_tol, cg_tol_action, cg_maxiter, cg_delta
        p.seed = int(seed)
        p.reunitarize = -1 if reunitarize is None else int(reunitarize)
        p.cuda_stream = stream
        self._lib = lib
        self._h = C.c_void_p()
        st = lib.fg_lattice_create(C.byref(p), C.byref(self._h))
        if st != FG_OK:
            raise FgError(st, "fg_lattice_create failed")
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        lx, ly, lz, lt = self.dims
        self.site_shape = (lt, lz, ly, lx)

    # -- lifetime
    def close(self):
        if self._h:
            self._lib.fg_lattice_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _call(self, name, *args):
        st = getattr(self._lib, name)(self._h, *args)
        if st != FG_OK:
            raise FgError(st, self._lib.fg_last_error(self._h).decode())
        return st

    # -- fields
    def set_gauge(self, u):
        a = _f64(u, (self.V, 4, 18))
        self._call("fg_set_gauge", _ptr(a))

    def get_gauge(self, out=None):
        """Links as complex128[Lt,Lz,Ly,Lx,4,3,3]; `out` (contiguous float64 or
        complex128 of the right size, e.g. pinned memory) is filled in place."""
        a = _out(out, self.V * 4 * 18)
        self._call("fg_get_gauge", _ptr(a))
        return a.reshape(-1).view(np.complex128).reshape(self.site_shape + (4, 3, 3))

    def set_momenta(self, p):
        self._call("fg_set_momenta", _ptr(_f64(p, (self.V, 4, 8))))

    def get_momenta(self, out=None):
        a = _out(out, self.V * 32)
        self._call("fg_get_momenta", _ptr(a))
        return a.reshape(self.site_shape + (4, 8))

    def refresh_momenta(self):
        self._call("fg_refresh_momenta")

    def set_pseudofermion(self, chi_even):
        self._call("fg_set_pseudofermion", _ptr(_f64(chi_even, (self.V // 2, 24))))

    def refresh_pseudofermion(self):
        self._call("fg_refresh_pseudofermion")

    # -- observables
    def force(self):
        a = np.empty(self.V * 32, dtype=np.float64)
        self._call("fg_force", _ptr(a))
        return a.reshape(self.site_shape + (4, 8))

    def action(self):
        sg, sf, t = C.c_double(), C.c_double(), C.c_double()
        self._call("fg_action", C.byref(sg), C.byref(sf), C.byref(t))
        return sg.value, sf.value, t.value

    def plaquette(self):
        x = C.c_double()
        self._call("fg_plaquette", C.byref(x))
        return x.value

    # -- molecular dynamics
    def md_step(self, integrator, dt):
        self._call("fg_md_step", INTEGRATORS[integrator], float(dt))

    def fg_step(self, dt):
        self._call("fg_fg_step", float(dt))

    def trajectory(self, integrator, dt, tau=1.0, refresh=True, u_accept=-1.0):
        r = FgTrajResult()
        self._call("fg_trajectory", INTEGRATORS[integrator], float(dt), float(tau), int(bool(refresh)),
                   float(u_accept), C.byref(r))
        return {k: getattr(r, k) for k, _ in FgTrajResult._fields_}

    def trajectory_nested(self, outer, inner, n_inner, dt, tau=1.0, refresh=True, u_accept=-1.0):
        r = FgTrajResult()
        self._call("fg_trajectory_nested", INTEGRATORS[outer], INTEGRATORS[inner], int(n_inner), float(dt),
                   float(tau), int(bool(refresh)), float(u_accept), C.byref(r))
        return {k: getattr(r, k) for k, _ in FgTrajResult._fields_}

    def trajectories_host_momenta(self, integrator, dt, tau, momenta, u_accept=None):
        """len(momenta) trajectories (refresh off), trajectory k from the host
        momenta ``momenta[k]``; uploads overlap the previous trajectory (use
        page-locked arrays for the overlap).  float32 arrays (all of them)
        are uploaded as FP32, anything else as FP64.  Returns one result dict
        each."""
        n = len(momenta)
        u = None if u_accept is None else _f64(u_accept, (n,))
        res = (FgTrajResult * max(n, 1))()
        if n > 0 and all(np.asarray(p).dtype == np.float32 for p in momenta):
            # FP32 arrays go up as they are (half the bytes)
            arrs = [np.ascontiguousarray(p, dtype=np.float32).reshape(-1) for p in momenta]
            for a in arrs:
                if a.size != self.V * 32:
                    raise ValueError(f"momenta: expected {self.V * 32} floats, got {a.size}")
            fp = C.POINTER(C.c_float)
            ptrs = (fp * n)(*[a.ctypes.data_as(fp) for a in arrs])
            self._call("fg_trajectories_host_momenta_f32", INTEGRATORS[integrator], float(dt), float(tau), n,
                       ptrs, _ptr(u) if u is not None else None, res)
        else:
            arrs = [_f64(p, (self.V, 4, 8)) for p in momenta]
            ptrs = (_dp * max(n, 1))(*[_ptr(a) for a in arrs])
            self._call("fg_trajectories_host_momenta", INTEGRATORS[integrator], float(dt), float(tau), n, ptrs,
                       _ptr(u) if u is not None else None, res)
        return [{k: getattr(r, k) for k, _ in FgTrajResult._fields_} for r in res[:n]]

    # -- fermion building blocks
    def apply_mhat(self, x_even, dagger=False):
        a = _f64(x_even, (self.V // 2, 24))
        out = np.empty(self.V // 2 * 24, dtype=np.float64)
        self._call("fg_apply_mhat", _ptr(a), _ptr(out), int(bool(dagger)))
        return out.view(np.complex128).reshape(self.V // 2, 4, 3)

    def apply_mhat_inner(self, x_even, dagger=False):
        a = _f64(x_even, (self.V // 2, 24))
        out = np.empty(self.V // 2 * 24, dtype=np.float64)
        self._call("fg_apply_mhat_inner", _ptr(a), _ptr(out), int(bool(dagger)))
        return out.view(np.complex128).reshape(self.V // 2, 4, 3)

    def cg_solve(self, b_even):
        a = _f64(b_even, (self.V // 2, 24))
        out = np.empty(self.V // 2 * 24, dtype=np.float64)
        r = FgCgResult()
        self._call("fg_cg_solve", _ptr(a), _ptr(out), C.byref(r))
        return out.view(np.complex128).reshape(self.V // 2, 4, 3), {
            k: getattr(r, k) for k, _ in FgCgResult._fields_}

    def reunitarize(self):
        self._call("fg_reunitarize")

    def random_gauge(self):
        self._call("fg_random_gauge")

    def set_rng_position(self, pos):
        self._call("fg_set_rng_position", C.c_ulonglong(int(pos)))

    # -- instrumentation
    def timing(self, on=True):
        self._call("fg_timing_enable", int(bool(on)))

    def timing_reset(self):
        self._call("fg_timing_reset")

    def kernel_time(self, cls):
        ms, n = C.c_double(), C.c_longlong()
        self._call("fg_kernel_time", cls.encode(), C.byref(ms), C.byref(n))
        return ms.value, n.value

    def launch_count(self):
        return int(self._lib.fg_launch_count(self._h))

    def set_wait_limit(self, seconds):
        self._call("fg_set_wait_limit", float(seconds))

    def sync(self):
        self._call("fg_sync")

    def device_bytes(self):
        return int(self._lib.fg_device_bytes(self._h))


class Batch:
    """Many independent pure-gauge chains advanced together (``fg_batch*``)."""

    def __init__(self, dims_list, betas, precision="fp32", link_reals=18, alpha=0.1932, tile=0,
                 use_graphs=True, seed=1, reunitarize=None, stream=None):
        lib = load()
        p = FgBatchParams()
        _check(lib.fg_batch_params_default(C.byref(p)), None)
        n = len(dims_list)
        self._dims = (C.c_int * (4 * n))(*[int(d) for dims in dims_list for d in dims])
        self._beta = (C.c_double * n)(*[float(b) for b in betas])
        p.nchains = n
        p.dims = self._dims
        p.beta = self._beta
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        p.link_reals, p.alpha, p.tile = int(link_reals), float(alpha), int(tile)
        p.use_graphs = int(bool(use_graphs))
        p.seed = int(seed)
        p.reunitarize = -1 if reunitarize is None else int(reunitarize)
        p.cuda_stream = stream
        self._lib = lib
        self._h = C.c_void_p()
        st = lib.fg_batch_create(C.byref(p), C.byref(self._h))
        if st != FG_OK:
            raise FgError(st, "fg_batch_create failed")
        self.dims = [tuple(int(x) for x in d) for d in dims_list]
        self.n = n

    def close(self):
        if self._h:
            self._lib.fg_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _call(self, name, *args):
        st = getattr(self._lib, name)(self._h, *args)
        if st != FG_OK:
            raise FgError(st, self._lib.fg_batch_last_error(self._h).decode())

    def _v(self, c):
        return int(np.prod(self.dims[c]))

    def _shape(self, c):
        lx, ly, lz, lt = self.dims[c]
        return (lt, lz, ly, lx)

    def set_gauge(self, c, u):
        self._call("fg_batch_set_gauge", int(c), _ptr(_f64(u, (self._v(c), 4, 18))))

    def get_gauge(self, c):
        a = np.empty(self._v(c) * 72, dtype=np.float64)
        self._call("fg_batch_get_gauge", int(c), _ptr(a))
        return a.view(np.complex128).reshape(self._shape(c) + (4, 3, 3))

    def set_momenta(self, c, p):
        self._call("fg_batch_set_momenta", int(c), _ptr(_f64(p, (self._v(c), 4, 8))))

    def get_momenta(self, c):
        a = np.empty(self._v(c) * 32, dtype=np.float64)
        self._call("fg_batch_get_momenta", int(c), _ptr(a))
        return a.reshape(self._shape(c) + (4, 8))

    def trajectory(self, integrator, dt, tau=1.0, refresh=True, always_accept=False):
        res = (FgTrajResult * self.n)()
        self._call("fg_batch_trajectory", INTEGRATORS[integrator], float(dt), float(tau), int(bool(refresh)),
                   int(bool(always_accept)), res)
        return [{k: getattr(r, k) for k, _ in FgTrajResult._fields_} for r in res]

    def set_wait_limit(self, seconds):
        self._call("fg_batch_set_wait_limit", float(seconds))

    def tile(self):
        t = C.c_int()
        self._call("fg_batch_tile", C.byref(t))
        return t.value

    def launch_count(self):
        return int(self._lib.fg_batch_launch_count(self._h))


def _check(st, h):
    if st != FG_OK:
        raise FgError(st, "call failed")
