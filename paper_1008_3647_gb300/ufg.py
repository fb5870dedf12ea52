"""Thin ctypes binding of libufg.so (the C ABI declared in include/ufg.h).

Argument marshalling only: every operator, solver step and reduction runs in the library's CUDA
kernels.  Vectors are torch CUDA tensors (contiguous [N_tau, N_x, N_x, N_x], float64 or float32);
their device pointers and the current CUDA stream are handed to the library.  There is no CPU
fallback: if the compiled library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libufg.so")

UFG_OK, UFG_INVALID_ARG, UFG_NOT_CONVERGED, UFG_BREAKDOWN, UFG_NONFINITE = 0, 1, 2, 3, 4
UFG_TIMEOUT, UFG_CUDA_ERROR, UFG_OOM, UFG_INTERNAL, UFG_UNSUPPORTED = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "UFG_OK", 1: "UFG_INVALID_ARG", 2: "UFG_NOT_CONVERGED", 3: "UFG_BREAKDOWN",
                4: "UFG_NONFINITE", 5: "UFG_TIMEOUT", 6: "UFG_CUDA_ERROR", 7: "UFG_OOM",
                8: "UFG_INTERNAL", 9: "UFG_UNSUPPORTED"}
UFG_FP64, UFG_FP32, UFG_MIXED, UFG_FP64_EMULATED = 0, 1, 2, 3
UFG_PC_NONE, UFG_PC_CHEB, UFG_PC_SCA, UFG_PC_WCE, UFG_PC_SCA_CHEB = 0, 1, 2, 3, 4
PC_KINDS = {"none": UFG_PC_NONE, "cheb": UFG_PC_CHEB, "sca": UFG_PC_SCA, "wce": UFG_PC_WCE,
            "sca_cheb": UFG_PC_SCA_CHEB}


class UfgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class PcParams(ctypes.Structure):
    _fields_ = [("degree", ctypes.c_int), ("eps", ctypes.c_double), ("scale", ctypes.c_double),
                ("alpha", ctypes.c_double), ("order", ctypes.c_int), ("euler", ctypes.c_int),
                ("euler_p", ctypes.c_double), ("vw_s", ctypes.c_double)]


UFG_ACCEL_NONE, UFG_ACCEL_EULER, UFG_ACCEL_EULER23, UFG_ACCEL_VANW = 0, 1, 2, 3
ACCEL = {False: 0, True: 1, 0: 0, 1: 1, 2: 2, 3: 3, "none": 0, "euler": 1, "euler23": 2,
         "vanw": 3}


class Params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("precision", ctypes.c_int),
                ("x0_given", ctypes.c_int), ("inner_tol", ctypes.c_double),
                ("check_every", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int),
                ("iterations_step", ctypes.c_int * 2), ("outer_iterations", ctypes.c_int),
                ("restarts", ctypes.c_int), ("n_M", ctypes.c_longlong),
                ("n_Mdag", ctypes.c_longlong), ("n_M1", ctypes.c_longlong),
                ("n_M1T", ctypes.c_longlong), ("n_M0inv", ctypes.c_longlong),
                ("n_M0invT", ctypes.c_longlong), ("n_sca", ctypes.c_longlong),
                ("mv_paper", ctypes.c_double), ("true_residual", ctypes.c_double),
                ("seconds", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("tile_slices", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["iterations_step"] = [self.iterations_step[0], self.iterations_step[1]]
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


class HmcStats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("accepted", ctypes.c_int), ("md_steps", ctypes.c_int),
                ("force_solves", ctypes.c_int), ("iterations", ctypes.c_longlong),
                ("H_old", ctypes.c_double), ("H_new", ctypes.c_double), ("dH", ctypes.c_double),
                ("action_old", ctypes.c_double), ("action_new", ctypes.c_double),
                ("seconds", ctypes.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        return d


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 64), ("launches", ctypes.c_longlong),
                ("total_ms", ctypes.c_double), ("bytes", ctypes.c_double)]


class Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ntau", ctypes.c_int), ("tau", ctypes.c_double),
                ("g", ctypes.c_double), ("sigma", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("x", ctypes.c_void_p)]


_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_SIGS = {
    "ufg_last_error": (ctypes.c_char_p, []),
    "ufg_version": (ctypes.c_char_p, []),
    "ufg_supported_nx": (ctypes.c_char_p, []),
    "ufg_kernel_launches": (ctypes.c_longlong, []),
    "ufg_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "ufg_measure_fma_rate": (ctypes.c_int, [ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_double)]),
    "ufg_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "ufg_wce_series_weights": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                              ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
    "ufg_lattice_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, ctypes.POINTER(_vp)]),
    "ufg_lattice_create_dim": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_int, ctypes.POINTER(_vp)]),
    "ufg_lattice_destroy": (None, [_vp]),
    "ufg_lattice_coupling": (ctypes.c_double, [_vp]),
    "ufg_lattice_check": (ctypes.c_int, [_vp, _vp]),
    "ufg_test_expire_waits": (None, [ctypes.c_int]),
    "ufg_lattice_autotune": (ctypes.c_int, [_vp, _vp]),
    "ufg_lattice_launch_shape": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                                ctypes.POINTER(ctypes.c_int)]),
    "ufg_field_create": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "ufg_field_update": (ctypes.c_int, [_vp, _vp, _vp]),
    "ufg_field_destroy": (None, [_vp]),
    "ufg_apply_M": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "ufg_apply_Mdag": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "ufg_apply_Q": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "ufg_apply_M1": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "ufg_apply_M1T": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "ufg_apply_kinetic": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "ufg_apply_M0inv": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "ufg_apply_M0invT": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "ufg_fourier": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp]),
    "ufg_apply_M_momentum": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, _vp]),
    "ufg_solver_create": (ctypes.c_int, [_vp, ctypes.POINTER(_vp)]),
    "ufg_solver_destroy": (None, [_vp]),
    "ufg_set_preconditioner": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.POINTER(PcParams)]),
    "ufg_apply_preconditioner": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int,
                                                _vp]),
    "ufg_solve_cg_normal": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.POINTER(Params),
                                           ctypes.POINTER(Stats), _vp]),
    "ufg_solve_bicgstab_two_step": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.POINTER(Params),
                                                   ctypes.POINTER(Stats), _vp]),
    "ufg_hmc_force": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(Params), ctypes.POINTER(Stats), _vp]),
    "ufg_force_from_solution": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_double, _vp]),
    "ufg_hmc_trajectory": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_double, ctypes.POINTER(Params), _vp, _vp,
                                          ctypes.POINTER(HmcStats), _vp]),
    "ufg_solve_batch": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(Problem), ctypes.c_int,
                                       ctypes.POINTER(PcParams), ctypes.POINTER(Params),
                                       ctypes.POINTER(Stats), _vp]),
    "ufg_batch_cache_clear": (None, []),
    "ufg_apply_Q_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_int, _vp, _vp, _vp, _vp]),
}
EXPORTED = tuple(_SIGS)


def load(path: str | None = None):
    """Loads the compiled library (once).  Raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError("libufg.so not found at %s: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`" % p)
        lib = ctypes.CDLL(p)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name, None)
            if fn is None:
                continue  # reported by the symbol-export test; calling it raises AttributeError
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def ufg_kernel_launches():
    return int(load().ufg_kernel_launches())


def ufg_profile_enable(on=True):
    """Per-kernel CUDA-event timing of the library's launches (direct launches, no graph replay)
    until disabled; enabling clears earlier records."""
    _check(load().ufg_profile_enable(1 if on else 0))


def ufg_measure_fma_rate(precision=UFG_FP64):
    """Measured FMA throughput of the current GPU in TFLOP/s (FP64 or FP32)."""
    v = ctypes.c_double(0.0)
    _check(load().ufg_measure_fma_rate(precision, _stream(), ctypes.byref(v)))
    return v.value


def ufg_wce_series_weights(order, euler=False, p=0.0, s=0.0):
    """The order + 1 weights of the weak-coupling series terms under acceleration `euler` (as in
    Solver.ufg_set_preconditioner); host only, no GPU needed."""
    w = (ctypes.c_double * (order + 1 if order >= 0 else 1))()
    _check(load().ufg_wce_series_weights(order, ACCEL[euler], p, s, w))
    return [w[i] for i in range(order + 1)]


def ufg_profile_read():
    """[{name, launches, total_ms, bytes, us_per_launch, gbs}] sorted by total time."""
    lib = load()
    n = ctypes.c_int(0)
    _check(lib.ufg_profile_read(None, 0, ctypes.byref(n)))
    arr = (KernelStat * max(1, n.value))()
    _check(lib.ufg_profile_read(ctypes.cast(arr, ctypes.c_void_p), n.value, ctypes.byref(n)))
    out = []
    for i in range(n.value):
        k = arr[i]
        ms = float(k.total_ms)
        out.append({"name": k.name.decode(), "launches": int(k.launches), "total_ms": ms,
                    "bytes": float(k.bytes),
                    "us_per_launch": 1e3 * ms / max(1, k.launches),
                    "gbs": float(k.bytes) / (ms * 1e-3) / 1e9 if ms > 0 else 0.0})
    return out


def _check(status):
    if status != UFG_OK:
        raise UfgError(status, load().ufg_last_error().decode())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _vec(t, shape, dtypes=(torch.float64, torch.float32), host_ok=False):
    if not isinstance(t, torch.Tensor) or not t.is_contiguous() or not (t.is_cuda or host_ok):
        raise ValueError("vectors must be contiguous CUDA tensors" +
                         (" (or host tensors)" if host_ok else ""))
    if tuple(t.shape) != tuple(shape) or t.dtype not in dtypes:
        raise ValueError("expected shape %s dtype in %s, got %s %s" % (shape, dtypes, tuple(t.shape),
                                                                       t.dtype))
    return t


class Lattice:
    """ufg_lattice: N_x^dim x N_tau lattice (dim 3 by default; 1 and 2: the lower dimensions),
    time step tau, coupling g (A = sqrt(2(e^{tau g}-1)))."""

    def __init__(self, nx, ntau, tau=0.05, g=5.0, dispersion=0, dim=3):
        lib = load()
        h = _vp()
        if dim == 3:
            _check(lib.ufg_lattice_create(nx, ntau, tau, g, dispersion, ctypes.byref(h)))
        else:
            _check(lib.ufg_lattice_create_dim(dim, nx, ntau, tau, g, dispersion, ctypes.byref(h)))
        self._h = h
        self.nx, self.ntau, self.tau, self.g, self.dispersion = nx, ntau, tau, g, dispersion
        self.dim = dim
        self.A = lib.ufg_lattice_coupling(h)

    @property
    def shape(self):
        return (self.ntau,) + (self.nx,) * self.dim

    def ufg_lattice_autotune(self):
        _check(load().ufg_lattice_autotune(self._h, _stream()))
        return {p: self.ufg_lattice_launch_shape(p) for p in (UFG_FP64, UFG_FP32)}

    def ufg_lattice_check(self):
        """Synchronises the current stream and raises UfgError(UFG_TIMEOUT) if a bounded device
        wait of a kernel launched on this lattice since the last check ran out."""
        _check(load().ufg_lattice_check(self._h, _stream()))

    def ufg_lattice_launch_shape(self, precision=UFG_FP32):
        c, s = ctypes.c_int(0), ctypes.c_int(0)
        _check(load().ufg_lattice_launch_shape(self._h, precision, ctypes.byref(c), ctypes.byref(s)))
        return c.value, s.value

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ufg_lattice_destroy(self._h)
            self._h = None


class Field:
    """ufg_field: auxiliary field sigma (CUDA float64 tensor) on a lattice."""

    def __init__(self, lattice: Lattice, sigma: torch.Tensor):
        lib = load()
        _vec(sigma, lattice.shape, (torch.float64,), host_ok=True)
        h = _vp()
        _check(lib.ufg_field_create(lattice._h, _ptr(sigma), _stream(), ctypes.byref(h)))
        self._h = h
        self.lattice = lattice

    def update(self, sigma: torch.Tensor):
        """New sigma from a CUDA tensor or a host tensor (pinned memory copies asynchronously)."""
        _vec(sigma, self.lattice.shape, (torch.float64,), host_ok=True)
        _check(load().ufg_field_update(self._h, _ptr(sigma), _stream()))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ufg_field_destroy(self._h)
            self._h = None


def _apply(name, field, x, y=None):
    _vec(x, field.lattice.shape)
    if y is None:
        y = torch.empty_like(x)
    _vec(y, field.lattice.shape, (x.dtype,))
    prec = UFG_FP64 if x.dtype == torch.float64 else UFG_FP32
    _check(getattr(load(), name)(field._h, _ptr(x), _ptr(y), prec, _stream()))
    return y


def ufg_apply_M(field, x, y=None):
    return _apply("ufg_apply_M", field, x, y)


def ufg_apply_Mdag(field, x, y=None):
    return _apply("ufg_apply_Mdag", field, x, y)


def ufg_apply_Q(field, x, y=None):
    return _apply("ufg_apply_Q", field, x, y)


def ufg_apply_M1(field, x, y=None):
    return _apply("ufg_apply_M1", field, x, y)


def ufg_apply_M1T(field, x, y=None):
    return _apply("ufg_apply_M1T", field, x, y)


def ufg_apply_kinetic(field, x, y=None):
    return _apply("ufg_apply_kinetic", field, x, y)


def ufg_apply_M0inv(field, x, y=None):
    return _apply("ufg_apply_M0inv", field, x, y)


def ufg_apply_M0invT(field, x, y=None):
    return _apply("ufg_apply_M0invT", field, x, y)


def _apply_flag(name, field, x, flag, y=None):
    _vec(x, field.lattice.shape)
    if y is None:
        y = torch.empty_like(x)
    _vec(y, field.lattice.shape, (x.dtype,))
    prec = UFG_FP64 if x.dtype == torch.float64 else UFG_FP32
    _check(getattr(load(), name)(field._h, _ptr(x), _ptr(y), prec, int(flag), _stream()))
    return y


def ufg_fourier(field, x, inverse=False, y=None):
    """Per-slice orthogonal real Fourier transform (inverse: its transpose)."""
    return _apply_flag("ufg_fourier", field, x, inverse, y)


def ufg_apply_M_momentum(field, x, transpose=False, y=None, emulated=False):
    """M (or M^T) in the momentum basis: F M F^T x per slice-stacked vector.  emulated=True (FP64
    vectors only): double-float arithmetic on the FP32 pipe."""
    if not emulated:
        return _apply_flag("ufg_apply_M_momentum", field, x, transpose, y)
    _vec(x, field.lattice.shape, (torch.float64,))
    y = torch.empty_like(x) if y is None else y
    _vec(y, field.lattice.shape, (torch.float64,))
    _check(load().ufg_apply_M_momentum(field._h, _ptr(x), _ptr(y), UFG_FP64_EMULATED,
                                       int(bool(transpose)), _stream()))
    return y


def _pc_params(kind, degree=16, eps=0.0, scale=0.0, alpha=2.0, order=2, euler=False, p=0.5,
               s=1.0):
    """euler: False/True, 0..3 or "none" / "euler" / "euler23" / "vanw" (ufg_accel); p: Euler
    parameter; s: van Wijngaarden parameter."""
    accel = ACCEL[euler] if euler in ACCEL else int(euler)  # unknown values: the library rejects
    return PC_KINDS[kind], PcParams(degree, eps, scale, alpha, order, accel, p, s)


def _params(tol=1e-10, maxit=20000, precision=UFG_FP64, x0_given=False, inner_tol=1e-5,
            check_every=8):
    return Params(tol, maxit, precision, int(bool(x0_given)), inner_tol, check_every)


class Solver:
    """ufg_solver: solver workspace for one lattice plus the preconditioner selection."""

    def __init__(self, lattice: Lattice):
        h = _vp()
        _check(load().ufg_solver_create(lattice._h, ctypes.byref(h)))
        self._h = h
        self.lattice = lattice

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.ufg_solver_destroy(self._h)
            self._h = None

    def ufg_set_preconditioner(self, kind="none", **kw):
        k, p = _pc_params(kind, **kw)
        _check(load().ufg_set_preconditioner(self._h, k, ctypes.byref(p)))

    def ufg_apply_preconditioner(self, field, r, z=None, transpose=False):
        """transpose: False / 0 -> P, True / 1 -> P^T, 2 -> the CG (normal-equation) form."""
        _vec(r, self.lattice.shape)
        z = torch.empty_like(r) if z is None else z
        prec = UFG_FP64 if r.dtype == torch.float64 else UFG_FP32
        _check(load().ufg_apply_preconditioner(self._h, field._h, _ptr(r), _ptr(z),
                                               int(transpose), prec, _stream()))
        return z

    def _solve(self, name, field, b, x, kw):
        """b, x: CUDA tensors or host tensors (host buffers are staged by the library)."""
        _vec(b, self.lattice.shape, (torch.float64,), host_ok=True)
        if x is not None:
            _vec(x, self.lattice.shape, (torch.float64,), host_ok=True)
        lib = load()
        p = _params(**kw)
        st = Stats()
        if x is None:
            x = torch.zeros_like(b)
        status = getattr(lib, name)(self._h, field._h, ctypes.c_void_p(b.data_ptr()),
                                    ctypes.c_void_p(x.data_ptr()), ctypes.byref(p),
                                    ctypes.byref(st), _stream())
        if status not in (UFG_OK, UFG_NOT_CONVERGED, UFG_BREAKDOWN, UFG_NONFINITE):
            _check(status)
        return x, st.as_dict()

    def ufg_solve_cg_normal(self, field, b, x=None, **kw):
        return self._solve("ufg_solve_cg_normal", field, b, x, kw)

    def ufg_solve_bicgstab_two_step(self, field, b, x=None, **kw):
        return self._solve("ufg_solve_bicgstab_two_step", field, b, x, kw)

    def ufg_hmc_force(self, field, phi, **kw):
        lib = load()
        p = _params(**kw)
        st = Stats()
        dS = torch.empty_like(phi)
        X = torch.empty_like(phi)
        S = ctypes.c_double(0.0)
        status = lib.ufg_hmc_force(self._h, field._h, _ptr(phi), _ptr(dS), _ptr(X),
                                   ctypes.byref(S), ctypes.byref(p), ctypes.byref(st), _stream())
        if status not in (UFG_OK, UFG_NOT_CONVERGED):
            _check(status)
        return dS, X, S.value, st.as_dict()

    def ufg_force_from_solution(self, field, X, dS=None, scale=1.0):
        dS = torch.empty_like(X) if dS is None else dS
        _check(load().ufg_force_from_solution(self._h, field._h, _ptr(X), _ptr(dS), float(scale),
                                              _stream()))
        return dS

    def ufg_hmc_trajectory(self, field, eta, pi0, u, n_steps, dt, **kw):
        """One HMC trajectory (heat bath phi = M^T eta, leapfrog, Metropolis against u);
        returns (sigma, pi, stats) with sigma the field's configuration afterwards."""
        shape = self.lattice.shape
        for t in (eta, pi0):
            _vec(t, shape, (torch.float64,))
        p = _params(**kw)
        st = HmcStats()
        sigma = torch.empty_like(eta)
        pi = torch.empty_like(eta)
        status = load().ufg_hmc_trajectory(self._h, field._h, _ptr(eta), _ptr(pi0), float(u),
                                           int(n_steps), float(dt), ctypes.byref(p), _ptr(sigma),
                                           _ptr(pi), ctypes.byref(st), _stream())
        if status not in (UFG_OK, UFG_NOT_CONVERGED, UFG_BREAKDOWN, UFG_NONFINITE):
            _check(status)
        return sigma, pi, st.as_dict()

    def ufg_pseudofermion_action(self, field, phi, **kw):
        """(S, X): S = phi^T Q^{-1} phi and X = Q^{-1} phi from ufg_hmc_force without the force."""
        lib = load()
        p = _params(**kw)
        st = Stats()
        X = torch.empty_like(phi)
        S = ctypes.c_double(0.0)
        status = lib.ufg_hmc_force(self._h, field._h, _ptr(phi), None, _ptr(X), ctypes.byref(S),
                                   ctypes.byref(p), ctypes.byref(st), _stream())
        if status not in (UFG_OK, UFG_NOT_CONVERGED):
            _check(status)
        return S.value, X, st.as_dict()


def ufg_test_expire_waits(launches):
    """Test hook: the next `launches` TMA-staged slice launches each run one bounded wait that is
    made to run out (results stay correct; the status becomes UFG_TIMEOUT)."""
    load().ufg_test_expire_waits(int(launches))


def ufg_batch_cache_clear():
    load().ufg_batch_cache_clear()


def ufg_solve_batch(problems, pc_kind="wce", pc=None, **kw):
    """problems: list of dicts with nx, ntau, tau, g, sigma, b, x (float64 tensors, CUDA or host
    memory; host tensors are staged by the library)."""
    lib = load()
    arr = (Problem * len(problems))()
    for i, pr in enumerate(problems):
        arr[i] = Problem(pr["nx"], pr["ntau"], pr.get("tau", 0.05), pr.get("g", 5.0),
                         pr["sigma"].data_ptr(), pr["b"].data_ptr(), pr["x"].data_ptr())
    k, pcp = _pc_params(pc_kind, **(pc or {}))
    p = _params(**kw)
    stats = (Stats * len(problems))()
    status = lib.ufg_solve_batch(len(problems), arr, k, ctypes.byref(pcp), ctypes.byref(p), stats,
                                 _stream())
    if status not in (UFG_OK, UFG_NOT_CONVERGED, UFG_BREAKDOWN, UFG_NONFINITE):
        _check(status)  # per-problem outcomes are in the returned stats
    return [s.as_dict() for s in stats]


class PseudofermionAction(torch.autograd.Function):
    """S(sigma) = phi^T (M^T M)^{-1} phi with backward dS/dsigma from the adjoint force kernel.

    forward solves X = Q^{-1} phi (two-step BiCGStab); backward reuses the saved X and
    recomputes Y = M X inside the force kernel's pipeline instead of storing intermediates."""

    @staticmethod
    def forward(ctx, sigma, phi, solver, solve_kw):
        field = Field(solver.lattice, sigma.detach().contiguous())
        S, x, st = solver.ufg_pseudofermion_action(field, phi, **(solve_kw or {}))
        ctx.save_for_backward(x)
        ctx.field = field
        ctx.solver = solver
        ctx.stats = st
        return torch.tensor(S, dtype=torch.float64, device=sigma.device)

    @staticmethod
    def backward(ctx, gS):
        (x,) = ctx.saved_tensors
        dS = ctx.solver.ufg_force_from_solution(ctx.field, x, scale=float(gS))
        return dS, None, None, None


def ufg_apply_Q_noalloc(nx, ntau, tau, g, sigma, x, y, dispersion=0):
    """y = M^T M x (FP64) through the allocation-free entry point: for callers that cannot
    allocate device memory where they need the operator.  Limited to N_x^3 N_tau <= 2^20 sites;
    calls that overlap on the GPU race on the library's static scratch."""
    shape = (ntau, nx, nx, nx)
    for t in (sigma, x, y):
        _vec(t, shape, (torch.float64,))
    _check(load().ufg_apply_Q_noalloc(nx, ntau, tau, g, dispersion, _ptr(sigma), _ptr(x), _ptr(y),
                                      _stream()))
    return y
