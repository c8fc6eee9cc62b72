"""Python binding of librsv (ctypes), one function per C-ABI entry point, same names.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Buffers are torch CUDA tensors (their data_ptr() is passed) or raw
integer device pointers; the operator's stream is torch's current stream at
creation unless one is given.  If librsv.so is missing or cannot be loaded,
`load()` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librsv.so")

RSV_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSTABLE", 3: "NOT_COMMENSURATE", 4: "DIVERGED", 5: "TIMEOUT",
          6: "OOM", 7: "CUDA", 8: "STATE"}
RSV_OP_GL1D, RSV_OP_DENSE, RSV_OP_ADR2D, RSV_OP_ADV3D = 0, 1, 2, 3
RSV_PREC_FP64, RSV_PREC_FP32, RSV_PREC_BF16_STATE = 0, 1, 2
RSV_SSRM, RSV_TRM = 0, 1
RSV_SCHEME_RK4, RSV_SCHEME_CN = 0, 1
RSV_INTERP_C0, RSV_INTERP_C1, RSV_INTERP_C2 = 0, 1, 2
_INTERP = {"c0": RSV_INTERP_C0, "c1": RSV_INTERP_C1, "c2": RSV_INTERP_C2}


class RsvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class rsv_operator_desc(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32), ("precision", ctypes.c_int32), ("dt", ctypes.c_double),
        ("n_instances", ctypes.c_int32), ("gl_n", ctypes.POINTER(ctypes.c_int32)),
        ("gl_mu0", ctypes.POINTER(ctypes.c_double)), ("x0", ctypes.c_double), ("x1", ctypes.c_double),
        ("nu_re", ctypes.c_double), ("nu_im", ctypes.c_double), ("gamma_re", ctypes.c_double),
        ("gamma_im", ctypes.c_double), ("mu_shift", ctypes.c_double), ("mu2", ctypes.c_double),
        ("dense_n", ctypes.c_int32), ("dense_a", ctypes.POINTER(ctypes.c_double)),
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
        ("visc", ctypes.c_double), ("kappa", ctypes.c_double), ("jet_delta", ctypes.c_double),
        ("sponge_amp", ctypes.c_double), ("sponge_cells", ctypes.c_int32),
        ("delta0", ctypes.c_double), ("delta1", ctypes.c_double),
        ("mu1", ctypes.c_double), ("scheme", ctypes.c_int32),
    ]


class rsv_march_opts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("n_transient_windows", ctypes.c_int32),
                ("tail_steps", ctypes.c_int64), ("tile_steps", ctypes.c_int32), ("group_vectors", ctypes.c_int32),
                ("tail_tol", ctypes.c_double), ("decay_tol", ctypes.c_double), ("decay_max_steps", ctypes.c_int64),
                ("decay_seed", ctypes.c_uint64)]


class rsv_series_opts(ctypes.Structure):
    _fields_ = [("every", ctypes.c_int32), ("interp", ctypes.c_int32), ("tail_tol", ctypes.c_double)]


class rsv_trm_opts(ctypes.Structure):
    _fields_ = [("series", rsv_series_opts), ("n_iter", ctypes.c_int32), ("filter_order", ctypes.c_int32),
                ("n_snap_max", ctypes.c_int64)]


_lib = None
_ENTRY_POINTS = {
    "rsv_create_operator": (ctypes.c_int, [ctypes.POINTER(rsv_operator_desc), ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_void_p)]),
    "rsv_destroy_operator": (None, [ctypes.c_void_p]),
    "rsv_operator_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "rsv_instance_range": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                          ctypes.POINTER(ctypes.c_int64)]),
    "rsv_set_frequencies": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                           ctypes.c_double, ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_double)]),
    "rsv_march_direct": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                        ctypes.POINTER(rsv_march_opts), ctypes.c_void_p]),
    "rsv_march_adjoint": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.POINTER(rsv_march_opts), ctypes.c_void_p]),
    "rsv_march_direct_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                             ctypes.POINTER(rsv_march_opts), ctypes.c_void_p]),
    "rsv_march_adjoint_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                              ctypes.POINTER(rsv_march_opts), ctypes.c_void_p]),
    "rsv_march_direct_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                               ctypes.POINTER(rsv_march_opts), ctypes.c_void_p]),
    "rsv_gains_modes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.POINTER(rsv_march_opts),
                                       ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_void_p]),
    "rsv_gains_modes_seeded": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_uint64, ctypes.POINTER(rsv_march_opts),
                                              ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_void_p]),
    "rsv_set_weights": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]),
    "rsv_decay_probe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_int64,
                                       ctypes.c_uint64, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_double)]),
    "rsv_refine_gains": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.POINTER(rsv_march_opts), ctypes.POINTER(ctypes.c_double),
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "rsv_arnoldi_gains": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(rsv_march_opts), ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "rsv_orthonormalize": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_double)]),
    "rsv_apply_operator": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_void_p]),
    "rsv_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(rsv_march_opts),
                                    ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
    "rsv_series_march": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                        ctypes.POINTER(rsv_series_opts), ctypes.c_void_p, ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "rsv_series_fourier": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                          ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                          ctypes.c_int32, ctypes.c_void_p]),
    "rsv_series_filter": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_void_p]),
    "rsv_fir_design": (ctypes.c_int, [ctypes.c_int32, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_double)]),
    "rsv_trm_power_iteration": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                               ctypes.POINTER(ctypes.c_double), ctypes.c_int32,
                                               ctypes.POINTER(rsv_trm_opts), ctypes.POINTER(ctypes.c_double),
                                               ctypes.c_void_p]),
    "rsv_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "rsv_profile_reset": (ctypes.c_int, [ctypes.c_void_p]),
    "rsv_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                        ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]),
    "rsv_describe": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int32]),
    "rsv_last_error": (ctypes.c_char_p, []),
    "rsv_version": (ctypes.c_char_p, []),
}


def load(path: str = LIB_PATH):
    """Load librsv.so (built by paper_2008_10904_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librsv.so not built at {path}: run paper_2008_10904_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _ENTRY_POINTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_ENTRY_POINTS)


def _check(status: int):
    if status != RSV_OK:
        raise RsvError(status, _lib.rsv_last_error().decode())


def _ptr(x) -> int:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("device buffers must be contiguous CUDA tensors")
        return x.data_ptr()
    raise TypeError(type(x))


def _opts(variant="ssrm", n_transient_windows=0, tail_steps=0, tile_steps=0, tail_tol=0.0, decay_tol=0.0,
          decay_max_steps=0, decay_seed=0, group_vectors=0):
    return rsv_march_opts(RSV_SSRM if variant == "ssrm" else RSV_TRM, int(n_transient_windows),
                          int(tail_steps), int(tile_steps), int(group_vectors), float(tail_tol), float(decay_tol),
                          int(decay_max_steps), int(decay_seed))


def _host_ptr(x) -> int:
    """Address of a host buffer: a CPU torch tensor (pinned for asynchronous copies) or a numpy array."""
    if hasattr(x, "data_ptr"):
        if x.is_cuda or not x.is_contiguous():
            raise ValueError("host buffers must be contiguous CPU tensors")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("host buffers must be C-contiguous")
        return x.ctypes.data
    raise TypeError(type(x))


class Operator:
    """Handle plus the host arrays its descriptor points to."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def __int__(self):
        return self.handle.value


def rsv_create_operator(desc: rsv_operator_desc, stream=None, keep=()) -> Operator:
    load()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    h = ctypes.c_void_p()
    _check(_lib.rsv_create_operator(ctypes.byref(desc), ctypes.c_void_p(stream), ctypes.byref(h)))
    return Operator(h, keep)


def rsv_destroy_operator(op: Operator):
    if op is not None and op.handle:
        _lib.rsv_destroy_operator(op.handle)
        op.handle = ctypes.c_void_p()


def rsv_operator_info(op: Operator):
    n, ni, rs = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.rsv_operator_info(op.handle, ctypes.byref(n), ctypes.byref(ni), ctypes.byref(rs)))
    return n.value, ni.value, bool(rs.value)


def rsv_instance_range(op: Operator, i: int):
    o, l = ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.rsv_instance_range(op.handle, i, ctypes.byref(o), ctypes.byref(l)))
    return o.value, l.value


def rsv_set_frequencies(op: Operator, omegas, dw: float = 0.0):
    om = np.ascontiguousarray(np.asarray(omegas, dtype=np.float64))
    nt, h = ctypes.c_int64(), ctypes.c_double()
    _check(_lib.rsv_set_frequencies(op.handle, om.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(om),
                                    float(dw), ctypes.byref(nt), ctypes.byref(h)))
    return nt.value, h.value


def rsv_march_direct(op: Operator, f_hat, k: int, y_hat, **opts):
    o = _opts(**opts)
    _check(_lib.rsv_march_direct(op.handle, _ptr(f_hat), int(k), ctypes.byref(o), _ptr(y_hat)))


def rsv_march_adjoint(op: Operator, y_hat, k: int, w_hat, **opts):
    o = _opts(**opts)
    _check(_lib.rsv_march_adjoint(op.handle, _ptr(y_hat), int(k), ctypes.byref(o), _ptr(w_hat)))


def rsv_march_direct_host(op: Operator, f_hat_host, k: int, y_hat, **opts):
    """Direct march of a host input block (copies overlapped with the march, per vector group)."""
    o = _opts(**opts)
    _check(_lib.rsv_march_direct_host(op.handle, _host_ptr(f_hat_host), int(k), ctypes.byref(o), _ptr(y_hat)))


def rsv_march_adjoint_host(op: Operator, y_hat_host, k: int, w_hat, **opts):
    o = _opts(**opts)
    _check(_lib.rsv_march_adjoint_host(op.handle, _host_ptr(y_hat_host), int(k), ctypes.byref(o), _ptr(w_hat)))


def rsv_march_direct_static(op: Operator, f_hat, k: int, y_hat, **opts):
    """rsv_march_direct with its scratch in the library's static device array (allocates nothing)."""
    o = _opts(**opts)
    _check(_lib.rsv_march_direct_static(op.handle, _ptr(f_hat), int(k), ctypes.byref(o), _ptr(y_hat)))


def rsv_gains_modes(op: Operator, omega_block, k: int, n_power_iter: int, n_modes: int, gains: np.ndarray,
                    forcing_modes=None, response_modes=None, **opts):
    """gains: host float64 array [n_instances][n_omega][n_modes], filled in place."""
    if gains.dtype != np.float64 or not gains.flags.c_contiguous:
        raise ValueError("gains must be a C-contiguous float64 array")
    o = _opts(**opts)
    _check(_lib.rsv_gains_modes(op.handle, _ptr(omega_block), int(k), int(n_power_iter), int(n_modes),
                                ctypes.byref(o), gains.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                _ptr(forcing_modes), _ptr(response_modes)))
    return gains


def rsv_gains_modes_seeded(op: Operator, k: int, n_power_iter: int, n_modes: int, seed: int, gains: np.ndarray,
                           forcing_modes=None, response_modes=None, **opts):
    """Randomized SVD from a library-drawn seeded Gaussian test block; gains filled in place."""
    if gains.dtype != np.float64 or not gains.flags.c_contiguous:
        raise ValueError("gains must be a C-contiguous float64 array")
    o = _opts(**opts)
    _check(_lib.rsv_gains_modes_seeded(op.handle, int(k), int(n_power_iter), int(n_modes), int(seed), ctypes.byref(o),
                                       gains.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(forcing_modes),
                                       _ptr(response_modes)))
    return gains


def rsv_set_weights(op: Operator, b=None, c=None, w_f=None, w_y=None):
    """Diagonal forcing / observation matrices and metrics (host arrays of n doubles, None = identity)."""
    arrs = [None if x is None else np.ascontiguousarray(np.asarray(x, dtype=np.float64)) for x in (b, c, w_f, w_y)]
    ptrs = [None if x is None else x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for x in arrs]
    _check(_lib.rsv_set_weights(op.handle, *ptrs))


def rsv_decay_probe(op: Operator, tol: float, max_steps: int, seed: int = 0, check_every: int = 0,
                    adjoint: bool = False):
    """(steps, ratio) of the decay run; raises RsvError (UNSTABLE) for a growing or non-decaying system."""
    st, r = ctypes.c_int64(), ctypes.c_double()
    _check(_lib.rsv_decay_probe(op.handle, int(bool(adjoint)), float(tol), int(max_steps), int(seed),
                                int(check_every), ctypes.byref(st), ctypes.byref(r)))
    return st.value, r.value


def rsv_refine_gains(op: Operator, basis, k: int, n_modes: int, gains: np.ndarray, forcing_modes=None,
                     response_modes=None, **opts):
    """Rayleigh-Ritz refinement on `basis`; gains: host float64 [n_instances][n_omega][n_modes], filled in place."""
    if gains.dtype != np.float64 or not gains.flags.c_contiguous:
        raise ValueError("gains must be a C-contiguous float64 array")
    o = _opts(**opts)
    _check(_lib.rsv_refine_gains(op.handle, _ptr(basis), int(k), int(n_modes), ctypes.byref(o),
                                 gains.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(forcing_modes),
                                 _ptr(response_modes)))
    return gains


def rsv_arnoldi_gains(op: Operator, f0, m: int, n_modes: int, gains: np.ndarray, forcing_modes=None,
                      response_modes=None, **opts):
    """Arnoldi gains from start vectors f0 [n_omega][1][n]; gains: host float64 [n_instances][n_omega][n_modes]."""
    if gains.dtype != np.float64 or not gains.flags.c_contiguous:
        raise ValueError("gains must be a C-contiguous float64 array")
    o = _opts(**opts)
    _check(_lib.rsv_arnoldi_gains(op.handle, _ptr(f0), int(m), int(n_modes), ctypes.byref(o),
                                  gains.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(forcing_modes),
                                  _ptr(response_modes)))
    return gains


def rsv_orthonormalize(op: Operator, block, k: int, r_factor: np.ndarray | None = None):
    """CholeskyQR2 of `block` in place; r_factor: optional host complex128 [n_omega][n_instances][k][k]."""
    rp = None
    if r_factor is not None:
        if r_factor.dtype != np.complex128 or not r_factor.flags.c_contiguous:
            raise ValueError("r_factor must be a C-contiguous complex128 array")
        rp = r_factor.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(_lib.rsv_orthonormalize(op.handle, _ptr(block), int(k), rp))
    return r_factor


def rsv_apply_operator(op: Operator, x, k: int, adjoint: bool, y):
    _check(_lib.rsv_apply_operator(op.handle, _ptr(x), int(k), int(bool(adjoint)), _ptr(y)))


def rsv_autotune(op: Operator, f_hat, k: int, **opts):
    """Measured (tile length, vector group) for marches of k vectors; kept in the operator."""
    o = _opts(**opts)
    t, g = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.rsv_autotune(op.handle, _ptr(f_hat), int(k), ctypes.byref(o), ctypes.byref(t), ctypes.byref(g)))
    return t.value, g.value


def _f64(x):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _series_opts(every=1, interp="c2", tail_tol=0.0):
    return rsv_series_opts(int(every), _INTERP[interp] if isinstance(interp, str) else int(interp), float(tail_tol))


def rsv_series_march(op: Operator, adjoint: bool, k: int, out, n_out_max: int, init=None, forcing=None,
                     n_in: int = 0, reverse_in: bool = False, **opts):
    """One series-driven run (device series [n][k][n_points]); returns (n_out, stops[k])."""
    o = _series_opts(**opts)
    n_out = ctypes.c_int64()
    stops = np.zeros(k, dtype=np.int64)
    _check(_lib.rsv_series_march(op.handle, int(bool(adjoint)), int(k), _ptr(init), _ptr(forcing), int(n_in),
                                 int(bool(reverse_in)), ctypes.byref(o), _ptr(out), int(n_out_max),
                                 ctypes.byref(n_out), stops.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return n_out.value, stops


def rsv_series_fourier(op: Operator, series, n_snap: int, k: int, d: float, t0: float, omegas, out):
    om, omp = _f64(omegas)
    _check(_lib.rsv_series_fourier(op.handle, _ptr(series), int(n_snap), int(k), float(d), float(t0), omp,
                                   len(om), _ptr(out)))


def rsv_series_filter(op: Operator, x, n_in: int, k: int, taps, out, reverse_taps: bool = False):
    """taps: complex [k][order + 1] (host)."""
    t = np.ascontiguousarray(np.asarray(taps, dtype=np.complex128).reshape(k, -1))
    _check(_lib.rsv_series_filter(op.handle, _ptr(x), int(n_in), int(k),
                                  t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), t.shape[1] - 1,
                                  int(bool(reverse_taps)), _ptr(out)))


def rsv_fir_design(order: int, d: float, w_pts, amp) -> np.ndarray:
    """Complex taps [order + 1] of the frequency-sampling design (host computation)."""
    w, wp = _f64(w_pts)
    a, ap = _f64(amp)
    taps = np.zeros(order + 1, dtype=np.complex128)
    _check(_lib.rsv_fir_design(int(order), float(d), wp, ap, len(w),
                               taps.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return taps


def rsv_trm_power_iteration(op: Operator, f0, k: int, omegas, n_iter: int, n_snap_max: int, filter_order: int = 0,
                            w_hat=None, **series_opts):
    """TRM power iteration; returns the gain estimates [n_iter][n_omega][k] (host)."""
    om, omp = _f64(omegas)
    o = rsv_trm_opts(_series_opts(**series_opts), int(n_iter), int(filter_order), int(n_snap_max))
    gains = np.zeros((n_iter, len(om), k))
    _check(_lib.rsv_trm_power_iteration(op.handle, _ptr(f0), int(k), omp, len(om), ctypes.byref(o),
                                        gains.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(w_hat)))
    return gains


PROFILE_CATEGORIES = ("synthesis", "march", "analysis", "glue")


def rsv_profile_enable(op: Operator, enable: bool):
    _check(_lib.rsv_profile_enable(op.handle, int(bool(enable))))


def rsv_profile_reset(op: Operator):
    _check(_lib.rsv_profile_reset(op.handle))


def rsv_profile_read(op: Operator, category: int):
    """(bracketed groups, kernels launched, summed event ms) of one category."""
    g, n, ms = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    _check(_lib.rsv_profile_read(op.handle, int(category), ctypes.byref(g), ctypes.byref(n), ctypes.byref(ms)))
    return g.value, n.value, ms.value


def rsv_describe(op: Operator) -> str:
    buf = ctypes.create_string_buffer(512)
    _check(_lib.rsv_describe(op.handle, buf, 512))
    return buf.value.decode()


def rsv_last_error() -> str:
    load()
    return _lib.rsv_last_error().decode()


def rsv_version() -> str:
    load()
    return _lib.rsv_version().decode()


# ---------------------------------------------------------------------------
# Descriptor marshalling from the workload parameter objects
# ---------------------------------------------------------------------------
def desc_for(system, dt: float, precision: int, scheme: int = RSV_SCHEME_RK4):
    """rsv_operator_desc for a workloads.GL1D / Dense / ADR2D / ADV3D object.

    Returns (desc, keep) where `keep` holds the host arrays the descriptor
    points to (they must stay alive until rsv_create_operator returns).
    """
    d = rsv_operator_desc()
    d.precision = precision
    d.dt = float(dt)
    d.scheme = int(scheme)
    keep = []
    name = type(system).__name__
    if name == "GL1D":
        d.kind = RSV_OP_GL1D
        n = np.ascontiguousarray(np.asarray(system.n, dtype=np.int32))
        mu0 = np.ascontiguousarray(np.asarray(system.mu0, dtype=np.float64))
        keep += [n, mu0]
        d.n_instances = len(n)
        d.gl_n = n.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        d.gl_mu0 = mu0.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.x0, d.x1 = system.x0, system.x1
        d.nu_re, d.nu_im = system.nu.real, system.nu.imag
        d.gamma_re, d.gamma_im = system.gamma.real, system.gamma.imag
        d.mu_shift, d.mu2 = system.mu_shift, system.mu2
        d.mu1 = getattr(system, "mu1", 0.0)
    elif name == "Dense":
        raise ValueError("a dense system needs its matrix: use desc_dense")
    elif name == "ADR2D":
        d.kind = RSV_OP_ADR2D
        d.nx, d.ny = system.nx, system.ny
        d.lx, d.ly = system.lx, system.ly
        d.visc, d.kappa, d.jet_delta = system.visc, system.kappa, system.jet_delta
        d.sponge_cells, d.sponge_amp = system.sponge_cells, system.sponge_amp
    elif name == "ADV3D":
        d.kind = RSV_OP_ADV3D
        d.nx, d.ny, d.nz = system.nx, system.ny, system.nz
        d.lx, d.ly, d.lz = system.lx, system.ly, system.lz
        d.visc, d.delta0, d.delta1 = system.visc, system.delta0, system.delta1
    else:
        raise ValueError(name)
    return d, keep


def desc_dense(a: np.ndarray, dt: float, precision: int):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    d = rsv_operator_desc()
    d.kind = RSV_OP_DENSE
    d.precision = precision
    d.dt = float(dt)
    d.dense_n = a.shape[0]
    d.dense_a = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return d, [a]


def create_for_workload(w, precision: int, stream=None, dense_matrix=None, scheme: int = RSV_SCHEME_RK4) -> Operator:
    """Create an operator for a workloads.Workload and set its frequencies."""
    if type(w.system).__name__ == "Dense":
        d, keep = desc_dense(dense_matrix, w.dt, precision)
        d.scheme = int(scheme)
    else:
        d, keep = desc_for(w.system, w.dt, precision, scheme)
    op = rsv_create_operator(d, stream, keep)
    rsv_set_frequencies(op, w.omegas)
    return op


def march_opts_for(w, tile_steps: int = 0) -> dict:
    return dict(variant=w.variant, n_transient_windows=w.n_transient_windows, tail_steps=w.tail_steps,
                tile_steps=tile_steps)
