"""Thin ctypes binding of the C ABI (``include/ssl_gsvd_music.h``).

Argument marshalling only: every step of the hot path runs in the CUDA
library.  Tensors are torch tensors (complex64 for complex data, float32,
int32); device tensors are passed as device pointers, CPU tensors (used only
by ``localize``'s host-buffer form) as host pointers.  The library must have
been built (``paper_2504_03373_gb300.build.build()``); there is no fallback.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

from .build import LIB as LIB_PATH

SSL_OK = 0
STATUS_NAMES = {
    0: "SSL_OK", 1: "SSL_E_INVALID_ARG", 2: "SSL_E_NOT_PD", 3: "SSL_E_NO_CONVERGENCE",
    4: "SSL_E_NONFINITE", 5: "SSL_E_OOM", 6: "SSL_E_ADMISSION", 7: "SSL_E_TIMEOUT",
    8: "SSL_E_CUDA", 9: "SSL_E_UNSUPPORTED", 10: "SSL_E_CAPACITY",
}
FORM = {"abs": 0, "sq": 1}
ANGLES = {"f64": 0, "f32": 1}
PRECISION = {"fp32": 0, "tf32": 1, "bf16": 2, "tf32x3": 3}
FLAG_NOT_PD, FLAG_NO_CONVERGENCE, FLAG_NONFINITE, FLAG_TIMEOUT, FLAG_BOUNDS = 1, 2, 4, 8, 16

# (name, argtypes) of every exported entry point; the CPU tests check that the
# library exports exactly what the header declares.
_P, _I, _U, _S = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_size_t
SIGNATURES = {
    "ssl_create": [ctypes.POINTER(_P), _I],
    "ssl_destroy": [_P],
    "ssl_last_error": [_P, ctypes.c_char_p, _S],
    "ssl_device_flags": [_P, _P, ctypes.POINTER(_U)],
    "ssl_set_wait_limit": [_P, ctypes.c_uint64],
    "ssl_set_test_stall": [_P, _I],
    "ssl_correlate": [_P, _P, _I, _I, _I, _I, _P, _P],
    "ssl_noise_inverse": [_P, _P, _I, _I, _P, _P, _P],
    "ssl_gsvd": [_P, _P, _P, _I, _I, _I, _P, _P, _P, _P, _P],
    "ssl_gsvd_kinv": [_P, _P, _P, _I, _I, _I, _P, _P, _P, _P, _P, _P],
    "ssl_gsvd_noalloc": [_P, _P, _I, _I, _I, _P, _P, _P, _P, _P],
    "ssl_sevd": [_P, _P, _I, _I, _I, _P, _P, _P, _P, _P],
    "ssl_gevd": [_P, _P, _P, _I, _I, _I, _P, _P, _P, _P, _P],
    "ssl_steering_create": [_P, _P, _I, _I, _I, ctypes.POINTER(_P)],
    "ssl_steering_destroy": [_P],
    "ssl_steering_set_search_range": [_P, _P],
    "ssl_steering_set_neighbours": [_P, _P, _P, _I],
    "ssl_steering_create_analytic": [_P, _P, _P, _P, ctypes.c_float, _I, _I, _I,
                                     ctypes.POINTER(_P)],
    "ssl_peaks_nbr": [_P, _P, _I, _P, _I, _P, _P, _P],
    "ssl_music_spectrum": [_P, _P, _I, _I, _I, _I, _P, _I, _I, _P, _P, _P],
    "ssl_peaks": [_P, _P, _I, _I, _I, _I, _P, _P, _P],
    "ssl_localize": [_P, _P, _I, _P, _P, _P, _P, _P, _P, _P],
    "ssl_localize_kinv": [_P, _P, _I, _P, _P, _P, _P, _P, _P, _P],
    "ssl_gsvd_f64": [_P, _P, _P, _I, _I, _I, _P, _P, _P, _P, _P, _P],
    "ssl_localize_f64": [_P, _P, _I, _P, _P, _P, _P, _P, _P, _P],
    "ssl_now_ns": [ctypes.POINTER(ctypes.c_uint64)],
    "ssl_server_create": [_P, _S, _I, ctypes.POINTER(_P)],
    "ssl_server_destroy": [_P],
    "ssl_session_create": [_P, _P, _P, _P, ctypes.POINTER(_P)],
    "ssl_session_destroy": [_P],
    "ssl_session_state_size": [_P, ctypes.POINTER(_S)],
    "ssl_session_save": [_P, _P, _S],
    "ssl_session_restore": [_P, _P, _S, _P, ctypes.POINTER(_P)],
    "ssl_session_submit": [_P, _P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)],
    "ssl_session_submit_after": [_P, _P, ctypes.c_uint64, _P, ctypes.POINTER(ctypes.c_uint64)],
    "ssl_session_poll": [_P, ctypes.c_uint64, _P],
    "ssl_session_wait": [_P, ctypes.c_uint64, ctypes.c_uint64, _P],
    "ssl_server_run_step": [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "ssl_server_stats": [_P, _P],
    "ssl_server_reset_stats": [_P],
    "ssl_stream_create": [_P, _P, _I, _P, _P, ctypes.POINTER(_P)],
    "ssl_stream_push": [_P, _P, _P, _P, _P, _P, _P],
    "ssl_stream_destroy": [_P],
    "ssl_plan_create": [_P, _I, _P, _U, ctypes.POINTER(_P)],
    "ssl_plan_run": [_P, _P],
    "ssl_plan_get_info": [_P, _P],
    "ssl_plan_destroy": [_P],
}
PLAN_GRAPH, PLAN_AUTOTUNE = 1, 2
MAX_M = 64


METHOD = {"jacobi": 0, "bidiag": 1, "split": 2}


class JacobiOpts(ctypes.Structure):
    _fields_ = [("max_sweeps", ctypes.c_int), ("rel_tol", ctypes.c_float),
                ("abs_tol", ctypes.c_float), ("angles", ctypes.c_int), ("method", ctypes.c_int),
                ("split_ns", ctypes.c_int)]


def jacobi_opts(max_sweeps=0, rel_tol=0.0, abs_tol=0.0, angles="f64",
                method="jacobi", split_ns=0) -> JacobiOpts:
    return JacobiOpts(max_sweeps, rel_tol, abs_tol, ANGLES[angles], METHOD[method], split_ns)


class Config(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in
                ("M", "T", "B", "Ns", "n_az", "n_el", "form", "precision")] + [
                    ("jacobi", JacobiOpts)]


MAX_NS = 16


class ArrayDesc(ctypes.Structure):
    _fields_ = [("cfg", Config), ("queue_depth", ctypes.c_int)]


class SessionStateHeader(ctypes.Structure):
    """Header of a saved session state (ssl_session_save)."""
    _fields_ = [("magic", ctypes.c_uint32), ("version", ctypes.c_uint32), ("cfg", Config),
                ("queue_depth", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("kinv_bytes", ctypes.c_uint64)]


class Result(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int32), ("status", ctypes.c_int32),
                ("peak_idx", ctypes.c_int32 * MAX_NS), ("peak_val", ctypes.c_float * MAX_NS),
                ("t_arrival_ns", ctypes.c_uint64), ("t_done_ns", ctypes.c_uint64)]


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("blocks_done", "batches", "sessions",
                                              "sessions_refused", "blocks_refused",
                                              "blocks_pending")] + \
               [(n, ctypes.c_size_t) for n in ("hbm_budget", "hbm_used", "hbm_work")] + \
               [(n, ctypes.c_double) for n in ("busy_ms", "latency_p50_ms", "latency_p99_ms",
                                               "latency_max_ms")]


class BatchItem(ctypes.Structure):
    _fields_ = [("cfg", Config), ("X", _P), ("Kinv", _P), ("steering", _P),
                ("peak_idx", _P), ("peak_val", _P), ("status", _P), ("Pbar", _P)]


class PlanInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("n_items", "n_bins", "gsvd_units", "gsvd_grid",
                                            "launches", "graph")] + \
               [("class_of_m", ctypes.c_int * (MAX_M + 1)), ("autotune_ms", ctypes.c_double)]


_lib = None


def load(path: str = None) -> ctypes.CDLL:
    """Load the library (once).  Raises if it has not been built.  The
    SSL_GSVD_LIB environment variable selects another build of it (the
    bounds-checked debug library, say)."""
    global _lib
    if path is None:
        path = os.environ.get("SSL_GSVD_LIB", LIB_PATH)
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is missing: call build() first "
                               "(there is no CPU fallback)")
        lib = ctypes.CDLL(path)
        for name, argt in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = argt
            fn.restype = ctypes.c_int32
        _lib = lib
    return _lib


class SSLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _need(t: torch.Tensor, dtype, shape, name, device=True):
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if device and not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")


def gsvd_noalloc(R: torch.Tensor, K: torch.Tensor, stream=None, **jacobi):
    """ssl_gsvd_noalloc: the generalised SVD without any device allocation by
    the library (for callers that cannot allocate, e.g. a real-time audio
    thread).  Outputs are allocated here by torch, as a caller would own them.
    The call runs on R's device (made current for its duration).  Returns
    (sigma, E, status); per-bin failures (SSL_E_NOT_PD for a K that cannot be
    inverted) come back in status; raises SSLError on a non-OK return."""
    nblk, B, M, _ = R.shape
    _need(R, torch.complex64, (nblk, B, M, M), "R")
    _need(K, torch.complex64, (B, M, M), "K")
    if K.device != R.device:
        raise ValueError(f"K is on {K.device}, R on {R.device}: one device per call")
    sigma = torch.empty((nblk, B, M), dtype=torch.float32, device=R.device)
    E = torch.empty((nblk, B, M, M), dtype=torch.complex64, device=R.device)
    status = torch.empty((nblk, B), dtype=torch.int32, device=R.device)
    opts = jacobi_opts(**jacobi)
    with torch.cuda.device(R.device):
        st = load().ssl_gsvd_noalloc(_ptr(R), _ptr(K), nblk, B, M, ctypes.byref(opts),
                                     _ptr(sigma), _ptr(E), _ptr(status), _stream(stream))
    if st != SSL_OK:
        raise SSLError(st, "ssl_gsvd_noalloc failed")
    return sigma, E, status


class Steering:
    """Library-owned steering table H [B][D][M] (eq. 5)."""

    def __init__(self, ctx: "Context", H: torch.Tensor):
        B, D, M = H.shape
        _need(H, torch.complex64, (B, D, M), "H", device=False)
        self.ctx, self.B, self.D, self.M = ctx, B, D, M
        h = ctypes.c_void_p()
        ctx._check(load().ssl_steering_create(ctx.handle, _ptr(H), B, D, M, ctypes.byref(h)))
        self.handle = h

    @classmethod
    def analytic(cls, ctx: "Context", pos, dirs, freqs, c: float = 343.0) -> "Steering":
        """Free-field steering from the geometry (ssl_steering_create_analytic):
        pos [M][3] metres, dirs [D][3] unit vectors, freqs [B] Hz (array-likes
        or tensors, host or device, copied as float32)."""
        pos = torch.as_tensor(pos, dtype=torch.float32).contiguous()
        dirs = torch.as_tensor(dirs, dtype=torch.float32).contiguous()
        freqs = torch.as_tensor(freqs, dtype=torch.float32).contiguous()
        M, D, B = pos.shape[0], dirs.shape[0], freqs.shape[0]
        if tuple(pos.shape) != (M, 3) or tuple(dirs.shape) != (D, 3):
            raise ValueError("pos must be [M][3] and dirs [D][3]")
        self = cls.__new__(cls)
        self.ctx, self.B, self.D, self.M = ctx, B, D, M
        h = ctypes.c_void_p()
        ctx._check(load().ssl_steering_create_analytic(ctx.handle, _ptr(pos), _ptr(dirs),
                                                       _ptr(freqs), float(c), B, D, M,
                                                       ctypes.byref(h)))
        self.handle = h
        return self

    def set_search_range(self, in_range=None):
        """Search range of the peak search (ssl_steering_set_search_range):
        a bool / uint8 mask over the D directions (array-like or tensor, host
        or device), nonzero inside; None removes it."""
        if in_range is None:
            self.ctx._check(load().ssl_steering_set_search_range(self.handle, None))
            return
        m = torch.as_tensor(in_range)
        if m.dtype != torch.uint8:
            m = m.to(torch.uint8)
        m = m.contiguous()
        if tuple(m.shape) != (self.D,):
            raise ValueError(f"search range: expected {self.D} entries, got {tuple(m.shape)}")
        self.ctx._check(load().ssl_steering_set_search_range(self.handle, _ptr(m)))

    def set_neighbours(self, nbr_ptr: torch.Tensor, nbr_idx: torch.Tensor):
        """Neighbour lists (compressed rows, int32, host or device) of a
        direction set that is not a grid; then ``n_el = 0`` selects them."""
        _need(nbr_ptr, torch.int32, (self.D + 1,), "nbr_ptr", device=False)
        _need(nbr_idx, torch.int32, (nbr_idx.numel(),), "nbr_idx", device=False)
        self.ctx._check(load().ssl_steering_set_neighbours(self.handle, _ptr(nbr_ptr),
                                                            _ptr(nbr_idx), nbr_idx.numel()))

    def close(self):
        if getattr(self, "handle", None):
            load().ssl_steering_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0):
        lib = load()
        h = ctypes.c_void_p()
        st = lib.ssl_create(ctypes.byref(h), device)
        if st != SSL_OK:
            raise SSLError(st, f"ssl_create(device={device}) failed")
        self.handle = h
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            load().ssl_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def last_error(self) -> str:
        buf = ctypes.create_string_buffer(512)
        load().ssl_last_error(self.handle, buf, 512)
        return buf.value.decode(errors="replace")

    def _check(self, st: int):
        if st != SSL_OK:
            raise SSLError(st, self.last_error())

    def device_flags(self, stream=None) -> int:
        f = ctypes.c_uint32()
        self._check(load().ssl_device_flags(self.handle, _stream(stream), ctypes.byref(f)))
        return int(f.value)

    def set_wait_limit(self, ns: int = 0):
        """Limit (ns) of each bounded wait in the tensor-core kernels; 0 = default."""
        self._check(load().ssl_set_wait_limit(self.handle, int(ns)))

    def set_test_stall(self, on: bool):
        """Test hook: tensor-core spectrum launches withhold their operand loads."""
        self._check(load().ssl_set_test_stall(self.handle, 1 if on else 0))

    # ---- stateless steps ----
    def correlate(self, X: torch.Tensor, R: Optional[torch.Tensor] = None, stream=None):
        nblk, T, B, M = X.shape
        _need(X, torch.complex64, (nblk, T, B, M), "X")
        if R is None:
            R = torch.empty((nblk, B, M, M), dtype=torch.complex64, device=X.device)
        _need(R, torch.complex64, (nblk, B, M, M), "R")
        self._check(load().ssl_correlate(self.handle, _ptr(X), nblk, T, B, M, _ptr(R),
                                         _stream(stream)))
        return R

    def noise_inverse(self, K: torch.Tensor, stream=None):
        B, M, _ = K.shape
        _need(K, torch.complex64, (B, M, M), "K")
        Kinv = torch.empty_like(K)
        status = torch.empty(B, dtype=torch.int32, device=K.device)
        self._check(load().ssl_noise_inverse(self.handle, _ptr(K), B, M, _ptr(Kinv),
                                             _ptr(status), _stream(stream)))
        return Kinv, status

    def gsvd(self, R: torch.Tensor, K: torch.Tensor, kinv: bool = False, stats: bool = False,
             stream=None, **jacobi):
        """eq. 4 per (block, bin).  With kinv=True, K is already K^{-1}; with
        stats=True (requires kinv) also returns int32 [nblk][B][2] (pairs
        tested, rotations applied).  Keyword arguments: max_sweeps, rel_tol, abs_tol, angles,
        method ("jacobi", "bidiag", "split") and split_ns (Ns, for "split")."""
        opts = jacobi_opts(**jacobi)
        nblk, B, M, _ = R.shape
        _need(R, torch.complex64, (nblk, B, M, M), "R")
        _need(K, torch.complex64, (B, M, M), "K")
        sigma = torch.empty((nblk, B, M), dtype=torch.float32, device=R.device)
        E = torch.empty((nblk, B, M, M), dtype=torch.complex64, device=R.device)
        status = torch.empty((nblk, B), dtype=torch.int32, device=R.device)
        if kinv:
            st = (torch.empty((nblk, B, 2), dtype=torch.int32, device=R.device)
                  if stats else None)
            self._check(load().ssl_gsvd_kinv(self.handle, _ptr(R), _ptr(K), nblk, B, M,
                                             ctypes.byref(opts), _ptr(sigma), _ptr(E),
                                             _ptr(status), _ptr(st), _stream(stream)))
            return (sigma, E, status, st) if stats else (sigma, E, status)
        self._check(load().ssl_gsvd(self.handle, _ptr(R), _ptr(K), nblk, B, M,
                                    ctypes.byref(opts), _ptr(sigma), _ptr(E), _ptr(status),
                                    _stream(stream)))
        return sigma, E, status

    def sevd(self, R: torch.Tensor, stream=None, **jacobi):
        """R = E Lambda E^H (the K = I case of eq. 4).  Returns (lambda, E, status)."""
        nblk, B, M, _ = R.shape
        _need(R, torch.complex64, (nblk, B, M, M), "R")
        lam = torch.empty((nblk, B, M), dtype=torch.float32, device=R.device)
        E = torch.empty_like(R)
        status = torch.empty((nblk, B), dtype=torch.int32, device=R.device)
        o = jacobi_opts(**jacobi)
        self._check(load().ssl_sevd(self.handle, _ptr(R), nblk, B, M, ctypes.byref(o), _ptr(lam),
                                    _ptr(E), _ptr(status), _stream(stream)))
        return lam, E, status

    def gevd(self, R: torch.Tensor, K: torch.Tensor, stream=None, **jacobi):
        """R e = lambda K e.  Returns (lambda, E, status), E's columns K-orthonormal."""
        nblk, B, M, _ = R.shape
        _need(R, torch.complex64, (nblk, B, M, M), "R")
        _need(K, torch.complex64, (B, M, M), "K")
        lam = torch.empty((nblk, B, M), dtype=torch.float32, device=R.device)
        E = torch.empty_like(R)
        status = torch.empty((nblk, B), dtype=torch.int32, device=R.device)
        o = jacobi_opts(**jacobi)
        self._check(load().ssl_gevd(self.handle, _ptr(R), _ptr(K), nblk, B, M, ctypes.byref(o),
                                    _ptr(lam), _ptr(E), _ptr(status), _stream(stream)))
        return lam, E, status

    def steering(self, H: torch.Tensor) -> Steering:
        return Steering(self, H)

    def music_spectrum(self, E: torch.Tensor, Ns: int, st: Steering, form: str = "abs",
                       precision: str = "fp32", want_P: bool = True, stream=None):
        nblk, B, M, _ = E.shape
        _need(E, torch.complex64, (nblk, B, M, M), "E")
        P = (torch.empty((nblk, B, st.D), dtype=torch.float32, device=E.device)
             if want_P else None)
        Pbar = torch.empty((nblk, st.D), dtype=torch.float32, device=E.device)
        self._check(load().ssl_music_spectrum(self.handle, _ptr(E), nblk, B, M, Ns, st.handle,
                                              FORM[form], PRECISION[precision], _ptr(P),
                                              _ptr(Pbar), _stream(stream)))
        return P, Pbar

    def peaks(self, Pbar: torch.Tensor, n_az: int, n_el: int, Ns: int, stream=None):
        nblk, D = Pbar.shape
        _need(Pbar, torch.float32, (nblk, n_az * n_el), "Pbar")
        idx = torch.empty((nblk, Ns), dtype=torch.int32, device=Pbar.device)
        val = torch.empty((nblk, Ns), dtype=torch.float32, device=Pbar.device)
        self._check(load().ssl_peaks(self.handle, _ptr(Pbar), nblk, n_az, n_el, Ns, _ptr(idx),
                                     _ptr(val), _stream(stream)))
        return idx, val

    # ---- the FP64 path ----
    def gsvd_f64(self, R: torch.Tensor, K: torch.Tensor, stats: bool = False, stream=None,
                 **jacobi):
        """eq. 4 in FP64: R complex128 [nblk][B][M][M], K complex64 [B][M][M].
        Returns (sigma float64, E complex128, status[, stats])."""
        nblk, B, M, _ = R.shape
        _need(R, torch.complex128, (nblk, B, M, M), "R")
        _need(K, torch.complex64, (B, M, M), "K")
        sigma = torch.empty((nblk, B, M), dtype=torch.float64, device=R.device)
        E = torch.empty_like(R)
        status = torch.empty((nblk, B), dtype=torch.int32, device=R.device)
        st = torch.empty((nblk, B, 2), dtype=torch.int32, device=R.device) if stats else None
        o = jacobi_opts(**jacobi)
        self._check(load().ssl_gsvd_f64(self.handle, _ptr(R), _ptr(K), nblk, B, M,
                                        ctypes.byref(o), _ptr(sigma), _ptr(E), _ptr(status),
                                        _ptr(st), _stream(stream)))
        return (sigma, E, status, st) if stats else (sigma, E, status)

    def localize_f64(self, X: torch.Tensor, K: torch.Tensor, st: Steering, Ns: int, n_az: int,
                     n_el: int, form: str = "sq", out=None, stream=None, **jacobi):
        """The whole path in FP64 (device tensors): X complex64 [nblk][T][B][M],
        K complex64 [B][M][M].  Returns (idx int32, val float64, Pbar float64)."""
        nblk, T, B, M = X.shape
        _need(X, torch.complex64, (nblk, T, B, M), "X")
        _need(K, torch.complex64, (B, M, M), "K")
        D = n_az * n_el if n_el else n_az
        if out is None:
            out = (torch.empty((nblk, Ns), dtype=torch.int32, device=X.device),
                   torch.empty((nblk, Ns), dtype=torch.float64, device=X.device),
                   torch.empty((nblk, D), dtype=torch.float64, device=X.device))
        idx, val, Pbar = out
        cfg = Config(M, T, B, Ns, n_az, n_el, FORM[form], 0, jacobi_opts(**jacobi))
        self._check(load().ssl_localize_f64(self.handle, _ptr(X), nblk, _ptr(K), st.handle,
                                            ctypes.byref(cfg), _ptr(idx), _ptr(val), _ptr(Pbar),
                                            _stream(stream)))
        return idx, val, Pbar

    def peaks_nbr(self, Pbar: torch.Tensor, st: Steering, Ns: int, stream=None):
        """Peak search over st's direction set and its neighbour lists."""
        nblk, D = Pbar.shape
        _need(Pbar, torch.float32, (nblk, st.D), "Pbar")
        idx = torch.empty((nblk, Ns), dtype=torch.int32, device=Pbar.device)
        val = torch.empty((nblk, Ns), dtype=torch.float32, device=Pbar.device)
        self._check(load().ssl_peaks_nbr(self.handle, _ptr(Pbar), nblk, st.handle, Ns, _ptr(idx),
                                         _ptr(val), _stream(stream)))
        return idx, val

    # ---- whole path ----
    def localize(self, X: torch.Tensor, K: torch.Tensor, st: Steering, Ns: int, n_az: int,
                 n_el: int, form: str = "abs", precision: str = "fp32", out=None,
                 want_pbar: bool = True, stream=None, kinv: bool = False, **jacobi):
        """X [nblk][T][B][M] and K [B][M][M]: CUDA tensors, or (pinned) CPU tensors
        whose copies then run inside the call.  With kinv=True, K is already
        K^{-1} (ssl_localize_kinv).  Returns (idx, val, Pbar) on the device of
        ``out`` (allocated like X when not given)."""
        nblk, T, B, M = X.shape
        _need(X, torch.complex64, (nblk, T, B, M), "X", device=False)
        _need(K, torch.complex64, (B, M, M), "K", device=False)
        D = n_az * n_el if n_el else n_az  # n_el = 0: st's direction set and neighbour lists
        if out is None:
            dev = X.device
            pin = dict(pin_memory=True) if not X.is_cuda and torch.cuda.is_available() else {}
            out = (torch.empty((nblk, Ns), dtype=torch.int32, device=dev, **pin),
                   torch.empty((nblk, Ns), dtype=torch.float32, device=dev, **pin),
                   torch.empty((nblk, D), dtype=torch.float32, device=dev, **pin)
                   if want_pbar else None)
        idx, val, Pbar = out
        cfg = Config(M, T, B, Ns, n_az, n_el, FORM[form], PRECISION[precision],
                     jacobi_opts(**jacobi))
        fn = load().ssl_localize_kinv if kinv else load().ssl_localize
        self._check(fn(self.handle, _ptr(X), nblk, _ptr(K), st.handle, ctypes.byref(cfg),
                       _ptr(idx), _ptr(val), _ptr(Pbar), _stream(stream)))
        return idx, val, Pbar


def now_ns() -> int:
    v = ctypes.c_uint64()
    load().ssl_now_ns(ctypes.byref(v))
    return int(v.value)


class Session:
    """One array served by a Server (ssl_session_*)."""

    def __init__(self, server: "Server", K: torch.Tensor, st: Steering, Ns: int, n_az: int,
                 n_el: int, T: int, form: str = "abs", precision: str = "bf16",
                 queue_depth: int = 4, **jacobi):
        B, M, _ = K.shape
        _need(K, torch.complex64, (B, M, M), "K", device=False)
        self.server, self.Ns, self.T, self.B, self.M = server, Ns, T, B, M
        desc = ArrayDesc(Config(M, T, B, Ns, n_az, n_el, FORM[form], PRECISION[precision],
                                jacobi_opts(**jacobi)), queue_depth)
        h = ctypes.c_void_p()
        st_ = load().ssl_session_create(server.handle, ctypes.byref(desc), _ptr(K), st.handle,
                                        ctypes.byref(h))
        if st_ != SSL_OK:
            raise SSLError(st_, "ssl_session_create")
        self.handle = h
        self._keep = st
        self._inputs = {}  # ticket -> submitted tensor, held until retired

    def submit(self, X: torch.Tensor, t_arrival_ns: Optional[int] = None, stream=None,
               ordered: bool = True) -> int:
        """Queue one block; X (device or pinned host tensor) is kept alive here
        until its result has been collected, since the copy is asynchronous.
        A device X is copied only after the work already issued to `stream`
        (default: torch's current stream, where X was presumably made);
        ordered=False skips that ordering for device data known to be
        complete (ssl_session_submit)."""
        _need(X, torch.complex64, (self.T, self.B, self.M), "X", device=False)
        t = ctypes.c_uint64()
        ta = now_ns() if t_arrival_ns is None else t_arrival_ns
        if X.is_cuda and ordered:
            st = load().ssl_session_submit_after(self.handle, _ptr(X), ta, _stream(stream),
                                                 ctypes.byref(t))
        else:
            st = load().ssl_session_submit(self.handle, _ptr(X), ta, ctypes.byref(t))
        if st != SSL_OK:
            raise SSLError(st, "ssl_session_submit")
        self._inputs[int(t.value)] = X
        return int(t.value)

    def _res(self, r: Result, ticket: int):
        if not r.done:
            return None
        self._inputs.pop(ticket, None)
        return {"status": int(r.status), "idx": [int(r.peak_idx[i]) for i in range(self.Ns)],
                "val": [float(r.peak_val[i]) for i in range(self.Ns)],
                "t_arrival_ns": int(r.t_arrival_ns), "t_done_ns": int(r.t_done_ns)}

    def poll(self, ticket: int):
        r = Result()
        st = load().ssl_session_poll(self.handle, ticket, ctypes.byref(r))
        if st != SSL_OK:
            raise SSLError(st, "ssl_session_poll")
        return self._res(r, ticket)

    def wait(self, ticket: int, timeout_s: float = 10.0):
        r = Result()
        st = load().ssl_session_wait(self.handle, ticket, int(timeout_s * 1e9), ctypes.byref(r))
        if st != SSL_OK:
            raise SSLError(st, "ssl_session_wait")
        return self._res(r, ticket)

    def save(self) -> bytes:
        """The session's state (config, queue depth, K^{-1}) as bytes
        (ssl_session_save); Session.restore makes a session from it."""
        n = ctypes.c_size_t()
        st = load().ssl_session_state_size(self.handle, ctypes.byref(n))
        if st != SSL_OK:
            raise SSLError(st, "ssl_session_state_size")
        buf = ctypes.create_string_buffer(n.value)
        st = load().ssl_session_save(self.handle, buf, n.value)
        if st != SSL_OK:
            raise SSLError(st, "ssl_session_save")
        return buf.raw

    @classmethod
    def restore(cls, server: "Server", state: bytes, st: Steering) -> "Session":
        """A session on `server` from a saved state and a steering object that
        matches its config (ssl_session_restore; no Cholesky of K)."""
        if len(state) < ctypes.sizeof(SessionStateHeader):
            raise SSLError(1, "ssl_session_restore")
        hdr = SessionStateHeader.from_buffer_copy(state[:ctypes.sizeof(SessionStateHeader)])
        buf = ctypes.create_string_buffer(state, len(state))
        h = ctypes.c_void_p()
        r = load().ssl_session_restore(server.handle, buf, len(state), st.handle, ctypes.byref(h))
        if r != SSL_OK:
            raise SSLError(r, "ssl_session_restore")
        self = cls.__new__(cls)
        c = hdr.cfg
        self.server, self.Ns, self.T, self.B, self.M = server, c.Ns, c.T, c.B, c.M
        self.handle = h
        self._keep = st
        self._inputs = {}
        return self

    def close(self):
        """Destroys the session, also with blocks in flight: queued ones are
        dropped, those on the GPU waited for (ssl_session_destroy)."""
        if getattr(self, "handle", None):
            st = load().ssl_session_destroy(self.handle)
            if st != SSL_OK:
                raise SSLError(st, "ssl_session_destroy")
            self.handle = None
            self._inputs.clear()  # no copy of a submitted block is pending now


class Server:
    """Continuous-batching server (ssl_server_*)."""

    def __init__(self, ctx: Context, hbm_budget_bytes: int, max_batch: int = 256):
        h = ctypes.c_void_p()
        st = load().ssl_server_create(ctx.handle, hbm_budget_bytes, max_batch, ctypes.byref(h))
        if st != SSL_OK:
            raise SSLError(st, "ssl_server_create")
        self.handle, self.ctx = h, ctx

    def session(self, *a, **kw) -> Session:
        return Session(self, *a, **kw)

    def run_step(self):
        la, re = ctypes.c_int(), ctypes.c_int()
        st = load().ssl_server_run_step(self.handle, ctypes.byref(la), ctypes.byref(re))
        if st != SSL_OK:
            raise SSLError(st, "ssl_server_run_step")
        return int(la.value), int(re.value)

    def stats(self) -> dict:
        s = Stats()
        load().ssl_server_stats(self.handle, ctypes.byref(s))
        return {n: getattr(s, n) for n, _ in Stats._fields_}

    def reset_stats(self):
        load().ssl_server_reset_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            load().ssl_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Mixed batch of arrays of different sizes (ssl_plan_*): one launch per
    stage over every (array, bin) pair, optionally replayed as a CUDA graph
    and with the Jacobi size class per M chosen by timing.

    arrays: list of dicts with X (complex64 [T][B][M], device), Kinv
    (complex64 [B][M][M], device), st (Steering), Ns, n_az, n_el.  The plan
    allocates per-array outputs (peak_idx, peak_val, status, Pbar) and
    keeps references to every tensor it points at."""

    def __init__(self, ctx: Context, arrays, form: str = "abs", precision: str = "bf16",
                 graph: bool = True, autotune: bool = False, **jacobi):
        self.ctx, self.arrays = ctx, arrays
        n = len(arrays)
        items = (BatchItem * n)()
        self.outputs = []
        for i, a in enumerate(arrays):
            T, B, M = a["X"].shape
            _need(a["X"], torch.complex64, (T, B, M), "X")
            _need(a["Kinv"], torch.complex64, (B, M, M), "Kinv")
            dev = a["X"].device
            D = a["n_az"] * a["n_el"] if a["n_el"] else a["n_az"]  # 0: a direction set
            out = {"peak_idx": torch.empty(a["Ns"], dtype=torch.int32, device=dev),
                   "peak_val": torch.empty(a["Ns"], dtype=torch.float32, device=dev),
                   "status": torch.empty(1, dtype=torch.int32, device=dev),
                   "Pbar": torch.empty(D, dtype=torch.float32, device=dev)}
            self.outputs.append(out)
            items[i].cfg = Config(M, T, B, a["Ns"], a["n_az"], a["n_el"], FORM[form],
                                  PRECISION[precision], jacobi_opts(**jacobi))
            items[i].X, items[i].Kinv = _ptr(a["X"]), _ptr(a["Kinv"])
            items[i].steering = a["st"].handle
            items[i].peak_idx, items[i].peak_val = _ptr(out["peak_idx"]), _ptr(out["peak_val"])
            items[i].status, items[i].Pbar = _ptr(out["status"]), _ptr(out["Pbar"])
        flags = (PLAN_GRAPH if graph else 0) | (PLAN_AUTOTUNE if autotune else 0)
        h = ctypes.c_void_p()
        ctx._check(load().ssl_plan_create(ctx.handle, n, items, flags, ctypes.byref(h)))
        self.handle = h

    def run(self, stream=None):
        self.ctx._check(load().ssl_plan_run(self.handle, _stream(stream)))

    def info(self) -> dict:
        i = PlanInfo()
        self.ctx._check(load().ssl_plan_get_info(self.handle, ctypes.byref(i)))
        return {"n_items": i.n_items, "n_bins": i.n_bins, "gsvd_units": i.gsvd_units,
                "gsvd_grid": i.gsvd_grid, "launches": i.launches, "graph": bool(i.graph),
                "class_of_m": {m: int(i.class_of_m[m]) for m in range(MAX_M + 1)
                               if i.class_of_m[m]},
                "autotune_ms": float(i.autotune_ms)}

    def close(self):
        if getattr(self, "handle", None):
            load().ssl_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Stream:
    """Per-frame processing of one array (ssl_stream_*): a sliding window of
    T frames, pushed `hop` frames at a time, with warm-started Jacobi."""

    def __init__(self, ctx: Context, K: torch.Tensor, st: Steering, Ns: int, n_az: int,
                 n_el: int, T: int, hop: int, form: str = "abs", precision: str = "bf16",
                 **jacobi):
        B, M, _ = K.shape
        _need(K, torch.complex64, (B, M, M), "K", device=False)
        D = n_az * n_el if n_el else n_az  # n_el = 0: st's direction set and neighbour lists
        self.ctx, self.st, self.Ns, self.D, self.B, self.M, self.hop = ctx, st, Ns, D, B, M, hop
        cfg = Config(M, T, B, Ns, n_az, n_el, FORM[form], PRECISION[precision],
                     jacobi_opts(**jacobi))
        h = ctypes.c_void_p()
        ctx._check(load().ssl_stream_create(ctx.handle, ctypes.byref(cfg), hop, _ptr(K), st.handle,
                                            ctypes.byref(h)))
        self.handle = h

    def push(self, X: torch.Tensor, want_pbar: bool = True, stats: bool = False, stream=None):
        """X [hop][B][M] complex64 (device, or CPU).  Returns (idx, val, Pbar,
        stats) as device tensors (Pbar / stats None unless asked for)."""
        _need(X, torch.complex64, (self.hop, self.B, self.M), "X", device=False)
        dev = torch.device("cuda", self.ctx.device)
        idx = torch.empty(self.Ns, dtype=torch.int32, device=dev)
        val = torch.empty(self.Ns, dtype=torch.float32, device=dev)
        Pbar = torch.empty(self.D, dtype=torch.float32, device=dev) if want_pbar else None
        st = torch.empty((self.B, 2), dtype=torch.int32, device=dev) if stats else None
        self.ctx._check(load().ssl_stream_push(self.handle, _ptr(X), _ptr(idx), _ptr(val),
                                               _ptr(Pbar), _ptr(st), _stream(stream)))
        return idx, val, Pbar, st

    def close(self):
        if getattr(self, "handle", None):
            load().ssl_stream_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
