"""Invalid sizes, enums and options are refused with SSL_E_INVALID_ARG before
anything is launched: every call below gets valid device buffers and exactly
one bad argument, and the context stays usable (no sticky flag, a valid call
afterwards succeeds)."""

import ctypes

import numpy as np
import pytest
import torch

from gpu_common import context, dev
from paper_2504_03373_gb300 import binding
from paper_2504_03373_gb300.binding import Config, JacobiOpts, jacobi_opts

pytestmark = pytest.mark.gpu

E_INVALID = 1


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def _buf(n):
    return torch.zeros(int(n), dtype=torch.float32, device="cuda")


@pytest.fixture(scope="module")
def env():
    ctx = context()
    B, D, M = 4, 16, 8
    st = ctx.steering(dev(np.ones((B, D, M), np.complex64)))
    big = _buf(1 << 22)  # 16 MB, larger than any call below reads
    return ctx, st, big, (B, D, M)


def _cfg(**kw):
    c = dict(M=8, T=10, B=4, Ns=1, n_az=16, n_el=1, form=1, precision=0)
    c.update(kw)
    jac = kw.pop("jacobi", None) or jacobi_opts()
    return Config(c["M"], c["T"], c["B"], c["Ns"], c["n_az"], c["n_el"], c["form"],
                  c["precision"], jac)


BAD_CFGS = [
    dict(M=0), dict(M=65), dict(T=0), dict(B=0), dict(Ns=0), dict(Ns=8), dict(Ns=17, M=40),
    dict(n_az=0), dict(n_el=-1), dict(n_az=8), dict(form=5), dict(precision=9),
    dict(jacobi=JacobiOpts(0, float("nan"), 0.0, 0, 0)),
    dict(jacobi=JacobiOpts(0, 0.0, float("inf"), 0, 0)),
    dict(jacobi=JacobiOpts(0, 0.0, 0.0, 7, 0)),
    dict(jacobi=JacobiOpts(0, 0.0, 0.0, 0, 5)),
]


@pytest.mark.parametrize("bad", BAD_CFGS, ids=lambda d: ",".join(f"{k}" for k in d))
def test_localize_refuses_an_inconsistent_config(env, bad):
    ctx, st, big, _ = env
    lib = binding.load()
    cfg = _cfg(**bad)
    idx = torch.zeros(64, dtype=torch.int32, device="cuda")
    r = lib.ssl_localize(ctx.handle, _p(big), 1, _p(big), st.handle, ctypes.byref(cfg), _p(idx),
                         _p(big), _p(big), None)
    assert r == E_INVALID, (bad, r)
    assert ctx.device_flags() == 0


def test_stateless_calls_refuse_bad_sizes(env):
    ctx, st, big, (B, D, M) = env
    lib = binding.load()
    h = ctx.handle
    bp = _p(big)
    idx = torch.zeros(64, dtype=torch.int32, device="cuda")
    jac = jacobi_opts()
    calls = {
        "correlate M=0": lambda: lib.ssl_correlate(h, bp, 1, 10, B, 0, bp, None),
        "correlate M=65": lambda: lib.ssl_correlate(h, bp, 1, 10, B, 65, bp, None),
        "correlate T=0": lambda: lib.ssl_correlate(h, bp, 1, 0, B, M, bp, None),
        "correlate nblk=0": lambda: lib.ssl_correlate(h, bp, 0, 10, B, M, bp, None),
        "noise_inverse B=0": lambda: lib.ssl_noise_inverse(h, bp, 0, M, bp, None, None),
        "gsvd M=65": lambda: lib.ssl_gsvd(h, bp, bp, 1, B, 65, ctypes.byref(jac), bp, bp, None,
                                          None),
        "gsvd bad method": lambda: lib.ssl_gsvd(h, bp, bp, 1, B, M,
                                                ctypes.byref(JacobiOpts(0, 0, 0, 0, 9)), bp, bp,
                                                None, None),
        "spectrum Ns=M": lambda: lib.ssl_music_spectrum(h, bp, 1, B, M, M, st.handle, 1, 0, None,
                                                        bp, None),
        "spectrum B mismatch": lambda: lib.ssl_music_spectrum(h, bp, 1, B + 1, M, 1, st.handle,
                                                              1, 0, None, bp, None),
        "spectrum bad form": lambda: lib.ssl_music_spectrum(h, bp, 1, B, M, 1, st.handle, 7, 0,
                                                            None, bp, None),
        "spectrum bad precision": lambda: lib.ssl_music_spectrum(h, bp, 1, B, M, 1, st.handle,
                                                                 1, 11, None, bp, None),
        "peaks D too large": lambda: lib.ssl_peaks(h, bp, 1, 8193, 1, 1, _p(idx), bp, None),
        "peaks Ns=17": lambda: lib.ssl_peaks(h, bp, 1, 16, 1, 17, _p(idx), bp, None),
        "peaks_nbr without lists": lambda: lib.ssl_peaks_nbr(h, bp, 1, st.handle, 1, _p(idx),
                                                             bp, None),
        "steering D=0": lambda: lib.ssl_steering_create(h, bp, B, 0, M,
                                                        ctypes.byref(ctypes.c_void_p())),
        "steering D too large": lambda: lib.ssl_steering_create(h, bp, B, 8193, M,
                                                                ctypes.byref(ctypes.c_void_p())),
        "analytic c=0": lambda: lib.ssl_steering_create_analytic(
            h, bp, bp, bp, ctypes.c_float(0.0), B, D, M, ctypes.byref(ctypes.c_void_p())),
    }
    for name, call in calls.items():
        assert call() == E_INVALID, name
    assert ctx.device_flags() == 0
    # the context still works
    X = dev(np.ones((1, 10, B, M), np.complex64))
    R = ctx.correlate(X)
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(R)).all()


def test_sessions_streams_and_plans_refuse_bad_configs(env):
    ctx, st, big, (B, D, M) = env
    lib = binding.load()
    srv = binding.Server(ctx, hbm_budget_bytes=1 << 30, max_batch=8)
    K = dev(np.broadcast_to(np.eye(M, dtype=np.complex64), (B, M, M)).copy())
    for bad in BAD_CFGS:
        desc = binding.ArrayDesc(_cfg(**bad), 2)
        out = ctypes.c_void_p()
        r = lib.ssl_session_create(srv.handle, ctypes.byref(desc), _p(K), st.handle,
                                   ctypes.byref(out))
        assert r == E_INVALID, ("session", bad, r)
        r = lib.ssl_stream_create(ctx.handle, ctypes.byref(_cfg(**bad)), 5, _p(K), st.handle,
                                  ctypes.byref(out))
        assert r == E_INVALID, ("stream", bad, r)
    desc = binding.ArrayDesc(_cfg(), 0)  # queue depth 0
    r = lib.ssl_session_create(srv.handle, ctypes.byref(desc), _p(K), st.handle,
                               ctypes.byref(ctypes.c_void_p()))
    assert r == E_INVALID
    for hop in (0, 11):  # hop outside 1..T
        r = lib.ssl_stream_create(ctx.handle, ctypes.byref(_cfg()), hop, _p(K), st.handle,
                                  ctypes.byref(ctypes.c_void_p()))
        assert r == E_INVALID, hop
    assert srv.stats()["sessions"] == 0
    srv.close()
    assert ctx.device_flags() == 0
