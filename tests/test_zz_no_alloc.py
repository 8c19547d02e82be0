"""ssl_gsvd_noalloc, the allocation-free form of the generalised SVD, against
the regular ssl_gsvd through the C ABI.

The entry point exists for callers that cannot allocate device memory on
their processing path (a real-time audition thread whose block deadline a
cudaMalloc could blow, a host framework that owns the device memory budget).
Its scratch (K^{-1} and a status word per bin) lives in a fixed array inside
the library; the status array is its only error channel.  This
file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""

import numpy as np
import pytest
import torch

import oracle.gsvd_music as O
from gpu_common import context, dev, host, projector
from paper_2504_03373_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def _inputs():
    w = synth.ball60_three_sources(seed=2, nblk=2)
    K = O.correlation(w.Xnoise).astype(np.complex64)
    R = np.stack([O.correlation(w.X[k]) for k in range(w.nblk)]).astype(np.complex64)
    return dev(R), dev(K)


@pytest.mark.parametrize("angles", ["f64", "f32"])
def test_noalloc_matches_regular_gsvd_twice(angles):
    ctx = context()
    R, K = _inputs()
    opts = dict(angles=angles, abs_tol=2.0 ** -23)
    sig_ref, E_ref, st_ref = ctx.gsvd(R, K, **opts)
    for call in range(2):  # the array keeps the previous call's contents
        sig, E, st = binding.gsvd_noalloc(R, K, **opts)
        s0, s1 = host(sig_ref), host(sig)
        assert (host(st) == host(st_ref)).all()
        assert np.abs(s1 - s0).max() <= 5e-5 * np.abs(s0).max(), call
        err = np.linalg.norm(projector(host(E), 3) - projector(host(E_ref), 3), axis=(-2, -1))
        assert err.max() < 1e-4, call


def test_noalloc_rejects_requests_beyond_its_capacity():
    context()
    M, B = 64, 257  # 257 * 64 * 64 > 2^20 complex values
    R = dev(np.zeros((1, B, M, M)))
    K = dev(np.broadcast_to(np.eye(M), (B, M, M)))
    with pytest.raises(binding.SSLError) as e:
        binding.gsvd_noalloc(R, K)
    assert e.value.status == 10  # SSL_E_CAPACITY


def test_noalloc_reports_a_k_it_cannot_invert_then_recovers():
    """With no context there is no sticky flag word, so the status array is
    the only error channel: a bin whose K is indefinite reports SSL_E_NOT_PD
    and a bin whose K holds a NaN reports SSL_E_NONFINITE, in every block;
    the other bins match the regular call.  A following call with a valid K
    reports every bin as 0 again (the per-bin words in the fixed array are
    rewritten by each call)."""
    ctx = context()
    R, K = _inputs()
    Kbad = K.clone()
    Kbad[5] = -Kbad[5]                 # negative definite: the first pivot is < 0
    Kbad[9][0, 0] = float("nan")       # non-finite
    sig_ref, E_ref, st_ref = ctx.gsvd(R, K, abs_tol=2.0 ** -23)
    sig, E, st = binding.gsvd_noalloc(R, Kbad, abs_tol=2.0 ** -23)
    st = host(st)
    assert (st[:, 5] == 2).all() and (st[:, 9] == 4).all()  # SSL_E_NOT_PD, SSL_E_NONFINITE
    assert (host(sig)[:, [5, 9]] == 0).all()                 # K^{-1} = 0 behind them
    good = np.ones(st.shape[1], dtype=bool)
    good[[5, 9]] = False
    assert (st[:, good] == host(st_ref)[:, good]).all()
    s0, s1 = host(sig_ref)[:, good], host(sig)[:, good]
    assert np.abs(s1 - s0).max() <= 5e-5 * np.abs(s0).max()
    sig2, E2, st2 = binding.gsvd_noalloc(R, K, abs_tol=2.0 ** -23)
    assert (host(st2) == host(st_ref)).all()
    assert np.abs(host(sig2) - host(sig_ref)).max() <= 5e-5 * np.abs(host(sig_ref)).max()


def test_noalloc_matches_the_oracle():
    """The allocation-free call against the FP64 oracle (eq. 4): singular
    values within 5e-5 of sigma_max for the three signal values (the
    absolute Jacobi tolerance makes the small ones accurate in absolute
    terms only, about abs_tol sigma_max^2 / sigma) and the noise-subspace
    projector within 1e-4 where the signal/noise gap is >= 1e-2 (else
    within 2e-6 / gap)."""
    context()
    R, K = _inputs()
    sig, E, st = binding.gsvd_noalloc(R, K, abs_tol=2.0 ** -23)
    assert (host(st) == 0).all()
    Rh, Kh = host(R).astype(np.complex128), host(K).astype(np.complex128)
    _, Eo, lo, _ = O.gsvd(Kh, Rh)
    sig, E = host(sig), host(E)
    smax = lo[..., :1].max()
    assert np.abs(sig[..., :3] - lo[..., :3]).max() / smax < 5e-5
    assert np.abs(sig - lo).max() / smax < 2e-3
    gap = (lo[..., 2] - lo[..., 3]) / lo[..., 0]
    err = np.linalg.norm(projector(E, 3) - projector(Eo, 3), axis=(-2, -1))
    bound = np.where(gap >= 1e-2, 1e-4, 2e-6 / np.maximum(gap, 1e-30))
    assert (err <= bound).all(), (err.max(), gap.min())


def test_noalloc_requires_a_status_array():
    """Without a status array a failure could not be reported: rejected."""
    from paper_2504_03373_gb300.binding import _ptr, jacobi_opts, load
    import ctypes
    context()
    R, K = _inputs()
    nblk, B, M, _ = R.shape
    sig = torch.empty((nblk, B, M), dtype=torch.float32, device=R.device)
    E = torch.empty_like(R)
    st = load().ssl_gsvd_noalloc(_ptr(R), _ptr(K), nblk, B, M, ctypes.byref(jacobi_opts()),
                                 _ptr(sig), _ptr(E), None, None)
    assert st == 1  # SSL_E_INVALID_ARG
