"""ssl_gsvd_noalloc, the allocation-free form of the generalised SVD, against
the regular ssl_gsvd through the C ABI.

The entry point exists for callers that cannot allocate device memory on
their processing path (a real-time audition thread whose block deadline a
cudaMalloc could blow, a host framework that owns the device memory budget).
It keeps its only scratch, K^{-1}, in a fixed array inside the library.  This
file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""

import numpy as np
import pytest

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
