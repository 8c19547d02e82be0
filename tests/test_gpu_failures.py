"""Failure paths of the device code, made to happen without faulting the GPU.

* The tensor-core spectrum's hand-offs (copies -> MMAs -> epilogue) are
  bounded waits.  A context's wait limit is set to 1 ns so that the first wait
  that is not satisfied at once gives up: the kernel must stop its pipeline,
  drain its own copies and MMAs, release its tensor memory, return, and raise
  SSL_FLAG_TIMEOUT; the next call with the default limit on the same context
  must give the same spectrum as before (tensor memory was released).
* The Jacobi iteration is bounded by max_sweeps: one sweep on the 60-mic
  workload ends with rotations still being applied, which every bin reports
  as SSL_E_NO_CONVERGENCE and the context as its sticky flag.
"""

import numpy as np
import pytest

import oracle.gsvd_music as O
from gpu_common import context, dev, host
from paper_2504_03373_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def _workload(nblk=2):
    w = synth.ball60_three_sources(seed=2, nblk=nblk)
    K = O.correlation(w.Xnoise).astype(np.complex64)
    R = np.stack([O.correlation(w.X[k]) for k in range(nblk)]).astype(np.complex64)
    return w, dev(R), dev(K)


@pytest.mark.parametrize("precision", ["bf16", "tf32"])
def test_spectrum_wait_limit_runs_out_and_the_context_recovers(precision):
    ctx = context()
    w, R, K = _workload()
    sig, E, st = ctx.gsvd(R, K, abs_tol=2.0 ** -23)
    H = ctx.steering(dev(w.H))
    assert ctx.device_flags() == 0
    P0, Pb0 = ctx.music_spectrum(E, 3, H, form="sq", precision=precision)
    assert ctx.device_flags() == 0
    ref = host(P0).copy()
    try:
        ctx.set_wait_limit(1)
        ctx.music_spectrum(E, 3, H, form="sq", precision=precision)
        flags = ctx.device_flags()  # synchronises: the launch returned
    finally:
        ctx.set_wait_limit(0)
    assert flags & binding.FLAG_TIMEOUT, flags
    # same context, default limit: the kernel allocates its tensor memory again
    P1, Pb1 = ctx.music_spectrum(E, 3, H, form="sq", precision=precision)
    assert ctx.device_flags() == 0
    assert np.array_equal(host(P1), ref)
    H.close()


def test_one_sweep_reports_no_convergence():
    ctx = context()
    _, R, K = _workload()
    assert ctx.device_flags() == 0
    sig, E, st = ctx.gsvd(R, K, max_sweeps=1, abs_tol=2.0 ** -23)
    flags = ctx.device_flags()
    assert (host(st) == 3).all()  # SSL_E_NO_CONVERGENCE in every (block, bin)
    assert flags & binding.FLAG_NO_CONVERGENCE, flags
    # the default limit converges on the same input
    sig, E, st = ctx.gsvd(R, K, abs_tol=2.0 ** -23)
    assert (host(st) == 0).all() and ctx.device_flags() == 0
