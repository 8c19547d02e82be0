"""Failure paths of the device code, made to happen without faulting the GPU.

* The tensor-core spectrum's hand-offs (copies -> MMAs -> epilogue) are
  bounded waits.  A test hook makes the load role issue no operand load at
  all (data that never arrives: a flag nothing sets), with the context's wait
  limit at 1 ms: the MMA role's wait must run out, the kernel must stop its
  pipeline, release its tensor memory, return, and raise SSL_FLAG_TIMEOUT;
  the next call on the same context, hook off and default limit, must give
  the same spectrum as before (tensor memory was released).  Every
  tensor-core form is covered: BF16 and TF32 from stored tables, BF16 with
  steering generated in the kernel, and 3xTF32.
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


@pytest.mark.parametrize("precision,analytic", [("bf16", False), ("tf32", False),
                                                ("bf16", True), ("tf32x3", False)])
def test_spectrum_wait_limit_runs_out_and_the_context_recovers(precision, analytic):
    ctx = context()
    w, R, K = _workload()
    sig, E, st = ctx.gsvd(R, K, abs_tol=2.0 ** -23)
    H = (binding.Steering.analytic(ctx, w.pos, w.grid.unit_vectors(), w.freqs) if analytic
         else ctx.steering(dev(w.H)))
    assert ctx.device_flags() == 0
    P0, Pb0 = ctx.music_spectrum(E, 3, H, form="sq", precision=precision)
    assert ctx.device_flags() == 0
    ref = host(P0).copy()
    try:
        ctx.set_wait_limit(1_000_000)
        ctx.set_test_stall(True)
        ctx.music_spectrum(E, 3, H, form="sq", precision=precision)
        flags = ctx.device_flags()  # synchronises: the launch returned
    finally:
        ctx.set_test_stall(False)
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
