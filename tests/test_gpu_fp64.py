"""The FP64 GPU path against the FP64 oracle on the same (FP32) inputs.

Both sides compute in double precision, so they differ by rounding only:
about 1e-16 per operation, amplified by the whitening (cond K = 1e3 here),
by 1 / gap for the noise subspace (relative signal/noise gap >= 1e-2 on the
graded bins) and by the small denominators of eq. 5 near the peaks.  The
bounds below (1e-12 for singular values and unitarity, 1e-10 for the
projector and for the max-normalised spectrum) leave two to three orders of
margin over those estimates while staying far below the FP32 path's 1e-4.
"""

import numpy as np
import pytest
import torch

import oracle.gsvd_music as O
from gpu_common import context, dev, host, max_rel, projector, signal_gap
from paper_2504_03373_gb300 import synth

pytestmark = pytest.mark.gpu


def _pd(rng, B, M, cond):
    G = synth.noise_mixing(rng, B, M, cond)
    return np.matmul(G, np.conj(np.swapaxes(G, 1, 2)))


def dev64(a):
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.complex128))).cuda()


@pytest.mark.parametrize("M", [2, 3, 8, 17, 33, 60, 64])
def test_gsvd_f64_random(M):
    ctx = context()
    rng = np.random.default_rng(1300 + M)
    nblk, B, T = 2, 5, max(2 * M, 20)
    K = _pd(rng, B, M, 1e2).astype(np.complex64)
    X = synth.cgauss(rng, (nblk, T, B, M))
    X[..., :3] *= 8.0
    R = np.stack([O.correlation(X[k]) for k in range(nblk)])
    sig, E, status = ctx.gsvd_f64(dev64(R), dev(K))
    assert (host(status) == 0).all() and ctx.device_flags() == 0
    sig, E = host(sig), host(E)
    for k in range(nblk):
        A, Eo, lo, _ = O.gsvd(K.astype(np.complex128), R[k])
        assert np.abs(sig[k] - lo).max() <= 1e-12 * lo.max()
        EH = np.conj(np.swapaxes(E[k], 1, 2))
        assert np.abs(np.matmul(EH, E[k]) - np.eye(M)).max() < 1e-12
        # A A^H e_i = sigma_i^2 e_i
        AAH = np.matmul(A, np.conj(np.swapaxes(A, 1, 2)))
        res = np.matmul(AAH, E[k]) - E[k] * (sig[k] ** 2)[:, None, :]
        assert np.abs(res).max() <= 1e-11 * (lo.max() ** 2)
        for Ns in (1, 2, 3):
            if Ns >= M:
                continue
            gap = signal_gap(lo, Ns)
            err = np.linalg.norm(projector(E[k], Ns) - projector(Eo, Ns), axis=(1, 2))
            bound = np.where(gap >= 1e-2, 1e-10, 1e-12 / np.maximum(gap, 1e-30))
            assert (err <= bound).all(), (Ns, err.max(), gap.min())


def _grade(w, K, idx, val, Pbar, form, nbr=None, tol=1e-10):
    graded = ok = 0
    for k in range(w.nblk):
        ref = O.localize_block(w.X[k], K, w.H.astype(np.complex64), w.Ns,
                               w.grid.n_az, w.grid.n_el, form, nbr=nbr)
        assert max_rel(host(Pbar)[k], ref["Pbar"]) < tol, k
        margin = (O.peak_margin(ref["Pbar"], w.grid.n_az, w.grid.n_el, w.Ns) if nbr is None
                  else O.peak_margin_nbr(ref["Pbar"], nbr[0], nbr[1], w.Ns))
        if margin > tol:
            graded += 1
            ok += list(host(idx)[k]) == list(ref["idx"])
            assert np.allclose(host(val)[k], ref["val"], rtol=tol)
    assert ok == graded
    return graded


def test_localize_f64_ball60_sq():
    ctx = context()
    w = synth.ball60_three_sources(seed=2, nblk=3)
    K = O.correlation(w.Xnoise).astype(np.complex64)
    st = ctx.steering(dev(w.H))
    idx, val, Pbar = ctx.localize_f64(dev(w.X), dev(K), st, 3, w.grid.n_az, w.grid.n_el,
                                      form="sq", abs_tol=2.0 ** -52)
    assert ctx.device_flags() == 0
    assert _grade(w, K, idx, val, Pbar, "sq") >= 1
    st.close()


def test_localize_f64_uca8_abs():
    """The 8-mic workload has separated noise singular values, so the ABS form
    (eq. 5 as printed) is determined and graded too."""
    ctx = context()
    w = synth.uca8_single_source(seed=1, nblk=2)
    K = O.correlation(w.Xnoise).astype(np.complex64)
    st = ctx.steering(dev(w.H))
    idx, val, Pbar = ctx.localize_f64(dev(w.X), dev(K), st, 1, w.grid.n_az, w.grid.n_el,
                                      form="abs")
    assert ctx.device_flags() == 0
    assert _grade(w, K, idx, val, Pbar, "abs") == 2
    st.close()


def test_localize_f64_paper_shape():
    ctx = context()
    w = synth.paper_shape(seed=3, nblk=2)
    K = O.correlation(w.Xnoise).astype(np.complex64)
    st = ctx.steering(dev(w.H))
    st.set_neighbours(torch.from_numpy(w.grid.nbr_ptr), torch.from_numpy(w.grid.nbr_idx))
    idx, val, Pbar = ctx.localize_f64(dev(w.X), dev(K), st, 2, w.D, 0, form="sq",
                                      abs_tol=2.0 ** -52)
    assert ctx.device_flags() == 0
    _grade(w, K, idx, val, Pbar, "sq", nbr=(w.grid.nbr_ptr, w.grid.nbr_idx))
    st.close()


def test_fp32_path_error_is_its_arithmetic():
    """On the same inputs the FP32 path's distance to the FP64 GPU path equals
    its distance to the oracle (to within the FP64 path's own 1e-10): the
    FP32 error is arithmetic, not method."""
    ctx = context()
    w = synth.ball60_three_sources(seed=2, nblk=2)
    K = O.correlation(w.Xnoise).astype(np.complex64)
    st = ctx.steering(dev(w.H))
    _, _, P64 = ctx.localize_f64(dev(w.X), dev(K), st, 3, 72, 19, form="sq",
                                 abs_tol=2.0 ** -52)
    _, _, P32 = ctx.localize(dev(w.X), dev(K), st, 3, 72, 19, form="sq", precision="fp32",
                             abs_tol=2.0 ** -23)
    for k in range(w.nblk):
        ref = O.localize_block(w.X[k], K, w.H.astype(np.complex64), 3, 72, 19, "sq")
        e_gpu = max_rel(host(P32)[k], host(P64)[k])
        e_ora = max_rel(host(P32)[k], ref["Pbar"])
        assert e_ora < 1e-4
        assert abs(e_gpu - e_ora) < 1e-9
    st.close()
