"""The paper's own SVD route (method="bidiag": Householder bidiagonalisation,
phase transform, implicit-shift QR, sort, back-transformation) against the
FP64 oracle, beside the one-sided Jacobi default: singular values, unitarity,
A A^H e_i = sigma_i^2 e_i, the noise-subspace projector, rank-deficient and
degenerate inputs, the full localization, and the batch / stream paths."""

import numpy as np
import pytest
import torch

import oracle.gsvd_music as O
from gpu_common import context, dev, host, projector
from paper_2504_03373_gb300 import binding, synth

pytestmark = pytest.mark.gpu

ABS_TOL = 2.0 ** -23


def _crand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _pd(rng, B, M, cond):
    Q = synth.haar_unitary(rng, B, M)
    s = np.logspace(0, -np.log10(cond), M)
    return np.matmul(Q * s[None, None, :], np.conj(np.swapaxes(Q, -1, -2)))


def _check(sig, E, K, R, Ns, sig_tol=2e-5, proj_tol=1e-3):
    A, E_ref, s_ref, _ = O.gsvd(K.astype(complex), R.astype(complex))
    s = sig.astype(float)
    assert np.abs(s - s_ref).max() / s_ref.max() < sig_tol
    assert np.all(np.diff(s, axis=-1) <= 0)
    Ec = E.astype(complex)
    EH = np.conj(np.swapaxes(Ec, -1, -2))
    M = E.shape[-1]
    assert np.abs(np.matmul(EH, Ec) - np.eye(M)).max() < 5e-5
    AAH = np.matmul(A, np.conj(np.swapaxes(A, -1, -2)))
    res = np.matmul(AAH, Ec) - Ec * (s ** 2)[..., None, :]
    assert np.abs(res).max() / (s_ref.max() ** 2) < 5e-5
    gap = (s_ref[..., Ns - 1] - s_ref[..., Ns]) / s_ref[..., 0]
    ok = gap > 1e-2
    perr = np.linalg.norm(projector(Ec, Ns) - projector(E_ref, Ns), axis=(-2, -1))
    assert perr[ok].max() < proj_tol, perr[ok].max()
    return perr[ok].max()


@pytest.mark.parametrize("M", [2, 8, 17, 32, 60, 64])
def test_bidiag_random(M):
    ctx = context()
    rng = np.random.default_rng(1100 + M)
    B, T = 9, 2 * M
    K = _pd(rng, B, M, 1e2).astype(np.complex64)
    X = _crand(rng, 2, T, B, M).astype(np.complex64)
    R = np.stack([O.correlation(X[k]) for k in range(2)]).astype(np.complex64)
    sig, E, status = ctx.gsvd(dev(R), dev(K), method="bidiag", abs_tol=ABS_TOL)
    assert (host(status) == 0).all()
    for k in range(2):
        _check(host(sig)[k], host(E)[k], K, R[k], Ns=min(3, M - 1))


@pytest.mark.parametrize("M,T", [(60, 50), (8, 3), (64, 20)])
def test_bidiag_rank_deficient(M, T):
    """M > T: the null space is spanned exactly by E's last M - T columns."""
    ctx = context()
    rng = np.random.default_rng(1200 + M + T)
    B = 6
    K = _pd(rng, B, M, 1e3).astype(np.complex64)
    X = _crand(rng, 1, T, B, M).astype(np.complex64)
    R = O.correlation(X[0])[None].astype(np.complex64)
    sig, E, status = ctx.gsvd(dev(R), dev(K), method="bidiag", abs_tol=ABS_TOL)
    assert (host(status) == 0).all()
    s = host(sig)[0]
    assert (s[:, T:] <= 1e-5 * s[:, :1]).all()
    _check(host(sig)[0], host(E)[0], K, R[0], Ns=1)


def test_bidiag_degenerate_inputs():
    ctx = context()
    M, B = 16, 4
    K = np.broadcast_to(np.eye(M), (B, M, M)).astype(np.complex64).copy()
    R = np.zeros((1, B, M, M), np.complex64)
    R[0, 1] = np.eye(M)                      # zero matrix, identity (all sigma equal)
    R[0, 2, 3, 3] = 2.0                      # rank one, real
    R[0, 3] = np.diag(np.arange(M, 0, -1))   # diagonal, distinct
    sig, E, status = ctx.gsvd(dev(R), dev(K), method="bidiag", abs_tol=ABS_TOL)
    assert (host(status) == 0).all()
    s, Eh = host(sig)[0], host(E)[0].astype(complex)
    assert np.allclose(s[0], 0) and np.allclose(s[1], 1, atol=1e-6)
    assert np.isclose(s[2, 0], 2) and np.allclose(s[2, 1:], 0, atol=1e-6)
    assert np.allclose(s[3], np.arange(M, 0, -1), rtol=1e-6)
    for b in range(B):
        assert np.abs(np.conj(Eh[b]).T @ Eh[b] - np.eye(M)).max() < 1e-5
    R[0, 0, 2, 5] = np.nan
    ctx.device_flags()  # read and clear
    _, _, status = ctx.gsvd(dev(R), dev(K), method="bidiag", abs_tol=ABS_TOL)
    assert int(host(status)[0, 0]) == 4  # SSL_E_NONFINITE
    assert ctx.device_flags() & binding.FLAG_NONFINITE  # read and clear


def test_bidiag_localization_matches_oracle():
    """The 60-mic workload (SQ form, FP32 spectrum) through the paper's
    route: P-bar within the FP32 tolerance, peaks where the margin allows,
    and the projector error beside the Jacobi default's."""
    ctx = context()
    w = synth.ball60_three_sources(seed=2, nblk=3)
    K = O.correlation(w.Xnoise).astype(np.complex64)
    st = ctx.steering(dev(w.H))
    idx, val, Pbar = ctx.localize(dev(w.X), dev(K), st, 3, w.grid.n_az, w.grid.n_el, form="sq",
                                  precision="fp32", method="bidiag", abs_tol=ABS_TOL)
    R = ctx.correlate(dev(w.X))
    _, Eb, sb = ctx.gsvd(R, dev(K), method="bidiag", abs_tol=ABS_TOL)
    _, Ej, sj = ctx.gsvd(R, dev(K), abs_tol=ABS_TOL)
    assert (host(sb) == 0).all() and (host(sj) == 0).all()
    pb, pj = [], []
    for k in range(w.nblk):
        ref = O.localize_block(w.X[k], K, w.H.astype(np.complex64), 3, w.grid.n_az,
                               w.grid.n_el, "sq")
        err = np.abs(host(Pbar)[k] - ref["Pbar"]).max() / ref["Pbar"].max()
        assert err < 1e-4, err
        if O.peak_margin(ref["Pbar"], w.grid.n_az, w.grid.n_el, 3) > 1e-3:
            assert list(host(idx)[k]) == list(ref["idx"])
        P0 = projector(ref["E"], 3)
        pb.append(np.linalg.norm(projector(host(Eb)[k], 3) - P0, axis=(-2, -1)).max())
        pj.append(np.linalg.norm(projector(host(Ej)[k], 3) - P0, axis=(-2, -1)).max())
    print(f"\nprojector error: bidiag {max(pb):.2e}, jacobi {max(pj):.2e}")
    assert max(pb) < 1e-4
    st.close()


def test_bidiag_in_batch_and_stream():
    ctx = context()
    w = synth.make_workload(M=17, T=40, nblk=2, Ns=2, geometry="ball", radius=0.3,
                            grid=synth.sphere_grid(15.0, 30.0), snr_db=6.0, cond=1e2, n_k=80,
                            bins=(16, 40), on_grid=True, seed=1300)
    K = O.correlation(w.Xnoise)
    Kinv, _ = ctx.noise_inverse(dev(K))
    st = ctx.steering(dev(w.H))
    plan = binding.Plan(ctx, [dict(X=dev(w.X[0]), Kinv=Kinv, st=st, Ns=2, n_az=w.grid.n_az,
                                   n_el=w.grid.n_el)], form="sq", precision="fp32",
                        method="bidiag", abs_tol=ABS_TOL)
    plan.run()
    torch.cuda.synchronize()
    _, _, Pbar = ctx.localize(dev(w.X[:1]), dev(K), st, 2, w.grid.n_az, w.grid.n_el, form="sq",
                              precision="fp32", method="bidiag", abs_tol=ABS_TOL)
    assert np.array_equal(host(plan.outputs[0]["Pbar"]), host(Pbar)[0])
    s = binding.Stream(ctx, dev(K), st, 2, w.grid.n_az, w.grid.n_el, 40, 10, form="sq",
                       precision="fp32", method="bidiag", abs_tol=ABS_TOL)
    X = np.concatenate(list(w.X), 0)
    for n in range(X.shape[0] // 10):
        _, _, Pb, _ = s.push(dev(X[n * 10:(n + 1) * 10]))
    ref = O.localize_block(X[-40:], K, w.H, 2, w.grid.n_az, w.grid.n_el, "sq")
    assert np.abs(host(Pb) - ref["Pbar"]).max() / ref["Pbar"].max() < 1e-4
    plan.close()
    s.close()
    st.close()
