"""SEVD and GEVD variants of the decomposition (ssl_sevd, ssl_gevd) against
the FP64 oracle: eigenvalues, the noise-subspace projector, the defining
identities (R E = K E Lambda, E^H K E = I) in FP32, the GEVD-MUSIC model's
exact orthogonality of the noise eigenvectors to the source, and the whole
localization with either variant feeding the spectrum."""

import numpy as np
import pytest

import oracle.gsvd_music as O
from gpu_common import context, dev, host
from paper_2504_03373_gb300 import synth

pytestmark = pytest.mark.gpu


def _crand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _psd(rng, B, M, T):
    X = _crand(rng, B, M, T)
    return np.matmul(X, np.conj(np.swapaxes(X, -1, -2))) / T


def _proj(E, n0):
    """Orthogonal projector onto the span of columns n0.. of E (any basis)."""
    Q, _ = np.linalg.qr(np.asarray(E, complex)[..., :, n0:])
    return np.matmul(Q, np.conj(np.swapaxes(Q, -1, -2)))


@pytest.mark.parametrize("M", [8, 17, 32, 60])
def test_sevd_matches_oracle(M):
    ctx = context()
    rng = np.random.default_rng(900 + M)
    B = 12
    R = _psd(rng, B, M, 2 * M)[None].astype(np.complex64)
    lam, E, status = ctx.sevd(dev(R))
    assert (host(status) == 0).all()
    E_ref, lam_ref = O.sevd(R[0].astype(complex))
    l = host(lam)[0].astype(float)
    assert np.abs(l - lam_ref).max() / lam_ref.max() < 2e-5
    Eh = host(E)[0].astype(complex)
    EH = np.conj(np.swapaxes(Eh, -1, -2))
    assert np.abs(np.matmul(EH, Eh) - np.eye(M)).max() < 5e-5
    rec = np.matmul(Eh * l[..., None, :], EH)
    assert np.abs(rec - R[0]).max() / np.abs(R[0]).max() < 5e-5
    gap = (lam_ref[:, 2] - lam_ref[:, 3]) / lam_ref[:, 0]
    ok = gap > 1e-2
    perr = np.linalg.norm(_proj(Eh, 3) - _proj(E_ref, 3), axis=(-2, -1))
    assert perr[ok].max() < 1e-3, perr


@pytest.mark.parametrize("M,cond", [(8, 1e2), (16, 1e3), (60, 1e2)])
def test_gevd_matches_oracle(M, cond):
    ctx = context()
    rng = np.random.default_rng(950 + M)
    B = 10
    Q = synth.haar_unitary(rng, B, M)
    s = np.logspace(0, -np.log10(cond), M)
    K = np.matmul(Q * s[None, None, :], np.conj(np.swapaxes(Q, -1, -2))).astype(np.complex64)
    R = _psd(rng, B, M, 2 * M)[None].astype(np.complex64)
    lam, E, status = ctx.gevd(dev(R), dev(K))
    assert (host(status) == 0).all()
    Kd, Rd = K.astype(complex), R[0].astype(complex)
    E_ref, lam_ref = O.gevd(Kd, Rd)
    l = host(lam)[0].astype(float)
    rel = np.abs(l - lam_ref).max() / lam_ref.max()
    Eh = host(E)[0].astype(complex)
    EH = np.conj(np.swapaxes(Eh, -1, -2))
    kortho = np.abs(np.matmul(EH, np.matmul(Kd, Eh)) - np.eye(M)).max()
    res = np.abs(np.matmul(Rd, Eh) - np.matmul(Kd, Eh) * l[..., None, :]).max()
    res /= np.abs(Rd).max() * np.abs(Eh).max()
    print(f"\nM {M} cond {cond:.0e}: lambda err {rel:.2e}, E^H K E - I {kortho:.2e}, "
          f"residual {res:.2e}")
    assert rel < 1e-4
    assert kortho < 1e-3
    assert res < 1e-4


def test_gevd_noise_vectors_orthogonal_to_source():
    """R = s a a^H + sigma^2 K (noiseless GEVD-MUSIC model): the noise
    eigenvectors are orthogonal to a, so |a^H E_n| is at the FP32 level,
    while the GSVD's are not: the left singular vectors of K^-1 R separate
    the source direction exactly only when K = I."""
    ctx = context()
    rng = np.random.default_rng(990)
    B, M, s, sigma2 = 6, 8, 5.0, 0.3
    Q = synth.haar_unitary(rng, B, M)
    sv = np.logspace(0, -3, M)
    K = np.matmul(Q * sv[None, None, :], np.conj(np.swapaxes(Q, -1, -2)))
    a = np.exp(1j * rng.uniform(0, 2 * np.pi, (B, M)))
    R = s * a[:, :, None] * np.conj(a[:, None, :]) + sigma2 * K
    lam, E, status = ctx.gevd(dev(R[None]), dev(K))
    assert (host(status) == 0).all()
    En = host(E)[0][:, :, 1:].astype(complex)
    En = En / np.linalg.norm(En, axis=1, keepdims=True)
    leak = np.abs(np.einsum("bm,bmi->bi", np.conj(a), En)).max() / np.sqrt(M)
    assert leak < 1e-4, leak
    sig, Eg, _ = ctx.gsvd(dev(R[None]), dev(K))
    Eg = host(Eg)[0][:, :, 1:].astype(complex)
    leak_g = np.abs(np.einsum("bm,bmi->bi", np.conj(a), Eg)).max() / np.sqrt(M)
    assert leak_g > 1e-2


@pytest.mark.parametrize("variant", ["sevd", "gevd"])
def test_localization_with_variant(variant):
    """The 8-mic workload localized through either variant's noise subspace
    (SQ form): P-bar within the FP32 tolerance of the oracle's same variant,
    and the same peaks where the margin allows."""
    ctx = context()
    w = synth.uca8_single_source(seed=31, nblk=2)
    K = O.correlation(w.Xnoise)
    R = ctx.correlate(dev(w.X))
    if variant == "sevd":
        _, E, status = ctx.sevd(R)
    else:
        _, E, status = ctx.gevd(R, dev(K))
    assert (host(status) == 0).all()
    st = ctx.steering(dev(w.H))
    _, Pbar = ctx.music_spectrum(E, 1, st, form="sq", precision="fp32", want_P=False)
    idx, _ = ctx.peaks(Pbar, w.grid.n_az, w.grid.n_el, 1)
    for k in range(2):
        Rk = O.correlation(w.X[k])
        Ek = O.sevd(Rk)[0] if variant == "sevd" else O.gevd(K, Rk)[0]
        ref = O.bin_sum(O.spectrum(w.H, O.noise_subspace(Ek, 1), "sq"))
        err = np.abs(host(Pbar)[k] - ref).max() / ref.max()
        assert err < 1e-4, (k, err)
        if O.peak_margin(ref, w.grid.n_az, w.grid.n_el, 1) > 1e-3:
            assert int(host(idx)[k][0]) == int(O.peaks(ref, w.grid.n_az, w.grid.n_el, 1)[0][0])
    st.close()
