"""The split decomposition (method "split"): the noise subspace of eq. 4
without its individual vectors, which is all the SQ form of eq. 5 needs
(it depends on E_n only through E_n E_n^H).  Graded against the FP64 oracle's
full SVD by the basis-invariant quantities:

* the Ns signal singular values (5e-5 of sigma_max) and vectors' projector
  (1e-4 Frobenius where the relative signal/noise gap is >= 1e-2, 2e-6 / gap
  below, as for the full iteration);
* E unitary (its trailing columns are an orthonormal basis of the
  complement of E_s) and the other columns' norms carrying the noise energy;
* Pbar of the whole path (SQ form) within the spectrum precision's
  tolerance, peaks exact where the oracle's margin exceeds it;
* the hand-back to the paper's bidiagonalisation route (matrices the rounds
  would not resolve within the split's sweep limit), the full iteration for
  the sizes the split does not take, and the refusals of the forms that need
  the individual noise vectors."""

import ctypes

import numpy as np
import pytest
import torch

import oracle.gsvd_music as O
from gpu_common import context, dev, host, max_rel, projector, signal_gap
from paper_2504_03373_gb300 import binding, synth

pytestmark = pytest.mark.gpu

ABS_TOL = 2.0 ** -23
E_INVALID_ARG, E_NO_CONVERGENCE, E_UNSUPPORTED = 1, 3, 9
TOL = {"fp32": 1e-4, "tf32x3": 1e-4, "tf32": 1e-3, "bf16": 1e-2}


def _bound(lo, Ns):
    gap = signal_gap(lo, Ns)
    return np.where(gap >= 1e-2, 1e-4, 2e-6 / np.maximum(gap, 1e-30))


def _check_split(sig, E, K, R, Ns):
    A, Eo, lo, _ = O.gsvd(K.astype(np.complex128), R.astype(np.complex128))
    nblk, B, M = sig.shape
    for k in range(nblk):
        smax = lo[k, :, :1]
        # the signal singular values, sorted
        assert (np.abs(sig[k][:, :Ns] - lo[k][:, :Ns]) / smax).max() < 5e-5
        assert (np.diff(sig[k][:, :Ns], axis=1) <= 0).all()
        # the other columns carry the noise energy sum_{i > Ns} sigma_i^2
        e_noise = (sig[k][:, Ns:].astype(np.float64) ** 2).sum(1)
        assert (np.abs(e_noise - (lo[k][:, Ns:] ** 2).sum(1)) / smax[:, 0] ** 2).max() < 1e-4
        assert (np.diff(sig[k][:, Ns:], axis=1) <= 0).all()
        EH = np.conj(np.swapaxes(E[k], 1, 2)).astype(np.complex128)
        assert np.abs(np.matmul(EH, E[k]) - np.eye(M)).max() < 1e-5
        err = np.linalg.norm(projector(E[k], Ns) - projector(Eo[k], Ns), axis=(1, 2))
        assert (err <= _bound(lo[k], Ns)).all(), (err.max(), signal_gap(lo[k], Ns).min())


@pytest.mark.parametrize("angles", ["f64", "f32"])
def test_split_on_the_60_mic_workload(angles):
    ctx = context()
    w = synth.ball60_three_sources(seed=2, nblk=2)
    K = O.correlation(w.Xnoise).astype(np.complex64)
    R = ctx.correlate(dev(w.X))
    sig, E, status = ctx.gsvd(R, dev(K), method="split", split_ns=3, abs_tol=ABS_TOL,
                              angles=angles)
    torch.cuda.synchronize()
    assert ctx.device_flags() == 0
    assert (host(status) == 0).all()
    _check_split(host(sig), host(E), K, host(R), 3)


@pytest.mark.parametrize("M,Ns", [(6, 2), (9, 3), (16, 1), (17, 5), (33, 4), (33, 8), (60, 2),
                                  (64, 8), (64, 3)])
def test_split_random(M, Ns):
    """Random matrices with a stretched signal subspace; (M, Ns) across the
    one- and two-row layouts and both pivot capacities."""
    ctx = context()
    rng = np.random.default_rng(700 + 10 * M + Ns)
    nblk, B, T = 2, 5, max(2 * M, 20)
    G = synth.noise_mixing(rng, B, M, 1e2)
    K = np.matmul(G, np.conj(np.swapaxes(G, 1, 2))).astype(np.complex64)
    X = synth.cgauss(rng, (nblk, T, B, M)).astype(np.complex64)
    X[..., :Ns] *= 8.0
    R = np.stack([O.correlation(X[k]) for k in range(nblk)]).astype(np.complex64)
    sig, E, status = ctx.gsvd(dev(R), dev(K), method="split", split_ns=Ns)
    torch.cuda.synchronize()
    assert ctx.device_flags() == 0
    assert (host(status) == 0).all()
    _check_split(host(sig), host(E), K, R, Ns)


def test_sizes_the_split_does_not_take_run_the_full_iteration():
    """Ns > M / 3 and Ns > 8: the full iteration (every column a singular vector)."""
    ctx = context()
    rng = np.random.default_rng(811)
    for M, Ns in [(8, 3), (40, 12)]:
        B = 3
        G = synth.noise_mixing(rng, B, M, 1e2)
        K = np.matmul(G, np.conj(np.swapaxes(G, 1, 2))).astype(np.complex64)
        X = synth.cgauss(rng, (1, 3 * M, B, M)).astype(np.complex64)
        R = O.correlation(X[0])[None].astype(np.complex64)
        sig, E, status = ctx.gsvd(dev(R), dev(K), method="split", split_ns=Ns)
        ref, Eref, stref = ctx.gsvd(dev(R), dev(K))
        torch.cuda.synchronize()
        assert (host(status) == 0).all()
        assert np.array_equal(host(sig), host(ref)) and np.array_equal(host(E), host(Eref))


def test_hand_back_to_the_bidiagonal_route():
    """An Ns above the number of sources leaves two noise values on either side
    of the split: the rounds would converge slowly, so the split hands those
    matrices to the paper's bidiagonalisation route, whose result they then
    carry bit for bit (the same kernel on the same R and K^-1), and the
    projector stays within its bound.  With a one-sweep limit the hand-back
    also covers the matrices the rounds leave unresolved, and the route
    reports its own limit (status 0 or NO_CONVERGENCE, flag raised with it).
    (Held to the relative test alone: the absolute test deliberately leaves
    pairs of noise-floor columns unconverged, so with abs_tol neither route
    resolves a split between two noise values.)"""
    ctx = context()
    w = synth.ball60_three_sources(seed=5, nblk=1)
    K = O.correlation(w.Xnoise).astype(np.complex64)
    R = ctx.correlate(dev(w.X))
    for sweeps in (1, 0):
        opts = dict(split_ns=5, max_sweeps=sweeps) if sweeps else dict(split_ns=5)
        sig, E, status = ctx.gsvd(R, dev(K), method="split", **opts)
        torch.cuda.synchronize()
        flags = ctx.device_flags()
        sgb, Eb, stb = ctx.gsvd(R, dev(K), method="bidiag", **opts)
        torch.cuda.synchronize()
        assert ctx.device_flags() == flags
        st, s_, sb = host(status), host(sig), host(sgb)
        handed = (s_ == sb).all(axis=-1)
        assert handed.any()
        assert np.array_equal(st[handed], host(stb)[handed])
        assert np.array_equal(host(E)[handed], host(Eb)[handed])
        assert np.isin(st, [0, E_NO_CONVERGENCE]).all()
        assert bool(flags & binding.FLAG_NO_CONVERGENCE) == bool((st == E_NO_CONVERGENCE).any())
    assert (st == 0).all()
    A, Eo, lo, _ = O.gsvd(K.astype(np.complex128), host(R)[0].astype(np.complex128))
    err = np.linalg.norm(projector(host(E)[0], 5) - projector(Eo, 5), axis=(1, 2))
    assert (err <= _bound(lo, 5)).all(), (err.max(), signal_gap(lo, 5).min())


@pytest.mark.parametrize("precision", ["fp32", "tf32x3", "bf16"])
def test_localize_with_the_split(precision):
    ctx = context()
    w = synth.ball60_three_sources(seed=2, nblk=3)
    K = O.correlation(w.Xnoise).astype(np.complex64)
    st = ctx.steering(dev(w.H))
    idx, val, Pbar = ctx.localize(dev(w.X), dev(K), st, 3, w.grid.n_az, w.grid.n_el, form="sq",
                                  precision=precision, abs_tol=ABS_TOL, method="split")
    torch.cuda.synchronize()
    assert ctx.device_flags() == 0
    graded = 0
    for k in range(w.nblk):
        ref = O.localize_block(w.X[k], K, w.H.astype(np.complex64), 3, w.grid.n_az, w.grid.n_el,
                               "sq")
        assert max_rel(host(Pbar)[k], ref["Pbar"]) < TOL[precision]
        if O.peak_margin(ref["Pbar"], w.grid.n_az, w.grid.n_el, 3) > TOL[precision]:
            graded += 1
            assert list(host(idx)[k]) == list(ref["idx"]), k
    assert graded > 0 or precision == "bf16"
    st.close()


def test_forms_that_need_the_noise_vectors_are_refused():
    ctx = context()
    w = synth.uca8_single_source(seed=1, nblk=1)
    K = dev(O.correlation(w.Xnoise).astype(np.complex64))
    st = ctx.steering(dev(w.H))
    with pytest.raises(binding.SSLError) as e:
        ctx.localize(dev(w.X), K, st, 1, w.grid.n_az, w.grid.n_el, form="abs", method="split")
    assert e.value.status == E_UNSUPPORTED
    R = ctx.correlate(dev(w.X))
    with pytest.raises(binding.SSLError) as e:
        ctx.sevd(R, method="split", split_ns=1)
    assert e.value.status == E_UNSUPPORTED
    with pytest.raises(binding.SSLError) as e:  # no Ns
        ctx.gsvd(R, K, method="split")
    assert e.value.status == E_INVALID_ARG
    srv = binding.Server(ctx, hbm_budget_bytes=1 << 30, max_batch=4)
    with pytest.raises(binding.SSLError) as e:
        srv.session(K, st, 1, w.grid.n_az, w.grid.n_el, w.T, form="abs", method="split")
    assert e.value.status == E_UNSUPPORTED
    srv.close()
    with pytest.raises(binding.SSLError) as e:
        binding.Stream(ctx, K, st, 1, w.grid.n_az, w.grid.n_el, w.T, w.T, form="abs",
                       method="split")
    assert e.value.status == E_UNSUPPORTED
    Kinv, _ = ctx.noise_inverse(K)
    with pytest.raises(binding.SSLError) as e:
        binding.Plan(ctx, [dict(X=dev(w.X[0]), Kinv=Kinv, st=st, Ns=1, n_az=w.grid.n_az,
                                n_el=w.grid.n_el)], form="sq", method="split")
    assert e.value.status == E_UNSUPPORTED
    assert ctx.device_flags() == 0
    st.close()


def test_split_in_sessions_and_streams():
    """A session on the split route gives each block the stateless call's
    result bit for bit; a stream with it matches the oracle on every window."""
    ctx = context()
    opts = dict(form="sq", precision="bf16", abs_tol=ABS_TOL, method="split")
    w = synth.ball60_three_sources(seed=7, nblk=2)
    Kn = O.correlation(w.Xnoise).astype(np.complex64)
    K = dev(Kn)
    st = ctx.steering(dev(w.H))
    ref = [ctx.localize(dev(w.X[k:k + 1]), K, st, 3, w.grid.n_az, w.grid.n_el, **opts)
           for k in range(2)]
    srv = binding.Server(ctx, hbm_budget_bytes=4 << 30, max_batch=8)
    se = srv.session(K, st, 3, w.grid.n_az, w.grid.n_el, w.T, queue_depth=2, **opts)
    tickets = [se.submit(dev(w.X[k])) for k in range(2)]
    for k, t in enumerate(tickets):
        r = se.wait(t, timeout_s=60.0)
        assert r["status"] == 0
        assert r["idx"] == [int(v) for v in host(ref[k][0])[0]]
        assert np.array_equal(np.array(r["val"], np.float32), host(ref[k][1])[0])
    se.close()
    srv.close()
    s = binding.Stream(ctx, K, st, 3, w.grid.n_az, w.grid.n_el, w.T, w.T, form="sq",
                       precision="fp32", abs_tol=ABS_TOL, method="split")
    for k in range(2):
        idx, _, Pbar, _ = s.push(dev(w.X[k]))
        torch.cuda.synchronize()
        r = O.localize_block(w.X[k], Kn, w.H.astype(np.complex64), 3, w.grid.n_az, w.grid.n_el,
                             "sq")
        assert max_rel(host(Pbar), r["Pbar"]) < 1e-4
        if O.peak_margin(r["Pbar"], w.grid.n_az, w.grid.n_el, 3) > 1e-4:
            assert list(host(idx)) == list(r["idx"])
    s.close()
    assert ctx.device_flags() == 0
    st.close()
