"""Stream processing (ssl_stream_*): the sliding-window form of eq. 3 with a
warm-started decomposition.  After every push the result matches the FP64
oracle on the window of the last T frames (including windows that wrap the
device ring), and continuing from the previous E takes far fewer rotations
than a cold start on the same window."""

import numpy as np
import pytest
import torch

import oracle.gsvd_music as O
from gpu_common import context, dev, host
from paper_2504_03373_gb300 import binding, synth

pytestmark = pytest.mark.gpu

ABS_TOL = 2.0 ** -23


def _frames(M, Ns, seed, nblk=4, bins=(16, 48)):
    w = synth.make_workload(M=M, T=50, nblk=nblk, Ns=Ns, geometry="ball", radius=0.3,
                            grid=synth.sphere_grid(15.0, 30.0), snr_db=6.0, cond=1e2,
                            n_k=max(50, 4 * M), bins=bins, on_grid=True, seed=seed)
    X = np.concatenate(list(w.X), axis=0)  # consecutive frames [nblk*T][B][M]
    return w, X


@pytest.mark.parametrize("M,Ns,T,hop", [(16, 2, 50, 5), (8, 1, 40, 7), (60, 3, 50, 10)])
def test_stream_matches_oracle_on_each_window(M, Ns, T, hop):
    ctx = context()
    w, X = _frames(M, Ns, seed=700 + M)
    K = O.correlation(w.Xnoise)
    st = ctx.steering(dev(w.H))
    s = binding.Stream(ctx, dev(K), st, Ns, w.grid.n_az, w.grid.n_el, T, hop, form="sq",
                       precision="fp32", abs_tol=ABS_TOL)
    n_push = X.shape[0] // hop
    checked = 0
    for n in range(n_push):
        idx, val, Pbar, _ = s.push(dev(X[n * hop:(n + 1) * hop]))
        end = (n + 1) * hop
        if end < T or (n % 3 != 2 and n != n_push - 1):
            continue
        ref = O.localize_block(X[end - T:end], K, w.H, Ns, w.grid.n_az, w.grid.n_el, "sq")
        err = np.abs(host(Pbar).astype(np.float64) - ref["Pbar"]).max() / ref["Pbar"].max()
        assert err < 1e-4, (n, err)
        if O.peak_margin(ref["Pbar"], w.grid.n_az, w.grid.n_el, Ns) > 1e-3:
            assert sorted(host(idx).tolist()) == sorted(ref["idx"].tolist()), n
        checked += 1
    assert checked >= 3
    s.close()
    st.close()


def test_warm_start_needs_fewer_rotations():
    ctx = context()
    M, Ns, T, hop = 32, 3, 50, 5
    w, X = _frames(M, Ns, seed=750, nblk=3)
    K = O.correlation(w.Xnoise)
    st = ctx.steering(dev(w.H))
    s = binding.Stream(ctx, dev(K), st, Ns, w.grid.n_az, w.grid.n_el, T, hop, form="abs",
                       precision="bf16", abs_tol=ABS_TOL)
    Kinv, _ = ctx.noise_inverse(dev(K))
    warm, cold = [], []
    for n in range(X.shape[0] // hop):
        _, _, _, stats = s.push(dev(X[n * hop:(n + 1) * hop]), stats=True)
        end = (n + 1) * hop
        if end >= T + 2 * hop:
            R = ctx.correlate(dev(X[end - T:end][None]))
            _, _, status, cst = ctx.gsvd(R, Kinv, kinv=True, stats=True, abs_tol=ABS_TOL)
            assert (host(status) == 0).all()
            warm.append(host(stats)[:, 1].mean())
            cold.append(host(cst)[0, :, 1].mean())
    assert len(warm) >= 5
    assert np.mean(warm) < 0.5 * np.mean(cold), (np.mean(warm), np.mean(cold))
    s.close()
    st.close()


def test_stream_rejects_bad_hop():
    ctx = context()
    w, _ = _frames(8, 1, seed=760, nblk=1)
    st = ctx.steering(dev(w.H))
    with pytest.raises(binding.SSLError):
        binding.Stream(ctx, dev(O.correlation(w.Xnoise)), st, 1, w.grid.n_az, w.grid.n_el,
                       T=20, hop=21)
    st.close()
