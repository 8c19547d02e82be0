"""Mixed batches (ssl_plan_*): arrays of different M, T, Ns and direction
grids in one launch per stage.  Every array's result equals the stateless
single-array call bit for bit (same kernels' arithmetic, same pair order),
matches the FP64 oracle within the path's tolerance, and follows new input
data when the captured graph is replayed."""

import numpy as np
import pytest
import torch

import oracle.gsvd_music as O
from gpu_common import context, dev, host
from paper_2504_03373_gb300 import binding, synth

pytestmark = pytest.mark.gpu

ABS_TOL = 2.0 ** -23
# (M, Ns, T, n_el): every Jacobi size class, ragged M, one- and
# two-dimensional grids, T above and below M
SHAPES = [(8, 1, 50, 1), (16, 2, 40, 3), (32, 3, 50, 3), (60, 3, 50, 3), (64, 1, 70, 1),
          (12, 1, 30, 1), (40, 2, 60, 3), (17, 3, 50, 3), (8, 2, 20, 3)]


def _grid(n_el):
    return synth.azimuth_grid(15.0) if n_el == 1 else synth.sphere_grid(15.0, 60.0)


def _arrays(bins=(16, 40), seed0=300, nblk=1):
    out = []
    for i, (M, Ns, T, n_el) in enumerate(SHAPES):
        w = synth.make_workload(M=M, T=T, nblk=nblk, Ns=Ns, geometry="ball", radius=0.4,
                                grid=_grid(n_el), snr_db=6.0, cond=1e2, n_k=max(50, 4 * M),
                                bins=bins, on_grid=True, seed=seed0 + i)
        out.append(w)
    return out


def _plan(ctx, ws, form, precision, k=0, **kw):
    arrays, keep = [], []
    for w in ws:
        K = dev(O.correlation(w.Xnoise))
        Kinv, st = ctx.noise_inverse(K)
        assert (host(st) == 0).all()
        steer = ctx.steering(dev(w.H))
        arrays.append(dict(X=dev(w.X[k]), Kinv=Kinv, st=steer, Ns=w.Ns, n_az=w.grid.n_az,
                           n_el=w.grid.n_el))
        keep.append((K, steer))
    plan = binding.Plan(ctx, arrays, form=form, precision=precision, abs_tol=ABS_TOL, **kw)
    return plan, arrays, keep


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_plan_equals_single_array_calls(precision):
    ctx = context()
    ws = _arrays()
    plan, arrays, keep = _plan(ctx, ws, "abs", precision, graph=True)
    info = plan.info()
    assert info["n_items"] == len(ws) and info["n_bins"] == sum(w.H.shape[0] for w in ws)
    assert info["graph"] and info["launches"] == 5
    assert info["class_of_m"] == {M: (16 if M <= 16 else 32 if M <= 32 else 64)
                                  for M, _, _, _ in SHAPES}
    plan.run()
    torch.cuda.synchronize()
    for w, a, out, (K, steer) in zip(ws, arrays, plan.outputs, keep):
        idx, val, Pbar = ctx.localize(a["X"][None], K, steer, w.Ns, w.grid.n_az, w.grid.n_el,
                                      form="abs", precision=precision, abs_tol=ABS_TOL)
        assert int(host(out["status"])[0]) == 0
        assert np.array_equal(host(out["Pbar"]), host(Pbar)[0])
        assert np.array_equal(host(out["peak_idx"]), host(idx)[0])
        assert np.array_equal(host(out["peak_val"]), host(val)[0])
    plan.close()


def test_plan_matches_oracle_and_autotunes():
    """SQ form (determined for every array), FP32 spectrum: P-bar within the
    FP32 tolerance of the oracle and the same peaks wherever the oracle's
    margin exceeds it; the autotuner's size classes all hold their M."""
    ctx = context()
    ws = _arrays(seed0=400)
    plan, arrays, keep = _plan(ctx, ws, "sq", "fp32", graph=True, autotune=True)
    info = plan.info()
    for M, cls in info["class_of_m"].items():
        assert cls in (16, 32, 64) and cls >= M
    assert info["autotune_ms"] > 0
    plan.run()
    torch.cuda.synchronize()
    for w, out in zip(ws, plan.outputs):
        K = O.correlation(w.Xnoise)
        ref = O.localize_block(w.X[0], K, w.H, w.Ns, w.grid.n_az, w.grid.n_el, "sq")
        Pbar = host(out["Pbar"]).astype(np.float64)
        err = np.abs(Pbar - ref["Pbar"]).max() / ref["Pbar"].max()
        assert err < 1e-4, (w.H.shape, err)
        if O.peak_margin(ref["Pbar"], w.grid.n_az, w.grid.n_el, w.Ns) > 1e-3:
            assert sorted(host(out["peak_idx"]).tolist()) == sorted(ref["idx"].tolist())
    plan.close()


def test_graph_replay_follows_new_input():
    ctx = context()
    ws = _arrays(seed0=500, nblk=2)
    plan, arrays, keep = _plan(ctx, ws, "abs", "bf16", graph=True)
    plan.run()
    torch.cuda.synchronize()
    first = [host(o["Pbar"]).copy() for o in plan.outputs]
    for w, a in zip(ws, arrays):  # the second block, in place
        a["X"].copy_(dev(w.X[1]))
    plan.run()
    torch.cuda.synchronize()
    for w, a, out, f, (K, steer) in zip(ws, arrays, plan.outputs, first, keep):
        _, _, Pbar = ctx.localize(a["X"][None], K, steer, w.Ns, w.grid.n_az, w.grid.n_el,
                                  form="abs", precision="bf16", abs_tol=ABS_TOL)
        assert np.array_equal(host(out["Pbar"]), host(Pbar)[0])
        assert not np.array_equal(host(out["Pbar"]), f)
    plan.close()


def test_plan_rejects_mixed_precision():
    ctx = context()
    ws = _arrays()[:2]
    arrays, keep = [], []
    for w in ws:
        Kinv, _ = ctx.noise_inverse(dev(O.correlation(w.Xnoise)))
        steer = ctx.steering(dev(w.H))
        keep.append(steer)
        arrays.append(dict(X=dev(w.X[0]), Kinv=Kinv, st=steer, Ns=w.Ns, n_az=w.grid.n_az,
                           n_el=w.grid.n_el))
    items = (binding.BatchItem * 2)()
    outs = []
    for i, a in enumerate(arrays):
        T, B, M = a["X"].shape
        o = torch.empty(4, dtype=torch.int32, device="cuda")
        v = torch.empty(4, dtype=torch.float32, device="cuda")
        outs.append((o, v))
        items[i].cfg = binding.Config(M, T, B, a["Ns"], a["n_az"], a["n_el"], 0,
                                      binding.PRECISION["bf16" if i == 0 else "fp32"],
                                      binding.jacobi_opts())
        items[i].X, items[i].Kinv = a["X"].data_ptr(), a["Kinv"].data_ptr()
        items[i].steering = a["st"].handle
        items[i].peak_idx, items[i].peak_val = o.data_ptr(), v.data_ptr()
    import ctypes
    h = ctypes.c_void_p()
    st = binding.load().ssl_plan_create(ctx.handle, 2, items, 0, ctypes.byref(h))
    assert st == 1  # SSL_E_INVALID_ARG
    assert "disagree" in ctx.last_error()
