"""The search range of the peak search (Sec. III-A, last step: peaks are
searched between theta_min and theta_max), attached to a steering object as a
direction mask: exact against the FP64 oracle on random spectra and lists,
within the spectrum tolerance on the 60-mic workload, and carried unchanged
through sessions, plans and streams (bit-identical to the stateless call)."""

import numpy as np
import pytest
import torch

import oracle.gsvd_music as O
from gpu_common import context, dev, host, max_rel
from paper_2504_03373_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def _random_lists(rng, D, k=4):
    sets = [set() for _ in range(D)]
    for d in range(D):
        for n in rng.choice(D, size=min(k, D), replace=False):
            if n != d:
                sets[d].add(int(n))
                sets[int(n)].add(d)
    ptr = np.zeros(D + 1, np.int32)
    ptr[1:] = np.cumsum([len(s) for s in sets])
    idx = np.concatenate([sorted(s) for s in sets]).astype(np.int32)
    return ptr, idx


@pytest.mark.parametrize("D,Ns", [(50, 3), (700, 8), (8192, 16)])
def test_peaks_with_a_range_match_the_oracle(D, Ns):
    ctx = context()
    rng = np.random.default_rng(900 + D)
    nblk, B, M = 3, 1, 4
    ptr, idx = _random_lists(rng, D)
    st = ctx.steering(dev(np.ones((B, D, M), np.complex64)))
    st.set_neighbours(torch.from_numpy(ptr), torch.from_numpy(idx))
    mask = rng.random(D) < 0.4
    st.set_search_range(mask)
    Pbar = rng.integers(0, 50, (nblk, D)).astype(np.float32)  # many ties
    gi, gv = ctx.peaks_nbr(torch.from_numpy(Pbar).cuda(), st, Ns)
    for k in range(nblk):
        io, vo = O.peaks_nbr(Pbar[k].astype(np.float64), ptr, idx, Ns, mask)
        assert list(host(gi)[k]) == list(io), k
        assert np.array_equal(host(gv)[k], vo.astype(np.float32)), k
    # removing the range gives the unrestricted search back
    st.set_search_range(None)
    gi, _ = ctx.peaks_nbr(torch.from_numpy(Pbar).cuda(), st, Ns)
    for k in range(nblk):
        io, _ = O.peaks_nbr(Pbar[k].astype(np.float64), ptr, idx, Ns)
        assert list(host(gi)[k]) == list(io)
    st.close()


def _azimuth_range(grid, lo_deg, hi_deg):
    """Mask of the grid directions whose azimuth lies in [lo_deg, hi_deg]."""
    u = grid.unit_vectors()
    az = np.degrees(np.arctan2(u[:, 1], u[:, 0])) % 360.0
    return (az >= lo_deg) & (az <= hi_deg)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_localize_with_an_azimuth_range(precision):
    ctx = context()
    w = synth.ball60_three_sources(seed=2, nblk=3)
    K = O.correlation(w.Xnoise).astype(np.complex64)
    mask = _azimuth_range(w.grid, 0.0, 180.0)
    st = ctx.steering(dev(w.H))
    st.set_search_range(mask)
    idx, val, Pbar = ctx.localize(dev(w.X), dev(K), st, 3, w.grid.n_az, w.grid.n_el, form="sq",
                                  precision=precision, abs_tol=2.0 ** -23)
    assert ctx.device_flags() == 0
    tol = {"fp32": 1e-4, "bf16": 1e-2}[precision]
    for k in range(w.nblk):
        ref = O.localize_block(w.X[k], K, w.H.astype(np.complex64), 3, w.grid.n_az,
                               w.grid.n_el, "sq", mask=mask)
        assert max_rel(host(Pbar)[k], ref["Pbar"]) < tol
        assert all(mask[d] for d in host(idx)[k] if d >= 0)
        if O.peak_margin(ref["Pbar"], w.grid.n_az, w.grid.n_el, 3, mask) > tol:
            assert list(host(idx)[k]) == list(ref["idx"]), k
    st.close()


def test_range_in_sessions_plans_and_streams():
    """Two 8-mic arrays in one serving class, one with a range over half of
    the azimuths and one without: every block's result equals the stateless
    call with the same steering object; likewise in a plan and a stream."""
    ctx = context()
    opts = dict(form="sq", precision="bf16", abs_tol=2.0 ** -23)
    arrays = []
    for i in range(2):
        w = synth.uca8_single_source(seed=40 + i, nblk=2)
        K = dev(O.correlation(w.Xnoise).astype(np.complex64))
        st = ctx.steering(dev(w.H))
        if i == 0:
            st.set_search_range(_azimuth_range(w.grid, 0.0, 175.0))
        ref = [ctx.localize(dev(w.X[k:k + 1]), K, st, 1, w.grid.n_az, w.grid.n_el, **opts)
               for k in range(2)]
        arrays.append(dict(w=w, K=K, st=st, ref=ref))
    srv = binding.Server(ctx, hbm_budget_bytes=2 << 30, max_batch=8)
    sess = [srv.session(a["K"], a["st"], 1, a["w"].grid.n_az, a["w"].grid.n_el, a["w"].T,
                        queue_depth=2, **opts) for a in arrays]
    tickets = [(i, k, sess[i].submit(dev(arrays[i]["w"].X[k]))) for k in range(2)
               for i in range(2)]
    for i, k, t in tickets:
        r = sess[i].wait(t, timeout_s=60.0)
        idx_ref, val_ref, _ = arrays[i]["ref"][k]
        assert r["status"] == 0
        assert r["idx"] == [int(v) for v in host(idx_ref)[0]], (i, k)
        assert np.array_equal(np.array(r["val"], np.float32), host(val_ref)[0]), (i, k)
    for se in sess:
        se.close()
    srv.close()
    items = []
    for a in arrays:
        Kinv, _ = ctx.noise_inverse(a["K"])
        items.append(dict(X=dev(a["w"].X[0]), Kinv=Kinv, st=a["st"], Ns=1,
                          n_az=a["w"].grid.n_az, n_el=a["w"].grid.n_el))
    plan = binding.Plan(ctx, items, form="sq", precision="bf16", abs_tol=2.0 ** -23)
    plan.run()
    torch.cuda.synchronize()
    for a, out in zip(arrays, plan.outputs):
        idx_ref, val_ref, _ = a["ref"][0]
        assert np.array_equal(host(out["peak_idx"]), host(idx_ref)[0])
        assert np.array_equal(host(out["peak_val"]), host(val_ref)[0])
    plan.close()
    a = arrays[0]
    w = a["w"]
    s = binding.Stream(ctx, a["K"], a["st"], 1, w.grid.n_az, w.grid.n_el, w.T, w.T, **opts)
    mask = _azimuth_range(w.grid, 0.0, 175.0)
    for k in range(2):
        idx, _, Pbar, _ = s.push(dev(w.X[k]))
        torch.cuda.synchronize()
        assert all(mask[d] for d in host(idx) if d >= 0)
        ref = O.localize_block(w.X[k], O.correlation(w.Xnoise).astype(np.complex64),
                               w.H.astype(np.complex64), 1, w.grid.n_az, w.grid.n_el, "sq",
                               mask=mask)
        if O.peak_margin(ref["Pbar"], w.grid.n_az, w.grid.n_el, 1, mask) > 1e-2:
            assert list(host(idx)) == list(ref["idx"])
    s.close()
    assert ctx.device_flags() == 0
    for a in arrays:
        a["st"].close()
