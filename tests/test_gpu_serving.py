"""Sessions and continuous batching through the C ABI: every block's result is
the same served alone (stateless ssl_localize) and in a mixed batch of many
arrays of two shape classes; admission refuses what does not fit."""

import numpy as np
import pytest
import torch

import oracle.gsvd_music as O
from gpu_common import context, dev, host
from paper_2504_03373_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def _arrays():
    """Four 8-mic arrays and two 16-mic arrays, each with its own geometry,
    noise field and sources."""
    out = []
    for i in range(4):
        w = synth.uca8_single_source(seed=20 + i, nblk=3)
        out.append(dict(w=w, Ns=1))
    for i in range(2):
        w = synth.make_workload(M=16, T=40, nblk=3, Ns=2, geometry="ball", radius=0.2,
                                grid=synth.sphere_grid(10.0, 30.0), snr_db=[5.0, 0.0],
                                cond=1e2, n_k=64, bins=(20, 60), on_grid=False, seed=40 + i)
        out.append(dict(w=w, Ns=2))
    return out


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_same_result_alone_and_in_the_mix(precision):
    ctx = context()
    arrays = _arrays()
    srv = binding.Server(ctx, hbm_budget_bytes=8 << 30, max_batch=64)
    sessions, steers = [], []
    for a in arrays:
        w = a["w"]
        K = O.correlation(w.Xnoise).astype(np.complex64)
        a["K"] = K
        st = ctx.steering(dev(w.H))
        steers.append(st)
        sessions.append(srv.session(dev(K), st, a["Ns"], w.grid.n_az, w.grid.n_el, w.T,
                                    form="abs", precision=precision, queue_depth=3,
                                    abs_tol=2.0 ** -23))
    # interleave the arrays' blocks; step the server between submissions so
    # that blocks arrive while earlier batches are on the GPU
    tickets = []
    for k in range(3):
        for i, (a, se) in enumerate(zip(arrays, sessions)):
            X = torch.from_numpy(np.ascontiguousarray(a["w"].X[k].astype(np.complex64)))
            tickets.append((i, k, se.submit(X.pin_memory())))
            if (len(tickets) % 4) == 0:
                srv.run_step()
    results = {}
    for i, k, t in tickets:
        results[(i, k)] = sessions[i].wait(t, timeout_s=60.0)
    stats = srv.stats()
    assert stats["blocks_done"] == len(tickets)
    assert stats["batches"] >= 2
    assert stats["latency_p99_ms"] > 0
    # alone: the stateless call, one block at a time
    for i, a in enumerate(arrays):
        w = a["w"]
        for k in range(3):
            idx, val, _ = ctx.localize(dev(w.X[k:k + 1]), dev(a["K"]), steers[i], a["Ns"],
                                       w.grid.n_az, w.grid.n_el, form="abs", precision=precision,
                                       abs_tol=2.0 ** -23)
            r = results[(i, k)]
            assert r["status"] == 0
            assert r["idx"] == [int(v) for v in host(idx)[0]], (i, k)
            assert np.array_equal(np.array(r["val"], np.float32), host(val)[0]), (i, k)
    for se in sessions:
        se.close()
    srv.close()
    for st in steers:
        st.close()


def test_admission_by_memory_budget_and_queue_depth():
    ctx = context()
    w = synth.uca8_single_source(seed=3, nblk=4)
    K = dev(O.correlation(w.Xnoise).astype(np.complex64))
    st = ctx.steering(dev(w.H))
    # footprint of one session: K^{-1} (209*8*8*8 B) + 2 slots of 50*209*8*8 B
    foot = 209 * 64 * 8 + 2 * 50 * 209 * 8 * 8
    srv = binding.Server(ctx, hbm_budget_bytes=int(1.5 * foot), max_batch=8)
    se = srv.session(K, st, 1, w.grid.n_az, 1, 50, queue_depth=2)
    with pytest.raises(binding.SSLError) as e:
        srv.session(K, st, 1, w.grid.n_az, 1, 50, queue_depth=2)
    assert e.value.status == 6  # SSL_E_ADMISSION
    X = [torch.from_numpy(np.ascontiguousarray(w.X[k].astype(np.complex64))) for k in range(3)]
    t0 = se.submit(X[0])
    t1 = se.submit(X[1])
    with pytest.raises(binding.SSLError) as e:
        se.submit(X[2])  # both slots in flight
    assert e.value.status == 6
    assert se.wait(t0)["status"] == 0
    assert se.wait(t1)["status"] == 0
    t2 = se.submit(X[2])  # a slot is free again
    assert se.wait(t2)["status"] == 0
    s = srv.stats()
    assert s["sessions_refused"] == 1 and s["blocks_refused"] == 1 and s["blocks_done"] == 3
    se.close()
    srv.close()
    st.close()


def test_same_result_alone_and_in_the_mix_with_60_mic_arrays_and_analytic_steering():
    """Three classes in one server (8-mic UCAs on stored tables, 32-mic and
    60-mic ball arrays each with its own analytic steering, generated in the
    spectrum kernel): every block's peaks and values are bit-identical served
    alone (the stateless call on one block) and in the mix."""
    ctx = context()
    arrays = []
    for i in range(3):
        arrays.append(dict(w=synth.uca8_single_source(seed=120 + i, nblk=2), Ns=1, analytic=False))
    for i, M in enumerate((32, 32, 60, 60, 60)):
        w = synth.make_workload(M=M, T=50, nblk=2, Ns=2, geometry="ball", radius=0.4,
                                grid=synth.sphere_grid(), snr_db=[8.0, 3.0], cond=1e2,
                                n_k=4 * M, bins=(16, 64), on_grid=False, seed=140 + i)
        arrays.append(dict(w=w, Ns=2, analytic=True))
    srv = binding.Server(ctx, hbm_budget_bytes=16 << 30, max_batch=64)
    sessions, steers = [], []
    for a in arrays:
        w = a["w"]
        a["K"] = O.correlation(w.Xnoise).astype(np.complex64)
        st = (binding.Steering.analytic(ctx, w.pos, w.grid.unit_vectors(), w.freqs)
              if a["analytic"] else ctx.steering(dev(w.H)))
        steers.append(st)
        sessions.append(srv.session(dev(a["K"]), st, a["Ns"], w.grid.n_az, w.grid.n_el, w.T,
                                    form="sq", precision="bf16", queue_depth=2,
                                    abs_tol=2.0 ** -23))
    tickets = []
    for k in range(2):
        for i, (a, se) in enumerate(zip(arrays, sessions)):
            X = dev(a["w"].X[k])  # device input, ordered after its producer
            tickets.append((i, k, se.submit(X)))
            if (len(tickets) % 3) == 0:
                srv.run_step()
    results = {(i, k): sessions[i].wait(t, timeout_s=120.0) for i, k, t in tickets}
    assert srv.stats()["blocks_done"] == len(tickets)
    for i, a in enumerate(arrays):
        w = a["w"]
        for k in range(2):
            idx, val, _ = ctx.localize(dev(w.X[k:k + 1]), dev(a["K"]), steers[i], a["Ns"],
                                       w.grid.n_az, w.grid.n_el, form="sq", precision="bf16",
                                       abs_tol=2.0 ** -23)
            r = results[(i, k)]
            assert r["status"] == 0
            assert r["idx"] == [int(v) for v in host(idx)[0]], (i, k)
            assert np.array_equal(np.array(r["val"], np.float32), host(val)[0]), (i, k)
    for se in sessions:
        se.close()
    srv.close()
    for st in steers:
        st.close()


def test_saved_session_restores_and_serves_the_same():
    """A session's saved state (config, queue depth, K^{-1}) restores on the
    same or another server and serves bit-identical results; states that do
    not fit the steering object, are corrupted or truncated are refused."""
    ctx = context()
    w = synth.uca8_single_source(seed=11, nblk=3)
    K = dev(O.correlation(w.Xnoise).astype(np.complex64))
    st = ctx.steering(dev(w.H))
    srv = binding.Server(ctx, hbm_budget_bytes=2 << 30, max_batch=8)
    se = srv.session(K, st, 1, w.grid.n_az, w.grid.n_el, w.T, form="sq", precision="bf16",
                     queue_depth=2, abs_tol=2.0 ** -23)
    X = [torch.from_numpy(np.ascontiguousarray(w.X[k].astype(np.complex64))).pin_memory()
         for k in range(3)]
    before = [se.wait(se.submit(x), timeout_s=60.0) for x in X]
    state = se.save()
    se.close()
    assert srv.stats()["sessions"] == 0
    srv2 = binding.Server(ctx, hbm_budget_bytes=2 << 30, max_batch=8)
    for server in (srv, srv2):
        se2 = binding.Session.restore(server, state, st)
        after = [se2.wait(se2.submit(x), timeout_s=60.0) for x in X]
        for a, b in zip(before, after):
            assert a["status"] == 0 and b["status"] == 0
            assert a["idx"] == b["idx"] and a["val"] == b["val"]
        se2.close()
    # refused: a steering object of another direction set, a damaged header,
    # a truncated state, a non-finite K^{-1}, a budget it does not fit
    st_other = ctx.steering(dev(np.ascontiguousarray(w.H[:, :36])))
    bad_header = bytearray(state)
    bad_header[0] ^= 0xFF
    nan_kinv = bytearray(state)
    nan_kinv[-4:] = np.array([np.nan], np.float32).tobytes()
    for args in ((srv, state, st_other), (srv, bytes(bad_header), st), (srv, state[:-8], st),
                 (srv, bytes(nan_kinv), st)):
        with pytest.raises(binding.SSLError) as e:
            binding.Session.restore(*args)
        assert e.value.status == 1  # SSL_E_INVALID_ARG
    tiny = binding.Server(ctx, hbm_budget_bytes=1 << 10, max_batch=8)
    with pytest.raises(binding.SSLError) as e:
        binding.Session.restore(tiny, state, st)
    assert e.value.status == 6  # SSL_E_ADMISSION
    assert ctx.device_flags() == 0
    for s_ in (tiny, srv2, srv):
        s_.close()
    st_other.close()
    st.close()
