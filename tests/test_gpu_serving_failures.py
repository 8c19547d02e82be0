"""Failure paths of the serving loop, injected on the host (no device fault):

* a session destroyed while its blocks are queued and on the GPU (its client
  went away): the other sessions' blocks in the same batches are served with
  the same results as alone, and the server drains;
* a malformed block (NaN frames): its result carries SSL_E_NONFINITE, the
  context raises the sticky flag, and the blocks batched with it are
  unaffected;
* a wedged poller (nobody steps the server for a while): submits beyond the
  queue depth are refused, the rest are served once stepping resumes, and
  their latency includes the stall;
* a late-stamped arrival counts its delay in the latency;
* ssl_session_wait with a deadline that has passed returns SSL_E_TIMEOUT and
  leaves the ticket to a later wait.
"""

import time

import numpy as np
import pytest
import torch

import oracle.gsvd_music as O
from gpu_common import context, dev, host
from paper_2504_03373_gb300 import binding, synth

pytestmark = pytest.mark.gpu

E_NONFINITE, E_ADMISSION, E_TIMEOUT = 4, 6, 7


def _uca(seed, nblk=3):
    w = synth.uca8_single_source(seed=seed, nblk=nblk)
    K = O.correlation(w.Xnoise).astype(np.complex64)
    return w, K


def _block(w, k):
    return torch.from_numpy(np.ascontiguousarray(w.X[k].astype(np.complex64))).pin_memory()


def _alone(ctx, w, K, st, k):
    idx, val, _ = ctx.localize(dev(w.X[k:k + 1]), dev(K), st, 1, w.grid.n_az, w.grid.n_el,
                               form="sq", precision="bf16", abs_tol=2.0 ** -23)
    return [int(v) for v in host(idx)[0]], host(val)[0]


def _setup(ctx, n, queue_depth=3, seed0=300):
    srv = binding.Server(ctx, hbm_budget_bytes=4 << 30, max_batch=64)
    arrays, sessions, steers = [], [], []
    for i in range(n):
        w, K = _uca(seed0 + i)
        st = ctx.steering(dev(w.H))
        arrays.append((w, K))
        steers.append(st)
        sessions.append(srv.session(dev(K), st, 1, w.grid.n_az, w.grid.n_el, w.T, form="sq",
                                    precision="bf16", queue_depth=queue_depth,
                                    abs_tol=2.0 ** -23))
    return srv, arrays, sessions, steers


def _teardown(srv, sessions, steers):
    for se in sessions:
        se.close()
    srv.close()
    for st in steers:
        st.close()


def test_session_destroyed_mid_flight():
    ctx = context()
    srv, arrays, sessions, steers = _setup(ctx, 4)
    tickets = []
    for k in range(3):
        for i, se in enumerate(sessions):
            tickets.append((i, k, se.submit(_block(arrays[i][0], k))))
        if k == 0:
            srv.run_step()  # the first blocks go to the GPU, the rest queue up
    # the client of session 0 goes away with blocks on the GPU and queued
    sessions[0].close()
    results = {}
    for i, k, t in tickets:
        if i != 0:
            results[(i, k)] = sessions[i].wait(t, timeout_s=60.0)
    st = srv.stats()
    assert st["sessions"] == 3 and st["blocks_pending"] == 0
    for i in range(1, 4):
        w, K = arrays[i]
        for k in range(3):
            r = results[(i, k)]
            assert r["status"] == 0
            idx, val = _alone(ctx, w, K, steers[i], k)
            assert r["idx"] == idx and np.array_equal(np.array(r["val"], np.float32), val)
    assert ctx.device_flags() == 0
    _teardown(srv, sessions, steers)


def test_malformed_block_is_flagged_and_isolated():
    ctx = context()
    srv, arrays, sessions, steers = _setup(ctx, 3)
    bad = _block(arrays[0][0], 0).clone()
    bad[7, 30, 3] = complex(float("nan"), 0.0)
    assert ctx.device_flags() == 0
    t_bad = sessions[0].submit(bad.pin_memory())
    t_ok = [sessions[i].submit(_block(arrays[i][0], 0)) for i in (1, 2)]
    r_bad = sessions[0].wait(t_bad, timeout_s=60.0)
    r_ok = [sessions[i].wait(t, timeout_s=60.0) for i, t in zip((1, 2), t_ok)]
    assert srv.stats()["batches"] == 1  # the three blocks shared one batch
    assert r_bad["status"] == E_NONFINITE
    assert ctx.device_flags() & binding.FLAG_NONFINITE
    for i, r in zip((1, 2), r_ok):
        w, K = arrays[i]
        idx, val = _alone(ctx, w, K, steers[i], 0)
        assert r["status"] == 0
        assert r["idx"] == idx and np.array_equal(np.array(r["val"], np.float32), val)
    # the session goes on serving well-formed blocks
    t = sessions[0].submit(_block(arrays[0][0], 1))
    assert sessions[0].wait(t, timeout_s=60.0)["status"] == 0
    assert ctx.device_flags() == 0
    _teardown(srv, sessions, steers)


def test_wedged_poller_then_recovery():
    ctx = context()
    srv, arrays, sessions, steers = _setup(ctx, 2, queue_depth=2)
    tickets = [(i, sessions[i].submit(_block(arrays[i][0], k))) for k in range(2)
               for i in range(2)]
    with pytest.raises(binding.SSLError) as e:  # both slots of session 0 are taken
        sessions[0].submit(_block(arrays[0][0], 2))
    assert e.value.status == E_ADMISSION
    stall_s = 0.2
    time.sleep(stall_s)  # nobody steps the server
    results = [(i, sessions[i].wait(t, timeout_s=60.0)) for i, t in tickets]
    for i, r in results:
        assert r["status"] == 0
        assert (r["t_done_ns"] - r["t_arrival_ns"]) * 1e-9 >= stall_s
    st = srv.stats()
    assert st["blocks_refused"] == 1 and st["blocks_done"] == 4 and st["blocks_pending"] == 0
    # slots are free again
    t = sessions[0].submit(_block(arrays[0][0], 2))
    assert sessions[0].wait(t, timeout_s=60.0)["status"] == 0
    _teardown(srv, sessions, steers)


def test_late_stamped_arrival_counts_its_delay():
    ctx = context()
    srv, arrays, sessions, steers = _setup(ctx, 1)
    delay_ns = 300_000_000
    t = sessions[0].submit(_block(arrays[0][0], 0), t_arrival_ns=binding.now_ns() - delay_ns)
    r = sessions[0].wait(t, timeout_s=60.0)
    assert r["status"] == 0
    assert r["t_done_ns"] - r["t_arrival_ns"] >= delay_ns
    assert srv.stats()["latency_max_ms"] >= delay_ns * 1e-6
    _teardown(srv, sessions, steers)


def test_wait_past_its_deadline_times_out_and_the_ticket_stays_valid():
    ctx = context()
    srv, arrays, sessions, steers = _setup(ctx, 1)
    t = sessions[0].submit(_block(arrays[0][0], 0))
    with pytest.raises(binding.SSLError) as e:
        sessions[0].wait(t, timeout_s=0.0)  # one step at most, then the deadline has passed
    assert e.value.status == E_TIMEOUT
    r = sessions[0].wait(t, timeout_s=60.0)
    assert r is not None and r["status"] == 0
    _teardown(srv, sessions, steers)
