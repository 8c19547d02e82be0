"""Direction sets that form no grid (the paper's 2522-direction measured
transfer functions, Sec. V): the neighbour-list peak search and the whole
path at the paper's own shape, against the FP64 oracle.

* Peaks: bit-exact indices and values on identical spectra (random neighbour
  graphs with many ties, the Fibonacci sphere's lists, and the grid's own
  8-neighbourhood lists, which must reproduce the grid search).
* Paper shape (60 mics, 73 bins, 2522 directions, Ns = 2): Pbar within the
  spectrum precision's tolerance (max-normalised), peak indices exact where
  the oracle's peak margin exceeds it.
"""

import numpy as np
import pytest
import torch

import oracle.gsvd_music as O
from gpu_common import context, dev, host, max_rel
from paper_2504_03373_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def _steering_with_lists(ctx, H, ptr, idx):
    st = ctx.steering(dev(H))
    st.set_neighbours(torch.from_numpy(np.asarray(ptr, np.int32)),
                      torch.from_numpy(np.asarray(idx, np.int32)))
    return st


def _random_lists(rng, D):
    sets = [set() for _ in range(D)]
    for _ in range(3 * D):
        a, b = rng.integers(0, D, 2)
        if a != b:
            sets[a].add(int(b))
            sets[b].add(int(a))
    if D > 2:
        sets[0].add(0)  # an entry equal to d is ignored
    ptr = np.zeros(D + 1, np.int32)
    ptr[1:] = np.cumsum([len(x) for x in sets])
    idx = np.array([n for x in sets for n in sorted(x)], np.int32)
    return ptr, idx


@pytest.mark.parametrize("D,Ns", [(1, 1), (2, 2), (37, 4), (500, 8), (2522, 16)])
def test_peaks_nbr_exact(D, Ns):
    ctx = context()
    rng = np.random.default_rng(900 + D)
    ptr, idx = (_random_lists(rng, D) if D != 2522 else
                (synth.fibonacci_sphere(D).nbr_ptr, synth.fibonacci_sphere(D).nbr_idx))
    st = _steering_with_lists(ctx, np.ones((1, D, 2)), ptr, idx)
    nblk = 4
    Pbar = rng.integers(0, 5, (nblk, D)).astype(np.float32)  # many ties
    Pbar[1] = rng.random(D).astype(np.float32)
    Pbar[2] = 3.0  # a plateau over the whole set
    gi, gv = ctx.peaks_nbr(torch.from_numpy(Pbar).cuda(), st, Ns)
    for k in range(nblk):
        io, vo = O.peaks_nbr(Pbar[k].astype(np.float64), ptr, idx, Ns)
        assert list(host(gi)[k]) == list(io), k
        assert np.array_equal(host(gv)[k], vo.astype(np.float32)), k
    st.close()


@pytest.mark.parametrize("n_az,n_el", [(72, 19), (6, 3), (8, 1)])
def test_grid_lists_reproduce_the_grid_search(n_az, n_el):
    ctx = context()
    rng = np.random.default_rng(950 + n_az)
    D = n_az * n_el
    ptr, idx = synth.grid_neighbours(n_az, n_el)
    st = _steering_with_lists(ctx, np.ones((1, D, 2)), ptr, idx)
    Pbar = torch.from_numpy(rng.integers(0, 4, (3, D)).astype(np.float32)).cuda()
    a_i, a_v = ctx.peaks(Pbar, n_az, n_el, 5)
    b_i, b_v = ctx.peaks_nbr(Pbar, st, 5)
    assert torch.equal(a_i, b_i) and torch.equal(a_v, b_v)
    st.close()


def test_bad_neighbour_lists_are_refused():
    ctx = context()
    st = ctx.steering(dev(np.ones((1, 4, 2))))
    for ptr, idx in (([0, 1, 2, 3, 4], [1, 2, 3, 4]),    # index D
                     ([0, 1, 2, 3, 4], [1, 2, 3, -1]),   # negative index
                     ([1, 1, 2, 3, 4], [1, 2, 3, 0]),    # does not start at 0
                     ([0, 2, 1, 3, 4], [1, 2, 3, 0])):   # decreasing
        with pytest.raises(binding.SSLError) as e:
            st.set_neighbours(torch.tensor(ptr, dtype=torch.int32),
                              torch.tensor(idx, dtype=torch.int32))
        assert e.value.status == 1
    # without lists, n_el = 0 and ssl_peaks_nbr are refused
    with pytest.raises(binding.SSLError):
        ctx.peaks_nbr(torch.zeros((1, 4), device="cuda"), st, 1)
    st.close()


TOL = {"tf32x3": 1e-4, "bf16": 1e-2}
_W = {}


def _paper_shape():
    if "w" not in _W:
        w = synth.paper_shape(seed=3, nblk=3)
        K = O.correlation(w.Xnoise).astype(np.complex64)
        nbr = (w.grid.nbr_ptr, w.grid.nbr_idx)
        refs = [O.localize_block(w.X[k], K, w.H.astype(np.complex64), 2, w.D, 0, "sq", nbr=nbr)
                for k in range(w.nblk)]
        _W["w"] = (w, K, refs)
    return _W["w"]


@pytest.mark.parametrize("precision", ["tf32x3", "bf16"])
@pytest.mark.parametrize("method", ["jacobi", "bidiag"])
def test_localize_paper_shape(precision, method):
    ctx = context()
    w, K, refs = _paper_shape()
    st = _steering_with_lists(ctx, w.H, w.grid.nbr_ptr, w.grid.nbr_idx)
    idx, val, Pbar = ctx.localize(dev(w.X), dev(K), st, 2, w.D, 0, form="sq",
                                  precision=precision, abs_tol=2.0 ** -23, method=method)
    assert ctx.device_flags() == 0
    graded = ok = 0
    for k, ref in enumerate(refs):
        assert max_rel(host(Pbar)[k], ref["Pbar"]) < TOL[precision]
        if O.peak_margin_nbr(ref["Pbar"], w.grid.nbr_ptr, w.grid.nbr_idx, 2) > TOL[precision]:
            graded += 1
            ok += list(host(idx)[k]) == list(ref["idx"])
    assert ok == graded
    st.close()


def _relabelled(w, seed):
    """The same direction set with its directions relabelled: steering table
    columns permuted and the neighbour lists rewritten to the new labels."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(w.D)  # new label j is old direction perm[j]
    new_of_old = np.argsort(perm)
    ptr, idx = np.asarray(w.grid.nbr_ptr), np.asarray(w.grid.nbr_idx)
    counts = np.diff(ptr)[perm]
    nptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    nidx = np.concatenate([new_of_old[idx[ptr[o]:ptr[o + 1]]] for o in perm]).astype(np.int32)
    return np.ascontiguousarray(w.H[:, perm]), nptr, nidx


def test_direction_sets_in_sessions_plans_and_streams():
    """Two 60-mic arrays on the paper's 2522-direction sphere (the second with
    its directions relabelled, so that the two arrays of one serving class and
    of one plan carry different neighbour lists): sessions and plans give
    bit-identical results to the stateless call with n_el = 0, and a stream
    whose hop is the whole window agrees with the oracle."""
    ctx = context()
    opts = dict(form="sq", precision="bf16", abs_tol=2.0 ** -23)
    arrays = []
    for i, seed in enumerate((3, 4)):
        w = synth.paper_shape(seed=seed, nblk=2)
        H, ptr, idx = (w.H, w.grid.nbr_ptr, w.grid.nbr_idx) if i == 0 else _relabelled(w, 9)
        K = dev(O.correlation(w.Xnoise).astype(np.complex64))
        st = _steering_with_lists(ctx, H, ptr, idx)
        ref = [ctx.localize(dev(w.X[k:k + 1]), K, st, 2, w.D, 0, **opts) for k in range(2)]
        arrays.append(dict(w=w, K=K, st=st, ref=ref, lists=(ptr, idx), H=H))
    # serving: both sessions in one shape class
    srv = binding.Server(ctx, hbm_budget_bytes=8 << 30, max_batch=8)
    sess = [srv.session(a["K"], a["st"], 2, a["w"].D, 0, a["w"].T, queue_depth=2, **opts)
            for a in arrays]
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
    # a plan over both arrays
    items = []
    for a in arrays:
        Kinv, kst = ctx.noise_inverse(a["K"])
        items.append(dict(X=dev(a["w"].X[0]), Kinv=Kinv, st=a["st"], Ns=2, n_az=a["w"].D,
                          n_el=0))
    plan = binding.Plan(ctx, items, form="sq", precision="bf16", abs_tol=2.0 ** -23)
    plan.run()
    torch.cuda.synchronize()
    for a, out in zip(arrays, plan.outputs):
        idx_ref, val_ref, Pb_ref = a["ref"][0]
        assert int(host(out["status"])[0]) == 0
        assert np.array_equal(host(out["peak_idx"]), host(idx_ref)[0])
        assert np.array_equal(host(out["peak_val"]), host(val_ref)[0])
        assert np.array_equal(host(out["Pbar"]), host(Pb_ref)[0])
    plan.close()
    # a stream: hop = T, so each push holds one whole block
    a = arrays[1]
    w = a["w"]
    s = binding.Stream(ctx, a["K"], a["st"], 2, w.D, 0, w.T, w.T, **opts)
    for k in range(2):
        idx, val, Pbar, _ = s.push(dev(w.X[k]))
        torch.cuda.synchronize()
        ref = O.localize_block(w.X[k], O.correlation(w.Xnoise).astype(np.complex64),
                               a["H"].astype(np.complex64), 2, w.D, 0, "sq", nbr=a["lists"])
        assert max_rel(host(Pbar), ref["Pbar"]) < 1e-2
        if O.peak_margin_nbr(ref["Pbar"], a["lists"][0], a["lists"][1], 2) > 1e-2:
            assert list(host(idx)) == list(ref["idx"])
    s.close()
    assert ctx.device_flags() == 0
    for a in arrays:
        a["st"].close()
