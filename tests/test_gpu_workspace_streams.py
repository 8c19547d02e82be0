"""One context driven from two streams at once.  The calls that keep
intermediates in the context's workspace (here the spectrum with P kept
inside, and the whole path with host frames, whose staging copy runs on the
context's own auxiliary stream) are ordered after one another by the library,
whatever stream each is issued on; results must equal those of the same calls
issued one at a time on one stream."""

import numpy as np
import pytest
import torch

import oracle.gsvd_music as O
from gpu_common import context, dev, host
from paper_2504_03373_gb300 import synth

pytestmark = pytest.mark.gpu


def test_calls_on_two_streams_share_the_workspace_safely():
    ctx = context()
    w = synth.ball60_three_sources(seed=2, nblk=6)
    K = dev(O.correlation(w.Xnoise).astype(np.complex64))
    st = ctx.steering(dev(w.H))
    R = ctx.correlate(dev(w.X))
    _, E, _ = ctx.gsvd(R, K, abs_tol=2.0 ** -23)
    opts = dict(form="sq", precision="bf16", abs_tol=2.0 ** -23)
    # one call at a time on the current stream
    _, Pb_ref = ctx.music_spectrum(E, 3, st, form="sq", precision="bf16", want_P=False)
    Xh = torch.from_numpy(np.ascontiguousarray(w.X[:3].astype(np.complex64))).pin_memory()
    i_ref, v_ref, Pl_ref = ctx.localize(Xh, K, st, 3, w.grid.n_az, w.grid.n_el, **opts)
    torch.cuda.synchronize()
    ref = (host(Pb_ref).copy(), host(i_ref).copy(), host(v_ref).copy(), host(Pl_ref).copy())
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    for _ in range(3):
        # issued back to back on two streams, without host synchronisation
        _, Pb1 = ctx.music_spectrum(E, 3, st, form="sq", precision="bf16", want_P=False,
                                    stream=s1)
        i2, v2, Pl2 = ctx.localize(Xh, K, st, 3, w.grid.n_az, w.grid.n_el, stream=s2, **opts)
        _, Pb3 = ctx.music_spectrum(E, 3, st, form="sq", precision="bf16", want_P=False,
                                    stream=s1)
        torch.cuda.synchronize()
        assert np.array_equal(host(Pb1), ref[0])
        assert np.array_equal(host(Pb3), ref[0])
        assert np.array_equal(host(i2), ref[1])
        assert np.array_equal(host(v2), ref[2])
        assert np.array_equal(host(Pl2), ref[3])
    assert ctx.device_flags() == 0
    st.close()
