"""Mixed-precision sweep on the 60-mic workload: the spectrum contraction in
FP32 (SIMT), TF32 and BF16 (tensor cores), the decomposition in FP32 with FP64
or FP32 Jacobi angles, with the preset noise correlation's condition number
swept over 1e2..1e6 (K = G G^H exactly).  Every setting is graded against the
FP64 oracle on sampled blocks: the max-normalised error of Pbar (SQ form),
the noise-subspace projector, and the peak indices where the oracle's margin
allows.  The errors are printed per setting."""

import numpy as np
import pytest

import oracle.gsvd_music as O
from gpu_common import context, dev, host, max_rel, projector

pytestmark = pytest.mark.gpu

# max-normalised Pbar tolerance per spectrum precision
TOL = {"fp32": 1e-4, "tf32": 1e-3, "bf16": 1e-2}
CONDS = [1e2, 1e3, 1e4, 1e5, 1e6]
_W = {}


def _workload(cond):
    from paper_2504_03373_gb300 import synth
    if cond not in _W:
        _W[cond] = synth.ball60_three_sources(seed=2, nblk=3, cond=cond)
    return _W[cond]


@pytest.mark.parametrize("cond", CONDS)
@pytest.mark.parametrize("precision", ["fp32", "tf32", "bf16"])
@pytest.mark.parametrize("angles", ["f64", "f32"])
def test_precision_and_conditioning(cond, precision, angles):
    ctx = context()
    w = _workload(cond)
    K = w.K_true.astype(np.complex64)
    st = ctx.steering(dev(w.H))
    idx, val, Pbar = ctx.localize(dev(w.X), dev(K), st, 3, w.grid.n_az, w.grid.n_el, form="sq",
                                  precision=precision, angles=angles, abs_tol=2.0 ** -23)
    R = ctx.correlate(dev(w.X))
    sig, E, status = ctx.gsvd(R, dev(K), angles=angles, abs_tol=2.0 ** -23)
    assert ctx.device_flags() == 0
    errs, perrs, peaks_ok, graded = [], [], 0, 0
    for k in range(w.nblk):
        ref = O.localize_block(w.X[k], K, w.H.astype(np.complex64), 3, w.grid.n_az,
                               w.grid.n_el, "sq")
        errs.append(max_rel(host(Pbar)[k], ref["Pbar"]))
        perrs.append(float(np.max(np.linalg.norm(projector(host(E)[k], 3) -
                                                 projector(ref["E"], 3), axis=(-2, -1)))))
        if O.peak_margin(ref["Pbar"], w.grid.n_az, w.grid.n_el, 3) > TOL[precision]:
            graded += 1
            peaks_ok += list(host(idx)[k]) == list(ref["idx"])
    print(f"\ncond {cond:.0e} spectrum {precision} angles {angles}: "
          f"Pbar err {max(errs):.2e}, projector err {max(perrs):.2e}, "
          f"peaks {peaks_ok}/{graded} graded blocks")
    st.close()
    assert max(errs) < TOL[precision]
    assert peaks_ok == graded
