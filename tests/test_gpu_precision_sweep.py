"""Mixed-precision sweep on the 60-mic workload: the spectrum contraction in
FP32 (SIMT), 3xTF32, TF32 and BF16 (tensor cores), the decomposition in FP32
by one-sided Jacobi with FP64 or FP32 angles, by the split iteration (the noise
subspace only) or by the paper's bidiagonalisation route, with the preset noise correlation's condition
number swept over 1e2..1e6 (K = G G^H exactly).  Every setting is graded
against the FP64 oracle on sampled blocks:

* Pbar (SQ form): max-normalised relative error below the spectrum
  precision's tolerance (1e-4 for the FP32-class forms, 1e-3 TF32, 1e-2 BF16);
* the noise-subspace projector (Frobenius) within 1e-4 on every bin whose
  relative signal/noise gap (sigma_3 - sigma_4) / sigma_1 is at least 1e-2,
  and within 2e-6 / gap below that (a subspace's sensitivity to a
  perturbation grows as 1 / gap);
* peak indices, exactly, wherever the oracle's peak margin exceeds the
  spectrum tolerance.
The errors are printed per setting."""

import numpy as np
import pytest

import oracle.gsvd_music as O
from gpu_common import context, dev, host, max_rel, projector

pytestmark = pytest.mark.gpu

# max-normalised Pbar tolerance per spectrum precision
TOL = {"fp32": 1e-4, "tf32x3": 1e-4, "tf32": 1e-3, "bf16": 1e-2}
CONDS = [1e2, 1e3, 1e4, 1e5, 1e6]
ROUTES = {"f64": dict(angles="f64"), "f32": dict(angles="f32"), "bidiag": dict(method="bidiag"),
          "split": dict(angles="f64", method="split", split_ns=3)}
_W, _REF = {}, {}


def _workload(cond):
    from paper_2504_03373_gb300 import synth
    if cond not in _W:
        w = synth.ball60_three_sources(seed=2, nblk=3, cond=cond)
        K = w.K_true.astype(np.complex64)
        refs = [O.localize_block(w.X[k], K, w.H.astype(np.complex64), 3, w.grid.n_az,
                                 w.grid.n_el, "sq") for k in range(w.nblk)]
        _W[cond], _REF[cond] = w, refs
    return _W[cond], _REF[cond]


def projector_bound(lam: np.ndarray, Ns: int) -> np.ndarray:
    gap = (lam[..., Ns - 1] - lam[..., Ns]) / lam[..., 0]
    return np.where(gap >= 1e-2, 1e-4, 2e-6 / np.maximum(gap, 1e-30))


@pytest.mark.parametrize("cond", CONDS)
@pytest.mark.parametrize("precision", ["fp32", "tf32x3", "tf32", "bf16"])
@pytest.mark.parametrize("route", list(ROUTES))
def test_precision_and_conditioning(cond, precision, route):
    ctx = context()
    w, refs = _workload(cond)
    K = w.K_true.astype(np.complex64)
    st = ctx.steering(dev(w.H))
    opts = dict(abs_tol=2.0 ** -23, **ROUTES[route])
    idx, val, Pbar = ctx.localize(dev(w.X), dev(K), st, 3, w.grid.n_az, w.grid.n_el, form="sq",
                                  precision=precision, **opts)
    R = ctx.correlate(dev(w.X))
    sig, E, status = ctx.gsvd(R, dev(K), **opts)
    assert ctx.device_flags() == 0
    assert (host(status) == 0).all()
    errs, pratio, perrs, peaks_ok, graded = [], [], [], 0, 0
    for k in range(w.nblk):
        ref = refs[k]
        errs.append(max_rel(host(Pbar)[k], ref["Pbar"]))
        perr = np.linalg.norm(projector(host(E)[k], 3) - projector(ref["E"], 3), axis=(-2, -1))
        perrs.append(float(perr.max()))
        pratio.append(float((perr / projector_bound(ref["lam"], 3)).max()))
        if O.peak_margin(ref["Pbar"], w.grid.n_az, w.grid.n_el, 3) > TOL[precision]:
            graded += 1
            peaks_ok += list(host(idx)[k]) == list(ref["idx"])
    print(f"\ncond {cond:.0e} spectrum {precision} route {route}: "
          f"Pbar err {max(errs):.2e}, projector err {max(perrs):.2e} "
          f"({max(pratio):.2f} of its bound), peaks {peaks_ok}/{graded} graded blocks")
    st.close()
    assert max(errs) < TOL[precision]
    assert max(pratio) <= 1.0, max(perrs)
    assert peaks_ok == graded
