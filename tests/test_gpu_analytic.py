"""Analytic (free-field) steering: the tensor-core spectrum generates each
steering tile from the array geometry inside the kernel instead of reading a
table.  Checked through the C ABI against the FP64 oracle and against the
table path:

* the generated tiles give the same denominators of eq. 5 as the oracle
  within the operand rounding of the precision (TF32 2e-3, BF16 1e-2,
  max-normalised; the same bounds as the table-driven tensor-core test), and
  the same P as the table path to well inside that;
* a path that reads a table (FP32 SIMT) builds it from the geometry (phases
  in FP64) and matches the oracle at the FP32 tolerance (1e-5) when the
  oracle uses the same single-precision geometry;
* the whole localization with analytic steering matches the oracle within
  the spectrum tolerance (BF16 1e-2, TF32 1e-3 on Pbar), peaks exact where
  the oracle's margin allows.
"""

import numpy as np
import pytest
import torch

import oracle.gsvd_music as O
from gpu_common import context, dev, host, max_rel
from paper_2504_03373_gb300 import binding, synth

pytestmark = pytest.mark.gpu

C = 343.0
TC_TOL = {"tf32": 2e-3, "bf16": 1e-2}


def _geometry(M, seed):
    rng = np.random.default_rng(seed)
    pos = synth.ball(M, 0.4, rng) if M > 8 else synth.uca(M, 0.1)
    grid = synth.sphere_grid()
    u = grid.unit_vectors()
    freqs = synth.bin_frequencies(16, 40)
    return pos, u, freqs


def _oracle_table(pos, u, freqs):
    """The steering the library forms from single-precision geometry: phase
    (u . p) (f / c) with the geometry and f / c rounded to float32."""
    p32 = pos.astype(np.float32).astype(np.float64)
    u32 = u.astype(np.float32).astype(np.float64)
    fc = (freqs.astype(np.float32) / np.float32(C)).astype(np.float64)
    ph = 2.0 * np.pi * fc[:, None, None] * (u32 @ p32.T)[None]
    return np.exp(1j * ph)


@pytest.mark.parametrize("precision", ["tf32", "bf16", "fp32"])
@pytest.mark.parametrize("M,Ns", [(8, 1), (33, 4), (60, 3)])
def test_generated_tiles(precision, M, Ns):
    ctx = context()
    pos, u, freqs = _geometry(M, 70 + M)
    B, D = freqs.size, u.shape[0]
    rng = np.random.default_rng(80 + M)
    nblk = 2
    E = np.stack([synth.haar_unitary(rng, B, M) for _ in range(nblk)])
    Ho = _oracle_table(pos, u, freqs)
    st_a = binding.Steering.analytic(ctx, pos, u, freqs, C)
    st_t = ctx.steering(dev(Ho))
    Pa, _ = ctx.music_spectrum(dev(E), Ns, st_a, form="sq", precision=precision)
    Pt, _ = ctx.music_spectrum(dev(E), Ns, st_t, form="sq", precision=precision)
    assert ctx.device_flags() == 0
    hh = float(M)
    for k in range(nblk):
        Po = O.spectrum(Ho, O.noise_subspace(E[k].astype(np.complex64).astype(complex), Ns), "sq")
        if precision == "fp32":
            assert max_rel(host(Pa)[k], Po) < 1e-5
        else:
            assert max_rel(hh / host(Pa)[k], hh / Po) < TC_TOL[precision]
            assert max_rel(host(Pa)[k], host(Pt)[k]) < TC_TOL[precision]
    st_a.close()
    st_t.close()


@pytest.mark.parametrize("precision", ["tf32", "bf16"])
def test_localize_with_analytic_steering(precision):
    ctx = context()
    w = synth.ball60_three_sources(seed=2, nblk=2)
    K = O.correlation(w.Xnoise).astype(np.complex64)
    st = binding.Steering.analytic(ctx, w.pos, w.grid.unit_vectors(), w.freqs, C)
    idx, val, Pbar = ctx.localize(dev(w.X), dev(K), st, 3, w.grid.n_az, w.grid.n_el, form="sq",
                                  precision=precision, abs_tol=2.0 ** -23)
    assert ctx.device_flags() == 0
    tol = {"tf32": 1e-3, "bf16": 1e-2}[precision]
    for k in range(w.nblk):
        ref = O.localize_block(w.X[k], K, w.H.astype(np.complex64), 3, w.grid.n_az,
                               w.grid.n_el, "sq")
        assert max_rel(host(Pbar)[k], ref["Pbar"]) < tol
        if O.peak_margin(ref["Pbar"], w.grid.n_az, w.grid.n_el, 3) > tol:
            assert list(host(idx)[k]) == list(ref["idx"])
    st.close()


def test_analytic_steering_rejects_bad_geometry():
    ctx = context()
    pos, u, freqs = _geometry(8, 1)
    with pytest.raises(binding.SSLError):
        binding.Steering.analytic(ctx, pos, u, freqs, c=0.0)
    bad = pos.copy()
    bad[0, 0] = np.nan
    with pytest.raises(binding.SSLError):
        binding.Steering.analytic(ctx, bad, u, freqs, C)
    bad_dev = torch.from_numpy(bad.astype(np.float32)).cuda()
    with pytest.raises(binding.SSLError):
        binding.Steering.analytic(ctx, bad_dev, u, freqs, C)


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_geometry_from_device_memory_gives_the_same_steering(precision):
    """The geometry may come from device memory: the spectrum is bit-identical
    to the one from the same geometry in host memory."""
    ctx = context()
    pos, u, freqs = _geometry(60, 5)
    B, M = freqs.size, pos.shape[0]
    rng = np.random.default_rng(9)
    E = dev(np.stack([synth.haar_unitary(rng, B, M)]))
    Hh = binding.Steering.analytic(ctx, pos, u, freqs, C)
    Hd = binding.Steering.analytic(ctx, torch.from_numpy(pos.astype(np.float32)).cuda(),
                                   torch.from_numpy(u.astype(np.float32)).cuda(),
                                   torch.from_numpy(freqs.astype(np.float32)).cuda(), C)
    Ph, _ = ctx.music_spectrum(E, 3, Hh, form="sq", precision=precision)
    Pd, _ = ctx.music_spectrum(E, 3, Hd, form="sq", precision=precision)
    assert ctx.device_flags() == 0
    assert np.array_equal(host(Ph), host(Pd))
    Hh.close()
    Hd.close()
