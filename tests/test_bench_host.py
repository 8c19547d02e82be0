"""Host-side logic of bench.py on the CPU: the clock record that decides
whether a timed run stands, the guard that drops a DRAM-traffic figure once
the kernel's source has changed, the whole-job throughput and the
algorithmic flop counts the roofline divides by."""

import json
import os
import sys
import tempfile

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _sampler_with(lines):
    cs = bench.ClockSampler(0)
    fd, cs.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    cs.proc = object()  # stands for a sampler that ran
    return cs


def test_clock_summary_median_max_and_reasons():
    na, act = "Not Active", "Active"
    lines = [f"0, {sm}, 2070, 900.5, 0x0, {na}, {na}, {na}, {pc}"
             for sm, pc in ((2070, na), (2055, act), (1995, na))]
    lines.insert(1, "garbage line")
    s = _sampler_with(lines).summary()
    assert s["sm_mhz"] == 2055 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_slowdowns():
    na, act = "Not Active", "Active"
    s = _sampler_with([f"0, 1500, 2070, 1300, 0x8, {act}, {na}, {act}, {na}"]).summary()
    assert s["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    assert _sampler_with([]).summary()["reasons"] == ["no samples"]
    cs = bench.ClockSampler(0)
    assert cs.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_measured_traffic_guards():
    rec = json.load(open(os.path.join(ROOT, "profiles", "roofline_traffic.json")))
    assert set(rec) >= {"gsvd_jacobi_kernel", "gsvd_bidiag_kernel"}
    for k, v in rec.items():
        assert v["passes"] == 1 and "--clock-control none" in v["command"]
        assert int(v["dram_bytes_read"]) > 0 and int(v["dram_bytes_write"]) > 0
    # unknown kernel, or a source other than the one the figure was taken on
    assert bench.measured_traffic("no_such_kernel", "bench.py") is None
    assert bench.measured_traffic("gsvd_jacobi_kernel",
                                  "paper_2504_03373_gb300/csrc/correlate.cu") is None
    got = bench.measured_traffic("gsvd_jacobi_kernel",
                                 "paper_2504_03373_gb300/csrc/gsvd_jacobi.cu")
    j = rec["gsvd_jacobi_kernel"]
    assert got in (None, int(j["dram_bytes_read"]) + int(j["dram_bytes_write"]))


def test_measured_traffic_of_the_split_route():
    """The split route's record sums its three launches and is keyed to the
    four sources they are built from, hashed in order."""
    rec = json.load(open(os.path.join(ROOT, "profiles", "roofline_traffic.json")))
    key = "whiten_kernel + gsvd_split_kernel + gsvd_bidiag_kernel"
    c = "paper_2504_03373_gb300/csrc/"
    srcs = [c + "whiten.cu", c + "gsvd_split.cu", c + "jacobi_rot.cuh", c + "gsvd_bidiag.cu"]
    v = rec[key]
    assert v["passes"] == 1 and "-c 3" in v["command"]
    got = bench.measured_traffic(key, srcs)
    assert got in (None, int(v["dram_bytes_read"]) + int(v["dram_bytes_write"]))
    assert bench.measured_traffic(key, srcs[::-1]) is None  # another order: another hash
    assert bench.measured_traffic(key, srcs[:2]) is None


def test_job_throughput():
    assert bench.job_throughput(100, 20, 1, 500.0) == 4000.0
    assert bench.job_throughput(100, 20, 4, 500.0) == 16000.0  # weak scaling: all ranks' blocks


def test_flop_counts_per_unit():
    M = 60
    zero = np.zeros((2, 3, 2))
    # no pair tested, no rotation: the whitening product alone, per bin
    assert bench.gsvd_flops(M, zero) == 6 * 8.0 * M ** 3
    one_rot = zero.copy()
    one_rot[0, 0, 1] = 1
    assert bench.gsvd_flops(M, one_rot) - bench.gsvd_flops(M, zero) == 40.0 * M
    sweep = zero.copy()
    sweep[0, 0, 0] = M * (M - 1) / 2  # one sweep's pair tests: dots plus one set of norms
    assert np.isclose(bench.gsvd_flops(M, sweep) - bench.gsvd_flops(M, zero),
                      8.0 * M * M * (M - 1) / 2 + 4.0 * M * M)
    # split route: a round tests Ns pairs (a dot and two norms each: 16 M),
    # an applied rotation updates two columns (20 M)
    Ns = 3
    assert bench.split_flops(M, Ns, one_rot) - bench.split_flops(M, Ns, zero) == 20.0 * M
    rnd = zero.copy()
    rnd[1, 2, 0] = 1
    assert bench.split_flops(M, Ns, rnd) - bench.split_flops(M, Ns, zero) == Ns * 16.0 * M
    fixed = bench.split_flops(M, Ns, zero) / 6
    assert fixed > 8.0 * M ** 3  # the whitening product plus the preconditioner and finalisation
    assert fixed < 8.0 * M ** 3 + 30.0 * M * M * Ns * 4  # O(M^2 Ns) beyond the product
    per_bin = 8.0 * M ** 3 + 32.0 * M ** 3 / 3 + 16.0 * M ** 3 / 3
    assert np.isclose(bench.bidiag_flops(M, zero), 6 * per_bin)
    assert np.isclose(bench.bidiag_flops(M, one_rot) - bench.bidiag_flops(M, zero), 12.0 * M)


def test_serving_pool_recipe_on_cpu():
    """The serving bench's per-session blocks: shapes, dtype, and noise of
    covariance K plus plane waves of the session's own geometry (the
    projection of X's sample covariance on a source's steering vector
    exceeds the noise-only value)."""
    import torch
    import bench
    from paper_2504_03373_gb300 import synth
    rng = np.random.default_rng(0)
    B, M, T = 3, 8, 400
    G = synth.noise_mixing(rng, B, M, 10.0)
    K = torch.from_numpy(np.matmul(G, np.conj(np.swapaxes(G, 1, 2))).astype(np.complex64))
    pos = synth.ball(M, 0.2, rng)
    freqs = synth.bin_frequencies(16, 18)
    pool = bench.serving_pool(K, pos, freqs, T, 2, np.random.default_rng(1), "cpu")
    assert len(pool) == 2 and pool[0].shape == (T, B, M) and pool[0].dtype == torch.complex64
    X = pool[0].numpy().astype(np.complex128)
    R = np.einsum("tbi,tbj->bij", X, np.conj(X)) / T
    assert np.all(np.real(np.einsum("bii->b", R)) > 0.9 * np.real(np.einsum("bii->b", K.numpy())))


def test_serving_pool_sources_drift_in_azimuth():
    """Consecutive blocks of a session's pool carry the sources rotated by
    DRIFT_DEG_PER_BLOCK about the z axis (10 degrees/s at 0.5 s per block):
    with one strong source, each block's principal eigenvector is the steering
    vector of the drifted direction, not of the initial one."""
    import torch
    import bench
    from paper_2504_03373_gb300 import synth
    assert bench.DRIFT_DEG_PER_BLOCK == 5.0
    seed = next(s for s in range(100) if np.random.default_rng(s).integers(1, 4) == 1)
    r = np.random.default_rng(seed)
    r.integers(1, 4)
    d = r.standard_normal((1, 3))
    d /= np.linalg.norm(d)
    sense = r.choice([-1.0, 1.0], 1)[0]
    B, M, T = 1, 12, 3000
    K = torch.from_numpy((1e-4 * np.eye(M, dtype=np.complex64))[None].copy())
    pos = synth.ball(M, 0.4, np.random.default_rng(7))
    freqs = np.array([2500.0])
    pool = bench.serving_pool(K, pos, freqs, T, 2, np.random.default_rng(seed), "cpu")

    def steer(deg):
        a = np.deg2rad(deg) * sense
        dk = np.array([np.cos(a) * d[0, 0] - np.sin(a) * d[0, 1],
                       np.sin(a) * d[0, 0] + np.cos(a) * d[0, 1], d[0, 2]])
        h = np.exp(2j * np.pi * freqs[0] * (pos @ dk) / synth.SPEED_OF_SOUND)
        return h / np.linalg.norm(h)

    for k in range(2):
        X = pool[k].numpy()[:, 0, :].astype(np.complex128)
        R = X.T @ np.conj(X) / T
        u = np.linalg.eigh(R)[1][:, -1]
        here = abs(np.vdot(u, steer(5.0 * k)))
        other = abs(np.vdot(u, steer(5.0 * (1 - k))))
        assert here > 0.999 and here > other, (k, here, other)
