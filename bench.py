"""Benchmark of the GSVD-MUSIC hot path on GB300.

Workload (one "step"): the 60-microphone array of the paper's scale — 60 mics
uniform in a 0.4 m ball, 209 bins (k = 16..224 of a 512-point STFT at
16 kHz), T = 50 frames per block, D = 72 x 19 = 1368 directions, Ns = 3
sources at SNR U[-5, 10] dB, K from 240 noise frames — processed as 100
consecutive blocks per step: correlation -> K^{-1} -> whitening + Jacobi SVD
-> E_n -> spectrum -> bin sum -> peaks, all in the library's kernels.
Synthetic, seeded inputs (the paper's recordings and measured transfer
functions are not available).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle (the only reference implementation there is) on a bounded sample of
the same workload.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "60-ch GSVD-MUSIC blocks/sec and p99 block latency; batched-mixed vs plain"
UNIT = "blocks/s"
NBLK = 100
NS, N_AZ, N_EL = 3, 72, 19
FP32_SIMT_LANES_PER_SM = 128
N_SM = 152


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="sq", choices=["abs", "sq"],
                    help="eq. 5 denominator: sq (basis-invariant; the form the parity tests "
                         "grade on this rank-deficient workload) or abs (as printed)")
    ap.add_argument("--precision", default="bf16", choices=["fp32", "tf32", "bf16", "tf32x3"])
    ap.add_argument("--angles", default="f64", choices=["f64", "f32"])
    ap.add_argument("--svd", default="split", choices=["split", "jacobi", "bidiag"],
                    help="decomposition of the whitened matrix: the split one-sided Jacobi "
                         "(the noise subspace the SQ spectrum needs: pairs with the Ns signal "
                         "columns only), the full one-sided Jacobi SVD, or the paper's "
                         "Householder bidiagonalisation + implicit QR")
    ap.add_argument("--abs-tol", type=float, default=2.0 ** -23,
                    help="absolute Jacobi tolerance relative to the largest squared column "
                         "norm (0 = relative test only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-blocks", type=int, default=20)
    ap.add_argument("--cpu-sample-blocks", type=int, default=12)
    ap.add_argument("--serving-sessions", type=int, default=1024,
                    help="sessions of the serving run (0 = skip it)")
    ap.add_argument("--serving-seconds", type=float, default=6.0)
    ap.add_argument("--serving-full-sessions", type=int, default=4096,
                    help="sessions of the full-size serving run (0 = skip it)")
    ap.add_argument("--batch-arrays", type=int, default=512,
                    help="arrays of the mixed-batch run (0 = skip it)")
    ap.add_argument("--streams", type=int, default=32,
                    help="concurrent streams of the per-frame run (0 = skip it)")
    ap.add_argument("--paper-shape", type=int, default=1,
                    help="1: also time the paper-shape configuration (73 bins, 2522 directions)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the extra timings of the FP32-angle, TF32, FP32-SIMT and "
                         "bidiagonal-QR SVD forms")
    ap.add_argument("--blocks", type=int, default=NBLK,
                    help="blocks per step (the measured workload is 100; smaller values are "
                         "for profiler captures)")
    args = ap.parse_args()
    if args.svd == "split" and args.form == "abs":
        ap.error("--svd split computes the noise subspace, which serves the SQ form; the ABS "
                 "form needs the individual noise vectors (--svd jacobi or bidiag)")
    return args


def workload_config(args, extra=None):
    nb = getattr(args, "blocks", NBLK)
    cfg = {
        "workload": "ball60 M=60 (0.4 m ball), 209 bins, T=50, D=1368 (72 az x 19 el), "
                    "Ns=3, SNR U[-5,10] dB, K from 240 noise frames, cond 1e3; "
                    f"{nb} blocks per step",
        "M": 60, "bins": 209, "T": 50, "D": N_AZ * N_EL, "Ns": NS, "blocks_per_step": nb,
        "form": args.form, "headline_form": args.form, "spectrum_precision": args.precision,
        "svd": getattr(args, "svd", "jacobi"),
        "jacobi": {"angles": getattr(args, "angles", "f64"),
                   "abs_tol": getattr(args, "abs_tol", 0.0), "rel_tol": "M*2^-24"},
        "l2": "inputs larger than L2 (X = 502 MB per step)",
    }
    if extra:
        cfg.update(extra)
    return cfg


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seed(rank: int) -> int:
    """Each replica (one per GPU) localises its own array's blocks: weak
    scaling with no data exchange between ranks."""
    return 2 + rank


def max_over_ranks(ms: float, device=None) -> float:
    """Slowest rank's timed-region length (the whole job ends with it)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(blocks_per_step: int, steps: int, world: int, max_ms: float) -> float:
    """Whole-job blocks/s: every rank's blocks over the slowest rank's time."""
    return blocks_per_step * steps * world / (max_ms / 1e3)


# ---------------------------------------------------------------------------
# CPU side: the oracle timed on the host cores
# ---------------------------------------------------------------------------

def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def time_oracle(w, K, nblocks: int, form: str = "sq"):
    import oracle.gsvd_music as O
    t0 = time.perf_counter()
    for k in range(nblocks):
        O.localize_block(w.X[k], K, w.H, NS, N_AZ, N_EL, form)
    return time.perf_counter() - t0


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2504_03373_gb300 import synth
    import oracle.gsvd_music as O
    nb = max(1, min(args.cpu_sample_blocks // 3, NBLK))
    w = synth.ball60_three_sources(seed=2, nblk=nb)
    K = O.correlation(w.Xnoise)
    for _ in range(args.warmup):
        time_oracle(w, K, 1, args.form)
    times = [time_oracle(w, K, nb, args.form) for _ in range(args.steps)]
    tot = sum(times)
    value = nb * args.steps / tot
    out = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * tot / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, {"reference_sample_blocks_per_step": nb}),
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": cpu_cores(),
                         "kind": "oracle",
                         "sample": f"{nb} blocks of the workload per step, FP64 NumPy oracle"},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# GPU side
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during a timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.dev)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks() -> dict:
    """The measured roofline denominators of this GPU model (HBM copy GB/s, cuBLAS
    bf16 TFLOP/s), from MEASURED_PEAKS.json at the repository root."""
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def measured_traffic(kernel: str, source):
    """DRAM bytes per launch of `kernel` (its launches) from the committed ncu
    capture, or None when the kernel's source files (one path or a list, hashed
    in order) have changed since the capture."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "roofline_traffic.json")))[kernel]
        h = hashlib.sha256()
        for src in ([source] if isinstance(source, str) else source):
            h.update(open(os.path.join(ROOT, src), "rb").read())
        cur = h.hexdigest()
    except (OSError, KeyError, ValueError):
        return None
    if rec.get("source_sha256") != cur:
        return None
    return int(rec["dram_bytes_read"]) + int(rec["dram_bytes_write"])


def gsvd_flops(M: int, stats: np.ndarray) -> float:
    """Algorithmic FP32 flops of one gsvd launch, per bin: the whitening
    product (8 M^3), the inner product g_p^H g_q of every pair tested (8 M),
    the squared column norms once per sweep-equivalent of tests (4 M^2), and
    the update of two columns of G and of V for every applied rotation (4 M
    complex outputs of 10 flops: 40 M).  Counts M real rows and columns, not
    the padded ones.  stats: [..., 2] = (pairs tested, rotations) per bin."""
    visits = stats[..., 0].astype(np.float64)
    rots = stats[..., 1].astype(np.float64)
    sweeps = visits / (M * (M - 1) / 2.0)
    return float(np.sum(8.0 * M ** 3 + visits * 8.0 * M + sweeps * 4.0 * M * M +
                        rots * 40.0 * M))


def split_flops(M: int, Ns: int, stats: np.ndarray) -> float:
    """Algorithmic FP32 flops of the split route (whitening launch, split
    launch), per bin, counting a complex multiply-add as 8 flops:
    the whitening product (8 M^3); the preconditioner: one power step and the
    transform A - (A V T) V^H (3 products of M x M by M x Ns: 24 M^2 Ns), then
    twice the pivots' Gram and rotation (16 M Ns^2) and the Cayley step (the
    pivot-partner inner products, A_n Z^H, G, the rank-Ns update: 24 M Ns nR +
    8 M Ns^2, nR = M - Ns); the batched test of every pair (per pair an inner
    product 8 M; per column a squared norm 4 M); per round, for each of the Ns
    pivot pairs, the inner product (8 M) and the two squared norms (4 M each);
    for every applied rotation two columns (2 M complex outputs of 10 flops:
    20 M); the Householder basis of the complement (16 M Ns^2) and the noise
    basis E_n = I - W V^H (8 M nR Ns).  stats: [..., 2] = (rounds, rotations)."""
    rounds = stats[..., 0].astype(np.float64)
    rots = stats[..., 1].astype(np.float64)
    nR = M - Ns
    fixed = (8.0 * M ** 3 + 24.0 * M * M * Ns
             + 2 * (16.0 * M * Ns * Ns + 24.0 * M * Ns * nR + 8.0 * M * Ns * Ns)
             + 8.0 * M * Ns * nR + 4.0 * M * M
             + 16.0 * M * Ns * Ns + 8.0 * M * nR * Ns)
    return float(np.sum(fixed + rounds * Ns * 16.0 * M + rots * 20.0 * M))


def bidiag_flops(M: int, stats: np.ndarray) -> float:
    """Algorithmic FP32 flops of one launch of the bidiagonalisation route, per
    bin: the whitening product (8 M^3), the two-sided Householder reduction
    (a dot and an update of 8 flops per trailing element and reflector:
    32 M^3 / 3), the backward accumulation of Q (16 M^3 / 3) and, for every
    left rotation of the QR iterations, two complex columns of Q times a real
    rotation (12 M).  stats: [..., 2] = (QR iterations, rotations) per bin."""
    rots = stats[..., 1].astype(np.float64)
    per_bin = 8.0 * M ** 3 + 32.0 * M ** 3 / 3.0 + 16.0 * M ** 3 / 3.0
    return float(per_bin * rots.size + np.sum(rots * 12.0 * M))


def run_ours(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    from __graft_entry__ import build
    build()
    from paper_2504_03373_gb300 import binding, synth

    NB = args.blocks
    w = synth.ball60_three_sources(seed=replica_seed(rank), nblk=NB)
    ctx = binding.Context(dev.index)
    Xd = torch.from_numpy(w.X.astype(np.complex64)).to(dev)
    Xn = torch.from_numpy(w.Xnoise.astype(np.complex64)).to(dev)[None]
    Kd = ctx.correlate(Xn)[0].contiguous()  # K from noise frames (session set-up)
    st = ctx.steering(torch.from_numpy(w.H.astype(np.complex64)).to(dev))
    out = (torch.empty((NB, NS), dtype=torch.int32, device=dev),
           torch.empty((NB, NS), dtype=torch.float32, device=dev),
           torch.empty((NB, N_AZ * N_EL), dtype=torch.float32, device=dev))
    stream = torch.cuda.current_stream()

    jac = dict(angles=args.angles, abs_tol=args.abs_tol, method=args.svd, split_ns=NS)

    def step():
        ctx.localize(Xd, Kd, st, NS, N_AZ, N_EL, form=args.form, precision=args.precision,
                     out=out, **jac)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    flags = ctx.device_flags()

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(dev.index) as clk:
        barrier()
        t0 = time.perf_counter()
        for i in range(args.steps):
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
        barrier()
        wall = time.perf_counter() - t0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dev)
    value = job_throughput(NB, args.steps, ws, total_ms)

    # ---- end to end through the C ABI with host buffers ----
    Xh = torch.from_numpy(w.X.astype(np.complex64)).pin_memory()
    Kh = Kd.cpu().pin_memory()
    outh = (torch.empty((NB, NS), dtype=torch.int32).pin_memory(),
            torch.empty((NB, NS), dtype=torch.float32).pin_memory(),
            torch.empty((NB, N_AZ * N_EL), dtype=torch.float32).pin_memory())

    def step_e2e():
        ctx.localize(Xh, Kh, st, NS, N_AZ, N_EL, form=args.form, precision=args.precision,
                     out=outh, **jac)

    for _ in range(2):
        step_e2e()
    e2e_steps = max(3, args.steps // 2)
    barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(e2e_steps):
        step_e2e()
    b.record(stream)
    barrier()
    e2e_ms = max_over_ranks(a.elapsed_time(b), dev)
    e2e_value = job_throughput(NB, e2e_steps, ws, e2e_ms)
    h2d = Xh.numel() * 8 + Kh.numel() * 8
    d2h = sum(t.numel() * t.element_size() for t in outh)

    # ---- variants of the batched step (a few steps each) ----
    variants = {}
    others = [m for m in ("split", "jacobi", "bidiag") if m != args.svd]
    route_name = {"split": "split_svd", "jacobi": "jacobi_svd", "bidiag": "bidiag_qr_svd"}
    # the ABS form needs the individual noise vectors: the split hands it to the full Jacobi
    abs_method = "jacobi" if args.svd == "split" else args.svd
    if not args.no_variants:
        for name, kw in (("paper_precision", dict(precision="tf32x3", angles=args.angles,
                                                  abs_tol=args.abs_tol, method=args.svd)),
                         ("abs_form", dict(precision=args.precision, angles=args.angles,
                                           abs_tol=args.abs_tol, method=abs_method, form="abs")),
                         ("angles_f32", dict(precision=args.precision, angles="f32",
                                             abs_tol=args.abs_tol, method=args.svd)),
                         ("tf32_spectrum", dict(precision="tf32", angles=args.angles,
                                                abs_tol=args.abs_tol, method=args.svd)),
                         ("fp32_simt_spectrum", dict(precision="fp32", angles=args.angles,
                                                     abs_tol=args.abs_tol, method=args.svd)),
                         ("relative_tol_only", dict(precision=args.precision, angles=args.angles,
                                                    abs_tol=0.0, method=args.svd)),
                         *((route_name[o], dict(precision=args.precision, angles=args.angles,
                                                abs_tol=args.abs_tol, method=o))
                           for o in others)):
            prec = kw.pop("precision")
            vform = kw.pop("form", args.form)
            for _ in range(2):
                ctx.localize(Xd, Kd, st, NS, N_AZ, N_EL, form=vform, precision=prec,
                             out=out, **kw)
            va, vb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            nst = 3
            va.record(stream)
            for _ in range(nst):
                ctx.localize(Xd, Kd, st, NS, N_AZ, N_EL, form=vform, precision=prec,
                             out=out, **kw)
            vb.record(stream)
            vb.synchronize()
            vms = va.elapsed_time(vb) / nst
            variants[name] = {"value": round(NB / (vms / 1e3), 3), "ms_per_step": round(vms, 3)}
            if name == "abs_form" and abs_method != args.svd:
                variants[name]["svd"] = abs_method

    # ---- the FP64 path (accuracy reference on the GPU) over the same blocks ----
    if not args.no_variants:
        o64 = (torch.empty((NB, NS), dtype=torch.int32, device=dev),
               torch.empty((NB, NS), dtype=torch.float64, device=dev),
               torch.empty((NB, N_AZ * N_EL), dtype=torch.float64, device=dev))

        def step64():
            ctx.localize_f64(Xd, Kd, st, NS, N_AZ, N_EL, form=args.form, out=o64,
                             abs_tol=2.0 ** -52)
        step64()
        va, vb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        va.record(stream)
        for _ in range(2):
            step64()
        vb.record(stream)
        vb.synchronize()
        vms = va.elapsed_time(vb) / 2
        variants["fp64_path"] = {"value": round(NB / (vms / 1e3), 3), "ms_per_step": round(vms, 3),
                                 "note": "correlation, K^-1, Jacobi (FP64 data, angles and tests, "
                                         "abs_tol 2^-52) and spectrum all in FP64"}

    # ---- plain form: one block per call, FP32 spectrum ----
    plain_ms = []
    pout = (torch.empty((1, NS), dtype=torch.int32, device=dev),
            torch.empty((1, NS), dtype=torch.float32, device=dev),
            torch.empty((1, N_AZ * N_EL), dtype=torch.float32, device=dev))
    for k in range(min(args.plain_blocks + 2, NB)):
        xa = Xd[k:k + 1]
        pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pa.record(stream)
        ctx.localize(xa, Kd, st, NS, N_AZ, N_EL, form=args.form, precision="fp32", out=pout,
                     **jac)
        pb.record(stream)
        pb.synchronize()
        if k >= 2:
            plain_ms.append(pa.elapsed_time(pb))

    # ---- dominant kernel: the whitening + Jacobi SVD launch ----
    R = ctx.correlate(Xd)
    Kinv, _ = ctx.noise_inverse(Kd)
    sig, E, status, stats = ctx.gsvd(R, Kinv, kinv=True, stats=True, **jac)
    torch.cuda.synchronize()
    reps = 3
    ka, kb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ka.record(stream)
    for _ in range(reps):
        ctx.gsvd(R, Kinv, kinv=True, stats=True, **jac)
    kb.record(stream)
    torch.cuda.synchronize()
    gsvd_ms = ka.elapsed_time(kb) / reps
    st_np = stats.cpu().numpy()
    def route_flops(method, stt):
        if method == "bidiag":
            return bidiag_flops(60, stt)
        if method == "split":
            return split_flops(60, NS, stt)
        return gsvd_flops(60, stt)

    flops = route_flops(args.svd, st_np)

    def route(ms, st, stt, method):
        r = {"launch_ms": round(ms, 4), "max_status": int(st.max())}
        if method == "split":
            r.update(mean_sweeps=round(float(stt[..., 0].mean()) / (60 - NS), 3),
                     mean_rotations=round(float(stt[..., 1].mean()), 1),
                     settled_by_batched_test=round(float((stt[..., 0] == 0).mean()), 4),
                     note="sweeps of 57 rounds of the 3 pivot-partner pairs after the batched "
                          "test; launch_ms covers the whitening launch (with the "
                          "preconditioner), the split launch and the retry launch (the "
                          "bidiagonalisation route on the matrices handed back)")
        elif method == "bidiag":
            r.update(mean_qr_iterations=round(float(stt[..., 0].mean()), 2),
                     mean_rotations=round(float(stt[..., 1].mean()), 1))
        else:
            r.update(mean_sweeps=round(float(stt[..., 0].mean()) / (60 * 59 / 2), 3),
                     mean_rotations=round(float(stt[..., 1].mean()), 1))
        return r

    # ---- each stage of the step alone (CUDA events on the launching stream) ----
    def stage_ms(fn, n=3):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / n

    T_, B_, M_ = Xd.shape[1], Xd.shape[2], Xd.shape[3]
    peaks_json = measured_peaks()
    hbm = peaks_json.get("hbm_gbs")
    tc_peak = peaks_json.get("bf16_tflops")
    if tc_peak and args.precision in ("tf32", "tf32x3"):
        tc_peak = tc_peak / 2  # nominal TF32 : BF16 dense ratio
    t_corr = stage_ms(lambda: ctx.correlate(Xd, R))
    t_inv = stage_ms(lambda: ctx.noise_inverse(Kd))
    Pb = torch.empty((NB, N_AZ * N_EL), dtype=torch.float32, device=dev)
    t_spec = stage_ms(lambda: ctx.music_spectrum(E, NS, st, form=args.form,
                                                 precision=args.precision, want_P=False))
    t_peaks = stage_ms(lambda: ctx.peaks(Pb, N_AZ, N_EL, NS))
    t_spec_gen = None
    if args.precision in ("bf16", "tf32"):
        # the same spectrum with analytic steering: tiles generated in the kernel
        st_an = binding.Steering.analytic(ctx, w.pos, w.grid.unit_vectors(), w.freqs)
        t_spec_gen = stage_ms(lambda: ctx.music_spectrum(E, NS, st_an, form=args.form,
                                                         precision=args.precision, want_P=False))
        st_an.close()
    corr_bytes = NB * T_ * B_ * M_ * 8 + NB * B_ * M_ * M_ * 8
    corr_flops = 8.0 * T_ * M_ * (M_ + 1) / 2 * NB * B_
    fp32_peak = N_SM * FP32_SIMT_LANES_PER_SM * 2 * 2070e6 / 1e12  # TFLOP/s, FMA at max clock
    spec_flops = 2.0 * NB * B_ * (N_AZ * N_EL) * (2 * (M_ - NS)) * (2 * M_)
    stages = {
        "correlate": {"ms": round(t_corr, 4), "bytes": corr_bytes,
                      "achieved_gbs": round(corr_bytes / t_corr / 1e6, 1),
                      "frac_of_hbm": (round(corr_bytes / t_corr / 1e6 / hbm, 4) if hbm else None),
                      "flops": corr_flops,
                      "achieved_tflops": round(corr_flops / t_corr / 1e9, 2),
                      "frac_of_fp32_peak": round(corr_flops / t_corr / 1e9 / fp32_peak, 4),
                      "binding_roof": "fp32" if hbm and corr_flops / corr_bytes > fp32_peak * 1e3 / hbm
                                      else "hbm",
                      "note": "X read + R written once, of measured HBM copy rate; flops "
                              "8 T M(M+1)/2 per bin (the Hermitian half), of derived FP32 peak "
                              "(152 SMs x 128 lanes x 2 x 2070 MHz)"},
        "noise_inverse": {"ms": round(t_inv, 4),
                          "note": "FP64 Cholesky and inverse of K (209 bins), in every call of "
                                  "the stateless step"},
        "gsvd": {"ms": round(gsvd_ms, 4),
                 "kernel": {"bidiag": "gsvd_bidiag_kernel",
                            "split": "whiten_kernel + gsvd_split_kernel + gsvd_bidiag_kernel"}.get(
                     args.svd, "gsvd_jacobi_kernel")},
        "spectrum": {"ms": round(t_spec, 4), "flops": spec_flops,
                     "achieved_tflops": round(spec_flops / t_spec / 1e9, 1),
                     "frac_of_tensor_peak": (round(spec_flops / t_spec / 1e9 / tc_peak, 4)
                                             if tc_peak else None),
                     "note": f"pack of E_n, {args.precision} tensor-core GEMM (real-embedded "
                             "2N x 2M per direction, useful flops) with the eq. 5 epilogue, bin "
                             "sum; of measured cuBLAS bf16 burst rate"
                             + (" / 2" if args.precision in ("tf32", "tf32x3") else "")
                             + (" (3xTF32 issues three MMAs per useful product)"
                                if args.precision == "tf32x3" else "")},
        "peaks": {"ms": round(t_peaks, 4)},
        "spectrum_generated_steering": (
            {"ms": round(t_spec_gen, 4),
             "achieved_tflops": round(spec_flops / t_spec_gen / 1e9, 1),
             "note": "the spectrum stage with analytic steering: the kernel's generator warps "
                     "write each steering tile (sine/cosine of the phase) instead of a TMA load"}
            if t_spec_gen else None),
    }

    # the other decomposition routes on the same launch
    svd_routes = None
    if not args.no_variants:
        svd_routes = {args.svd: route(gsvd_ms, status, st_np, args.svd)}
        for other in others:
            ojac = dict(jac, method=other)
            _, _, ostatus, ostats = ctx.gsvd(R, Kinv, kinv=True, stats=True, **ojac)
            torch.cuda.synchronize()
            ba, bb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ba.record(stream)
            for _ in range(reps):
                ctx.gsvd(R, Kinv, kinv=True, **ojac)
            bb.record(stream)
            torch.cuda.synchronize()
            oms = ba.elapsed_time(bb) / reps
            ost = ostats.cpu().numpy()
            svd_routes[other] = route(oms, ostatus, ost, other)
            svd_routes[other]["tflops"] = round(route_flops(other, ost) / (oms / 1e3) / 1e12, 3)
        svd_routes["note"] = "one launch over all blocks x bins of the step, same R and K^-1"
    clock = clk.summary()
    peak_tflops = N_SM * FP32_SIMT_LANES_PER_SM * 2 * 2070e6 / 1e12  # FP32 FMA at max clock
    achieved = flops / (gsvd_ms / 1e3) / 1e12

    if rank != 0:
        return
    kernel = {"bidiag": "gsvd_bidiag_kernel",
              "split": "whiten_kernel + gsvd_split_kernel + gsvd_bidiag_kernel"}.get(
        args.svd, "gsvd_jacobi_kernel")
    csrc = "paper_2504_03373_gb300/csrc/"
    kernel_src = ([csrc + "whiten.cu", csrc + "gsvd_split.cu", csrc + "jacobi_rot.cuh",
                   csrc + "gsvd_bidiag.cu"]
                  if args.svd == "split" else
                  csrc + "gsvd_bidiag.cu" if args.svd == "bidiag" else
                  [csrc + "gsvd_jacobi.cu", csrc + "jacobi_rot.cuh"])
    svd_desc = {"split": f"split one-sided Jacobi with {args.angles} angles (noise subspace)",
                "jacobi": f"one-sided Jacobi with {args.angles} angles",
                "bidiag": "bidiagonalisation + implicit QR"}[args.svd]
    plain_ms = plain_ms or [float("nan")]
    res = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": (f"mixed: {args.precision} spectrum, f32 correlation and SVD, "
                  + (f"{args.angles} Jacobi angles, " if args.svd != "bidiag" else "")
                  + "f64 Cholesky of K"),
        "data": "synthetic (seeded STFT-domain frames, free-field steering)",
        "config": workload_config(args, {"parallelism": f"replicas x{ws}",
                                         "form_note": f"{args.precision} spectrum, FP32 "
                                                      f"decomposition by {svd_desc}, FP64 "
                                                      "Cholesky of K"}),
        "latency_ms": {"p50": round(statistics.median(step_ms), 4),
                       "p99": round(float(np.percentile(step_ms, 99)), 4),
                       "note": "batched form: every block of a step completes with the step"},
        "plain": {"value": round(1e3 / statistics.mean(plain_ms), 3), "unit": UNIT,
                  "p50_ms": round(statistics.median(plain_ms), 4),
                  "p99_ms": round(float(np.percentile(plain_ms, 99)), 4),
                  "form": "one block per call, FP32 spectrum"},
        "paper_precision": (dict(variants["paper_precision"], unit=UNIT,
                                 form=f"the same step with the FP32-class 3xTF32 spectrum "
                                      f"(the paper computes in FP32), {args.form} form")
                            if "paper_precision" in variants else None),
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        # noise inverse, correlation, [whitening,] decomposition, [retry,] spectrum, bin sum, peaks
        "gpu_launches": (8 if args.svd == "split" else 6) * args.steps,
        "roofline": {"kernel": kernel, "bound": "alu",
                     "achieved": round(achieved, 3), "peak": round(peak_tflops, 2),
                     "unit": "TFLOP/s", "frac": round(achieved / peak_tflops, 4),
                     "traffic": (measured_traffic(kernel, kernel_src)
                                 if NB == NBLK and (args.angles == "f64" or args.svd == "bidiag")
                                 else None),
                     "traffic_unit": "bytes per launch (ncu dram read + write)",
                     "peak_note": "of derived peak: FP32 FMA, 152 SMs x 128 lanes x 2 flop x "
                                  "2070 MHz (measured FFMA microbenchmark: 74.1 TFLOP/s)",
                     **route(gsvd_ms, status, st_np, args.svd)},
        "variants": variants,
        "svd_routes": svd_routes,
        "stages": stages,
        "clocks": clock,
        "device_flags": flags,
        "wall_s_timed_region": round(wall, 3),
    }
    if args.serving_sessions > 0 and ws == 1:
        res["serving"] = run_serving(ctx, args, dev, args.serving_sessions, args.serving_seconds)
    if args.serving_full_sessions > 0 and ws == 1:
        res["serving_full"] = run_serving(ctx, args, dev, args.serving_full_sessions,
                                          args.serving_seconds)
    if args.serving_full_sessions > 0 and ws == 1 and not args.no_variants:
        # the same full-size serving run with the other decomposition routes
        for other in others:
            oargs = argparse.Namespace(**dict(vars(args), svd=other))
            res[f"serving_full_{other}"] = run_serving(ctx, oargs, dev,
                                                       args.serving_full_sessions,
                                                       args.serving_seconds)
    if args.batch_arrays > 0 and ws == 1:
        res["batching"] = run_batching(ctx, args, dev, args.batch_arrays)
    if args.streams > 0 and ws == 1:
        res["streaming"] = run_streaming(ctx, args, dev, args.streams)
    if not args.no_variants and ws == 1:
        res["plain_uca8"] = run_uca8(ctx, args, dev)
    if args.paper_shape and ws == 1:
        res["paper_shape"] = run_paper_shape(ctx, args, dev)
    if not args.no_cpu_baseline and ws == 1:
        import oracle.gsvd_music as O
        Kc = Kd.cpu().numpy().astype(np.complex128)
        nb = min(args.cpu_sample_blocks, NB)
        t = time_oracle(w, Kc, nb, args.form)
        res["cpu_baseline"] = {"value": round(nb / t, 4), "unit": UNIT, "cores": cpu_cores(),
                               "kind": "oracle",
                               "sample": f"first {nb} of the {NB} blocks, FP64 NumPy oracle, "
                                         f"{args.form.upper()} form"}
    print(json.dumps(res), flush=True)
    st.close()
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()


def batching_arrays(ctx, n: int, dev, seed: int = 4):
    """The mixed-batch workload: n arrays, M drawn from {8, 16, 32, 60, 64},
    Ns from 1..3, each with its own random geometry (uniform in a 0.4 m
    ball), noise field and sources (directions uniform on the sphere, SNR
    U[-5, 10] dB); 209 bins, T = 50, D = 72 x 19.  Frames, noise and the
    free-field steering tables are generated on the device (seeded) and the
    tables handed to the library; K^{-1} comes from the library's FP64
    Cholesky of the sample noise correlation.  One block per array."""
    import torch
    from paper_2504_03373_gb300 import synth
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    grid = synth.sphere_grid()
    u = torch.from_numpy(grid.unit_vectors()).to(dev)                     # [D][3]
    kf = torch.from_numpy(2.0 * np.pi * synth.bin_frequencies() / 343.0).to(dev)  # [B]
    T, B = 50, kf.numel()

    def cn(*shape):
        re = torch.randn(*shape, generator=gen, device=dev, dtype=torch.float32)
        im = torch.randn(*shape, generator=gen, device=dev, dtype=torch.float32)
        return torch.complex(re, im) * (0.5 ** 0.5)

    arrays = []
    for i in range(n):
        M = int(rng.choice([8, 16, 32, 60, 64]))
        Ns = int(rng.integers(1, 4))
        pos = []
        while len(pos) < M:
            q = rng.uniform(-0.4, 0.4, 3)
            if q @ q <= 0.16:
                pos.append(q)
        pos = torch.from_numpy(np.array(pos)).to(dev)                    # [M][3]
        ph = kf[:, None, None] * (u @ pos.T)[None]                       # [B][D][M]
        H = torch.polar(torch.ones_like(ph), ph).to(torch.complex64).contiguous()
        st = ctx.steering(H)
        del H, ph
        G = cn(B, M, M) / M ** 0.5                                       # noise mixing
        nk = max(50, 4 * M)
        Nk = G @ cn(B, M, nk)
        K = (Nk @ Nk.conj().transpose(1, 2) / nk).contiguous()
        Kinv, kst = ctx.noise_inverse(K)
        N = G @ cn(B, M, T)                                              # [B][M][T]
        p_noise = float(N.abs().square().mean())
        az = rng.uniform(0.0, 2 * np.pi, Ns)
        el = np.arcsin(rng.uniform(-1.0, 1.0, Ns))
        us = torch.from_numpy(np.stack([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az),
                                        np.sin(el)], 1)).to(dev)           # [Ns][3]
        phs = kf[:, None, None] * (us @ pos.T)[None]                     # [B][Ns][M]
        hs = torch.polar(torch.ones_like(phs), phs).to(torch.complex64)
        amp = torch.from_numpy((10.0 ** (rng.uniform(-5, 10, Ns) / 20.0)) * p_noise ** 0.5)
        S = cn(B, Ns, T) * amp.to(dev, torch.float32)[None, :, None]
        X = (hs.transpose(1, 2) @ S + N).permute(2, 0, 1).contiguous()   # [T][B][M]
        arrays.append(dict(X=X, Kinv=Kinv, K=K, st=st, Ns=Ns, n_az=grid.n_az, n_el=grid.n_el,
                           M=M, kst=kst))
    return arrays


def run_batching(ctx, args, dev, n_arrays: int, passes: int = 3):
    """Mixed batch of n_arrays arrays of uneven size: the plan (one launch per
    stage over all (array, bin) pairs, autotuned Jacobi size classes, replayed
    as a CUDA graph) against one launch sequence per array through the
    stateless calls.  Both passes recompute every array's block; time with
    CUDA events on the current stream after one untimed pass each."""
    import torch
    from paper_2504_03373_gb300 import binding
    t0 = time.perf_counter()
    arrays = batching_arrays(ctx, n_arrays, dev)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    # (plans run the full one-sided Jacobi or the paper's route)
    jac = dict(angles=args.angles, abs_tol=args.abs_tol,
               method="jacobi" if args.svd == "split" else args.svd)
    t0 = time.perf_counter()
    plan = binding.Plan(ctx, arrays, form=args.form, precision=args.precision, graph=True,
                        autotune=True, **jac)
    t_plan = time.perf_counter() - t0
    plain = binding.Plan(ctx, arrays, form=args.form, precision=args.precision, graph=False,
                         **jac)

    def per_array():
        out = []
        for a in arrays:
            R = ctx.correlate(a["X"][None])
            _, E, _ = ctx.gsvd(R, a["Kinv"], kinv=True, **jac)
            _, Pbar = ctx.music_spectrum(E, a["Ns"], a["st"], form=args.form,
                                         precision=args.precision, want_P=False)
            out.append(ctx.peaks(Pbar, a["n_az"], a["n_el"], a["Ns"])[0])
        return out

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0 = time.perf_counter()
        e0.record()
        res = None
        for _ in range(passes):
            res = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / passes, (time.perf_counter() - w0) * 1e3 / passes, res

    ms_graph, _, _ = timed(plan.run)
    ms_plain, _, _ = timed(plain.run)
    ms_arr, _, idx_arr = timed(per_array)
    same = sum(int(np.array_equal(o["peak_idx"].cpu().numpy(), r.cpu().numpy()[0]))
               for o, r in zip(plan.outputs, idx_arr))
    status_ok = sum(int(o["status"].item() == 0) for o in plan.outputs)
    info = plan.info()
    ms_of = {m: int(sum(a["M"] == m for a in arrays)) for m in (8, 16, 32, 60, 64)}
    res = {
        "config": f"{n_arrays} arrays, M in {{8,16,32,60,64}} (counts {ms_of}), Ns 1..3, "
                  "own random 0.4 m ball geometry, noise field and sources per array; 209 bins, "
                  "T=50, D=1368 (72 az x 19 el); one block per array per pass",
        "unit": "blocks/s",
        "plan_graph": {"value": round(n_arrays / (ms_graph / 1e3), 1),
                       "ms_per_pass": round(ms_graph, 3), "launches_per_pass": info["launches"]},
        "plan_no_graph": {"value": round(n_arrays / (ms_plain / 1e3), 1),
                          "ms_per_pass": round(ms_plain, 3)},
        "per_array_calls": {"value": round(n_arrays / (ms_arr / 1e3), 1),
                            "ms_per_pass": round(ms_arr, 3),
                            "note": "correlate, gsvd, music_spectrum, peaks per array"},
        "speedup_vs_per_array": round(ms_arr / ms_graph, 2),
        "peaks_identical_to_per_array": f"{same}/{n_arrays}",
        "status_ok": f"{status_ok}/{n_arrays}",
        "jacobi_class_of_m": info["class_of_m"], "gsvd_units": info["gsvd_units"],
        "gsvd_grid": info["gsvd_grid"], "autotune_ms": round(info["autotune_ms"], 1),
        "setup_s": {"inputs": round(t_gen, 2), "plan_with_autotune_and_graph": round(t_plan, 2)},
    }
    plan.close()
    plain.close()
    for a in arrays:
        a["st"].close()
    return res


def run_paper_shape(ctx, args, dev, nblk: int = 100, steps: int = 5):
    """The paper's own shape (Sec. V): 60 mics, 73 bins (k = 16..88), a
    2522-direction set over the sphere (Fibonacci spiral, neighbour-list peak
    search), Ns = 2; the batched step over nblk blocks, and one block per call."""
    import torch
    from paper_2504_03373_gb300 import synth

    w = synth.paper_shape(seed=3, nblk=nblk)
    ctx_X = torch.from_numpy(w.X.astype(np.complex64)).to(dev)
    Kd = ctx.correlate(torch.from_numpy(w.Xnoise.astype(np.complex64)).to(dev)[None])[0]
    Kd = Kd.contiguous()
    st = ctx.steering(torch.from_numpy(w.H.astype(np.complex64)).to(dev))
    st.set_neighbours(torch.from_numpy(w.grid.nbr_ptr), torch.from_numpy(w.grid.nbr_idx))
    jac = dict(angles=args.angles, abs_tol=args.abs_tol, method=args.svd)
    out = (torch.empty((nblk, 2), dtype=torch.int32, device=dev),
           torch.empty((nblk, 2), dtype=torch.float32, device=dev),
           torch.empty((nblk, w.D), dtype=torch.float32, device=dev))
    stream = torch.cuda.current_stream()
    res = {"config": "M=60 (0.4 m ball), 73 bins (k=16..88), D=2522 Fibonacci-sphere "
                     "directions with 6-nearest-neighbour lists, Ns=2, T=50, SNR U[-5,10] dB, "
                     f"K from 240 noise frames; {nblk} blocks per step, {args.form} form",
           "unit": UNIT}
    for prec in (args.precision, "tf32x3"):
        def step():
            ctx.localize(ctx_X, Kd, st, 2, w.D, 0, form=args.form, precision=prec, out=out, **jac)
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            step()
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        res[f"{prec}_spectrum"] = {"value": round(nblk / (ms / 1e3), 1), "ms_per_step": round(ms, 3)}
    lat = []
    o1 = tuple(t[:1] for t in out)
    for k in range(12):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.localize(ctx_X[k:k + 1], Kd, st, 2, w.D, 0, form=args.form, precision="tf32x3",
                     out=o1, **jac)
        b.record(stream)
        b.synchronize()
        if k >= 2:
            lat.append(a.elapsed_time(b))
    res["plain_tf32x3"] = {"value": round(1e3 / statistics.mean(lat), 1),
                           "p50_ms": round(statistics.median(lat), 4),
                           "p99_ms": round(float(np.percentile(lat, 99)), 4),
                           "form": "one block per call"}
    st.close()
    return res


def run_uca8(ctx, args, dev, blocks: int = 40):
    """The plain 8-mic configuration: a uniform circular array (r = 0.1 m), one
    source at 0 dB, 72 azimuths, one block per call with the FP32 spectrum;
    per-call latency for both SVD routes."""
    import torch
    from paper_2504_03373_gb300 import synth

    w = synth.uca8_single_source(seed=5, nblk=blocks)
    X = torch.from_numpy(w.X.astype(np.complex64)).to(dev)
    K = ctx.correlate(torch.from_numpy(w.Xnoise.astype(np.complex64)).to(dev)[None])[0]
    st = ctx.steering(torch.from_numpy(w.H.astype(np.complex64)).to(dev))
    D = w.grid.n_az * w.grid.n_el
    out = (torch.empty((1, 1), dtype=torch.int32, device=dev),
           torch.empty((1, 1), dtype=torch.float32, device=dev),
           torch.empty((1, D), dtype=torch.float32, device=dev))
    stream = torch.cuda.current_stream()
    res = {"config": "8-mic UCA r = 0.1 m, 1 source at 0 dB, K cond 1e3 from 50 noise frames, "
                     "209 bins, T = 50, D = 72 azimuths, Ns = 1; one block per call, FP32 "
                     f"spectrum, {args.form.upper()} form"}
    # (the split route serves the SQ form only)
    for method in ("split", "jacobi", "bidiag") if args.form == "sq" else ("jacobi", "bidiag"):
        lat = []
        for k in range(blocks + 3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.localize(X[k % blocks:k % blocks + 1], K, st, 1, w.grid.n_az, w.grid.n_el,
                         form=args.form, precision="fp32", out=out, angles=args.angles,
                         abs_tol=args.abs_tol, method=method)
            b.record(stream)
            b.synchronize()
            if k >= 3:
                lat.append(a.elapsed_time(b))
        res[method] = {"value": round(1e3 / statistics.mean(lat), 1), "unit": UNIT,
                       "p50_ms": round(statistics.median(lat), 4),
                       "p99_ms": round(float(np.percentile(lat, 99)), 4)}
    st.close()
    return res


def run_streaming(ctx, args, dev, n_streams: int = 32, hop: int = 5, pushes: int = 20):
    """Per-frame processing of 60-mic streams (the benchmark array, K, grid):
    a sliding window of T = 50 frames advanced by `hop` frames per push (50 ms
    of audio at 100 frames/s for hop 5), warm-started Jacobi.  Reports the
    latency of one stream's pushes (CUDA events, one push at a time), the
    rotations per bin warm vs a cold start on the same window, and the
    throughput of n_streams streams pushing concurrently on their own CUDA
    streams (real-time capacity = pushes/s / (100 / hop))."""
    import torch
    from paper_2504_03373_gb300 import binding, synth
    w = synth.ball60_three_sources(seed=2, nblk=4)
    X = torch.from_numpy(np.ascontiguousarray(np.concatenate(list(w.X), 0))).to(dev)
    Xn = torch.from_numpy(w.Xnoise).to(dev)[None]
    K = ctx.correlate(Xn)[0].contiguous()
    st = ctx.steering(torch.from_numpy(w.H.astype(np.complex64)).to(dev))
    # streams continue the full Jacobi from the previous window (warm start)
    jac = dict(angles=args.angles, abs_tol=args.abs_tol,
               method="jacobi" if args.svd == "split" else args.svd)
    nf = X.shape[0]

    def frames(n):
        i = (n * hop) % (nf - hop)
        return X[i:i + hop]

    s = binding.Stream(ctx, K, st, NS, N_AZ, N_EL, 50, hop, form=args.form,
                       precision=args.precision, **jac)
    for n in range(12):
        s.push(frames(n))
    lat, warm_rot = [], []
    for n in range(12, 12 + pushes):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, _, _, stt = s.push(frames(n), stats=True)
        e1.record()
        torch.cuda.synchronize()
        lat.append(e0.elapsed_time(e1))
        warm_rot.append(float(stt[:, 1].float().mean()))
    Kinv, _ = ctx.noise_inverse(K)
    cold_rot = []
    for n in range(12, 12 + 4):
        end = (n + 1) * hop % (nf - hop) + 0
        R = ctx.correlate(X[max(0, end - 50):max(50, end)][None].contiguous())
        _, _, _, cst = ctx.gsvd(R, Kinv, kinv=True, stats=True, **jac)
        cold_rot.append(float(cst[0, :, 1].float().mean()))
    s.close()
    streams = [binding.Stream(ctx, K, st, NS, N_AZ, N_EL, 50, hop, form=args.form,
                              precision=args.precision, **jac) for _ in range(n_streams)]
    cuda_streams = [torch.cuda.Stream() for _ in range(n_streams)]
    for n in range(12):
        for k, (ss, cs) in enumerate(zip(streams, cuda_streams)):
            with torch.cuda.stream(cs):
                ss.push(frames(n + k), want_pbar=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for n in range(12, 12 + pushes):
        for k, (ss, cs) in enumerate(zip(streams, cuda_streams)):
            with torch.cuda.stream(cs):
                ss.push(frames(n + k), want_pbar=False)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    for ss in streams:
        ss.close()
    st.close()
    rate = n_streams * pushes / wall
    return {"config": f"60-mic array (ball60 workload), T = 50 frame window, hop {hop} frames, "
                      f"{args.precision} spectrum, {args.angles} Jacobi angles",
            "single_stream_push_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                                      "p99": round(float(np.percentile(lat, 99)), 3)},
            "rotations_per_bin": {"warm": round(float(np.mean(warm_rot)), 1),
                                  "cold": round(float(np.mean(cold_rot)), 1)},
            "concurrent_streams": n_streams,
            "pushes_per_s": round(rate, 1),
            "realtime_streams_at_100_frames_per_s": round(rate / (100.0 / hop), 1)}


# azimuth drift of the serving sources per 0.5 s block (10 degrees per second)
DRIFT_DEG_PER_BLOCK = 5.0


def serving_pool(K, pos, freqs, T: int, nblk: int, rng, dev):
    """nblk consecutive blocks [T][B][M] (complex64, on dev) of one session:
    1-3 plane-wave sources of the session's own geometry pos [M][3] (initial
    directions uniform on the sphere, each drifting in azimuth by
    DRIFT_DEG_PER_BLOCK per block, in a random sense; SNR U[-5, 10] dB against
    the mean noise power tr(K)/M per bin) over noise n = L w with K = L L^H
    (K: [B][M][M] tensor on dev)."""
    import torch
    from paper_2504_03373_gb300 import synth
    B, M = K.shape[0], K.shape[1]
    ns = int(rng.integers(1, 4))
    d = rng.standard_normal((ns, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    sense = rng.choice([-1.0, 1.0], ns)
    amp = torch.from_numpy(np.sqrt(10.0 ** (rng.uniform(-5, 10, ns) / 10.0))).to(dev)
    fr = torch.from_numpy(np.asarray(freqs, np.float64)).to(dev)
    K64 = K.to(torch.complex128)
    L = torch.linalg.cholesky(K64)
    Wn = torch.randn((B, M, nblk * T), dtype=torch.complex128, device=dev)
    N = torch.matmul(L, Wn).permute(2, 0, 1).reshape(nblk, T, B, M)
    p_n = torch.diagonal(K64, dim1=-2, dim2=-1).real.mean(-1)  # [B]
    S = torch.randn((nblk, T, B, ns), dtype=torch.complex128, device=dev)
    S = S * amp * torch.sqrt(p_n)[None, None, :, None]
    out = []
    for k in range(nblk):
        a = np.deg2rad(DRIFT_DEG_PER_BLOCK * k) * sense  # [ns], about the z axis
        c, s_ = np.cos(a), np.sin(a)
        dk = np.stack([c * d[:, 0] - s_ * d[:, 1], s_ * d[:, 0] + c * d[:, 1], d[:, 2]], 1)
        delay = torch.from_numpy(dk @ np.asarray(pos).T / synth.SPEED_OF_SOUND).to(dev)
        h = torch.exp(2j * np.pi * fr[:, None, None] * delay[None])  # [B][ns][M]
        X = N[k] + torch.einsum("tbs,bsm->tbm", S[k], h)
        out.append(X.to(torch.complex64).contiguous())
    return out


def run_serving(ctx, args, dev, n_sessions: int, seconds: float):
    """Continuous-batching serving run: n_sessions arrays (60 % M=60, 25 % M=32,
    15 % M=16), each sending a 50-frame block every 0.5 s with exponential
    jitter (mean 20 ms), for `seconds` of wall time after a 1 s warm-up.
    With a tensor-core spectrum every session is a distinct array: its own
    random ball geometry, held as analytic steering (the spectrum kernel
    generates the steering tiles from it), and its own two-block pool whose
    sources (1-3, at random directions drifting 10 degrees/s in azimuth, SNR
    U[-5, 10] dB) are synthesised for
    that geometry over one of four noise fields per channel count (K).  With
    the FP32 spectrum, sessions share four stored steering tables per channel
    count instead.  Returns the server's throughput, the latency
    t_done - t_arrival of retired blocks and the device memory held."""
    import torch
    from paper_2504_03373_gb300 import binding, synth
    rng = np.random.default_rng(5)
    mix = [(60, 0.60, 0.4, 3), (32, 0.25, 0.2, 2), (16, 0.15, 0.1, 1)]
    grid = synth.sphere_grid()
    u = grid.unit_vectors()
    analytic = args.precision in ("bf16", "tf32")
    freqs = synth.bin_frequencies()
    T = 50
    noise = {}  # (M, field) -> (K, [noise-only blocks])
    steer_bytes = 0
    for M, frac, radius, Ns in mix:
        for gidx in range(4):
            w = synth.make_workload(M=M, T=T, nblk=2, Ns=Ns, geometry="ball", radius=radius,
                                    grid=grid, snr_db=rng.uniform(-5, 10, Ns), cond=1e3,
                                    n_k=max(50, 4 * M), on_grid=False, seed=100 + M + gidx,
                                    drift_deg_per_blk=5.0)
            Xn = torch.from_numpy(w.Xnoise).to(dev)[None]
            K = ctx.correlate(Xn)[0].contiguous()
            if analytic:
                noise[(M, gidx)] = (K, None, None, Ns)
            else:
                st = ctx.steering(torch.from_numpy(w.H.astype(np.complex64)).to(dev))
                steer_bytes += w.H.size * 8 + w.H.shape[0] * w.H.shape[1] * (128 * 2 + 4)
                pool = [torch.from_numpy(np.ascontiguousarray(w.X[k])).to(dev) for k in range(2)]
                noise[(M, gidx)] = (K, pool, st, Ns)
    srv = binding.Server(ctx, hbm_budget_bytes=160 << 30, max_batch=1024)
    counts = [int(round(f * n_sessions)) for _, f, _, _ in mix]
    counts[0] += n_sessions - sum(counts)
    sessions, keep = [], []
    t_setup = time.perf_counter()
    for (M, _, radius, Ns), cnt in zip(mix, counts):
        for i in range(cnt):
            K, Wn, st, Ns_ = noise[(M, i % 4)]
            if analytic:
                pos = synth.ball(M, radius, rng)
                st = binding.Steering.analytic(ctx, pos, u, freqs)
                steer_bytes += 256 + 4 * (3 * M + 3 * grid.D + freqs.size)
                pool = serving_pool(K, pos, freqs, T, 2, rng, dev)
                keep.append(st)
            else:
                pool = Wn
            se = srv.session(K, st, Ns_, grid.n_az, grid.n_el, T, form=args.form,
                             precision=args.precision, queue_depth=2, angles=args.angles,
                             abs_tol=args.abs_tol, method=args.svd)
            sessions.append((se, pool))
    setup_s = time.perf_counter() - t_setup
    torch.cuda.synchronize()  # every pool block is complete: submits need no ordering
    period = 0.5e9
    t_start = binding.now_ns() + 50_000_000
    nxt = [t_start + rng.uniform(0, period) for _ in sessions]
    outstanding = [[] for _ in sessions]
    sent = [0] * len(sessions)
    submitted = refused = 0
    t_warm = t_start + 1e9
    t_end = t_warm + seconds * 1e9
    measuring = False
    while True:
        now = binding.now_ns()
        if not measuring and now >= t_warm:
            srv.reset_stats()
            submitted = refused = 0
            measuring = True
        if now >= t_end:
            break
        for i, (se, pool) in enumerate(sessions):
            if nxt[i] <= now:
                try:
                    t = se.submit(pool[sent[i] % len(pool)], int(nxt[i]), ordered=False)
                    sent[i] += 1
                    outstanding[i].append(t)
                    submitted += 1
                except binding.SSLError:
                    refused += 1
                nxt[i] += period + rng.exponential(20e6)
        srv.run_step()
        for i, (se, _) in enumerate(sessions):
            if outstanding[i] and se.poll(outstanding[i][0]) is not None:
                outstanding[i].pop(0)
    st = srv.stats()
    wall = (binding.now_ns() - t_warm) * 1e-9
    srv.close()
    for x in keep:
        x.close()
    offered = n_sessions / 0.5
    return {"sessions": n_sessions, "mix": "60% M=60, 25% M=32, 15% M=16",
            "distinct_geometries": n_sessions if analytic else 12,
            "steering": ("analytic, tiles generated in the spectrum kernel" if analytic
                         else "stored tables shared by geometry"),
            "gpu_busy_frac": round(st["busy_ms"] / (wall * 1e3), 3),
            "hbm_sessions_bytes": int(st["hbm_used"]), "hbm_batch_work_bytes": int(st["hbm_work"]),
            "hbm_steering_bytes": int(steer_bytes),
            "setup_s": round(setup_s, 1),
            "offered_blocks_per_s": round(offered, 1),
            "served_blocks_per_s": round(st["blocks_done"] / wall, 1),
            "p50_ms": round(st["latency_p50_ms"], 3), "p99_ms": round(st["latency_p99_ms"], 3),
            "max_ms": round(st["latency_max_ms"], 3), "batches": int(st["batches"]),
            "refused_submits": refused, "pending_at_end": int(st["blocks_pending"]),
            "seconds": round(wall, 2), "budget_s": 0.5,
            "meets_budget": bool(st["latency_p99_ms"] < 500.0 and refused == 0),
            "note": "4 noise fields (K) per channel count; each session's own geometry and "
                    "sources (tensor-core spectra) or 4 shared geometries per channel count "
                    "(FP32); sources drift 10 deg/s in azimuth; the two-block pool repeats; "
                    "latency = retirement time - scheduled "
                    "arrival time; a submit to a full two-slot ring is refused"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
