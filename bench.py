"""Benchmark: SVD forward + backward of one 4096 x 4096 FP32 matrix (kappa = 10
geometric spectrum, the square-matrix setting of Section 4.1 / Tables 1-2), FP32-accurate.

One step = psvd_svd_fwd (Algorithm 1) + psvd_svd_bwd (Algorithm 4, eps = 1e-8) of the
loss <G_U, U> + <g_S, sigma> + <G_V, V> with seeded N(0,1) weights.  The headline
`value` is the mixed-precision path (BF16 -> TF32 -> split-TF32 polish, eigenbasis
correction); the plain FP32-accurate path (split-TF32 throughout) is timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs N independent replicas (one process per GPU, launched by torchrun); the
batch shards with no data-path collective ("scaling": "weak").  `--impl reference`
times the FP64 CPU oracle (the paper's method restated plainly) on the host cores.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 4096
KAPPA = 10.0
EPS = 1e-8
METRIC = "SVD fwd+bwd ms at 4096^2, f32-accurate: mixed vs plain path; % tensor-core peak"
# DRAM bytes (read + written) of one sytrd_kernel launch at n = 4096, from an ncu capture of
# the current kernel (dram__bytes.sum.per_second x gpu__time_duration.sum = 148.13 GB/s x
# 39.116 ms); valid while the kernel is unchanged
TRD_DRAM_BYTES = 5794092046
WORKLOAD = (f"SVD fwd+bwd of one {N}x{N} fp32 matrix A = Q1 diag(s) Q2^T, s_i = {KAPPA:g}^((n-i)/(n-1)), "
            f"eps=1e-8, kreg Algorithm 4")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    def __init__(self, index: int = 0):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                     timeout=5).stdout.strip()
                f = [x.strip() for x in out.split(",")]
                if len(f) >= 7:
                    self.samples.append(f)
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def _dist():
    from paper_2609_32505_gb300 import replicas
    return replicas.init("nccl")


def _oracle_step_seconds(n: int) -> float:
    """Wall time of the FP64 oracle's fwd + bwd of one n x n matrix of the headline construction."""
    from oracle import psvd_oracle as O
    import workloads as W
    a, _ = W.kappa_square(0, n, KAPPA)
    gu, gs, gv = W.loss_weights(0, n, n)
    t0 = time.perf_counter()
    u, s, vt, _ = O.svd(a)
    O.svd_bwd(a, u, s, vt, gu, gs, gv.T, eps=EPS, kreg_mode=0)
    return time.perf_counter() - t0


def _oracle_scaling():
    """The oracle timed at 256^2 (the small configuration's own size) and 512^2 (the clustered
    backward configuration's size); its cost grows faster than n^3 (cyclic Jacobi sweeps grow
    with n and leave the caches), so the exponent is measured between the two, not assumed."""
    t256 = min(_oracle_step_seconds(256) for _ in range(2))
    t512 = _oracle_step_seconds(512)
    p = math.log(t512 / t256) / math.log(2.0)
    return t256, t512, p


def _cpu_line(t256, t512, p):
    ms = t512 * (N / 512) ** p * 1e3
    return ms, {"value": ms, "unit": "ms", "cores": os.cpu_count() or 1, "kind": "oracle",
                "sample": f"FP64 oracle fwd+bwd measured at 256^2 ({t256:.2f} s, the small configuration) and "
                          f"512^2 ({t512:.2f} s), extrapolated to one 4096^2 step by (4096/512)^p with the "
                          f"measured exponent p = {p:.2f} (Jacobi EVD single-threaded, numpy products on the "
                          f"host's BLAS threads)",
                "measured_ms": {"256x256": t256 * 1e3, "512x512": t512 * 1e3}}


def reference_arm(args):
    """The FP64 oracle timed on the host cores on a bounded sample of the workload."""
    rank, ws = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    t256, t512, p = _oracle_scaling()
    for _ in range(max(0, min(args.warmup, 1))):
        _oracle_step_seconds(256)
    ts = [_oracle_step_seconds(256) for _ in range(max(1, args.steps))]
    sec = float(np.median(ts))
    ms = sec * (N / 256) ** p * 1e3
    _, cpu = _cpu_line(t256, t512, p)
    cpu["value"] = ms
    cpu["sample"] = (f"per step one 256^2 fwd+bwd (median {sec:.2f} s of {len(ts)}), extrapolated to 4096^2 by "
                     f"(4096/256)^p, p = {p:.2f} measured between 256^2 and 512^2 ({t512:.2f} s) in this run")
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "reference": "FP64 oracle (the method restated plainly) on the host cores, measured at "
                                    "256^2 and 512^2 and extrapolated with the measured growth exponent"},
            "cpu_baseline": cpu,
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_leg():
    t256, t512, p = _oracle_scaling()
    return _cpu_line(t256, t512, p)[1]


def l2_rmw_gbs(dev) -> float:
    """Read-modify-write bandwidth of a 48 MB buffer that stays in L2 (torch's elementwise
    kernel, CUDA events, best of 5 runs of 20 passes): the ceiling of a pass that streams an
    L2-resident matrix, as the tridiagonalization's row pass does."""
    import torch
    x = torch.ones(12 * 1024 * 1024, device=dev)
    best = float("inf")
    for _ in range(6):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(20):
            x.mul_(1.0000001)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return 2.0 * x.numel() * 4 * 20 / (best * 1e-3) / 1e9


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
        return

    import torch
    import paper_2609_32505_gb300 as P
    import workloads as W

    env_ws = int(os.environ.get("WORLD_SIZE", "1"))
    if args.gpus != env_ws:
        # N GPUs are N processes under torchrun; a plain `python bench.py --gpus N` would run
        # one replica on one GPU and report it as N
        sys.exit(f"bench.py --gpus {args.gpus}: launch one process per GPU, e.g. python -m torch.distributed.run "
                 f"--nproc-per-node {args.gpus} bench.py --gpus {args.gpus} (WORLD_SIZE is {env_ws})")
    rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    P.build()
    L = P.lib()

    s0 = W.kappa_spectrum(N, KAPPA)
    A = W.torch_constructed(1000 + rank, N, N, s0, device=dev)
    rng = W.rng_for(2000 + rank)
    GU = torch.from_numpy(rng.standard_normal((N, N)).astype(np.float32)).to(dev)
    GS = torch.from_numpy(rng.standard_normal(N).astype(np.float32)).to(dev)
    GVT = torch.from_numpy(rng.standard_normal((N, N)).astype(np.float32)).T.contiguous().to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 512 MB > L2

    # learned lower bound: network trained by paper_2609_32505_gb300.train_schedule, probes
    # drawn once; the features, the network and the bound run inside the timed step
    from paper_2609_32505_gb300 import train_schedule
    mlp_params, mlp_margin, nprobe = train_schedule.load(device=dev)
    Zp = P.rademacher_probes(1, N, nprobe, seed=5, device=dev)
    Fp = torch.empty(1, 8, device=dev)
    wsk = P._workspace(L.psvd_sketch_workspace_bytes(1, N, N, nprobe), dev)

    def make(precision, learned=False, schedule=None):
        lb = torch.full((1,), 0.5, device=dev)
        sched = schedule if schedule is not None else (P.SCHED_LEARNED if learned else P.SCHED_CANS)
        o = P.make_opts(precision=precision, schedule=sched, lower_bound=lb if learned else None)
        U = torch.empty(1, N, N, device=dev)
        S = torch.empty(1, N, device=dev)
        VT = torch.empty(1, N, N, device=dev)
        dA = torch.empty(1, N, N, device=dev)
        info = torch.zeros(1, P.INFO_WORDS, dtype=torch.int32, device=dev)
        wsf = P._workspace(L.psvd_svd_workspace_bytes(1, N, N, ctypes.byref(o)), dev)
        wsb = P._workspace(L.psvd_svd_bwd_workspace_bytes(1, N, N), dev)
        return o, U, S, VT, dA, info, wsf, wsb, (lb if learned else None)

    def step(bufs, a_dev):
        o, U, S, VT, dA, info, wsf, wsb, lb = bufs
        st = P._stream()
        if lb is not None:
            P._check(L.psvd_sketch_features(P._ptr(a_dev), P._ptr(Zp), nprobe, P._ptr(Fp), 1, N, N, P._ptr(wsk),
                                            wsk.numel(), st), "sketch")
            P._check(L.psvd_mlp_lower_bound(P._ptr(mlp_params), P._ptr(Fp), P._ptr(lb), 1, float(mlp_margin), st),
                     "lower_bound")
        P._check(L.psvd_svd_fwd(P._ptr(a_dev), P._ptr(U), P._ptr(S), P._ptr(VT), 1, N, N, ctypes.byref(o),
                                P._ptr(wsf), wsf.numel(), P._ptr(info), st), "svd_fwd")
        P._check(L.psvd_svd_bwd(P._ptr(a_dev), P._ptr(U), P._ptr(S), P._ptr(VT), P._ptr(GU), P._ptr(GS),
                                P._ptr(GVT), P._ptr(dA), 1, N, N, EPS, 0, P._ptr(wsb), wsb.numel(), st), "svd_bwd")

    def timed_one(bufs):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step(bufs, A)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    mixed = make(P.PREC_MIXED, learned=True)
    plain = make(P.PREC_FP32)
    for _ in range(max(3, args.warmup)):
        step(mixed, A)
        step(plain, A)
    torch.cuda.synchronize()

    # the two paths alternate step by step, and which one goes first alternates too, so
    # that both see the same clocks and box state
    t_mixed, t_plain = [], []
    launches = launches_plain = 0
    with ClockSampler(local) as clk:
        for it in range(args.steps):
            for arm in ((0, 1) if it % 2 == 0 else (1, 0)):
                c0 = P.kernel_launches()
                if arm == 0:
                    t_mixed.append(timed_one(mixed))
                    launches += P.kernel_launches() - c0   # over the K timed headline steps
                else:
                    t_plain.append(timed_one(plain))
                    launches_plain += P.kernel_launches() - c0
    ms_mixed, ms_plain = float(np.mean(t_mixed)), float(np.mean(t_plain))
    if ws > 1:
        from paper_2609_32505_gb300 import replicas
        ms_mixed, ms_plain = replicas.max_over_ranks([ms_mixed, ms_plain], device=dev)

    # accuracy of this very run (factors of the timed input against its known spectrum)
    info_m = P.info_dict(mixed[5])[0]

    def accuracy(bufs, a_in=None, spec=None):
        _, U, S, VT, *_ = bufs
        a_in = A if a_in is None else a_in
        spec = s0 if spec is None else spec
        u, sg, vt, a = U[0].double(), S[0].double(), VT[0].double(), a_in[0].double()
        eye = torch.eye(N, dtype=torch.float64, device=dev)
        return {"sigma_err_rel_smax": float((sg.cpu() - torch.from_numpy(spec)).abs().max() / spec[0]),
                "recon": float(torch.linalg.matrix_norm(a - (u * sg) @ vt) / torch.linalg.matrix_norm(a)),
                "ortho_u": float(torch.linalg.matrix_norm(u.T @ u - eye) / N ** 0.5),
                "ortho_v": float(torch.linalg.matrix_norm(vt @ vt.T - eye) / N ** 0.5)}

    acc_m, acc_p = accuracy(mixed), accuracy(plain)
    sched_m = {"steps": [info_m["steps_bf16"], info_m["steps_tf32"], info_m["steps_3xtf32"]],
               "lower_bound": float(mixed[8][0]), "sched_fallback": info_m["sched_fallback"]}

    # the BF16-first ladder (PSVD_PREC_MIXED_BF16), reported beside the headline
    bf16 = make(P.PREC_MIXED_BF16, learned=True)
    for _ in range(2):
        step(bf16, A)
    t_bf16 = [timed_one(bf16) for _ in range(3)]
    info_b = P.info_dict(bf16[5])[0]
    bf16_report = {"median_ms": float(np.median(t_bf16)), "accuracy": accuracy(bf16),
                   "corr_max": info_b["corr_max"], "prec_fallback": info_b["prec_fallback"],
                   "polar_steps": [info_b["steps_bf16"], info_b["steps_tf32"], info_b["steps_3xtf32"]]}
    del bf16
    sig_err = acc_m["sigma_err_rel_smax"]

    # roofline: CUDA events around each launch of the tridiagonalization (the dominant
    # kernel) and of the tcgen05 product kernel, on their stream, in one extra step of each path
    peaks, peak_src = _peaks()
    NCLS = 5                                   # PSVD_PROF_CLASSES
    L.psvd_profile_enable(1)
    step(mixed, A)
    torch.cuda.synchronize()
    prof_m = (ctypes.c_double * (4 * NCLS))()
    L.psvd_profile_read(prof_m)
    step(plain, A)
    torch.cuda.synchronize()
    prof_p = (ctypes.c_double * (4 * NCLS))()
    L.psvd_profile_read(prof_p)
    L.psvd_profile_enable(0)

    def cls(arr, c):
        return {"launches": int(arr[4 * c]), "ms": arr[4 * c + 1], "work": arr[4 * c + 2], "max_ms": arr[4 * c + 3]}

    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    bf16_burst = float(peaks.get("bf16_tflops", 1900.0))
    bf16_peak = float(peaks.get("bf16_tflops_sustained", bf16_burst))
    tf32_peak = bf16_peak * (1.1 / 2.25)
    l2_gbs = l2_rmw_gbs(dev)
    trd = cls(prof_m, 4)
    trd_gbs = trd["work"] / (trd["ms"] * 1e-3) / 1e9 if trd["ms"] > 0 else 0.0
    trd_flops = 4.0 / 3.0 * N ** 3                     # Householder tridiagonalization, symmetric
    # polar GEMM chain (per-matrix precision launches of the mixed path) against the
    # precision-weighted peak of the steps it ran, burst and sustained
    mix = cls(prof_m, 3)
    st = [info_m["steps_bf16"], info_m["steps_tf32"], info_m["steps_3xtf32"]]

    def weighted(bf16):
        pk = [bf16, bf16 * 1.1 / 2.25, bf16 * 1.1 / 2.25 / 3.0]
        return sum(st) / sum(k / p for k, p in zip(st, pk)) if sum(st) else bf16

    # Algorithmic flops of the chain from the steps the matrix actually took: K steps of a
    # Gram (n(n+1)m, one triangle) and an apply (2mn^2), plus the final Gram that found the
    # residual below tol.  The time is that of every per-matrix-precision launch, including
    # the launches of the step budget that found nothing left to do.
    k_steps = sum(st)
    chain_flops = (k_steps + 1) * N * (N + 1) * N + k_steps * 2.0 * N * N * N
    chain_tf = chain_flops / (mix["ms"] * 1e-3) / 1e12 if mix["ms"] > 0 else 0.0
    roofline = {"bound": "l2", "achieved": trd_gbs, "peak": l2_gbs, "unit": "GB/s", "frac": trd_gbs / l2_gbs,
                "traffic": TRD_DRAM_BYTES if N == 4096 else None,
                "kernel": "sytrd_kernel (Householder tridiagonalization of H, eigensolver stage 1; one launch)",
                "algorithmic_bytes": trd["work"], "ms": trd["ms"], "share_of_step": trd["ms"] / ms_mixed,
                "peak_src": "measured in this run: read-modify-write of a 48 MB L2-resident buffer",
                "note": (f"every step reads and writes the trailing matrix, 8 sum (n-k-2)^2 bytes, served from "
                         f"L2 (DRAM sees the traffic above); against the measured HBM copy ({hbm_peak:.0f} GB/s) "
                         f"that is {trd_gbs / hbm_peak:.2f}; in flops (4/3 n^3) "
                         f"{trd_flops / (trd['ms'] * 1e-3) / 1e12 if trd['ms'] > 0 else 0:.2f} TFLOP/s; the "
                         f"kernel waits on one grid barrier per reflector"),
                "polar_chain": {"bound": "tensor", "achieved": chain_tf, "unit": "TFLOP/s",
                                "peak_sustained": weighted(bf16_peak), "frac_sustained": chain_tf / weighted(bf16_peak),
                                "peak_burst": weighted(bf16_burst), "frac_burst": chain_tf / weighted(bf16_burst),
                                "steps": st, "launches": mix["launches"], "ms": mix["ms"],
                                "peak_src": f"{peak_src} bf16 {bf16_burst:.0f} burst / {bf16_peak:.0f} sustained, "
                                            f"TF32 x1.1/2.25, split-TF32 /3, weighted by the steps taken"}}
    x3 = cls(prof_p, 2)
    plain_tf = x3["work"] / (x3["ms"] * 1e-3) / 1e12 if x3["ms"] > 0 else 0.0
    tensor = {"split_tf32_all_plain": {"achieved": plain_tf, "peak": tf32_peak / 3.0, "unit": "TFLOP/s",
                                       "frac": plain_tf / (tf32_peak / 3.0), "launches": x3["launches"],
                                       "ms": x3["ms"]},
              "product_kernel_ms_share_mixed": sum(cls(prof_m, c)["ms"] for c in range(4)) / ms_mixed}

    # end to end through the C ABI with host buffers: H2D of A, D2H of dA and sigma
    A_host = A.cpu().pin_memory()
    dA_host = torch.empty(N, N).pin_memory()
    S_host = torch.empty(N).pin_memory()
    a_dev = torch.empty_like(A)
    e2e = []
    for _ in range(max(2, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        a_dev.copy_(A_host, non_blocking=True)
        step(mixed, a_dev)
        dA_host.copy_(mixed[4][0], non_blocking=True)
        S_host.copy_(mixed[2][0], non_blocking=True)
        torch.cuda.synchronize()
        e2e.append((time.perf_counter() - t0) * 1e3)
    e2e_ms = float(np.median(e2e))

    # reported beside the headline, outside its timed region: the same construction at the
    # other condition numbers of the study (both paths) and the classical Newton-Schulz
    # schedule on the headline matrix
    def timed_on(bufs, a_in):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        step(bufs, a_in)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def path_report(bufs, a_in, spec):
        step(bufs, a_in)
        ts = [timed_on(bufs, a_in) for _ in range(2)]
        inf = P.info_dict(bufs[5])[0]
        return {"median_ms": float(np.median(ts)), "accuracy": accuracy(bufs, a_in, spec),
                "polar_steps": [inf["steps_bf16"], inf["steps_tf32"], inf["steps_3xtf32"]],
                "status": inf["status"], "sched_fallback": inf["sched_fallback"],
                "prec_fallback": inf["prec_fallback"], "qr_fallback": inf["qr_fallback"]}

    def extra_reports():
        gen = torch.Generator()
        gen.manual_seed(1000 + rank)                       # the headline matrix's factors
        q1 = W.torch_orthonormal(gen, N, N).to(dev)
        q2 = W.torch_orthonormal(gen, N, N).to(dev)
        sweep = []
        for kappa in (1e2, 1e3, 1e4, 1e6):
            spec = W.kappa_spectrum(N, kappa)
            a_k = ((q1 * torch.from_numpy(spec).to(dev)[None, :]) @ q2.T).float()[None].contiguous()
            sweep.append({"kappa": kappa, "mixed": path_report(mixed, a_k, spec),
                          "plain": path_report(plain, a_k, spec)})
            del a_k
        del q1, q2
        ns = make(P.PREC_FP32, schedule=P.SCHED_NS)
        ns_rep = path_report(ns, A, s0)
        del ns
        return {"kappa_sweep": sweep, "classical_ns_plain": ns_rep}

    def rect_report():
        # the rectangular configuration: 8 x (4096 x 1024), iid N(0, 1/1024), forward only;
        # mixed and plain, on M directly and through the QR preprocessing (Section 4.1)
        a = np.stack([W.marchenko_pastur(100 + i, 4096, 1024) for i in range(8)]).astype(np.float32)
        Ar = torch.from_numpy(a).to(dev)
        out = {}
        for name, prec, preqr in (("plain", P.PREC_FP32, 0), ("mixed", P.PREC_MIXED, 0),
                                  ("plain_preqr", P.PREC_FP32, 1), ("mixed_preqr", P.PREC_MIXED, 1)):
            o = P.make_opts(precision=prec, preqr=preqr)
            U, S, VT, info = P.svd_fwd(Ar, o, return_info=True)
            ts = []
            for _ in range(3):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                P.svd_fwd(Ar, o)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            rec = max(float(torch.linalg.matrix_norm(Ar[b].double() - (U[b].double() * S[b].double()) @ VT[b].double())
                            / torch.linalg.matrix_norm(Ar[b].double())) for b in range(8))
            out[name] = {"median_ms": float(np.median(ts)), "max_recon": rec,
                         "prec_fallback": sum(i["prec_fallback"] for i in info),
                         "status": sorted({i["status"] for i in info})}
            del U, S, VT
        return {"workload": "8 x (4096 x 1024) iid N(0, 1/1024), svd_fwd", **out}

    def small_report():
        # the small configuration: one 256 x 256 matrix (singular values log-uniform in
        # [1e-3, 1]), plain FP32 path with the classical Newton-Schulz polar iteration, full
        # U, S, V^T; latency of svd_fwd and of svd_fwd + svd_bwd in microseconds (launch-bound
        # at this size), and the errors against the matrix's own factors
        a, s = W.small_square(1, 256)
        As = torch.from_numpy(a.astype(np.float32))[None].to(dev).contiguous()
        out = {}
        for name, sched in (("newton_schulz", P.SCHED_NS), ("cans", P.SCHED_CANS)):
            o = P.make_opts(precision=P.PREC_FP32, schedule=sched)
            U, S, VT, info = P.svd_fwd(As, o, return_info=True)
            gU, gS, gV = torch.ones_like(U), torch.ones_like(S), torch.ones_like(VT)
            ts_f, ts_fb = [], []
            for _ in range(25):
                for ts, bwd in ((ts_f, False), (ts_fb, True)):
                    torch.cuda.synchronize()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    u, sv, vt = P.svd_fwd(As, o)
                    if bwd:
                        P.svd_bwd(As, u, sv, vt, gU, gS, gV, eps=EPS)
                    e1.record()
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1) * 1e3)
            ad = As[0].double()
            rec = float(torch.linalg.matrix_norm(ad - (U[0].double() * S[0].double()) @ VT[0].double())
                        / torch.linalg.matrix_norm(ad))
            serr = float(np.max(np.abs(S[0].double().cpu().numpy() - np.sort(s)[::-1])) / np.max(s))
            out[name] = {"fwd_us": float(np.median(ts_f[5:])), "fwd_bwd_us": float(np.median(ts_fb[5:])),
                         "polar_steps": info[0]["iters"], "recon": rec, "sigma_err_rel_smax": serr}
        return {"workload": "one 256 x 256 fp32 matrix, sigma log-uniform in [1e-3, 1], plain path", **out}

    reports = {}
    try:
        reports["small_256"] = small_report()
    except Exception as exc:
        reports["small_256_error"] = f"{type(exc).__name__}: {exc}"
    for key, fn in (("sweep", extra_reports), ("rectangular_preqr", rect_report)):
        try:
            r = fn()
            reports.update(r) if key == "sweep" else reports.__setitem__(key, r)
        except Exception as exc:          # a report must not cost the headline line
            reports[key + "_error"] = f"{type(exc).__name__}: {exc}"
    try:
        from paper_2609_32505_gb300 import schedules
        sc = schedules.run(n=1024, kappa=1e6, batch=4, reps=2)
        for v in sc["schedules"].values():
            v.pop("residual_curve", None)
        reports["schedule_comparison"] = sc
    except Exception as exc:
        reports["schedule_comparison_error"] = f"{type(exc).__name__}: {exc}"
    # the learned schedule at the size of its study: 2048 held-out 1024^2 matrices of the three
    # training families, conservative vs learned (steps, device time, final residual); ~1 min,
    # most of it generating the inputs
    if rank == 0:
        try:
            from paper_2609_32505_gb300 import train_schedule
            reports["learned_eval"] = train_schedule.evaluate(2048, quiet=True)
        except Exception as exc:
            reports["learned_eval_error"] = f"{type(exc).__name__}: {exc}"

    if rank == 0:
        line = {"metric": METRIC, "value": ms_mixed, "unit": "ms", "n_gpus": ws, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms_mixed, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD,
                           "path": "mixed: learned lower bound (sketch + MLP kernels) -> greedy cubics, TF32 steps "
                                   "-> split-TF32 polish, eigenbasis correction; plain: conservative CANS "
                                   "(delta=0.99), split-TF32 throughout",
                           "schedule_mixed": sched_m,
                           "bf16_ladder": bf16_report,
                           "plain_ms": ms_plain, "speedup_mixed_vs_plain": ms_plain / ms_mixed,
                           "median_ms": {"mixed": float(np.median(t_mixed)), "plain": float(np.median(t_plain))},
                           "step_ms": {"mixed": [round(t, 2) for t in t_mixed], "plain": [round(t, 2) for t in t_plain]},
                           "accuracy_plain": acc_p,
                           "l2": "512 MB buffer written between timed steps",
                           "launches_per_step": {"mixed": launches // max(1, args.steps),
                                                 "plain": launches_plain // max(1, args.steps)},
                           "accuracy_mixed": {**acc_m, "polar_ortho_resid": info_m["ortho_resid"],
                                              "corr_max": info_m["corr_max"],
                                              "prec_fallback": info_m["prec_fallback"],
                                              "polar_steps": [info_m["steps_bf16"], info_m["steps_tf32"],
                                                              info_m["steps_3xtf32"]]}},
                "roofline": roofline,
                "tensor": tensor,
                "measured_l2_rmw_gbs": l2_gbs,
                "clocks": clk.summary(),
                "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": N * N * 4,
                        "d2h_bytes_per_step": N * N * 4 + N * 4},
                "gpu_launches": int(launches),
                "reports": reports}
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline_leg()
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
