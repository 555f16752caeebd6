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
    import torch.distributed as dist
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1 and not dist.is_initialized():
        dist.init_process_group("nccl")
    return (dist.get_rank() if ws > 1 else 0), ws


def reference_arm(args):
    """The FP64 oracle timed on the host cores on a bounded sample of the workload."""
    rank, ws = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    from oracle import psvd_oracle as O
    import workloads as W
    n = 256
    a, _ = W.kappa_square(0, n, KAPPA)
    gu, gs, gv = W.loss_weights(0, n, n)
    threads = os.cpu_count() or 1

    def step():
        u, s, vt, _ = O.svd(a)
        O.svd_bwd(a, u, s, vt, gu, gs, gv.T, eps=EPS, kreg_mode=0)

    for _ in range(max(0, min(args.warmup, 1))):
        step()
    ts = []
    for _ in range(max(1, args.steps)):
        t0 = time.perf_counter()
        step()
        ts.append(time.perf_counter() - t0)
    sec = float(np.median(ts))
    scale = (N / n) ** 3          # dense O(n^3) work throughout (NS products, Jacobi sweeps, backward)
    ms = sec * scale * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": ms, "unit": "ms", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"SVD fwd+bwd {N}x{N} fp32 input, kappa={KAPPA:g} geometric spectrum, "
                                   f"FP64 oracle timed at {n}x{n} and scaled by (4096/{n})^3"},
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": threads, "kind": "oracle",
                             "sample": f"one {n}x{n} fwd+bwd per step (median of {len(ts)}), x{scale:.0f}"},
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_leg():
    from oracle import psvd_oracle as O
    import workloads as W
    n = 256
    a, _ = W.kappa_square(0, n, KAPPA)
    gu, gs, gv = W.loss_weights(0, n, n)
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        u, s, vt, _ = O.svd(a)
        O.svd_bwd(a, u, s, vt, gu, gs, gv.T, eps=EPS, kreg_mode=0)
        ts.append(time.perf_counter() - t0)
    sec = float(np.median(ts))
    scale = (N / n) ** 3
    return {"value": sec * scale * 1e3, "unit": "ms", "cores": os.cpu_count() or 1, "kind": "oracle",
            "sample": f"FP64 oracle fwd+bwd of one {n}x{n} kappa=10 matrix (median of 3, {sec:.2f} s), "
                      f"scaled by (4096/{n})^3 to one 4096^2 step"}


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

    def make(precision):
        o = P.make_opts(precision=precision)
        U = torch.empty(1, N, N, device=dev)
        S = torch.empty(1, N, device=dev)
        VT = torch.empty(1, N, N, device=dev)
        dA = torch.empty(1, N, N, device=dev)
        info = torch.zeros(1, 9, dtype=torch.int32, device=dev)
        wsf = P._workspace(L.psvd_svd_workspace_bytes(1, N, N, ctypes.byref(o)), dev)
        wsb = P._workspace(L.psvd_svd_bwd_workspace_bytes(1, N, N), dev)
        return o, U, S, VT, dA, info, wsf, wsb

    def step(bufs, a_dev):
        o, U, S, VT, dA, info, wsf, wsb = bufs
        st = P._stream()
        P._check(L.psvd_svd_fwd(P._ptr(a_dev), P._ptr(U), P._ptr(S), P._ptr(VT), 1, N, N, ctypes.byref(o),
                                P._ptr(wsf), wsf.numel(), P._ptr(info), st), "svd_fwd")
        P._check(L.psvd_svd_bwd(P._ptr(a_dev), P._ptr(U), P._ptr(S), P._ptr(VT), P._ptr(GU), P._ptr(GS),
                                P._ptr(GVT), P._ptr(dA), 1, N, N, EPS, 0, P._ptr(wsb), wsb.numel(), st), "svd_bwd")

    def timed(bufs, steps):
        times = []
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            if ws > 1:
                torch.distributed.barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            step(bufs, A)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return times

    mixed = make(P.PREC_MIXED)
    plain = make(P.PREC_FP32)
    for _ in range(max(3, args.warmup)):
        step(mixed, A)
        step(plain, A)
    torch.cuda.synchronize()

    launches0 = P.kernel_launches()
    with ClockSampler(local) as clk:
        t_mixed = timed(mixed, args.steps)
        launches = P.kernel_launches() - launches0     # over the K timed headline steps
        t_plain = timed(plain, args.steps)
    launches_plain = P.kernel_launches() - launches0 - launches
    ms_mixed, ms_plain = float(np.mean(t_mixed)), float(np.mean(t_plain))
    if ws > 1:
        t = torch.tensor([ms_mixed, ms_plain], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_mixed, ms_plain = t.tolist()

    # accuracy of this very run (factors of the timed input against its known spectrum)
    info_m = P.info_dict(mixed[5])[0]
    sig = mixed[2][0].double().cpu().numpy()
    sig_err = float(np.max(np.abs(sig - s0)) / s0[0])

    # roofline of the product kernel: CUDA events around each launch on its stream
    peaks, peak_src = _peaks()
    L.psvd_profile_enable(1)
    step(mixed, A)
    torch.cuda.synchronize()
    prof = (ctypes.c_double * 16)()
    L.psvd_profile_read(prof)
    step(plain, A)
    torch.cuda.synchronize()
    prof_p = (ctypes.c_double * 16)()
    L.psvd_profile_read(prof_p)
    L.psvd_profile_enable(0)
    bf16_peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1700.0)))
    tf32_peak = bf16_peak * (1.1 / 2.25)
    # per class: (launches, ms, flops, max ms); split-TF32 issues 3 TF32 products per flop
    cls_peak = [bf16_peak, tf32_peak, tf32_peak / 3.0, None]
    per = {}
    for c, name in enumerate(["bf16", "tf32", "tf32x3", "mixed"]):
        nl, ms, fl = prof[4 * c], prof[4 * c + 1], prof[4 * c + 2]
        if nl > 0:
            per[name] = {"launches": int(nl), "ms": ms, "tflops": fl / (ms * 1e-3) / 1e12}
    # the per-matrix-precision launches (polar steps) dominate the mixed path
    pm = prof[12:16]
    pp = prof_p[8:12]     # plain path: split-TF32 class
    ach_m = pm[2] / (pm[1] * 1e-3) / 1e12 if pm[1] > 0 else 0.0
    ach_p = pp[2] / (pp[1] * 1e-3) / 1e12 if pp[1] > 0 else 0.0
    roofline = {"bound": "tensor", "achieved": ach_p, "peak": tf32_peak / 3.0, "unit": "TFLOP/s",
                "frac": ach_p / (tf32_peak / 3.0), "traffic": None,
                "kernel": "gemm_tn_kernel (tcgen05 split-TF32, plain path, all launches of one step)",
                "peak_src": f"{peak_src} bf16 sustained {bf16_peak:.0f} x 1.1/2.25 (TF32) / 3 (split-TF32)",
                "mixed_path_kernel_tflops": ach_m, "mixed_path_classes": per,
                "gemm_ms_share_plain": pp[1] / ms_plain if ms_plain else None}

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

    if rank == 0:
        line = {"metric": METRIC, "value": ms_mixed / ws, "unit": "ms", "n_gpus": ws, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms_mixed, "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"SVD fwd+bwd of one {N}x{N} fp32 matrix A = Q1 diag(s) Q2^T, "
                                       f"s_i = {KAPPA:g}^((n-i)/(n-1)), eps=1e-8, kreg Algorithm 4",
                           "path": "mixed: BF16->TF32->split-TF32 polish + eigenbasis correction, CANS delta=0.99",
                           "plain_ms": ms_plain, "speedup_mixed_vs_plain": ms_plain / ms_mixed,
                           "l2": "512 MB buffer written between timed steps",
                           "launches_per_step": {"mixed": launches // max(1, args.steps),
                                                 "plain": launches_plain // max(1, args.steps)},
                           "accuracy_mixed": {"sigma_err_rel_smax": sig_err, "ortho_resid": info_m["ortho_resid"],
                                              "polar_steps": [info_m["steps_bf16"], info_m["steps_tf32"],
                                                              info_m["steps_3xtf32"]]}},
                "roofline": roofline,
                "clocks": clk.summary(),
                "e2e": {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": N * N * 4,
                        "d2h_bytes_per_step": N * N * 4 + N * 4},
                "gpu_launches": int(launches)}
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline_leg()
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
