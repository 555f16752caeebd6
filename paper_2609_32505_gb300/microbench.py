"""Per-stage timings of the SVD pipeline through the C ABI (CUDA events, after warm-up).

  python -m paper_2609_32505_gb300.microbench gemm  --n 4096 --prec 0|1|2   (BF16, TF32, split-TF32)
  python -m paper_2609_32505_gb300.microbench polar --n 4096 --prec 0|1 [--learned]
  python -m paper_2609_32505_gb300.microbench eigh  --n 4096
  python -m paper_2609_32505_gb300.microbench svd   --n 4096 --prec 0|1
  python -m paper_2609_32505_gb300.microbench stages --n 4096
  python -m paper_2609_32505_gb300.microbench eigh_dc --n 4096     (divide and conquer, against eigh)
  python -m paper_2609_32505_gb300.microbench step --n 4096 [--prec 0]
      (the benchmark's step: learned bound, svd_fwd, svd_bwd; mixed unless --prec 0 -- the
       command the profiles' launch lists and kernel captures run)
  python -m paper_2609_32505_gb300.microbench qr --m 4096 --n 4096 [--batch B]
      (psvd_qr, with the time of its product-kernel launches)
  python -m paper_2609_32505_gb300.microbench budget --n 4096 --prec 0|1 [--learned]
      (polar_fwd with the default step budget against one trimmed to the steps the input needs:
       the difference is the time of the launches that found nothing left to do)

Inputs are A = Q1 diag(s) Q2^T with s_i = kappa^((n-i)/(n-1)) (kappa = 10 by default),
generated on the device.  `--reps 1 --warmup 1` keeps a profiler capture to a couple of
launches of each kernel.
"""
from __future__ import annotations

import argparse
import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_2609_32505_gb300 as P  # noqa: E402
import workloads as W  # noqa: E402


def _time(f, reps: int, warmup: int) -> float:
    for _ in range(warmup):
        f()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        f()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["gemm", "polar", "eigh", "svd", "stages", "budget", "qr", "eigh_dc", "step"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--m", type=int, default=0)
    ap.add_argument("--batch", type=int, default=1)
    ap.add_argument("--prec", type=int, default=0)
    ap.add_argument("--kappa", type=float, default=10.0)
    ap.add_argument("--learned", action="store_true")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=2)
    a = ap.parse_args(argv)
    n, m = a.n, a.m or a.n
    dev = torch.device("cuda")
    P.lib()
    A = W.torch_constructed(1, m, n, W.kappa_spectrum(n, a.kappa), device=dev, batch=a.batch)
    if a.what == "gemm":
        g = torch.Generator(device=dev)
        g.manual_seed(0)
        x = torch.randn(n, n, device=dev, generator=g)
        y = torch.randn(n, n, device=dev, generator=g)
        ms = _time(lambda: P.gemm_tn(x, y, a.prec), a.reps, a.warmup)
        print(f"gemm_tn n={n} prec={a.prec}: {ms:.3f} ms, {2 * n ** 3 / ms / 1e9:.1f} TFLOP/s (operand split included)")
        return
    o = P.make_opts(precision=a.prec)
    lb = None
    if a.learned:
        # an oracle-free stand-in for the learned bound: 0.9 sigma_min(X0), from the known
        # spectrum (sigma_min(A) = 1) and the normalization scale the iteration reports
        _, _, info = P.polar(A, o, want_h=False, return_info=True)
        lb = torch.tensor([0.9 / i["scale"] for i in info], device=dev, dtype=torch.float32)
        o = P.make_opts(precision=a.prec, schedule=P.SCHED_LEARNED, lower_bound=lb)
    if a.what == "step":
        import ctypes
        from paper_2609_32505_gb300 import train_schedule
        L = P.lib()
        params, margin, nprobe = train_schedule.load(device=dev)
        Z = P.rademacher_probes(1, n, nprobe, seed=5, device=dev)
        mixed = a.prec != 0
        g = torch.Generator(device="cpu")
        g.manual_seed(2000)
        GU = torch.randn(1, m, n, generator=g).to(dev)
        GS = torch.randn(1, n, generator=g).to(dev)
        GVT = torch.randn(1, n, n, generator=g).to(dev)

        def one():
            if mixed:
                lb = P.predict_lower_bound(A, params, margin=margin, z=Z)
                o = P.make_opts(precision=P.PREC_MIXED, schedule=P.SCHED_LEARNED, lower_bound=lb)
            else:
                o = P.make_opts()
            u, s, vt = P.svd_fwd(A, o)
            P.svd_bwd(A, u, s, vt, GU, GS, GVT, eps=1e-8, kreg_mode=0)
        ms = _time(one, a.reps, a.warmup)
        print(f"step n={n} {'mixed' if mixed else 'plain'}: {ms:.3f} ms, {P.kernel_launches()} launches so far",
              flush=True)
        return
    if a.what == "eigh_dc":
        _, H = P.polar(A, P.make_opts())
        ms = _time(lambda: P.eigh_dc(H), a.reps, a.warmup)
        ms_t = _time(lambda: P.eigh(H), a.reps, a.warmup)
        s1, v1 = P.eigh_dc(H)
        s2, v2 = P.eigh(H)
        h = H[0].double()
        v = v1[0].double().T
        res = float(torch.linalg.matrix_norm(h @ v - v * s1[0].double()) / torch.linalg.matrix_norm(h))
        print(f"eigh_dc n={n}: {ms:.3f} ms (tridiagonal eigh {ms_t:.3f} ms); max |s_dc - s_tri| / s_max "
              f"{float((s1 - s2).abs().max() / s2.abs().max()):.2e}; ||H V - V S|| / ||H|| {res:.2e}", flush=True)
        return
    if a.what == "qr":
        import ctypes
        L = P.lib()
        ms = _time(lambda: P.qr(A), a.reps, a.warmup)
        L.psvd_profile_enable(1)
        P.qr(A)
        torch.cuda.synchronize()
        prof = (ctypes.c_double * 20)()
        L.psvd_profile_read(prof)
        L.psvd_profile_enable(0)
        q, r = P.qr(A)
        a64 = A.double()
        rec = max(float(torch.linalg.matrix_norm(a64[b] - q[b].double() @ r[b].double()) /
                        torch.linalg.matrix_norm(a64[b])) for b in range(A.shape[0]))
        print(f"qr {a.batch} x {m} x {n}: {ms:.3f} ms; product-kernel launches {int(prof[8])} taking "
              f"{prof[9]:.3f} ms (with event overhead); recon {rec:.2e}", flush=True)
        return
    if a.what == "budget":
        _, _, info = P.polar(A, o, want_h=False, return_info=True)
        used = max(i["iters"] for i in info)
        full = _time(lambda: P.polar(A, o, want_h=False), a.reps, a.warmup)
        kw = dict(precision=a.prec, max_iter=max(1, used + 1 - (2 if not a.learned else 0)))
        if a.learned:
            kw.update(schedule=P.SCHED_LEARNED, lower_bound=lb, budget=used + 1)
        ot = P.make_opts(**kw)
        _, _, info_t = P.polar(A, ot, want_h=False, return_info=True)
        assert all(i["status"] == 0 for i in info_t), info_t
        trim = _time(lambda: P.polar(A, ot, want_h=False), a.reps, a.warmup)
        print(f"budget n={n} prec={a.prec} learned={a.learned}: steps used {used}; default budget {full:.3f} ms, "
              f"trimmed {trim:.3f} ms, empty launches {full - trim:.3f} ms", flush=True)
        return
    if a.what in ("polar", "stages"):
        ms = _time(lambda: P.polar(A, o), a.reps, a.warmup)
        _, _, info = P.polar(A, o, return_info=True)
        i = info[0]
        print(f"polar n={n} prec={a.prec}: {ms:.3f} ms steps bf16/tf32/3xtf32 = "
              f"{i['steps_bf16']}/{i['steps_tf32']}/{i['steps_3xtf32']} ortho {i['ortho_resid']:.2e}", flush=True)
    if a.what in ("eigh", "stages"):
        import ctypes
        _, H = P.polar(A, P.make_opts())
        ms = _time(lambda: P.eigh(H), a.reps, a.warmup)
        L = P.lib()
        L.psvd_profile_enable(1)
        P.eigh(H)
        torch.cuda.synchronize()
        prof = (ctypes.c_double * 20)()
        L.psvd_profile_read(prof)
        L.psvd_profile_enable(0)
        print(f"eigh n={n}: {ms:.3f} ms (tridiagonalization {prof[4 * 4 + 1]:.3f} ms of one call)", flush=True)
    if a.what in ("svd", "stages"):
        ms = _time(lambda: P.svd_fwd(A, o), a.reps, a.warmup)
        print(f"svd_fwd n={n} prec={a.prec}: {ms:.3f} ms", flush=True)
        if a.what == "stages":
            u, s, vt = P.svd_fwd(A, o)
            g = torch.randn_like(u)
            ms = _time(lambda: P.svd_bwd(A, u, s, vt, g, torch.ones_like(s), g.transpose(-1, -2).contiguous()),
                       a.reps, a.warmup)
            print(f"svd_bwd n={n}: {ms:.3f} ms", flush=True)


if __name__ == "__main__":
    main()
