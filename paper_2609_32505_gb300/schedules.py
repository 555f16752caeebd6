"""Schedule comparison for the polar iteration (the polar-iteration ablation of Appendix B):
classical Newton-Schulz, a Polar-Express-style damped schedule, conservative CANS and the
learned lower bound, on the ablation's setting -- square 1024 x 1024 matrices with
kappa = 1e6 (A = Q1 diag(s) Q2^T, s_i = kappa^((n-i)/(n-1))).

    python -m paper_2609_32505_gb300.schedules [--n 1024] [--kappa 1e6] [--batch 4] [--prec 0]

For every schedule: polynomial steps per matrix, device time of psvd_polar_fwd (CUDA events,
best of a few after warm-up), the relative orthogonality ||W^T W - I||_F / sqrt(n) after every
step (the ablation figure's curve, from opts.res_history), the final residual, the
reconstruction ||A - W H||_F / ||A||_F (FP64 on the device), and, for the learned schedule,
how many matrices fell back to the conservative rerun.  The learned and the damped schedules
start from the same predicted lower bound (the sketch + network of the learned schedule).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_2609_32505_gb300 as P  # noqa: E402
import workloads as W  # noqa: E402

NAMES = {P.SCHED_NS: "newton_schulz", P.SCHED_PE: "polar_express_style", P.SCHED_CANS: "cans",
         P.SCHED_LEARNED: "learned"}


def _time(f, reps=3, warmup=1):
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


def compare(A: torch.Tensor, lower_bound: torch.Tensor, precision: int = P.PREC_FP32, reps: int = 3,
            schedules=(P.SCHED_NS, P.SCHED_PE, P.SCHED_CANS, P.SCHED_LEARNED)):
    bt, m, n = A.shape
    out = {}
    a64 = A.double()
    for sched in schedules:
        kw = dict(precision=precision, schedule=sched)
        if sched in (P.SCHED_LEARNED, P.SCHED_PE):
            kw["lower_bound"] = lower_bound
        kcap = 50 + (2 if sched == P.SCHED_CANS else 0)
        hist = torch.zeros((kcap + 1) * bt, dtype=torch.float64, device=A.device)
        o = P.make_opts(res_history=hist, **kw)
        w, h, info = P.polar(A, o, return_info=True)
        torch.cuda.synchronize()
        curves = hist.view(kcap + 1, bt).T.cpu().tolist()
        rec = [float(torch.linalg.matrix_norm(a64[b] - w[b].double() @ h[b].double()) /
                     torch.linalg.matrix_norm(a64[b])) for b in range(bt)]
        o_t = P.make_opts(**kw)
        ms = _time(lambda: P.polar(A, o_t, want_h=False), reps)
        out[NAMES[sched]] = {
            "steps": [i["iters"] for i in info], "status": [i["status"] for i in info],
            "sched_fallback": [i["sched_fallback"] for i in info],
            "ortho_resid": [i["ortho_resid"] for i in info], "recon": rec, "ms_polar_batch": ms,
            "residual_curve": [[c for c in cur[: i["iters"] + 1]] for cur, i in zip(curves, info)]}
    return out


def run(n=1024, kappa=1e6, batch=4, precision=P.PREC_FP32, seed=1200, reps=3):
    dev = torch.device("cuda")
    A = W.torch_constructed(seed, n, n, W.kappa_spectrum(n, kappa), device=dev, batch=batch)
    from paper_2609_32505_gb300 import train_schedule
    params, margin, nprobe = train_schedule.load(device=dev)
    lb = P.predict_lower_bound(A, params, margin=margin, probes=nprobe, seed=7)
    res = compare(A, lb, precision, reps)
    return {"n": n, "kappa": kappa, "batch": batch, "precision": precision,
            "lower_bound": lb.cpu().tolist(), "schedules": res}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--kappa", type=float, default=1e6)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--prec", type=int, default=0)
    a = ap.parse_args(argv)
    P.lib()
    print(json.dumps(run(a.n, a.kappa, a.batch, a.prec)))


if __name__ == "__main__":
    main()
