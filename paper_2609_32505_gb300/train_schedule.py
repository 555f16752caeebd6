"""Trains the lower-bound network of the learned polynomial schedule on the GPU.

    python -m paper_2609_32505_gb300.train_schedule [--out paper_2609_32505_gb300/schedule_mlp.npz]
    python -m paper_2609_32505_gb300.train_schedule --evaluate 2048      (held-out comparison)

Training data are spectra the method itself produces: seeded matrices from the three
families of the learned-schedule study (geometric spectra with kappa in [1e1, 1e6], power
laws i^-p with p in [0.3, 1.5], rank 64 plus 1e-4 Gaussian noise) at sizes 256 to 4096
(Haar orthogonal factors from a device QR of seeded Gaussians), whose
smallest singular value and normalization scale come from the library's own FP32-accurate
svd_fwd.  The target is log sigma_min(X0), X0 = M / sqrt(||M||_1 ||M||_inf); the features
are the eight sketch features (psvd_sketch_features) with seeded Rademacher probes.  The
network is fitted with the library's Adam kernels (mlp_fit), and the safety margin is a
quantile of the over-prediction on held-out matrices.  The file holds the parameters, the
margin, the number of probes and the fit statistics.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_2609_32505_gb300 as P  # noqa: E402
import workloads as W  # noqa: E402

DEFAULT_OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "schedule_mlp.npz")
PROBES = 8


def _orthonormal(gen, n, device):
    """Haar orthogonal n x n: Q of the device QR of a Gaussian, signs fixed by diag(R) > 0.
    FP32 (GB300's FP64 rate is low, and the labels come from svd_fwd on the matrix as built)."""
    g = torch.randn(n, n, generator=gen, dtype=torch.float32).to(device)
    q, r = torch.linalg.qr(g)
    d = torch.sign(torch.diagonal(r))
    return q * torch.where(d == 0, torch.ones_like(d), d)[None, :]


def family_batch(seeds, n, device):
    """Matrices of the three families (seeded) as one (len(seeds), n, n) FP32 batch."""
    out = torch.empty(len(seeds), n, n, device=device)
    for i, s in enumerate(seeds):
        fam, spec = W.schedule_family(int(s), n)
        gen = torch.Generator()
        gen.manual_seed(50_000 + int(s))
        q1, q2 = _orthonormal(gen, n, device), _orthonormal(gen, n, device)
        sp = torch.as_tensor(np.ascontiguousarray(spec), dtype=torch.float32, device=device)
        a = (q1 * sp[None, :]) @ q2.T
        if fam == 2:
            a = a + 1e-4 * torch.randn(n, n, generator=gen).to(device)
        out[i] = a
    return out


def features_and_labels(seeds, n, device):
    chunk = max(1, min(32, (1 << 24) // (n * n)))
    feats, labels = [], []
    for c in range(0, len(seeds), chunk):
        sd = seeds[c:c + chunk]
        A = family_batch(sd, n, device)
        _, s, _, info = P.svd_fwd(A, P.make_opts(), return_info=True)
        scale = torch.tensor([i["scale"] for i in info], device=device)
        labels.append(torch.log(s[:, -1].clamp_min(1e-30) / scale))
        Z = P.rademacher_probes(len(sd), n, PROBES, seed=int(sd[0]), device=device)
        feats.append(P.sketch_features(A, Z))
        del A
    return torch.cat(feats), torch.cat(labels)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_OUT)
    ap.add_argument("--sizes", default="256:6000,512:6000,1024:5000,2048:2400,4096:600")
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--quantile", type=float, default=0.95)
    ap.add_argument("--evaluate", type=int, default=0, help="evaluate the stored network on this many matrices")
    a = ap.parse_args(argv)
    if a.evaluate:
        P.lib()
        evaluate(a.evaluate, path=a.out)
        return
    dev = torch.device("cuda")
    P.lib()
    F, Y = [], []
    seed = 10_000
    for item in a.sizes.split(","):
        n, cnt = (int(x) for x in item.split(":"))
        f, y = features_and_labels(list(range(seed, seed + cnt)), n, dev)
        seed += cnt
        F.append(f)
        Y.append(y)
        print(f"n={n}: {cnt} matrices, labels in [{y.min().item():.2f}, {y.max().item():.2f}]", flush=True)
    F, Y = torch.cat(F), torch.cat(Y)
    g = torch.Generator(device="cpu")
    g.manual_seed(1)
    perm = torch.randperm(F.shape[0], generator=g).to(dev)
    F, Y = F[perm].contiguous(), Y[perm].contiguous()
    nh = max(1, F.shape[0] // 5)                     # held out for the margin
    params, curve = P.mlp_fit(F[nh:], Y[nh:], steps=a.steps, lr=3e-3, batch=256, seed=0)
    margin = P.mlp_calibrate(params, F[:nh], Y[:nh], quantile=a.quantile)
    resid = (P.mlp_forward(params, F[:nh]) - Y[:nh]).abs()
    np.savez(a.out, params=params.cpu().numpy().astype(np.float32), margin=np.float32(margin),
             probes=np.int32(PROBES), loss_first=np.float32(curve[0]), loss_last=np.float32(curve[-1]),
             heldout_median_abs=np.float32(resid.median().item()), count=np.int32(F.shape[0]))
    print(f"trained on {F.shape[0] - nh}, held out {nh}: loss {curve[0]:.3f} -> {curve[-1]:.4f}, "
          f"held-out median |log error| {resid.median().item():.3f}, margin {margin:.3f} -> {a.out}")


def evaluate(count: int, n: int = 1024, chunk: int = 64, path: str = DEFAULT_OUT, quiet: bool = False):
    """Held-out matrices of the three families (seeds 400, 401, ...): steps and device time of
    the conservative and the learned schedule (bound prediction included), same tolerance."""
    dev = torch.device("cuda")
    params, margin, nprobe = load(path, dev)
    tot = {"cons_ms": 0.0, "learn_ms": 0.0, "pred_ms": 0.0}
    steps_c, steps_l, n_ok, n_fb, n_fail = [], [], 0, 0, 0

    def timed(f):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        r = f()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    ortho_c, ortho_l = [], []
    for c in range(0, count, chunk):
        seeds = list(range(400 + c, 400 + min(count, c + chunk)))
        A = family_batch(seeds, n, dev)
        Z = P.rademacher_probes(len(seeds), n, nprobe, seed=400 + c, device=dev)
        lb, t = timed(lambda: P.predict_lower_bound(A, params, margin, z=Z))
        tot["pred_ms"] += t
        (_, _, ic), t = timed(lambda: P.polar(A, P.make_opts(), want_h=False, return_info=True))
        tot["cons_ms"] += t
        o = P.make_opts(schedule=P.SCHED_LEARNED, lower_bound=lb)
        (_, _, il), t = timed(lambda: P.polar(A, o, want_h=False, return_info=True))
        tot["learn_ms"] += t
        for a, b in zip(ic, il):
            if a["status"] != 0:
                n_fail += 1
                continue
            n_ok += 1
            n_fb += b["sched_fallback"]
            steps_c.append(a["iters"])
            steps_l.append(b["iters"])
            ortho_c.append(a["ortho_resid"])
            ortho_l.append(b["ortho_resid"])
        del A
    res = {"matrices": count, "n": n, "converged": n_ok, "hit_cap": n_fail,
           "mean_steps_conservative": float(np.mean(steps_c)), "mean_steps_learned": float(np.mean(steps_l)),
           "conservative_reruns": int(n_fb), "device_ms_conservative": tot["cons_ms"],
           "device_ms_learned": tot["learn_ms"], "device_ms_bound_prediction": tot["pred_ms"],
           "max_ortho_resid_conservative": float(np.max(ortho_c)), "max_ortho_resid_learned": float(np.max(ortho_l))}
    if not quiet:
        print(f"{count} matrices of {n} x {n}: {n_ok} converged under the conservative schedule ({n_fail} hit the "
              f"cap); mean steps conservative {res['mean_steps_conservative']:.2f}, learned "
              f"{res['mean_steps_learned']:.2f} ({n_fb} conservative reruns); device time conservative "
              f"{tot['cons_ms']:.1f} ms, learned {tot['learn_ms']:.1f} ms + bound prediction {tot['pred_ms']:.1f} ms; "
              f"largest final residual {res['max_ortho_resid_conservative']:.2e} / {res['max_ortho_resid_learned']:.2e}")
    return res


def load(path: str = DEFAULT_OUT, device="cuda"):
    """(params on `device`, margin, probes) from a file written by main()."""
    d = np.load(path)
    return torch.from_numpy(d["params"]).to(device), float(d["margin"]), int(d["probes"])


if __name__ == "__main__":
    main()
