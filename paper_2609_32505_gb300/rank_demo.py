"""Layer-wise rank selection by differentiating through the SVD of activations (the rank
learning of Section 5's compression experiment, Dobi-SVD style), on synthetic activations.

    python -m paper_2609_32505_gb300.rank_demo [--layers 4] [--d 256] [--tokens 1024]
                                               [--ratio 0.35] [--eps 0.1 1 10] [--iters 150]

A small synthetic network stands in for the language model (whose weights and data are not
available): L residual blocks h <- h + tanh(h W_i^T) of width d, with seeded weights whose
spectra have a knee at a layer-specific rank (the layers differ in how compressible their
activations are, as the layers of a real model do) and a seeded full-rank input of `tokens`
rows.  Each layer i has a trainable continuous rank gamma_i.  At every step the activations A_i = H_{i-1} W_i^T are
factored by the library (psvd.svd, forward Algorithm 1 and backward Algorithm 4 with the
chosen eps), truncated softly -- A_i ~ U diag(sigma o m(gamma_i)) V^T with
m_j(gamma) = sigmoid((gamma - j) / tau) -- and passed on; the loss is the relative distance
of the last layer's output to the uncompressed network's plus a penalty that pulls the mean
kept fraction sum_i gamma_i / (L d) to the target ratio.  Gradients reach gamma_i through
its own mask and through every later layer's SVD, which is where the regularized backward
matters.  After training, the ranks round_i(gamma_i) are applied as hard truncations and
compared with the uniform allocation of the same total rank.

The model around the SVD (products with W, tanh, the masks, Adam on L scalars) is ordinary
PyTorch: it stands for the user's network; every SVD and its backward run in libpsvd.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_2609_32505_gb300 as P  # noqa: E402
import workloads as W  # noqa: E402


# knee position of each layer's weight spectrum, as a fraction of d (cycled over the layers)
KNEES = (12 / 128, 80 / 128, 32 / 128, 56 / 128)


def make_problem(layers: int, d: int, tokens: int, seed: int = 0, device="cuda"):
    """Seeded weights and input.  Weight i: s_j = 1 - j / (2 r_i) up to its knee r_i, then
    0.5 exp(-(j - r_i) / 4); input: s_j = 0.5 sqrt(tokens) exp(-2 j / d) (full rank)."""
    ws = []
    j = np.arange(d, dtype=np.float64)
    for i in range(layers):
        r = max(1, int(round(KNEES[i % len(KNEES)] * d)))
        s = np.where(j < r, 1.0 - 0.5 * j / r, 0.5 * np.exp(-(j - r) / 4.0))
        a, _, _ = W.constructed(seed * 100 + i, d, d, s)
        ws.append(torch.from_numpy(a.astype(np.float32)).to(device))
    sx = np.exp(-2.0 * j / d) * math.sqrt(tokens) * 0.5
    x, _, _ = W.constructed(seed * 100 + 99, tokens, d, sx)
    return ws, torch.from_numpy(x.astype(np.float32)).to(device)


def soft_mask(gamma: torch.Tensor, d: int, tau: float) -> torch.Tensor:
    j = torch.arange(d, device=gamma.device, dtype=torch.float32)
    return torch.sigmoid((gamma - j) / tau)


def forward(ws, x, gammas=None, ranks=None, eps=1e-8, kreg_mode=0, tau=2.0):
    """Output of the network with soft (gammas) or hard (ranks) truncation of every layer's
    activations, or uncompressed (neither)."""
    h = x
    for i, w in enumerate(ws):
        a = h @ w.T
        if gammas is not None or ranks is not None:
            u, s, vt = P.svd(a, eps=eps, kreg_mode=kreg_mode)
            d = s.shape[-1]
            if gammas is not None:
                s = s * soft_mask(gammas[i], d, tau)
            else:
                keep = torch.zeros(d, device=s.device)
                keep[:int(ranks[i])] = 1.0
                s = s * keep
            a = (u * s[None, :]) @ vt
        h = h + torch.tanh(a)
    return h


def rel_err(y, ref):
    return torch.linalg.matrix_norm(y - ref) / torch.linalg.matrix_norm(ref)


def demo_loss(ws, x, ref, gammas, ratio, lam, eps, kreg_mode, tau=2.0):
    d = ws[0].shape[0]
    y = forward(ws, x, gammas=gammas, eps=eps, kreg_mode=kreg_mode, tau=tau)
    kept = torch.stack(list(gammas)).sum() / (len(ws) * d)
    return rel_err(y, ref) ** 2 + lam * (kept - ratio) ** 2, y


def train(ws, x, ratio: float, eps: float, kreg_mode: int = 0, iters: int = 150, lr: float = 1.0,
          lam: float = 50.0, tau: float = 2.0):
    d = ws[0].shape[0]
    ref = forward(ws, x)
    gammas = [torch.tensor(ratio * d, device=x.device, requires_grad=True) for _ in ws]
    opt = torch.optim.Adam(gammas, lr=lr)
    curve, grad_norms = [], []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in range(iters):
        opt.zero_grad()
        loss, _ = demo_loss(ws, x, ref, gammas, ratio, lam, eps, kreg_mode, tau)
        loss.backward()
        g = torch.stack([gm.grad for gm in gammas])
        if not torch.isfinite(g).all():
            raise FloatingPointError(f"non-finite gradient at iteration {it}")
        grad_norms.append(float(g.norm()))
        opt.step()
        with torch.no_grad():
            for gm in gammas:
                gm.clamp_(1.0, float(d))
        if it % 10 == 0 or it == iters - 1:
            curve.append(float(loss.detach()))
    torch.cuda.synchronize()
    sec = (time.perf_counter() - t0) / iters
    return [float(gm) for gm in gammas], curve, grad_norms, sec


def hard_ranks(gammas, total: int, d: int):
    """Integer ranks with the same total as `total`, proportional to the learned gammas."""
    g = np.asarray(gammas, dtype=np.float64)
    r = np.floor(g / g.sum() * total).astype(int)
    for i in np.argsort(-(g / g.sum() * total - r))[: total - r.sum()]:
        r[i] += 1
    return np.clip(r, 1, d)


def run(layers=4, d=256, tokens=1024, ratio=0.35, eps_list=(0.1, 1.0, 10.0), iters=150, kreg_mode=0, seed=0):
    ws, x = make_problem(layers, d, tokens, seed)
    ref = forward(ws, x)
    total = int(round(ratio * d * layers))
    uniform = [total // layers + (1 if i < total % layers else 0) for i in range(layers)]
    with torch.no_grad():
        err_uniform = float(rel_err(forward(ws, x, ranks=uniform), ref))
    out = {"layers": layers, "d": d, "tokens": tokens, "ratio": ratio, "kreg_mode": kreg_mode,
           "uniform": {"ranks": uniform, "rel_err": err_uniform}, "learned": []}
    for eps in eps_list:
        gam, curve, gn, sec = train(ws, x, ratio, eps, kreg_mode, iters)
        ranks = hard_ranks(gam, total, d)
        with torch.no_grad():
            err = float(rel_err(forward(ws, x, ranks=ranks), ref))
        out["learned"].append({"eps": eps, "gammas": gam, "ranks": ranks.tolist(), "rel_err": err,
                               "loss_curve": curve, "max_grad_norm": max(gn), "sec_per_iter": sec})
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--layers", type=int, default=4)
    ap.add_argument("--d", type=int, default=256)
    ap.add_argument("--tokens", type=int, default=1024)
    ap.add_argument("--ratio", type=float, default=0.35)
    ap.add_argument("--eps", type=float, nargs="+", default=[0.1, 1.0, 10.0])
    ap.add_argument("--iters", type=int, default=150)
    ap.add_argument("--kreg", type=int, default=0)
    a = ap.parse_args(argv)
    P.lib()
    print(json.dumps(run(a.layers, a.d, a.tokens, a.ratio, tuple(a.eps), a.iters, a.kreg)))


if __name__ == "__main__":
    main()
