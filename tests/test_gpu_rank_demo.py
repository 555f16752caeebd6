"""The rank-selection demo (differentiating through the SVD of activations, Section 5's
compression experiment on synthetic data): its gradient with respect to the continuous
ranks against a central finite difference of the same loss evaluated in FP64 with the
oracle's SVD, and a short training run for each eps of the paper's ablation."""
import math

import numpy as np
import pytest
import torch

from oracle import psvd_oracle as O

pytestmark = pytest.mark.gpu


def _np_forward(ws, x, gammas, tau):
    """The demo's soft-truncated network in FP64, every SVD by the oracle (Algorithm 1)."""
    h = x
    for w, g in zip(ws, gammas):
        a = h @ w.T
        u, s, vt, _ = O.svd(a)
        d = s.shape[0]
        m = 1.0 / (1.0 + np.exp(-(g - np.arange(d)) / tau))
        h = h + np.tanh((u * (s * m)[None, :]) @ vt)
    return h


def _np_loss(ws, x, ref, gammas, ratio, lam, tau):
    y = _np_forward(ws, x, gammas, tau)
    kept = sum(gammas) / (len(ws) * ws[0].shape[0])
    return (np.linalg.norm(y - ref) / np.linalg.norm(ref)) ** 2 + lam * (kept - ratio) ** 2


def test_rank_gradient_matches_fp64_finite_differences():
    from paper_2609_32505_gb300 import rank_demo as R
    layers, d, tokens, ratio, lam, tau = 3, 32, 96, 0.4, 50.0, 2.0
    ws, x = R.make_problem(layers, d, tokens, seed=3)
    gam0 = [9.3, 14.1, 11.7]
    # library: FP32 forward, Algorithm 4 backward with the exact mask (kreg_mode 2)
    ref = R.forward(ws, x)
    gammas = [torch.tensor(g, device="cuda", requires_grad=True) for g in gam0]
    loss, _ = R.demo_loss(ws, x, ref, gammas, ratio, lam, eps=0.0, kreg_mode=2, tau=tau)
    loss.backward()
    g_lib = np.array([float(g.grad) for g in gammas])
    # FP64: the same loss with the oracle's SVD, central differences h = 1e-4
    ws64 = [w.cpu().double().numpy() for w in ws]
    x64 = x.cpu().double().numpy()
    ref64 = _np_forward(ws64, x64, [1e9] * layers, tau)      # masks at 1: uncompressed
    g_fd = np.zeros(layers)
    for i in range(layers):
        gp, gm = list(gam0), list(gam0)
        gp[i] += 1e-4
        gm[i] -= 1e-4
        g_fd[i] = (_np_loss(ws64, x64, ref64, gp, ratio, lam, tau) -
                   _np_loss(ws64, x64, ref64, gm, ratio, lam, tau)) / 2e-4
    assert np.linalg.norm(g_lib - g_fd) <= 1e-3 * np.linalg.norm(g_fd), (g_lib, g_fd)


@pytest.mark.parametrize("eps", [0.1, 1.0, 10.0])
def test_rank_demo_trains(eps):
    # the layers' knees differ, so the learned allocation must beat the uniform one of the same
    # total rank (hard truncation of both), and the loss must fall
    from paper_2609_32505_gb300 import rank_demo as R
    layers, d, ratio = 4, 128, 0.35
    ws, x = R.make_problem(layers, d, 512, seed=0)
    gam, curve, gn, sec = R.train(ws, x, ratio=ratio, eps=eps, iters=120)
    assert all(math.isfinite(g) for g in gam) and all(math.isfinite(g) for g in gn)
    assert curve[-1] < 0.5 * curve[0]
    total = int(round(ratio * d * layers))
    ranks = R.hard_ranks(gam, total, d)
    assert ranks.sum() == total
    uniform = [total // layers + (1 if i < total % layers else 0) for i in range(layers)]
    ref = R.forward(ws, x)
    with torch.no_grad():
        e_l = float(R.rel_err(R.forward(ws, x, ranks=ranks), ref))
        e_u = float(R.rel_err(R.forward(ws, x, ranks=uniform), ref))
    assert e_l < 0.7 * e_u, (ranks, e_l, e_u)
