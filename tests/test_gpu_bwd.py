"""GPU backward (Algorithm 4 / Algorithm 3) against the FP64 oracle.

The backward is a function of the factors, so both sides get the same ones: the exact
factors the input generator built the matrix from (A = Q1 diag(s) Q2^T), rounded to
FP32, which isolates the backward kernels.  The end-to-end autograd case compares the
library's own forward + backward with the oracle's forward + backward on a matrix with
well-separated singular values.  Bar: relative Frobenius error <= 1e-3."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import psvd_oracle as O

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _factor_inputs(q1, s, q2):
    """The generator's exact factors rounded to FP32: (CUDA tensors U, S, V^T for the
    library, the same values in FP64 for the oracle)."""
    host = [np.ascontiguousarray(x).astype(np.float32) for x in (q1, s, q2.T)]
    return [torch.from_numpy(x).cuda() for x in host], [x.astype(np.float64) for x in host]


@pytest.mark.parametrize("m,n", [(330, 300), (256, 256), (70, 33)])
@pytest.mark.parametrize("kreg,eps", [(0, 1e-8), (1, 1e-8), (2, 0.0)])
def test_svd_bwd_parity(m, n, kreg, eps):
    import paper_2609_32505_gb300 as P
    if m == n:
        a, q1, s0, q2 = W.small_square_factors(3, n)
    else:
        s0 = W.kappa_spectrum(n, 100.0)
        a, q1, q2 = W.constructed(4, m, n, s0)
    a32 = a.astype(np.float32).astype(np.float64)
    (u, s, vt), (U, S, VT) = _factor_inputs(q1, s0, q2)
    gu, gs, gv = W.loss_weights(9, m, n)
    du = torch.from_numpy(gu.astype(np.float32)).cuda()
    ds = torch.from_numpy(gs.astype(np.float32)).cuda()
    dvt = torch.from_numpy(gv.T.astype(np.float32)).cuda()     # loss <G_V, V>: gradient of V^T is G_V^T
    da = P.svd_bwd(torch.from_numpy(a32.astype(np.float32)).cuda(), u, s, vt, du, ds, dvt, eps, kreg)
    torch.cuda.synchronize()
    ref = O.svd_bwd(a32, U, S, VT, gu, gs, gv.T, eps=eps, kreg_mode=kreg, tie_tol=1e-6)
    assert _rel(da.cpu().double().numpy(), ref) <= 1e-3


def test_svd_bwd_null_gradients_and_clusters():
    import paper_2609_32505_gb300 as P
    a, q1, s0, q2 = W.clustered_square_factors(seed=300, n=128, n_clusters=32, mult=4)
    a32 = a.astype(np.float32).astype(np.float64)
    (u, s, vt), (U, S, VT) = _factor_inputs(q1, s0, q2)
    gu, gs, gv = W.loss_weights(301, 128, 128)
    A = torch.from_numpy(a32.astype(np.float32)).cuda()
    for du, ds, dvt in [(gu, None, None), (None, gs, None), (None, None, gv.T), (gu, gs, gv.T)]:
        t = lambda x: None if x is None else torch.from_numpy(np.ascontiguousarray(x).astype(np.float32)).cuda()
        da = P.svd_bwd(A, u, s, vt, t(du), t(ds), t(dvt), 1e-8, 0).cpu().double().numpy()
        ref = O.svd_bwd(a32, U, S, VT, du, ds, dvt, eps=1e-8, kreg_mode=0)
        assert _rel(da, ref) <= 1e-3


@pytest.mark.parametrize("eps", [1e-8, 0.0])
def test_polar_bwd_parity(eps):
    import paper_2609_32505_gb300 as P
    s0 = W.kappa_spectrum(150, 50.0)
    a, q1, q2 = W.constructed(11, 200, 150, s0)
    a32 = a.astype(np.float32).astype(np.float64)
    A = torch.from_numpy(a32.astype(np.float32)).cuda()
    # the exact polar factors of the constructed matrix, W = Q1 Q2^T, H = Q2 diag(s) Q2^T
    h_exact = (q2 * s0[None, :]) @ q2.T
    Wn = (q1 @ q2.T).astype(np.float32).astype(np.float64)
    Hn = ((h_exact + h_exact.T) / 2).astype(np.float32).astype(np.float64)
    w = torch.from_numpy(Wn.astype(np.float32)).cuda()
    h = torch.from_numpy(Hn.astype(np.float32)).cuda()
    rng = W.rng_for(12)
    gw, gh = rng.standard_normal((200, 150)), rng.standard_normal((150, 150))
    da = P.polar_bwd(A, w, h, torch.from_numpy(gw.astype(np.float32)).cuda(),
                     torch.from_numpy(gh.astype(np.float32)).cuda(), eps).cpu().double().numpy()
    ref = O.polar_bwd(a32, Wn, Hn, gw, O.sym(gh), eps=eps)
    assert _rel(da, ref) <= 1e-3


def test_autograd_matches_oracle():
    import paper_2609_32505_gb300 as P
    # linear spectrum 1 .. 0.1 at n = 64: relative gaps 1.4e-2, so the library's and the
    # oracle's factors agree column by column to ~1e-5; the sign convention (largest |V| entry
    # of a column positive) has a margin of 1.5e-2 for this seed, so both pick the same signs
    n = 64
    a, _, _ = W.constructed(12, n, n, W.linear_spectrum(n))
    a32 = a.astype(np.float32)
    A = torch.from_numpy(a32).cuda().requires_grad_(True)
    u, s, vt = P.svd(A, eps=1e-8, kreg_mode=0)
    gu, gs, gv = W.loss_weights(6, n, n)
    loss = (u * torch.from_numpy(gu).float().cuda()).sum() + (s * torch.from_numpy(gs).float().cuda()).sum() + \
        (vt.T * torch.from_numpy(gv).float().cuda()).sum()
    (g,) = torch.autograd.grad(loss, A)
    U, S, VT, _ = O.svd(a32.astype(np.float64))                # the oracle's own forward
    ref = O.svd_bwd(a32.astype(np.float64), U, S, VT, gu, gs, gv.T, eps=1e-8, kreg_mode=0)
    assert _rel(g.cpu().double().numpy(), ref) <= 1e-3
