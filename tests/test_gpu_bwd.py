"""GPU backward (Algorithm 4 / Algorithm 3) against the FP64 oracle fed with the GPU's
own factors (the backward is a function of the factors; feeding both sides the same
U, S, V^T isolates the backward kernels).  Bar: relative Frobenius error <= 1e-3."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import psvd_oracle as O

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _factors(a32, precision=0):
    import paper_2609_32505_gb300 as P
    u, s, vt = P.svd_fwd(torch.from_numpy(a32.astype(np.float32)).cuda(), P.make_opts(precision=precision))
    return u, s, vt


@pytest.mark.parametrize("m,n", [(330, 300), (256, 256), (70, 33)])
@pytest.mark.parametrize("kreg,eps", [(0, 1e-8), (1, 1e-8), (2, 0.0)])
def test_svd_bwd_parity(m, n, kreg, eps):
    import paper_2609_32505_gb300 as P
    a, _ = W.small_square(seed=3, n=n) if m == n else (W.constructed(4, m, n, W.kappa_spectrum(n, 100.0))[0], None)
    a32 = a.astype(np.float32).astype(np.float64)
    u, s, vt = _factors(a32)
    gu, gs, gv = W.loss_weights(9, m, n)
    du = torch.from_numpy(gu.astype(np.float32)).cuda()
    ds = torch.from_numpy(gs.astype(np.float32)).cuda()
    dvt = torch.from_numpy(gv.T.astype(np.float32)).cuda()     # loss <G_V, V>: gradient of V^T is G_V^T
    da = P.svd_bwd(torch.from_numpy(a32.astype(np.float32)).cuda(), u, s, vt, du, ds, dvt, eps, kreg)
    torch.cuda.synchronize()
    U, S, VT = (x.cpu().double().numpy() for x in (u, s, vt))
    ref = O.svd_bwd(a32, U, S, VT, gu, gs, gv.T, eps=eps, kreg_mode=kreg, tie_tol=1e-6)
    assert _rel(da.cpu().double().numpy(), ref) <= 1e-3


def test_svd_bwd_null_gradients_and_clusters():
    import paper_2609_32505_gb300 as P
    a, s0 = W.clustered_square(seed=300, n=128, n_clusters=32, mult=4)
    a32 = a.astype(np.float32).astype(np.float64)
    u, s, vt = _factors(a32)
    gu, gs, gv = W.loss_weights(301, 128, 128)
    U, S, VT = (x.cpu().double().numpy() for x in (u, s, vt))
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
    w, h = P.polar(A)
    rng = W.rng_for(12)
    gw, gh = rng.standard_normal((200, 150)), rng.standard_normal((150, 150))
    da = P.polar_bwd(A, w, h, torch.from_numpy(gw.astype(np.float32)).cuda(),
                     torch.from_numpy(gh.astype(np.float32)).cuda(), eps).cpu().double().numpy()
    Wn, Hn = w.cpu().double().numpy(), h.cpu().double().numpy()
    ref = O.polar_bwd(a32, Wn, Hn, gw, O.sym(gh), eps=eps)
    assert _rel(da, ref) <= 1e-3


def test_autograd_matches_oracle():
    import paper_2609_32505_gb300 as P
    a, _ = W.small_square(seed=5, n=160)
    a32 = a.astype(np.float32)
    A = torch.from_numpy(a32).cuda().requires_grad_(True)
    u, s, vt = P.svd(A, eps=1e-8, kreg_mode=0)
    gu, gs, gv = W.loss_weights(6, 160, 160)
    loss = (u * torch.from_numpy(gu).float().cuda()).sum() + (s * torch.from_numpy(gs).float().cuda()).sum() + \
        (vt.T * torch.from_numpy(gv).float().cuda()).sum()
    (g,) = torch.autograd.grad(loss, A)
    U, S, VT = (x.detach().cpu().double().numpy() for x in (u, s, vt))
    ref = O.svd_bwd(a32.astype(np.float64), U, S, VT, gu, gs, gv.T, eps=1e-8, kreg_mode=0)
    assert _rel(g.cpu().double().numpy(), ref) <= 1e-3
