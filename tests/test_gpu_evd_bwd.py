"""GPU EVD backward (Theorem 4.3 with the K_eps regularization of Section 5.2) through the
C ABI, against the FP64 oracle's evd_bwd on the same FP32-rounded factors.

Both sides take V and sigma rounded to FP32 and the same incoming gradients, so the
comparison sees only the GPU's arithmetic (split-TF32 products, FP32 masks): the relative
Frobenius error bound 1e-3 is the gradient tolerance used for every backward here."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import psvd_oracle as O

pytestmark = pytest.mark.gpu


def _factors(seed, n, spectrum):
    rng = W.rng_for(seed)
    v = W.orthonormal(rng, n, n).astype(np.float32).astype(np.float64)
    s = np.asarray(spectrum, dtype=np.float32).astype(np.float64)
    vbar = rng.standard_normal((n, n)).astype(np.float32).astype(np.float64)
    sbar = rng.standard_normal(n).astype(np.float32).astype(np.float64)
    return v, s, vbar, sbar


def _gpu(vs, ss, vbars, sbars, eps, mode, with_v=True, with_s=True):
    import paper_2609_32505_gb300 as P
    cu = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    VT = cu(np.stack([v.T for v in vs]))
    S = cu(np.stack(ss))
    dVT = cu(np.stack([vb.T for vb in vbars])) if with_v else None
    dS = cu(np.stack(sbars)) if with_s else None
    dH = P.eigh_bwd(S, VT, dS, dVT, eps=eps, kreg_mode=mode)
    torch.cuda.synchronize()
    return dH.cpu().double().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("n", [64, 200, 300])
@pytest.mark.parametrize("mode,eps", [(0, 1e-8), (0, 1e-2), (1, 1e-3), (1, 1.0), (2, 0.0)])
def test_eigh_bwd_parity(n, mode, eps):
    # two matrices per batch: a linear spectrum and a kappa = 1e3 geometric one (distinct values)
    specs = [np.linspace(2.0, 0.5, n), W.kappa_spectrum(n, 1e3)]
    fac = [_factors(800 + 7 * k + n, n, sp) for k, sp in enumerate(specs)]
    got = _gpu([f[0] for f in fac], [f[1] for f in fac], [f[2] for f in fac], [f[3] for f in fac], eps, mode)
    for b, (v, s, vbar, sbar) in enumerate(fac):
        ref = O.evd_bwd(v, s, vbar, sbar, eps=eps, kreg_mode=mode)
        assert _rel(got[b], ref) <= 1e-3, (b, _rel(got[b], ref))
        assert np.abs(got[b] - got[b].T).max() <= 1e-5 * np.abs(got[b]).max()


def test_eigh_bwd_null_gradients_and_clusters():
    # repeated eigenvalues (clusters of 4) with the Algorithm 4 regularizer, and the two
    # one-sided cases: only Sbar (Hbar = V diag(Sbar) V^T exactly) and only Vbar
    n = 96
    spec = np.repeat(np.linspace(1.5, 0.2, n // 4), 4)
    v, s, vbar, sbar = _factors(830, n, spec)
    got = _gpu([v], [s], [vbar], [sbar], 1e-8, 0)[0]
    assert _rel(got, O.evd_bwd(v, s, vbar, sbar, eps=1e-8, kreg_mode=0)) <= 1e-3
    only_s = _gpu([v], [s], [vbar], [sbar], 1e-8, 0, with_v=False)[0]
    assert _rel(only_s, (v * sbar[None, :]) @ v.T) <= 1e-5
    only_v = _gpu([v], [s], [vbar], [sbar], 1e-8, 0, with_s=False)[0]
    assert _rel(only_v, O.evd_bwd(v, s, vbar, None, eps=1e-8, kreg_mode=0)) <= 1e-3


def test_eigh_autograd_through_library():
    # eigh_ad: forward psvd_eigh, backward psvd_eigh_bwd; the loss <G, V> + <g, S> on a
    # symmetric matrix with well-separated eigenvalues, against the oracle on the library's
    # own factors (the pseudo-gradient is defined at the factorization)
    import paper_2609_32505_gb300 as P
    n = 128
    rng = W.rng_for(840)
    q = W.orthonormal(rng, n, n)
    lam = np.linspace(3.0, 0.3, n)
    h = ((q * lam[None, :]) @ q.T).astype(np.float32)
    g_v, g_s = rng.standard_normal((n, n)), rng.standard_normal(n)
    H = torch.from_numpy(h).cuda().requires_grad_(True)
    s, vt = P.eigh_ad(H, eps=1e-8, kreg_mode=0)
    loss = (vt.T * torch.from_numpy(g_v).float().cuda()).sum() + (s * torch.from_numpy(g_s).float().cuda()).sum()
    (dh,) = torch.autograd.grad(loss, H)
    torch.cuda.synchronize()
    v = vt.detach().cpu().double().numpy().T
    sv = s.detach().cpu().double().numpy()
    ref = O.evd_bwd(v, sv, g_v, g_s, eps=1e-8, kreg_mode=0)
    assert _rel(dh.cpu().double().numpy(), ref) <= 1e-3
