"""GPU polar factor (the polar-factor part of Algorithm 1) against the FP64 oracle.

W is unique for full-rank inputs (Definition 2.1), so the CUDA path's W and H are
compared element by element with the oracle's, whatever schedule reached them.
Tolerances: FP32-accurate products give W to ~1e-6 * kappa-independent accuracy
(the polar factor is well conditioned in the entries of W when sigma_min is not
tiny); the bound used is 2e-5 max abs on W and 2e-5 * ||A||_2 on H."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import psvd_oracle as O

pytestmark = pytest.mark.gpu


def _run(a, **kw):
    import paper_2609_32505_gb300 as P
    o = P.make_opts(**kw)
    w, h, info = P.polar(torch.from_numpy(a.astype(np.float32)).cuda(), o, return_info=True)
    torch.cuda.synchronize()
    return w.cpu().double().numpy(), h.cpu().double().numpy(), info


@pytest.mark.parametrize("m,n,kappa", [(256, 256, 1e2), (300, 200, 1e3), (130, 129, 10.0), (64, 1, 1.0)])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_polar_parity(m, n, kappa, precision):
    s = W.kappa_spectrum(n, kappa)
    a, q1, q2 = W.constructed(3, m, n, s)
    a32 = a.astype(np.float32).astype(np.float64)
    w_ref, h_ref, _ = O.polar_newton_schulz(a32)
    w, h, info = _run(a32, precision=precision)
    assert all(i["status"] == 0 for i in info), info
    assert info[0]["ortho_resid"] <= 1e-5
    assert O.ortho_error(w) <= 2e-5
    if precision == 0:
        assert np.abs(w - w_ref).max() < 2e-5 * max(1.0, kappa / 1e3)
        assert np.abs(h - h_ref).max() < 2e-5 * s[0]
    else:
        # BF16/TF32 steps rotate X inside low-sigma subspaces and, for m > n, tilt it out of
        # its column space (invisible to the orthogonality residual, kept by later steps); H is
        # still an FP32-accurate product, so ||A - W H||_F / ||A||_F is that rounding's footprint.
        # A rounding error made at step k in the direction of a right singular vector v_i is
        # amplified by the growth still ahead of sigma_i (1 / sigma_i^(k)) and weighted by
        # sigma_i(A) in A, so each step contributes O(u) relative to ||A||, independently of
        # kappa; the steps' errors are independent, so they add like sqrt(K).  Bound:
        # 4 u sqrt(K), u the unit roundoff of the step precision (TF32 2^-11, BF16 2^-8) and K
        # the number of low-precision steps.  (Measured at 300 x 200, kappa = 1e3: 4.2e-3 TF32,
        # 3.4e-2 BF16 -- the ratio of the two unit roundoffs; the paper's all-TF32 variant gives
        # about 1e-3 at 4096^2, Table 1.)
        low = "steps_bf16" if precision == 2 else "steps_tf32"
        assert info[0][low] > 0 and info[0]["steps_3xtf32"] > 0
        k_low = info[0]["steps_bf16"] + info[0]["steps_tf32"]
        u = 2.0 ** -11 if precision == 1 else 2.0 ** -8
        assert np.linalg.norm(a32 - w @ h) / np.linalg.norm(a32) < 4.0 * u * np.sqrt(k_low)


def test_polar_batch_and_schedules():
    a = np.stack([W.small_square(seed=s, n=192)[0] for s in range(3)]).astype(np.float32).astype(np.float64)
    refs = [O.polar_newton_schulz(x)[0] for x in a]
    for sched in (0, 2):
        w, h, info = _run(a, schedule=sched)
        for b in range(3):
            assert np.abs(w[b] - refs[b]).max() < 1e-4
            assert info[b]["status"] == 0


def test_polar_zero_and_nonfinite():
    import paper_2609_32505_gb300 as P
    a = np.zeros((2, 40, 30), dtype=np.float32)
    a[1, 3, 4] = np.nan
    w, h, info = P.polar(torch.from_numpy(a).cuda(), P.make_opts(), return_info=True)
    assert info[0]["status"] == 0 and not w[0].abs().sum().item()
    assert info[1]["status"] == -3 and torch.isnan(w[1]).all()
