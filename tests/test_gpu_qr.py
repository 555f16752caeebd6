"""Blocked Householder QR on the GPU (psvd_qr: the QR fallback of Appendix A.2 and the QR
preprocessing of Section 4.1), and the pre-QR route of svd_fwd / polar_fwd.

For full-rank A the thin QR with diag(R) > 0 is unique, so Q and R are compared element
by element with the oracle's (LAPACK QR with the signs fixed, a library step pinned in
tests/test_oracle_forward.py).  The perturbation of Q and R is about kappa(A) times the
backward error, so the element bound is 2e-5 kappa on inputs with kappa <= 1e2.  Shapes
cover every panel configuration (64- and 32-column panels, clusters of 8 and 16 CTAs) and
ragged edges (m, n not multiples of the panel or tile)."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import psvd_oracle as O

pytestmark = pytest.mark.gpu


def _qr(a):
    import paper_2609_32505_gb300 as P
    A = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    q, r = P.qr(A)
    torch.cuda.synchronize()
    return q.cpu().double().numpy(), r.cpu().double().numpy()


@pytest.mark.parametrize("m,n,kappa", [(300, 200, 10.0), (129, 129, 1e2), (77, 40, 1.0), (1000, 64, 10.0),
                                       (1030, 190, 10.0), (5000, 130, 10.0), (7000, 70, 10.0),
                                       (14336, 40, 10.0)])
def test_qr_parity(m, n, kappa):
    a, _, _ = W.constructed(900 + m + n, m, n, W.kappa_spectrum(n, kappa))
    a32 = a.astype(np.float32).astype(np.float64)
    q, r = _qr(a32)
    q_ref, r_ref = O.qr_nonneg(a32)
    assert np.abs(np.tril(r, -1)).max() == 0.0
    assert (np.diag(r) >= 0).all()
    assert np.linalg.norm(a32 - q @ r) / np.linalg.norm(a32) <= 1e-5
    assert O.ortho_error(q) <= 1e-5
    bound = 2e-5 * kappa
    assert np.abs(q - q_ref).max() <= bound
    assert np.abs(r - r_ref).max() <= bound * np.abs(r_ref).max()


def test_qr_batch_and_rank_deficient():
    # a batch of three: full rank, exactly rank 5 of 30 (zero singular values), zero matrix
    m, n = 90, 30
    a0, _, _ = W.constructed(940, m, n, W.kappa_spectrum(n, 10.0))
    a1, _, _ = W.constructed(941, m, n, W.kappa_spectrum(n, 10.0, rank=5))
    a = np.stack([a0, a1, np.zeros((m, n))]).astype(np.float32).astype(np.float64)
    q, r = _qr(a)
    for b in range(3):
        assert np.abs(np.tril(r[b], -1)).max() == 0.0 and (np.diag(r[b]) >= 0).all()
        assert O.ortho_error(q[b]) <= 1e-5                 # Householder Q stays orthonormal
        nrm = max(np.linalg.norm(a[b]), 1e-30)
        assert np.linalg.norm(a[b] - q[b] @ r[b]) / nrm <= 1e-5 or np.linalg.norm(a[b]) == 0.0
    q_ref, _ = O.qr_nonneg(a[0])
    assert np.abs(q[0] - q_ref).max() <= 2e-4


@pytest.mark.parametrize("precision", [0, 1])
def test_svd_preqr_parity(precision):
    # tall input: the QR preprocessing route against the oracle's (svd_preqr), and the mixed
    # result is kept (the square problem on R has no column space to lose)
    import paper_2609_32505_gb300 as P
    m, n = 1500, 300
    a, _, _ = W.constructed(950, m, n, W.kappa_spectrum(n, 10.0))
    a32 = a.astype(np.float32).astype(np.float64)
    A = torch.from_numpy(a32.astype(np.float32)).cuda()
    U, S, VT, info = P.svd_fwd(A, P.make_opts(precision=precision, preqr=1), return_info=True)
    torch.cuda.synchronize()
    u, s, vt = U.cpu().double().numpy(), S.cpu().double().numpy(), VT.cpu().double().numpy()
    u_ref, s_ref, vt_ref, _ = O.svd_preqr(a32)
    assert info[0]["status"] == 0
    assert np.abs(s - s_ref).max() <= 1e-5 * s_ref[0]
    assert O.recon_error(a32, u, s, vt) <= 1e-5
    assert O.ortho_error(u) <= 1e-4 and O.ortho_error(vt.T) <= 1e-4
    # distinct singular values: the factors agree column by column with the oracle's
    assert np.abs(np.abs((u * u_ref).sum(0)) - 1.0).max() <= 1e-3
    if precision:
        assert info[0]["prec_fallback"] == 0 and info[0]["steps_tf32"] > 0


def test_polar_preqr_parity():
    import paper_2609_32505_gb300 as P
    m, n = 900, 250
    a, _, _ = W.constructed(960, m, n, W.kappa_spectrum(n, 1e2))
    a32 = a.astype(np.float32).astype(np.float64)
    A = torch.from_numpy(a32.astype(np.float32)).cuda()
    w, h, info = P.polar(A, P.make_opts(preqr=1), return_info=True)
    torch.cuda.synchronize()
    w_ref, h_ref = O.polar_preqr(a32)
    assert info[0]["status"] == 0
    assert np.abs(w.cpu().double().numpy() - w_ref).max() <= 2e-5
    assert np.abs(h.cpu().double().numpy() - h_ref).max() <= 2e-5 * np.abs(h_ref).max()
