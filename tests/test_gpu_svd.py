"""GPU SVD forward (Algorithm 1) against the FP64 oracle.

Gates from the benchmark spec, read as in the design notes: |sigma_i - sigma_i*| <=
1e-5 sigma_max, ||A - U S V^T||_F / ||A||_F <= 1e-5, orthogonality
||Q^T Q - I||_F / sqrt(n) <= 1e-4 (relative, the paper's metric) for U and V.
Singular vectors are compared through the polar factor U V^T where it is unique."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import psvd_oracle as O

pytestmark = pytest.mark.gpu


def _svd(a, **kw):
    import paper_2609_32505_gb300 as P
    u, s, vt, info = P.svd_fwd(torch.from_numpy(a.astype(np.float32)).cuda(), P.make_opts(**kw), return_info=True)
    torch.cuda.synchronize()
    return u.cpu().double().numpy(), s.cpu().double().numpy(), vt.cpu().double().numpy(), info


def _gates(a, u, s, vt, s_ref, precision=0):
    # Both paths meet the same gates: the mixed path keeps its BF16/TF32 result only
    # when the eigenbasis correction stays below PSVD_MIXED_CORR_MAX (error ~ corr^2)
    # and recomputes the matrix on the FP32-accurate path otherwise.
    assert np.abs(s - s_ref).max() <= 1e-5 * s_ref[0]
    assert O.recon_error(a, u, s, vt) <= 1e-5
    assert O.ortho_error(u) <= 1e-4 and O.ortho_error(vt.T) <= 1e-4


def _fallback_consistent(info):
    import paper_2609_32505_gb300 as P
    for i in info:
        bad = not (i["corr_max"] <= P.MIXED_CORR_MAX) or not (i["recon_est"] <= P.MIXED_RECON_MAX)
        assert i["prec_fallback"] == int(bad)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_svd_small_square(precision):
    a, s_true = W.small_square(seed=1, n=256)
    a32 = a.astype(np.float32).astype(np.float64)
    u_ref, s_ref, vt_ref, _ = O.svd(a32)
    u, s, vt, info = _svd(a32, precision=precision)
    _gates(a32, u, s, vt, s_ref, precision)
    if precision >= 1:
        _fallback_consistent(info)


@pytest.mark.parametrize("m,n,kappa", [(300, 200, 1e3), (130, 129, 10.0), (77, 40, 1e4)])
def test_svd_rect_parity(m, n, kappa):
    s0 = W.kappa_spectrum(n, kappa)
    a, q1, q2 = W.constructed(5, m, n, s0)
    a32 = a.astype(np.float32).astype(np.float64)
    u_ref, s_ref, vt_ref, _ = O.svd(a32)
    for precision in (0, 1, 2):
        u, s, vt, info = _svd(a32, precision=precision)
        _gates(a32, u, s, vt, s_ref, precision)
        if precision >= 1:
            _fallback_consistent(info)
        if precision == 0:
            # distinct, well separated spectrum: the factors themselves are unique
            np.testing.assert_allclose(u @ vt, u_ref @ vt_ref, atol=2e-4 * max(1, kappa / 1e3))


def test_svd_batch_marchenko_pastur():
    a = np.stack([W.marchenko_pastur(100 + i, 512, 128) for i in range(3)]).astype(np.float32).astype(np.float64)
    for precision in (0, 1, 2):
        u, s, vt, info = _svd(a, precision=precision)
        for b in range(3):
            s_ref = np.linalg.svd(a[b], compute_uv=False)
            _gates(a[b], u[b], s[b], vt[b], s_ref, precision)


def test_svd_rank_deficient():
    # generic rank deficiency: over the 50-step cap FP32 rounding in the null space
    # grows into an orthonormal completion, so the result is a valid SVD either way
    n, r = 96, 20
    s0 = W.kappa_spectrum(n, 10.0, rank=r)
    a, q1, q2 = W.constructed(7, 120, n, s0)
    a32 = a.astype(np.float32).astype(np.float64)
    u, s, vt, info = _svd(a32)
    s_ref = np.linalg.svd(a32, compute_uv=False)
    assert np.abs(s - s_ref).max() <= 1e-5 * s_ref[0]
    assert O.recon_error(a32, u, s, vt) <= 1e-5
    assert O.ortho_error(u) <= 1e-4
    p_ref = q1[:, :r] @ q1[:, :r].T          # the leading r left vectors span a unique subspace
    assert np.abs(u[:, :r] @ u[:, :r].T - p_ref).max() <= 1e-4


def test_svd_qr_fallback_zero_columns():
    # exactly zero columns stay exactly zero through X <- X (c1 I + c3 X^T X), so U = W V
    # has zero columns and the QR step of Appendix A.2 must supply them (diag R >= 0)
    rng = W.rng_for(8)
    a = np.zeros((80, 48))
    a[:, :40] = rng.standard_normal((80, 40))
    a32 = a.astype(np.float32).astype(np.float64)
    u, s, vt, info = _svd(a32)
    assert info[0]["qr_fallback"] == 1
    s_ref = np.linalg.svd(a32, compute_uv=False)
    assert np.abs(s - s_ref).max() <= 1e-5 * s_ref[0]
    assert O.recon_error(a32, u, s, vt) <= 1e-5
    assert O.ortho_error(u) <= 1e-5 and O.ortho_error(vt.T) <= 1e-4
    np.testing.assert_allclose(u[:, :40].T @ u[:, :40], np.eye(40), atol=1e-4)


def test_svd_zero_matrix():
    u, s, vt, info = _svd(np.zeros((1, 20, 12)))
    assert not s.any()
    np.testing.assert_allclose(u[0], np.eye(20)[:, :12], atol=1e-6)
    np.testing.assert_allclose(vt[0], np.eye(12), atol=1e-6)


@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_fallback_on_ill_conditioned_input(precision):
    # kappa = 1e3 at n = 200: the low-precision steps leave rotations in the small-sigma
    # directions larger than the first-order correction can undo, so the matrix is
    # recomputed on the FP32-accurate path
    n = 200
    a, _, _ = W.constructed(5, n, n, W.kappa_spectrum(n, 1e3))
    a = a.astype(np.float32).astype(np.float64)
    u, s, vt, info = _svd(a, precision=precision)
    _fallback_consistent(info)
    assert info[0]["prec_fallback"] == 1
    _gates(a, u, s, vt, O.svd(a)[1], precision)


def test_mixed_keeps_large_well_conditioned_result():
    # n = 1024, kappa = 10, TF32 steps: the correction stays small and the mixed result is kept; the
    # spectrum is known (Weyl: FP32 rounding of A moves it by <= ||A32 - A||_2)
    n = 1024
    s0 = W.kappa_spectrum(n, 10.0)
    a, _, _ = W.constructed(9, n, n, s0)
    a32 = a.astype(np.float32).astype(np.float64)
    weyl = np.linalg.norm(a32 - a, 2)
    u, s, vt, info = _svd(a32, precision=1)
    _fallback_consistent(info)
    assert info[0]["prec_fallback"] == 0 and info[0]["steps_tf32"] > 0
    assert np.abs(s - s0).max() <= 1e-5 * s0[0] + weyl
    assert O.recon_error(a32, u, s, vt) <= 1e-5
    assert O.ortho_error(u) <= 1e-4 and O.ortho_error(vt.T) <= 1e-4


def test_mixed_batch_of_different_spectra():
    # one batch, three condition numbers: the correction's first-order products drop to TF32
    # matrix by matrix (when 2^-11 max|K| / (2 s_min) and 2^-11 max|X| stay below FP32
    # resolution), so the matrices of one launch take different precisions; each must meet
    # the gates on its own and agree with the plain path's singular values
    n = 512
    a = np.stack([W.constructed(30 + i, n, n, W.kappa_spectrum(n, k))[0]
                  for i, k in enumerate((10.0, 1e2, 1e3))]).astype(np.float32).astype(np.float64)
    u, s, vt, info = _svd(a, precision=1)
    _, s_plain, _, _ = _svd(a, precision=0)
    _fallback_consistent(info)
    for b in range(3):
        s_ref = O.svd(a[b])[1]
        _gates(a[b], u[b], s[b], vt[b], s_ref, 1)
        assert np.abs(s[b] - s_plain[b]).max() <= 1e-5 * s_ref[0]
    assert info[0]["steps_tf32"] > 0 and info[0]["prec_fallback"] == 0


def test_mixed_reconstruction_check_on_tall_input():
    # m > n: the low-precision steps tilt the column space of W; the probe estimate of the
    # reconstruction error sees it, and the result still meets the gates
    a, _, _ = W.constructed(8, 260, 100, W.kappa_spectrum(100, 10.0))
    a = a.astype(np.float32).astype(np.float64)
    u, s, vt, info = _svd(a, precision=1)
    _fallback_consistent(info)
    assert info[0]["recon_est"] > 0
    _gates(a, u, s, vt, O.svd(a)[1], 1)


@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_reconstruction_estimate_tracks_the_error(precision):
    # the 8-probe estimate of ||A - U S V^T||_F / ||A||_F against the error of the returned
    # factors, where the mixed result was kept (after a fallback the record still holds the
    # mixed attempt's estimate, while the factors come from the FP32-accurate rerun)
    a, _, _ = W.constructed(9, 1024, 1024, W.kappa_spectrum(1024, 10.0))
    a = a.astype(np.float32).astype(np.float64)
    u, s, vt, info = _svd(a, precision=precision)
    _fallback_consistent(info)
    if info[0]["prec_fallback"] == 0:
        err = O.recon_error(a, u, s, vt)
        assert 0.3 * err <= info[0]["recon_est"] <= 3.0 * err + 1e-7


def test_mixed_learned_gate_on_small_lower_bound():
    # PSVD_MIXED_LB_MIN: with the learned schedule, a matrix whose lower bound is below the
    # threshold starts on the split-TF32 rung (no TF32 step, nothing to recompute); one with
    # a larger bound makes its TF32 attempt.  Batch of two: kappa = 1e3 with a bound below
    # the threshold, kappa = 10 with a bound above it; both bounds are valid (<= sigma_min(X0)).
    import paper_2609_32505_gb300 as P
    n = 512
    mats = [W.constructed(21, n, n, W.kappa_spectrum(n, k))[0].astype(np.float32).astype(np.float64)
            for k in (1e3, 10.0)]
    lbs = []
    for a in mats:
        scale = np.sqrt(np.abs(a).sum(0).max() * np.abs(a).sum(1).max())
        lbs.append(0.5 * O.svd(a)[1][-1] / scale)          # half of sigma_min(X0)
    lbs[0] = min(lbs[0], 0.5 * P.MIXED_LB_MIN)
    assert lbs[0] < P.MIXED_LB_MIN <= lbs[1]
    A = torch.from_numpy(np.stack(mats).astype(np.float32)).cuda()
    lb = torch.tensor(lbs, dtype=torch.float32, device="cuda")
    U, S, VT, info = P.svd_fwd(A, P.make_opts(precision=P.PREC_MIXED, schedule=P.SCHED_LEARNED, lower_bound=lb),
                               return_info=True)
    torch.cuda.synchronize()
    _fallback_consistent(info)
    assert info[0]["status"] == 0 and info[0]["sched_fallback"] == 0
    assert info[0]["steps_tf32"] == 0 and info[0]["steps_bf16"] == 0 and info[0]["steps_3xtf32"] > 0
    assert info[0]["prec_fallback"] == 0
    assert info[1]["steps_tf32"] > 0 or info[1]["prec_fallback"] == 1
    u, s, vt = U.cpu().double().numpy(), S.cpu().double().numpy(), VT.cpu().double().numpy()
    for b, a in enumerate(mats):
        _gates(a, u[b], s[b], vt[b], O.svd(a)[1], 1)


@pytest.mark.parametrize("precision", [0, 1])
def test_learned_schedule_miss_is_recomputed_on_the_plain_path(precision):
    # svd_fwd with the learned schedule and a deliberately over-predicted bound for the first
    # matrix: that matrix misses tol within its budget, and instead of a conservative rerun of
    # the polar iteration inside the call (as psvd_polar_fwd does) it joins the one recompute
    # of flagged matrices on the plain FP32-accurate path; the record says why.
    import paper_2609_32505_gb300 as P
    n = 200
    mats = [W.constructed(31 + k, n, n, W.kappa_spectrum(n, k_))[0].astype(np.float32).astype(np.float64)
            for k, k_ in enumerate((1e3, 10.0))]
    lbs = []
    for a in mats:
        scale = np.sqrt(np.abs(a).sum(0).max() * np.abs(a).sum(1).max())
        lbs.append(0.5 * O.svd(a)[1][-1] / scale)
    lbs[0] = 0.9                                            # far above sigma_min(X0)
    A = torch.from_numpy(np.stack(mats).astype(np.float32)).cuda()
    lb = torch.tensor(lbs, dtype=torch.float32, device="cuda")
    U, S, VT, info = P.svd_fwd(A, P.make_opts(precision=precision, schedule=P.SCHED_LEARNED, lower_bound=lb),
                               return_info=True)
    torch.cuda.synchronize()
    assert info[0]["sched_fallback"] == 1 and info[0]["status"] == 0
    assert info[0]["steps_3xtf32"] > 0 and info[0]["qr_fallback"] == 0
    assert info[1]["sched_fallback"] == 0
    if precision:
        _fallback_consistent(info)
    u, s, vt = U.cpu().double().numpy(), S.cpu().double().numpy(), VT.cpu().double().numpy()
    for b, a in enumerate(mats):
        _gates(a, u[b], s[b], vt[b], O.svd(a)[1], precision)
