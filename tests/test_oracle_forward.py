"""Pins for the oracle's forward pieces (CPU only).

Each test checks the FP64 oracle against something other than itself: closed
forms (2x2 polar, constructed spectra), invariants of Definition 2.1, LAPACK
routines on cases that reduce to them, and brute-force minimax checks of the CANS
cubic."""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import psvd_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- normalization
def test_normalize_worked_example():
    # Algorithm 2 on [[1,2],[3,4]]: max column l1 = 6, max row l1 = 7 -> X0 = M / sqrt(42)
    m = np.array([[1.0, 2.0], [3.0, 4.0]])
    x0, s = O.normalize(m)
    assert s == pytest.approx(math.sqrt(42.0), rel=1e-15)
    np.testing.assert_allclose(x0, m / math.sqrt(42.0), rtol=1e-15)


@pytest.mark.parametrize("shape", [(7, 5), (40, 40), (64, 9)])
def test_normalize_spectral_bound(shape):
    # ||X0||_2 <= 1 because ||M||_2 <= sqrt(||M||_1 ||M||_inf) (Appendix A.1)
    rng = W.rng_for(5)
    for _ in range(20):
        m = rng.standard_normal(shape) * rng.uniform(0.01, 100)
        x0, _ = O.normalize(m)
        assert np.linalg.norm(x0, 2) <= 1.0 + 1e-14


def test_normalize_zero():
    x0, s = O.normalize(np.zeros((4, 3)))
    assert s == 0.0 and not x0.any()


# ---------------------------------------------------------------- CANS cubic
def _maxerr(c1, c3, a, b, pts=200001):
    x = np.linspace(a, b, pts)
    return np.max(np.abs(1.0 - (c1 * x + c3 * x ** 3)))


def test_cans_degenerate_interval_is_newton_schulz():
    c1, c3, e = O.cans_cubic(1.0, 1.0)
    assert (c1, c3) == pytest.approx((1.5, -0.5), abs=1e-15) and abs(e) < 1e-15


@pytest.mark.parametrize("a,b", [(0.1, 1.0), (0.01, 1.99), (0.5, 1.5), (1e-4, 1.0), (0.9, 1.1)])
def test_cans_equioscillation(a, b):
    c1, c3, e = O.cans_cubic(a, b)
    p = lambda x: c1 * x + c3 * x ** 3
    ex = math.sqrt(-c1 / (3 * c3))          # interior extremum, p'(ex) = 0
    assert a <= ex <= b
    # error alternates +E, -E, +E at a, ex, b
    assert 1 - p(a) == pytest.approx(e, abs=1e-13)
    assert 1 - p(ex) == pytest.approx(-e, abs=1e-13)
    assert 1 - p(b) == pytest.approx(e, abs=1e-13)
    # the max over a dense grid equals E
    assert _maxerr(c1, c3, a, b) == pytest.approx(e, rel=1e-9)


@pytest.mark.parametrize("a,b", [(0.1, 1.0), (0.01, 1.99), (0.6, 1.4)])
def test_cans_cubic_is_minimax_bruteforce(a, b):
    # brute force: no (c1, c3) on a fine neighbourhood grid beats the closed form
    c1, c3, e = O.cans_cubic(a, b)
    best = math.inf
    for d1 in np.linspace(-0.02, 0.02, 41):
        for d3 in np.linspace(-0.02, 0.02, 41):
            if d1 == 0 and d3 == 0:
                continue
            best = min(best, _maxerr(c1 * (1 + d1), c3 * (1 + d3), a, b, 4001))
    assert best >= e * (1 - 1e-9)


def test_cans_small_a_limit():
    _, _, e = O.cans_cubic(1e-12, 1.0)
    assert e == pytest.approx(1.0, abs=1e-10)


def test_cans_golden_values():
    # the minimax cubics solved as a linear program on a dense grid, with no closed form
    # (tests/golden/make_cans_cubic.py), against the oracle's equioscillation closed form
    rows = np.loadtxt(os.path.join(GOLDEN, "cans_cubic.txt"))
    for a, b, c1, c3, e in rows:
        got = O.cans_cubic(a, b)
        assert got == pytest.approx((c1, c3, e), abs=2e-6)


def test_cans_preprocess_maps_into_delta_band():
    for delta in (0.9, 0.99, 0.999):
        t, pre = O.cans_preprocess(delta, 2)
        x = np.geomspace(t, 1.0, 20001)
        for c1, c3 in pre:
            x = c1 * x + c3 * x ** 3
        assert np.min(x) >= 1 - delta - 1e-9 and np.max(x) <= 1 + delta + 1e-9
        assert np.min(x) == pytest.approx(1 - delta, abs=1e-8)   # t is the largest such interval


def test_cans_schedule_intervals_shrink():
    sched = O.cans_schedule(0.99, 2, 30)
    es = [e for _, _, e in sched[2:]]
    assert all(e2 < e1 for e1, e2 in zip(es, es[1:]) if e1 > 1e-15)
    assert es[-1] < 1e-12


# ---------------------------------------------------------------- polar factor
def _polar_2x2_closed(a):
    (p, q), (r, s) = a
    cof = np.array([[s, -r], [-q, p]])
    if np.linalg.det(a) > 0:
        return (a + cof) / math.hypot(p + s, q - r)
    return (a - cof) / math.hypot(p - s, q + r)


@pytest.mark.parametrize("seed", range(6))
def test_polar_2x2_closed_form(seed):
    rng = W.rng_for(100 + seed)
    a = rng.standard_normal((2, 2))
    w, h, _ = O.polar_newton_schulz(a)
    np.testing.assert_allclose(w, _polar_2x2_closed(a), atol=1e-12)
    (p, q), (r, s) = a
    s1 = 0.5 * (math.hypot(p + s, q - r) + math.hypot(p - s, q + r))
    s2 = 0.5 * abs(math.hypot(p + s, q - r) - math.hypot(p - s, q + r))
    sig, _ = O.eigh(h)
    np.testing.assert_allclose(sig, [s1, s2], atol=1e-12)


@pytest.mark.parametrize("m,n,kappa", [(30, 30, 10.0), (40, 25, 1e3), (24, 24, 1e6)])
def test_polar_constructed(m, n, kappa):
    s = W.kappa_spectrum(n, kappa)
    a, q1, q2 = W.constructed(7, m, n, s)
    w, h, _ = O.polar_newton_schulz(a)
    tol = 1e-13 * kappa
    np.testing.assert_allclose(w, q1 @ q2.T, atol=tol)
    np.testing.assert_allclose(h, (q2 * s[None, :]) @ q2.T, atol=1e-13 * kappa)


def test_polar_invariants():
    rng = W.rng_for(3)
    a = rng.standard_normal((12, 8))
    w, h, _ = O.polar_newton_schulz(a)
    np.testing.assert_allclose(w.T @ w, np.eye(8), atol=1e-13)
    np.testing.assert_allclose(w @ h, a, atol=1e-12)
    np.testing.assert_allclose(h, h.T, atol=0)
    assert np.linalg.eigvalsh(h).min() > 0
    # polar(c A) = polar(A), H(cA) = c H(A)
    w2, h2, _ = O.polar_newton_schulz(3.7 * a)
    np.testing.assert_allclose(w2, w, atol=1e-13)
    np.testing.assert_allclose(h2, 3.7 * h, atol=1e-12)
    # polar(Q1 A Q2) = Q1 polar(A) Q2
    q1 = W.orthonormal(rng, 12, 12)
    q2 = W.orthonormal(rng, 8, 8)
    w3, _, _ = O.polar_newton_schulz(q1 @ a @ q2)
    np.testing.assert_allclose(w3, q1 @ w @ q2, atol=1e-12)
    # polar(Q) = Q, H = I
    q = W.orthonormal(rng, 10, 6)
    wq, hq, _ = O.polar_newton_schulz(q)
    np.testing.assert_allclose(wq, q, atol=1e-13)
    np.testing.assert_allclose(hq, np.eye(6), atol=1e-13)


def test_polar_matches_lapack_svd():
    rng = W.rng_for(11)
    a = rng.standard_normal((20, 13))
    u, s, vt = np.linalg.svd(a, full_matrices=False)
    w, h, _ = O.polar_newton_schulz(a)
    np.testing.assert_allclose(w, u @ vt, atol=1e-12)
    np.testing.assert_allclose(h, (vt.T * s) @ vt, atol=1e-12)


def test_polar_cans_route_agrees():
    a, _ = W.kappa_square(4, 32, 1e4)
    w1, h1, _ = O.polar_newton_schulz(a)
    w2, h2, it, res = O.polar_cans(a, tol=1e-13)
    assert res[-1] <= 1e-13
    np.testing.assert_allclose(w2, w1, atol=1e-11)
    np.testing.assert_allclose(h2, h1, atol=1e-11)


# ---------------------------------------------------------------- EVD
@pytest.mark.parametrize("n", [1, 2, 9, 40])
def test_eigh_against_lapack(n):
    rng = W.rng_for(20 + n)
    b = rng.standard_normal((n, n))
    h = b + b.T
    sig, v = O.eigh(h)
    np.testing.assert_allclose(sig, np.sort(np.linalg.eigvalsh(h))[::-1], atol=1e-12)
    np.testing.assert_allclose(h @ v, v * sig[None, :], atol=1e-12)
    np.testing.assert_allclose(v.T @ v, np.eye(n), atol=1e-13)
    idx = np.argmax(np.abs(v), axis=0)
    assert np.all(v[idx, np.arange(n)] > 0)


def test_eigh_repeated_eigenvalues_projectors():
    rng = W.rng_for(31)
    q = W.orthonormal(rng, 12, 12)
    lam = np.array([5, 5, 5, 3, 3, 2, 1, 1, 1, 1, 0.5, 0.1], dtype=float)
    h = (q * lam) @ q.T
    sig, v = O.eigh(h)
    np.testing.assert_allclose(sig, lam, atol=1e-13)
    for val in np.unique(lam):
        sel = np.abs(lam - val) < 1e-9
        p_true = q[:, sel] @ q[:, sel].T
        p_got = v[:, sel] @ v[:, sel].T
        np.testing.assert_allclose(p_got, p_true, atol=1e-12)


# ---------------------------------------------------------------- SVD (Algorithm 1)
@pytest.mark.parametrize("m,n,kappa", [(24, 24, 10.0), (35, 20, 1e4), (16, 16, 1e6)])
def test_svd_constructed_spectrum(m, n, kappa):
    s = W.kappa_spectrum(n, kappa)
    a, q1, q2 = W.constructed(9, m, n, s)
    u, sig, vt, info = O.svd(a)
    assert not info["qr"]
    np.testing.assert_allclose(sig, s, atol=1e-13 * s[0])
    assert O.recon_error(a, u, sig, vt) < 1e-13
    assert O.ortho_error(u) < 1e-13 and O.ortho_error(vt.T) < 1e-13


def test_svd_matches_lapack_and_onesided():
    rng = W.rng_for(41)
    a = rng.standard_normal((30, 18))
    u, sig, vt, _ = O.svd(a)
    s_ref = np.linalg.svd(a, compute_uv=False)
    np.testing.assert_allclose(sig, s_ref, atol=1e-13)
    u2, sig2, vt2 = O.svd_onesided(a)
    np.testing.assert_allclose(sig2, s_ref, atol=1e-13)
    np.testing.assert_allclose(u @ vt, u2 @ vt2, atol=1e-12)          # same polar factor
    np.testing.assert_allclose(vt, vt2, atol=1e-10)                     # same canonical V
    np.testing.assert_allclose(u, u2, atol=1e-10)


def test_svd_two_routes_ill_conditioned():
    s = W.kappa_spectrum(20, 1e6)
    a, q1, q2 = W.constructed(13, 20, 20, s)
    u, sig, vt, _ = O.svd(a)
    u2, sig2, vt2 = O.svd_onesided(a)
    np.testing.assert_allclose(u @ vt, u2 @ vt2, atol=1e-9)
    np.testing.assert_allclose(sig, sig2, atol=1e-13)


def test_qr_nonneg():
    rng = W.rng_for(51)
    u = rng.standard_normal((15, 6))
    q, r = O.qr_nonneg(u)
    assert np.all(np.diag(r) >= 0)
    np.testing.assert_allclose(q @ r, u, atol=1e-13)
    np.testing.assert_allclose(q.T @ q, np.eye(6), atol=1e-13)


def test_svd_rank_deficient_uses_qr():
    # W_r = (U_r 0) V^T limit of Appendix A.2: U = W V has zero columns -> QR fallback
    n, r = 16, 5
    s = W.kappa_spectrum(n, 10.0, rank=r)
    a, q1, q2 = W.constructed(17, 22, n, s)
    w, h, _ = O.polar_newton_schulz(a)
    np.testing.assert_allclose(w, q1[:, :r] @ q2[:, :r].T, atol=1e-8)
    u, sig, vt, info = O.svd(a)
    assert info["qr"]
    np.testing.assert_allclose(sig, s, atol=1e-12)
    assert O.ortho_error(u) < 1e-12
    assert O.recon_error(a, u, sig, vt) < 1e-12
    # the first r columns are unique up to the canonical V sign
    np.testing.assert_allclose(np.abs(u[:, :r].T @ q1[:, :r]), np.eye(r), atol=1e-8)


def test_svd_zero_matrix():
    u, sig, vt, info = O.svd(np.zeros((6, 4)))
    assert not sig.any()
    np.testing.assert_allclose(vt, np.eye(4))
    np.testing.assert_allclose(u, np.eye(6)[:, :4])


def test_gram_evd_fails_sigma_tolerance():
    # Remark 2.1: the Gram-matrix route in FP32 loses sigma accuracy at kappa >= 1e3
    s = W.kappa_spectrum(64, 1e4)
    a, _, _ = W.constructed(19, 64, 64, s)
    a32 = a.astype(np.float32)
    lam = np.linalg.eigvalsh((a32.T @ a32).astype(np.float32))
    sg = np.sqrt(np.clip(np.sort(lam)[::-1].astype(np.float64), 0, None))
    assert np.max(np.abs(sg - s)) > 1e-5 * s[0]
    u, sig, vt, _ = O.svd(a32.astype(np.float64))
    assert np.max(np.abs(sig - s)) < 1e-5 * s[0]


def test_preqr_constructed_tall():
    # the QR preprocessing of rectangular inputs (Section 4.1) on a constructed tall matrix:
    # the spectrum, the polar factor Q1 Q2^T and H = Q2 diag(s) Q2^T are known exactly
    m, n = 40, 12
    s = W.kappa_spectrum(n, 1e3)
    a, q1, q2 = W.constructed(31, m, n, s)
    u, sg, vt, _ = O.svd_preqr(a)
    assert np.abs(sg - s).max() <= 1e-12 * s[0]
    np.testing.assert_allclose(u @ vt, q1 @ q2.T, atol=1e-11)
    w, h = O.polar_preqr(a)
    np.testing.assert_allclose(w, q1 @ q2.T, atol=1e-11)
    np.testing.assert_allclose(h, (q2 * s) @ q2.T, atol=1e-12 * s[0])


def test_preqr_agrees_with_direct_route():
    # the QR route and Algorithm 1 on M itself give the same singular values and the same
    # (unique) polar factor U V^T, and the QR route's factors reconstruct M
    a = W.rng_for(32).standard_normal((50, 20))
    u1, s1, vt1, _ = O.svd(a)
    u2, s2, vt2, _ = O.svd_preqr(a)
    assert np.abs(s1 - s2).max() <= 1e-12 * s1[0]
    np.testing.assert_allclose(u1 @ vt1, u2 @ vt2, atol=1e-12)
    assert O.recon_error(a, u2, s2, vt2) <= 1e-13
    assert O.ortho_error(u2) <= 1e-13 and O.ortho_error(vt2.T) <= 1e-13
