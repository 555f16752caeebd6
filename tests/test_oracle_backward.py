"""Pins for the oracle's backward formulas (CPU only).

Algorithm 4 / Algorithm 3 are checked against: Theorem 3.1's closed-form
consequences, central finite differences through the oracle's own forward
(tiny generic inputs), Townsend's formula (Theorem G.1) on distinct spectra,
Theorem H.1 on exactly repeated spectra for gauge-invariant losses, explicit
factor paths at degenerate points (no SVD differentiated), the eps^(1/4) rate of
Proposition 3.2, Lemma D.1 and Example C.1; Theorem 4.3 (the EVD pseudo-gradient)
against central finite differences."""
import math

import numpy as np
import pytest
from scipy.linalg import expm

import workloads as W
from oracle import psvd_oracle as O


def _rand_skew(rng, n):
    a = rng.standard_normal((n, n))
    return a - a.T


def _factors(seed, m, n, s):
    a, q1, q2 = W.constructed(seed, m, n, s)
    return a, q1, np.asarray(s, float), q2


# ---------------------------------------------------------------- closed forms
def test_thm31_trace_loss_gives_w():
    # l = <I, H> = sum sigma  ->  Abar = W (C = I, X = H^-1 / 2, 2 A X = W)
    rng = W.rng_for(1)
    a = rng.standard_normal((9, 6))
    w, h, _ = O.polar_newton_schulz(a)
    z = np.zeros_like(w)
    np.testing.assert_allclose(O.polar_bwd(a, w, h, z, np.eye(6), eps=0.0), w, atol=1e-12)
    np.testing.assert_allclose(O.polar_bwd_thm31(a, w, h, z, np.eye(6)), w, atol=1e-12)


def test_thm31_frobenius_loss_gives_a():
    # l = 1/2 ||H||_F^2 = 1/2 ||A||_F^2  ->  Abar = A
    rng = W.rng_for(2)
    a = rng.standard_normal((8, 8))
    w, h, _ = O.polar_newton_schulz(a)
    np.testing.assert_allclose(O.polar_bwd(a, w, h, np.zeros_like(w), h, eps=0.0), a, atol=1e-11)


def test_sigma_loss_constant_on_clusters():
    # l = <w, sigma> with w constant on clusters -> Abar = U diag(w) V^T
    s = np.array([3.0, 3.0, 2.0, 1.0, 1.0, 1.0, 0.5])
    a, u, s, v = _factors(3, 10, 7, s)
    wv = np.array([0.3, 0.3, -1.2, 2.0, 2.0, 2.0, 0.7])
    g = O.svd_bwd(a, u, s, v.T, None, wv, None, kreg_mode=2)
    np.testing.assert_allclose(g, (u * wv[None, :]) @ v.T, atol=1e-10)
    # regularized: C = V diag(w) V^T, X = V diag(w_i * 2 s_i / (4 s_i^2 + eps^(1/4))) V^T,
    # 2 M X = U diag(w_i * 4 s_i^2 / (4 s_i^2 + eps^(1/4))) V^T
    eps = 1e-8
    g = O.svd_bwd(a, u, s, v.T, None, wv, None, eps=eps, kreg_mode=0)
    scale = 4 * s ** 2 / (4 * s ** 2 + eps ** 0.25)
    np.testing.assert_allclose(g, (u * (wv * scale)[None, :]) @ v.T, atol=1e-10)


def test_lyapunov_identity_lemma_d1():
    rng = W.rng_for(4)
    q = W.orthonormal(rng, 7, 7)
    lam = rng.uniform(0.2, 3.0, 7)
    h = (q * lam) @ q.T
    a = rng.standard_normal((7, 7))
    b = rng.standard_normal((7, 7))
    y = O.lyapunov_eigenbasis(lam, q, a)
    x = O.lyapunov_eigenbasis(lam, q, b)
    np.testing.assert_allclose(h @ x + x @ h, b, atol=1e-12)
    np.testing.assert_allclose(h @ y + y @ h, a, atol=1e-12)
    assert np.sum(a * x) == pytest.approx(np.sum(y * b), rel=1e-12)


# ---------------------------------------------------------------- finite differences
def _fd(f, a, d, h=1e-6):
    return (f(a + h * d) - f(a - h * d)) / (2 * h)


@pytest.mark.parametrize("m,n", [(4, 4), (7, 4), (6, 6)])
def test_polar_bwd_finite_differences(m, n):
    rng = W.rng_for(10 * m + n)
    a = rng.standard_normal((m, n))
    gw = rng.standard_normal((m, n))
    gh = rng.standard_normal((n, n))

    def loss(x):
        w, h, _ = O.polar_newton_schulz(x)
        return float(np.sum(gw * w) + np.sum(gh * h))

    w, h, _ = O.polar_newton_schulz(a)
    # H is symmetric, so only the symmetric part of its incoming gradient matters
    g = O.polar_bwd(a, w, h, gw, O.sym(gh), eps=0.0)
    g31 = O.polar_bwd_thm31(a, w, h, gw, O.sym(gh))
    np.testing.assert_allclose(g, g31, atol=1e-11)
    for k in range(4):
        d = rng.standard_normal((m, n))
        assert np.sum(g * d) == pytest.approx(_fd(loss, a, d), rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("m,n", [(5, 5), (8, 5), (3, 3)])
def test_svd_bwd_finite_differences(m, n):
    rng = W.rng_for(100 + 10 * m + n)
    a = rng.standard_normal((m, n))
    gu, gs, gv = rng.standard_normal((m, n)), rng.standard_normal(n), rng.standard_normal((n, n))

    def loss(x):
        u, s, vt, _ = O.svd(x)
        return float(np.sum(gu * u) + np.sum(gs * s) + np.sum(gv * vt.T))

    u, s, vt, _ = O.svd(a)
    g = O.svd_bwd(a, u, s, vt, gu, gs, gv.T, kreg_mode=2)
    for k in range(4):
        d = rng.standard_normal((m, n))
        assert np.sum(g * d) == pytest.approx(_fd(loss, a, d), rel=1e-6, abs=1e-8)


# ---------------------------------------------------------------- cross-formula agreement
@pytest.mark.parametrize("m,n", [(9, 9), (14, 9)])
def test_alg4_matches_townsend_distinct(m, n):
    rng = W.rng_for(200 + m)
    s = np.sort(rng.uniform(0.3, 4.0, n))[::-1]
    a, u, s, v = _factors(21, m, n, s)
    gu, gs, gv = rng.standard_normal((m, n)), rng.standard_normal(n), rng.standard_normal((n, n))
    g4 = O.svd_bwd(a, u, s, v.T, gu, gs, gv.T, kreg_mode=2)
    gt = O.svd_bwd_townsend(u, s, v.T, gu, gs, gv.T)
    np.testing.assert_allclose(g4, gt, atol=1e-10 * np.abs(gt).max())


def test_alg3_and_alg4_agree_for_polar_losses():
    # a loss in (W, H) routed through (U, sigma, V) gives Algorithm 3's gradient
    rng = W.rng_for(7)
    m, n = 10, 6
    s = np.sort(rng.uniform(0.5, 2.0, n))[::-1]
    a, u, s, v = _factors(8, m, n, s)
    gw, gh = rng.standard_normal((m, n)), O.sym(rng.standard_normal((n, n)))
    w, h = u @ v.T, (v * s) @ v.T
    ubar = gw @ v
    vbar = gw.T @ u + 2 * gh @ v * s[None, :]
    sbar = np.diag(v.T @ gh @ v)
    g4 = O.svd_bwd(a, u, s, v.T, ubar, sbar, vbar.T, kreg_mode=2)
    g3 = O.polar_bwd(a, w, h, gw, gh, eps=0.0)
    np.testing.assert_allclose(g4, g3, atol=1e-10)


def _cluster_case(seed, n=8):
    s = np.array([2.0, 2.0, 2.0, 1.3, 0.7, 0.7, 0.4, 0.1])[:n]
    return _factors(seed, n, n, s)


def test_alg4_matches_thm_h1_gauge_invariant():
    # on exact clusters the two pseudo-gradients coincide for gauge-invariant losses
    a, u, s, v = _cluster_case(31)
    rng = W.rng_for(32)
    gw, gh = rng.standard_normal((8, 8)), O.sym(rng.standard_normal((8, 8)))
    ubar = gw @ v
    vbar = gw.T @ u + 2 * gh @ v * s[None, :]
    sbar = np.diag(v.T @ gh @ v)
    g4 = O.svd_bwd(a, u, s, v.T, ubar, sbar, vbar.T, kreg_mode=2)
    gh1 = O.svd_bwd_degenerate(u, s, v.T, ubar, sbar, vbar.T)
    np.testing.assert_allclose(g4, gh1, atol=1e-10)


def _path_check(a, u, s, v, omega_u, omega_v, dd, grad, rng):
    gu, gs, gv = rng
    def ell(t):
        uu = u @ expm(t * omega_u)
        vv = v @ expm(t * omega_v)
        return float(np.sum(gu * uu) + np.sum(gs * (s + t * dd)) + np.sum(gv * vv))
    h = 1e-6
    fd = (ell(h) - ell(-h)) / (2 * h)
    mdot = u @ (omega_u @ np.diag(s) + np.diag(dd) - np.diag(s) @ omega_v) @ v.T
    return fd, float(np.sum(grad * mdot))


def test_degenerate_path_alg4_gauge():
    # explicit factor paths M(t) = U e^{t Om_U} (S + t D) (V e^{t Om_V})^T with Om_V's
    # within-cluster blocks zero (V does not rotate inside an eigenspace of H)
    a, u, s, v = _cluster_case(41)
    rng = W.rng_for(42)
    gu, gs, gv = rng.standard_normal((8, 8)), rng.standard_normal(8), rng.standard_normal((8, 8))
    g4 = O.svd_bwd(a, u, s, v.T, gu, gs, gv.T, kreg_mode=2)
    same = np.abs(s[:, None] - s[None, :]) < 1e-12
    for _ in range(4):
        om_u = _rand_skew(rng, 8)
        om_v = _rand_skew(rng, 8)
        om_v[same] = 0.0
        dd = rng.standard_normal(8)
        fd, lin = _path_check(a, u, s, v, om_u, om_v, dd, g4, (gu, gs, gv))
        assert lin == pytest.approx(fd, rel=1e-7, abs=1e-9)


def test_degenerate_path_thm_h1_gauge():
    # Theorem H.1 fixes the common rotation instead: Om_U = -Om_V inside clusters
    a, u, s, v = _cluster_case(51)
    rng = W.rng_for(52)
    gu, gs, gv = rng.standard_normal((8, 8)), rng.standard_normal(8), rng.standard_normal((8, 8))
    gh1 = O.svd_bwd_degenerate(u, s, v.T, gu, gs, gv.T)
    same = np.abs(s[:, None] - s[None, :]) < 1e-12
    for _ in range(4):
        om_u = _rand_skew(rng, 8)
        om_v = _rand_skew(rng, 8)
        om_v[same] = -om_u[same]
        dd = rng.standard_normal(8)
        fd, lin = _path_check(a, u, s, v, om_u, om_v, dd, gh1, (gu, gs, gv))
        assert lin == pytest.approx(fd, rel=1e-7, abs=1e-9)


def test_alg4_and_thm_h1_differ_for_gauge_dependent_loss():
    a, u, s, v = _cluster_case(61)
    rng = W.rng_for(62)
    gu, gs, gv = rng.standard_normal((8, 8)), rng.standard_normal(8), rng.standard_normal((8, 8))
    g4 = O.svd_bwd(a, u, s, v.T, gu, gs, gv.T, kreg_mode=2)
    gh1 = O.svd_bwd_degenerate(u, s, v.T, gu, gs, gv.T)
    assert np.linalg.norm(g4 - gh1) > 1e-3 * np.linalg.norm(g4)


# ---------------------------------------------------------------- regularization
def test_regularization_rate_quarter():
    # Proposition 3.2: ||Abar_eps - Abar_0|| = O(eps^(1/4))
    rng = W.rng_for(71)
    n = 8
    s = np.linspace(3.0, 0.5, n)          # well separated, so the eps^(1/4) term of T dominates
    a, u, s, v = _factors(72, n, n, s)
    gu, gs, gv = rng.standard_normal((n, n)), rng.standard_normal(n), rng.standard_normal((n, n))
    g0 = O.svd_bwd(a, u, s, v.T, gu, gs, gv.T, kreg_mode=2)
    eps = np.array([1e-8, 1e-12, 1e-16, 1e-20, 1e-24])
    gaps = [np.linalg.norm(O.svd_bwd(a, u, s, v.T, gu, gs, gv.T, eps=e, kreg_mode=0) - g0)
            / np.linalg.norm(g0) for e in eps]
    slope = np.polyfit(np.log10(eps), np.log10(gaps), 1)[0]
    assert 0.22 < slope < 0.28
    assert gaps[-1] < 1e-5


def test_example_c1_identity_consistency():
    # at M = I (U = V = I, all sigma equal): a U-only loss and a V-only loss built from
    # the same G agree on every symmetric direction (the only ones keeping U = V);
    # the pseudo-gradient is skew(G) and 0 respectively
    n = 5
    rng = W.rng_for(81)
    g = rng.standard_normal((n, n))
    i = np.eye(n)
    s = np.ones(n)
    gu_only = O.svd_bwd(i, i, s, i, g, None, None, kreg_mode=2)
    gv_only = O.svd_bwd(i, i, s, i, None, None, g.T, kreg_mode=2)
    np.testing.assert_allclose(gu_only, O.skew(g), atol=1e-13)
    np.testing.assert_allclose(gv_only, 0.0, atol=1e-13)
    np.testing.assert_allclose(O.sym(gu_only), O.sym(gv_only), atol=1e-13)


def test_table3_qualitative_gradient_norm():
    # Table 3's shape: the regularized norm equals the analytic one at large gaps and
    # stays bounded at tiny gaps, where the analytic one blows up (exact table values
    # are parity unpinned)
    n = 48
    rng = W.rng_for(91)
    ga, gb, gc = rng.standard_normal((n, n)), rng.standard_normal(n), rng.standard_normal((n, n))
    norms_t, norms_r = [], []
    for gap in (1.0, 1e-1, 1e-6):
        s = W.gap_spectrum(n, gap)
        a, u, s, v = _factors(92, n, n, s)
        norms_t.append(np.linalg.norm(O.svd_bwd_townsend(u, s, v.T, ga, gb, gc.T)))
        norms_r.append(np.linalg.norm(O.svd_bwd(a, u, s, v.T, ga, gb, gc.T, eps=1e-8, kreg_mode=0)))
    assert norms_r[0] == pytest.approx(norms_t[0], rel=1e-3)
    assert norms_t[2] > 100 * norms_t[0]
    assert norms_r[2] < 2 * norms_r[0]


def test_evd_bwd_thm43_finite_differences():
    # Theorem 4.3 on a symmetric matrix with distinct eigenvalues: the directional
    # derivative of <Vbar, V> + <sbar, s> along a symmetric E (central differences through
    # LAPACK's eigh with the oracle's sign convention, locally constant here) equals
    # <Mbar*, E>; Mbar* is symmetric
    rng = W.rng_for(51)
    n = 7
    g = rng.standard_normal((n, n))
    a = (g + g.T) / 2
    vbar = rng.standard_normal((n, n))
    sbar = rng.standard_normal(n)

    def fwd(x):
        w, v = np.linalg.eigh(x)
        order = np.argsort(-w, kind="stable")
        return w[order], O.canonical_signs(v[:, order])

    s, v = fwd(a)
    assert np.min(np.abs(np.diff(s))) > 1e-2
    mbar = O.evd_bwd(v, s, vbar, sbar)
    np.testing.assert_allclose(mbar, mbar.T, atol=1e-13)
    h = 1e-6
    for _ in range(4):
        e = rng.standard_normal((n, n))
        e = (e + e.T) / 2
        sp, vp = fwd(a + h * e)
        sm, vm = fwd(a - h * e)
        fd = (np.sum(vbar * (vp - vm)) + np.sum(sbar * (sp - sm))) / (2 * h)
        assert abs(fd - np.sum(mbar * e)) <= 1e-7 * max(1.0, abs(fd)), (fd, np.sum(mbar * e))
