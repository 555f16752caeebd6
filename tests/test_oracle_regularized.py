"""Pins for the regularized branches of the oracle's backward (CPU only).

Each expected value below is derived by hand from the formulas of Algorithm 4
(complete pipeline), Algorithm 3 / Proposition 3.2 and the K_eps regularizer of
Section 5.2, for inputs where the chain collapses to diagonal or 2 x 2 algebra.
The expressions are written out here term by term; none of them calls the oracle's
mask or R_eps helpers.  Each exponent of eps that the oracle uses -- 1/2 in R_eps,
1/4 in T_eps, 1/2 (Algorithm 4) or 2 (Section 5.2) in K_eps -- moves at least one of
these values, so a swapped exponent fails a test (checked by the planted-mistake
tests at the end, which patch the oracle on the CPU)."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import psvd_oracle as O


def _rotation(theta):
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, -s], [s, c]])


def _phi_diag_ubar(s, g, eps):
    """Algorithm 4 with Ubar = U diag(g), Sbar = 0, Vbar = 0 (derivation).

    Vbar_tot = W^T Ubar = V U^T U diag(g) = V diag(g), so B = (diag(g) - diag(g))/2 = 0 and
    Hbar = 0.  With D = diag(s_i / (s_i^2 + eps^(1/2))), R_eps = V D V^T and
    M^T Wbar = V diag(s_i g_i) V^T, so C = -V diag(d_i^2 s_i g_i) V^T.  T_eps is diagonal on
    the diagonal: t_i = 2 s_i / (4 s_i^2 + eps^(1/4)).  Then X = -V diag(t_i d_i^2 s_i g_i) V^T
    and Mbar = Wbar R_eps + 2 M X = U diag(phi) V^T with
    phi_i = g_i d_i - 2 s_i^2 t_i d_i^2 g_i
          = g_i s_i / (s_i^2 + eps^(1/2)) - 4 s_i^2 / (4 s_i^2 + eps^(1/4)) * g_i s_i^3 / (s_i^2 + eps^(1/2))^2."""
    s = np.asarray(s, float)
    g = np.asarray(g, float)
    r = math.sqrt(eps)
    q = eps ** 0.25
    return g * s / (s * s + r) - (4 * s * s / (4 * s * s + q)) * g * s ** 3 / (s * s + r) ** 2


@pytest.mark.parametrize("eps", [1e-8, 1e-4, 1e-2])
@pytest.mark.parametrize("m,n", [(6, 6), (9, 5)])
def test_svd_bwd_regularized_ubar_diagonal(eps, m, n):
    rng = W.rng_for(700 + m + n)
    s = rng.uniform(0.05, 2.0, n)
    a, u, v = W.constructed(710 + m, m, n, s)
    g = rng.standard_normal(n)
    got = O.svd_bwd(a, u, s, v.T, u * g[None, :], None, None, eps=eps, kreg_mode=0)
    want = (u * _phi_diag_ubar(s, g, eps)[None, :]) @ v.T
    np.testing.assert_allclose(got, want, atol=1e-12 * max(1.0, np.abs(want).max()))
    # K_eps drops out (B = 0): modes 0 and 1 agree on this input
    got1 = O.svd_bwd(a, u, s, v.T, u * g[None, :], None, None, eps=eps, kreg_mode=1)
    np.testing.assert_allclose(got1, want, atol=1e-12 * max(1.0, np.abs(want).max()))


@pytest.mark.parametrize("eps", [1e-8, 1e-4, 1e-2])
def test_polar_bwd_regularized_wbar_diagonal(eps):
    # Algorithm 3 with Wbar = U diag(g) V^T and Hbar = 0 is the same collapse:
    # B = -(H_eps^-1 M^T Wbar H_eps^-1)_sym = -V diag(d_i^2 s_i g_i) V^T, Mbar = U diag(phi) V^T.
    m, n = 8, 5
    rng = W.rng_for(720)
    s = rng.uniform(0.05, 2.0, n)
    a, u, v = W.constructed(721, m, n, s)
    g = rng.standard_normal(n)
    w = u @ v.T
    h = (v * s[None, :]) @ v.T
    got = O.polar_bwd(a, w, h, (u * g[None, :]) @ v.T, np.zeros((n, n)), eps=eps)
    want = (u * _phi_diag_ubar(s, g, eps)[None, :]) @ v.T
    np.testing.assert_allclose(got, want, atol=1e-11 * max(1.0, np.abs(want).max()))


@pytest.mark.parametrize("eps", [1e-8, 1e-4, 1e-2])
def test_polar_bwd_regularized_hbar_diagonal(eps):
    # Algorithm 3 with Wbar = 0 and Hbar = V diag(h) V^T: B = Hbar, X = V diag(t_i h_i) V^T with
    # t_i = 2 s_i / (4 s_i^2 + eps^(1/4)), Mbar = 2 M X = U diag(4 s_i^2 h_i / (4 s_i^2 + eps^(1/4))) V^T.
    m, n = 7, 4
    rng = W.rng_for(730)
    s = rng.uniform(0.05, 2.0, n)
    a, u, v = W.constructed(731, m, n, s)
    hv = rng.standard_normal(n)
    w = u @ v.T
    h = (v * s[None, :]) @ v.T
    got = O.polar_bwd(a, w, h, np.zeros((m, n)), (v * hv[None, :]) @ v.T, eps=eps)
    want = (u * (4 * s * s * hv / (4 * s * s + eps ** 0.25))[None, :]) @ v.T
    np.testing.assert_allclose(got, want, atol=1e-11 * max(1.0, np.abs(want).max()))


def _two_by_two(s1, s2, a_skew, eps, mode, th_u, th_v):
    """Algorithm 4 by hand for M = U diag(s1, s2) V^T (2 x 2, U, V rotations), Ubar = 0,
    Sbar = 0, Vbar = V [[0, a], [-a, 0]].

    W^T Ubar = 0, so Vbar_tot = Vbar, V^T Vbar_tot = Omega = [[0, a], [-a, 0]] and B = Omega.
    K_12 = d / (d^2 + reg) with d = s1 - s2 (reg = eps^(1/2) in mode 0, eps^2 in mode 1;
    mode 2: K_12 = 1/d); K_21 = -K_12.  (K^T o B)_12 = K_21 B_12 = -K_12 a and
    (K^T o B)_21 = K_12 B_21 = -K_12 a, so V^T Hbar V = [[0, -K_12 a], [-K_12 a, 0]].
    Wbar = 0, so V^T C V = V^T Hbar V.  T_12 = (s1 + s2) / ((s1 + s2)^2 + eps^(1/4)) (mode 2:
    1 / (s1 + s2)), x = -T_12 K_12 a, V^T X V = [[0, x], [x, 0]].
    Mbar = 2 M X = U [[0, 2 s1 x], [2 s2 x, 0]] V^T."""
    d = s1 - s2
    if mode == 0:
        k12 = d / (d * d + math.sqrt(eps))
    elif mode == 1:
        k12 = d / (d * d + eps * eps)
    else:
        k12 = 1.0 / d
    ssum = s1 + s2
    t12 = 1.0 / ssum if mode == 2 else ssum / (ssum * ssum + eps ** 0.25)
    x = -t12 * k12 * a_skew
    core = np.array([[0.0, 2 * s1 * x], [2 * s2 * x, 0.0]])
    u = _rotation(th_u)
    v = _rotation(th_v)
    return u @ core @ v.T, u, v


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("s1,s2,eps", [(1.01, 1.0, 1e-4), (1.1, 1.0, 1e-4), (0.7, 0.3, 1e-2), (2.0, 1.999, 1e-8)])
def test_svd_bwd_kreg_two_by_two(mode, s1, s2, eps):
    a_skew = 0.37
    th_u, th_v = 0.61, -1.27
    want, u, v = _two_by_two(s1, s2, a_skew, eps, mode, th_u, th_v)
    s = np.array([s1, s2])
    m = (u * s[None, :]) @ v.T
    vbar = v @ np.array([[0.0, a_skew], [-a_skew, 0.0]])
    got = O.svd_bwd(m, u, s, v.T, None, None, vbar.T, eps=eps, kreg_mode=mode)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-13 * max(1.0, np.abs(want).max()))


def test_kreg_modes_are_distinguished():
    # on (s1, s2) = (1.01, 1.0), eps = 1e-4 the three modes give clearly different values
    vals = [_two_by_two(1.01, 1.0, 0.37, 1e-4, md, 0.0, 0.0)[0][0, 1] for md in (0, 1, 2)]
    assert abs(vals[0] - vals[1]) > 0.5 * abs(vals[1])
    assert abs(vals[1] - vals[2]) > 1e-3 * abs(vals[2])


# ---------------------------------------------------------------- planted mistakes
# Each case patches one eps exponent of the oracle (on the CPU, for this test only)
# and checks that the pins above catch it.
_ORIG_R, _ORIG_T, _ORIG_K = O._r_mat, O._t_mask, O._k_mask


def _patched_r(s, v, eps):
    if eps == 0.0:
        return _ORIG_R(s, v, eps)
    d = s / (s * s + eps)                      # eps instead of eps^(1/2)
    return (v * d[None, :]) @ v.T


def _patched_t(s, eps):
    if eps == 0.0:
        return _ORIG_T(s, eps)
    ssum = s[:, None] + s[None, :]
    return ssum / (ssum * ssum + math.sqrt(eps))   # eps^(1/2) instead of eps^(1/4)


def _patched_k(s, eps, kreg_mode, tie_tol):
    d = s[:, None] - s[None, :]
    if kreg_mode == 0:
        return d / (d * d + eps ** 0.25)       # eps^(1/4) instead of eps^(1/2)
    if kreg_mode == 1:
        return d / (d * d + eps)               # eps instead of eps^2
    return _ORIG_K(s, eps, kreg_mode, tie_tol)


@pytest.mark.parametrize("which", ["r", "t", "k0", "k1"])
def test_pins_catch_swapped_exponents(monkeypatch, which):
    patch = {"r": ("_r_mat", _patched_r), "t": ("_t_mask", _patched_t),
             "k0": ("_k_mask", _patched_k), "k1": ("_k_mask", _patched_k)}[which]
    monkeypatch.setattr(O, *patch)
    with pytest.raises(AssertionError):
        if which in ("r", "t"):
            test_svd_bwd_regularized_ubar_diagonal(1e-4, 6, 6)
            test_polar_bwd_regularized_wbar_diagonal(1e-4)
        else:
            test_svd_bwd_kreg_two_by_two(0 if which == "k0" else 1, 1.01, 1.0, 1e-4)


# ---------------------------------------------------------------- EVD backward (Theorem 4.3 with K_eps)
def _evd_two_by_two(s1, s2, a_skew, sb1, sb2, eps, mode, th):
    """Theorem 4.3 by hand for H = V diag(s1, s2) V^T (V a rotation), Vbar = V Omega with
    Omega = [[0, a], [-a, 0]], Sbar = diag(sb1, sb2).

    V^T Vbar = Omega and V^T Vbar - Vbar^T V = 2 Omega, so S = K^T o Omega:
    S_12 = K_21 a = -K_12 a and S_21 = K_12 (-a) = -K_12 a, with K_12 = d / (d^2 + reg),
    d = s1 - s2 (reg = eps^(1/2) in mode 0, eps^2 in mode 1; mode 2: 1/d).
    Hbar = V [[sb1, -K_12 a], [-K_12 a, sb2]] V^T."""
    d = s1 - s2
    k12 = d / (d * d + math.sqrt(eps)) if mode == 0 else (d / (d * d + eps * eps) if mode == 1 else 1.0 / d)
    core = np.array([[sb1, -k12 * a_skew], [-k12 * a_skew, sb2]])
    v = _rotation(th)
    return v @ core @ v.T, v


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("s1,s2,eps", [(1.01, 1.0, 1e-4), (3.0, 0.5, 1.0), (2.0, 1.999, 1e-8), (1.2, 1.0, 10.0)])
def test_evd_bwd_kreg_two_by_two(mode, s1, s2, eps):
    want, v = _evd_two_by_two(s1, s2, 0.53, 0.7, -1.3, eps, mode, 0.83)
    vbar = v @ np.array([[0.0, 0.53], [-0.53, 0.0]])
    got = O.evd_bwd(v, np.array([s1, s2]), vbar, np.array([0.7, -1.3]), eps=eps, kreg_mode=mode)
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14 * max(1.0, np.abs(want).max()))


def test_evd_bwd_regularized_tends_to_thm43():
    # K_eps -> K as eps -> 0 on a distinct spectrum (the limit stated after Theorem 4.3)
    rng = W.rng_for(740)
    n = 6
    v = W.orthonormal(rng, n, n)
    s = np.sort(rng.uniform(0.5, 3.0, n))[::-1]
    vbar, sbar = rng.standard_normal((n, n)), rng.standard_normal(n)
    exact = O.evd_bwd(v, s, vbar, sbar)
    for mode in (0, 1):
        gaps = []
        for eps in (1e-2, 1e-4, 1e-8, 1e-12, 1e-16):
            gaps.append(np.linalg.norm(O.evd_bwd(v, s, vbar, sbar, eps=eps, kreg_mode=mode) - exact))
        ref = np.linalg.norm(exact)
        assert all(b < a or b < 1e-14 * ref for a, b in zip(gaps, gaps[1:]))
        assert gaps[-1] < 1e-5 * ref
