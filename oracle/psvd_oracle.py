"""FP64 CPU oracle for the SVD-via-polar-decomposition pipeline and its backward.

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by ``bench.py``'s CPU-baseline leg; the product
path (``paper_2609_32505_gb300``) never imports, links or calls it, and this
module imports nothing from the product path.  Everything is plain FP64 numpy
(matrix products and a LAPACK QR used as library steps) plus the Jacobi routines
in ``jacobi.c`` (loaded through ctypes).

What each function computes, with the passage it follows:

* ``normalize``            Algorithm 2 (Appendix A.1): X0 = M / sqrt(||M||_1 ||M||_inf).
* ``cans_cubic``           optimal odd cubic p(x) = c1 x + c3 x^3 on [a, b] (the degree-3
                           CANS polynomial, Appendix A.4 / B.8), derived here from
                           Chebyshev equioscillation at a, e, b with p'(e) = 0.
* ``cans_preprocess``      the preprocessing of Appendix B.8: the largest [t, 1] that two
                           greedy optimal cubics map into [1 - delta, 1 + delta].
* ``cans_schedule``        preprocessing + main CANS iteration from [1 - delta, 1 + delta].
* ``polar_newton_schulz``  the unique polar factor of Definition 2.1 by the classical
                           Newton-Schulz iteration X <- X (3 I - X^T X) / 2 (Section 3,
                           Appendix A.1), run to FP64 convergence.
* ``polar_cans``           the same limit by the CANS schedule (the iteration of Algorithm 1).
* ``eigh``                 cyclic Jacobi EVD (the EVD of Algorithm 1), sigma descending,
                           each eigenvector's largest-magnitude entry made positive.
* ``qr_nonneg``            QR with non-negative diag(R) (Appendix A.2).
* ``svd``                  Algorithm 1 end to end with the FP64 pieces above.
* ``svd_onesided``         an independent SVD route (Hestenes one-sided Jacobi).
* ``svd_preqr`` / ``polar_preqr``  the QR preprocessing of rectangular inputs (Section 4.1,
                           rectangular matrices): M = Q R (thin), the SVD or polar
                           decomposition of the n x n factor R, then U = Q U_R, W = Q W_R,
                           H = H_R.
* ``polar_bwd``            Algorithm 3 / Proposition 3.2 (regularized), Theorem 3.1 (eps=0).
* ``evd_bwd``              Theorem 4.3 (EVD pseudo-gradient), and its K_eps regularization
                           (Section 5.2).
* ``svd_bwd``              Algorithm 4 (complete pipeline), kreg modes 0/1/2.
* ``svd_bwd_townsend``     Theorem G.1 (distinct spectra, thin, m >= n).
* ``svd_bwd_degenerate``   Theorem H.1 (square, repeated singular values allowed).
* ``lyapunov_eigenbasis``  Proposition D.3.
* ``sketch_features`` / ``mlp_*``  the learned lower-bound predictor's features and
                           a plain FP64 MLP (8 -> 64 -> 64 -> 1) forward/backward.

Readings taken where the paper is silent or garbled:
the closed-form CANS cubic and the bisection reading of the preprocessing;
stopping residual ||X^T X - I||_F / sqrt(n); skew(X) = (X - X^T)/2; the sign of the
(I - U U^T) Ubar S^-1 V^T term is '+' (Theorem G.1); eigenvector sign convention;
the K_eps regularizer uses eps^(1/2) as printed in Algorithm 4 (kreg_mode 0) with
the main text's eps^2 as kreg_mode 1 and the exact eps = 0 mask as kreg_mode 2.

Parity status: every function above is pinned by tests under ``tests/`` against
closed forms, invariants, library routines or finite differences (the regularized
branches -- R_eps's eps^(1/2), T_eps's eps^(1/4), K_eps's eps^(1/2) / eps^2 and
``polar_bwd`` at eps > 0 -- by hand-derived diagonal and 2 x 2 closed forms of
Algorithm 4 / Algorithm 3 in ``tests/test_oracle_regularized.py``), except the
exact numbers of Table 3 (parity unpinned: the table matches neither smooth
regularizer exactly; only its qualitative shape is tested) and the CANS
iteration counts (parity unpinned: the paper prints none).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def build_c(force: bool = False) -> str:
    """Compile jacobi.c into a shared object next to it (gcc, -O2, portable flags)."""
    src = os.path.join(_HERE, "jacobi.c")
    so = os.path.join(_HERE, "_jacobi.so")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(build_c())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_eigh_jacobi.argtypes = [ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_int]
        lib.oracle_eigh_jacobi.restype = ctypes.c_int
        lib.oracle_svd_onesided.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_double, ctypes.c_int]
        lib.oracle_svd_onesided.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def sym(a: np.ndarray) -> np.ndarray:
    """A_sym = (A + A^T) / 2 (Section 2.1 notation)."""
    return 0.5 * (a + a.T)


def skew(a: np.ndarray) -> np.ndarray:
    """skew(A) = (A - A^T) / 2 (reading of Theorem H.1's undefined skew)."""
    return 0.5 * (a - a.T)


# ---------------------------------------------------------------------------
# Forward: normalization, CANS coefficients, polar factor
# ---------------------------------------------------------------------------

def normalize(m: np.ndarray):
    """Algorithm 2: a = ||M||_1 ||M||_inf (max column / max row l1 norm), X0 = M / sqrt(a).

    Returns (X0, s) with s = sqrt(a); a zero matrix gives (0, 0)."""
    m = np.asarray(m, dtype=np.float64)
    n1 = np.abs(m).sum(axis=0).max() if m.size else 0.0
    ninf = np.abs(m).sum(axis=1).max() if m.size else 0.0
    s = math.sqrt(n1 * ninf)
    if s == 0.0:
        return np.zeros_like(m), 0.0
    return m / s, s


def cans_cubic(a: float, b: float):
    """Optimal odd cubic p(x) = c1 x + c3 x^3 minimizing max_{[a,b]} |1 - p(x)|.

    Equioscillation at a, e, b with p'(e) = 0 and p(a) = p(b) gives
    s = a^2 + ab + b^2, e = sqrt(s/3), c3 = -c1/s,
    c1 = 2 / ((2/3) e + ab(a+b)/s), E = (2/3) c1 e - 1; p maps [a,b] onto [1-E, 1+E].
    Returns (c1, c3, E)."""
    a = float(a)
    b = float(b)
    s = a * a + a * b + b * b
    e = math.sqrt(s / 3.0)
    c1 = 2.0 / ((2.0 / 3.0) * e + a * b * (a + b) / s)
    c3 = -c1 / s
    big_e = (2.0 / 3.0) * c1 * e - 1.0
    return c1, c3, big_e


def _greedy(a: float, b: float, steps: int):
    coeffs = []
    for _ in range(steps):
        c1, c3, e = cans_cubic(a, b)
        coeffs.append((c1, c3))
        a, b = 1.0 - e, 1.0 + e
    return coeffs, a, b


def cans_preprocess(delta: float = 0.99, steps: int = 2):
    """Largest [t, 1] whose image under ``steps`` greedy optimal cubics lies in
    [1 - delta, 1 + delta] (Appendix B.8, read as a bisection on t).
    Returns (t, [(c1, c3), ...])."""
    if steps == 0:
        return 1.0 - delta, []
    lo, hi = 1e-300, 1.0
    for _ in range(200):   # bisection on log t: E after `steps` steps decreases in t
        mid = math.sqrt(lo * hi) if lo > 0 else 0.5 * hi
        _, a, b = _greedy(mid, 1.0, steps)
        if 1.0 - a <= delta:
            hi = mid
        else:
            lo = mid
    t = hi
    coeffs, _, _ = _greedy(t, 1.0, steps)
    return t, coeffs


def cans_schedule(delta: float = 0.99, pre_steps: int = 2, max_iter: int = 50, lower: float | None = None):
    """Coefficient list of the conservative CANS schedule: ``pre_steps`` preprocessing
    cubics for [t, 1], then greedy optimal cubics starting from [1 - delta, 1 + delta].
    With ``lower`` given, the schedule instead starts from [lower, 1] (greedy, no
    preprocessing) -- the form the learned lower bound plugs into.
    Returns a list of (c1, c3, E_after) triples, ``max_iter`` main steps long."""
    out = []
    if lower is None:
        t, pre = cans_preprocess(delta, pre_steps)
        a, b = t, 1.0
        for c1, c3 in pre:
            _, _, e = cans_cubic(a, b)
            out.append((c1, c3, e))
            a, b = 1.0 - e, 1.0 + e
        a, b = 1.0 - delta, 1.0 + delta
    else:
        a, b = float(lower), 1.0
    for _ in range(max_iter):
        c1, c3, e = cans_cubic(a, b)
        out.append((c1, c3, e))
        a, b = 1.0 - e, 1.0 + e
    return out


def ortho_residual(x: np.ndarray) -> float:
    """||X^T X - I||_F / sqrt(n) (the relative orthogonality measure of Section 4.1)."""
    n = x.shape[1]
    g = x.T @ x
    return float(np.linalg.norm(g - np.eye(n)) / math.sqrt(n))


def polar_newton_schulz(m: np.ndarray, tol: float = 1e-14, max_iter: int = 300):
    """Polar factor W (Definition 2.1) by X <- 1.5 X - 0.5 X X^T X from X0 of Algorithm 2.

    Stops when ||X^T X - I||_F/sqrt(n) <= tol; or when the residual has stagnated
    (changes by <= 1e-14) while a step moves X by <= 1e-10 ||X||_F, which is the
    rank-deficient limit W_r = (U_r 0) V^T of Appendix A.2 (continuing would only
    amplify rounding noise in the null space by 3/2 per step); or at max_iter.
    Returns (W, H, iters) with H = (W^T M)_sym."""
    m = np.asarray(m, dtype=np.float64)
    x, s = normalize(m)
    n = m.shape[1]
    it = 0
    r_prev = math.inf
    for it in range(1, max_iter + 1):
        g = x.T @ x
        r = np.linalg.norm(g - np.eye(n)) / math.sqrt(n)
        if r <= tol:
            it -= 1
            break
        x_new = x @ (1.5 * np.eye(n) - 0.5 * g)
        change = np.linalg.norm(x_new - x)
        if abs(r_prev - r) <= 1e-14 and change <= 1e-10 * max(np.linalg.norm(x), 1e-300):
            it -= 1
            break
        x = x_new
        r_prev = r
    h = sym(x.T @ m)
    return x, h, it


def polar_cans(m: np.ndarray, schedule=None, tol: float = 1e-14, max_iter: int = 60):
    """Polar factor by the CANS coefficients (Algorithm 1, steps 1-3), continued with
    Newton-Schulz steps once the schedule is exhausted.  Returns (W, H, iters, residuals)."""
    m = np.asarray(m, dtype=np.float64)
    x, _ = normalize(m)
    n = m.shape[1]
    sched = cans_schedule() if schedule is None else schedule
    res = []
    for k in range(max_iter):
        g = x.T @ x
        r = float(np.linalg.norm(g - np.eye(n)) / math.sqrt(n))
        res.append(r)
        if r <= tol:
            break
        c1, c3 = (sched[k][0], sched[k][1]) if k < len(sched) else (1.5, -0.5)
        x = x @ (c1 * np.eye(n) + c3 * g)
    h = sym(x.T @ m)
    return x, h, len(res) - 1, res


# ---------------------------------------------------------------------------
# EVD, QR, SVD
# ---------------------------------------------------------------------------

def canonical_signs(v: np.ndarray) -> np.ndarray:
    """Flip each column so that its largest-|.| entry (lowest index on ties) is positive."""
    v = v.copy()
    idx = np.argmax(np.abs(v), axis=0)
    sgn = np.sign(v[idx, np.arange(v.shape[1])])
    sgn[sgn == 0] = 1.0
    return v * sgn[None, :]


def eigh(h: np.ndarray, rel_tol: float = 1e-15, max_sweeps: int = 100):
    """Cyclic Jacobi EVD of symmetric h (FP64): returns (sigma descending, V)."""
    h = np.asarray(h, dtype=np.float64)
    n = h.shape[0]
    a = np.ascontiguousarray(sym(h))
    v = np.zeros((n, n))
    sweeps = _lib().oracle_eigh_jacobi(n, _ptr(a), _ptr(v), rel_tol, max_sweeps)
    if sweeps < 0:
        raise RuntimeError("Jacobi EVD did not converge")
    w = np.diag(a).copy()
    order = np.argsort(-w, kind="stable")
    return w[order], canonical_signs(v[:, order])


def qr_nonneg(u: np.ndarray):
    """Householder QR (LAPACK) with the signs fixed so that diag(R) >= 0 (Appendix A.2)."""
    q, r = np.linalg.qr(np.asarray(u, dtype=np.float64), mode="reduced")
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d[None, :], r * d[:, None]


def svd(m: np.ndarray, eps_qr: float = 1e-10, polar: str = "ns"):
    """Algorithm 1 in FP64: normalize, polar factor W, H = (W^T M)_sym, EVD H = V S V^T,
    U = W V, then QR of U (diag R >= 0) if any column norm is off 1 by more than eps_qr.
    Returns (U, sigma, V^T, info) with info = dict(qr=bool, iters=int)."""
    m = np.asarray(m, dtype=np.float64)
    if polar == "ns":
        w, h, it = polar_newton_schulz(m)
    else:
        w, h, it, _ = polar_cans(m)
    sigma, v = eigh(h)
    u = w @ v
    norms = np.linalg.norm(u, axis=0)
    used_qr = bool(np.any(np.abs(norms - 1.0) > eps_qr))
    if used_qr:
        u, _ = qr_nonneg(u)
    return u, sigma, v.T, {"qr": used_qr, "iters": it}


def svd_preqr(m: np.ndarray, eps_qr: float = 1e-10, polar: str = "ns"):
    """SVD of a rectangular M (m >= n) through its thin QR (Section 4.1, rectangular
    matrices): M = Q R, R = U_R S V^T by Algorithm 1, U = Q U_R.  Returns (U, sigma, V^T,
    info) like ``svd``."""
    m = np.asarray(m, dtype=np.float64)
    q, r = qr_nonneg(m)
    u_r, sigma, vt, info = svd(r, eps_qr=eps_qr, polar=polar)
    return q @ u_r, sigma, vt, info


def polar_preqr(m: np.ndarray):
    """Polar decomposition of a rectangular M (m >= n) through its thin QR: with M = Q R and
    R = W_R H_R, the factor Q W_R has orthonormal columns and (Q W_R) H_R = M, so it is the
    polar factor of M (unique for full rank, Definition 2.1) and H_R is H.  Returns (W, H)."""
    m = np.asarray(m, dtype=np.float64)
    q, r = qr_nonneg(m)
    w_r, h_r, _ = polar_newton_schulz(r)
    return q @ w_r, h_r


def svd_onesided(m: np.ndarray, tol: float = 1e-15, max_sweeps: int = 100):
    """Hestenes one-sided Jacobi SVD (independent of the polar route).
    Returns (U, sigma descending, V^T) for full-rank m x n, m >= n."""
    m = np.asarray(m, dtype=np.float64)
    mm, n = m.shape
    at = np.ascontiguousarray(m.T)
    vt = np.zeros((n, n))
    if _lib().oracle_svd_onesided(mm, n, _ptr(at), _ptr(vt), tol, max_sweeps) < 0:
        raise RuntimeError("one-sided Jacobi did not converge")
    sig = np.linalg.norm(at, axis=1)
    order = np.argsort(-sig, kind="stable")
    sig = sig[order]
    u = (at[order] / np.where(sig > 0, sig, 1.0)[:, None]).T
    v = vt[order].T
    v = canonical_signs(v)
    # keep U consistent with the sign-fixed V
    flip = np.sign(np.sum(v * vt[order].T, axis=0))
    u = u * flip[None, :]
    return u, sig, v.T


# ---------------------------------------------------------------------------
# Backward
# ---------------------------------------------------------------------------

def lyapunov_eigenbasis(sigma: np.ndarray, q: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Proposition D.3: the solution of H X + X H = C for H = Q diag(sigma) Q^T, sigma > 0."""
    s = np.asarray(sigma, dtype=np.float64)
    return q @ ((q.T @ c @ q) / (s[:, None] + s[None, :])) @ q.T


def _t_mask(s: np.ndarray, eps: float) -> np.ndarray:
    ssum = s[:, None] + s[None, :]
    if eps == 0.0:
        out = np.zeros_like(ssum)
        nz = ssum > 0
        out[nz] = 1.0 / ssum[nz]
        return out
    return ssum / (ssum * ssum + eps ** 0.25)


def _k_mask(s: np.ndarray, eps: float, kreg_mode: int, tie_tol: float) -> np.ndarray:
    d = s[:, None] - s[None, :]          # d_ij = sigma_i - sigma_j
    if kreg_mode == 0:
        return d / (d * d + math.sqrt(eps))
    if kreg_mode == 1:
        return d / (d * d + eps * eps)
    if kreg_mode == 2:
        smax = float(np.max(np.abs(s))) if s.size else 0.0
        tie = np.abs(d) <= tie_tol * smax
        out = np.zeros_like(d)
        out[~tie] = 1.0 / d[~tie]
        return out
    raise ValueError("kreg_mode must be 0, 1 or 2")


def _r_mat(s: np.ndarray, v: np.ndarray, eps: float) -> np.ndarray:
    """R_eps = V Sigma (Sigma^2 + eps^(1/2) I)^(-1) V^T; eps = 0 gives the pseudo-inverse H^+."""
    if eps == 0.0:
        d = np.zeros_like(s)
        nz = s > 0
        d[nz] = 1.0 / s[nz]
    else:
        d = s / (s * s + math.sqrt(eps))
    return (v * d[None, :]) @ v.T


def polar_bwd(m, w, h, wbar, hbar, eps: float = 1e-8):
    """Algorithm 3 (Proposition 3.2); eps = 0 gives Theorem 3.1 exactly.

    EVD of H, H_eps^-1 = V Sigma (Sigma^2 + eps^(1/2))^-1 V^T,
    B = (Hbar - H_eps^-1 M^T Wbar H_eps^-1)_sym,
    Xt_ij = (s_i + s_j) / ((s_i + s_j)^2 + eps^(1/4)) (V^T B V)_ij, X = V Xt V^T,
    Mbar = Wbar H_eps^-1 + 2 M X."""
    m = np.asarray(m, dtype=np.float64)
    s, v = eigh(h)
    r = _r_mat(s, v, eps)
    b = sym(hbar - r @ m.T @ wbar @ r)
    xt = _t_mask(s, eps) * (v.T @ b @ v)
    x = v @ xt @ v.T
    return wbar @ r + 2.0 * m @ x


def polar_bwd_thm31(m, w, h, wbar, hbar):
    """Theorem 3.1 as printed: C = (Hbar - W^T Wbar H^-1)_sym, X = V (T o V^T C V) V^T,
    Mbar = Wbar H^-1 + 2 M X (full-rank M)."""
    s, v = eigh(h)
    hinv = (v / s[None, :]) @ v.T
    c = sym(hbar - w.T @ wbar @ hinv)
    x = v @ (_t_mask(s, 0.0) * (v.T @ c @ v)) @ v.T
    return wbar @ hinv + 2.0 * np.asarray(m, dtype=np.float64) @ x


def evd_bwd(v, sigma, vbar, sigmabar, tie_tol: float = 0.0, eps: float = 0.0, kreg_mode: int = 2):
    """Theorem 4.3: K_ij = 1/(s_i - s_j) (0 on equal values), S = 1/2 K^T o (V^T Vbar - Vbar^T V),
    Mbar_star = V (S + diag(sigmabar)) V^T.

    With kreg_mode 0 or 1, K is replaced by its Tikhonov regularization K_eps (Section 5.2,
    the paragraph after Theorem 4.3): (s_i - s_j) / ((s_i - s_j)^2 + reg) with reg = eps^(1/2)
    (the form Algorithm 4 prints, mode 0) or eps^2 (the form Section 5.2 prints, mode 1).
    ``vbar`` or ``sigmabar`` may be None (zero)."""
    v = np.asarray(v, dtype=np.float64)
    s = np.asarray(sigma, dtype=np.float64)
    n = s.shape[0]
    vbar = np.zeros((n, n)) if vbar is None else np.asarray(vbar, dtype=np.float64)
    sbar = np.zeros(n) if sigmabar is None else np.asarray(sigmabar, dtype=np.float64)
    k = _k_mask(s, eps, kreg_mode, tie_tol)
    smat = 0.5 * k.T * (v.T @ vbar - vbar.T @ v)
    return v @ (smat + np.diag(sbar)) @ v.T


def svd_bwd(m, u, sigma, vt, ubar, sigmabar, vtbar, eps: float = 1e-8,
            kreg_mode: int = 0, tie_tol: float = 1e-10):
    """Algorithm 4, backward pass, in the order printed:

    W = U V^T; Wbar = Ubar V^T; Vbar_tot = Vbar + W^T Ubar;
    B = (V^T Vbar_tot - Vbar_tot^T V) / 2;
    (K_eps)_ij = (s_i - s_j) / ((s_i - s_j)^2 + reg)  [reg: eps^(1/2) mode 0, eps^2 mode 1,
                                                      exact 1/(s_i - s_j) with ties masked mode 2];
    Hbar = V (diag(sigmabar) + K_eps^T o B) V^T;
    R_eps = V Sigma (Sigma^2 + eps^(1/2))^-1 V^T;  C = (Hbar - R_eps M^T Wbar R_eps)_sym;
    (T_eps)_ij = (s_i + s_j) / ((s_i + s_j)^2 + eps^(1/4));  X = V (T_eps o V^T C V) V^T;
    Mbar = Wbar R_eps + 2 M X.
    ``vtbar`` is the gradient of V^T (transposed to Vbar as the appendix states).
    Mode 2 uses eps = 0 in R and T (the unregularized limit)."""
    m = np.asarray(m, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    s = np.asarray(sigma, dtype=np.float64)
    v = np.asarray(vt, dtype=np.float64).T
    n = v.shape[0]
    ubar = np.zeros_like(u) if ubar is None else np.asarray(ubar, dtype=np.float64)
    sbar = np.zeros(n) if sigmabar is None else np.asarray(sigmabar, dtype=np.float64)
    vbar = np.zeros((n, n)) if vtbar is None else np.asarray(vtbar, dtype=np.float64).T
    e = 0.0 if kreg_mode == 2 else eps
    w = u @ v.T
    wbar = ubar @ v.T
    vbar_tot = vbar + w.T @ ubar
    b = 0.5 * (v.T @ vbar_tot - vbar_tot.T @ v)
    k = _k_mask(s, eps, kreg_mode, tie_tol)
    hbar = v @ (np.diag(sbar) + k.T * b) @ v.T
    r = _r_mat(s, v, e)
    c = sym(hbar - r @ m.T @ wbar @ r)
    x = v @ (_t_mask(s, e) * (v.T @ c @ v)) @ v.T
    return wbar @ r + 2.0 * m @ x


def svd_bwd_townsend(u, sigma, vt, ubar, sigmabar, vtbar):
    """Theorem G.1 with k = n (thin SVD, distinct positive singular values, m >= n):
    Abar = [U (F o (U^T Ubar - Ubar^T U)) S + (I - U U^T) Ubar S^-1] V^T + U diag(sbar) V^T
           + U [S (F o (V^T Vbar - Vbar^T V)) V^T + S^-1 Vbar^T (I - V V^T)],
    F_ij = 1/(s_j^2 - s_i^2), F_ii = 0."""
    u = np.asarray(u, dtype=np.float64)
    s = np.asarray(sigma, dtype=np.float64)
    v = np.asarray(vt, dtype=np.float64).T
    mm, n = u.shape
    ubar = np.zeros_like(u) if ubar is None else np.asarray(ubar, dtype=np.float64)
    sbar = np.zeros(n) if sigmabar is None else np.asarray(sigmabar, dtype=np.float64)
    vbar = np.zeros((n, n)) if vtbar is None else np.asarray(vtbar, dtype=np.float64).T
    d = s[None, :] ** 2 - s[:, None] ** 2
    f = np.zeros_like(d)
    off = ~np.eye(n, dtype=bool)
    f[off] = 1.0 / d[off]
    smat = np.diag(s)
    sinv = np.diag(1.0 / s)
    term1 = (u @ (f * (u.T @ ubar - ubar.T @ u)) @ smat + (np.eye(mm) - u @ u.T) @ ubar @ sinv) @ v.T
    term2 = u @ np.diag(sbar) @ v.T
    term3 = u @ (smat @ (f * (v.T @ vbar - vbar.T @ v)) @ v.T + sinv @ vbar.T @ (np.eye(n) - v @ v.T))
    return term1 + term2 + term3


def svd_bwd_degenerate(u, sigma, vt, ubar, sigmabar, vtbar, tie_tol: float = 1e-10):
    """Theorem H.1 (square M, repeated singular values allowed):
    A = U^T Ubar, B = V^T Vbar, F_ij = 1/(s_j^2 - s_i^2) off ties (else 0),
    G_ij = 1/(2 s_i) on ties with s_i > 0 (else 0),
    Mbar = U [F o ((A - A^T) S + S (B - B^T)) + diag(sbar) + G o skew(A - B)] V^T."""
    u = np.asarray(u, dtype=np.float64)
    s = np.asarray(sigma, dtype=np.float64)
    v = np.asarray(vt, dtype=np.float64).T
    n = v.shape[0]
    ubar = np.zeros_like(u) if ubar is None else np.asarray(ubar, dtype=np.float64)
    sbar = np.zeros(n) if sigmabar is None else np.asarray(sigmabar, dtype=np.float64)
    vbar = np.zeros((n, n)) if vtbar is None else np.asarray(vtbar, dtype=np.float64).T
    smax = float(np.max(np.abs(s)))
    tie = np.abs(s[:, None] - s[None, :]) <= tie_tol * smax
    d = s[None, :] ** 2 - s[:, None] ** 2
    f = np.zeros_like(d)
    f[~tie] = 1.0 / d[~tie]
    g = np.zeros_like(d)
    pos = tie & (s[:, None] > 0)
    g[pos] = (1.0 / (2.0 * s[:, None] * np.ones((1, n))))[pos]
    a = u.T @ ubar
    b = v.T @ vbar
    smat = np.diag(s)
    core = f * ((a - a.T) @ smat + smat @ (b - b.T)) + np.diag(sbar) + g * skew(a - b)
    return u @ core @ v.T


# ---------------------------------------------------------------------------
# Accuracy metrics (Section 4.1)
# ---------------------------------------------------------------------------

def recon_error(m, u, sigma, vt) -> float:
    m = np.asarray(m, dtype=np.float64)
    return float(np.linalg.norm(m - (np.asarray(u, np.float64) * np.asarray(sigma, np.float64)[None, :])
                                @ np.asarray(vt, np.float64)) / np.linalg.norm(m))


def ortho_error(q) -> float:
    """||Q^T Q - I||_F / sqrt(n) (relative orthogonality, Section 4.1)."""
    return ortho_residual(np.asarray(q, dtype=np.float64))


# ---------------------------------------------------------------------------
# Learned lower bound: sketch features and a plain MLP (8 -> 64 -> 64 -> 1)
# ---------------------------------------------------------------------------

def sketch_features(x0: np.ndarray, probes: np.ndarray) -> np.ndarray:
    """Eight features of the normalized matrix X0 (sigma(X0) in [0, 1]):
    f_k = log( (1/(n s)) sum_probes z^T G^k z ) for k = 1..4 with G = X0^T X0 and the
    given Rademacher probes z (n x s) -- logs of Hutchinson estimates of tr(G^k)/n;
    f_5 = log ||X0||_F^2 / n;  f_6 = log of f_4 / f_3 (ratio of power traces);
    f_7 = log(n) / 10;  f_8 = log(m / n)."""
    x0 = np.asarray(x0, dtype=np.float64)
    mm, n = x0.shape
    z = np.asarray(probes, dtype=np.float64)
    s = z.shape[1]
    t = []
    y = z
    for _ in range(4):
        y = x0.T @ (x0 @ y)
        t.append(float(np.sum(z * y)) / (n * s))
    fro2 = float(np.sum(x0 * x0)) / n
    tiny = 1e-30
    lt = [math.log(max(v, tiny)) for v in t]
    return np.array([lt[0], lt[1], lt[2], lt[3],
                     math.log(max(fro2, tiny)),
                     math.log(max(t[3], tiny) / max(t[2], tiny)),
                     math.log(n) / 10.0,
                     math.log(mm / n)])


def mlp_forward(params, feats):
    """y = W3 relu(W2 relu(W1 f + b1) + b2) + b3, the predicted log lower bound.
    params = (W1 [64x8], b1, W2 [64x64], b2, W3 [1x64], b3); feats: (B, 8)."""
    w1, b1, w2, b2, w3, b3 = [np.asarray(p, dtype=np.float64) for p in params]
    f = np.asarray(feats, dtype=np.float64)
    z1 = f @ w1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3.T + b3
    return y[:, 0], (f, z1, h1, z2, h2)


def mlp_loss_grad(params, feats, target):
    """Mean squared error 0.5 mean (y - target)^2 and its gradient w.r.t. every parameter."""
    w1, b1, w2, b2, w3, b3 = [np.asarray(p, dtype=np.float64) for p in params]
    y, (f, z1, h1, z2, h2) = mlp_forward(params, feats)
    nb = y.shape[0]
    r = (y - np.asarray(target, dtype=np.float64)) / nb
    loss = 0.5 * float(np.sum((y - target) ** 2)) / nb
    dy = r[:, None]
    gw3 = dy.T @ h2
    gb3 = dy.sum(axis=0)
    dh2 = dy @ w3
    dz2 = dh2 * (z2 > 0)
    gw2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ w2
    dz1 = dh1 * (z1 > 0)
    gw1 = dz1.T @ f
    gb1 = dz1.sum(axis=0)
    return loss, (gw1, gb1, gw2, gb2, gw3, gb3)
