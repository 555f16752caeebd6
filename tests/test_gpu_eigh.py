"""GPU symmetric eigensolver (the EVD of Algorithm 1) against the FP64 oracle (cyclic Jacobi).

Eigenvalues: |lambda_i - lambda_i*| <= 2e-6 ||H||_2 (FP32 Householder reduction is
backward stable with error ~ sqrt(n) u ||H||).  Eigenvectors are unique only up to
sign (fixed by the convention) for simple eigenvalues, and only as a subspace for
repeated ones: simple ones are compared directly with a gap-scaled bound, clusters
through their projectors, and every basis must satisfy ||H V - V Lambda|| and
V^T V = I to FP32 level."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import psvd_oracle as O

pytestmark = pytest.mark.gpu


def _sym(rng, n):
    b = rng.standard_normal((n, n))
    return ((b + b.T) / 2).astype(np.float32).astype(np.float64)


def _run(h):
    import paper_2609_32505_gb300 as P
    s, vt = P.eigh(torch.from_numpy(h.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    return s.cpu().double().numpy(), vt.cpu().double().numpy()


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 129, 256, 300])
def test_eigh_parity(n):
    rng = W.rng_for(500 + n)
    h = np.stack([_sym(rng, n), _sym(rng, n)])
    s, vt = _run(h)
    for b in range(2):
        lam, v = O.eigh(h[b])
        nrm = max(np.abs(lam).max(), 1e-30)
        assert np.abs(s[b] - lam).max() <= 2e-6 * nrm * max(1.0, np.sqrt(n) / 8)
        V = vt[b].T
        assert np.linalg.norm(h[b] @ V - V * s[b][None, :]) <= 1e-5 * nrm * np.sqrt(n)
        assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-5
        idx = np.argmax(np.abs(V), axis=0)
        assert np.all(V[idx, np.arange(n)] > 0)
        gaps = np.full(n, np.inf)
        if n > 1:
            d = np.abs(np.diff(lam))
            gaps[:-1] = d
            gaps[1:] = np.minimum(gaps[1:], d)
        for i in range(n):
            if gaps[i] > 1e-3 * nrm:
                err = np.abs(V[:, i] - v[:, i]).max()
                assert err <= 2e-5 * nrm / gaps[i] + 1e-5, (i, err, gaps[i])


def test_eigh_clusters_projectors():
    rng = W.rng_for(77)
    n = 96
    q = W.orthonormal(rng, n, n)
    lam = np.repeat(np.array([3.0, 2.0, 1.5, 1.0, 0.5, 0.25]), 16)
    h = (q * lam) @ q.T
    s, vt = _run(h[None])
    V = vt[0].T
    assert np.abs(s[0] - lam).max() <= 2e-6 * 3
    assert np.abs(V.T @ V - np.eye(n)).max() <= 2e-5
    for val in np.unique(lam):
        sel = lam == val
        p_true = q[:, sel] @ q[:, sel].T
        p_got = V[:, sel] @ V[:, sel].T
        assert np.abs(p_got - p_true).max() <= 1e-4


def test_eigh_diagonal_and_zero():
    d = np.diag(np.array([5.0, -1.0, 3.0, 3.0, 0.0]))
    s, vt = _run(np.stack([d, np.zeros((5, 5))]))
    np.testing.assert_allclose(s[0], [5, 3, 3, 0, -1], atol=1e-6)
    np.testing.assert_allclose(s[1], 0.0, atol=0)
    assert np.abs(vt[1] @ vt[1].T - np.eye(5)).max() < 1e-6


@pytest.mark.parametrize("kappa", [1e3, 1e6])
def test_eigh_graded_spectrum(kappa):
    # geometric eigenvalues kappa^(-(i)/(n-1)): the small ones are closer than 1e-5 ||H||
    # to each other, so their FP32 estimates are refined in FP64 before inverse iteration;
    # the vectors must come out orthonormal and satisfy H V = V Lambda to FP32 level
    n = 400
    rng = W.rng_for(91)
    q = W.orthonormal(rng, n, n)
    lam0 = kappa ** (-np.arange(n) / (n - 1))
    h = ((q * lam0[None, :]) @ q.T).astype(np.float32).astype(np.float64)
    s, vt = _run(h[None])
    lam, _ = O.eigh(h)
    assert np.abs(s[0] - lam).max() <= 2e-6 * np.sqrt(n) / 8
    V = vt[0].T
    assert np.abs(V.T @ V - np.eye(n)).max() <= 1e-5
    assert np.linalg.norm(h @ V - V * s[0][None, :]) <= 1e-5 * np.sqrt(n)
