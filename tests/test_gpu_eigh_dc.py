"""The matmul-only eigensolver (spectral divide and conquer on the polar decomposition,
psvd_eigh_dc) against the FP64 oracle's cyclic Jacobi EVD.

Sizes take every path: a leaf (n <= 512, the tridiagonal solver directly), one split
(n = 700) and two levels of splits (n = 1500), plus the degenerate H = c I (no split
possible).  The splits' backward error comes from the FP32-accurate polar factors
(orthogonality ~1e-6), so the bounds are: eigenvalues within 1e-5 ||H||, ||H V - V Lambda||_F
and ||V^T V - I||_F / sqrt(n) within 1e-5 ||H||_F resp. 1e-5, and simple eigenvalues with a
relative gap above 1e-3 give eigenvectors parallel to the oracle's to 1e-4."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import psvd_oracle as O

pytestmark = pytest.mark.gpu


def _run(h):
    import paper_2609_32505_gb300 as P
    s, vt = P.eigh_dc(torch.from_numpy(h.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    return s.cpu().double().numpy(), vt.cpu().double().numpy()


def _spd(seed, n, spec):
    rng = W.rng_for(seed)
    q = W.orthonormal(rng, n, n)
    return ((q * np.asarray(spec)[None, :]) @ q.T).astype(np.float32).astype(np.float64)


def _check(h, s, vt):
    lam, v_ref = O.eigh(h)
    n = h.shape[0]
    hn = np.linalg.norm(h, 2)
    assert np.abs(s - lam).max() <= 1e-5 * hn
    v = vt.T
    assert np.linalg.norm(h @ v - v * s[None, :]) <= 1e-5 * np.linalg.norm(h)
    assert np.linalg.norm(v.T @ v - np.eye(n)) / np.sqrt(n) <= 1e-5
    gap = np.full(n, np.inf)
    gap[:-1] = np.minimum(gap[:-1], lam[:-1] - lam[1:])
    gap[1:] = np.minimum(gap[1:], lam[:-1] - lam[1:])
    simple = gap > 1e-3 * hn
    if simple.any():
        dots = np.abs((v[:, simple] * v_ref[:, simple]).sum(0))
        assert dots.min() >= 1 - 1e-4


@pytest.mark.parametrize("n", [300, 700, 1500])
def test_eigh_dc_parity(n):
    h = _spd(600 + n, n, np.linspace(2.0, 0.2, n))
    s, vt = _run(h)
    _check(h, s, vt)


def test_eigh_dc_indefinite_and_clustered():
    # indefinite symmetric matrix with clusters of four (projectors for the clusters are the
    # only well-defined objects; the residual and orthogonality checks cover them)
    n = 900
    base = np.linspace(-1.0, 1.0, n // 4)
    h = _spd(610, n, np.repeat(base, 4)[::-1])
    s, vt = _run(h)
    _check(h, s, vt)


def test_eigh_dc_scalar_matrix_and_batch():
    import paper_2609_32505_gb300 as P
    n = 640
    h = np.stack([2.5 * np.eye(n), _spd(620, n, np.linspace(1.0, 0.01, n))])
    s, vt = _run(h)
    assert np.abs(s[0] - 2.5).max() <= 1e-5 * 2.5
    assert np.linalg.norm(vt[0] @ vt[0].T - np.eye(n)) / np.sqrt(n) <= 1e-5
    _check(h[1], s[1], vt[1])
    # the same eigenvalues as the tridiagonal solver
    s2, _ = P.eigh(torch.from_numpy(h[1].astype(np.float32)).cuda())
    assert np.abs(s[1] - s2.cpu().double().numpy()).max() <= 1e-5
