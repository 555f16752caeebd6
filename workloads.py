"""Seeded synthetic inputs for the polar-decomposition SVD.

This module only draws inputs; it holds none of the method's arithmetic, so both
the FP64 oracle and the CUDA path may use it.  Every generator is deterministic in
its seed.

Recipes (the paper's generator, Appendix A.3 "Matrix Generation Scheme"):

* ``orthonormal(rng, m, n)`` -- thin QR of an m x n standard-normal draw with the
  sign of each column fixed so that diag(R) > 0 (Householder QR from LAPACK used
  only as a random-orthogonal sampler).
* ``constructed(seed, m, n, s)`` -- A = Q1 diag(s) Q2^T with Q1 m x n and Q2 n x n
  orthonormal; the singular values of A are exactly ``sorted(s)`` in exact
  arithmetic, which is what the tests pin against.
* ``kappa_spectrum(n, kappa, rank)`` -- s_i = kappa^((r-i)/(r-1)) for i <= r, else 0
  (Appendix A.3, the kappa-controlled spectrum).
* ``gap_spectrum(n, gap)`` -- s_i = i for i < n and s_n = n-1+gap (Appendix A.3,
  the spectral-gap family of Table 3).

The named workloads below mirror the shapes and value distributions of the paper's
experiments (Section 4.1 / Tables 1-2 at 4096^2, kappa = 10; the rectangular
4096 x n family; the degenerate-spectrum backward study of Section 5).
"""
from __future__ import annotations

import math

import numpy as np


def rng_for(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.PCG64(int(seed)))


def orthonormal(rng: np.random.Generator, m: int, n: int) -> np.ndarray:
    """m x n matrix with orthonormal columns (m >= n), FP64."""
    g = rng.standard_normal((m, n))
    q, r = np.linalg.qr(g, mode="reduced")
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d[None, :]


def kappa_spectrum(n: int, kappa: float, rank: int | None = None) -> np.ndarray:
    r = n if rank is None else int(rank)
    s = np.zeros(n)
    if r == 1:
        s[0] = 1.0
        return s
    i = np.arange(1, r + 1, dtype=np.float64)
    s[:r] = float(kappa) ** ((r - i) / (r - 1))
    return s


def gap_spectrum(n: int, gap: float) -> np.ndarray:
    s = np.arange(1, n + 1, dtype=np.float64)
    s[-1] = n - 1 + gap
    return s[::-1].copy()


def linear_spectrum(n: int, lo: float = 0.1, hi: float = 1.0) -> np.ndarray:
    """s_i linearly spaced from hi down to lo: well-separated singular values."""
    return np.linspace(hi, lo, n)


def loguniform_spectrum(rng: np.random.Generator, n: int, lo: float, hi: float) -> np.ndarray:
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))


def constructed(seed: int, m: int, n: int, s: np.ndarray):
    """A = Q1 diag(s) Q2^T (FP64), with the factors it was built from."""
    rng = rng_for(seed)
    q1 = orthonormal(rng, m, n)
    q2 = orthonormal(rng, n, n)
    a = (q1 * np.asarray(s, dtype=np.float64)[None, :]) @ q2.T
    return a, q1, q2


def clustered_spectrum(rng: np.random.Generator, n_clusters: int, mult: int,
                       lo: float, hi: float, min_rel_gap: float) -> np.ndarray:
    """Cluster centres log-uniform in [lo, hi], redrawn until every pair of adjacent
    centres is at least ``min_rel_gap`` apart relative to the larger; each centre is
    repeated ``mult`` times exactly."""
    for _ in range(10000):
        c = np.sort(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_clusters)))
        rel = np.diff(c) / c[1:]
        if rel.size == 0 or rel.min() >= min_rel_gap:
            return np.repeat(c[::-1], mult)
    raise RuntimeError("could not draw separated cluster centres")


# --------------------------------------------------------------------------
# Named workloads (shapes and distributions of the paper's experiments)
# --------------------------------------------------------------------------

def small_square_factors(seed: int = 1, n: int = 256):
    """One n x n matrix with singular values log-uniform in [1e-3, 1], with the factors it
    was built from: (A, Q1, s, Q2), A = Q1 diag(s) Q2^T, s descending."""
    rng = rng_for(10_000 + seed)
    s = np.sort(loguniform_spectrum(rng, n, 1e-3, 1.0))[::-1]
    a, q1, q2 = constructed(seed, n, n, s)
    return a, q1, s, q2


def small_square(seed: int = 1, n: int = 256):
    """One n x n matrix with singular values log-uniform in [1e-3, 1]: (A, s)."""
    a, _, s, _ = small_square_factors(seed, n)
    return a, s


def kappa_square(seed: int, n: int, kappa: float, rank: int | None = None):
    """n x n matrix with the kappa-controlled spectrum of Appendix A.3."""
    s = kappa_spectrum(n, kappa, rank)
    a, q1, q2 = constructed(seed, n, n, s)
    return a, s


def marchenko_pastur(seed: int, m: int = 4096, n: int = 1024) -> np.ndarray:
    """iid N(0, 1/n) entries (singular values near [1 - sqrt(n/m), 1 + sqrt(n/m)] * sqrt(m/n))."""
    rng = rng_for(seed)
    return rng.standard_normal((m, n)) / math.sqrt(n)


def clustered_square_factors(seed: int, n: int = 512, n_clusters: int = 128, mult: int = 4):
    """Square matrix with exactly repeated singular values (clusters of ``mult``), with the
    factors it was built from: (A, Q1, s, Q2), s descending."""
    rng = rng_for(20_000 + seed)
    s = clustered_spectrum(rng, n_clusters, mult, 1e-2, 1.0, 1e-3)
    a, q1, q2 = constructed(seed, n, n, s)
    return a, q1, s, q2


def clustered_square(seed: int, n: int = 512, n_clusters: int = 128, mult: int = 4):
    """Square matrix with exactly repeated singular values (clusters of ``mult``): (A, s)."""
    a, _, s, _ = clustered_square_factors(seed, n, n_clusters, mult)
    return a, s


def rademacher(seed: int, batch: int, n: int, s: int) -> np.ndarray:
    """Seeded Rademacher probes (batch, n, s) with entries +-1, float32."""
    rng = rng_for(70_000 + seed)
    return np.where(rng.random((batch, n, s)) < 0.5, -1.0, 1.0).astype(np.float32)


def mlp_params(seed: int) -> np.ndarray:
    """Seeded parameters of the 8-64-64-1 lower-bound network as one float32 vector in the
    C ABI's layout [W1 64x8 | b1 64 | W2 64x64 | b2 64 | W3 1x64 | b3 1] (row-major
    blocks): He-scaled weights, biases N(0, 0.1^2)."""
    rng = rng_for(80_000 + seed)
    blocks = [rng.standard_normal((64, 8)) * (2.0 / 8) ** 0.5, 0.1 * rng.standard_normal(64),
              rng.standard_normal((64, 64)) * (2.0 / 64) ** 0.5, 0.1 * rng.standard_normal(64),
              rng.standard_normal((1, 64)) * (1.0 / 64) ** 0.5, 0.1 * rng.standard_normal(1)]
    return np.concatenate([x.ravel() for x in blocks]).astype(np.float32)


def loss_weights(seed: int, m: int, n: int):
    """Seeded N(0,1) weights for the loss <G_U, U> + <g_S, sigma> + <G_V, V>."""
    rng = rng_for(30_000 + seed)
    return rng.standard_normal((m, n)), rng.standard_normal(n), rng.standard_normal((n, n))


def schedule_family(seed: int, n: int):
    """One draw from the three spectrum families of the learned-schedule study:
    0: geometric spectrum with kappa log-uniform in [1e1, 1e6];
    1: power law s_i = i^-p with p uniform in [0.3, 1.5];
    2: rank-64 plus 1e-4 * N(0,1) noise (returned as a spectrum of the low-rank part;
       the noise is added to the matrix by ``schedule_matrix``)."""
    rng = rng_for(40_000 + seed)
    fam = int(rng.integers(0, 3))
    if fam == 0:
        kappa = math.exp(rng.uniform(math.log(1e1), math.log(1e6)))
        s = kappa_spectrum(n, kappa)
    elif fam == 1:
        p = rng.uniform(0.3, 1.5)
        s = np.arange(1, n + 1, dtype=np.float64) ** (-p)
    else:
        s = np.zeros(n)
        s[:64] = np.exp(rng.uniform(math.log(1e-2), 0.0, size=64))
        s = np.sort(s)[::-1]
    return fam, s


# --------------------------------------------------------------------------
# Large workloads (same recipe, torch RNG): the Gaussian factors and their QR are
# made on the host in FP64 (LAPACK), the product on the device in FP64.  These
# inputs are checked through properties that hold at any size (known spectrum, Weyl).
# --------------------------------------------------------------------------

def torch_orthonormal(gen, m: int, n: int):
    import torch
    g = torch.randn(m, n, generator=gen, dtype=torch.float64)
    q, r = torch.linalg.qr(g, mode="reduced")
    d = torch.sign(torch.diagonal(r))
    d = torch.where(d == 0, torch.ones_like(d), d)
    return q * d[None, :]


def torch_constructed(seed: int, m: int, n: int, s, device="cuda", batch: int = 1):
    """Batch of A_b = Q1_b diag(s_b) Q2_b^T (Q from the host QR of seeded Gaussians),
    formed on ``device`` in FP64 and returned as FP32 (batch, m, n).  ``s`` is (n,) or
    (batch, n)."""
    import torch
    gen = torch.Generator()
    gen.manual_seed(int(seed))
    s = torch.as_tensor(np.ascontiguousarray(s, dtype=np.float64), device=device)
    if s.dim() == 1:
        s = s[None, :].expand(batch, -1)
    out = torch.empty(batch, m, n, device=device, dtype=torch.float32)
    for b in range(batch):
        q1 = torch_orthonormal(gen, m, n).to(device)
        q2 = torch_orthonormal(gen, n, n).to(device)
        out[b] = ((q1 * s[b][None, :]) @ q2.T).float()
        del q1, q2
    return out
