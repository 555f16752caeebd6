"""Pins of the oracle's learned-schedule pieces: the sketch features and the FP64 MLP.

Each check rests on something other than the oracle's own formula: exact trace
identities (Hadamard probes make the Hutchinson estimate exact; a scaled orthonormal X0
has every power trace in closed form), eigenvalues from LAPACK, properties of ReLU
networks (zero weights, positive homogeneity, a hand-built network computing the sum of
its inputs), and central finite differences of the loss."""
import math

import numpy as np

import workloads as W
from oracle import psvd_oracle as O


def _hadamard(n):
    h = np.ones((1, 1))
    while h.shape[0] < n:
        h = np.block([[h, h], [h, -h]])
    return h


def test_sketch_features_exact_with_hadamard_probes():
    # s = n Hadamard probes: Z Z^T = n I, so (1/(n s)) sum_z z^T G^k z = tr(G^k) / n exactly
    m, n = 24, 16
    rng = W.rng_for(41)
    x0 = 0.2 * rng.standard_normal((m, n))
    f = O.sketch_features(x0, _hadamard(n))
    lam = np.linalg.eigvalsh(x0.T @ x0)
    tr = [float(np.sum(lam ** k)) for k in range(1, 5)]
    for k in range(4):
        assert abs(f[k] - math.log(tr[k] / n)) <= 1e-12
    assert abs(f[4] - math.log(np.sum(x0 * x0) / n)) <= 1e-12
    assert abs(f[5] - math.log(tr[3] / tr[2])) <= 1e-12
    assert abs(f[6] - math.log(n) / 10) <= 1e-15 and abs(f[7] - math.log(m / n)) <= 1e-15


def test_sketch_features_scaled_orthonormal():
    # X0 = c Q with orthonormal columns: G = c^2 I, so every probe gives z^T G^k z = c^(2k) n
    m, n, c = 30, 12, 0.37
    q = W.orthonormal(W.rng_for(42), m, n)
    z = np.where(W.rng_for(43).random((n, 5)) < 0.5, -1.0, 1.0)
    f = O.sketch_features(c * q, z)
    for k in range(4):
        assert abs(f[k] - 2 * (k + 1) * math.log(c)) <= 1e-12
    assert abs(f[4] - 2 * math.log(c)) <= 1e-12 and abs(f[5] - 2 * math.log(c)) <= 1e-12


def _random_params(rng, scale=0.3):
    return [scale * rng.standard_normal(s) for s in ((64, 8), (64,), (64, 64), (64,), (1, 64), (1,))]


def test_mlp_zero_weights_give_the_output_bias():
    p = [np.zeros((64, 8)), np.zeros(64), np.zeros((64, 64)), np.zeros(64), np.zeros((1, 64)), np.array([0.7])]
    y, _ = O.mlp_forward(p, W.rng_for(44).standard_normal((5, 8)))
    np.testing.assert_array_equal(y, np.full(5, 0.7))


def test_mlp_positive_homogeneity_without_biases():
    rng = W.rng_for(45)
    p = _random_params(rng)
    p[1][:] = 0.0
    p[3][:] = 0.0
    p[5][:] = 0.0
    f = rng.standard_normal((7, 8))
    y1, _ = O.mlp_forward(p, f)
    y2, _ = O.mlp_forward(p, 2.5 * f)
    np.testing.assert_allclose(y2, 2.5 * y1, rtol=1e-13, atol=1e-15)


def test_mlp_handbuilt_network_sums_its_inputs():
    # layer 1 holds relu(f_i) and relu(-f_i); layer 2 permutes units; layer 3 weighs them
    # +1 / -1 at their permuted positions, so y = sum_i f_i + b3 (a transposed W1 or W2,
    # or layers applied in the wrong order, break the alignment)
    w1 = np.zeros((64, 8))
    for i in range(8):
        w1[i, i] = 1.0
        w1[8 + i, i] = -1.0
    perm = W.rng_for(46).permutation(64)
    w2 = np.zeros((64, 64))
    w2[perm, np.arange(64)] = 1.0            # unit j of layer 1 -> unit perm[j] of layer 2
    w3 = np.zeros((1, 64))
    w3[0, perm[:8]] = 1.0
    w3[0, perm[8:16]] = -1.0
    p = [w1, np.zeros(64), w2, np.zeros(64), w3, np.array([-0.25])]
    f = W.rng_for(47).standard_normal((6, 8))
    y, _ = O.mlp_forward(p, f)
    np.testing.assert_allclose(y, f.sum(axis=1) - 0.25, rtol=0, atol=1e-14)


def test_mlp_loss_gradient_finite_differences():
    rng = W.rng_for(48)
    p = _random_params(rng)
    f = rng.standard_normal((9, 8))
    t = rng.standard_normal(9)
    _, g = O.mlp_loss_grad(p, f, t)
    h = 1e-6
    for blk in range(6):
        flat = p[blk].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = O.mlp_loss_grad(p, f, t)
            flat[idx] = old - h
            lm, _ = O.mlp_loss_grad(p, f, t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[blk].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-7 * max(1.0, abs(an)), (blk, idx, fd, an)
