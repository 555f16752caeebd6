"""GPU parity of the tcgen05 TN product kernel against FP64 products (CPU).

Tolerances follow from the operand rounding: BF16 (8-bit significand) gives a
relative error per product of 2^-8 and TF32 (11-bit) 2^-11, so with random-sign
accumulation over K terms the error is ~ u * sqrt(K) * |A||B| entrywise; split
hi+lo TF32 drops the lo*lo term (<= 2^-22 relative) and is FP32-accurate."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _ref(a, b):
    return np.einsum("bik,bjk->bij", a.astype(np.float64), b.astype(np.float64))


@pytest.mark.parametrize("prec,rtol", [(0, 2e-2), (1, 3e-3), (2, 2e-6)])
@pytest.mark.parametrize("batch,M,N,K", [(1, 128, 128, 32), (1, 256, 384, 512), (2, 200, 77, 300),
                                         (3, 1, 5, 7), (1, 130, 129, 1000), (2, 2048, 2048, 96),
                                         (1, 300, 1100, 200)])
def test_gemm_tn_parity(prec, rtol, batch, M, N, K):
    import paper_2609_32505_gb300 as P
    rng = W.rng_for(M * 7 + N * 3 + K)
    a = rng.standard_normal((batch, M, K)).astype(np.float32)
    b = rng.standard_normal((batch, N, K)).astype(np.float32)
    d = P.gemm_tn(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), prec)
    torch.cuda.synchronize()
    ref = _ref(a, b)
    scale = np.sqrt(K)   # |A_i||B_j| ~ K, error ~ u sqrt(K) * sqrt(K) for random signs
    err = np.abs(d.cpu().double().numpy() - ref).max() / scale
    assert err < rtol * 4, f"max scaled error {err}"


def test_gemm_tn_split_beats_single_tf32():
    import paper_2609_32505_gb300 as P
    rng = W.rng_for(99)
    a = rng.standard_normal((1, 256, 1024)).astype(np.float32)
    b = rng.standard_normal((1, 256, 1024)).astype(np.float32)
    ref = _ref(a, b)
    errs = []
    for prec in (0, 1, 2):
        d = P.gemm_tn(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), prec).cpu().double().numpy()
        errs.append(np.abs(d - ref).max())
    assert errs[2] < errs[1] / 50 < errs[0] / 50
