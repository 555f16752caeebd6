"""Failure detection without a GPU fault: the grid barriers of the cooperative kernels are
bounded waits.  With the bound lowered to a couple of polls (psvd_debug_set_barrier_spin)
the tridiagonalization's barrier expires at once; every CTA records the timeout and runs
on, the call returns, psvd_svd_fwd reports PSVD_ERR_TIMEOUT in every record, and the
context stays usable: with the default bound restored the next call is correct.  Nothing
is injected on the device beyond the shorter wait, and the product kernel's pipeline waits
(TMA / mbarrier) are not touched."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W
from oracle import psvd_oracle as O

pytestmark = pytest.mark.gpu


def test_expired_grid_barrier_reports_timeout_and_the_context_survives():
    import paper_2609_32505_gb300 as P
    L = P.lib()
    L.psvd_debug_set_barrier_spin.argtypes = [ctypes.c_uint32]
    L.psvd_debug_set_barrier_spin.restype = ctypes.c_int
    n = 512
    a, _ = W.kappa_square(77, n, 10.0)
    a32 = a.astype(np.float32).astype(np.float64)
    A = torch.from_numpy(np.stack([a32, a32]).astype(np.float32)).cuda()
    try:
        assert L.psvd_debug_set_barrier_spin(2) == 0
        _, _, _, info = P.svd_fwd(A, P.make_opts(), return_info=True)
        torch.cuda.synchronize()
        assert [i["status"] for i in info] == [-5, -5]
    finally:
        L.psvd_debug_set_barrier_spin(0)
    U, S, VT, info = P.svd_fwd(A, P.make_opts(), return_info=True)
    torch.cuda.synchronize()
    assert [i["status"] for i in info] == [0, 0]
    s_ref = O.svd(a32)[1]
    u, s, vt = U[0].cpu().double().numpy(), S[0].cpu().double().numpy(), VT[0].cpu().double().numpy()
    assert np.abs(s - s_ref).max() <= 1e-5 * s_ref[0]
    assert O.recon_error(a32, u, s, vt) <= 1e-5
