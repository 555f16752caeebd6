"""psvd_polar_fwd_noalloc: the polar decomposition for callers that cannot allocate
device memory (code running under CUDA graph capture, allocator-free real-time loops,
or a memory manager that owns every cudaMalloc).  Its scratch is a fixed device array
inside the library; the results must match psvd_polar_fwd's, call after call, because
every call reuses (and re-clears) the same array."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _entry():
    import paper_2609_32505_gb300 as P
    L = P.lib()
    fn = L.psvd_polar_fwd_noalloc
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    fn.restype = ctypes.c_int
    fn.argtypes = [vp, vp, vp, i64, i64, i64, vp, vp, vp]
    L.psvd_polar_noalloc_capacity.restype = ctypes.c_size_t
    return P, L, fn


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_polar_fwd_on_consecutive_calls(precision):
    P, L, fn = _entry()
    opts = P.make_opts(precision=precision)
    for seed in (11, 12):                      # two calls in a row, different inputs
        a = np.stack([W.constructed(seed + k, 200, 160, W.kappa_spectrum(160, 10.0 ** (1 + k)))[0]
                      for k in range(2)]).astype(np.float32)
        A = torch.from_numpy(a).cuda()
        w_ref, h_ref, info_ref = P.polar(A, opts, return_info=True)
        Wt = torch.empty_like(A)
        Ht = torch.empty(2, 160, 160, device="cuda")
        info = torch.zeros(2, P.INFO_WORDS, dtype=torch.int32, device="cuda")
        rc = fn(P._ptr(A), P._ptr(Wt), P._ptr(Ht), 2, 200, 160, ctypes.byref(opts), P._ptr(info), P._stream())
        assert rc == 0, P.lib().psvd_last_error()
        torch.cuda.synchronize()
        assert [i["status"] for i in P.info_dict(info)] == [i["status"] for i in info_ref]
        assert (Wt - w_ref).abs().max().item() <= 2e-5
        assert (Ht - h_ref).abs().max().item() <= 2e-5 * float(h_ref.abs().max())


def test_noalloc_rejects_problems_beyond_its_scratch():
    P, L, fn = _entry()
    opts = P.make_opts()
    cap = L.psvd_polar_noalloc_capacity()
    n = 1024
    assert L.psvd_polar_workspace_bytes(4, n, n, ctypes.byref(opts)) > cap
    A = torch.zeros(4, n, n, device="cuda")
    Wt = torch.empty_like(A)
    rc = fn(P._ptr(A), P._ptr(Wt), None, 4, n, n, ctypes.byref(opts), None, P._stream())
    assert rc == -2
