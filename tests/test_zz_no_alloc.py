"""psvd_polar_fwd_noalloc: the polar decomposition for callers that cannot allocate
device memory -- real-time loops that forbid allocator calls, embeddings whose memory
manager owns all device memory, plugins handed only their input and output buffers.
Its scratch is a fixed device array inside the library that every call reuses, so a
call must give the same results as psvd_polar_fwd however the previous call left the
array: the calls below change shape, precision and schedule from one to the next, and
psvd_polar_fwd gets a workspace filled with NaN bytes, so that anything either entry
point failed to clear would show.  The products are deterministic (no atomics touch
W or H), so W and H must agree exactly.

This file is collected last on purpose (a failure here leaves every other test run)."""
import ctypes

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

INT_FIELDS = ["status", "iters", "qr_fallback", "sched_fallback", "prec_fallback", "steps_bf16", "steps_tf32",
              "steps_3xtf32"]


def _entry():
    import paper_2609_32505_gb300 as P
    L = P.lib()
    fn = L.psvd_polar_fwd_noalloc
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    fn.restype = ctypes.c_int
    fn.argtypes = [vp, vp, vp, i64, i64, i64, vp, vp, vp]
    L.psvd_polar_noalloc_capacity.restype = ctypes.c_size_t
    return P, L, fn


def _reference(P, L, A, opts):
    """psvd_polar_fwd through the C ABI with a workspace of NaN bytes."""
    B, m, n = A.shape
    nbytes = L.psvd_polar_workspace_bytes(B, m, n, ctypes.byref(opts))
    ws = torch.full((max(int(nbytes), 256),), 0xFF, dtype=torch.uint8, device="cuda")
    Wt = torch.empty_like(A)
    Ht = torch.empty(B, n, n, device="cuda")
    info = torch.zeros(B, P.INFO_WORDS, dtype=torch.int32, device="cuda")
    rc = L.psvd_polar_fwd(P._ptr(A), P._ptr(Wt), P._ptr(Ht), B, m, n, ctypes.byref(opts), P._ptr(ws), ws.numel(),
                          P._ptr(info), P._stream())
    assert rc == 0, L.psvd_last_error()
    return Wt, Ht, info


def _noalloc(P, fn, A, opts):
    B, m, n = A.shape
    Wt = torch.empty_like(A)
    Ht = torch.empty(B, n, n, device="cuda")
    info = torch.zeros(B, P.INFO_WORDS, dtype=torch.int32, device="cuda")
    rc = fn(P._ptr(A), P._ptr(Wt), P._ptr(Ht), B, m, n, ctypes.byref(opts), P._ptr(info), P._stream())
    assert rc == 0, P.lib().psvd_last_error()
    return Wt, Ht, info


def _batch(seed, B, m, n, kappas):
    return torch.from_numpy(np.stack([W.constructed(seed + k, m, n, W.kappa_spectrum(n, kappas[k]))[0]
                                      for k in range(B)]).astype(np.float32)).cuda()


def test_noalloc_matches_polar_fwd_on_consecutive_calls():
    P, L, fn = _entry()
    calls = [
        # (input, options): larger mixed-precision problem first, then a smaller one of another
        # shape in FP32, then the learned schedule with one over-estimated bound (its matrix
        # misses tol within budget and is rerun with the conservative schedule), then FP32 again
        (_batch(11, 2, 300, 256, [10.0, 1e2]), dict(precision=P.PREC_MIXED)),
        (_batch(21, 3, 150, 100, [10.0, 1e3, 1e2]), dict(precision=P.PREC_FP32)),
        (_batch(31, 2, 200, 160, [10.0, 1e3]), dict(precision=P.PREC_FP32, schedule=P.SCHED_LEARNED,
                                                    lower_bound=[0.05, 0.9])),
        (_batch(41, 2, 200, 160, [10.0, 1e2]), dict(precision=P.PREC_FP32)),
    ]
    for A, kw in calls:
        if "lower_bound" in kw:
            kw = dict(kw, lower_bound=torch.tensor(kw["lower_bound"], dtype=torch.float32, device="cuda"))
        opts = P.make_opts(**kw)
        w_ref, h_ref, info_ref = _reference(P, L, A, opts)
        w_na, h_na, info_na = _noalloc(P, fn, A, opts)
        torch.cuda.synchronize()
        ir, ia = P.info_dict(info_ref), P.info_dict(info_na)
        for r, a in zip(ir, ia):
            assert r["status"] == 0, r
            assert [r[k] for k in INT_FIELDS] == [a[k] for k in INT_FIELDS]
            assert a["ortho_resid"] == pytest.approx(r["ortho_resid"], rel=1e-5, abs=1e-12)
            assert a["scale"] == r["scale"]
        if "lower_bound" in kw:
            assert [i["sched_fallback"] for i in ia] == [0, 1]
        assert torch.isfinite(w_na).all() and torch.isfinite(h_na).all()
        assert torch.equal(w_na, w_ref)
        assert torch.equal(h_na, h_ref)


def test_noalloc_rejects_problems_beyond_its_scratch():
    P, L, fn = _entry()
    opts = P.make_opts()
    cap = L.psvd_polar_noalloc_capacity()
    n = 1024
    need = L.psvd_polar_workspace_bytes(4, n, n, ctypes.byref(opts))
    assert need > cap
    A = torch.zeros(4, n, n, device="cuda")
    Wt = torch.empty_like(A)
    rc = fn(P._ptr(A), P._ptr(Wt), None, 4, n, n, ctypes.byref(opts), None, P._stream())
    assert rc == -2
    msg = L.psvd_last_error().decode()
    assert str(need) in msg and str(cap) in msg
    # the same argument checks as psvd_polar_fwd
    assert fn(P._ptr(A), P._ptr(Wt), None, 4, n - 1, n, ctypes.byref(opts), None, P._stream()) == -1
