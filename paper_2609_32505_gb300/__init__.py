"""psvd: SVD via polar decomposition on GB300 -- thin Python binding.

Every numerical step runs in ``libpsvd.so`` (hand-written sm_103a kernels behind a
C ABI, declared in ``include/psvd.h``).  This module only marshals arguments:
it allocates device tensors (outputs and workspaces) with PyTorch, passes raw
pointers and the current CUDA stream, and wraps forward/backward in a
``torch.autograd.Function``.  There is no CPU or eager fallback: if the library
cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libpsvd.so")
_lib = None

PREC_FP32, PREC_MIXED = 0, 1
SCHED_CANS, SCHED_LEARNED, SCHED_NS = 0, 1, 2
GEMM_BF16, GEMM_TF32, GEMM_TF32X3 = 0, 1, 2

STATUS = {0: "ok", 1: "not_converged", -1: "arg", -2: "workspace", -3: "nonfinite", -4: "cuda",
          -5: "timeout", -6: "unsupported"}

MLP_NPARAMS = 64 * 8 + 64 + 64 * 64 + 64 + 64 + 1


class PsvdError(RuntimeError):
    pass


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("schedule", ctypes.c_int), ("delta", ctypes.c_double),
                ("pre_iters", ctypes.c_int), ("max_iter", ctypes.c_int), ("tol", ctypes.c_double),
                ("eps_qr", ctypes.c_double), ("lower_bound", ctypes.c_void_p), ("budget", ctypes.c_int)]


INFO_FIELDS = ["status", "iters", "qr_fallback", "sched_fallback", "steps_bf16", "steps_tf32",
               "steps_3xtf32", "ortho_resid", "scale"]
INFO_INTS = 7   # the first 7 fields are int32, the last 2 float32


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def lib():
    """Loads libpsvd.so (built in-tree by ``build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise PsvdError(f"{_LIB_PATH} is missing: run paper_2609_32505_gb300.build() first "
                        "(there is no fallback implementation)")
    L = ctypes.CDLL(_LIB_PATH)
    vp, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
    sig = {
        "psvd_default_opts": (None, [vp]),
        "psvd_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "psvd_kernel_launch_count": (ctypes.c_uint64, []),
        "psvd_gemm_workspace_bytes": (sz, [i64, i64, i64, i64]),
        "psvd_gemm_tn": (ctypes.c_int, [vp, vp, vp, i64, i64, i64, i64, ctypes.c_int, vp, sz, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _check(rc: int, what: str):
    if rc != 0:
        msg = lib().psvd_status_string(rc).decode()
        raise PsvdError(f"{what} failed: {msg} (status {rc})")


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def kernel_launches() -> int:
    return int(lib().psvd_kernel_launch_count())


def gemm_tn(a: torch.Tensor, b: torch.Tensor, precision: int = GEMM_TF32X3) -> torch.Tensor:
    """D[i] = A[i] @ B[i]^T on the tcgen05 tensor cores (A: (batch,)M x K, B: (batch,)N x K)."""
    squeeze = a.dim() == 2
    A = a.unsqueeze(0) if squeeze else a
    B = b.unsqueeze(0) if squeeze else b
    A = A.contiguous().float()
    B = B.contiguous().float()
    bt, M, K = A.shape
    N = B.shape[1]
    D = torch.empty(bt, M, N, device=A.device, dtype=torch.float32)
    L = lib()
    ws = _workspace(L.psvd_gemm_workspace_bytes(bt, M, N, K), A.device)
    _check(L.psvd_gemm_tn(_ptr(A), _ptr(B), _ptr(D), bt, M, N, K, precision, _ptr(ws), ws.numel(), _stream()),
           "psvd_gemm_tn")
    return D[0] if squeeze else D
