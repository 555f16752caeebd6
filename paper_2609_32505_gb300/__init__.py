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

PREC_FP32, PREC_MIXED, PREC_MIXED_BF16 = 0, 1, 2
SCHED_CANS, SCHED_LEARNED, SCHED_NS, SCHED_PE = 0, 1, 2, 3
GEMM_BF16, GEMM_TF32, GEMM_TF32X3 = 0, 1, 2

STATUS = {0: "ok", 1: "not_converged", -1: "arg", -2: "workspace", -3: "nonfinite", -4: "cuda",
          -5: "timeout", -6: "unsupported"}

MLP_NPARAMS = 64 * 8 + 64 + 64 * 64 + 64 + 64 + 1


class PsvdError(RuntimeError):
    pass


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("schedule", ctypes.c_int), ("delta", ctypes.c_double),
                ("pre_iters", ctypes.c_int), ("max_iter", ctypes.c_int), ("tol", ctypes.c_double),
                ("eps_qr", ctypes.c_double), ("lower_bound", ctypes.c_void_p), ("budget", ctypes.c_int),
                ("res_history", ctypes.c_void_p), ("preqr", ctypes.c_int)]


INFO_FIELDS = ["status", "iters", "qr_fallback", "sched_fallback", "prec_fallback", "steps_bf16", "steps_tf32",
               "steps_3xtf32", "ortho_resid", "scale", "corr_max", "recon_est"]
INFO_INTS = 8   # the first 8 fields are int32, the rest float32
INFO_WORDS = len(INFO_FIELDS)
MIXED_CORR_MAX = 2e-3    # PSVD_MIXED_CORR_MAX of psvd.h
MIXED_RECON_MAX = 5e-6   # PSVD_MIXED_RECON_MAX of psvd.h
MIXED_LB_MIN = 5e-5      # PSVD_MIXED_LB_MIN of psvd.h


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
        "psvd_last_error": (ctypes.c_char_p, []),
        "psvd_kernel_launch_count": (ctypes.c_uint64, []),
        "psvd_gemm_workspace_bytes": (sz, [i64, i64, i64, i64]),
        "psvd_gemm_tn": (ctypes.c_int, [vp, vp, vp, i64, i64, i64, i64, ctypes.c_int, vp, sz, vp]),
        "psvd_polar_workspace_bytes": (sz, [i64, i64, i64, vp]),
        "psvd_polar_fwd": (ctypes.c_int, [vp, vp, vp, i64, i64, i64, vp, vp, sz, vp, vp]),
        "psvd_svd_workspace_bytes": (sz, [i64, i64, i64, vp]),
        "psvd_svd_fwd": (ctypes.c_int, [vp, vp, vp, vp, i64, i64, i64, vp, vp, sz, vp, vp]),
        "psvd_eigh_workspace_bytes": (sz, [i64, i64]),
        "psvd_eigh": (ctypes.c_int, [vp, vp, vp, i64, i64, vp, sz, vp]),
        "psvd_svd_bwd_workspace_bytes": (sz, [i64, i64, i64]),
        "psvd_svd_bwd": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, vp, vp, i64, i64, i64, ctypes.c_double,
                                        ctypes.c_int, vp, sz, vp]),
        "psvd_polar_bwd_workspace_bytes": (sz, [i64, i64, i64]),
        "psvd_polar_bwd": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, i64, i64, i64, ctypes.c_double, vp, sz, vp]),
        "psvd_eigh_bwd_workspace_bytes": (sz, [i64, i64]),
        "psvd_eigh_bwd": (ctypes.c_int, [vp, vp, vp, vp, vp, i64, i64, ctypes.c_double, ctypes.c_int, vp, sz, vp]),
        "psvd_eigh_dc_workspace_bytes": (sz, [i64]),
        "psvd_eigh_dc": (ctypes.c_int, [vp, vp, vp, i64, i64, vp, sz, vp]),
        "psvd_qr_workspace_bytes": (sz, [i64, i64, i64]),
        "psvd_qr": (ctypes.c_int, [vp, vp, vp, i64, i64, i64, vp, sz, vp]),
        "psvd_profile_enable": (ctypes.c_int, [ctypes.c_int]),
        "psvd_sketch_workspace_bytes": (sz, [i64, i64, i64, i64]),
        "psvd_sketch_features": (ctypes.c_int, [vp, vp, i64, vp, i64, i64, i64, vp, sz, vp]),
        "psvd_mlp_fwd": (ctypes.c_int, [vp, vp, vp, i64, vp]),
        "psvd_mlp_lower_bound": (ctypes.c_int, [vp, vp, vp, i64, ctypes.c_float, vp]),
        "psvd_mlp_grad": (ctypes.c_int, [vp, vp, vp, i64, vp, vp, vp]),
        "psvd_mlp_train_step": (ctypes.c_int, [vp, vp, vp, vp, vp, vp, i64, ctypes.c_float, ctypes.c_int, vp, vp]),
        "psvd_profile_read": (ctypes.c_int, [vp]),
        "psvd_mlp_standardize": (ctypes.c_int, [vp, i64, vp, vp, vp]),
        "psvd_mlp_fold": (ctypes.c_int, [vp, vp, vp]),
        "psvd_mlp_gather": (ctypes.c_int, [vp, vp, vp, i64, vp, vp, vp]),
        "psvd_mlp_calibrate": (ctypes.c_int, [vp, vp, vp, i64, ctypes.c_float, vp, vp, vp]),
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
        where = lib().psvd_last_error().decode() if rc == -4 else ""
        raise PsvdError(f"{what} failed: {msg} (status {rc}) {where}")


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


def make_opts(precision: int = PREC_FP32, schedule: int = SCHED_CANS, delta: float = 0.99, pre_iters: int = 2,
              max_iter: int = 50, tol: float = 1e-5, eps_qr: float = 1e-5, lower_bound=None, budget: int = 0,
              res_history=None, preqr: int = 0):
    o = Opts()
    lib().psvd_default_opts(ctypes.byref(o))
    o.precision, o.schedule, o.delta, o.pre_iters = precision, schedule, delta, pre_iters
    o.max_iter, o.tol, o.eps_qr, o.budget = max_iter, tol, eps_qr, budget
    o.lower_bound = None if lower_bound is None else lower_bound.data_ptr()
    o.res_history = None if res_history is None else res_history.data_ptr()
    o.preqr = int(preqr)
    return o


def info_dict(info: torch.Tensor):
    """Decodes a (batch, INFO_WORDS) int32 device info array into a list of dicts."""
    raw = info.cpu()
    ints = raw[:, :INFO_INTS].tolist()
    flts = raw[:, INFO_INTS:].contiguous().view(torch.float32).tolist()
    return [dict(zip(INFO_FIELDS, i + f)) for i, f in zip(ints, flts)]


def _batched(a):
    if a.dim() == 2:
        return a.unsqueeze(0), True
    return a, False


def polar(a: torch.Tensor, opts: Opts | None = None, want_h: bool = True, return_info: bool = False):
    """Right polar decomposition A = W H (batch of m x n, m >= n) by the polynomial iteration."""
    A, sq = _batched(a.contiguous().float())
    bt, m, n = A.shape
    o = opts or make_opts()
    W = torch.empty_like(A)
    H = torch.empty(bt, n, n, device=A.device, dtype=torch.float32) if want_h else None
    info = torch.zeros(bt, INFO_WORDS, device=A.device, dtype=torch.int32)
    L = lib()
    ws = _workspace(L.psvd_polar_workspace_bytes(bt, m, n, ctypes.byref(o)), A.device)
    _check(L.psvd_polar_fwd(_ptr(A), _ptr(W), _ptr(H), bt, m, n, ctypes.byref(o), _ptr(ws), ws.numel(),
                            _ptr(info), _stream()), "psvd_polar_fwd")
    out = (W[0] if sq else W, None if H is None else (H[0] if sq else H))
    return out + (info_dict(info),) if return_info else out


def qr(a: torch.Tensor, want_r: bool = True):
    """Thin QR A = Q R with diag(R) >= 0 (batch of m x n, m >= n) on the GPU (psvd_qr)."""
    A, sq = _batched(a.contiguous().float())
    bt, m, n = A.shape
    Q = torch.empty_like(A)
    R = torch.empty(bt, n, n, device=A.device, dtype=torch.float32) if want_r else None
    L = lib()
    ws = _workspace(L.psvd_qr_workspace_bytes(bt, m, n), A.device)
    _check(L.psvd_qr(_ptr(A), _ptr(Q), _ptr(R), bt, m, n, _ptr(ws), ws.numel(), _stream()), "psvd_qr")
    if sq:
        return Q[0], None if R is None else R[0]
    return Q, R


def eigh(h: torch.Tensor):
    """Symmetric EVD H = V diag(S) V^T: returns (S descending, V^T) for a batch of n x n."""
    Hs, sq = _batched(h.contiguous().float())
    bt, n, _ = Hs.shape
    S = torch.empty(bt, n, device=Hs.device, dtype=torch.float32)
    VT = torch.empty(bt, n, n, device=Hs.device, dtype=torch.float32)
    L = lib()
    ws = _workspace(L.psvd_eigh_workspace_bytes(bt, n), Hs.device)
    _check(L.psvd_eigh(_ptr(Hs), _ptr(S), _ptr(VT), bt, n, _ptr(ws), ws.numel(), _stream()), "psvd_eigh")
    return (S[0], VT[0]) if sq else (S, VT)


def eigh_dc(h: torch.Tensor):
    """Symmetric EVD by spectral divide and conquer on the polar decomposition (psvd_eigh_dc):
    returns (S descending, V^T) for a batch of n x n."""
    Hs, sq = _batched(h.contiguous().float())
    bt, n, _ = Hs.shape
    S = torch.empty(bt, n, device=Hs.device, dtype=torch.float32)
    VT = torch.empty(bt, n, n, device=Hs.device, dtype=torch.float32)
    L = lib()
    ws = _workspace(L.psvd_eigh_dc_workspace_bytes(n), Hs.device)
    _check(L.psvd_eigh_dc(_ptr(Hs), _ptr(S), _ptr(VT), bt, n, _ptr(ws), ws.numel(), _stream()), "psvd_eigh_dc")
    return (S[0], VT[0]) if sq else (S, VT)


def svd_fwd(a: torch.Tensor, opts: Opts | None = None, return_info: bool = False):
    """Thin SVD A = U diag(S) V^T by Algorithm 1 (batch of m x n, m >= n); returns (U, S, V^T)."""
    A, sq = _batched(a.contiguous().float())
    bt, m, n = A.shape
    o = opts or make_opts()
    U = torch.empty_like(A)
    S = torch.empty(bt, n, device=A.device, dtype=torch.float32)
    VT = torch.empty(bt, n, n, device=A.device, dtype=torch.float32)
    info = torch.zeros(bt, INFO_WORDS, device=A.device, dtype=torch.int32)
    L = lib()
    ws = _workspace(L.psvd_svd_workspace_bytes(bt, m, n, ctypes.byref(o)), A.device)
    _check(L.psvd_svd_fwd(_ptr(A), _ptr(U), _ptr(S), _ptr(VT), bt, m, n, ctypes.byref(o), _ptr(ws), ws.numel(),
                          _ptr(info), _stream()), "psvd_svd_fwd")
    out = (U[0], S[0], VT[0]) if sq else (U, S, VT)
    return out + (info_dict(info),) if return_info else out


def _opt(x, shape_like):
    return None if x is None else x.contiguous().float().reshape(shape_like)


def svd_bwd(a, u, s, vt, du=None, ds=None, dvt=None, eps: float = 1e-8, kreg_mode: int = 0):
    """Algorithm 4 backward: dA from the cached factors and incoming gradients (None = zero)."""
    A, sq = _batched(a.contiguous().float())
    bt, m, n = A.shape
    U = u.contiguous().float().reshape(bt, m, n)
    S = s.contiguous().float().reshape(bt, n)
    VT = vt.contiguous().float().reshape(bt, n, n)
    dU, dS, dVT = _opt(du, (bt, m, n)), _opt(ds, (bt, n)), _opt(dvt, (bt, n, n))
    dA = torch.empty_like(A)
    L = lib()
    ws = _workspace(L.psvd_svd_bwd_workspace_bytes(bt, m, n), A.device)
    _check(L.psvd_svd_bwd(_ptr(A), _ptr(U), _ptr(S), _ptr(VT), _ptr(dU), _ptr(dS), _ptr(dVT), _ptr(dA), bt, m, n,
                          float(eps), int(kreg_mode), _ptr(ws), ws.numel(), _stream()), "psvd_svd_bwd")
    return dA[0] if sq else dA


def polar_bwd(a, w, h, dw=None, dh=None, eps: float = 1e-8):
    """Algorithm 3 backward of the polar decomposition A = W H."""
    A, sq = _batched(a.contiguous().float())
    bt, m, n = A.shape
    Wt = w.contiguous().float().reshape(bt, m, n)
    H = h.contiguous().float().reshape(bt, n, n)
    dW, dH = _opt(dw, (bt, m, n)), _opt(dh, (bt, n, n))
    dA = torch.empty_like(A)
    L = lib()
    ws = _workspace(L.psvd_polar_bwd_workspace_bytes(bt, m, n), A.device)
    _check(L.psvd_polar_bwd(_ptr(A), _ptr(Wt), _ptr(H), _ptr(dW), _ptr(dH), _ptr(dA), bt, m, n, float(eps),
                            _ptr(ws), ws.numel(), _stream()), "psvd_polar_bwd")
    return dA[0] if sq else dA


def eigh_bwd(s, vt, ds=None, dvt=None, eps: float = 1e-8, kreg_mode: int = 0):
    """Theorem 4.3 backward of H = V diag(S) V^T (psvd_eigh_bwd): the symmetric dH from the
    gradients of S and V^T (None = zero), with K_eps chosen by kreg_mode."""
    S = s.contiguous().float()
    sq = S.dim() == 1
    S = S.reshape(-1, S.shape[-1])
    bt, n = S.shape
    VT = vt.contiguous().float().reshape(bt, n, n)
    dS, dVT = _opt(ds, (bt, n)), _opt(dvt, (bt, n, n))
    dH = torch.empty(bt, n, n, device=S.device, dtype=torch.float32)
    L = lib()
    ws = _workspace(L.psvd_eigh_bwd_workspace_bytes(bt, n), S.device)
    _check(L.psvd_eigh_bwd(_ptr(S), _ptr(VT), _ptr(dS), _ptr(dVT), _ptr(dH), bt, n, float(eps), int(kreg_mode),
                           _ptr(ws), ws.numel(), _stream()), "psvd_eigh_bwd")
    return dH[0] if sq else dH


class _EighFunction(torch.autograd.Function):
    """Forward: psvd_eigh.  Backward: psvd_eigh_bwd (Theorem 4.3 with K_eps)."""

    @staticmethod
    def forward(ctx, h, eps, kreg_mode):
        s, vt = eigh(h)
        ctx.save_for_backward(s, vt)
        ctx.eps, ctx.kreg = eps, kreg_mode
        return s, vt

    @staticmethod
    def backward(ctx, gs, gvt):
        s, vt = ctx.saved_tensors
        return eigh_bwd(s, vt, gs, gvt, ctx.eps, ctx.kreg), None, None


def eigh_ad(h: torch.Tensor, eps: float = 1e-8, kreg_mode: int = 0):
    """Differentiable symmetric EVD: returns (S descending, V^T); gradients by Theorem 4.3."""
    return _EighFunction.apply(h, eps, kreg_mode)


class _SVDFunction(torch.autograd.Function):
    """Forward: Algorithm 1 (psvd_svd_fwd).  Backward: Algorithm 4 (psvd_svd_bwd), which
    recomputes W = U V^T from the cached factors; no polar iterate is stored."""

    @staticmethod
    def forward(ctx, a, opts_args, eps, kreg_mode):
        u, s, vt = svd_fwd(a, make_opts(**opts_args))
        ctx.save_for_backward(a, u, s, vt)
        ctx.eps, ctx.kreg = eps, kreg_mode
        return u, s, vt

    @staticmethod
    def backward(ctx, gu, gs, gvt):
        a, u, s, vt = ctx.saved_tensors
        da = svd_bwd(a, u, s, vt, gu, gs, gvt, ctx.eps, ctx.kreg)
        return da, None, None, None


def svd(a: torch.Tensor, precision: int = PREC_FP32, schedule: int = SCHED_CANS, eps: float = 1e-8,
        kreg_mode: int = 0, **opts):
    """Differentiable thin SVD: returns (U, S, V^T) with autograd through Algorithm 4."""
    args = dict(precision=precision, schedule=schedule, **opts)
    return _SVDFunction.apply(a, args, eps, kreg_mode)


# ---------------------------------------------------------------- learned schedule
def rademacher_probes(batch: int, n: int, s: int = 8, seed: int = 0, device="cuda") -> torch.Tensor:
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    z = torch.randint(0, 2, (batch, n, s), generator=g).float() * 2 - 1
    return z.to(device)


def sketch_features(a: torch.Tensor, probes: torch.Tensor) -> torch.Tensor:
    """Eight sketch features per matrix (see include/psvd.h): (batch, 8)."""
    A, _ = _batched(a.contiguous().float())
    bt, m, n = A.shape
    Z = probes.contiguous().float().reshape(bt, n, -1)
    s = Z.shape[2]
    F = torch.empty(bt, 8, device=A.device, dtype=torch.float32)
    L = lib()
    ws = _workspace(L.psvd_sketch_workspace_bytes(bt, m, n, s), A.device)
    _check(L.psvd_sketch_features(_ptr(A), _ptr(Z), s, _ptr(F), bt, m, n, _ptr(ws), ws.numel(), _stream()),
           "psvd_sketch_features")
    return F


def mlp_init(seed: int = 0, device="cuda") -> torch.Tensor:
    """He-initialized parameters [W1 64x8 | b1 | W2 64x64 | b2 | W3 1x64 | b3]."""
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    w1 = torch.randn(64, 8, generator=g) * (2.0 / 8) ** 0.5
    w2 = torch.randn(64, 64, generator=g) * (2.0 / 64) ** 0.5
    w3 = torch.randn(1, 64, generator=g) * (1.0 / 64) ** 0.5
    p = torch.cat([w1.flatten(), torch.zeros(64), w2.flatten(), torch.zeros(64), w3.flatten(), torch.zeros(1)])
    return p.to(device)


def mlp_unpack(p: torch.Tensor):
    p = p.detach().cpu().double()
    o = [0]

    def take(k, shape):
        x = p[o[0]:o[0] + k].reshape(shape)
        o[0] += k
        return x.numpy()
    return (take(512, (64, 8)), take(64, (64,)), take(4096, (64, 64)), take(64, (64,)), take(64, (1, 64)),
            take(1, (1,)))


def mlp_forward(params: torch.Tensor, feats: torch.Tensor) -> torch.Tensor:
    F = feats.contiguous().float()
    y = torch.empty(F.shape[0], device=F.device, dtype=torch.float32)
    _check(lib().psvd_mlp_fwd(_ptr(params), _ptr(F), _ptr(y), F.shape[0], _stream()), "psvd_mlp_fwd")
    return y


def mlp_grad(params: torch.Tensor, feats: torch.Tensor, target: torch.Tensor):
    F = feats.contiguous().float()
    tg = target.contiguous().float()
    g = torch.empty_like(params)
    loss = torch.zeros(1, device=params.device)
    _check(lib().psvd_mlp_grad(_ptr(params), _ptr(F), _ptr(tg), F.shape[0], _ptr(g), _ptr(loss), _stream()),
           "psvd_mlp_grad")
    return float(loss.item()), g


def mlp_train(params: torch.Tensor, feats: torch.Tensor, target: torch.Tensor, steps: int = 500, lr: float = 3e-3,
              batch: int = 1024, seed: int = 0):
    """Adam on 0.5 mean (y - target)^2 with the library's own kernels; returns the loss curve.
    The minibatch indices are drawn on the host (seeded) and copied once; the rows are
    gathered on the device (psvd_mlp_gather)."""
    F = feats.contiguous().float()
    tg = target.contiguous().float()
    grads = torch.zeros_like(params)
    m1 = torch.zeros_like(params)
    m2 = torch.zeros_like(params)
    loss = torch.zeros(1, device=params.device)
    L = lib()
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    nb = F.shape[0]
    bs = min(batch, nb)
    idx = torch.randint(0, nb, (steps, bs), generator=g, dtype=torch.int32).to(F.device)
    Fb = torch.empty(bs, 8, device=F.device)
    tb = torch.empty(bs, device=F.device)
    curve = []
    for it in range(1, steps + 1):
        _check(L.psvd_mlp_gather(_ptr(F), _ptr(tg), _ptr(idx[it - 1]), bs, _ptr(Fb), _ptr(tb), _stream()),
               "psvd_mlp_gather")
        _check(L.psvd_mlp_train_step(_ptr(params), _ptr(grads), _ptr(m1), _ptr(m2), _ptr(Fb), _ptr(tb), bs,
                                     float(lr), it, _ptr(loss), _stream()), "psvd_mlp_train_step")
        if it % 50 == 0 or it == 1:
            curve.append(float(loss.item()))
    return curve


def mlp_fit(feats: torch.Tensor, target: torch.Tensor, steps: int = 2000, lr: float = 3e-3, batch: int = 256,
            seed: int = 0):
    """Trains the MLP with the library's Adam kernels on standardized features
    (psvd_mlp_standardize), then folds the standardization into the first layer
    (psvd_mlp_fold), so the returned parameters act on raw features.  Returns (params, curve)."""
    F = feats.contiguous().float()
    L = lib()
    stats = torch.empty(16, device=F.device)
    Fs = torch.empty_like(F)
    _check(L.psvd_mlp_standardize(_ptr(F), F.shape[0], _ptr(Fs), _ptr(stats), _stream()), "psvd_mlp_standardize")
    params = mlp_init(seed=seed, device=F.device)
    curve = mlp_train(params, Fs, target, steps=steps, lr=lr, batch=batch, seed=seed)
    _check(L.psvd_mlp_fold(_ptr(params), _ptr(stats), _stream()), "psvd_mlp_fold")
    return params, curve


def mlp_calibrate(params: torch.Tensor, feats: torch.Tensor, target: torch.Tensor, quantile: float = 0.98) -> float:
    """Safety margin for the predicted lower bound: exp(-q) with q the given quantile of the
    over-prediction y - target on (held-out) training data (psvd_mlp_calibrate), so that about
    that fraction of bounds are true lower bounds; over-predictions are caught by the
    conservative rerun."""
    F = feats.contiguous().float()
    tg = target.contiguous().float()
    y = torch.empty(F.shape[0], device=F.device)
    margin = torch.empty(1, device=F.device)
    _check(lib().psvd_mlp_calibrate(_ptr(params), _ptr(F), _ptr(tg), F.shape[0], float(quantile), _ptr(y),
                                    _ptr(margin), _stream()), "psvd_mlp_calibrate")
    return float(margin.item())


def predict_lower_bound(a: torch.Tensor, params: torch.Tensor, margin: float = 0.5, probes: int = 8,
                        seed: int = 0, z: torch.Tensor | None = None) -> torch.Tensor:
    """Per-matrix lower bound of sigma_min(X0) for the learned schedule: margin * exp(MLP(features)),
    all on the device (sketch kernels, then psvd_mlp_lower_bound).  `z`: probes drawn in advance."""
    A, _ = _batched(a)
    Z = z if z is not None else rademacher_probes(A.shape[0], A.shape[2], probes, seed, A.device)
    F = sketch_features(A, Z)
    lb = torch.empty(F.shape[0], device=F.device, dtype=torch.float32)
    _check(lib().psvd_mlp_lower_bound(_ptr(params), _ptr(F), _ptr(lb), F.shape[0], float(margin), _stream()),
           "psvd_mlp_lower_bound")
    return lb
