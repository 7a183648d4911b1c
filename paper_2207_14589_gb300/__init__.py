"""Thin Python binding of libsped (the C ABI in include/sped.h) for PyTorch tensors.

Argument marshalling only: every step of the hot path runs in the CUDA kernels of libsped.
PyTorch provides device memory (inputs, outputs and the scratch buffers the library asks for)
and the current CUDA stream. There is no CPU fallback: if the extension is missing or no CUDA
device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsped.so")

# enums (mirror include/sped.h)
OK, ERR_INVALID_ARG, ERR_BAD_CSR, ERR_UNSUPPORTED, ERR_NUMERIC, ERR_NOT_CONVERGED, \
    ERR_TIMEOUT, ERR_CUDA, ERR_SCRATCH = range(9)
BF16, F32, F64 = 0, 1, 2
POLY_LIMIT_EXP, POLY_TAYLOR_EXP, POLY_TAYLOR_LOG, POLY_MONOMIAL, POLY_SHIFT, POLY_CHEBYSHEV = range(6)
(EXACT, STOCHASTIC_IS, STOCHASTIC_REJECT, STOCHASTIC_MINIBATCH,
 STOCHASTIC_MINIBATCH_STRATIFIED) = range(5)
MU_EG, OJA = 0, 1

_STATUS = {0: "OK", 1: "INVALID_ARG", 2: "BAD_CSR", 3: "UNSUPPORTED", 4: "NUMERIC",
           5: "NOT_CONVERGED", 6: "TIMEOUT", 7: "CUDA", 8: "SCRATCH"}

_TORCH_DT = {torch.bfloat16: BF16, torch.float32: F32, torch.float64: F64}
_DT_TORCH = {v: k for k, v in _TORCH_DT.items()}
_DT_SIZE = {BF16: 2, F32: 4, F64: 8}


class SpedError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"sped {_STATUS.get(status, status)}: {msg}")
        self.status = status


class sped_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("n_edges", ctypes.c_int64),
                ("max_degree", ctypes.c_int32), ("max_wdegree", ctypes.c_double),
                ("lambda_bound", ctypes.c_double), ("weighted", ctypes.c_int),
                ("poly_kind", ctypes.c_int), ("degree", ctypes.c_int),
                ("scale_s", ctypes.c_double), ("shift", ctypes.c_double),
                ("lambda_star", ctypes.c_double)]


class sped_step_opts(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("eta", ctypes.c_double), ("chain_t", ctypes.c_int),
                ("y_t", ctypes.c_int), ("mode", ctypes.c_int), ("walkers", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("ev_chain_begin", ctypes.c_void_p),
                ("ev_chain_end", ctypes.c_void_p), ("v_shadow", ctypes.c_void_p),
                ("shadow_ld", ctypes.c_int), ("shadow_valid", ctypes.c_int)]


class sped_solve_opts(ctypes.Structure):
    _fields_ = [("step", sped_step_opts), ("max_steps", ctypes.c_int),
                ("check_every", ctypes.c_int), ("tol", ctypes.c_double),
                ("switch_tol", ctypes.c_double), ("phase1_steps", ctypes.c_int),
                ("refine_chain_t", ctypes.c_int)]


class sped_tune_report(ctypes.Structure):
    _fields_ = [("split", ctypes.c_int), ("merge_ipg", ctypes.c_int), ("cached", ctypes.c_int),
                ("n_candidates", ctypes.c_int), ("ms", ctypes.c_double * 8)]


class sped_batch_tune_report(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("cached", ctypes.c_int),
                ("n_candidates", ctypes.c_int), ("ms", ctypes.c_double * 8)]


class sped_solve_report(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("phase1_steps", ctypes.c_int),
                ("spmm_count", ctypes.c_int64), ("final_residual", ctypes.c_double),
                ("converged", ctypes.c_int)]


_lib = None


def lib():
    """The loaded libsped (ctypes). Raises if the extension has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libsped.so not built ({LIB_PATH}); run "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u64, dbl, sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                  ctypes.c_double, ctypes.c_size_t)
    P = ctypes.POINTER
    sigs = {
        "sped_workspace_size": [i64, i64, P(sz)],
        "sped_build_laplacian": [i64, i64, vp, vp, vp, vp, sz, i32, vp, P(vp)],
        "sped_graph_get_info": [vp, P(sped_graph_info)],
        "sped_graph_edges": [vp, vp, vp, vp],
        "sped_set_edge_weights": [vp, vp, vp],
        "sped_set_polynomial": [vp, i32, i32, dbl, dbl, P(dbl), dbl],
        "sped_get_power_coeffs": [vp, P(dbl), i32],
        "sped_poly_step": [vp, i32, vp, i32, i32, vp, i32, i32, vp, i32, i32, dbl, dbl, dbl, i32,
                           vp, sz, vp],
        "sped_poly_step_scratch_size": [vp, i32, i32, i32, P(sz)],
        "sped_apply_poly": [vp, i32, vp, i32, i32, vp, i32, i32, i32, i32, i64, u64, vp, sz, vp],
        "sped_apply_poly_scratch_size": [vp, i32, i32, i32, P(sz)],
        "sped_apply_poly_backward": [vp, i32, vp, i32, i32, vp, i32, i32, i32, vp, sz, vp],
        "sped_gram": [i64, vp, i32, i32, i32, vp, i32, i32, i32, vp, vp, sz, vp],
        "sped_gram_scratch_size": [i64, i32, i32, P(sz)],
        "sped_eig_step": [vp, P(sped_step_opts), vp, i32, i32, i32, vp, vp, sz, vp],
        "sped_eig_step_scratch_size": [vp, P(sped_step_opts), i32, P(sz)],
        "sped_rayleigh": [vp, vp, i32, i32, i32, vp, vp, sz, vp],
        "sped_rayleigh_scratch_size": [vp, i32, P(sz)],
        "sped_rayleigh_ritz": [vp, vp, i32, i32, i32, vp, vp, i32, vp, sz, vp],
        "sped_rayleigh_ritz_scratch_size": [vp, i32, P(sz)],
        "sped_solve_bottom_k": [vp, P(sped_solve_opts), vp, i32, i32, i32, P(dbl),
                                P(sped_solve_report), vp, sz, vp],
        "sped_solve_scratch_size": [vp, P(sped_solve_opts), i32, P(sz)],
        "sped_cluster_assign": [vp, i32, i64, i32, i32, i32, u64, i32, vp, P(i32), vp, sz, vp],
        "sped_cluster_scratch_size": [i64, i32, i32, P(sz)],
        "sped_autotune_scratch_size": [vp, i32, i32, P(sz)],
        "sped_autotune": [vp, i32, i32, vp, sz, vp, P(sped_tune_report)],
        "sped_set_schedule": [vp, i32, i32],
        "sped_poly_moments": [vp, vp, i32, i32, i32, i32, i32, dbl, dbl, vp, vp, sz, vp],
        "sped_poly_moments_scratch_size": [vp, i32, i32, P(sz)],
        "sped_device_status": [vp],
        "sped_test_gram_waits": [ctypes.c_uint32, i32],
        "sped_sample_edges": [vp, u64, ctypes.c_uint32, i64, i32, vp, vp, vp, vp, vp],
        "sped_edge_step": [i64, i32, vp, vp, vp, i64, dbl, vp, i32, i32, vp, i32, i32, vp, i32,
                           i32, dbl, dbl, dbl, vp, vp],
    }
    for name, args in sigs.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.sped_graph_destroy.argtypes = [vp]
    L.sped_graph_destroy.restype = None
    L.sped_last_error.restype = ctypes.c_char_p
    L.sped_version.restype = ctypes.c_char_p
    _lib = L
    return L


def _check(status):
    if status != OK:
        raise SpedError(status, lib().sped_last_error().decode())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _scratch(nbytes, device):
    # 256-byte aligned raw device bytes (torch's caching allocator aligns to >= 512)
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def padded_ld(k, dtype):
    e = 16 // _DT_SIZE[_TORCH_DT[dtype]]
    return (k + e - 1) // e * e


def alloc_block(n, k, dtype=torch.float32, device="cuda", fill=None):
    """n x k block with the row padding the vector path wants; returns the (n, ld) storage."""
    ld = padded_ld(k, dtype)
    t = torch.zeros((n, ld), dtype=dtype, device=device) if fill is None else \
        torch.full((n, ld), fill, dtype=dtype, device=device)
    return t


def _block(t, k):
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("block tensors must be 2-D with unit column stride")
    if t.dtype not in _TORCH_DT:
        raise TypeError(f"unsupported dtype {t.dtype}")
    if not t.is_cuda:
        raise ValueError("block tensors must live on a CUDA device")
    return _TORCH_DT[t.dtype], t.stride(0)


def version():
    return lib().sped_version().decode()


@dataclass
class GraphInfo:
    n: int
    nnz: int
    n_edges: int
    max_degree: int
    max_wdegree: float
    lambda_bound: float
    weighted: bool
    poly_kind: int
    degree: int
    scale_s: float
    shift: float
    lambda_star: float


class Graph:
    """A graph Laplacian L = D - A resident on the GPU (Section 2 of the paper).

    Holds the CSR tensors, the library workspace and the opaque handle."""

    def __init__(self, row_ptr, col_idx, w=None, check=True, stream=None):
        L = lib()
        dev = row_ptr.device
        self.row_ptr = row_ptr.to(torch.int32).contiguous()
        self.col_idx = col_idx.to(torch.int32).contiguous()
        self.w = None if w is None else w.to(torch.float32).contiguous()
        self.n = self.row_ptr.numel() - 1
        self.nnz = self.col_idx.numel()
        ws = ctypes.c_size_t()
        _check(L.sped_workspace_size(self.n, self.nnz, ctypes.byref(ws)))
        self.workspace = _scratch(ws.value, dev)
        h = ctypes.c_void_p()
        _check(L.sped_build_laplacian(self.n, self.nnz, _ptr(self.row_ptr), _ptr(self.col_idx),
                                      _ptr(self.w), _ptr(self.workspace), ws.value, int(check),
                                      _stream(stream), ctypes.byref(h)))
        self.handle = h
        self.device = dev
        self._edge_w = None

    @classmethod
    def from_csr(cls, g, device="cuda", check=True):
        """From a host CSR graph (an object with n, row_ptr, col_idx and optional w arrays)."""
        rp = torch.from_numpy(g.row_ptr).to(device)
        ci = torch.from_numpy(g.col_idx).to(device)
        w = None if g.w is None else torch.from_numpy(g.w).to(device)
        return cls(rp, ci, w, check=check)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.sped_graph_destroy(h)
            self.handle = None

    def info(self) -> GraphInfo:
        i = sped_graph_info()
        _check(lib().sped_graph_get_info(self.handle, ctypes.byref(i)))
        return GraphInfo(i.n, i.nnz, i.n_edges, i.max_degree, i.max_wdegree, i.lambda_bound,
                         bool(i.weighted), i.poly_kind, i.degree, i.scale_s, i.shift,
                         i.lambda_star)

    def edges(self, stream=None):
        ne = self.info().n_edges
        a = torch.empty(ne, dtype=torch.int32, device=self.device)
        b = torch.empty(ne, dtype=torch.int32, device=self.device)
        _check(lib().sped_graph_edges(self.handle, _ptr(a), _ptr(b), _stream(stream)))
        return a, b

    def set_edge_weights(self, w_edge, stream=None):
        self._edge_w = w_edge.to(torch.float32).contiguous()
        _check(lib().sped_set_edge_weights(self.handle, _ptr(self._edge_w), _stream(stream)))

    def set_polynomial(self, kind=POLY_LIMIT_EXP, degree=1, scale=0.0, eps=0.0, coeffs=None,
                       lambda_star=0.0):
        c = None
        if coeffs is not None:
            arr = (ctypes.c_double * len(coeffs))(*[float(x) for x in coeffs])
            c = arr
        _check(lib().sped_set_polynomial(self.handle, kind, degree, float(scale), float(eps),
                                         c, float(lambda_star)))
        return self.info()

    def autotune(self, k, chain_dtype=torch.bfloat16, stream=None):
        """Time the chain-step schedules on this graph and keep the fastest (sped_autotune)."""
        ct = _TORCH_DT[chain_dtype]
        nb = ctypes.c_size_t()
        _check(lib().sped_autotune_scratch_size(self.handle, k, ct, ctypes.byref(nb)))
        scr = _scratch(nb.value, self.device)
        rep = sped_tune_report()
        _check(lib().sped_autotune(self.handle, k, ct, _ptr(scr), nb.value, _stream(stream),
                                   ctypes.byref(rep)))
        return {"split": rep.split, "merge_ipg": rep.merge_ipg, "cached": bool(rep.cached),
                "ms": list(rep.ms[:rep.n_candidates])}

    def set_schedule(self, split=0, merge_ipg=0):
        _check(lib().sped_set_schedule(self.handle, int(split), int(merge_ipg)))

    def power_coeffs(self):
        d = self.info().degree
        out = (ctypes.c_double * (d + 1))()
        _check(lib().sped_get_power_coeffs(self.handle, out, d + 1))
        return list(out)


# ----------------------------------------------------------------------------------------
# operations
# ----------------------------------------------------------------------------------------
def poly_step(g: Graph, X, Y, k, alpha=0.0, beta=1.0, gamma=0.0, V=None, split=0, stream=None):
    """Y = alpha V + gamma X + beta L X (the fused chain step)."""
    xt, ldx = _block(X, k)
    yt, ldy = _block(Y, k)
    vt, ldv = _block(V, k) if V is not None else (F32, k)
    nb = ctypes.c_size_t()
    _check(lib().sped_poly_step_scratch_size(g.handle, k, xt, split, ctypes.byref(nb)))
    scr = _scratch(nb.value, X.device) if nb.value else None
    _check(lib().sped_poly_step(g.handle, k, _ptr(X), xt, ldx, _ptr(V), vt, ldv, _ptr(Y), yt,
                                ldy, float(alpha), float(beta), float(gamma), split, _ptr(scr),
                                nb.value, _stream(stream)))
    return Y


def apply_poly_scratch_bytes(g: Graph, k, chain_dtype=torch.float32, mode=EXACT):
    nb = ctypes.c_size_t()
    _check(lib().sped_apply_poly_scratch_size(g.handle, k, _TORCH_DT[chain_dtype], mode,
                                              ctypes.byref(nb)))
    return nb.value


def apply_poly(g: Graph, V, Y, k, chain_dtype=None, mode=EXACT, walkers=0, seed=0,
               scratch=None, stream=None):
    """Y = M V for the graph's polynomial (exact chain or stochastic estimate)."""
    vt, ldv = _block(V, k)
    yt, ldy = _block(Y, k)
    ct = _TORCH_DT[chain_dtype] if chain_dtype is not None else vt
    if scratch is None:
        nb = apply_poly_scratch_bytes(g, k, _DT_TORCH[ct], mode)
        scratch = _scratch(nb, V.device)
    _check(lib().sped_apply_poly(g.handle, k, _ptr(V), vt, ldv, _ptr(Y), yt, ldy, ct, mode,
                                 int(walkers), int(seed), _ptr(scratch), scratch.numel(),
                                 _stream(stream)))
    return Y


def poly_moments(g: Graph, V, k, n_moments, basis="chebyshev", a=0.0, b=0.0, stream=None):
    """Block moments V^T B_l V (FP64, n_moments x k x k) of the power ("power") or Chebyshev
    ("chebyshev", on [a, b]; b = 0: the spectral bound) basis."""
    vt, ld = _block(V, k)
    nb = ctypes.c_size_t()
    _check(lib().sped_poly_moments_scratch_size(g.handle, k, vt, ctypes.byref(nb)))
    scr = _scratch(nb.value, V.device)
    out = torch.empty((n_moments, k, k), dtype=torch.float64, device=V.device)
    _check(lib().sped_poly_moments(g.handle, _ptr(V), vt, k, ld, 0 if basis == "power" else 1,
                                   int(n_moments), float(a), float(b), _ptr(out), _ptr(scr),
                                   nb.value, _stream(stream)))
    return out


def sample_edges(g: Graph, seed, step, count, stratified=False, stream=None):
    """The edge minibatch that STOCHASTIC_MINIBATCH (or, stratified, STOCHASTIC_MINIBATCH_
    STRATIFIED) draws for multiplication `step`: (a, b, w) device tensors (int32, int32,
    float32) of length count, a < b; stratified draws add the stratum sizes (int32)."""
    dev = torch.device("cuda", torch.cuda.current_device())
    a = torch.empty(max(int(count), 1), dtype=torch.int32, device=dev)
    b = torch.empty_like(a)
    w = torch.empty(max(int(count), 1), dtype=torch.float32, device=dev)
    size = torch.empty_like(a) if stratified else None
    _check(lib().sped_sample_edges(g.handle, int(seed), int(step), int(count), int(stratified),
                                   _ptr(a), _ptr(b), _ptr(w), _ptr(size), _stream(stream)))
    if stratified:
        return a[:count], b[:count], w[:count], size[:count]
    return a[:count], b[:count], w[:count]


def edge_step(n, X, Y, k, a, b, w=None, edge_scale=1.0, alpha=0.0, beta=1.0, gamma=0.0, V=None,
              skipped=None, stream=None):
    """Y = alpha V + gamma X + beta * edge_scale * sum_j w_j x_j x_j^T X for the caller's edge
    minibatch (a, b, w: int32 / int32 / float32 device tensors)."""
    xt, ldx = _block(X, k)
    yt, ldy = _block(Y, k)
    vt, ldv = _block(V, k) if V is not None else (F32, k)
    for t, dt in ((a, torch.int32), (b, torch.int32)) + (((w, torch.float32),) if w is not None
                                                         else ()):
        if t.dtype != dt or not t.is_contiguous():
            raise TypeError("edge arrays: contiguous int32 endpoints, float32 weights")
        if t.numel() != a.numel():
            raise ValueError("edge arrays of different lengths")
    _check(lib().sped_edge_step(int(n), k, _ptr(a), _ptr(b), _ptr(w), int(a.numel()),
                                float(edge_scale), _ptr(X), xt, ldx, _ptr(V), vt, ldv, _ptr(Y), yt,
                                ldy, float(alpha), float(beta), float(gamma), _ptr(skipped),
                                _stream(stream)))
    return Y


def apply_poly_backward(g: Graph, dY, dV, k, chain_dtype=None, scratch=None, stream=None):
    """dV = M^T dY = M dY (M = p(L) symmetric): the backward of Y = M V with respect to V."""
    yt, ldy = _block(dY, k)
    vt, ldv = _block(dV, k)
    ct = _TORCH_DT[chain_dtype] if chain_dtype is not None else yt
    if scratch is None:
        scratch = _scratch(apply_poly_scratch_bytes(g, k, _DT_TORCH[ct]), dY.device)
    _check(lib().sped_apply_poly_backward(g.handle, k, _ptr(dY), yt, ldy, _ptr(dV), vt, ldv, ct,
                                          _ptr(scratch), scratch.numel(), _stream(stream)))
    return dV


def gram(A, ka, B=None, kb=0, G=None, scratch=None, stream=None):
    """G = [A B]^T [A B] in FP64 ((ka+kb) x (ka+kb))."""
    at, lda = _block(A, ka)
    bt, ldb = _block(B, kb) if B is not None else (at, lda)
    n = A.shape[0]
    K2 = ka + kb
    if G is None:
        G = torch.empty((K2, K2), dtype=torch.float64, device=A.device)
    if scratch is None:
        nb = ctypes.c_size_t()
        _check(lib().sped_gram_scratch_size(n, ka, kb, ctypes.byref(nb)))
        scratch = _scratch(nb.value, A.device)
    _check(lib().sped_gram(n, _ptr(A), at, lda, ka, _ptr(B), bt, ldb, kb, _ptr(G),
                           _ptr(scratch), scratch.numel(), _stream(stream)))
    return G


def device_status(stream=None):
    """Synchronise the stream and raise SpedError(ERR_TIMEOUT) if a bounded device-side wait gave
    up since the last check (sped_device_status); the status word is cleared."""
    _check(lib().sped_device_status(_stream(stream)))


def test_gram_waits(wait_limit=0, skip_fills=False):
    """Test control of the tensor-core Gram's bounded waits (sped_test_gram_waits)."""
    _check(lib().sped_test_gram_waits(int(wait_limit), int(bool(skip_fills))))


def step_opts(solver=MU_EG, eta=1.0, chain_dtype=torch.float32, y_dtype=torch.float32,
              mode=EXACT, walkers=0, seed=0, v_shadow=None, shadow_valid=False):
    """Options of one solver step. v_shadow: optional BF16 block (alloc_block(n, k, bfloat16))
    that the update keeps equal to bf16(V); shadow_valid says it already holds bf16(V), so a
    BF16 chain starts from it."""
    o = sped_step_opts(solver, float(eta), _TORCH_DT[chain_dtype], _TORCH_DT[y_dtype], mode,
                       int(walkers), int(seed), None, None, None, 0, 0)
    if v_shadow is not None:
        if v_shadow.dtype != torch.bfloat16:
            raise ValueError("the shadow of V is a bfloat16 block")
        o.v_shadow = v_shadow.data_ptr()
        o.shadow_ld = v_shadow.stride(0)
        o.shadow_valid = int(bool(shadow_valid))
    return o


def eig_step_scratch_bytes(g: Graph, opts: sped_step_opts, k):
    nb = ctypes.c_size_t()
    _check(lib().sped_eig_step_scratch_size(g.handle, ctypes.byref(opts), k, ctypes.byref(nb)))
    return nb.value


def eig_step(g: Graph, V, k, opts: sped_step_opts, stats=None, scratch=None, stream=None):
    """One solver step on the graph's operator, V updated in place."""
    vt, ld = _block(V, k)
    if scratch is None:
        scratch = _scratch(eig_step_scratch_bytes(g, opts, k), V.device)
    _check(lib().sped_eig_step(g.handle, ctypes.byref(opts), _ptr(V), vt, k, ld, _ptr(stats),
                               _ptr(scratch), scratch.numel(), _stream(stream)))
    return V


def rayleigh(g: Graph, V, k, out=None, stream=None):
    vt, ld = _block(V, k)
    nb = ctypes.c_size_t()
    _check(lib().sped_rayleigh_scratch_size(g.handle, k, ctypes.byref(nb)))
    scr = _scratch(nb.value, V.device)
    if out is None:
        out = torch.empty(k, dtype=torch.float64, device=V.device)
    _check(lib().sped_rayleigh(g.handle, _ptr(V), vt, k, ld, _ptr(out), _ptr(scr), nb.value,
                               _stream(stream)))
    return out


def rayleigh_ritz(g: Graph, V, k, rotate=False, stream=None):
    """Ritz values (ascending, FP64) and coefficients W (V W = Ritz vectors) of L on span(V);
    rotate=True also replaces V by V W."""
    vt, ld = _block(V, k)
    nb = ctypes.c_size_t()
    _check(lib().sped_rayleigh_ritz_scratch_size(g.handle, k, ctypes.byref(nb)))
    scr = _scratch(nb.value, V.device)
    theta = torch.empty(k, dtype=torch.float64, device=V.device)
    W = torch.empty((k, k), dtype=torch.float64, device=V.device)
    _check(lib().sped_rayleigh_ritz(g.handle, _ptr(V), vt, k, ld, _ptr(theta), _ptr(W),
                                    int(bool(rotate)), _ptr(scr), nb.value, _stream(stream)))
    return theta, W


def solve_opts(solver=MU_EG, eta=1.0, chain_dtype=torch.bfloat16, y_dtype=torch.float32,
               max_steps=100, check_every=1, tol=1e-6, switch_tol=3e-3, phase1_steps=50,
               refine_dtype=torch.float32, mode=EXACT, walkers=0, seed=0):
    return sped_solve_opts(step_opts(solver, eta, chain_dtype, y_dtype, mode, walkers, seed),
                           int(max_steps), int(check_every), float(tol), float(switch_tol),
                           int(phase1_steps), _TORCH_DT[refine_dtype])


def solve_bottom_k(g: Graph, V, k, opts: sped_solve_opts, raise_not_converged=False, stream=None):
    """Iterate eig_step to convergence; returns (eigenvalues of L as a list, report dict)."""
    vt, ld = _block(V, k)
    nb = ctypes.c_size_t()
    _check(lib().sped_solve_scratch_size(g.handle, ctypes.byref(opts), k, ctypes.byref(nb)))
    scr = _scratch(nb.value, V.device)
    lam = (ctypes.c_double * k)()
    rep = sped_solve_report()
    st = lib().sped_solve_bottom_k(g.handle, ctypes.byref(opts), _ptr(V), vt, k, ld, lam,
                                   ctypes.byref(rep), _ptr(scr), nb.value, _stream(stream))
    if st != OK and not (st == ERR_NOT_CONVERGED and not raise_not_converged):
        _check(st)
    return list(lam), dict(steps=rep.steps, phase1_steps=rep.phase1_steps,
                           spmm_count=rep.spmm_count, final_residual=rep.final_residual,
                           converged=bool(rep.converged))


def cluster_assign(V, k, n_clusters, seed=0, max_iter=100, stream=None):
    """k-means labels (int32) of the rows of V."""
    vt, ld = _block(V, k)
    n = V.shape[0]
    nb = ctypes.c_size_t()
    _check(lib().sped_cluster_scratch_size(n, k, n_clusters, ctypes.byref(nb)))
    scr = _scratch(nb.value, V.device)
    labels = torch.empty(n, dtype=torch.int32, device=V.device)
    iters = ctypes.c_int()
    _check(lib().sped_cluster_assign(_ptr(V), vt, n, k, ld, n_clusters, int(seed), int(max_iter),
                                     _ptr(labels), ctypes.byref(iters), _ptr(scr), nb.value,
                                     _stream(stream)))
    return labels, iters.value


# ----------------------------------------------------------------------------------------
# batched: many graphs in one persistent launch
# ----------------------------------------------------------------------------------------
class Batch:
    """Independent graphs stored as one block-diagonal CSR (global node ids), solved together
    by sped_batch_eig_steps."""

    def __init__(self, node_off, row_ptr, col_idx, w=None, degree=31, check=True, stream=None):
        L = lib()
        _batch_sigs(L)
        self.node_off = [int(x) for x in node_off]
        self.n_graphs = len(self.node_off) - 1
        self.row_ptr = row_ptr.to(torch.int32).contiguous()
        self.col_idx = col_idx.to(torch.int32).contiguous()
        self.w = None if w is None else w.to(torch.float32).contiguous()
        self.n_total = self.node_off[-1]
        self.device = self.row_ptr.device
        nb = ctypes.c_size_t()
        _check(L.sped_batch_workspace_size(self.n_graphs, ctypes.byref(nb)))
        self.workspace = _scratch(nb.value, self.device)
        off = (ctypes.c_int64 * (self.n_graphs + 1))(*self.node_off)
        h = ctypes.c_void_p()
        _check(L.sped_batch_create(self.n_graphs, off, _ptr(self.row_ptr), _ptr(self.col_idx),
                                   _ptr(self.w), int(degree), int(check), _ptr(self.workspace),
                                   nb.value, _stream(stream), ctypes.byref(h)))
        self.handle = h
        self.degree = degree

    @classmethod
    def from_graphs(cls, graphs, degree=31, device="cuda", check=True):
        """Block-diagonal union of host CSR graphs (objects with n, row_ptr, col_idx and an
        optional w, all or none weighted), column ids shifted to global node ids."""
        import numpy as np
        n = np.array([g.n for g in graphs], dtype=np.int64)
        nnz = np.array([len(g.col_idx) for g in graphs], dtype=np.int64)
        node_off = np.concatenate([[0], np.cumsum(n)])
        nnz_off = np.concatenate([[0], np.cumsum(nnz)])
        if nnz_off[-1] > np.iinfo(np.int32).max or node_off[-1] > np.iinfo(np.int32).max:
            raise ValueError("batch exceeds int32 indexing")
        rp = np.empty(node_off[-1] + 1, dtype=np.int32)
        ci = np.empty(nnz_off[-1], dtype=np.int32)
        weighted = graphs[0].w is not None
        if any((g.w is not None) != weighted for g in graphs):
            raise ValueError("batch mixes weighted and unweighted graphs")
        wv = np.empty(nnz_off[-1], dtype=np.float32) if weighted else None
        rp[0] = 0
        for i, g in enumerate(graphs):
            rp[node_off[i] + 1: node_off[i + 1] + 1] = np.asarray(g.row_ptr[1:], np.int64) + nnz_off[i]
            ci[nnz_off[i]: nnz_off[i + 1]] = np.asarray(g.col_idx, np.int64) + node_off[i]
            if weighted:
                wv[nnz_off[i]: nnz_off[i + 1]] = g.w
        w = None if wv is None else torch.from_numpy(wv).to(device)
        return cls(node_off, torch.from_numpy(rp).to(device), torch.from_numpy(ci).to(device),
                   w, degree=degree, check=check)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h and _lib is not None:
            _lib.sped_batch_destroy(h)
            self.handle = None

    def scales(self):
        out = (ctypes.c_double * self.n_graphs)()
        _check(lib().sped_batch_scale(self.handle, out, self.n_graphs))
        return list(out)

    def scratch_bytes(self, k, chain_dtype=torch.bfloat16):
        nb = ctypes.c_size_t()
        _check(lib().sped_batch_scratch_size(self.handle, k, _TORCH_DT[chain_dtype],
                                             ctypes.byref(nb)))
        return nb.value

    def set_schedule(self, threads=512, ctas_per_sm=2):
        _check(lib().sped_batch_set_schedule(self.handle, int(threads), int(ctas_per_sm)))

    def autotune(self, V, k, chain_dtype=torch.bfloat16, stream=None):
        """Time the candidate schedules on a copy of V; the fastest is kept (dict report)."""
        nb = ctypes.c_size_t()
        _check(lib().sped_batch_autotune_scratch_size(self.handle, k, _TORCH_DT[chain_dtype],
                                                      ctypes.byref(nb)))
        scr = _scratch(nb.value, V.device)
        rep = sped_batch_tune_report()
        _check(lib().sped_batch_autotune(self.handle, k, _TORCH_DT[chain_dtype], _ptr(V),
                                         V.stride(0), _ptr(scr), nb.value, _stream(stream),
                                         ctypes.byref(rep)))
        return dict(threads=rep.threads, ctas_per_sm=rep.ctas_per_sm, cached=bool(rep.cached),
                    ms=[rep.ms[i] for i in range(rep.n_candidates)])

    def eig_steps(self, V, k, steps=1, eta=1.0, chain_dtype=torch.bfloat16, ritz=None,
                  scratch=None, stream=None):
        if V.dtype != torch.float32 or V.dim() != 2 or V.stride(1) != 1:
            raise ValueError("batched V must be a 2-D float32 block")
        if ritz is None:
            ritz = torch.empty((self.n_graphs, k), dtype=torch.float64, device=V.device)
        if scratch is None:
            scratch = _scratch(self.scratch_bytes(k, chain_dtype), V.device)
        _check(lib().sped_batch_eig_steps(self.handle, int(steps), float(eta),
                                          _TORCH_DT[chain_dtype], _ptr(V), k, V.stride(0),
                                          _ptr(ritz), _ptr(scratch), scratch.numel(),
                                          _stream(stream)))
        return V, ritz


def batch_block(n_total, k, device="cuda"):
    """Float32 master block for the batched solver (ld 8 for k <= 8, else 16)."""
    return torch.zeros((n_total, 8 if k <= 8 else 16), dtype=torch.float32, device=device)


_batch_ready = False


def _batch_sigs(L):
    global _batch_ready
    if _batch_ready:
        return
    vp, i32, i64, dbl, sz = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                             ctypes.c_size_t)
    P = ctypes.POINTER
    for name, args in {
        "sped_batch_workspace_size": [i64, P(sz)],
        "sped_batch_create": [i64, P(ctypes.c_int64), vp, vp, vp, i32, i32, vp, sz, vp, P(vp)],
        "sped_batch_scale": [vp, P(dbl), i32],
        "sped_batch_scratch_size": [vp, i32, i32, P(sz)],
        "sped_batch_eig_steps": [vp, i32, dbl, i32, vp, i32, i32, vp, vp, sz, vp],
        "sped_batch_set_schedule": [vp, i32, i32],
        "sped_batch_autotune_scratch_size": [vp, i32, i32, P(sz)],
        "sped_batch_autotune": [vp, i32, i32, vp, i32, vp, sz, vp, P(sped_batch_tune_report)],
    }.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.sped_batch_destroy.argtypes = [vp]
    L.sped_batch_destroy.restype = None
    _batch_ready = True


# ----------------------------------------------------------------------------------------
# differentiable utilities
# ----------------------------------------------------------------------------------------
_diff_ready = False


def _diff_sigs(L):
    global _diff_ready
    if _diff_ready:
        return
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    P = ctypes.POINTER
    for name, args in {
        "sped_eg_utilities": [i32, vp, i32, vp, vp, vp, vp, vp],
        "sped_block_combine": [i64, i32, vp, i32, vp, vp, i32, vp, vp, i32, i32, vp],
        "sped_edge_grad": [vp, vp, i32, i32, i32, vp, vp, vp, sz, vp],
        "sped_edge_grad_scratch_size": [vp, i32, i32, P(sz)],
    }.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    _diff_ready = True


def eg_utilities(G, k, g_u=None, stream=None):
    """From the Gram G = [V Y]^T [V Y] (2k x 2k FP64, Y = M V): utilities u (k), and when
    g_u is given Hbar = d(sum g_i u_i)/dH; also the detached-parents coefficients S."""
    L = lib()
    _diff_sigs(L)
    dev = G.device
    H = G[:, k:]  # rows 0..k-1 used, row stride 2k
    u = torch.empty(k, dtype=torch.float64, device=dev)
    S = torch.empty((k, k), dtype=torch.float64, device=dev)
    Hbar = None
    gg = None
    if g_u is not None:
        gg = g_u.to(dtype=torch.float64, device=dev).contiguous()
        Hbar = torch.empty((k, k), dtype=torch.float64, device=dev)
    _check(L.sped_eg_utilities(k, ctypes.c_void_p(H.data_ptr()), G.stride(0), _ptr(gg), _ptr(u),
                               _ptr(Hbar), _ptr(S), _stream(stream)))
    return u, Hbar, S


def block_combine(A, k, P, B=None, Q=None, out=None, stream=None):
    """out = A P + B Q (n x k blocks, k x k FP64 coefficient matrices)."""
    L = lib()
    _diff_sigs(L)
    t, lda = _block(A, k)
    ldb = B.stride(0) if B is not None else 0
    if out is None:
        out = torch.zeros_like(A)
    _check(L.sped_block_combine(A.shape[0], k, _ptr(A), lda, _ptr(P.contiguous()), _ptr(B), ldb,
                                _ptr(Q.contiguous() if Q is not None else None), _ptr(out),
                                out.stride(0), t, _stream(stream)))
    return out


def edge_grad(g: Graph, V, k, HbarT, stream=None):
    """d f / d w_e for every undirected edge (FP64), f(H) with df/dH = Hbar."""
    L = lib()
    _diff_sigs(L)
    t, ld = _block(V, k)
    nb = ctypes.c_size_t()
    _check(L.sped_edge_grad_scratch_size(g.handle, k, t, ctypes.byref(nb)))
    scr = _scratch(nb.value, V.device)
    out = torch.empty(g.info().n_edges, dtype=torch.float64, device=V.device)
    _check(L.sped_edge_grad(g.handle, _ptr(V), t, k, ld, _ptr(HbarT.contiguous()), _ptr(out),
                            _ptr(scr), nb.value, _stream(stream)))
    return out


class EigenGameUtility(torch.autograd.Function):
    """u = EigenGame utilities of the columns of V under M = (I - sL(w))^l.

    Inputs: V (n x ld padded block, F32 or F64; the first k columns are the players), w (one
    weight per undirected edge, the graph's learnable weights), the Graph (limit form set) and
    k. Backward: dV = Y Hbar^T + M (V Hbar) (adjoint polynomial chain) and dw by the
    checkpointed SDDMM (sped_edge_grad). Every step runs in libsped's kernels."""

    @staticmethod
    def forward(ctx, V, w, graph, k):
        graph.set_edge_weights(w.detach().to(torch.float32))
        Y = torch.zeros_like(V)
        apply_poly(graph, V, Y, k, chain_dtype=V.dtype)
        G = gram(V, k, Y, k)
        u, _, _ = eg_utilities(G, k)
        ctx.save_for_backward(V, Y, G)
        ctx.graph, ctx.k, ctx.w_dtype = graph, k, w.dtype
        return u

    @staticmethod
    def backward(ctx, g_u):
        V, Y, G = ctx.saved_tensors
        graph, k = ctx.graph, ctx.k
        _, Hbar, _ = eg_utilities(G, k, g_u)
        T = block_combine(V, k, Hbar)                      # V Hbar
        MT = torch.zeros_like(V)
        apply_poly(graph, T, MT, k, chain_dtype=V.dtype)   # adjoint chain: M^T = M
        eye = torch.eye(k, dtype=torch.float64, device=V.device)
        dV = block_combine(Y, k, Hbar.t().contiguous(), MT, eye)
        dw = edge_grad(graph, V, k, Hbar.t().contiguous())
        return dV, dw.to(ctx.w_dtype), None, None


def eigengame_utilities(V, w, graph, k):
    return EigenGameUtility.apply(V, w, graph, k)
