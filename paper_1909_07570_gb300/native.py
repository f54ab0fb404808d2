"""Thin ctypes binding of libnncandelinc.so (include/nncandelinc.h).

Argument marshalling only: every step of the computation runs in the CUDA
library. Tensors are torch CUDA tensors; the binding passes their data
pointers and the current torch stream. If the library is missing, every call
raises - there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

NNC_FP64, NNC_FP32, NNC_BF16_REFINE, NNC_FP32_SIMT = 0, 1, 2, 3

_STATUS = {
    0: "ok", -1: "invalid argument", -2: "negative input", -3: "non-finite value",
    -4: "CUDA error", -5: "allocation failed", -6: "unsupported", -7: "device wait timed out",
}

# Every symbol include/nncandelinc.h declares.
EXPORTED = ("ntd_fit", "ntd_fit_batched", "ntd_fit_small_batched", "nmf_fit_batched",
            "lifted_rel_err_batched", "nncp_core_fit", "nncp_core_fit_batched",
            "nncp_core_fit_batched_noalloc", "nnc_mode_product", "candelinc_lift",
            "recon_residual", "candelinc_lifted_grad", "candelinc_pg_fit",
            "nncp_tensor_fit", "nmf_fit", "candelinc_alg2",
            "nnc_status_string", "nnc_last_error_detail",
            "nnc_profile_enable", "nnc_profile_read", "nnc_kernel_launches",
            "nnc_autotune_enable", "nnc_wait_selftest", "nnc_debug_fail_alloc",
            "nnc_last_refine_sweep")


class NncError(RuntimeError):
    def __init__(self, fn, status, detail):
        self.status = status
        super().__init__(f"{fn} failed: {_STATUS.get(status, status)} ({status}) {detail}".rstrip())


class nnc_opts(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("refine_iters", ctypes.c_int), ("eps", ctypes.c_double),
                ("exact_every", ctypes.c_int), ("refine_tol", ctypes.c_double)]


class ntd_job(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("d", ctypes.c_int), ("dims", ctypes.c_int64 * 4),
                ("m", ctypes.c_int * 4), ("F", ctypes.c_void_p * 4), ("G", ctypes.c_void_p),
                ("trace", ctypes.c_void_p)]


class ntd_small_job(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("dims", ctypes.c_int * 3), ("m", ctypes.c_int * 3),
                ("F", ctypes.c_void_p * 3), ("G", ctypes.c_void_p)]


class nmf_job(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("N", ctypes.c_int), ("r", ctypes.c_int),
                ("m", ctypes.c_int), ("F", ctypes.c_void_p), ("B", ctypes.c_void_p)]


class lifted_job(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("dims", ctypes.c_int * 3), ("m", ctypes.c_int * 3),
                ("r", ctypes.c_int), ("F", ctypes.c_void_p * 3), ("B", ctypes.c_void_p * 3)]


class nncp_job(ctypes.Structure):
    _fields_ = [("G", ctypes.c_void_p), ("d", ctypes.c_int), ("m", ctypes.c_int * 4),
                ("r", ctypes.c_int), ("B", ctypes.c_void_p * 4)]


_lib = None


def load(path: str | None = None):
    """Load the library (once). Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"libnncandelinc.so not found at {path}: run "
                           "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(path)
    vp, i64p, ip, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int), \
        ctypes.POINTER(ctypes.c_double)
    vpp = ctypes.POINTER(ctypes.c_void_p)
    lib.ntd_fit.argtypes = [vp, ctypes.c_int, i64p, ip, ctypes.c_int, ctypes.POINTER(nnc_opts), vpp,
                            vp, vp, dp, vp]
    lib.nncp_core_fit.argtypes = [vp, ctypes.c_int, ip, ctypes.c_int, ctypes.c_int,
                                  ctypes.POINTER(nnc_opts), vpp, dp, vp]
    lib.nncp_core_fit_batched.argtypes = [ctypes.c_int, ctypes.POINTER(nncp_job), ctypes.c_int,
                                          ctypes.POINTER(nnc_opts), vp, vp, vp]
    lib.candelinc_lift.argtypes = [ctypes.c_int, i64p, ip, ctypes.c_int, ctypes.c_int, vpp, vpp,
                                   vpp, vp]
    lib.recon_residual.argtypes = [vp, ctypes.c_int, i64p, ctypes.c_int, ctypes.c_int, ip,
                                   ctypes.c_int, vpp, vp, dp, dp, vp]
    lib.nncp_core_fit_batched_noalloc.argtypes = lib.nncp_core_fit_batched.argtypes
    lib.nnc_mode_product.argtypes = [vp, ctypes.c_int, i64p, ctypes.c_int, vp, ctypes.c_int,
                                     ctypes.c_int, vp, vp]
    lib.candelinc_lifted_grad.argtypes = [vp, ctypes.c_int, i64p, ip, ctypes.c_int, ctypes.c_int,
                                          vpp, vpp, vpp, vpp, dp, vp]
    lib.candelinc_pg_fit.argtypes = [vp, ctypes.c_int, i64p, ip, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, vpp, vpp, vp, dp, vp]
    lib.ntd_fit_batched.argtypes = [ctypes.c_int, ctypes.POINTER(ntd_job), ctypes.c_int,
                                    ctypes.POINTER(nnc_opts), ctypes.c_int, dp, ip, vp]
    lib.ntd_fit_small_batched.argtypes = [ctypes.c_int, ctypes.POINTER(ntd_small_job), ctypes.c_int,
                                          ctypes.POINTER(nnc_opts), vp, vp]
    lib.nmf_fit_batched.argtypes = [ctypes.c_int, ctypes.POINTER(nmf_job), ctypes.c_int,
                                    ctypes.POINTER(nnc_opts), vp, vp]
    lib.lifted_rel_err_batched.argtypes = [ctypes.c_int, ctypes.POINTER(lifted_job), ctypes.c_int,
                                           vp, vp]
    lib.nncp_tensor_fit.argtypes = [vp, ctypes.c_int, i64p, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(nnc_opts), vpp, vp, dp, vp]
    lib.nmf_fit.argtypes = [vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                            ctypes.POINTER(nnc_opts), vp, vp, vp, dp, vp]
    lib.candelinc_alg2.argtypes = [vp, ctypes.c_int, i64p, ip, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(nnc_opts), ctypes.POINTER(nnc_opts), vpp, vpp,
                                   vpp, dp, dp, vp]
    for fn in ("ntd_fit", "nncp_core_fit", "nncp_core_fit_batched",
               "nncp_core_fit_batched_noalloc", "nnc_mode_product", "candelinc_lift", "recon_residual",
               "candelinc_lifted_grad", "candelinc_pg_fit", "nncp_tensor_fit", "nmf_fit",
               "candelinc_alg2", "ntd_fit_batched", "ntd_fit_small_batched", "nmf_fit_batched",
               "lifted_rel_err_batched"):
        getattr(lib, fn).restype = ctypes.c_int
    lib.nnc_status_string.argtypes = [ctypes.c_int]
    lib.nnc_status_string.restype = ctypes.c_char_p
    lib.nnc_last_error_detail.argtypes = []
    lib.nnc_last_error_detail.restype = ctypes.c_char_p
    lib.nnc_profile_enable.argtypes = [ctypes.c_int]
    lib.nnc_profile_enable.restype = ctypes.c_int
    lib.nnc_profile_read.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                     ctypes.POINTER(ctypes.c_double)]
    lib.nnc_profile_read.restype = ctypes.c_int
    lib.nnc_kernel_launches.argtypes = []
    lib.nnc_kernel_launches.restype = ctypes.c_longlong
    lib.nnc_autotune_enable.argtypes = [ctypes.c_int]
    lib.nnc_autotune_enable.restype = ctypes.c_int
    lib.nnc_wait_selftest.argtypes = [ctypes.c_longlong, vp]
    lib.nnc_wait_selftest.restype = ctypes.c_int
    lib.nnc_debug_fail_alloc.argtypes = [ctypes.c_int]
    lib.nnc_debug_fail_alloc.restype = ctypes.c_int
    lib.nnc_last_refine_sweep.argtypes = []
    lib.nnc_last_refine_sweep.restype = ctypes.c_int
    _lib = lib
    return lib


def _check(fn, status):
    if status != 0:
        detail = load().nnc_last_error_detail().decode()
        raise NncError(fn, status, detail)


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _require(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _precision(X, precision):
    if precision is None:
        precision = "fp64" if X.dtype == torch.float64 else "fp32"
    code = {"fp64": NNC_FP64, "fp32": NNC_FP32, "bf16": NNC_BF16_REFINE,
            "fp32_simt": NNC_FP32_SIMT}[precision]
    dtype = torch.float64 if code == NNC_FP64 else torch.float32
    return code, dtype


def _i64(vals):
    return (ctypes.c_int64 * len(vals))(*[int(v) for v in vals])


def _i32(vals):
    return (ctypes.c_int * len(vals))(*[int(v) for v in vals])


def _ptrs(ts):
    return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


def ntd_fit(X, F, G, iters, precision=None, eps=1e-12, refine_iters=0, trace=True,
            rel_err=True, stream=None, exact_every=0, refine_tol=0.0):
    """nnTD of X in place on F (list of N_n x m_n) and G. Returns
    (final relative error or None, per-sweep relative-error trace or None).
    exact_every / refine_tol: see nnc_opts (exact trace checkpoints, and the
    switch from BF16 to FP32 sweeps when progress slows)."""
    code, dtype = _precision(X, precision)
    _require(X, dtype, "X")
    for n, f in enumerate(F):
        _require(f, dtype, f"F[{n}]")
    _require(G, dtype, "G")
    d = X.dim()
    m = [f.shape[1] for f in F]
    tr = torch.empty(max(iters, 1), dtype=torch.float64, device=X.device) if trace else None
    err = ctypes.c_double(float("nan"))
    opts = nnc_opts(int(iters), int(refine_iters), float(eps), int(exact_every), float(refine_tol))
    st = load().ntd_fit(_ptr(X), d, _i64(X.shape), _i32(m), code, ctypes.byref(opts), _ptrs(F),
                        _ptr(G), _ptr(tr) if trace else None,
                        ctypes.byref(err) if rel_err else None, _stream(stream))
    _check("ntd_fit", st)
    return (err.value if rel_err else None), (tr[:iters] if trace else None)


def ntd_fit_batched(problems, iters, precision=None, eps=1e-12, refine_iters=0, concurrency=0,
                    trace=True, stream=None):
    """Many nnTD problems of uneven shapes, in place: problems is a list of
    (X, F list, G). Returns (relative errors, device FP64 traces or None,
    statuses)."""
    if not problems:
        return [], [], []
    code, dtype = _precision(problems[0][0], precision)
    n = len(problems)
    jobs = (ntd_job * n)()
    traces = []
    for j, (X, F, G) in enumerate(problems):
        _require(X, dtype, f"X[{j}]")
        _require(G, dtype, f"G[{j}]")
        for k, f in enumerate(F):
            _require(f, dtype, f"F[{j}][{k}]")
        jobs[j].X = X.data_ptr()
        jobs[j].d = X.dim()
        for k in range(X.dim()):
            jobs[j].dims[k] = X.shape[k]
            jobs[j].m[k] = F[k].shape[1]
            jobs[j].F[k] = F[k].data_ptr()
        jobs[j].G = G.data_ptr()
        tr = torch.empty(max(iters, 1), dtype=torch.float64, device=X.device) if trace else None
        jobs[j].trace = tr.data_ptr() if trace else None
        traces.append(tr[:iters] if trace else None)
    opts = nnc_opts(int(iters), int(refine_iters), float(eps))
    errs = (ctypes.c_double * n)()
    sts = (ctypes.c_int * n)()
    st = load().ntd_fit_batched(n, jobs, code, ctypes.byref(opts), int(concurrency), errs, sts,
                                _stream(stream))
    _check("ntd_fit_batched", st)
    return list(errs), traces, list(sts)


def ntd_fit_small_batched(problems, iters, precision=None, eps=1e-12, stream=None):
    """nnTD of many tiny 3-way tensors, one block each, in place: problems is a
    list of (X, F list, G). Returns a device FP64 tensor of relative errors."""
    code, dtype = _precision(problems[0][0], precision)
    n = len(problems)
    jobs = (ntd_small_job * n)()
    for j, (X, F, G) in enumerate(problems):
        _require(X, dtype, f"X[{j}]")
        _require(G, dtype, f"G[{j}]")
        jobs[j].X = X.data_ptr()
        for k in range(3):
            _require(F[k], dtype, f"F[{j}][{k}]")
            jobs[j].dims[k] = X.shape[k]
            jobs[j].m[k] = F[k].shape[1]
            jobs[j].F[k] = F[k].data_ptr()
        jobs[j].G = G.data_ptr()
    errs = torch.empty(n, dtype=torch.float64, device=problems[0][0].device)
    opts = nnc_opts(int(iters), 0, float(eps))
    st = load().ntd_fit_small_batched(n, jobs, code, ctypes.byref(opts), _ptr(errs), _stream(stream))
    _check("ntd_fit_small_batched", st)
    return errs


def nmf_fit_batched(problems, iters, precision=None, eps=1e-12, stream=None):
    """Many small NMFs A ~ F B in place: problems is a list of (A, F, B).
    Returns a device FP64 tensor of relative errors."""
    code, dtype = _precision(problems[0][0], precision)
    n = len(problems)
    jobs = (nmf_job * n)()
    for j, (A, F, B) in enumerate(problems):
        for name, t in (("A", A), ("F", F), ("B", B)):
            _require(t, dtype, f"{name}[{j}]")
        jobs[j].A, jobs[j].F, jobs[j].B = A.data_ptr(), F.data_ptr(), B.data_ptr()
        jobs[j].N, jobs[j].r, jobs[j].m = A.shape[0], A.shape[1], F.shape[1]
    errs = torch.empty(n, dtype=torch.float64, device=problems[0][0].device)
    opts = nnc_opts(int(iters), 0, float(eps))
    st = load().nmf_fit_batched(n, jobs, code, ctypes.byref(opts), _ptr(errs), _stream(stream))
    _check("nmf_fit_batched", st)
    return errs


def lifted_rel_err_batched(problems, precision=None, stream=None):
    """||X - I x_k F^(k) B^(k)|| / ||X|| for many small (X, F list, B list)."""
    code, dtype = _precision(problems[0][0], precision)
    n = len(problems)
    jobs = (lifted_job * n)()
    for j, (X, F, B) in enumerate(problems):
        _require(X, dtype, f"X[{j}]")
        jobs[j].X = X.data_ptr()
        jobs[j].r = B[0].shape[1]
        for k in range(3):
            _require(F[k], dtype, f"F[{j}][{k}]")
            _require(B[k], dtype, f"B[{j}][{k}]")
            jobs[j].dims[k] = X.shape[k]
            jobs[j].m[k] = F[k].shape[1]
            jobs[j].F[k], jobs[j].B[k] = F[k].data_ptr(), B[k].data_ptr()
    errs = torch.empty(n, dtype=torch.float64, device=problems[0][0].device)
    st = load().lifted_rel_err_batched(n, jobs, code, _ptr(errs), _stream(stream))
    _check("lifted_rel_err_batched", st)
    return errs


def nncp_core_fit(G, B, iters, precision=None, eps=1e-12, rel_err=True, stream=None):
    """nnCPD of the core G in place on B (list of m_n x r). Returns the final
    relative error (or None)."""
    code, dtype = _precision(G, precision)
    _require(G, dtype, "G")
    for n, b in enumerate(B):
        _require(b, dtype, f"B[{n}]")
    err = ctypes.c_double(float("nan"))
    opts = nnc_opts(int(iters), 0, float(eps))
    st = load().nncp_core_fit(_ptr(G), G.dim(), _i32(G.shape), B[0].shape[1], code,
                              ctypes.byref(opts), _ptrs(B),
                              ctypes.byref(err) if rel_err else None, _stream(stream))
    _check("nncp_core_fit", st)
    return err.value if rel_err else None


def nncp_core_fit_batched(problems, iters, precision=None, eps=1e-12, stream=None,
                          statuses=None, _entry="nncp_core_fit_batched"):
    """Many core fits in one launch. ``problems`` is a list of (G, [B^(n)]);
    every B is updated in place. Returns a float64 CUDA tensor of the final
    relative errors. ``statuses``, if given, is an int32 CUDA tensor of
    len(problems) entries that receives each fit's status code."""
    if not problems:
        return None
    G0 = problems[0][0]
    code, dtype = _precision(G0, precision)
    jobs = (nncp_job * len(problems))()
    for i, (G, B) in enumerate(problems):
        _require(G, dtype, f"problems[{i}].G")
        j = jobs[i]
        j.G = G.data_ptr()
        j.d = G.dim()
        j.r = B[0].shape[1]
        for n in range(G.dim()):
            _require(B[n], dtype, f"problems[{i}].B[{n}]")
            j.m[n] = G.shape[n]
            j.B[n] = B[n].data_ptr()
    errs = torch.empty(len(problems), dtype=torch.float64, device=G0.device)
    if statuses is not None:
        _require(statuses, torch.int32, "statuses")
        if statuses.numel() != len(problems):
            raise ValueError("statuses must have one entry per problem")
    opts = nnc_opts(int(iters), 0, float(eps))
    st = getattr(load(), _entry)(len(problems), jobs, code, ctypes.byref(opts), _ptr(errs),
                                 _ptr(statuses) if statuses is not None else None,
                                 _stream(stream))
    _check(_entry, st)
    return errs


def nncp_core_fit_batched_noalloc(problems, iters, precision=None, eps=1e-12, stream=None,
                                  statuses=None):
    """As nncp_core_fit_batched, through the entry point that allocates no
    device memory (its job table is a fixed array of 4096 descriptors inside the
    library). For callers whose memory manager forbids allocations by a
    library. Batches that need the two-pass kernel are refused (UNSUPPORTED)."""
    return nncp_core_fit_batched(problems, iters, precision, eps, stream, statuses,
                                 _entry="nncp_core_fit_batched_noalloc")


def mode_product(X, F, mode, precision=None, stream=None):
    """Y = X x_mode F^T for a 3-way X (F is dims[mode] x Q); returns Y."""
    code, dtype = _precision(X, precision)
    _require(X, dtype, "X")
    _require(F, dtype, "F")
    Q = F.shape[1]
    shape = list(X.shape)
    shape[mode] = Q
    out = torch.empty(shape, dtype=dtype, device=X.device)
    st = load().nnc_mode_product(_ptr(X), X.dim(), _i64(X.shape), int(mode), _ptr(F), int(Q), code,
                                 _ptr(out), _stream(stream))
    _check("nnc_mode_product", st)
    return out


def candelinc_lift(F, B, out=None, stream=None):
    """A^(n) = F^(n) B^(n) for every mode; returns the list of A^(n)."""
    dtype = F[0].dtype
    code = NNC_FP64 if dtype == torch.float64 else NNC_FP32
    for n in range(len(F)):
        _require(F[n], dtype, f"F[{n}]")
        _require(B[n], dtype, f"B[{n}]")
    r = B[0].shape[1]
    A = out if out is not None else [torch.empty(f.shape[0], r, dtype=dtype, device=f.device)
                                     for f in F]
    st = load().candelinc_lift(len(F), _i64([f.shape[0] for f in F]), _i32([f.shape[1] for f in F]),
                               r, code, _ptrs(F), _ptrs(B), _ptrs(A), _stream(stream))
    _check("candelinc_lift", st)
    return A


def candelinc_lifted_grad(X, F, B, precision=None, grads=True, stream=None):
    """Loss and gradients of L = 1/2 ||X - I x_n F^(n) B^(n)||^2.

    Returns (loss, gF, gB) with gF[n], gB[n] shaped like F[n], B[n]; with
    grads=False only the loss is computed (gF = gB = None). precision: "fp64",
    "fp32" (TF32x3 tensor-core passes) or "fp32_simt"."""
    code, dtype = _precision(X, precision)
    _require(X, dtype, "X")
    d = X.dim()
    for n in range(d):
        _require(F[n], dtype, f"F[{n}]")
        _require(B[n], dtype, f"B[{n}]")
    r = B[0].shape[1]
    gF = [torch.empty_like(f) for f in F] if grads else None
    gB = [torch.empty_like(b) for b in B] if grads else None
    loss = ctypes.c_double()
    st = load().candelinc_lifted_grad(
        _ptr(X), d, _i64(X.shape), _i32([f.shape[1] for f in F]), r, code, _ptrs(F), _ptrs(B),
        _ptrs(gF) if grads else None, _ptrs(gB) if grads else None, ctypes.byref(loss),
        _stream(stream))
    _check("candelinc_lifted_grad", st)
    return loss.value, gF, gB


def candelinc_pg_fit(X, F, B, steps, precision=None, trace=True, stream=None):
    """Block projected-gradient steps on the lifted loss, in place on F and B.
    Returns (final loss, trace) with trace a device FP64 tensor of the loss after
    each step (None if trace=False)."""
    code, dtype = _precision(X, precision)
    _require(X, dtype, "X")
    d = X.dim()
    for n in range(d):
        _require(F[n], dtype, f"F[{n}]")
        _require(B[n], dtype, f"B[{n}]")
    r = B[0].shape[1]
    tr = torch.empty(max(steps, 1), dtype=torch.float64, device=X.device) if trace else None
    loss = ctypes.c_double()
    st = load().candelinc_pg_fit(_ptr(X), d, _i64(X.shape), _i32([f.shape[1] for f in F]), r,
                                 code, int(steps), _ptrs(F), _ptrs(B),
                                 _ptr(tr) if trace else None, ctypes.byref(loss), _stream(stream))
    _check("candelinc_pg_fit", st)
    return loss.value, (tr[:steps] if trace else None)


def nncp_tensor_fit(X, A, iters, precision=None, eps=1e-12, trace=True, stream=None,
                    exact_every=0):
    """nnCPD of X itself (Alg. 2, first step), in place on A (list of N_n x r).
    Returns (relative error, device FP64 trace or None); exact_every as in
    nnc_opts (exact trace checkpoints)."""
    code, dtype = _precision(X, precision)
    _require(X, dtype, "X")
    for n, a in enumerate(A):
        _require(a, dtype, f"A[{n}]")
    r = A[0].shape[1]
    opts = nnc_opts(int(iters), 0, float(eps), int(exact_every), 0.0)
    tr = torch.empty(max(iters, 1), dtype=torch.float64, device=X.device) if trace else None
    err = ctypes.c_double()
    st = load().nncp_tensor_fit(_ptr(X), X.dim(), _i64(X.shape), r, code, ctypes.byref(opts),
                                _ptrs(A), _ptr(tr) if trace else None, ctypes.byref(err),
                                _stream(stream))
    _check("nncp_tensor_fit", st)
    return err.value, (tr[:iters] if trace else None)


def nmf_fit(A, F, B, iters, precision=None, eps=1e-12, trace=True, stream=None):
    """NMF A ~ F B by MU (Alg. 2, second step), in place on F, B.
    Returns (relative error, device FP64 trace or None)."""
    code, dtype = _precision(A, precision)
    for name, t in (("A", A), ("F", F), ("B", B)):
        _require(t, dtype, name)
    opts = nnc_opts(int(iters), 0, float(eps))
    tr = torch.empty(max(iters, 1), dtype=torch.float64, device=A.device) if trace else None
    err = ctypes.c_double()
    st = load().nmf_fit(_ptr(A), A.shape[0], A.shape[1], F.shape[1], code, ctypes.byref(opts),
                        _ptr(F), _ptr(B), _ptr(tr) if trace else None, ctypes.byref(err),
                        _stream(stream))
    _check("nmf_fit", st)
    return err.value, (tr[:iters] if trace else None)


def candelinc_alg2(X, A, F, B, cp_iters, nmf_iters, precision=None, eps=1e-12, stream=None):
    """Alg. 2 in place on A, F, B: nnCPD of X, then an NMF of every CP factor.
    Returns (CP relative error, list of NMF relative errors)."""
    code, dtype = _precision(X, precision)
    _require(X, dtype, "X")
    d = X.dim()
    for n in range(d):
        _require(A[n], dtype, f"A[{n}]")
        _require(F[n], dtype, f"F[{n}]")
        _require(B[n], dtype, f"B[{n}]")
    cp = nnc_opts(int(cp_iters), 0, float(eps))
    nm = nnc_opts(int(nmf_iters), 0, float(eps))
    cp_err = ctypes.c_double()
    nmf_err = (ctypes.c_double * d)()
    st = load().candelinc_alg2(_ptr(X), d, _i64(X.shape), _i32([f.shape[1] for f in F]),
                               A[0].shape[1], code, ctypes.byref(cp), ctypes.byref(nm), _ptrs(A),
                               _ptrs(F), _ptrs(B), ctypes.byref(cp_err), nmf_err, _stream(stream))
    _check("candelinc_alg2", st)
    return cp_err.value, list(nmf_err)


def recon_residual(X, factors, G=None, stream=None):
    """(||X - X_hat||_F, ||X||_F): Tucker model when G is given, else CP."""
    dtype = X.dtype
    code = NNC_FP64 if dtype == torch.float64 else NNC_FP32
    _require(X, dtype, "X")
    for n, f in enumerate(factors):
        _require(f, dtype, f"factors[{n}]")
    model = 0 if G is not None else 1
    if G is not None:
        _require(G, dtype, "G")
    m = [f.shape[1] for f in factors]
    r = factors[0].shape[1]
    rn, xn = ctypes.c_double(), ctypes.c_double()
    st = load().recon_residual(_ptr(X), X.dim(), _i64(X.shape), code, model, _i32(m), r,
                               _ptrs(factors), _ptr(G) if G is not None else None,
                               ctypes.byref(rn), ctypes.byref(xn), _stream(stream))
    _check("recon_residual", st)
    return rn.value, xn.value


PASS_KINDS = {0: "simt_x3", 1: "simt_x1", 2: "tc_bf16_x3", 3: "tc_bf16_x1", 4: "tc_tf32x3_x3",
              5: "tc_tf32x3_x1"}


def nnc_profile_enable(on=True):
    """Switch event timing of the passes over X on or off (clears the totals)."""
    _check("nnc_profile_enable", load().nnc_profile_enable(1 if on else 0))


def nnc_profile_read(kind):
    """(timed launches, total ms) of one pass kind (see PASS_KINDS)."""
    n, ms = ctypes.c_longlong(), ctypes.c_double()
    _check("nnc_profile_read", load().nnc_profile_read(int(kind), ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def nnc_kernel_launches():
    """Kernels this library has launched in this process so far."""
    return int(load().nnc_kernel_launches())


def nnc_autotune_enable(on=True):
    """Switch the launch-shape autotuner of the batched fits; returns the
    previous setting."""
    return bool(load().nnc_autotune_enable(1 if on else 0))


def nnc_last_refine_sweep():
    """Sweep at which this thread's last BF16 ntd_fit began its FP32 sweeps."""
    return int(load().nnc_last_refine_sweep())


def nnc_debug_fail_alloc(nth):
    """Test hook: make the nth scratch allocation from now fail on the host
    (0 disarms). Returns the previous countdown."""
    return int(load().nnc_debug_fail_alloc(int(nth)))


def nnc_wait_selftest(cycles=2_000_000, stream=None):
    """Status of the bounded-wait self-test (NNC_ERR_TIMEOUT = -7 expected)."""
    return int(load().nnc_wait_selftest(int(cycles), _stream(stream)))
