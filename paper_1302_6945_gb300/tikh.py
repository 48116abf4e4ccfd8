"""Python binding of the C-ABI in include/tikh.h (argument marshalling only).

Every arithmetic step runs in the CUDA kernels of libtikh.so; this module only converts arguments
(torch device tensors or numpy host arrays) to pointers, sizes and the current CUDA stream.  It
raises if the library has not been built: there is no other implementation to fall back on.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtikh.so")

TIKH_OK, TIKH_EINVAL, TIKH_ENOMEM, TIKH_ECUDA, TIKH_ENUMERIC, TIKH_EDIFFICULT, TIKH_ENOTCONVERGED, \
    TIKH_ETIMEOUT, TIKH_EDEGREE = 0, -1, -2, -3, -4, -5, -6, -7, -8
TIKH_R64, TIKH_C128 = 0, 1
TIKH_PREC_FP64, TIKH_PREC_FP32_REFINE, TIKH_PREC_FP32 = 0, 1, 2
PRECISIONS = {"fp64": TIKH_PREC_FP64, "fp32_refine": TIKH_PREC_FP32_REFINE, "fp32": TIKH_PREC_FP32}


class tikh_opts(ctypes.Structure):
    _fields_ = [("n_lim", ctypes.c_int), ("m_min", ctypes.c_int), ("fill", ctypes.c_int),
                ("eps_diff", ctypes.c_double), ("max_difficult", ctypes.c_int), ("refine_steps", ctypes.c_int),
                ("batch", ctypes.c_int), ("graph", ctypes.c_int),
                ("prod_direct_max", ctypes.c_int), ("eval_direct_max", ctypes.c_int), ("wait_polls", ctypes.c_int),
                ("refine_tol", ctypes.c_double), ("fft_radix", ctypes.c_int), ("fft_tile", ctypes.c_int)]


class tikh_stats(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int64), ("M", ctypes.c_int64), ("k", ctypes.c_int64), ("p", ctypes.c_int),
                ("dual", ctypes.c_int), ("n_difficult", ctypes.c_int64), ("delta", ctypes.c_int * 7),
                ("jstar", ctypes.c_int), ("retries", ctypes.c_int), ("kernel_launches", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_int64), ("refine_steps", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("batch", ctypes.c_int), ("prof_leaf_ms", ctypes.c_double), ("prof_leaf_launches", ctypes.c_int64),
                ("graph", ctypes.c_int), ("prof_kind_ms", ctypes.c_double * 4), ("prof_kind_count", ctypes.c_int64 * 4),
                ("model_flops", ctypes.c_double * 4), ("model_flops_fp32", ctypes.c_double * 4),
                ("last_correction", ctypes.c_double)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        for f in ("delta", "prof_kind_ms", "prof_kind_count", "model_flops", "model_flops_fp32"):
            d[f] = list(getattr(self, f))
        return d


class tikh_batch_stats(ctypes.Structure):
    _fields_ = [("ngroups", ctypes.c_int), ("max_waves", ctypes.c_int), ("items", ctypes.c_int64),
                ("kernel_launches", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64), ("graph", ctypes.c_int),
                ("retries", ctypes.c_int), ("n_difficult", ctypes.c_int64), ("rel_residual", ctypes.c_double),
                ("last_correction", ctypes.c_double), ("model_flops", ctypes.c_double * 4),
                ("model_flops_fp32", ctypes.c_double * 4), ("prof_kind_ms", ctypes.c_double * 4),
                ("prof_kind_count", ctypes.c_int64 * 4)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_}
        for f in ("model_flops", "model_flops_fp32", "prof_kind_ms", "prof_kind_count"):
            d[f] = list(getattr(self, f))
        return d


class TikhError(RuntimeError):
    def __init__(self, status, what):
        super().__init__("%s failed: %s (status %d)" % (what, tikh_strerror(status), status))
        self.status = status


_lib = None

EXPORTED = ["tikh_plan_create", "tikh_solve", "tikh_solve_async", "tikh_solve_normal", "tikh_solve_host",
            "tikh_solve_strided", "tikh_batch_plan_create", "tikh_solve_batched", "tikh_batch_get_stats",
            "tikh_batch_plan_destroy", "tikh_test_fft32", "tikh_batch_set_profiling", "tikh_plan_create_gramian",
            "tikh_solve_gramian", "tikh_nufft_gramian", "tikh_test_rcp", "tikh_solve_grad_strided",
            "tikh_sync", "tikh_get_stats", "tikh_plan_destroy", "tikh_strerror", "tikh_test_fft", "tikh_test_leaf",
            "tikh_fft_noalloc", "tikh_set_profiling", "tikh_solve_grad", "tikh_get_difficult", "tikh_test_peak",
            "tikh_plan_create_general", "tikh_solve_general", "tikh_solve_general_normal",
            "tikh_solve_general_strided", "tikh_test_scale", "tikh_inverse_create", "tikh_inverse_apply",
            "tikh_inverse_generators", "tikh_inverse_info", "tikh_inverse_destroy"]


def lib():
    """Load libtikh.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtikh.so is not built (%s): run __graft_entry__.build() or "
                               "python paper_1302_6945_gb300/build.py" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, dbl, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        L.tikh_plan_create.argtypes = [ctypes.POINTER(vp), i64, i64, ci, ci, ctypes.POINTER(tikh_opts), vp]
        for f in ("tikh_solve", "tikh_solve_async", "tikh_solve_normal", "tikh_solve_host"):
            getattr(L, f).argtypes = [vp, vp, vp, vp, dbl, vp]
        L.tikh_solve_strided.argtypes = [vp, ci, vp, i64, vp, i64, vp, i64, vp, vp, i64]
        L.tikh_batch_plan_create.argtypes = [ctypes.POINTER(vp), ci, vp, vp, ci, ci, ci, ctypes.POINTER(tikh_opts),
                                             i64, vp]
        L.tikh_solve_batched.argtypes = [vp, ci, vp, vp, vp, vp, vp, ci, vp, vp]
        L.tikh_batch_get_stats.argtypes = [vp, ctypes.POINTER(tikh_batch_stats)]
        L.tikh_plan_create_gramian.argtypes = [ctypes.POINTER(vp), i64, i64, ci, ci, ctypes.POINTER(tikh_opts), vp]
        L.tikh_solve_gramian.argtypes = [vp, vp, vp, vp, vp, vp]
        L.tikh_plan_create_general.argtypes = [ctypes.POINTER(vp), i64, i64, i64, ci, ctypes.POINTER(tikh_opts), vp]
        L.tikh_solve_general.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.tikh_solve_general_normal.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.tikh_solve_general_strided.argtypes = [vp, ci, vp, i64, vp, i64, vp, i64, vp, i64, vp, i64, vp, i64]
        L.tikh_nufft_gramian.argtypes = [i64, vp, vp, vp, i64, vp, vp, vp]
        L.tikh_batch_set_profiling.argtypes = [vp, ci]
        L.tikh_batch_plan_destroy.argtypes = [vp]
        L.tikh_batch_plan_destroy.restype = None
        L.tikh_sync.argtypes = [vp]
        L.tikh_set_profiling.argtypes = [vp, ci]
        L.tikh_solve_grad.argtypes = [vp, vp, vp, vp, dbl, vp, vp, vp, vp, vp, ctypes.POINTER(dbl)]
        L.tikh_solve_grad_strided.argtypes = [vp, ci, vp, i64, vp, i64, vp, i64, vp, vp, i64, vp, i64, vp, vp, vp, vp]
        L.tikh_get_stats.argtypes = [vp, ctypes.POINTER(tikh_stats)]
        L.tikh_get_difficult.argtypes = [vp, vp, i64, ctypes.POINTER(i64)]
        L.tikh_plan_destroy.argtypes = [vp]
        L.tikh_plan_destroy.restype = None
        L.tikh_strerror.argtypes = [ci]
        L.tikh_strerror.restype = ctypes.c_char_p
        L.tikh_test_fft.argtypes = [i64, vp, ci, vp]
        L.tikh_test_fft32.argtypes = [i64, vp, ci, vp]
        L.tikh_test_rcp.argtypes = [i64, vp, vp, vp]
        L.tikh_test_scale.argtypes = [i64, vp, vp, vp, vp, vp]
        L.tikh_fft_noalloc.argtypes = [i64, vp, ci, vp]
        L.tikh_test_peak.argtypes = [ci, ctypes.POINTER(dbl), vp]
        L.tikh_test_leaf.argtypes = [ci, vp, vp, vp, dbl, vp, vp, vp, vp, vp, vp, vp, vp]
        L.tikh_inverse_create.argtypes = [ctypes.POINTER(vp), vp, vp, vp, dbl, ci]
        L.tikh_inverse_apply.argtypes = [vp, ci, vp, i64, vp, i64, ci, ci]
        L.tikh_inverse_generators.argtypes = [vp, vp]
        L.tikh_inverse_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.tikh_inverse_destroy.argtypes = [vp]
        L.tikh_inverse_destroy.restype = None
        _lib = L
    return _lib


def tikh_strerror(status):
    return lib().tikh_strerror(int(status)).decode()


def _check(rc, what):
    if rc != TIKH_OK:
        raise TikhError(rc, what)


# ---------------------------------------------------------------------------------------------
# C-ABI mirrors
# ---------------------------------------------------------------------------------------------

def tikh_plan_create(m, n, dtype=TIKH_R64, prec=TIKH_PREC_FP64, opts=None, stream=0):
    h = ctypes.c_void_p()
    o = ctypes.byref(opts) if opts is not None else None
    _check(lib().tikh_plan_create(ctypes.byref(h), int(m), int(n), int(dtype), int(prec), o,
                                  ctypes.c_void_p(int(stream))), "tikh_plan_create")
    return h


def tikh_plan_create_gramian(n, p, dtype=TIKH_R64, prec=TIKH_PREC_FP64, opts=None, stream=0):
    h = ctypes.c_void_p()
    o = ctypes.byref(opts) if opts is not None else None
    _check(lib().tikh_plan_create_gramian(ctypes.byref(h), int(n), int(p), int(dtype), int(prec), o,
                                          ctypes.c_void_p(int(stream))), "tikh_plan_create_gramian")
    return h


def tikh_solve_gramian(plan, g, lcol, lrow, y, x):
    _check(lib().tikh_solve_gramian(plan, g, lcol, lrow, y, x), "tikh_solve_gramian")


def tikh_plan_create_general(m, n, pl, dtype=TIKH_R64, opts=None, stream=0):
    h = ctypes.c_void_p()
    o = ctypes.byref(opts) if opts is not None else None
    _check(lib().tikh_plan_create_general(ctypes.byref(h), int(m), int(n), int(pl), int(dtype), o,
                                          ctypes.c_void_p(int(stream))), "tikh_plan_create_general")
    return h


def tikh_solve_general(plan, col, row, lcol, lrow, b, x):
    _check(lib().tikh_solve_general(plan, col, row, lcol, lrow, b, x), "tikh_solve_general")


def tikh_solve_general_normal(plan, col, row, lcol, lrow, y, x):
    _check(lib().tikh_solve_general_normal(plan, col, row, lcol, lrow, y, x), "tikh_solve_general_normal")


def tikh_solve_general_strided(plan, batch, col, col_stride, row, row_stride, lcol, lcol_stride, lrow, lrow_stride,
                               b, b_stride, x, x_stride):
    _check(lib().tikh_solve_general_strided(plan, int(batch), col, int(col_stride), row, int(row_stride), lcol,
                                            int(lcol_stride), lrow, int(lrow_stride), b, int(b_stride), x,
                                            int(x_stride)), "tikh_solve_general_strided")


def tikh_nufft_gramian(K, f, w, X, n, g, y, stream=0):
    _check(lib().tikh_nufft_gramian(int(K), f, w, X, int(n), g, y, ctypes.c_void_p(int(stream))),
           "tikh_nufft_gramian")


def nufft_gramian(f, w, X, n):
    """(g, y) of the weighted non-uniform Fourier Gramian from CUDA tensors f, w (float64) and X (complex128)."""
    import torch
    g = torch.empty(int(n), dtype=torch.complex128, device=f.device)
    y = torch.empty(int(n), dtype=torch.complex128, device=f.device)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    tikh_nufft_gramian(f.numel(), p(f), p(w), p(X), n, p(g), p(y), torch.cuda.current_stream().cuda_stream)
    return g, y


def tikh_solve(plan, col, row, b, lam, x):
    _check(lib().tikh_solve(plan, col, row, b, float(lam), x), "tikh_solve")


def tikh_solve_async(plan, col, row, b, lam, x):
    _check(lib().tikh_solve_async(plan, col, row, b, float(lam), x), "tikh_solve_async")


def tikh_solve_normal(plan, col, row, y, lam, x):
    _check(lib().tikh_solve_normal(plan, col, row, y, float(lam), x), "tikh_solve_normal")


def tikh_solve_strided(plan, batch, col, col_stride, row, row_stride, b, b_stride, lambdas, x, x_stride):
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    _check(lib().tikh_solve_strided(plan, int(batch), col, int(col_stride), row, int(row_stride), b, int(b_stride),
                                    lam.ctypes.data_as(ctypes.c_void_p), x, int(x_stride)), "tikh_solve_strided")


def _i64s(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int64).reshape(-1))
    return a, a.ctypes.data_as(ctypes.c_void_p)


def _ptrs(v):
    a = (ctypes.c_void_p * len(v))(*[int(p) for p in v])
    return a, ctypes.cast(a, ctypes.c_void_p)


def tikh_batch_plan_create(m, n, nlambda, dtype=TIKH_R64, prec=TIKH_PREC_FP64, opts=None, max_workspace_bytes=0,
                           stream=0):
    h = ctypes.c_void_p()
    ma, mp = _i64s(m)
    na, npt = _i64s(n)
    o = ctypes.byref(opts) if opts is not None else None
    _check(lib().tikh_batch_plan_create(ctypes.byref(h), int(ma.size), mp, npt, int(nlambda), int(dtype), int(prec), o,
                                        int(max_workspace_bytes), ctypes.c_void_p(int(stream))),
           "tikh_batch_plan_create")
    return h


def tikh_solve_batched(plan, m, n, col_ptrs, row_ptrs, b_ptrs, lambdas, x_ptrs):
    """Pointer lists are device addresses (ints); lambdas a host sequence."""
    ma, mp = _i64s(m)
    na, npt = _i64s(n)
    ca, cp = _ptrs(col_ptrs)
    ra, rp = _ptrs(row_ptrs)
    ba, bp = _ptrs(b_ptrs)
    xa, xp = _ptrs(x_ptrs)
    lam = np.ascontiguousarray(lambdas, dtype=np.float64)
    _check(lib().tikh_solve_batched(plan, int(ma.size), mp, npt, cp, rp, bp, int(lam.size),
                                    lam.ctypes.data_as(ctypes.c_void_p), xp), "tikh_solve_batched")


def tikh_batch_get_stats(plan):
    st = tikh_batch_stats()
    _check(lib().tikh_batch_get_stats(plan, ctypes.byref(st)), "tikh_batch_get_stats")
    return st.as_dict()


def tikh_batch_set_profiling(plan, flags):
    _check(lib().tikh_batch_set_profiling(plan, int(flags)), "tikh_batch_set_profiling")


def tikh_batch_plan_destroy(plan):
    lib().tikh_batch_plan_destroy(plan)


def tikh_solve_grad(plan, col, row, b, lam, x, dldx, dcol, drow, db):
    out = ctypes.c_double()
    _check(lib().tikh_solve_grad(plan, col, row, b, float(lam), x, dldx, dcol, drow, db, ctypes.byref(out)),
           "tikh_solve_grad")
    return out.value


def tikh_solve_host(plan, col, row, b, lam, x):
    _check(lib().tikh_solve_host(plan, col, row, b, float(lam), x), "tikh_solve_host")


def tikh_sync(plan):
    _check(lib().tikh_sync(plan), "tikh_sync")


def tikh_get_stats(plan):
    st = tikh_stats()
    _check(lib().tikh_get_stats(plan, ctypes.byref(st)), "tikh_get_stats")
    return st.as_dict()


def tikh_get_difficult(plan, cap=1 << 16):
    """(count, sorted ids 2e + f) of the conditions deferred as difficult in the last solve."""
    ids = np.zeros(max(int(cap), 1), np.int64)
    cnt = ctypes.c_int64()
    _check(lib().tikh_get_difficult(plan, ids.ctypes.data_as(ctypes.c_void_p), int(cap), ctypes.byref(cnt)),
           "tikh_get_difficult")
    return int(cnt.value), sorted(int(v) for v in ids[:min(int(cnt.value), int(cap))])


def tikh_plan_destroy(plan):
    lib().tikh_plan_destroy(plan)


def tikh_inverse_create(plan, col, row, lam, max_rhs):
    h = ctypes.c_void_p()
    _check(lib().tikh_inverse_create(ctypes.byref(h), plan, col, row, float(lam), int(max_rhs)), "tikh_inverse_create")
    return h


def tikh_inverse_apply(inv, nrhs, b, b_stride, x, x_stride, normal, refine_steps):
    _check(lib().tikh_inverse_apply(inv, int(nrhs), b, int(b_stride), x, int(x_stride), int(normal),
                                    int(refine_steps)), "tikh_inverse_apply")


def tikh_inverse_generators(inv, out):
    _check(lib().tikh_inverse_generators(inv, out), "tikh_inverse_generators")


def tikh_inverse_info(inv):
    nl, nb = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().tikh_inverse_info(inv, ctypes.byref(nl), ctypes.byref(nb)), "tikh_inverse_info")
    return {"kernel_launches": nl.value, "workspace_bytes": nb.value}


def tikh_inverse_destroy(inv):
    lib().tikh_inverse_destroy(inv)


def tikh_set_profiling(plan, flags):
    _check(lib().tikh_set_profiling(plan, int(flags)), "tikh_set_profiling")


def tikh_test_fft(n, data, sign, stream=0):
    _check(lib().tikh_test_fft(int(n), data, int(sign), ctypes.c_void_p(int(stream))), "tikh_test_fft")


def tikh_test_fft32(n, data, sign, stream=0):
    _check(lib().tikh_test_fft32(int(n), data, int(sign), ctypes.c_void_p(int(stream))), "tikh_test_fft32")


def tikh_test_rcp(n, d, out, stream=0):
    _check(lib().tikh_test_rcp(int(n), d, out, ctypes.c_void_p(int(stream))), "tikh_test_rcp")


def tikh_test_scale(n, v, bits, out_exp, out_mul, stream=0):
    _check(lib().tikh_test_scale(int(n), v, bits, out_exp, out_mul, ctypes.c_void_p(int(stream))), "tikh_test_scale")


def tikh_test_peak(kind, stream=0):
    """Measured FMA rate of the device in GFLOP/s: kind 0 = FP64, 1 = FP32."""
    out = ctypes.c_double()
    _check(lib().tikh_test_peak(int(kind), ctypes.byref(out), ctypes.c_void_p(int(stream))), "tikh_test_peak")
    return out.value


def tikh_fft_noalloc(n, data, sign, stream=0):
    _check(lib().tikh_fft_noalloc(int(n), data, int(sign), ctypes.c_void_p(int(stream))), "tikh_fft_noalloc")


def tikh_test_leaf(K, sigma, r, delta_in, eps, B, length, delta_out, order, pivot, deferred, n_def, stream=0):
    _check(lib().tikh_test_leaf(int(K), sigma, r, delta_in, float(eps), B, length, delta_out, order, pivot, deferred,
                                n_def, ctypes.c_void_p(int(stream))), "tikh_test_leaf")


def fft(x, sign=+1):
    """DFT of a complex128 CUDA tensor through the library's FFT engine (test hook)."""
    import torch
    y = x.detach().to(torch.complex128).contiguous().clone()
    tikh_test_fft(y.numel(), ctypes.c_void_p(y.data_ptr()), sign, torch.cuda.current_stream().cuda_stream)
    return y


def leaf(sigma, r, delta, eps=1e-8):
    """Run one leaf kernel on CUDA tensors sigma (K,) and r (K, 5) (test hook); returns a dict."""
    import torch
    K = sigma.numel()
    dev = sigma.device
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    sig = sigma.to(torch.complex128).contiguous()
    rr = r.to(torch.complex128).contiguous()
    din = torch.tensor(list(delta), dtype=torch.int32, device=dev)
    B = torch.zeros(25 * (K + 1), dtype=torch.complex128, device=dev)
    ln = torch.zeros(25, dtype=torch.int32, device=dev)
    dout = torch.zeros(5, dtype=torch.int32, device=dev)
    order = torch.zeros(K, dtype=torch.int32, device=dev)
    piv = torch.zeros(K, dtype=torch.int32, device=dev)
    dq = torch.zeros(K, dtype=torch.int64, device=dev)
    nd = torch.zeros(1, dtype=torch.int32, device=dev)
    tikh_test_leaf(K, ptr(sig), ptr(rr), ptr(din), eps, ptr(B), ptr(ln), ptr(dout), ptr(order), ptr(piv), ptr(dq),
                   ptr(nd), torch.cuda.current_stream().cuda_stream)
    n = int(nd.item())
    return dict(B=B.view(25, K + 1).cpu().numpy(), len=ln.cpu().numpy(), delta=dout.cpu().numpy(),
                order=order.cpu().numpy(), pivot=piv.cpu().numpy(), deferred=sorted(dq[:n].cpu().tolist()))


# ---------------------------------------------------------------------------------------------
# convenience wrapper over torch CUDA tensors / numpy host arrays
# ---------------------------------------------------------------------------------------------

def _dtype_code(t):
    import torch
    if t.dtype == torch.float64:
        return TIKH_R64
    if t.dtype == torch.complex128:
        return TIKH_C128
    raise TypeError("tensors must be float64 or complex128, got %s" % t.dtype)


class Plan:
    """A solver plan for m x n Toeplitz problems of one dtype ('r64' or 'c128')."""

    def __init__(self, m, n, dtype="r64", n_lim=32, m_min=0, fill=0, eps_diff=1e-8, max_difficult=4096,
                 refine_steps=0, batch=1, graph=False, prod_direct_max=0, eval_direct_max=0, wait_polls=0,
                 refine_tol=0.0, precision="fp64", fft_radix=0, fft_tile=0, stream=None):
        import torch
        self.m, self.n = int(m), int(n)
        self.dtype = TIKH_C128 if dtype in ("c128", TIKH_C128, torch.complex128) else TIKH_R64
        self.batch = int(batch)
        self.opts = tikh_opts(int(n_lim), int(m_min), int(fill), float(eps_diff), int(max_difficult),
                              int(refine_steps), self.batch, 1 if graph else 0, int(prod_direct_max),
                              int(eval_direct_max), int(wait_polls), float(refine_tol),
                              int(fft_radix), int(fft_tile))
        self.prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self.h = tikh_plan_create(self.m, self.n, self.dtype, self.prec, self.opts, handle)

    def _args(self, col, row, v, vlen):
        import torch
        for t, ln in ((col, self.m), (row, self.n), (v, vlen)):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
                raise TypeError("expected contiguous CUDA tensors")
            if _dtype_code(t) != self.dtype or t.numel() != ln:
                raise ValueError("tensor dtype/size does not match the plan")
        return ctypes.c_void_p(col.data_ptr()), ctypes.c_void_p(row.data_ptr()), ctypes.c_void_p(v.data_ptr())

    def _out(self, ref, x):
        import torch
        if x is None:
            x = torch.empty(self.n, dtype=ref.dtype, device=ref.device)
        return x

    def solve(self, col, row, b, lam, x=None, sync=True):
        """x = argmin ||Tx-b||^2 + lam ||x||^2 on the plan's stream."""
        c, r, bb = self._args(col, row, b, self.m)
        x = self._out(b, x)
        f = tikh_solve if sync else tikh_solve_async
        f(self.h, c, r, bb, lam, ctypes.c_void_p(x.data_ptr()))
        return x

    def solve_strided(self, col, row, b, lams, x=None):
        """Solve a batch: col (B, m) or (m,), row (B, n) or (n,), b (B, m) or (m,), lams (B,) on the host.
        A 1-D argument is shared by every problem of the batch (stride 0)."""
        import torch
        lams = np.ascontiguousarray(np.asarray(lams, dtype=np.float64).reshape(-1))
        B = lams.size

        def arg(t, ln):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
                raise TypeError("expected contiguous CUDA tensors")
            if _dtype_code(t) != self.dtype or t.shape[-1] != ln or (t.dim() == 2 and t.shape[0] != B) or t.dim() > 2:
                raise ValueError("tensor dtype/shape does not match the plan and batch")
            return ctypes.c_void_p(t.data_ptr()), (ln if t.dim() == 2 else 0)

        c, cs = arg(col, self.m)
        r, rs = arg(row, self.n)
        bb, bs = arg(b, self.m)
        if x is None:
            x = torch.empty((B, self.n), dtype=b.dtype, device=b.device)
        tikh_solve_strided(self.h, B, c, cs, r, rs, bb, bs, lams, ctypes.c_void_p(x.data_ptr()), self.n)
        return x

    def grad(self, col, row, b, lam, x, dldx):
        """Adjoint: returns (dL/dcol, dL/drow, dL/db, dL/dlambda) for dL/dx = dldx (m >= n)."""
        c, r, bb = self._args(col, row, b, self.m)
        _, _, xx = self._args(col, row, x, self.n)
        dl = dldx.contiguous()  # kept alive for the call
        _, _, gg = self._args(col, row, dl, self.n)
        dcol, drow, db = torch_empty_like(col), torch_empty_like(row), torch_empty_like(b)
        dlam = tikh_solve_grad(self.h, c, r, bb, lam, xx, gg, ctypes.c_void_p(dcol.data_ptr()),
                               ctypes.c_void_p(drow.data_ptr()), ctypes.c_void_p(db.data_ptr()))
        return dcol, drow, db, dlam

    def grad_strided(self, col, row, b, lams, x, dldx):
        """Adjoint of a batch: col (B, m), row (B, n), b (B, m), x and dldx (B, n) contiguous CUDA tensors, lams (B,)
        on the host.  Returns (dL/dcol (B, m), dL/drow (B, n), dL/db (B, m), dL/dlambda (B,) numpy)."""
        import torch
        B = col.shape[0]
        lam = np.ascontiguousarray(np.asarray(lams, dtype=np.float64).reshape(-1))
        dcol, drow, db = torch.empty_like(col), torch.empty_like(row), torch.empty_like(b)
        dlam = np.zeros(B, np.float64)
        dl = dldx.contiguous()  # kept alive for the call
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        _check(lib().tikh_solve_grad_strided(self.h, int(B), p(col), self.m, p(row), self.n, p(b), self.m,
                                             lam.ctypes.data_as(ctypes.c_void_p), p(x), self.n, p(dl),
                                             self.n, p(dcol), p(drow), p(db),
                                             dlam.ctypes.data_as(ctypes.c_void_p)), "tikh_solve_grad_strided")
        return dcol, drow, db, dlam

    def solve_normal(self, col, row, y, lam, x=None):
        """x = (T^H T + lam I)^{-1} y (requires m >= n)."""
        c, r, yy = self._args(col, row, y, self.n)
        x = self._out(y, x)
        tikh_solve_normal(self.h, c, r, yy, lam, ctypes.c_void_p(x.data_ptr()))
        return x

    def solve_host(self, col, row, b, lam, x=None):
        """Same as solve for host numpy arrays (copies in and out inside the call)."""
        np_dt = np.complex128 if self.dtype == TIKH_C128 else np.float64
        col = np.ascontiguousarray(col, dtype=np_dt)
        row = np.ascontiguousarray(row, dtype=np_dt)
        b = np.ascontiguousarray(b, dtype=np_dt)
        if x is None:
            x = np.empty(self.n, dtype=np_dt)
        tikh_solve_host(self.h, col.ctypes.data_as(ctypes.c_void_p), row.ctypes.data_as(ctypes.c_void_p),
                        b.ctypes.data_as(ctypes.c_void_p), lam, x.ctypes.data_as(ctypes.c_void_p))
        return x

    def sync(self):
        tikh_sync(self.h)

    def set_profiling(self, flags):
        tikh_set_profiling(self.h, flags)

    def stats(self):
        d = tikh_get_stats(self.h)
        d["delta"] = d["delta"][:getattr(self, "w", 5)]  # basis size: 5, or 7 for the general problem
        return d

    def difficult(self):
        """(count, sorted ids 2e + f) of the conditions deferred in the last solve (problem 0)."""
        return tikh_get_difficult(self.h)

    def close(self):
        if getattr(self, "h", None):
            tikh_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GramianPlan(Plan):
    """A plan for the Toeplitz-Gramian problem x = (G + L^H L)^{-1} y (G n x n Hermitian Toeplitz, L p x n)."""

    def __init__(self, n, p, dtype="r64", n_lim=32, m_min=0, fill=0, eps_diff=1e-8, max_difficult=4096,
                 refine_steps=0, graph=False, prod_direct_max=0, eval_direct_max=0, wait_polls=0, refine_tol=0.0,
                 precision="fp64", fft_radix=0, fft_tile=0, stream=None):
        import torch
        self.m, self.n = int(p), int(n)
        self.dtype = TIKH_C128 if dtype in ("c128", TIKH_C128, torch.complex128) else TIKH_R64
        self.batch = 1
        self.opts = tikh_opts(int(n_lim), int(m_min), int(fill), float(eps_diff), int(max_difficult),
                              int(refine_steps), 1, 1 if graph else 0, int(prod_direct_max), int(eval_direct_max),
                              int(wait_polls), float(refine_tol), int(fft_radix), int(fft_tile))
        self.prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self.h = tikh_plan_create_gramian(self.n, self.m, self.dtype, self.prec, self.opts, handle)

    def solve(self, g, lcol, lrow, y, x=None):
        """x = (G + L^H L)^{-1} y from contiguous CUDA tensors g (n), lcol (p), lrow (n), y (n)."""
        import torch
        for t, ln in ((g, self.n), (lcol, self.m), (lrow, self.n), (y, self.n)):
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
                raise TypeError("expected contiguous CUDA tensors")
            if _dtype_code(t) != self.dtype or t.numel() != ln:
                raise ValueError("tensor dtype/size does not match the plan")
        if x is None:
            x = torch.empty(self.n, dtype=y.dtype, device=y.device)
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        tikh_solve_gramian(self.h, p(g), p(lcol), p(lrow), p(y), p(x))
        return x


class GeneralPlan(Plan):
    """A plan for the general problem (Sec. 3.2): x = (T^H T + L^H L)^{-1} T^H b, T m x n, L pl x n Toeplitz."""

    def __init__(self, m, n, pl, dtype="r64", n_lim=30, m_min=0, fill=0, eps_diff=1e-12, max_difficult=4096,
                 refine_steps=0, batch=1, graph=False, prod_direct_max=0, eval_direct_max=0, wait_polls=0,
                 refine_tol=0.0, fft_radix=0, fft_tile=0, stream=None):
        import torch
        self.m, self.n, self.pl = int(m), int(n), int(pl)
        self.w = 7
        self.dtype = TIKH_C128 if dtype in ("c128", TIKH_C128, torch.complex128) else TIKH_R64
        self.batch = int(batch)
        self.opts = tikh_opts(int(n_lim), int(m_min), int(fill), float(eps_diff), int(max_difficult),
                              int(refine_steps), int(batch), 1 if graph else 0, int(prod_direct_max),
                              int(eval_direct_max), int(wait_polls), float(refine_tol), int(fft_radix), int(fft_tile))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self.h = tikh_plan_create_general(self.m, self.n, self.pl, self.dtype, self.opts, handle)

    def _check_args(self, pairs):
        import torch
        for t, ln in pairs:
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
                raise TypeError("expected contiguous CUDA tensors")
            if _dtype_code(t) != self.dtype or t.shape[-1] != ln:
                raise ValueError("tensor dtype/size does not match the plan")

    def solve(self, col, row, lcol, lrow, b, x=None, normal=False):
        """x = (T^H T + L^H L)^{-1} T^H b from contiguous CUDA tensors col (m), row (n), lcol (pl), lrow (n),
        b (m); with normal=True the last argument is y (n) and x = (T^H T + L^H L)^{-1} y."""
        import torch
        self._check_args(((col, self.m), (row, self.n), (lcol, self.pl), (lrow, self.n),
                          (b, self.n if normal else self.m)))
        if x is None:
            x = torch.empty(self.n, dtype=b.dtype, device=b.device)
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        f = tikh_solve_general_normal if normal else tikh_solve_general
        f(self.h, p(col), p(row), p(lcol), p(lrow), p(b), p(x))
        return x

    def solve_strided(self, col, row, lcol, lrow, b, x=None):
        """A batch: col (B, m), row (B, n), lcol (B, pl), lrow (B, n), b (B, m) contiguous CUDA tensors (a 1-D
        argument is shared by every problem, stride 0)."""
        import torch
        B = b.shape[0] if b.dim() == 2 else col.shape[0]
        self._check_args(((col, self.m), (row, self.n), (lcol, self.pl), (lrow, self.n), (b, self.m)))
        st = lambda t, ln: ln if t.dim() == 2 else 0
        if x is None:
            x = torch.empty((B, self.n), dtype=b.dtype, device=b.device)
        p = lambda t: ctypes.c_void_p(t.data_ptr())
        tikh_solve_general_strided(self.h, B, p(col), st(col, self.m), p(row), st(row, self.n), p(lcol),
                                   st(lcol, self.pl), p(lrow), st(lrow, self.n), p(b), st(b, self.m), p(x), self.n)
        return x


class Inverse:
    """(T^H T + lam I)^{-1} of one T and lam as four Hankel-product pairs, from eight superfast solves on `plan`
    (an l2 Plan with m >= n, which must stay open): every further right-hand side costs FFTs only."""

    def __init__(self, plan, col, row, lam, max_rhs=8):
        c, r, _ = plan._args(col, row, row, plan.n)
        self.plan, self.m, self.n, self.dtype, self.max_rhs = plan, plan.m, plan.n, plan.dtype, int(max_rhs)
        self.h = tikh_inverse_create(plan.h, c, r, lam, self.max_rhs)

    def apply(self, b, normal=False, refine_steps=1, x=None):
        """x for b of shape (R, m) or (m,) (normal: y of shape (R, n) or (n,)); R right-hand sides."""
        import torch
        ln = self.n if normal else self.m
        if not (isinstance(b, torch.Tensor) and b.is_cuda and b.is_contiguous()):
            raise TypeError("expected a contiguous CUDA tensor")
        if _dtype_code(b) != self.dtype or b.shape[-1] != ln or b.dim() > 2:
            raise ValueError("tensor dtype/shape does not match the plan")
        R = b.shape[0] if b.dim() == 2 else 1
        if x is None:
            x = torch.empty(b.shape[:-1] + (self.n,), dtype=b.dtype, device=b.device)
        tikh_inverse_apply(self.h, R, ctypes.c_void_p(b.data_ptr()), ln, ctypes.c_void_p(x.data_ptr()), self.n,
                           1 if normal else 0, refine_steps)
        return x

    def generators(self):
        """u_0..u_3, w_0..w_3 as an (8, n) complex128 tensor."""
        import torch
        out = torch.empty((8, self.n), dtype=torch.complex128, device="cuda")
        tikh_inverse_generators(self.h, ctypes.c_void_p(out.data_ptr()))
        return out

    def info(self):
        return tikh_inverse_info(self.h)

    def close(self):
        if getattr(self, "h", None):
            tikh_inverse_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchPlan:
    """A plan for problems of different shapes m[i] x n[i], each solved for the same nlambda weights."""

    def __init__(self, m, n, nlambda, dtype="r64", n_lim=32, m_min=0, fill=0, eps_diff=1e-8, max_difficult=4096,
                 refine_steps=0, graph=False, prod_direct_max=0, eval_direct_max=0, wait_polls=0,
                 refine_tol=0.0, precision="fp64", fft_radix=0, fft_tile=0, max_workspace_bytes=0, stream=None):
        import torch
        self.m = [int(v) for v in m]
        self.n = [int(v) for v in n]
        self.nlambda = int(nlambda)
        self.dtype = TIKH_C128 if dtype in ("c128", TIKH_C128, torch.complex128) else TIKH_R64
        self.opts = tikh_opts(int(n_lim), int(m_min), int(fill), float(eps_diff), int(max_difficult),
                              int(refine_steps), 1, 1 if graph else 0, int(prod_direct_max), int(eval_direct_max),
                              int(wait_polls), float(refine_tol), int(fft_radix), int(fft_tile))
        self.prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self.h = tikh_batch_plan_create(self.m, self.n, self.nlambda, self.dtype, self.prec, self.opts,
                                        int(max_workspace_bytes), handle)

    def solve(self, cols, rows, bs, lams, xs=None):
        """cols[i], rows[i], bs[i]: contiguous CUDA tensors of problem i; lams: nlambda weights.  Returns xs,
        a list of nprob * nlambda tensors, xs[i * nlambda + l] for problem i and weight l."""
        import torch
        npb = len(self.m)
        if not (len(cols) == len(rows) == len(bs) == npb):
            raise ValueError("one col, row and b per problem")
        for i in range(npb):
            for t, ln in ((cols[i], self.m[i]), (rows[i], self.n[i]), (bs[i], self.m[i])):
                if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
                    raise TypeError("expected contiguous CUDA tensors")
                if _dtype_code(t) != self.dtype or t.numel() != ln:
                    raise ValueError("tensor dtype/size does not match the plan")
        lams = np.ascontiguousarray(np.asarray(lams, dtype=np.float64).reshape(-1))
        if lams.size != self.nlambda:
            raise ValueError("expected %d lambdas" % self.nlambda)
        if xs is None:
            xs = [torch.empty(self.n[i], dtype=cols[i].dtype, device=cols[i].device)
                  for i in range(npb) for _ in range(self.nlambda)]
        tikh_solve_batched(self.h, self.m, self.n, [t.data_ptr() for t in cols], [t.data_ptr() for t in rows],
                           [t.data_ptr() for t in bs], lams, [t.data_ptr() for t in xs])
        return xs

    def stats(self):
        return tikh_batch_get_stats(self.h)

    def set_profiling(self, flags):
        tikh_batch_set_profiling(self.h, flags)

    def close(self):
        if getattr(self, "h", None):
            tikh_batch_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def torch_empty_like(t):
    import torch
    return torch.empty_like(t)


_autograd_fn = None


def _make_autograd():
    import torch

    class TikhSolve(torch.autograd.Function):
        """x = argmin ||Tx - b||^2 + lam ||x||^2 with the library's hand-written adjoint as backward."""

        @staticmethod
        def forward(ctx, col, row, b, lam, plan):
            lam_v = float(lam)
            x = plan.solve(col.contiguous(), row.contiguous(), b.contiguous(), lam_v)
            ctx.save_for_backward(col, row, b, x)
            ctx.plan, ctx.lam = plan, lam_v
            ctx.lam_is_tensor = isinstance(lam, torch.Tensor)
            return x

        @staticmethod
        def backward(ctx, gx):
            col, row, b, x = ctx.saved_tensors
            dcol, drow, db, dlam = ctx.plan.grad(col.contiguous(), row.contiguous(), b.contiguous(), ctx.lam, x,
                                                 gx.contiguous())
            glam = torch.tensor(dlam, dtype=torch.float64, device=col.device) if ctx.lam_is_tensor else None
            return dcol, drow, db, glam, None

    return TikhSolve


def tikh_solve_autograd(col, row, b, lam, plan):
    """Differentiable solve: gradients flow to col, row, b and (if a tensor) lam."""
    global _autograd_fn
    if _autograd_fn is None:
        _autograd_fn = _make_autograd()
    return _autograd_fn.apply(col, row, b, lam, plan)


def solve(col, row, b, lam, **kw):
    """One-shot solve of CUDA tensors (builds and frees a plan)."""
    p = Plan(col.numel(), row.numel(), "c128" if col.is_complex() else "r64", **kw)
    try:
        return p.solve(col, row, b, lam)
    finally:
        p.close()


# ---- tuning ----------------------------------------------------------------------------------------

TUNE_SPACE = {
    "n_lim": (24, 32, 40),
    "prod_direct_max": (36, 72, 192, 360),
    "eval_direct_max": (10, 20, 40, 80),
    "fft_radix": (8, 4),
    "fft_tile": (256, 512, 1024),
}


def coordinate_search(time_fn, start, space=None):
    """Minimise time_fn(opts) one key at a time (n_lim, then the product and evaluation thresholds),
    keeping the best value of each key before moving to the next.  Returns (best opts, {opts: time})."""
    space = space or TUNE_SPACE
    best = dict(start)
    seen = {}

    def t(o):
        k = tuple(sorted(o.items()))
        if k not in seen:
            seen[k] = float(time_fn(dict(o)))
        return seen[k]

    best_t = t(best)
    for key in ("n_lim", "prod_direct_max", "eval_direct_max", "fft_radix", "fft_tile"):
        if key not in space:
            continue
        for v in space[key]:
            cand = dict(best)
            cand[key] = v
            ct = t(cand)
            if ct < best_t:
                best, best_t = cand, ct
    return best, {k: v for k, v in seen.items()}


def autotune(m, n, dtype="c128", batch=1, refine_steps=0, reps=2, seed=0, time_fn=None):
    """Pick N_lim and the direct/FFT thresholds of steps 2 and 4 for m x n problems solved `batch` at a
    time: each candidate plan solves a seeded random Toeplitz problem of that shape (generated on the
    device), timed with CUDA events on the plan's stream after one warm-up solve, best of `reps`.
    Returns (Plan keyword arguments, {candidate: seconds}).  time_fn replaces the timing (for tests)."""
    import torch
    if time_fn is None:
        g = torch.Generator(device="cuda").manual_seed(int(seed))
        tdt = torch.complex128 if dtype in ("c128", TIKH_C128) else torch.float64
        B = int(batch)
        col = torch.randn((B, m), generator=g, device="cuda", dtype=tdt)
        row = torch.randn((B, n), generator=g, device="cuda", dtype=tdt)
        b = torch.randn((B, m), generator=g, device="cuda", dtype=tdt)
        lams = [1e-2] * B
        stream = torch.cuda.Stream()

        def time_fn(o):
            with torch.cuda.stream(stream):
                p = Plan(m, n, dtype, refine_steps=refine_steps, batch=B, graph=True, stream=stream, **o)
                try:
                    x = torch.empty((B, n), dtype=tdt, device="cuda")
                    p.solve_strided(col, row, b, lams, x)
                    best = float("inf")
                    for _ in range(max(1, int(reps))):
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        p.solve_strided(col, row, b, lams, x)
                        e1.record(stream)
                        e1.synchronize()
                        best = min(best, e0.elapsed_time(e1) * 1e-3)
                    return best
                finally:
                    p.close()

    start = {"n_lim": 32, "prod_direct_max": 0, "eval_direct_max": 0, "fft_radix": 0, "fft_tile": 0}
    return coordinate_search(time_fn, start)
