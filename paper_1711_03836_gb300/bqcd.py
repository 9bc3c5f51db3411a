"""Thin ctypes binding of ``libbqcd_gb300.so`` (C ABI in ``include/bqcd.h``).

Argument marshalling only: every step of the operator and the solvers runs in
the CUDA library.  Functions keep the C names.  Device buffers are torch CUDA
tensors (``torch`` supplies device memory and the stream); host arrays are
numpy arrays or CPU tensors.  A missing or unloadable library raises at import
time of the first call: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbqcd_gb300.so")

BQ_OK, BQ_ERR_ARG, BQ_ERR_CUDA, BQ_ERR_NOT_CONVERGED, BQ_ERR_TIMEOUT, BQ_ERR_CLOVER_SINGULAR, BQ_ERR_STATE, \
    BQ_ERR_NOMEM = range(8)
BQ_PREC_DOUBLE, BQ_PREC_SINGLE, BQ_PREC_HALF = 0, 1, 2
BQ_RECON_18, BQ_RECON_12, BQ_RECON_8 = 18, 12, 8
BQ_HOST, BQ_DEVICE = 0, 1
BQ_FP64_NATIVE, BQ_FP64_DF64 = 0, 1
BQ_SOLVER_CG, BQ_SOLVER_BICGSTAB = 0, 1
SOLVER_NAMES = {"cg": BQ_SOLVER_CG, "bicgstab": BQ_SOLVER_BICGSTAB, 0: 0, 1: 1}
PREC_NAMES = {"double": 0, "single": 1, "half": 2, 0: 0, 1: 1, 2: 2}


class bq_params(ctypes.Structure):
    _fields_ = [("kappa", ctypes.c_double), ("csw", ctypes.c_double), ("mu", ctypes.c_double),
                ("t_bc", ctypes.c_double), ("charge", ctypes.c_double)]


class bq_solver_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precision", ctypes.c_int),
                ("delta", ctypes.c_double), ("check_every", ctypes.c_int), ("shift", ctypes.c_double),
                ("initial_guess", ctypes.c_int)]


class bq_solver_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("converged", ctypes.c_int),
                ("true_residual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("dslash_calls", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class bq_counters(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("dslash_launches", (ctypes.c_longlong * 5) * 3),
                ("dslash_bytes", (ctypes.c_double * 5) * 3), ("dslash_flops", (ctypes.c_double * 5) * 3),
                ("dslash_ms", (ctypes.c_double * 5) * 3), ("fused_bytes", (ctypes.c_double * 5) * 3)]

    def as_dict(self):
        return {
            "launches": int(self.launches),
            "dslash_launches": [[int(v) for v in row] for row in self.dslash_launches],
            "dslash_bytes": [list(row) for row in self.dslash_bytes],
            "dslash_flops": [list(row) for row in self.dslash_flops],
            "dslash_ms": [list(row) for row in self.dslash_ms],
            "fused_bytes": [list(row) for row in self.fused_bytes],
        }


class BqError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        lib = _lib_handle()
        msg = lib.bq_strerror(status).decode() + ": " + lib.bq_last_error().decode()
        super().__init__(f"{where}: {msg} (status {status})")


_lock = threading.Lock()
_lib = None

_SIGS = {
    "bq_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "bq_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "bq_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "bq_last_error": (ctypes.c_char_p, []),
    "bq_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(bq_params)]),
    "bq_reset_counters": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "bq_get_counters": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(bq_counters)]),
    "bq_set_recon": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "bq_set_fp64_arith": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "bq_set_cuda_graphs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "bq_set_gauge": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "bq_set_u1": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "bq_build_clover": (ctypes.c_int, [ctypes.c_void_p]),
    "bq_set_clover": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "bq_spinor_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.c_int]),
    "bq_spinor_pack": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "bq_spinor_unpack": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "bq_spinor_dot": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_double)]),
    "bq_spinor_dot_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int,
                                             ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "bq_apply_dhop": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int]),
    "bq_apply_clover": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int]),
    "bq_apply_mhat": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "bq_apply_mdagm": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "bq_apply_mdagm_batch": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                            ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                            ctypes.c_int]),
    "bq_solve_cg": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                   ctypes.POINTER(bq_solver_params), ctypes.POINTER(bq_solver_stats)]),
    "bq_solve_cg_batch": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                         ctypes.c_int, ctypes.POINTER(bq_solver_params),
                                         ctypes.POINTER(bq_solver_stats)]),
    "bq_solve_multishift_cg": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.c_void_p,
                                              ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(bq_solver_params), ctypes.POINTER(bq_solver_stats),
                                              ctypes.POINTER(ctypes.c_double)]),
    "bq_solve_multishift_cg_block": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                                    ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int,
                                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(bq_solver_params),
                                                    ctypes.POINTER(bq_solver_stats), ctypes.POINTER(ctypes.c_double)]),
    "bq_set_batch_mapping": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "bq_get_batch_mapping": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "bq_set_stout": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int]),
    "bq_get_hop_links": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "bq_clover_logdet": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int)]),
    "bq_solve_full": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(bq_solver_params), ctypes.POINTER(bq_solver_stats)]),
    "bq_trace_samples": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(ctypes.c_void_p), ctypes.c_int,
                                        ctypes.POINTER(bq_solver_params), ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(bq_solver_stats)]),
}


def _lib_handle():
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"CUDA library {LIB_PATH} is not built; run __graft_entry__.build()")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _check(status, where):
    if status != BQ_OK:
        raise BqError(status, where)


def _ptr_where(a):
    """(pointer, BQ_HOST/BQ_DEVICE) of a numpy array or torch tensor (contiguous)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, BQ_HOST
    import torch

    if isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), (BQ_DEVICE if a.is_cuda else BQ_HOST)
    raise TypeError(f"unsupported buffer type {type(a)}")


def _dev_ptr(t):
    p, w = _ptr_where(t)
    if w != BQ_DEVICE:
        raise ValueError("native spinor buffers must be CUDA tensors")
    return p


# ---------------------------------------------------------------- the C functions

def bq_create(dims, stream=None):
    ctx = ctypes.c_void_p()
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    if stream is None:
        import torch

        stream = torch.cuda.current_stream().cuda_stream
    _check(_lib_handle().bq_create(ctypes.byref(ctx), d, ctypes.c_void_p(stream)), "bq_create")
    return ctx


def bq_destroy(ctx):
    _check(_lib_handle().bq_destroy(ctx), "bq_destroy")


def bq_set_params(ctx, kappa, csw=0.0, mu=0.0, t_bc=-1.0, charge=0.0):
    p = bq_params(kappa, csw, mu, t_bc, charge)
    _check(_lib_handle().bq_set_params(ctx, ctypes.byref(p)), "bq_set_params")


def bq_reset_counters(ctx, timing=False):
    _check(_lib_handle().bq_reset_counters(ctx, int(bool(timing))), "bq_reset_counters")


def bq_get_counters(ctx):
    c = bq_counters()
    _check(_lib_handle().bq_get_counters(ctx, ctypes.byref(c)), "bq_get_counters")
    return c.as_dict()


def bq_set_recon(ctx, precision, recon):
    _check(_lib_handle().bq_set_recon(ctx, PREC_NAMES[precision], int(recon)), "bq_set_recon")


def bq_set_fp64_arith(ctx, mode):
    """"native" (FP64 units) or "df64" (double-float on the FP32 units) for FP64-storage operator kernels."""
    m = {"native": BQ_FP64_NATIVE, "df64": BQ_FP64_DF64, 0: 0, 1: 1}[mode]
    _check(_lib_handle().bq_set_fp64_arith(ctx, m), "bq_set_fp64_arith")


def bq_set_cuda_graphs(ctx, enable):
    _check(_lib_handle().bq_set_cuda_graphs(ctx, int(bool(enable))), "bq_set_cuda_graphs")


def bq_set_gauge(ctx, U):
    p, w = _ptr_where(U)
    _check(_lib_handle().bq_set_gauge(ctx, p, w), "bq_set_gauge")


def bq_set_u1(ctx, A):
    if A is None:
        _check(_lib_handle().bq_set_u1(ctx, None, BQ_HOST), "bq_set_u1")
        return
    p, w = _ptr_where(A)
    _check(_lib_handle().bq_set_u1(ctx, p, w), "bq_set_u1")


def bq_build_clover(ctx):
    _check(_lib_handle().bq_build_clover(ctx), "bq_build_clover")


def bq_set_clover(ctx, A):
    """Caller-supplied clover field A[V][2][36] float64 (host or device), or None to build it from the links."""
    if A is None:
        _check(_lib_handle().bq_set_clover(ctx, None, BQ_HOST), "bq_set_clover")
        return
    p, w = _ptr_where(A)
    _check(_lib_handle().bq_set_clover(ctx, p, w), "bq_set_clover")


def bq_spinor_bytes(ctx, precision):
    return int(_lib_handle().bq_spinor_bytes(ctx, PREC_NAMES[precision]))


def bq_spinor_pack(ctx, native, canonical, precision):
    p, w = _ptr_where(canonical)
    _check(_lib_handle().bq_spinor_pack(ctx, _dev_ptr(native), p, PREC_NAMES[precision], w), "bq_spinor_pack")


def bq_spinor_unpack(ctx, canonical, native, precision):
    p, w = _ptr_where(canonical)
    _check(_lib_handle().bq_spinor_unpack(ctx, p, _dev_ptr(native), PREC_NAMES[precision], w), "bq_spinor_unpack")


def bq_spinor_dot(ctx, a, b, precision):
    """<a, b> over the half lattice (complex), FP64 accumulation."""
    r = (ctypes.c_double * 2)()
    _check(_lib_handle().bq_spinor_dot(ctx, _dev_ptr(a), _dev_ptr(b), PREC_NAMES[precision], r), "bq_spinor_dot")
    return complex(r[0], r[1])


def bq_spinor_dot_noalloc(a, b, n_sites, precision, stream=None):
    """<a, b> of two native buffers of n_sites sites without a context and without allocating."""
    if stream is None:
        import torch

        stream = torch.cuda.current_stream().cuda_stream
    r = (ctypes.c_double * 2)()
    _check(_lib_handle().bq_spinor_dot_noalloc(_dev_ptr(a), _dev_ptr(b), int(n_sites), PREC_NAMES[precision],
                                               ctypes.c_void_p(stream), r), "bq_spinor_dot_noalloc")
    return complex(r[0], r[1])


def bq_apply_dhop(ctx, out, inp, out_parity, dagger, precision):
    _check(_lib_handle().bq_apply_dhop(ctx, _dev_ptr(out), _dev_ptr(inp), int(out_parity), int(bool(dagger)),
                                       PREC_NAMES[precision]), "bq_apply_dhop")


def bq_apply_clover(ctx, out, inp, parity, inverse, precision):
    _check(_lib_handle().bq_apply_clover(ctx, _dev_ptr(out), _dev_ptr(inp), int(parity), int(bool(inverse)),
                                         PREC_NAMES[precision]), "bq_apply_clover")


def bq_apply_mhat(ctx, out, inp, dagger, precision):
    _check(_lib_handle().bq_apply_mhat(ctx, _dev_ptr(out), _dev_ptr(inp), int(bool(dagger)), PREC_NAMES[precision]),
           "bq_apply_mhat")


def bq_apply_mdagm(ctx, out, inp, precision):
    _check(_lib_handle().bq_apply_mdagm(ctx, _dev_ptr(out), _dev_ptr(inp), PREC_NAMES[precision]), "bq_apply_mdagm")


def bq_apply_mdagm_batch(ctxs, outs, ins, precision):
    """outs[i] = Mhat^dag Mhat ins[i] on lattice ctxs[i] for every i (native CUDA buffers)."""
    n = len(ctxs)
    if len(outs) != n or len(ins) != n:
        raise ValueError("one output and one input per system")
    carr = (ctypes.c_void_p * n)(*[c.value for c in ctxs])
    oarr = (ctypes.c_void_p * n)(*[_dev_ptr(o) for o in outs])
    iarr = (ctypes.c_void_p * n)(*[_dev_ptr(i) for i in ins])
    _check(_lib_handle().bq_apply_mdagm_batch(carr, n, oarr, iarr, PREC_NAMES[precision]), "bq_apply_mdagm_batch")


def bq_solve_cg(ctx, x, b, tol=1e-10, max_iter=10000, precision="double", delta=1e-3, check_every=8, shift=0.0,
                raise_on_nonconvergence=True, initial_guess=False):
    """Solve (Mhat^dag Mhat + shift) x = b; x, b canonical [V/2][4][3] complex128 (host or device);
    initial_guess=True starts from the x passed in."""
    px, wx = _ptr_where(x)
    pb, wb = _ptr_where(b)
    if wx != wb:
        raise ValueError("x and b must both be host or both be device buffers")
    sp = bq_solver_params(tol, int(max_iter), PREC_NAMES[precision], delta, int(check_every), shift,
                          int(bool(initial_guess)))
    st = bq_solver_stats()
    s = _lib_handle().bq_solve_cg(ctx, px, pb, wx, ctypes.byref(sp), ctypes.byref(st))
    if s != BQ_OK and (raise_on_nonconvergence or s != BQ_ERR_NOT_CONVERGED):
        raise BqError(s, "bq_solve_cg")
    return st.as_dict()


def bq_solve_cg_batch(ctxs, xs, bs, tol=1e-10, max_iter=20000, precision="double", delta=1e-3, check_every=8,
                      shift=0.0, raise_on_nonconvergence=True, initial_guess=False):
    """Solve (Mhat^dag Mhat + shift) xs[i] = bs[i] on lattice ctxs[i] for every i in one batched solve."""
    n = len(ctxs)
    if len(xs) != n or len(bs) != n:
        raise ValueError("one x and one b per system")
    where = None
    px, pb = [], []
    for x, b in zip(xs, bs):
        p1, w1 = _ptr_where(x)
        p2, w2 = _ptr_where(b)
        if w1 != w2 or (where is not None and w1 != where):
            raise ValueError("all x and b must be host buffers or all device buffers")
        where = w1
        px.append(p1)
        pb.append(p2)
    carr = (ctypes.c_void_p * n)(*[c.value for c in ctxs])
    xarr = (ctypes.c_void_p * n)(*px)
    barr = (ctypes.c_void_p * n)(*pb)
    sp = bq_solver_params(tol, int(max_iter), PREC_NAMES[precision], delta, int(check_every), shift,
                          int(bool(initial_guess)))
    st = (bq_solver_stats * n)()
    s = _lib_handle().bq_solve_cg_batch(carr, n, xarr, barr, where, ctypes.byref(sp), st)
    if s != BQ_OK and (raise_on_nonconvergence or s != BQ_ERR_NOT_CONVERGED):
        raise BqError(s, "bq_solve_cg_batch")
    return [st[i].as_dict() for i in range(n)]


def bq_solve_multishift_cg(ctx, xs, b, shifts, tol=1e-10, max_iter=20000, precision="double", delta=1e-3,
                           check_every=8, raise_on_nonconvergence=True):
    """Solve (Mhat^dag Mhat + shifts[k]) xs[k] = b for all k; xs, b canonical, all host or all device."""
    n = len(shifts)
    if len(xs) != n:
        raise ValueError("one solution buffer per shift")
    pb, wb = _ptr_where(b)
    ptrs = []
    for x in xs:
        px, wx = _ptr_where(x)
        if wx != wb:
            raise ValueError("solutions and b must all be host or all be device buffers")
        ptrs.append(px)
    parr = (ctypes.c_void_p * n)(*ptrs)
    sarr = (ctypes.c_double * n)(*[float(v) for v in shifts])
    res = (ctypes.c_double * n)()
    sp = bq_solver_params(tol, int(max_iter), PREC_NAMES[precision], delta, int(check_every), 0.0)
    st = bq_solver_stats()
    s = _lib_handle().bq_solve_multishift_cg(ctx, parr, pb, wb, n, sarr, ctypes.byref(sp), ctypes.byref(st), res)
    if s != BQ_OK and (raise_on_nonconvergence or s != BQ_ERR_NOT_CONVERGED):
        raise BqError(s, "bq_solve_multishift_cg")
    d = st.as_dict()
    d["residuals"] = list(res)
    return d


def bq_solve_multishift_cg_block(ctx, xs, bs, shifts, tol=1e-10, max_iter=20000, precision="double", delta=1e-3,
                                 check_every=8, raise_on_nonconvergence=True):
    """(Mhat^dag Mhat + shifts[k]) xs[r][k] = bs[r] for every right-hand side r and shift k."""
    nrhs, n = len(bs), len(shifts)
    if len(xs) != nrhs or any(len(row) != n for row in xs):
        raise ValueError("xs must hold one row of len(shifts) solutions per right-hand side")
    ptrs = [_ptr_where(v) for v in bs] + [_ptr_where(v) for row in xs for v in row]
    where = ptrs[0][1]
    if any(w != where for _, w in ptrs):
        raise ValueError("all right-hand sides and solutions must be host or all device buffers")
    barr = (ctypes.c_void_p * nrhs)(*[p for p, _ in ptrs[:nrhs]])
    xarr = (ctypes.c_void_p * (nrhs * n))(*[p for p, _ in ptrs[nrhs:]])
    sarr = (ctypes.c_double * n)(*[float(v) for v in shifts])
    res = (ctypes.c_double * (nrhs * n))()
    sp = bq_solver_params(tol, int(max_iter), PREC_NAMES[precision], delta, int(check_every), 0.0)
    st = (bq_solver_stats * nrhs)()
    s = _lib_handle().bq_solve_multishift_cg_block(ctx, nrhs, xarr, barr, where, n, sarr, ctypes.byref(sp), st, res)
    if s != BQ_OK and (raise_on_nonconvergence or s != BQ_ERR_NOT_CONVERGED):
        raise BqError(s, "bq_solve_multishift_cg_block")
    out = [st[r].as_dict() for r in range(nrhs)]
    for r in range(nrhs):
        out[r]["residuals"] = [res[r * n + k] for k in range(n)]
    return out


def bq_set_batch_mapping(ctx, mapping):
    """0 autotuned, -1 block-interleaved, -2 one rhs per warp, -3 shared-memory tiles, 1..8 rhs
    interleaved in a warp."""
    _check(_lib_handle().bq_set_batch_mapping(ctx, int(mapping)), "bq_set_batch_mapping")


def bq_get_batch_mapping(ctx):
    """Mapping used by the last batched call with ctx first (0: none yet)."""
    m = ctypes.c_int()
    _check(_lib_handle().bq_get_batch_mapping(ctx, ctypes.byref(m)), "bq_get_batch_mapping")
    return m.value


def bq_set_stout(ctx, rho, n_iter=1):
    _check(_lib_handle().bq_set_stout(ctx, float(rho), int(n_iter)), "bq_set_stout")


def bq_get_hop_links(ctx, U):
    """Links of the hopping term into U ([V][4][3][3] complex128, host or device)."""
    p, w = _ptr_where(U)
    _check(_lib_handle().bq_get_hop_links(ctx, p, w), "bq_get_hop_links")
    return U


def bq_clover_logdet(ctx, parity):
    """(sum over the parity's sites of log|det A(x)|, number of blocks with det < 0)."""
    ld = ctypes.c_double()
    neg = ctypes.c_int()
    _check(_lib_handle().bq_clover_logdet(ctx, int(parity), ctypes.byref(ld), ctypes.byref(neg)), "bq_clover_logdet")
    return ld.value, neg.value


def bq_solve_full(ctx, x_e, x_o, b_e, b_o, method="bicgstab", tol=1e-10, max_iter=20000, precision="double",
                  delta=1e-3, check_every=8, dagger=False, raise_on_nonconvergence=True):
    """Solve M x = b (or M^dag x = b) on the full lattice (even and odd halves, canonical, all host or all device)."""
    ptrs = [_ptr_where(v) for v in (x_e, x_o, b_e, b_o)]
    where = ptrs[0][1]
    if any(w != where for _, w in ptrs):
        raise ValueError("x_e, x_o, b_e, b_o must all be host or all be device buffers")
    sp = bq_solver_params(tol, int(max_iter), PREC_NAMES[precision], delta, int(check_every), 0.0)
    st = bq_solver_stats()
    s = _lib_handle().bq_solve_full(ctx, ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[3][0], where,
                                    SOLVER_NAMES[method], int(bool(dagger)), ctypes.byref(sp), ctypes.byref(st))
    if s != BQ_OK and (raise_on_nonconvergence or s != BQ_ERR_NOT_CONVERGED):
        raise BqError(s, "bq_solve_full")
    return st.as_dict()


def bq_trace_samples(ctx, etas_e, etas_o, tol=1e-10, max_iter=20000, precision="double", delta=1e-3,
                     check_every=8, raise_on_nonconvergence=True):
    """Per noise vector: (eta^dag M^-1 eta, eta^dag gamma_5 M^-1 eta, eta^dag (M^dag M)^-1 eta) as a
    numpy array [nnoise, 3] (complex, complex, real), and the per-solve stats (M solves, then M^dag solves)."""
    n = len(etas_e)
    if len(etas_o) != n or n < 1:
        raise ValueError("one odd half per even half, at least one noise vector")
    pe = [_ptr_where(v) for v in etas_e]
    po = [_ptr_where(v) for v in etas_o]
    where = pe[0][1]
    if any(w != where for _, w in pe + po):
        raise ValueError("noise vectors must all be host or all be device buffers")
    earr = (ctypes.c_void_p * n)(*[p for p, _ in pe])
    oarr = (ctypes.c_void_p * n)(*[p for p, _ in po])
    sp = bq_solver_params(tol, int(max_iter), PREC_NAMES[precision], delta, int(check_every), 0.0)
    out = (ctypes.c_double * (5 * n))()
    st = (bq_solver_stats * (2 * n))()
    s = _lib_handle().bq_trace_samples(ctx, n, earr, oarr, where, ctypes.byref(sp), out, st)
    if s != BQ_OK and (raise_on_nonconvergence or s != BQ_ERR_NOT_CONVERGED):
        raise BqError(s, "bq_trace_samples")
    v = np.array(out[:], dtype=np.float64).reshape(n, 5)
    res = np.empty((n, 3), np.complex128)
    res[:, 0] = v[:, 0] + 1j * v[:, 1]
    res[:, 1] = v[:, 2] + 1j * v[:, 3]
    res[:, 2] = v[:, 4]
    return res, [st[i].as_dict() for i in range(2 * n)]


# ---------------------------------------------------------------- convenience

class Lattice:
    """A context plus torch-allocated native buffers (device memory only)."""

    def __init__(self, dims, kappa, csw=0.0, mu=0.0, t_bc=-1.0, charge=0.0, stream=None):
        import torch

        self.torch = torch
        self.dims = tuple(int(d) for d in dims)
        self.Vh = int(np.prod(self.dims)) // 2
        self.ctx = bq_create(self.dims, stream)
        bq_set_params(self.ctx, kappa, csw, mu, t_bc, charge)

    def close(self):
        if self.ctx is not None:
            bq_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def spinor(self, precision="double"):
        n = bq_spinor_bytes(self.ctx, precision)
        return self.torch.empty(n, dtype=self.torch.uint8, device="cuda")

    def pack(self, canonical, precision="double"):
        buf = self.spinor(precision)
        bq_spinor_pack(self.ctx, buf, np.ascontiguousarray(canonical, np.complex128)
                       if isinstance(canonical, np.ndarray) else canonical, precision)
        return buf

    def unpack(self, native, precision="double"):
        out = np.empty((self.Vh, 4, 3), np.complex128)
        bq_spinor_unpack(self.ctx, out, native, precision)
        return out
