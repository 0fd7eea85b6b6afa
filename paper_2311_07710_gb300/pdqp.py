"""Thin ctypes binding of libpdqp.so (include/pdqp.h).

Functions carry the C names and only marshal arguments: numpy arrays are
passed as host pointers (PDQP_MEM_HOST), torch CUDA tensors as device pointers
(PDQP_MEM_DEVICE).  Every step of the solver runs in the library's CUDA
kernels; importing this module fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpdqp.so")

PDQP_OK, PDQP_ERR_INVALID, PDQP_ERR_CUDA, PDQP_ERR_OOM = 0, 1, 2, 3
PDQP_ITER_LIMIT, PDQP_TIME_LIMIT, PDQP_NUMERICAL, PDQP_DEVICE_TIMEOUT = 10, 11, 12, 13
PDQP_PRIMAL_INFEASIBLE, PDQP_DUAL_INFEASIBLE = 14, 15
PDQP_MEM_HOST, PDQP_MEM_DEVICE = 0, 1
PDQP_PREC_FP64, PDQP_PREC_MIXED = 0, 1
PDQP_STEP_ADAPTIVE, PDQP_STEP_THEORY = 0, 1
PDQP_RESTART_PDQP, PDQP_RESTART_HALVING, PDQP_RESTART_FIXED, PDQP_RESTART_NONE = 0, 1, 2, 3


class pdqp_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32), ("step_rule", ctypes.c_int32), ("restart_rule", ctypes.c_int32),
        ("accelerate", ctypes.c_int32), ("scaling", ctypes.c_int32), ("ruiz_iters", ctypes.c_int32),
        ("l2_scaling", ctypes.c_int32), ("pock_chambolle", ctypes.c_int32), ("fixed_K", ctypes.c_int32),
        ("check_period", ctypes.c_int32), ("max_iter", ctypes.c_int64), ("eps", ctypes.c_double),
        ("time_limit", ctypes.c_double), ("beta_suff", ctypes.c_double), ("beta_nec", ctypes.c_double),
        ("beta_art", ctypes.c_double), ("pw_theta", ctypes.c_double), ("eps_zero", ctypes.c_double),
        ("norm_A", ctypes.c_double), ("norm_Q", ctypes.c_double), ("norm_iters", ctypes.c_int32),
        ("norm_tol", ctypes.c_double), ("spmv_threads", ctypes.c_int32), ("no_graphs", ctypes.c_int32),
        ("detect_infeasibility", ctypes.c_int32), ("eps_infeasible", ctypes.c_double),
        ("maintained_products", ctypes.c_int32),
    ]


class pdqp_info(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("iterations", ctypes.c_int64), ("restarts", ctypes.c_int64),
        ("rel_kkt", ctypes.c_double), ("r_primal", ctypes.c_double), ("r_dual", ctypes.c_double),
        ("r_gap", ctypes.c_double), ("primal_obj", ctypes.c_double), ("dual_obj", ctypes.c_double),
        ("seconds", ctypes.c_double), ("norm_A", ctypes.c_double), ("norm_Q", ctypes.c_double),
        ("omega", ctypes.c_double), ("setup_seconds", ctypes.c_double),
        ("iterate_seconds", ctypes.c_double), ("norm_iters", ctypes.c_int32), ("spmv_threads", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class pdqp_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 4), ("ms", ctypes.c_double * 4), ("bytes", ctypes.c_double * 4)]


class pdqp_ws_train_options(ctypes.Structure):
    _fields_ = [("epochs", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("seed", ctypes.c_uint64)]


class PdqpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_string(status)} ({status}): {msg}")
        self.status = status


_P = ctypes.c_void_p
_lib = None

# exported symbols and their signatures: (restype, argtypes)
SIGNATURES = {
    "pdqp_default_options": (None, [ctypes.POINTER(pdqp_options)]),
    "pdqp_status_string": (ctypes.c_char_p, [ctypes.c_int32]),
    "pdqp_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                   _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int32, _P]),
    "pdqp_set_lowrank_Q": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.c_int32, _P]),
    "pdqp_solve": (ctypes.c_int, [_P, ctypes.POINTER(pdqp_options), _P, _P, _P, _P,
                                  ctypes.POINTER(pdqp_info), ctypes.c_int32, _P]),
    "pdqp_solve_batch": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(_P), ctypes.POINTER(pdqp_options),
                                        ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P),
                                        ctypes.POINTER(_P), ctypes.POINTER(pdqp_info), ctypes.c_int32, _P]),
    "pdqp_get_iterates": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int32, _P]),
    "pdqp_get_state": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_size_t), _P]),
    "pdqp_set_state": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P]),
    "pdqp_kkt": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_double), ctypes.c_int32, _P]),
    "pdqp_get_sizes": (ctypes.c_int, [_P] + [ctypes.POINTER(ctypes.c_int64)] * 5),
    "pdqp_last_error": (ctypes.c_char_p, [_P]),
    "pdqp_destroy": (None, [_P]),
    "pdqp_launch_count": (ctypes.c_int64, []),
    "pdqp_profile_enable": (ctypes.c_int, [_P, ctypes.c_int32]),
    "pdqp_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(pdqp_profile)]),
    "pdqp_create_batch": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32] + [ctypes.POINTER(ctypes.c_int64)] * 3
                          + [ctypes.POINTER(_P)] * 10 + [ctypes.c_int32, _P]),
    "pdqp_create_batch_packed": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32]
                                 + [ctypes.POINTER(ctypes.c_int64)] * 3 + [_P] * 10 + [ctypes.c_int32, _P]),
    "pdqp_create_family": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_int64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int32, _P]),
    "pdqp_batch_count": (ctypes.c_int32, [_P]),
    "pdqp_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(pdqp_info), ctypes.c_int32]),
    "pdqp_kkt_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _P, _P, _P,
                                        ctypes.c_int64, _P, _P, _P, _P, _P, _P, ctypes.c_int64,
                                        _P, _P, _P, _P, _P, _P, _P, _P]),
    # include/pdqp_ws.h
    "pdqp_ws_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int64, ctypes.c_int64, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P]),
    "pdqp_ws_destroy": (None, [_P]),
    "pdqp_ws_last_error": (ctypes.c_char_p, [_P]),
    "pdqp_ws_set_params": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_int32, _P]),
    "pdqp_ws_get_params": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_int32, _P]),
    "pdqp_ws_set_normalization": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_int32, _P]),
    "pdqp_ws_get_normalization": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_int32, _P]),
    "pdqp_ws_fit": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int64, ctypes.c_int32, _P]),
    "pdqp_ws_grad": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_double),
                                    ctypes.c_int32, _P]),
    "pdqp_ws_train": (ctypes.c_int, [_P, ctypes.POINTER(pdqp_ws_train_options), _P, _P, _P, _P, ctypes.c_int64,
                                     _P, ctypes.c_int32, _P]),
    "pdqp_ws_infer": (ctypes.c_int, [_P, _P, _P, ctypes.c_int64, _P, _P, ctypes.c_int32, _P]),
    "pdqp_gemm_bf16": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int32, _P,
                                      ctypes.c_int32, _P, ctypes.c_int32, _P, ctypes.c_int32, _P, _P,
                                      ctypes.c_int32, ctypes.c_int32, _P, ctypes.c_int64, _P]),
    "pdqp_gemm_bf16_check": (ctypes.c_int, [_P]),
    "pdqp_gemm_bf16_wait_probe": (ctypes.c_int, [_P]),
    "pdqp_gemm_bf16_splits": (ctypes.c_int32, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
}


def load(path: str = LIB_PATH):
    """Load libpdqp.so (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().pdqp_status_string(int(status)).decode()


# ---------------------------------------------------------------------------
# argument marshalling
# ---------------------------------------------------------------------------
def _is_torch_cuda(a) -> bool:
    return a is not None and type(a).__module__.startswith("torch") and getattr(a, "is_cuda", False)


def _ptr(a, dtype):
    """(pointer, keepalive, mem_space) of an array argument."""
    if a is None:
        return None, None, None
    if _is_torch_cuda(a):
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32, np.float32: torch.float32}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"device array must be a contiguous {want} tensor")
        return ctypes.c_void_p(a.data_ptr()), a, PDQP_MEM_DEVICE
    arr = np.ascontiguousarray(a, dtype=dtype)
    return ctypes.c_void_p(arr.ctypes.data), arr, PDQP_MEM_HOST


def _stream(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _check(status, handle=None):
    if status not in (PDQP_OK, PDQP_ITER_LIMIT, PDQP_TIME_LIMIT, PDQP_NUMERICAL, PDQP_PRIMAL_INFEASIBLE,
                      PDQP_DUAL_INFEASIBLE):
        msg = load().pdqp_last_error(handle).decode()
        raise PdqpError(status, msg)
    return status


def _one_space(spaces):
    s = {x for x in spaces if x is not None}
    if len(s) > 1:
        raise TypeError("mix of host (numpy) and device (torch CUDA) arrays in one call")
    return s.pop() if s else PDQP_MEM_HOST


# ---------------------------------------------------------------------------
# the C functions
# ---------------------------------------------------------------------------
def pdqp_default_options(**overrides) -> pdqp_options:
    o = pdqp_options()
    load().pdqp_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o


def pdqp_create(n, m, m_eq, Q_rowptr, Q_col, Q_val, A_rowptr, A_col, A_val, c, b, l, u, stream=None):
    args = [_ptr(Q_rowptr, np.int32), _ptr(Q_col, np.int32), _ptr(Q_val, np.float64),
            _ptr(A_rowptr, np.int32), _ptr(A_col, np.int32), _ptr(A_val, np.float64),
            _ptr(c, np.float64), _ptr(b, np.float64), _ptr(l, np.float64), _ptr(u, np.float64)]
    mem = _one_space([a[2] for a in args])
    h = ctypes.c_void_p()
    st = load().pdqp_create(ctypes.byref(h), int(n), int(m), int(m_eq), *[a[0] for a in args], mem,
                            _stream(stream))
    _check(st, None)
    return h


def pdqp_set_lowrank_Q(h, r, F, stream=None):
    p, keep, mem = _ptr(F, np.float32)
    return _check(load().pdqp_set_lowrank_Q(h, int(r), p, mem, _stream(stream)), h)


def pdqp_solve(h, opt: Optional[pdqp_options] = None, x0=None, y0=None, x_out=None, y_out=None, stream=None):
    """Returns (status, pdqp_info).  x_out / y_out (numpy float64 or torch CUDA
    float64) receive the returned iterate."""
    args = [_ptr(x0, np.float64), _ptr(y0, np.float64)]
    outs = [x_out, y_out]
    for o in outs:
        if o is not None and not _is_torch_cuda(o):
            if not (isinstance(o, np.ndarray) and o.dtype == np.float64 and o.flags.c_contiguous):
                raise TypeError("host outputs must be contiguous float64 numpy arrays")
    oargs = [_ptr(o, np.float64) for o in outs]
    mem = _one_space([a[2] for a in args + oargs])
    info = pdqp_info()
    opt = opt if opt is not None else pdqp_default_options()
    st = load().pdqp_solve(h, ctypes.byref(opt), args[0][0], args[1][0], oargs[0][0], oargs[1][0],
                           ctypes.byref(info), mem, _stream(stream))
    return _check(st, h), info


def pdqp_solve_batch(hs: Sequence, opt: Optional[pdqp_options] = None, x0=None, y0=None, x_out=None,
                     y_out=None, stream=None):
    """Solve len(hs) problems.  x0/y0/x_out/y_out are None or per-problem lists."""
    count = len(hs)
    keep = []

    def arr_of(lst, writable):
        if lst is None:
            return None, []
        ptrs = []
        for a in lst:
            if a is not None and writable and not _is_torch_cuda(a):
                assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
            p = _ptr(a, np.float64)
            keep.append(p[1])
            ptrs.append(p)
        return (ctypes.c_void_p * count)(*[p[0] for p in ptrs]), [p[2] for p in ptrs]

    a0, s0 = arr_of(x0, False)
    a1, s1 = arr_of(y0, False)
    a2, s2 = arr_of(x_out, True)
    a3, s3 = arr_of(y_out, True)
    mem = _one_space(s0 + s1 + s2 + s3)
    hs_arr = (ctypes.c_void_p * count)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in hs])
    infos = (pdqp_info * count)()
    opt = opt if opt is not None else pdqp_default_options()
    st = load().pdqp_solve_batch(count, hs_arr, ctypes.byref(opt), a0, a1, a2, a3, infos, mem, _stream(stream))
    return _check(st, None), list(infos)


def pdqp_get_iterates(h, x=None, y=None, xbar=None, ybar=None, stream=None):
    args = [_ptr(a, np.float64) for a in (x, y, xbar, ybar)]
    mem = _one_space([a[2] for a in args])
    return _check(load().pdqp_get_iterates(h, *[a[0] for a in args], mem, _stream(stream)), h)


def pdqp_get_state(h, stream=None):
    """The handle's complete solver state after its last solve (checkpoint), as bytes."""
    lib = load()
    size = ctypes.c_size_t(0)
    _check(lib.pdqp_get_state(h, None, ctypes.byref(size), _stream(stream)), h)
    buf = ctypes.create_string_buffer(size.value)
    _check(lib.pdqp_get_state(h, buf, ctypes.byref(size), _stream(stream)), h)
    return buf.raw[:size.value]


def pdqp_set_state(h, state: bytes, stream=None):
    """Load a checkpoint from pdqp_get_state; the next pdqp_solve continues from it."""
    buf = ctypes.create_string_buffer(bytes(state), len(state))
    return _check(load().pdqp_set_state(h, buf, len(state), _stream(stream)), h)


def pdqp_kkt(h, x, y, stream=None):
    """[r_primal, r_dual, r_gap, rel_kkt, primal_obj, dual_obj] of (x, y)."""
    a, b = _ptr(x, np.float64), _ptr(y, np.float64)
    mem = _one_space([a[2], b[2]])
    parts = (ctypes.c_double * 6)()
    _check(load().pdqp_kkt(h, a[0], b[0], parts, mem, _stream(stream)), h)
    return list(parts)


def pdqp_create_batch(instances, stream=None):
    """One handle for a list of problems; each entry is a tuple
    (n, m, m_eq, Q_rowptr, Q_col, Q_val, A_rowptr, A_col, A_val, c, b, l, u)."""
    count = len(instances)
    keep = []
    cols = [[] for _ in range(10)]
    dtypes = [np.int32, np.int32, np.float64] * 2 + [np.float64] * 4
    spaces = []
    for inst in instances:
        for k, (arr, t) in enumerate(zip(inst[3:], dtypes)):
            ptr, ka, sp_ = _ptr(arr, t)
            keep.append(ka)
            cols[k].append(ptr)
            spaces.append(sp_)
    mem = _one_space(spaces)
    I64 = ctypes.c_int64 * count
    ns, ms, meqs = I64(*[int(i[0]) for i in instances]), I64(*[int(i[1]) for i in instances]), \
        I64(*[int(i[2]) for i in instances])
    ptr_arrays = [(ctypes.c_void_p * count)(*c) for c in cols]
    h = ctypes.c_void_p()
    st = load().pdqp_create_batch(ctypes.byref(h), count, ns, ms, meqs, *ptr_arrays, mem, _stream(stream))
    _check(st, None)
    return h


def pdqp_create_batch_packed(n, m, m_eq, Q_rowptr, Q_col, Q_val, A_rowptr, A_col, A_val, c, b, l, u,
                             stream=None):
    """One handle for a batch handed over as one block-diagonal problem: n, m,
    m_eq are the instances' sizes (sequences of count ints); the CSR arrays
    span the whole stack with global column indices and c, b, l, u are the
    instances' vectors concatenated (pack_instances builds them)."""
    count = len(n)
    I64 = ctypes.c_int64 * count
    ns, ms, meqs = I64(*[int(v) for v in n]), I64(*[int(v) for v in m]), I64(*[int(v) for v in m_eq])
    dtypes = [np.int32, np.int32, np.float64] * 2 + [np.float64] * 4
    args = [_ptr(a, t) for a, t in zip((Q_rowptr, Q_col, Q_val, A_rowptr, A_col, A_val, c, b, l, u), dtypes)]
    mem = _one_space([a[2] for a in args])
    h = ctypes.c_void_p()
    st = load().pdqp_create_batch_packed(ctypes.byref(h), count, ns, ms, meqs, *[a[0] for a in args], mem,
                                         _stream(stream))
    _check(st, None)
    return h


def pdqp_create_family(count, n, m, m_eq, Q_rowptr, Q_col, Q_val, A_rowptr, A_col, A_val, C, B, l, u,
                       stream=None):
    """One handle for `count` family members sharing Q, A, l, u; C [count x n]
    and B [count x m] hold each member's c and b."""
    args = [_ptr(Q_rowptr, np.int32), _ptr(Q_col, np.int32), _ptr(Q_val, np.float64),
            _ptr(A_rowptr, np.int32), _ptr(A_col, np.int32), _ptr(A_val, np.float64),
            _ptr(C, np.float64), _ptr(B, np.float64), _ptr(l, np.float64), _ptr(u, np.float64)]
    mem = _one_space([a[2] for a in args])
    h = ctypes.c_void_p()
    st = load().pdqp_create_family(ctypes.byref(h), int(count), int(n), int(m), int(m_eq), *[a[0] for a in args],
                                   mem, _stream(stream))
    _check(st, None)
    return h


def family_from_base(base, C, B, device=False, stream=None):
    """A family handle from a base instance (n, m, m_eq, Q, A, l, u; scipy CSR)
    and per-member rows C [count x n], B [count x m] (numpy, or torch CUDA
    float64 tensors, which put the whole call on device pointers)."""
    device = device or _is_torch_cuda(C)
    arrays = [base.Q.indptr, base.Q.indices, base.Q.data, base.A.indptr, base.A.indices, base.A.data,
              base.l, base.u]
    dtypes = [np.int32, np.int32, np.float64] * 2 + [np.float64] * 2
    arrays = [np.ascontiguousarray(a, dtype=t) for a, t in zip(arrays, dtypes)]
    if device:
        import torch
        arrays = [torch.from_numpy(a).cuda() for a in arrays]
        C = C if _is_torch_cuda(C) else torch.from_numpy(np.ascontiguousarray(C, dtype=np.float64)).cuda()
        B = B if _is_torch_cuda(B) else torch.from_numpy(np.ascontiguousarray(B, dtype=np.float64)).cuda()
        torch.cuda.synchronize()
    else:
        C = np.ascontiguousarray(C, dtype=np.float64)
        B = np.ascontiguousarray(B, dtype=np.float64)
    return pdqp_create_family(C.shape[0], base.n, base.m, base.m_eq, *arrays[:6], C, B, *arrays[6:],
                              stream=stream)


def pdqp_batch_count(h) -> int:
    return int(load().pdqp_batch_count(h))


def pdqp_batch_info(h):
    count = pdqp_batch_count(h)
    infos = (pdqp_info * count)()
    _check(load().pdqp_batch_info(h, infos, count), h)
    return list(infos)


def pdqp_kkt_noalloc(n, m, m_eq, Q_rowptr, Q_col, Q_val, A_rowptr, A_col, A_val, At_rowptr, At_col, At_val,
                     c, b, l, u, x, y, parts, stream=None):
    """Allocation-free relKKT of (x, y): every array is a torch CUDA tensor
    (int32 / float64); parts (float64, 6 entries) receives the result.  The
    call is asynchronous on `stream` and returns the status."""
    dev = [Q_rowptr, Q_col, Q_val, A_rowptr, A_col, A_val, At_rowptr, At_col, At_val, c, b, l, u, x, y, parts]
    types = [np.int32, np.int32, np.float64] * 3 + [np.float64] * 7
    ptrs = []
    for a, t in zip(dev, types):
        if a is None:
            ptrs.append(None)
            continue
        if not _is_torch_cuda(a):
            raise TypeError("pdqp_kkt_noalloc takes device (torch CUDA) arrays only")
        ptrs.append(_ptr(a, t)[0])
    nnz_Q = int(Q_col.numel()) if Q_col is not None else 0
    nnz_A = int(A_col.numel()) if A_col is not None else 0
    return load().pdqp_kkt_noalloc(int(n), int(m), int(m_eq), ptrs[0], ptrs[1], ptrs[2], nnz_Q, ptrs[3],
                                   ptrs[4], ptrs[5], ptrs[6], ptrs[7], ptrs[8], nnz_A, *ptrs[9:],
                                   _stream(stream))


def pdqp_get_sizes(h):
    vals = [ctypes.c_int64() for _ in range(5)]
    _check(load().pdqp_get_sizes(h, *[ctypes.byref(v) for v in vals]), h)
    return tuple(v.value for v in vals)


def pdqp_last_error(h=None) -> str:
    return load().pdqp_last_error(h).decode()


def pdqp_destroy(h):
    load().pdqp_destroy(h)


def pdqp_launch_count() -> int:
    return int(load().pdqp_launch_count())


def pdqp_profile_enable(h, on=True):
    return _check(load().pdqp_profile_enable(h, 1 if on else 0), h)


def pdqp_profile_read(h) -> dict:
    pr = pdqp_profile()
    _check(load().pdqp_profile_read(h, ctypes.byref(pr)), h)
    names = ("dual", "primal", "check", "other")
    return {nm: dict(launches=int(pr.launches[k]), ms=float(pr.ms[k]), bytes=float(pr.bytes[k]))
            for k, nm in enumerate(names)}


# ---------------------------------------------------------------------------
# convenience: a handle from scipy CSR data (marshalling only)
# ---------------------------------------------------------------------------
def batch_from_instances(insts, device=False, stream=None):
    """A batch handle from objects with n, m, m_eq, Q, A (scipy CSR), c, b, l, u."""
    entries = []
    for it in insts:
        arrays = [it.Q.indptr, it.Q.indices, it.Q.data, it.A.indptr, it.A.indices, it.A.data, it.c, it.b, it.l, it.u]
        dtypes = [np.int32, np.int32, np.float64] * 2 + [np.float64] * 4
        arrays = [np.ascontiguousarray(a, dtype=t) for a, t in zip(arrays, dtypes)]
        if device:
            import torch
            arrays = [torch.from_numpy(a).cuda() for a in arrays]
        entries.append((it.n, it.m, it.m_eq, *arrays))
    if device:
        import torch
        torch.cuda.synchronize()
    return pdqp_create_batch(entries, stream=stream)


def pack_instances(insts):
    """The block-diagonal form pdqp_create_batch_packed takes, from objects with
    n, m, m_eq, Q, A (scipy CSR), c, b, l, u: a dict of the sizes (n, m, m_eq)
    and the ten arrays (int32 row pointers and global columns, float64 values
    and vectors)."""
    n = np.array([it.n for it in insts], np.int64)
    m = np.array([it.m for it in insts], np.int64)
    xoff = np.concatenate([[0], np.cumsum(n)])

    def stack(mats, rows):
        nnz = np.array([M.indptr[rows[k]] for k, M in enumerate(mats)], np.int64)
        eoff = np.concatenate([[0], np.cumsum(nnz)])
        rp = np.concatenate([[0]] + [M.indptr[1:rows[k] + 1].astype(np.int64) + eoff[k]
                                     for k, M in enumerate(mats)]).astype(np.int32)
        col = np.concatenate([np.zeros(0, np.int64)] + [M.indices[:nnz[k]].astype(np.int64) + xoff[k]
                                                        for k, M in enumerate(mats)]).astype(np.int32)
        val = np.concatenate([np.zeros(0)] + [np.asarray(M.data[:nnz[k]], np.float64) for k, M in enumerate(mats)])
        return rp, col, val

    Qrp, Qcol, Qval = stack([it.Q for it in insts], n)
    Arp, Acol, Aval = stack([it.A for it in insts], m)
    cat = lambda f: np.concatenate([np.zeros(0)] + [np.asarray(getattr(it, f), np.float64) for it in insts])
    return dict(n=n, m=m, m_eq=np.array([it.m_eq for it in insts], np.int64), Q_rowptr=Qrp, Q_col=Qcol,
                Q_val=Qval, A_rowptr=Arp, A_col=Acol, A_val=Aval, c=cat("c"), b=cat("b"), l=cat("l"), u=cat("u"))


def create_from_csr(n, m, m_eq, Q, A, c, b, l, u, device=False, stream=None):
    """Q, A: scipy.sparse CSR (int32 indices).  device=True uploads the arrays
    as torch CUDA tensors first, exercising the PDQP_MEM_DEVICE path."""
    arrays = [Q.indptr, Q.indices, Q.data, A.indptr, A.indices, A.data, c, b, l, u]
    dtypes = [np.int32, np.int32, np.float64] * 2 + [np.float64] * 4
    arrays = [np.ascontiguousarray(a, dtype=t) for a, t in zip(arrays, dtypes)]
    if device:
        import torch
        arrays = [torch.from_numpy(a).cuda() for a in arrays]
        torch.cuda.synchronize()
    return pdqp_create(n, m, m_eq, *arrays, stream=stream)


# ---------------------------------------------------------------------------
# learned warm start (include/pdqp_ws.h)
# ---------------------------------------------------------------------------
def _ws_check(status, w=None):
    if status != PDQP_OK:
        raise PdqpError(status, load().pdqp_ws_last_error(w).decode())
    return status


def _ws_arrays(arrays, dtype):
    args = [_ptr(a, dtype) for a in arrays]
    return [a[0] for a in args], [a[1] for a in args], _one_space([a[2] for a in args])


def pdqp_ws_create(n, m, d=1024, width=1024, depth=3, max_batch=512, stream=None):
    w = ctypes.c_void_p()
    _ws_check(load().pdqp_ws_create(ctypes.byref(w), int(n), int(m), int(d), int(width), int(depth),
                                    int(max_batch), _stream(stream)), None)
    return w


def pdqp_ws_destroy(w):
    load().pdqp_ws_destroy(w)


def pdqp_ws_set_params(w, layer, W, b=None, stream=None):
    ptrs, keep, mem = _ws_arrays([W, b], np.float32)
    return _ws_check(load().pdqp_ws_set_params(w, int(layer), ptrs[0], ptrs[1], mem, _stream(stream)), w)


def pdqp_ws_get_params(w, layer, what=0, W=None, b=None, stream=None):
    """Fill W and/or b (float32 numpy arrays or torch CUDA tensors) in place."""
    for a in (W, b):
        if a is not None and not _is_torch_cuda(a):
            assert isinstance(a, np.ndarray) and a.dtype == np.float32 and a.flags.c_contiguous
    ptrs, keep, mem = _ws_arrays([W, b], np.float32)
    return _ws_check(load().pdqp_ws_get_params(w, int(layer), int(what), ptrs[0], ptrs[1], mem, _stream(stream)), w)


def pdqp_ws_set_normalization(w, in_mean, in_scale, out_mean, out_std, out_inv, stream=None):
    ptrs, keep, mem = _ws_arrays([in_mean, in_scale, out_mean, out_std, out_inv], np.float32)
    return _ws_check(load().pdqp_ws_set_normalization(w, *ptrs, mem, _stream(stream)), w)


def pdqp_ws_get_normalization(w, F, stream=None):
    out = [np.zeros(F, np.float32) for _ in range(5)]
    ptrs = [ctypes.c_void_p(a.ctypes.data) for a in out]
    _ws_check(load().pdqp_ws_get_normalization(w, *ptrs, PDQP_MEM_HOST, _stream(stream)), w)
    return dict(zip(("in_mean", "in_scale", "out_mean", "out_std", "out_inv"), out))


def pdqp_ws_fit(w, C, B, X, Y, stream=None):
    ptrs, keep, mem = _ws_arrays([C, B, X, Y], np.float64)
    return _ws_check(load().pdqp_ws_fit(w, *ptrs, int(C.shape[0]), mem, _stream(stream)), w)


def pdqp_ws_grad(w, C, B, X, Y, stream=None) -> float:
    ptrs, keep, mem = _ws_arrays([C, B, X, Y], np.float64)
    loss = ctypes.c_double()
    _ws_check(load().pdqp_ws_grad(w, *ptrs, int(C.shape[0]), ctypes.byref(loss), mem, _stream(stream)), w)
    return loss.value


def pdqp_ws_train(w, C, B, X, Y, epochs=10, batch=256, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, seed=0,
                  stream=None):
    """Returns the mean minibatch loss of every epoch (numpy float64)."""
    opt = pdqp_ws_train_options(int(epochs), int(batch), float(lr), float(beta1), float(beta2), float(eps),
                                int(seed))
    ptrs, keep, mem = _ws_arrays([C, B, X, Y], np.float64)
    losses = np.zeros(max(int(epochs), 1))
    _ws_check(load().pdqp_ws_train(w, ctypes.byref(opt), *ptrs, int(C.shape[0]),
                                   ctypes.c_void_p(losses.ctypes.data), mem, _stream(stream)), w)
    return losses[:int(epochs)]


def pdqp_ws_infer(w, C, B, X0, Y0, stream=None):
    """Write the predicted warm starts into X0 [count x n] and Y0 [count x m]
    (float64 numpy arrays or torch CUDA tensors, in place)."""
    for a in (X0, Y0):
        if a is not None and not _is_torch_cuda(a):
            assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous
    ptrs, keep, mem = _ws_arrays([C, B, X0, Y0], np.float64)
    return _ws_check(load().pdqp_ws_infer(w, ptrs[0], ptrs[1], int(C.shape[0]), ptrs[2], ptrs[3], mem,
                                          _stream(stream)), w)


def pdqp_gemm_bf16(A, B, bias=None, relu=False, mask=None, D_f32=None, D_bf16=None, splits=0, workspace=None,
                   M=None, N=None, K=None, stream=None):
    """D = A B' on torch CUDA tensors: A (M x lda) and B (N x ldb) bfloat16,
    bias float32 [N], mask bfloat16 (M x ldm), D_f32 float32 / D_bf16 bfloat16
    (M x ldd), workspace float32.  M, N, K default to the shapes of A and B."""
    M = A.shape[0] if M is None else M
    N = B.shape[0] if N is None else N
    K = A.shape[1] if K is None else K
    D = D_f32 if D_f32 is not None else D_bf16
    p = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    st = load().pdqp_gemm_bf16(int(M), int(N), int(K), p(A), int(A.stride(0)), p(B), int(B.stride(0)), p(bias),
                               int(bool(relu)), p(mask), int(mask.stride(0)) if mask is not None else 0,
                               p(D_f32), p(D_bf16), int(D.stride(0)), int(splits), p(workspace),
                               int(workspace.numel() * 4) if workspace is not None else 0, _stream(stream))
    if st != PDQP_OK:
        raise PdqpError(st, "pdqp_gemm_bf16 rejected its arguments")
    return st


def pdqp_gemm_bf16_check(stream=None):
    return int(load().pdqp_gemm_bf16_check(_stream(stream)))


def pdqp_gemm_bf16_wait_probe(stream=None):
    """Status of a bounded device wait that runs out (PDQP_DEVICE_TIMEOUT)."""
    return int(load().pdqp_gemm_bf16_wait_probe(_stream(stream)))


def pdqp_gemm_bf16_splits(M, N, K, splits=0):
    return int(load().pdqp_gemm_bf16_splits(int(M), int(N), int(K), int(splits)))
