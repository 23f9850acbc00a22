"""Thin ctypes binding of libbm.so (include/bm.h).

Argument marshalling only: every computation runs in the CUDA library.  The
functions carry the C names; arrays may be numpy arrays (host) or torch
tensors (host or CUDA).  A failing status raises BMError with the library's
message.  If libbm.so is missing the import of a function fails loudly; there
is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("BM_LIB", os.path.join(HERE, "libbm.so"))
HEADER = os.path.join(os.path.dirname(HERE), "include", "bm.h")

BM_OK, BM_ERR_INVALID, BM_ERR_OOM, BM_ERR_CUDA, BM_ERR_TIMEOUT, BM_ERR_NUMERIC, BM_ERR_NOT_CONVERGED = range(7)
STATUS_NAMES = ["BM_OK", "BM_ERR_INVALID", "BM_ERR_OOM", "BM_ERR_CUDA", "BM_ERR_TIMEOUT",
                "BM_ERR_NUMERIC", "BM_ERR_NOT_CONVERGED"]


class BMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class bm_options(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("bm_epochs", ctypes.c_int32), ("pg_steps", ctypes.c_int32),
                ("lmsvd_p", ctypes.c_int32), ("lmsvd_imax", ctypes.c_int32), ("lmsvd_min_iter", ctypes.c_int32),
                ("lmsvd_tol", ctypes.c_double), ("tau", ctypes.c_double), ("ritz_rel", ctypes.c_double),
                ("psi0", ctypes.c_double), ("k_init", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("autotune", ctypes.c_int32), ("step_rule", ctypes.c_int32),
                ("value_codec", ctypes.c_int32), ("bm_solver", ctypes.c_int32), ("tensor_grams", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


class bm_bb_options(ctypes.Structure):
    _fields_ = [("alpha_min", ctypes.c_double), ("alpha_max", ctypes.c_double), ("beta", ctypes.c_double),
                ("delta", ctypes.c_double), ("max_backtracks", ctypes.c_int32), ("pad_", ctypes.c_int32)]


class bm_bb_info(ctypes.Structure):
    _fields_ = [("alpha_bb", ctypes.c_double), ("alpha", ctypes.c_double), ("backtracks", ctypes.c_int32),
                ("accepted_by", ctypes.c_int32)]


BM_PASS_KINDS = 5
BM_MAX_PANELS = 16
PASS_NAMES = ("grad_csr", "grad_csc", "linesearch_csr", "spmm_csr", "spmm_csc")


class bm_tune_info(ctypes.Structure):
    _fields_ = [("panels", ctypes.c_int32 * BM_PASS_KINDS), ("timed", ctypes.c_int32),
                ("ms", ctypes.c_double * BM_PASS_KINDS), ("ms_single", ctypes.c_double * BM_PASS_KINDS),
                ("layout", ctypes.c_int32 * BM_PASS_KINDS), ("pad_", ctypes.c_int32)]


class bm_prox_info(ctypes.Structure):
    _fields_ = [("k_new", ctypes.c_int32), ("warm_cols", ctypes.c_int32), ("lmsvd_iters", ctypes.c_int32),
                ("n_L", ctypes.c_int32), ("cap_hit", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("eps", ctypes.c_double), ("F", ctypes.c_double)]


class bm_solve_opts(ctypes.Structure):
    _fields_ = [("max_outer", ctypes.c_int32), ("pad_", ctypes.c_int32), ("tol", ctypes.c_double),
                ("F_target", ctypes.c_double), ("time_limit_s", ctypes.c_double)]


class bm_solve_info(ctypes.Structure):
    _fields_ = [("outer", ctypes.c_int32), ("k", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("pad_", ctypes.c_int32), ("F", ctypes.c_double), ("seconds", ctypes.c_double)]


_lib = None
_c = ctypes
_P = ctypes.c_void_p
_SIGS = {
    "bm_default_options": (_c.c_int, [_c.POINTER(bm_options)]),
    "bm_create": (_c.c_int, [_c.c_int64, _c.c_int64, _c.c_int64, _P, _P, _P, _c.c_double, _c.c_int32,
                             _c.POINTER(bm_options), _c.POINTER(_P)]),
    "bm_destroy": (None, [_P]),
    "bm_last_error": (_c.c_char_p, [_P]),
    "bm_set_stream": (_c.c_int, [_P, _P]),
    "bm_dims": (_c.c_int, [_P, _P, _P, _P, _P, _P]),
    "bm_get_index": (_c.c_int, [_P, _P, _P, _P, _P, _P, _P, _P]),
    "bm_set_factors": (_c.c_int, [_P, _c.c_int32, _P, _P]),
    "bm_get_factors": (_c.c_int, [_P, _P, _P, _P]),
    "bm_loss_grad": (_c.c_int, [_P, _P, _P, _P, _P]),
    "bm_bm_phase": (_c.c_int, [_P, _c.c_int32, _P]),
    "bm_init": (_c.c_int, [_P, _c.POINTER(bm_prox_info)]),
    "bm_prox_step": (_c.c_int, [_P, _c.c_double, _c.POINTER(bm_prox_info)]),
    "bm_bb_default_options": (_c.c_int, [_c.POINTER(bm_bb_options)]),
    "bm_bcd_phase": (_c.c_int, [_P, _c.c_int32, _c.POINTER(_c.c_double)]),
    "bm_get_codes": (_c.c_int, [_P, _c.POINTER(_c.c_int32), _c.POINTER(_c.c_float), _P, _P]),
    "bm_set_bb_options": (_c.c_int, [_P, _c.POINTER(bm_bb_options)]),
    "bm_prox_step_bb": (_c.c_int, [_P, _c.POINTER(bm_prox_info), _c.POINTER(bm_bb_info)]),
    "bm_solve": (_c.c_int, [_P, _c.POINTER(bm_solve_opts), _c.POINTER(bm_solve_info)]),
    "bm_profile_enable": (_c.c_int, [_P, _c.c_int32]),
    "bm_autotune": (_c.c_int, [_P, _c.c_int32, _c.POINTER(bm_tune_info)]),
    "bm_get_state": (_c.c_int, [_P, _P, _c.POINTER(_c.c_size_t)]),
    "bm_set_state": (_c.c_int, [_P, _P, _c.c_size_t]),
    "bm_set_panels": (_c.c_int, [_P, _c.POINTER(_c.c_int32)]),
    "bm_get_panels": (_c.c_int, [_P, _c.POINTER(_c.c_int32)]),
    "bm_set_layout": (_c.c_int, [_P, _c.POINTER(_c.c_int32)]),
    "bm_gather_roof": (_c.c_int, [_P, _c.c_int32, _c.POINTER(_c.c_double), _c.POINTER(_c.c_double)]),
    "bm_dense_gram": (_c.c_int, [_P, _c.c_int64, _c.c_int32, _c.c_int32, _P, _c.c_int32, _c.c_int32, _P, _c.c_int32,
                                 _P]),
    "bm_dense_last_error": (_c.c_char_p, []),
    "bm_sym_eig": (_c.c_int, [_P, _c.c_int32, _P, _P, _c.c_int32, _P]),
    "bm_get_layout": (_c.c_int, [_P, _c.POINTER(_c.c_int32)]),
    "bm_profile_read": (_c.c_int, [_P, _c.c_int32, _P, _P, _P, _P]),
}


def header_symbols() -> list:
    """Function names declared in include/bm.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bm_[a-z_0-9]+)\s*\(", txt)))


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing; build it with paper_2204_14067_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(x):
    """Address of a numpy array / torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def _check(status: int, h=None):
    if status != BM_OK:
        msg = lib().bm_last_error(h)
        raise BMError(status, msg.decode() if msg else "")


def bm_default_options() -> bm_options:
    o = bm_options()
    _check(lib().bm_default_options(ctypes.byref(o)))
    return o


def bm_create(m, n, rows, cols, vals, lam, k_max, opt: bm_options | None = None):
    """Returns an opaque handle (int).  rows/cols int32, vals float32."""
    for a, dt in ((rows, "int32"), (cols, "int32"), (vals, "float32")):
        if str(a.dtype).replace("torch.", "") != dt:
            raise TypeError(f"expected {dt}, got {a.dtype}")
    nnz = int(rows.shape[0])
    h = _P()
    st = lib().bm_create(int(m), int(n), nnz, _ptr(rows), _ptr(cols), _ptr(vals), float(lam), int(k_max),
                         ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    _check(st, None)
    return h.value


def bm_destroy(h):
    lib().bm_destroy(h)


def bm_last_error(h=None) -> str:
    return lib().bm_last_error(h).decode()


def bm_set_stream(h, stream):
    """stream: torch.cuda.Stream, a raw cudaStream_t int, or None."""
    raw = getattr(stream, "cuda_stream", stream)
    _check(lib().bm_set_stream(h, raw), h)


def bm_dims(h):
    m, n, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    tr, k = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().bm_dims(h, ctypes.byref(m), ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(tr),
                         ctypes.byref(k)), h)
    return dict(m=m.value, n=n.value, nnz=nnz.value, transposed=bool(tr.value), k=k.value)


def bm_get_index(h):
    """Index arrays (internal orientation) as numpy host arrays."""
    d = bm_dims(h)
    m, n, nnz = d["m"], d["n"], d["nnz"]
    out = dict(row_ptr=np.empty(m + 1, np.int64), col=np.empty(nnz, np.int32), val=np.empty(nnz, np.float32),
               col_ptr=np.empty(n + 1, np.int64), row=np.empty(nnz, np.int32), cval=np.empty(nnz, np.float32),
               csr2csc=np.empty(nnz, np.int64))
    _check(lib().bm_get_index(h, *(_ptr(out[k]) for k in
                                   ("row_ptr", "col", "val", "col_ptr", "row", "cval", "csr2csc"))), h)
    return out


def bm_set_factors(h, k, W, H):
    _check(lib().bm_set_factors(h, int(k), _ptr(W), _ptr(H)), h)


def bm_get_factors(h, m, n, W=None, H=None):
    """Caller-orientation factors; allocates host arrays if W/H are None."""
    kk = ctypes.c_int32()
    _check(lib().bm_dims(h, None, None, None, None, ctypes.byref(kk)), h)
    k = kk.value
    if W is None:
        W = np.zeros((m, k), np.float32)
    if H is None:
        H = np.zeros((n, k), np.float32)
    _check(lib().bm_get_factors(h, ctypes.byref(kk), _ptr(W), _ptr(H)), h)
    return W, H


def bm_loss_grad(h, gW=None, gH=None):
    """Returns (f, F); writes gradients into gW / gH if given."""
    f, F = ctypes.c_double(), ctypes.c_double()
    _check(lib().bm_loss_grad(h, ctypes.byref(f), ctypes.byref(F), _ptr(gW), _ptr(gH)), h)
    return f.value, F.value


def bm_bm_phase(h, epochs):
    F = ctypes.c_double()
    _check(lib().bm_bm_phase(h, int(epochs), ctypes.byref(F)), h)
    return F.value


def _info_dict(info: bm_prox_info):
    return {name: getattr(info, name) for name, _ in bm_prox_info._fields_ if name != "pad_"}


def bm_init(h):
    info = bm_prox_info()
    _check(lib().bm_init(h, ctypes.byref(info)), h)
    return _info_dict(info)


def bm_prox_step(h, alpha=0.0):
    info = bm_prox_info()
    _check(lib().bm_prox_step(h, float(alpha), ctypes.byref(info)), h)
    return _info_dict(info)


def bm_bcd_phase(h, epochs):
    """`epochs` sweeps of the column-block BM solver; returns F after them."""
    F = ctypes.c_double()
    _check(lib().bm_bcd_phase(h, int(epochs), ctypes.byref(F)), h)
    return F.value


def bm_get_codes(h, nnz=None):
    """(active, offset, csr_codes, csc_codes); the code arrays only when active and nnz is given."""
    act = ctypes.c_int32()
    off = ctypes.c_float()
    _check(lib().bm_get_codes(h, ctypes.byref(act), ctypes.byref(off), None, None), h)
    if not act.value or nnz is None:
        return bool(act.value), off.value, None, None
    a = np.zeros(nnz, np.uint8)
    b = np.zeros(nnz, np.uint8)
    _check(lib().bm_get_codes(h, None, None, _ptr(a), _ptr(b)), h)
    return True, off.value, a, b


def bm_bb_default_options() -> bm_bb_options:
    o = bm_bb_options()
    _check(lib().bm_bb_default_options(ctypes.byref(o)))
    return o


def bm_set_bb_options(h, o: bm_bb_options):
    _check(lib().bm_set_bb_options(h, ctypes.byref(o)), h)


def bm_prox_step_bb(h):
    """One PG step with the SpaRSA step rule: (prox info dict, step record dict)."""
    info = bm_prox_info()
    bb = bm_bb_info()
    _check(lib().bm_prox_step_bb(h, ctypes.byref(info), ctypes.byref(bb)), h)
    return _info_dict(info), {"alpha_bb": bb.alpha_bb, "alpha": bb.alpha, "backtracks": bb.backtracks,
                              "accepted_by": bb.accepted_by}


def bm_solve(h, max_outer=100, tol=1e-10, F_target=0.0, time_limit_s=0.0, raise_not_converged=False):
    o = bm_solve_opts(max_outer=int(max_outer), tol=float(tol), F_target=float(F_target),
                      time_limit_s=float(time_limit_s))
    info = bm_solve_info()
    st = lib().bm_solve(h, ctypes.byref(o), ctypes.byref(info))
    if st != BM_OK and not (st == BM_ERR_NOT_CONVERGED and not raise_not_converged):
        _check(st, h)
    return dict(outer=info.outer, k=info.k, converged=bool(info.converged), F=info.F, seconds=info.seconds,
                status=st)


def bm_autotune(h, max_panels=BM_MAX_PANELS):
    """Time the sparse passes' work splits and kernel layouts and keep the
    fastest; returns {pass name: (panels, ms chosen, ms with one panel and the
    automatic layout, layout)}."""
    info = bm_tune_info()
    _check(lib().bm_autotune(h, int(max_panels), ctypes.byref(info)), h)
    return {nm: (int(info.panels[i]), float(info.ms[i]), float(info.ms_single[i]), int(info.layout[i]))
            for i, nm in enumerate(PASS_NAMES)}


def bm_state_size(h) -> int:
    """Bytes of the solve-state checkpoint."""
    n = ctypes.c_size_t(0)
    _check(lib().bm_get_state(h, None, ctypes.byref(n)), h)
    return n.value


def bm_get_state(h, out=None):
    """Checkpoint of the solve state.  Without `out`: host bytes.  With `out`
    (a contiguous host numpy uint8 array or CPU torch tensor, e.g. pinned, of
    at least bm_state_size bytes): written in place, returns the byte count."""
    if out is not None:
        n = ctypes.c_size_t(int(out.nbytes) if hasattr(out, "nbytes") else out.numel() * out.element_size())
        _check(lib().bm_get_state(h, _ptr(out), ctypes.byref(n)), h)
        return n.value
    n = ctypes.c_size_t(0)
    _check(lib().bm_get_state(h, None, ctypes.byref(n)), h)
    buf = ctypes.create_string_buffer(n.value)
    _check(lib().bm_get_state(h, buf, ctypes.byref(n)), h)
    return buf.raw[: n.value]


def bm_set_state(h, state, nbytes=None):
    """Restore a checkpoint: bytes, or a host numpy uint8 array / CPU torch
    tensor (read in place; nbytes = the state's length when the buffer is larger)."""
    if isinstance(state, (bytes, bytearray)):
        buf = ctypes.create_string_buffer(bytes(state), len(state))
        _check(lib().bm_set_state(h, buf, len(state)), h)
        return
    n = int(nbytes) if nbytes is not None else (int(state.nbytes) if hasattr(state, "nbytes")
                                                 else state.numel() * state.element_size())
    _check(lib().bm_set_state(h, _ptr(state), n), h)


def bm_set_panels(h, panels):
    arr = (ctypes.c_int32 * BM_PASS_KINDS)(*[int(x) for x in panels])
    _check(lib().bm_set_panels(h, arr), h)


def bm_get_panels(h):
    arr = (ctypes.c_int32 * BM_PASS_KINDS)()
    _check(lib().bm_get_panels(h, arr), h)
    return [int(x) for x in arr]


def bm_gather_roof(h, kind):
    """(ms, GB/s) of a gather-only pass over pass kind `kind` (index into PASS_NAMES or its name)."""
    if isinstance(kind, str):
        kind = PASS_NAMES.index(kind)
    ms, gbs = ctypes.c_double(), ctypes.c_double()
    _check(lib().bm_gather_roof(h, int(kind), ctypes.byref(ms), ctypes.byref(gbs)), h)
    return ms.value, gbs.value


def bm_dense_gram(A, B, C, mode, stream=None):
    """C (a x b float64 CUDA tensor) = A^T B for CUDA float32 tensors A (L x lda), B (L x ldb) whose
    leading a, b columns are used (a = C.shape[0], b = C.shape[1]); mode 0 FP32 pipes, 1 compensated,
    2 tensor cores."""
    raw = getattr(stream, "cuda_stream", stream)
    a, b = int(C.shape[0]), int(C.shape[1])
    st = lib().bm_dense_gram(_ptr(A), int(A.shape[0]), a, int(A.shape[1]), _ptr(B), b, int(B.shape[1]), _ptr(C),
                             int(mode), raw)
    if st != BM_OK:
        msg = lib().bm_dense_last_error()
        raise BMError(st, msg.decode() if msg else "")


def bm_sym_eig(S, evals, evecs, mode, stream=None):
    """evals (n float64 CUDA tensor, descending) and evecs (n x n, column j = vector j) of the symmetric
    n x n float64 CUDA tensor S; mode 0 FP32 QL, 1 with relative FP32 Jacobi refinement, 2 FP64 refinement."""
    raw = getattr(stream, "cuda_stream", stream)
    st = lib().bm_sym_eig(_ptr(S), int(S.shape[0]), _ptr(evals), _ptr(evecs), int(mode), raw)
    if st != BM_OK:
        msg = lib().bm_dense_last_error()
        raise BMError(st, msg.decode() if msg else "")


def bm_set_layout(h, layout):
    """Kernel layout per pass kind: -1 automatic, 0 lane group per segment, 1 warp per segment."""
    arr = (ctypes.c_int32 * BM_PASS_KINDS)(*[int(x) for x in layout])
    _check(lib().bm_set_layout(h, arr), h)


def bm_get_layout(h):
    arr = (ctypes.c_int32 * BM_PASS_KINDS)()
    _check(lib().bm_get_layout(h, arr), h)
    return [int(x) for x in arr]


def bm_profile_enable(h, enable=True):
    _check(lib().bm_profile_enable(h, 1 if enable else 0), h)


def bm_profile_read(h, cap=64):
    """{kernel name: (launches, total_ms)} since the last bm_profile_enable."""
    names = ctypes.create_string_buffer(48 * cap)
    launches = np.zeros(cap, np.int64)
    ms = np.zeros(cap, np.float64)
    cnt = ctypes.c_int32()
    _check(lib().bm_profile_read(h, cap, names, _ptr(launches), _ptr(ms), ctypes.byref(cnt)), h)
    out = {}
    for i in range(min(cnt.value, cap)):
        nm = names.raw[48 * i:48 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (int(launches[i]), float(ms[i]))
    return out


_SIGS.update({
    "bm_edm_create": (_c.c_int, [_c.c_int64, _c.c_int64, _P, _P, _P, _P, _c.c_double, _c.c_int32,
                                 _c.POINTER(_P)]),
    "bm_edm_destroy": (None, [_P]),
    "bm_edm_last_error": (_c.c_char_p, [_P]),
    "bm_edm_set_factor": (_c.c_int, [_P, _c.c_int32, _P]),
    "bm_edm_loss_grad": (_c.c_int, [_P, _P, _P]),
    "bm_edm_set_stream": (_c.c_int, [_P, _P]),
    "bm_edm_set_options": (_c.c_int, [_P, _c.POINTER(bm_options)]),
    "bm_edm_init": (_c.c_int, [_P, _c.POINTER(bm_prox_info)]),
    "bm_edm_bm_phase": (_c.c_int, [_P, _c.c_int32, _c.POINTER(_c.c_double)]),
    "bm_edm_prox_step": (_c.c_int, [_P, _c.POINTER(bm_prox_info)]),
    "bm_edm_solve": (_c.c_int, [_P, _c.POINTER(bm_solve_opts), _c.POINTER(bm_solve_info)]),
    "bm_edm_get_factor": (_c.c_int, [_P, _c.POINTER(_c.c_int32), _P]),
    "bm_edm_profile_enable": (_c.c_int, [_P, _c.c_int32]),
    "bm_edm_profile_read": (_c.c_int, [_P, _c.c_int32, _P, _P, _P, _c.POINTER(_c.c_int32)]),
})


def _check_edm(status: int, h=None):
    if status != BM_OK:
        msg = lib().bm_edm_last_error(h)
        raise BMError(status, msg.decode() if msg else "")


def bm_edm_create(n, i, j, d, lam, k_max, w=None):
    h = _P()
    _check_edm(lib().bm_edm_create(int(n), int(i.shape[0]), _ptr(i), _ptr(j), _ptr(d), _ptr(w), float(lam),
                                   int(k_max), ctypes.byref(h)))
    return h.value


def bm_edm_destroy(h):
    lib().bm_edm_destroy(h)


def bm_edm_set_factor(h, k, V):
    _check_edm(lib().bm_edm_set_factor(h, int(k), _ptr(V)), h)


def _edm_info(info: bm_prox_info):
    return {"rank": info.k_new, "computed": info.warm_cols, "lmsvd_iters": info.lmsvd_iters,
            "k_next": info.n_L, "all_positive": bool(info.cap_hit), "sigma": info.eps, "F": info.F}


def bm_edm_set_options(h, o: bm_options):
    _check_edm(lib().bm_edm_set_options(h, ctypes.byref(o)), h)


def bm_edm_init(h):
    info = bm_prox_info()
    _check_edm(lib().bm_edm_init(h, ctypes.byref(info)), h)
    return _edm_info(info)


def bm_edm_bm_phase(h, epochs):
    F = ctypes.c_double()
    _check_edm(lib().bm_edm_bm_phase(h, int(epochs), ctypes.byref(F)), h)
    return F.value


def bm_edm_prox_step(h):
    info = bm_prox_info()
    _check_edm(lib().bm_edm_prox_step(h, ctypes.byref(info)), h)
    return _edm_info(info)


def bm_edm_solve(h, max_outer=100, tol=1e-10, F_target=0.0, time_limit_s=0.0):
    o = bm_solve_opts(max_outer=int(max_outer), tol=float(tol), F_target=float(F_target),
                      time_limit_s=float(time_limit_s))
    info = bm_solve_info()
    st = lib().bm_edm_solve(h, ctypes.byref(o), ctypes.byref(info))
    if st not in (BM_OK, BM_ERR_NOT_CONVERGED):
        _check_edm(st, h)
    return {"outer": info.outer, "k": info.k, "converged": bool(info.converged), "F": info.F,
            "seconds": info.seconds}


def bm_edm_get_factor(h, n):
    kk = ctypes.c_int32()
    _check_edm(lib().bm_edm_get_factor(h, ctypes.byref(kk), None), h)
    V = np.zeros((n, kk.value), np.float32)
    if kk.value:
        _check_edm(lib().bm_edm_get_factor(h, None, _ptr(V)), h)
    return V


def bm_edm_profile_enable(h, enable=True):
    _check_edm(lib().bm_edm_profile_enable(h, 1 if enable else 0), h)


def bm_edm_profile_read(h, cap=64):
    """{kernel name: (launches, total_ms)} since the last bm_edm_profile_enable."""
    names = ctypes.create_string_buffer(48 * cap)
    launches = np.zeros(cap, np.int64)
    ms = np.zeros(cap, np.float64)
    cnt = ctypes.c_int32()
    _check_edm(lib().bm_edm_profile_read(h, cap, names, _ptr(launches), _ptr(ms), ctypes.byref(cnt)), h)
    out = {}
    for i in range(min(cnt.value, cap)):
        nm = names.raw[48 * i:48 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (int(launches[i]), float(ms[i]))
    return out


def bm_edm_set_stream(h, stream):
    ptr = stream.cuda_stream if hasattr(stream, "cuda_stream") else (stream or 0)
    _check_edm(lib().bm_edm_set_stream(h, ctypes.c_void_p(ptr)), h)


def bm_edm_loss_grad(h, gV=None):
    g = ctypes.c_double()
    _check_edm(lib().bm_edm_loss_grad(h, ctypes.byref(g), _ptr(gV)), h)
    return g.value


_SIGS.update({
    "bm_loss_grad_csr_noalloc": (_c.c_int, [_c.c_int64, _c.c_int64, _P, _P, _P, _P, _P, _c.c_int32, _c.c_int32,
                                            _c.c_double, _P, _P, _P]),
    "bm_noalloc_last_error": (_c.c_char_p, []),
})


def bm_loss_grad_csr_noalloc(m, n, row_ptr, col, val, W, H, k, ld, lam, gW, f, stream=None):
    """Allocation-free CSR loss/gradient; all arrays are CUDA tensors, f a 1-element float64 tensor."""
    raw = getattr(stream, "cuda_stream", stream)
    st = lib().bm_loss_grad_csr_noalloc(int(m), int(n), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(W), _ptr(H),
                                         int(k), int(ld), float(lam), _ptr(gW), _ptr(f), raw)
    if st != BM_OK:
        msg = lib().bm_noalloc_last_error()
        raise BMError(st, msg.decode() if msg else "")


_SIGS.update({
    "bm_batch_create": (_c.c_int, [_P, _c.c_int32, _c.POINTER(_P)]),
    "bm_batch_destroy": (None, [_P]),
    "bm_batch_last_error": (_c.c_char_p, [_P]),
    "bm_batch_bm_phase": (_c.c_int, [_P, _c.c_int32, _P]),
    "bm_batch_prox_step": (_c.c_int, [_P, _c.c_double, _c.POINTER(bm_prox_info), _P]),
    "bm_batch_stats": (_c.c_int, [_P, _c.POINTER(_c.c_int64), _c.POINTER(_c.c_int64)]),
})


def _check_batch(status: int, b=None):
    if status != BM_OK:
        msg = lib().bm_batch_last_error(b)
        raise BMError(status, msg.decode() if msg else "")


def bm_batch_create(handles):
    arr = (_P * len(handles))(*handles)
    b = _P()
    _check_batch(lib().bm_batch_create(arr, len(handles), ctypes.byref(b)))
    return b.value


def bm_batch_destroy(b):
    lib().bm_batch_destroy(b)


def bm_batch_bm_phase(b, count, epochs):
    F = np.zeros(count, np.float64)
    _check_batch(lib().bm_batch_bm_phase(b, int(epochs), _ptr(F)), b)
    return F


def bm_batch_prox_step(b, count, alpha=0.0):
    """One PG step on every handle of the batch (shared SpMM launches); a list of info dicts."""
    infos = (bm_prox_info * count)()
    _check_batch(lib().bm_batch_prox_step(b, float(alpha), infos, None), b)
    return [_info_dict(infos[i]) for i in range(count)]


def bm_batch_stats(b):
    """(products handed to the shared SpMM launches, launches made for them) so far."""
    p, n = ctypes.c_int64(), ctypes.c_int64()
    _check_batch(lib().bm_batch_stats(b, ctypes.byref(p), ctypes.byref(n)), b)
    return p.value, n.value


class bm_server_opts(ctypes.Structure):
    _fields_ = [("max_active", ctypes.c_int32), ("precision", ctypes.c_int32), ("batched", ctypes.c_int32),
                ("workers", ctypes.c_int32), ("mem_budget_gb", ctypes.c_double), ("max_outer", ctypes.c_int32),
                ("keep_factors", ctypes.c_int32), ("tol", ctypes.c_double)]


class bm_request_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("k", ctypes.c_int32),
                ("outer", ctypes.c_int32), ("pad_", ctypes.c_int32), ("F", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


_SIGS.update({
    "bm_server_create": (_c.c_int, [_c.POINTER(bm_server_opts), _c.POINTER(_P)]),
    "bm_server_submit": (_c.c_int, [_P, _c.c_int64, _c.c_int64, _c.c_int64, _P, _P, _P, _c.c_double, _c.c_int32,
                                    _P]),
    "bm_server_drain": (_c.c_int, [_P, _c.c_double]),
    "bm_server_results": (_c.c_int, [_P, _P, _c.c_int32, _P]),
    "bm_server_factors": (_c.c_int, [_P, _c.c_int64, _P, _P, _P]),
    "bm_server_now": (_c.c_double, [_P]),
    "bm_server_last_error": (_c.c_char_p, [_P]),
    "bm_server_destroy": (None, [_P]),
})


def _check_server(status: int, s=None):
    if status != BM_OK:
        msg = lib().bm_server_last_error(s)
        raise BMError(status, msg.decode() if msg else "")


def bm_server_create(max_active=16, precision=0, batched=1, workers=8, mem_budget_gb=0.0, max_outer=100,
                     tol=1e-6, keep_factors=0):
    o = bm_server_opts(max_active=max_active, precision=precision, batched=batched, workers=workers,
                       mem_budget_gb=mem_budget_gb, max_outer=max_outer, tol=tol, keep_factors=keep_factors)
    s = _P()
    _check_server(lib().bm_server_create(ctypes.byref(o), ctypes.byref(s)))
    return s.value


def bm_server_submit(s, m, n, rows, cols, vals, lam, k_max):
    rid = ctypes.c_int64()
    _check_server(lib().bm_server_submit(s, int(m), int(n), int(rows.shape[0]), _ptr(rows), _ptr(cols), _ptr(vals),
                                         float(lam), int(k_max), ctypes.byref(rid)), s)
    return rid.value


def bm_server_drain(s, timeout_s=0.0):
    _check_server(lib().bm_server_drain(s, float(timeout_s)), s)


def bm_server_results(s):
    cnt = ctypes.c_int32()
    _check_server(lib().bm_server_results(s, None, 0, ctypes.byref(cnt)), s)
    arr = (bm_request_result * max(1, cnt.value))()
    _check_server(lib().bm_server_results(s, arr, cnt.value, ctypes.byref(cnt)), s)
    return [{n: getattr(arr[i], n) for n, _ in bm_request_result._fields_ if n != "pad_"} for i in range(cnt.value)]


def bm_server_factors(s, rid, m, n):
    """Factors (W m x k, H n x k, caller orientation) of finished request rid
    (server created with keep_factors=1); the server's copy is released."""
    k = ctypes.c_int32()
    _check_server(lib().bm_server_factors(s, int(rid), ctypes.byref(k), None, None), s)
    W = np.zeros((int(m), k.value), np.float32)
    H = np.zeros((int(n), k.value), np.float32)
    _check_server(lib().bm_server_factors(s, int(rid), ctypes.byref(k), _ptr(W), _ptr(H)), s)
    return W, H


def bm_server_now(s):
    return lib().bm_server_now(s)


def bm_server_destroy(s):
    lib().bm_server_destroy(s)
