"""ctypes binding of libcurid.so: argument marshalling only.

Every function here takes torch tensors that live on a CUDA device, passes
their device pointers and the current torch stream to the C ABI declared in
``include/curid.h``, and returns torch tensors the C library wrote.  No step
of the decomposition runs in Python.  The library allocates nothing itself:
the workspace is a torch uint8 tensor owned by the per-device handle here.
"""
import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libcurid.so")

OK, INVALID_ARG, RANK_DEFICIENT, BREAKDOWN, NONFINITE, TIMEOUT, CUDA_ERROR, NO_WORKSPACE, \
    UNSUPPORTED = range(9)
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "RANK_DEFICIENT", 3: "BREAKDOWN",
                4: "NONFINITE", 5: "TIMEOUT", 6: "CUDA_ERROR", 7: "NO_WORKSPACE",
                8: "UNSUPPORTED", 9: "TOL_NOT_MET"}
F64, F32, BF16 = 0, 1, 2


class CuridError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: curid status {STATUS_NAMES.get(status, status)}")


class Sketch(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("q", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("omega", ctypes.c_void_p), ("tf32", ctypes.c_int),
                ("srft_rows", ctypes.c_void_p), ("srft_signs", ctypes.c_void_p)]


class Srft:
    """The structured Omega of Eq. (5.2) given by its sampled rows (int32)
    and signs (int8), both on the device.  Passed as ``omega`` to the
    decompositions, it is applied by the fast transform (curid_srft_sketch)
    instead of being formed."""

    def __init__(self, rows, signs):
        if rows.dtype != torch.int32 or signs.dtype != torch.int8:
            raise ValueError("rows must be int32 and signs int8")
        self.rows, self.signs = rows.contiguous(), signs.contiguous()


class Sparse(ctypes.Structure):
    _fields_ = [("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("row_val", ctypes.c_void_p),
                ("col_ptr", ctypes.c_void_p), ("row_idx", ctypes.c_void_p),
                ("col_val", ctypes.c_void_p)]


_vp, _i64, _int, _dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
SIGNATURES = {
    "curid_create": [ctypes.POINTER(_vp), _int],
    "curid_destroy": [_vp],
    "curid_set_stream": [_vp, _vp],
    "curid_set_workspace": [_vp, _vp, ctypes.c_size_t],
    "curid_set_timeout": [_vp, ctypes.c_longlong],
    "curid_set_concurrency": [_vp, _int],
    "curid_workspace_size": [_vp, _int, _i64, _i64, _int, Sketch, ctypes.POINTER(ctypes.c_size_t)],
    "curid_last_status": [_vp, ctypes.POINTER(_int)],
    "curid_profile": [_vp, _int],
    "curid_profile_read": [_vp, ctypes.POINTER(_dbl), ctypes.POINTER(_int),
                           ctypes.POINTER(ctypes.c_longlong)],
    "curid_gaussian": [_vp, _int, _i64, _i64, ctypes.c_uint64, _vp],
    "curid_srft_omega": [_vp, _int, _i64, _i64, _vp, _vp, _vp, _i64],
    "curid_srft_draw": [_vp, _i64, _i64, ctypes.c_uint64, _vp, _vp],
    "curid_srft_sketch": [_vp, _int, _vp, _i64, _i64, _i64, _i64, _vp, _vp, _vp, _i64],
    "curid_sketch_matrix": [_vp, _int, _vp, _i64, _i64, _i64, _int, _int, _int, _vp, _vp],
    "curid_cpqr": [_vp, _int, _vp, _i64, _i64, _i64, _int, _dbl, _vp, _vp],
    "curid_cpqr_static": [_vp, _int, _vp, _i64, _i64, _i64, _int, _dbl, _vp, _vp, _vp],
    "curid_id_col": [_vp, _int, _vp, _i64, _i64, _i64, _int, _dbl, Sketch, _vp, _vp, _i64],
    "curid_id_row": [_vp, _int, _vp, _i64, _i64, _i64, _int, _dbl, Sketch, _vp, _vp, _i64],
    "curid_tsid": [_vp, _int, _vp, _i64, _i64, _i64, _int, _dbl, Sketch, _vp, _vp, _i64, _vp,
                   _vp, _i64],
    "curid_cur": [_vp, _int, _vp, _i64, _i64, _i64, _int, _dbl, Sketch, _vp, _vp, _vp, _vp, _vp,
                  _vp, _i64, _vp, _i64],
    "curid_interp_tikhonov_workspace_size": [_vp, _int, _i64, _int,
                                             ctypes.POINTER(ctypes.c_size_t)],
    "curid_interp_tikhonov": [_vp, _int, _vp, _i64, _vp, _i64, _int, _dbl, _vp, _i64],
    "curid_interp_tsvd_workspace_size": [_vp, _int, _i64, _int, ctypes.POINTER(ctypes.c_size_t)],
    "curid_interp_tsvd": [_vp, _int, _vp, _i64, _vp, _i64, _int, _dbl, _vp, _i64],
    "curid_sparse_workspace_size": [_vp, _int, _i64, _i64, _int, Sketch,
                                    ctypes.POINTER(ctypes.c_size_t)],
    "curid_cur_sparse": [_vp, _int, _i64, _i64, ctypes.POINTER(Sparse), _int, Sketch, _int, _vp,
                         _vp, _vp, _vp, _vp, _vp, _i64, _vp, _i64],
    "curid_complex_workspace_size": [_vp, _int, _i64, _i64, _int, Sketch,
                                     ctypes.POINTER(ctypes.c_size_t)],
    "curid_cur_complex": [_vp, _int, _vp, _i64, _i64, _i64, _int, Sketch, _vp, _vp, _vp, _vp,
                          _i64],
    "curid_cur_corrected": [_vp, _int, _vp, _i64, _i64, _i64, _int, _dbl, Sketch, _vp, _vp, _vp,
                            _vp, _vp, _vp, _i64, _vp, _i64],
    "curid_cur_adjoint_workspace_size": [_vp, _int, _i64, _i64, _int,
                                         ctypes.POINTER(ctypes.c_size_t)],
    "curid_id_col_batched_workspace_size": [_vp, _int, _int, _int, _int,
                                            ctypes.POINTER(ctypes.c_size_t)],
    "curid_id_col_batched": [_vp, _int, _int, _vp, _vp, _vp, _vp, _vp, _int, _int, _dbl, _int,
                             _vp, _vp, _vp, _vp],
    "curid_id_col_batched_autotune": [_vp, _int, _int, _vp, _vp, _vp, _vp, _vp, _int, _int, _dbl,
                                      _int, _vp, _vp, _vp, _vp, ctypes.POINTER(_int),
                                      ctypes.POINTER(_int)],
    "curid_cur_adjoint": [_vp, _int, _vp, _i64, _i64, _i64, _int, _vp, _vp, _vp, _i64, _vp, _vp,
                          _vp, _vp, _i64],
}

_lib = None
_lock = threading.Lock()


def load_library():
    """Load libcurid.so (raises if it has not been built: there is no
    fallback implementation)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing; build it with "
                                  "`python -m paper_1412_8447_gb300.build`")
            lib = ctypes.CDLL(LIB_PATH)
            for name, args in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dtype_code(t):
    if t == torch.float64:
        return F64
    if t == torch.float32:
        return F32
    if t == torch.bfloat16:
        return BF16
    raise TypeError(f"unsupported dtype {t}; use float32, float64 or bfloat16")


def _work_dtype(t):
    """dtype of T and TW: float32 for bfloat16 storage, else that of A."""
    return torch.float32 if t == torch.bfloat16 else t


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _check(st, where):
    if st != OK:
        raise CuridError(st, where)


class _Handle:
    """A library handle on one CUDA device, with a growable workspace; each
    call binds torch's current stream."""

    def __init__(self, device):
        self.lib = load_library()
        self.device = device
        h = ctypes.c_void_p()
        _check(self.lib.curid_create(ctypes.byref(h), device), "curid_create")
        self.h = h
        self.ws = None

    def prepare(self, nbytes):
        if self.ws is None or self.ws.numel() < nbytes:
            self.ws = torch.empty(max(nbytes, 1 << 20), dtype=torch.uint8,
                                  device=f"cuda:{self.device}")
            _check(self.lib.curid_set_workspace(self.h, _ptr(self.ws), self.ws.numel()),
                   "curid_set_workspace")
        stream = torch.cuda.current_stream(self.device).cuda_stream
        _check(self.lib.curid_set_stream(self.h, ctypes.c_void_p(stream)), "curid_set_stream")

    def status(self):
        k = ctypes.c_int(0)
        st = self.lib.curid_last_status(self.h, ctypes.byref(k))
        return st, k.value


_handles = {}
_slot = threading.local()


class inflight:
    """Context in which library calls use handle ``slot`` of their device
    (its own workspace and status): decompositions queued on different
    streams under different slots can run on the GPU at the same time.
    Outside any context, slot 0."""

    def __init__(self, slot):
        self.slot = int(slot)

    def __enter__(self):
        self.prev = getattr(_slot, "v", 0)
        _slot.v = self.slot
        return self

    def __exit__(self, *exc):
        _slot.v = self.prev
        return False


def handle(device):
    key = (device, getattr(_slot, "v", 0))
    if key not in _handles:
        _handles[key] = _Handle(device)
    return _handles[key]


def _dev(t):
    if not t.is_cuda:
        raise ValueError("tensors must be on a CUDA device")
    return t.device.index if t.device.index is not None else torch.cuda.current_device()


def _mat(A):
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("expected a 2-D row-major tensor (stride(1) == 1)")
    return A


def _sketch(p, q, seed, omega, tf32):
    if isinstance(omega, Srft):
        return Sketch(int(p), int(q), int(seed) & ((1 << 64) - 1), None, 1 if tf32 else 0,
                      ctypes.c_void_p(omega.rows.data_ptr()),
                      ctypes.c_void_p(omega.signs.data_ptr()))
    return Sketch(int(p), int(q), int(seed) & ((1 << 64) - 1),
                  ctypes.c_void_p(omega.data_ptr()) if omega is not None else None,
                  1 if tf32 else 0, None, None)


def workspace_bytes(h, dt, m, n, k, sk):
    b = ctypes.c_size_t(0)
    _check(h.lib.curid_workspace_size(h.h, dt, m, n, k, sk, ctypes.byref(b)),
           "curid_workspace_size")
    return b.value


class Result:
    """Outputs of one call; ``status`` is the device status (0 = OK,
    2 = RANK_DEFICIENT) and ``k`` the rank produced, both filled when the
    call ran with ``check=True``."""

    def __init__(self, **kw):
        self.status = None
        self.k = None
        self.__dict__.update(kw)

    def __repr__(self):
        keys = ", ".join(k for k in self.__dict__)
        return f"Result({keys})"


def _finish(h, res, check, where):
    if check:
        st, k = h.status()
        if st not in (OK, RANK_DEFICIENT):
            raise CuridError(st, where)
        res.status, res.k = st, k
    return res


PHASES = ["omega", "sketch", "orth", "cpqr_col", "t_solve", "gather", "cpqr_row", "u_solve"]


def profile(enable=True, device=0):
    """Turn per-phase CUDA-event timing and launch counting on or off."""
    h = handle(device)
    _check(h.lib.curid_profile(h.h, 1 if enable else 0), "curid_profile")


def profile_read(device=0):
    """({phase: ms}, {phase: intervals}, launches) since the last read."""
    h = handle(device)
    n = len(PHASES)
    ms = (ctypes.c_double * n)()
    calls = (ctypes.c_int * n)()
    launches = ctypes.c_longlong(0)
    _check(h.lib.curid_profile_read(h.h, ms, calls, ctypes.byref(launches)), "curid_profile_read")
    return ({p: ms[i] for i, p in enumerate(PHASES)},
            {p: calls[i] for i, p in enumerate(PHASES)}, launches.value)


def status_block(device=0):
    """The raw device status block of the last call (synchronises): flags,
    k_done, k_eff, k_row, timeout site."""
    h = handle(device)
    torch.cuda.synchronize(device)
    return h.ws[:20].view(torch.int32).cpu().tolist() if h.ws is not None else None


def set_concurrency(inflight, device=0):
    """Tell the library how many decompositions are kept in flight on
    ``device`` (applies to the current ``inflight`` slot's handle)."""
    h = handle(device)
    _check(h.lib.curid_set_concurrency(h.h, int(inflight)), "curid_set_concurrency")


def set_timeout(cycles, device=0):
    """Bound of the waits between blocks of the persistent kernels, in SM
    clock cycles (0: the default, about 2 s)."""
    h = handle(device)
    _check(h.lib.curid_set_timeout(h.h, int(cycles)), "curid_set_timeout")


def last_status(device=0):
    """(status, k) recorded by the last call on ``device`` (synchronises)."""
    return handle(device).status()


def gaussian(rows, cols, seed, dtype=torch.float32, device=None):
    """N(0, 1) rows x cols matrix from the library's Philox4x32-10 generator."""
    device = torch.cuda.current_device() if device is None else device
    h = handle(device)
    h.prepare(0)
    out = torch.empty((rows, cols), dtype=dtype, device=f"cuda:{device}")
    _check(h.lib.curid_gaussian(h.h, _dtype_code(dtype), rows, cols, int(seed) & ((1 << 64) - 1),
                                _ptr(out)), "curid_gaussian")
    return out


def srft_draw(m, l, seed, device=None):
    """Random signs (int8, [m]) and l distinct rows (int32, [l]) of the
    structured sampling matrix of Section 5.2, drawn on the device from
    ``seed`` (curid_srft_draw)."""
    dev = device if device is not None else torch.cuda.current_device()
    h = handle(dev)
    h.prepare(0)
    rows = torch.empty(l, dtype=torch.int32, device=f"cuda:{dev}")
    signs = torch.empty(m, dtype=torch.int8, device=f"cuda:{dev}")
    _check(h.lib.curid_srft_draw(h.h, int(m), int(l), int(seed) & ((1 << 64) - 1), _ptr(rows),
                                 _ptr(signs)), "curid_srft_draw")
    return rows, signs


def srft_omega(rows, signs, dtype=torch.float32):
    """Omega = sqrt(m/l) R F D of Eq. (5.2) (real form: DCT-II and random
    signs), l x m, from device ``rows`` (int32) and ``signs`` (int8)
    (curid_srft_omega).  Pass it as ``omega`` with p = l - k and q = 0 for
    the accelerated scheme."""
    if rows.dtype != torch.int32 or signs.dtype != torch.int8:
        raise ValueError("rows must be int32 and signs int8")
    rows, signs = rows.contiguous(), signs.contiguous()
    dev = _dev(rows)
    h = handle(dev)
    h.prepare(0)
    l, m = rows.numel(), signs.numel()
    out = torch.empty((l, m), dtype=dtype, device=rows.device)
    _check(h.lib.curid_srft_omega(h.h, _dtype_code(out.dtype), m, l, _ptr(rows), _ptr(signs),
                                  _ptr(out), m), "curid_srft_omega")
    return out


def srft_sketch(A, rows, signs):
    """Y = Omega A (l x n) for the structured Omega of Eq. (5.2) given by
    ``rows`` and ``signs``, by the fast transform, without forming Omega
    (curid_srft_sketch).  A float32 or float64, row-major, on the device."""
    A = _mat(A)
    if rows.dtype != torch.int32 or signs.dtype != torch.int8:
        raise ValueError("rows must be int32 and signs int8")
    rows, signs = rows.contiguous(), signs.contiguous()
    m, n = A.shape
    if signs.numel() != m:
        raise ValueError("signs must have one entry per row of A")
    dev = _dev(A)
    h = handle(dev)
    h.prepare(0)
    l = rows.numel()
    Y = torch.empty((l, n), dtype=A.dtype, device=A.device)
    _check(h.lib.curid_srft_sketch(h.h, _dtype_code(A.dtype), _ptr(A), m, n, A.stride(0), l,
                                   _ptr(rows), _ptr(signs), _ptr(Y), n), "curid_srft_sketch")
    return Y


def sketch_matrix(A, omega, q=0, tf32=False):
    """Y = Omega A (A^T A)^q with row orthonormalisation between products."""
    A = _mat(A)
    dev = _dev(A)
    h = handle(dev)
    m, n = A.shape
    l = omega.shape[0]
    dt = _dtype_code(A.dtype)
    h.prepare(workspace_bytes(h, dt, m, n, 1, _sketch(max(0, l - 1), q, 0, omega, tf32)))
    Y = torch.empty((l, n), dtype=_work_dtype(A.dtype), device=A.device)
    _check(h.lib.curid_sketch_matrix(h.h, dt, _ptr(A), m, n, A.stride(0), l, q,
                                     1 if tf32 else 0, _ptr(omega.contiguous()), _ptr(Y)),
           "curid_sketch_matrix")
    return Y


def cpqr(Y, k=0, tol=0.0, check=True):
    """Truncated column-pivoted QR of Y: J (int32, n) and S (k_max x n,
    original column order)."""
    Y = _mat(Y)
    dev = _dev(Y)
    h = handle(dev)
    l, n = Y.shape
    k_max = k if k > 0 else min(l, n)
    dt = _dtype_code(Y.dtype)
    # the workspace of a rank-1 deterministic decomposition of an l x n
    # matrix contains the CPQR scratch for l x n
    h.prepare(workspace_bytes(h, dt, max(l, 1), n, 1, _sketch(-1, 0, 0, None, 0)))
    J = torch.empty(n, dtype=torch.int32, device=Y.device)
    S = torch.zeros((k_max, n), dtype=Y.dtype, device=Y.device)
    _check(h.lib.curid_cpqr(h.h, dt, _ptr(Y), l, n, Y.stride(0), k, float(tol), _ptr(J), _ptr(S)),
           "curid_cpqr")
    return _finish(h, Result(J=J, S=S), check, "curid_cpqr")


def _interp(kind, S, J, k, param):
    S = _mat(S)
    dev = _dev(S)
    h = handle(dev)
    kk, n = S.shape
    if kk < k:
        raise ValueError("S has fewer than k rows")
    b = ctypes.c_size_t(0)
    ws = getattr(h.lib, f"curid_interp_{kind}_workspace_size")
    _check(ws(h.h, _dtype_code(S.dtype), n, k, ctypes.byref(b)),
           f"curid_interp_{kind}_workspace_size")
    h.prepare(b.value)
    T = torch.empty((k, max(n - k, 1)), dtype=S.dtype, device=S.device)
    fn = getattr(h.lib, f"curid_interp_{kind}")
    _check(fn(h.h, _dtype_code(S.dtype), _ptr(S), S.stride(0), _ptr(J.contiguous()), n, k,
              float(param), _ptr(T), T.stride(0)), f"curid_interp_{kind}")
    return T[:, :n - k]


def interp_tsvd(S, J, k, rtol):
    """Truncated-SVD T = V diag(1/sigma, sigma > rtol sigma_1) U^T S12
    (Section 4.1) from the S and J that ``cpqr`` returns."""
    return _interp("tsvd", S, J, k, rtol)


def interp_tikhonov(S, J, k, lam):
    """Regularised T = argmin ||S11 T - S12||^2 + lam^2 ||T||^2 (Section 4.1
    with a Tikhonov term) from the S (k x n, original column order) and J
    that ``cpqr`` returns; T is k x (n - k), columns following J[k:]."""
    return _interp("tikhonov", S, J, k, lam)


def _prep(A, k, p, q, seed, omega, tf32):
    A = _mat(A)
    dev = _dev(A)
    h = handle(dev)
    m, n = A.shape
    dt = _dtype_code(A.dtype)
    sk = _sketch(p, q, seed, omega, tf32)
    h.prepare(workspace_bytes(h, dt, m, n, k, sk))
    return A, h, m, n, dt, sk


def _steps_done(h):
    """CPQR steps of the last call (status block word 1): the rank an adaptive
    call ran its decomposition at (its outputs' shapes)."""
    torch.cuda.synchronize(h.device)
    return int(h.ws[4:8].view(torch.int32).item())


def _adaptive(k, tol, p):
    if k == 0:
        if not tol > 0:
            raise ValueError("k == 0 needs tol > 0 (adaptive rank)")
        return True
    return False


def id_col(A, k, p=-1, q=0, seed=0, omega=None, tf32=False, tol=0.0, check=True):
    """Column ID A ~ A(:, J[:k]) [I T] P^T (Algorithm 1; p >= 0: Algorithm 4).
    k == 0 with tol > 0: adaptive rank (deterministic method)."""
    adaptive = _adaptive(k, tol, p)
    A, h, m, n, dt, sk = _prep(A, k, p, q, seed, omega, tf32)
    kb = min(m, n) if adaptive else k
    J = torch.empty(n, dtype=torch.int32, device=A.device)
    T = torch.empty((kb, n if adaptive else max(n - k, 1)), dtype=_work_dtype(A.dtype),
                    device=A.device)
    _check(h.lib.curid_id_col(h.h, dt, _ptr(A), m, n, A.stride(0), k, float(tol), sk, _ptr(J),
                              _ptr(T), T.stride(0)), "curid_id_col")
    res = _finish(h, Result(J=J, T=T), check or adaptive, "curid_id_col")
    kk = _steps_done(h) if adaptive else k
    res.T = T[:kk, :n - kk]
    return res


def id_row(A, k, p=-1, q=0, seed=0, omega=None, tf32=False, check=True):
    """Row ID A ~ W A(I[:k], :) (the column ID of A^T)."""
    A, h, m, n, dt, sk = _prep(A, k, p, q, seed, omega, tf32)
    I = torch.empty(m, dtype=torch.int32, device=A.device)
    TW = torch.empty((k, max(m - k, 1)), dtype=A.dtype, device=A.device)
    _check(h.lib.curid_id_row(h.h, dt, _ptr(A), m, n, A.stride(0), k, 0.0, sk, _ptr(I),
                              _ptr(TW), TW.stride(0)), "curid_id_row")
    return _finish(h, Result(I=I, TW=TW[:, :m - k]), check, "curid_id_row")


def tsid(A, k, p=-1, q=0, seed=0, omega=None, tf32=False, tol=0.0, check=True):
    """Two-sided ID A ~ W A(I[:k], J[:k]) V* (Algorithm 2); k == 0 with
    tol > 0: adaptive rank (deterministic method)."""
    adaptive = _adaptive(k, tol, p)
    A, h, m, n, dt, sk = _prep(A, k, p, q, seed, omega, tf32)
    kb = min(m, n) if adaptive else k
    J = torch.empty(n, dtype=torch.int32, device=A.device)
    I = torch.empty(m, dtype=torch.int32, device=A.device)
    T = torch.empty((kb, n if adaptive else max(n - k, 1)), dtype=_work_dtype(A.dtype),
                    device=A.device)
    TW = torch.empty((kb, m if adaptive else max(m - k, 1)), dtype=_work_dtype(A.dtype),
                     device=A.device)
    _check(h.lib.curid_tsid(h.h, dt, _ptr(A), m, n, A.stride(0), k, float(tol), sk, _ptr(J),
                            _ptr(T), T.stride(0), _ptr(I), _ptr(TW), TW.stride(0)), "curid_tsid")
    res = _finish(h, Result(J=J, T=T, I=I, TW=TW), check or adaptive, "curid_tsid")
    kk = _steps_done(h) if adaptive else k
    res.T, res.TW = T[:kk, :n - kk], TW[:kk, :m - kk]
    return res


def cur_outputs(A, k, want_c=False, want_r=False, want_t=False, want_tw=False):
    """Preallocated output tensors for ``cur(..., out=...)``."""
    m, n = A.shape
    dev = A.device
    return Result(
        J=torch.empty(n, dtype=torch.int32, device=dev),
        I=torch.empty(m, dtype=torch.int32, device=dev),
        U=torch.empty((k, k), dtype=torch.float64, device=dev),
        C=torch.empty((m, k), dtype=A.dtype, device=dev) if want_c else None,
        R=torch.empty((k, n), dtype=A.dtype, device=dev) if want_r else None,
        T=torch.empty((k, max(n - k, 1)), dtype=_work_dtype(A.dtype), device=dev)
        if want_t else None,
        TW=torch.empty((k, max(m - k, 1)), dtype=_work_dtype(A.dtype), device=dev)
        if want_tw else None)


def cur(A, k, p=-1, q=0, seed=0, omega=None, tf32=False, want_c=False, want_r=False,
        want_t=False, want_tw=False, out=None, check=True, tol=0.0, corrected=False):
    """CUR-ID A ~ C U R (Algorithm 3); U is float64 (k x k).  k == 0 with
    tol > 0: adaptive rank (deterministic method); outputs are views at the
    rank reached (res.k).  corrected=True: U from the error-corrected system
    of Eq. (4.3), U = C^+ A R^+ (curid_cur_corrected)."""
    adaptive = _adaptive(k, tol, p)
    A, h, m, n, dt, sk = _prep(A, k, p, q, seed, omega, tf32)
    kb = min(m, n) if adaptive else k
    if adaptive:
        dev = A.device
        o = Result(
            J=torch.empty(n, dtype=torch.int32, device=dev),
            I=torch.empty(m, dtype=torch.int32, device=dev),
            U=torch.empty(kb * kb, dtype=torch.float64, device=dev),
            C=torch.empty(m * kb, dtype=A.dtype, device=dev) if want_c else None,
            R=torch.empty((kb, n), dtype=A.dtype, device=dev) if want_r else None,
            T=torch.empty((kb, n), dtype=_work_dtype(A.dtype), device=dev) if want_t else None,
            TW=torch.empty((kb, m), dtype=_work_dtype(A.dtype), device=dev)
            if want_tw else None)
    else:
        o = out if out is not None else cur_outputs(A, k, want_c, want_r, want_t, want_tw)
    fn = h.lib.curid_cur_corrected if corrected else h.lib.curid_cur
    st = fn(h.h, dt, _ptr(A), m, n, A.stride(0), k, float(tol), sk, _ptr(o.J),
            _ptr(o.I), _ptr(o.U), _ptr(o.C), _ptr(o.R), _ptr(o.T),
            o.T.stride(0) if o.T is not None else 0, _ptr(o.TW),
            o.TW.stride(0) if o.TW is not None else 0)
    _check(st, "curid_cur")
    res = _finish(h, o, check or adaptive, "curid_cur")
    if adaptive:
        kk = _steps_done(h)
        res.U = o.U[:kk * kk].view(kk, kk)
        if want_c:
            res.C = o.C[:m * kk].view(m, kk)
        if want_r:
            res.R = o.R[:kk]
        if want_t:
            res.T = o.T[:kk, :n - kk]
        if want_tw:
            res.TW = o.TW[:kk, :m - kk]
    return res

def cur_complex(A, k, p=-1, q=0, seed=0, tf32=False, want_t=False, check=True):
    """CUR-ID of a complex A (torch complex64 / complex128, row-major, on a
    CUDA device) through curid_cur_complex: J, I (int32), U (complex128
    k x k), T (complex, k x (n - k), when want_t)."""
    if A.dtype not in (torch.complex64, torch.complex128):
        raise ValueError("expected a complex64 or complex128 tensor")
    A = _mat(A)
    dev = _dev(A)
    h = handle(dev)
    m, n = A.shape
    dt = F32 if A.dtype == torch.complex64 else F64
    sk = _sketch(p, q, seed, None, tf32)
    b = ctypes.c_size_t(0)
    _check(h.lib.curid_complex_workspace_size(h.h, dt, m, n, k, sk, ctypes.byref(b)),
           "curid_complex_workspace_size")
    h.prepare(b.value)
    o = Result(J=torch.empty(n, dtype=torch.int32, device=A.device),
               I=torch.empty(m, dtype=torch.int32, device=A.device),
               U=torch.empty((k, k), dtype=torch.complex128, device=A.device),
               T=torch.empty((k, max(n - k, 1)), dtype=A.dtype, device=A.device)
               if want_t else None)
    _check(h.lib.curid_cur_complex(h.h, dt, _ptr(A), m, n, A.stride(0), k, sk, _ptr(o.J),
                                   _ptr(o.I), _ptr(o.U), _ptr(o.T),
                                   o.T.stride(0) if o.T is not None else 0),
           "curid_cur_complex")
    res = _finish(h, o, check, "curid_cur_complex")
    if want_t:
        res.T = o.T[:, :n - k]
    return res


def sparse_operand(A):
    """The two compressed forms curid_cur_sparse reads, from a torch sparse
    CSR tensor on a CUDA device: its rows, and its columns from torch's
    CSR -> CSC conversion (indices as int32, pointers as int64).  Returns
    (tensors to keep alive, the ctypes struct)."""
    if A.layout != torch.sparse_csr or not A.is_cuda:
        raise ValueError("expected a torch sparse CSR tensor on a CUDA device")
    crow = A.crow_indices().to(torch.int64).contiguous()
    col = A.col_indices().to(torch.int32).contiguous()
    val = A.values().contiguous()
    Ac = A.to_sparse_csc()
    ccol = Ac.ccol_indices().to(torch.int64).contiguous()
    row = Ac.row_indices().to(torch.int32).contiguous()
    cval = Ac.values().contiguous()
    keep = (crow, col, val, ccol, row, cval)
    st = Sparse(int(val.numel()), _ptr(crow), _ptr(col), _ptr(val), _ptr(ccol), _ptr(row),
                _ptr(cval))
    return keep, st


def cur_sparse(A, k, p, q=0, seed=0, omega=None, corrected=False, want_c=False, want_r=False,
               want_t=False, want_tw=False, out=None, check=True):
    """Randomized CUR-ID of a sparse A (torch sparse CSR tensor, float32 or
    float64, on a CUDA device) through curid_cur_sparse; outputs as ``cur``
    (C and R dense)."""
    keep, st = sparse_operand(A)
    m, n = A.shape
    dev = A.device.index if A.device.index is not None else torch.cuda.current_device()
    h = handle(dev)
    dt = _dtype_code(A.dtype)
    sk = _sketch(p, q, seed, omega, False)
    b = ctypes.c_size_t(0)
    _check(h.lib.curid_sparse_workspace_size(h.h, dt, m, n, k, sk, ctypes.byref(b)),
           "curid_sparse_workspace_size")
    h.prepare(b.value)
    if out is None:
        out = Result(
            J=torch.empty(n, dtype=torch.int32, device=A.device),
            I=torch.empty(m, dtype=torch.int32, device=A.device),
            U=torch.empty((k, k), dtype=torch.float64, device=A.device),
            C=torch.empty((m, k), dtype=A.dtype, device=A.device) if want_c else None,
            R=torch.empty((k, n), dtype=A.dtype, device=A.device) if want_r else None,
            T=torch.empty((k, max(n - k, 1)), dtype=A.dtype, device=A.device) if want_t else None,
            TW=torch.empty((k, max(m - k, 1)), dtype=A.dtype, device=A.device)
            if want_tw else None)
    o = out
    _check(h.lib.curid_cur_sparse(h.h, dt, m, n, ctypes.byref(st), k, sk, 1 if corrected else 0,
                                  _ptr(o.J), _ptr(o.I), _ptr(o.U), _ptr(o.C), _ptr(o.R),
                                  _ptr(o.T), o.T.stride(0) if o.T is not None else 0,
                                  _ptr(o.TW), o.TW.stride(0) if o.TW is not None else 0),
           "curid_cur_sparse")
    res = _finish(h, o, check, "curid_cur_sparse")
    res._keep = keep  # the compressed forms stay alive until the work is done
    return res


def cur_adjoint(A, J, I, T, k, Cbar=None, Ubar=None, Rbar=None, out=None, check=True):
    """Gradient with respect to A of <Cbar, C> + <Ubar, U> + <Rbar, R> for the
    deterministic CUR-ID with the skeletons J, I frozen (T from the same
    decomposition).  Cotangents may be None (zero); Ubar is float64 like U."""
    A = _mat(A)
    dev = _dev(A)
    h = handle(dev)
    m, n = A.shape
    dt = _dtype_code(A.dtype)
    b = ctypes.c_size_t(0)
    _check(h.lib.curid_cur_adjoint_workspace_size(h.h, dt, m, n, k, ctypes.byref(b)),
           "curid_cur_adjoint_workspace_size")
    h.prepare(b.value)
    Cb = Cbar.to(A.dtype).contiguous() if Cbar is not None else None
    Ub = Ubar.to(torch.float64).contiguous() if Ubar is not None else None
    Rb = Rbar.to(A.dtype).contiguous() if Rbar is not None else None
    Tc = T if (T is None or T.stride(-1) == 1) else T.contiguous()
    Ab = out if out is not None else torch.empty((m, n), dtype=A.dtype, device=A.device)
    st = h.lib.curid_cur_adjoint(h.h, dt, _ptr(A), m, n, A.stride(0), k, _ptr(J), _ptr(I),
                                 _ptr(Tc if n > k else None),
                                 Tc.stride(0) if (Tc is not None and n > k) else 1,
                                 _ptr(Cb), _ptr(Ub), _ptr(Rb), _ptr(Ab), Ab.stride(0))
    _check(st, "curid_cur_adjoint")
    if check:
        st, _ = h.status()
        if st != OK:
            raise CuridError(st, "curid_cur_adjoint")
    return Ab


class CURFunction(torch.autograd.Function):
    """(C, U, R) of the deterministic CUR-ID (Algorithm 3) as a function of A,
    differentiable with the skeletons frozen at the forward pass's J and I;
    the backward pass is the library's adjoint (curid_cur_adjoint)."""

    @staticmethod
    def forward(ctx, A, k):
        r = cur(A, k, want_c=True, want_r=True, want_t=True)
        ctx.k = k
        ctx.save_for_backward(A, r.J, r.I, r.T)
        ctx.mark_non_differentiable(r.J, r.I)
        return r.C, r.U, r.R, r.J, r.I

    @staticmethod
    def backward(ctx, Cbar, Ubar, Rbar, _J, _I):
        A, J, I, T = ctx.saved_tensors
        k = ctx.k
        Ab = cur_adjoint(A, J, I, T[:, :A.shape[1] - k], k, Cbar, Ubar, Rbar)
        return Ab, None


def cur_differentiable(A, k):
    """C, U, R, J, I with C, U, R differentiable in A (skeletons frozen)."""
    return CURFunction.apply(A, k)


class BatchedID:
    """Column IDs of many independent blocks in one persistent launch
    (curid_id_col_batched).  ``flat`` holds the row-major blocks back to back
    (block b of shape ``shapes[b]`` starting at element ``offsets[b]``);
    outputs live in flat device buffers allocated here.  ``run()`` only
    enqueues work (two memsets and one kernel) on the current stream, so it
    can be captured into a CUDA graph."""

    def __init__(self, flat, shapes, offsets, tol, k_max=64, largest_first=True):
        self.flat = flat
        dev = _dev(flat)
        self.h = handle(dev)
        self.dtype = flat.dtype
        self.dt = _dtype_code(flat.dtype)
        self.nb = len(shapes)
        self.shapes = list(shapes)
        self.tol = float(tol)
        self.k_max = int(k_max)
        d = flat.device
        esz = flat.element_size()
        m = [s[0] for s in shapes]
        n = [s[1] for s in shapes]
        self.max_m, self.max_n = max(m), max(n)
        base = flat.data_ptr()
        self.A_ptr = torch.tensor([base + esz * o for o in offsets], dtype=torch.int64, device=d)
        self.lda = torch.tensor(n, dtype=torch.int64, device=d)
        self.m = torch.tensor(m, dtype=torch.int32, device=d)
        self.n = torch.tensor(n, dtype=torch.int32, device=d)
        self.joff, self.toff = [], []
        jt = tt = 0
        for mb, nb_ in shapes:
            self.joff.append(jt)
            self.toff.append(tt)
            jt += nb_
            tt += self.k_max * nb_
        self.Jflat = torch.zeros(max(jt, 1), dtype=torch.int32, device=d)
        self.Tflat = torch.zeros(max(tt, 1), dtype=flat.dtype, device=d)
        self.J_ptr = torch.tensor([self.Jflat.data_ptr() + 4 * o for o in self.joff],
                                  dtype=torch.int64, device=d)
        self.T_ptr = torch.tensor([self.Tflat.data_ptr() + esz * o for o in self.toff],
                                  dtype=torch.int64, device=d)
        self.k_out = torch.zeros(self.nb, dtype=torch.int32, device=d)
        self.block_status = torch.zeros(self.nb, dtype=torch.int32, device=d)
        order = sorted(range(self.nb), key=lambda b: -m[b] * n[b]) if largest_first else None
        self.order = torch.tensor(order, dtype=torch.int32, device=d) if order else None
        b = ctypes.c_size_t(0)
        _check(self.h.lib.curid_id_col_batched_workspace_size(
            self.h.h, self.dt, self.max_m, self.max_n, self.k_max, ctypes.byref(b)),
            "curid_id_col_batched_workspace_size")
        self.ws_bytes = b.value

    def _args(self):
        return (self.h.h, self.dt, self.nb, _ptr(self.A_ptr), _ptr(self.lda), _ptr(self.m),
                _ptr(self.n), _ptr(self.order), self.max_m, self.max_n, self.tol, self.k_max,
                _ptr(self.J_ptr), _ptr(self.T_ptr), _ptr(self.k_out), _ptr(self.block_status))

    def prepare(self):
        """Attach a large enough workspace and bind the current stream (call
        before capturing ``run`` into a graph)."""
        self.h.prepare(self.ws_bytes)

    def run(self):
        self.prepare()
        _check(self.h.lib.curid_id_col_batched(*self._args()), "curid_id_col_batched")

    def autotune(self):
        """Time every feasible launch shape on this batch and keep the fastest
        on the handle; returns (threads per CTA, CTAs per SM)."""
        self.prepare()
        t, c = ctypes.c_int(0), ctypes.c_int(0)
        _check(self.h.lib.curid_id_col_batched_autotune(*self._args(), ctypes.byref(t),
                                                        ctypes.byref(c)),
               "curid_id_col_batched_autotune")
        return t.value, c.value

    def results(self):
        """[(J_b, T_b, k_b, status_b)]: J_b int32 (n_b), T_b k_b x (n_b - k_b)."""
        k = self.k_out.cpu().tolist()
        st = self.block_status.cpu().tolist()
        out = []
        for b, (mb, nb_) in enumerate(self.shapes):
            J = self.Jflat[self.joff[b]:self.joff[b] + nb_]
            T = self.Tflat[self.toff[b]:self.toff[b] + self.k_max * nb_].view(self.k_max, nb_)
            out.append((J, T[:k[b], :nb_ - k[b]], k[b], st[b]))
        return out


class HostStream:
    """CUR-IDs of a sequence of host matrices, each copied to the device and
    its skeletons and U copied back, with the host-to-device copies
    overlapped with the decompositions.

    ``inflight`` decompositions run at once, each on its own stream and
    library handle (``inflight`` slots); inflight + 1 device buffers for A
    rotate, so the copy of the next matrix runs while ``inflight``
    decompositions use the others.  The copies of A run on three side
    streams (consecutive matrices in turn),
    each waiting until the decomposition that last read its buffer has
    finished; the copies of (J, I, U) back to the host run on the stream of
    their decomposition.  Host matrices should be pinned
    (``tensor.pin_memory()``) so the copies are asynchronous.  Only stream
    and event bookkeeping happens here: every step of each decomposition is
    the same library call ``cur`` makes.
    """

    def __init__(self, m, n, k, dtype=torch.float32, device=None, p=-1, q=0, tf32=False,
                 inflight=1):
        dev = torch.device("cuda", device if device is not None else torch.cuda.current_device())
        self.device, self.k, self.p, self.q, self.tf32 = dev, int(k), int(p), int(q), bool(tf32)
        self.inflight = max(1, int(inflight))
        nbuf = self.inflight + 1
        self.A = [torch.empty((m, n), dtype=dtype, device=dev) for _ in range(nbuf)]
        self.out = [cur_outputs(self.A[0], k) for _ in range(self.inflight)]
        # three copy streams, consecutive matrices in turn: a copy can start
        # as soon as its buffer is free (host-to-device bandwidth, about 210
        # GB/s on GB300 from pinned memory, is the same with one stream)
        self.copy_streams = [torch.cuda.Stream(dev) for _ in range(3)]
        self.streams = [None] + [torch.cuda.Stream(dev) for _ in range(self.inflight - 1)]
        self.ready = [torch.cuda.Event() for _ in range(nbuf)]
        self.free = [torch.cuda.Event() for _ in range(nbuf)]

    def host_results(self, count):
        """Pinned host buffers (J, I, U) for ``count`` decompositions."""
        m, n = self.A[0].shape
        k = self.k
        return [(torch.empty(n, dtype=torch.int32).pin_memory(),
                 torch.empty(m, dtype=torch.int32).pin_memory(),
                 torch.empty((k, k), dtype=torch.float64).pin_memory()) for _ in range(count)]

    def run(self, A_hosts, results, seeds=None):
        """Decompose every matrix of ``A_hosts`` (host tensors of the stream's
        shape and dtype) into ``results[i] = (J, I, U)`` host tensors.  Work is
        queued behind the current stream and returns before it finishes;
        synchronize before reading ``results``.  Device status is not checked
        (read it with ``last_status`` inside ``inflight(slot)``)."""
        cur_s = torch.cuda.current_stream(self.device)
        streams = [cur_s] + self.streams[1:]
        count = len(A_hosts)
        nbuf = len(self.A)
        if len(results) < count:
            raise ValueError("one (J, I, U) result triple per matrix is needed")
        # no copy or decomposition may start before work already queued on
        # the current stream
        for cs in self.copy_streams:
            cs.wait_stream(cur_s)
        for st in streams[1:]:
            st.wait_stream(cur_s)
        first = [True] * nbuf

        def copy_in(i):
            b = i % nbuf
            cs = self.copy_streams[i % len(self.copy_streams)]
            with torch.cuda.stream(cs):
                if not first[b]:
                    cs.wait_event(self.free[b])
                first[b] = False
                self.A[b].copy_(A_hosts[i], non_blocking=True)
                self.ready[b].record(cs)

        for slot in range(self.inflight):
            with torch.cuda.stream(streams[slot]), inflight(slot):
                set_concurrency(self.inflight, self.device.index)
        for i in range(min(count, self.inflight)):
            copy_in(i)
        for i in range(count):
            b, slot = i % nbuf, i % self.inflight
            if i + self.inflight < count:
                copy_in(i + self.inflight)
            st = streams[slot]
            st.wait_event(self.ready[b])
            seed = seeds[i] if seeds is not None else i
            with torch.cuda.stream(st), inflight(slot):
                cur(self.A[b], self.k, p=self.p, q=self.q, seed=seed, tf32=self.tf32,
                    out=self.out[slot], check=False)
                self.free[b].record(st)
                J, I, U = results[i]
                J.copy_(self.out[slot].J, non_blocking=True)
                I.copy_(self.out[slot].I, non_blocking=True)
                U.copy_(self.out[slot].U, non_blocking=True)
        # the A buffers must not be reused by a later run before these copies,
        # and the current stream ends after every decomposition
        for cs in self.copy_streams:
            cur_s.wait_stream(cs)
        for st in streams[1:]:
            cur_s.wait_stream(st)
