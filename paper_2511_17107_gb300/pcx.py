"""ctypes binding of libpcx (include/pcx.h).  Argument marshalling only:
every step of the computation runs inside the CUDA library.  The library
must have been built (``paper_2511_17107_gb300.build.build()``); without it
every call raises.

Functions keep the C names (``pcx_setup``, ``pcx_apply``, ...).  Device
buffers are torch tensors (complex64 for PCX_FP32, complex128 for PCX_FP64),
contiguous, shaped (nvec, 3, N, N, N); streams default to torch's current
stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PCX_OK, PCX_EINVAL, PCX_ENOMEM, PCX_ENOTHPD, PCX_ENOCONV, PCX_ENUMERIC, PCX_ECUDA = 0, -1, -2, -3, -4, -5, -6
PCX_FP64, PCX_FP32 = 0, 1
PCX_CT_SUMMED, PCX_CT_LITERAL = 0, 1
PCX_APPLY_AUTO, PCX_APPLY_FIVE_PASS, PCX_APPLY_THREE_PASS = 0, 1, 2
PCX_PENALTY_SCALAR, PCX_PENALTY_PER_MODE, PCX_PENALTY_PROJECTOR = 0, 1, 2
STATUS_NAMES = {0: "PCX_OK", -1: "PCX_EINVAL", -2: "PCX_ENOMEM", -3: "PCX_ENOTHPD", -4: "PCX_ENOCONV",
                -5: "PCX_ENUMERIC", -6: "PCX_ECUDA"}

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libpcx.so")


class PcxError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class pcx_shape(C.Structure):
    _fields_ = [("kind", C.c_int), ("material", C.c_int), ("p", C.c_double * 9)]


class pcx_setup_desc(C.Structure):
    _fields_ = [("n", C.c_int), ("stencil_m", C.c_int), ("ct_reading", C.c_int), ("lattice", C.c_double * 9),
                ("n_mat", C.c_int), ("eps", C.POINTER(C.c_double)), ("background", C.c_int),
                ("n_shape", C.c_int), ("shapes", C.POINTER(pcx_shape)), ("cell_blocks", C.POINTER(C.c_double)),
                ("m_kind", C.c_int), ("crossdof_unchecked", C.c_int)]


class pcx_solve_stats(C.Structure):
    _fields_ = [("iters_fp32", C.c_int), ("iters_fp64", C.c_int), ("applies_fp32", C.c_longlong),
                ("applies_fp64", C.c_longlong), ("ms_total", C.c_double), ("ms_apply", C.c_double),
                ("ms_gram", C.c_double), ("ms_rr", C.c_double), ("ms_other", C.c_double),
                ("gamma_raises", C.c_int), ("gamma_last", C.c_double), ("ms_precond", C.c_double),
                ("learned_fallbacks", C.c_int), ("dumped", C.c_int), ("history_len", C.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class pcx_tune_result(C.Structure):
    _fields_ = [("chunk", C.c_int), ("graphs", C.c_int), ("us_per_vector", C.c_double), ("candidates", C.c_int),
                ("from_cache", C.c_int), ("path", C.c_int), ("x_variant", C.c_int), ("z_variant", C.c_int)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class pcx_solve_opts(C.Structure):
    _fields_ = [("block", C.c_int), ("maxit", C.c_int), ("precision", C.c_int), ("switch_tol", C.c_double),
                ("seed", C.c_uint64), ("verbose", C.c_int), ("stats", C.POINTER(pcx_solve_stats)),
                ("gamma", C.c_double), ("penalty_tol", C.c_double), ("cnn_params", C.c_void_p),
                ("dump_R", C.c_void_p), ("dump_cap", C.c_int), ("dump_every", C.c_int), ("precond_kind", C.c_int),
                ("learned_patience", C.c_int), ("fp32_floor", C.c_double), ("x0", C.c_void_p),
                ("k_concurrency", C.c_int), ("res_history", C.POINTER(C.c_double)), ("res_history_cap", C.c_int)]


_lib = None


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpcx.so is missing at {LIB_PATH}: build it first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        try:   # make torch's CUDA runtime the one libpcx binds to
            import torch  # noqa: F401
        except ImportError:
            pass
        L = C.CDLL(LIB_PATH)
        vp, dp, ip, st = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int), C.c_int
        sig = {
            "pcx_setup": (st, [C.POINTER(pcx_setup_desc), C.POINTER(vp)]),
            "pcx_destroy": (None, [vp]),
            "pcx_sample_host": (st, [C.POINTER(pcx_setup_desc), dp, C.POINTER(C.c_int32), C.POINTER(C.c_longlong)]),
            "pcx_last_error": (C.c_char_p, [vp]),
            "pcx_grid_n": (C.c_int, [vp]),
            "pcx_vector_length": (C.c_size_t, [vp]),
            "pcx_cell_blocks": (st, [vp, dp, dp]),
            "pcx_symbols": (st, [vp, dp, C.c_double, dp, dp, dp, dp]),
            "pcx_set_apply_chunk": (st, [vp, C.c_int]),
            "pcx_get_apply_chunk": (C.c_int, [vp, C.c_int]),
            "pcx_apply": (st, [vp, dp, C.c_double, vp, vp, C.c_int, C.c_int, vp]),
            "pcx_apply_noalloc": (st, [vp, dp, C.c_double, vp, vp, C.c_int, C.c_int, vp]),
            "pcx_apply_host": (st, [vp, dp, C.c_double, vp, vp, C.c_int, C.c_int, vp]),
            "pcx_precond": (st, [vp, dp, C.c_double, vp, vp, C.c_int, C.c_int, vp]),
            "pcx_gram": (st, [vp, vp, C.c_int, vp, C.c_int, C.c_size_t, C.c_int, vp, vp]),
            "pcx_set_gram_path": (st, [C.c_int]),
            "pcx_get_gram_path": (C.c_int, []),
            "pcx_div_norms": (st, [vp, dp, vp, C.c_int, C.c_int, vp, vp]),
            "pcx_apply_kbatch": (st, [vp, dp, C.c_int, C.c_double, vp, vp, C.c_int, C.c_int, vp]),
            "pcx_apply_kbatch_host": (st, [vp, dp, C.c_int, C.c_double, vp, C.c_int, vp, C.c_int, C.c_int, C.c_int,
                                           vp]),
            "pcx_set_apply_graphs": (st, [vp, C.c_int]),
            "pcx_set_apply_path": (st, [vp, C.c_int]),
            "pcx_set_cnn_form": (st, [vp, C.c_int]),
            "pcx_get_apply_path": (C.c_int, [vp, C.c_int]),
            "pcx_set_penalty_form": (st, [vp, C.c_int]),
            "pcx_set_apply_variant": (st, [vp, C.c_int, C.c_int]),
            "pcx_get_apply_variant": (st, [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
            "pcx_get_penalty_form": (C.c_int, [vp]),
            "pcx_autotune": (st, [vp, C.c_int, C.c_int, vp, C.POINTER(pcx_tune_result)]),
            "pcx_sandwich_precond": (st, [vp, dp, C.c_double, vp, vp, C.c_int, C.c_int, vp]),
            "pcx_cnn_init": (st, [C.c_uint64, vp, vp]),
            "pcx_cnn_gates": (st, [vp, vp, vp, vp]),
            "pcx_cnn_forward": (st, [vp, vp, vp, vp, vp, C.c_int, vp]),
            "pcx_cnn_grad": (st, [vp, vp, vp, vp, dp, C.c_int, vp, C.c_int, dp, vp]),
            "pcx_cnn_adam": (st, [vp, vp, vp, vp, C.c_int, C.c_float, vp]),
            "pcx_cnn_precond": (st, [vp, dp, C.c_double, vp, vp, vp, vp, C.c_int, vp]),
            "pcx_cnn_pairs": (st, [vp, dp, C.c_double, vp, vp, vp, vp, dp, C.c_int, vp]),
            "pcx_cg_solve": (st, [vp, dp, C.c_double, vp, vp, C.c_int, C.c_double, C.c_int, ip, dp, vp]),
            "pcx_gram_mixed": (st, [vp, vp, C.c_int, vp, C.c_int, C.c_size_t, vp, vp]),
            "pcx_combine": (st, [vp, vp, C.c_int, vp, C.c_int, C.c_double, vp, C.c_size_t, C.c_int, vp]),
            "pcx_residual": (st, [vp, vp, vp, vp, vp, vp, C.c_int, C.c_size_t, C.c_int, vp]),
            "pcx_rr_eig": (st, [C.c_int, dp, dp, C.c_double, dp, dp, ip]),
            "pcx_solve": (st, [vp, dp, C.c_int, C.c_int, C.c_double, C.POINTER(pcx_solve_opts), dp, dp, ip, vp, vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return [n for n in ("pcx_setup", "pcx_sample_host", "pcx_destroy", "pcx_last_error", "pcx_grid_n", "pcx_vector_length",
                        "pcx_cell_blocks", "pcx_symbols", "pcx_set_apply_chunk", "pcx_get_apply_chunk", "pcx_apply", "pcx_apply_noalloc", "pcx_apply_host", "pcx_precond",
                        "pcx_div_norms", "pcx_apply_kbatch", "pcx_apply_kbatch_host", "pcx_set_apply_graphs", "pcx_set_apply_path", "pcx_get_apply_path", "pcx_set_penalty_form", "pcx_get_penalty_form", "pcx_set_apply_variant", "pcx_get_apply_variant", "pcx_set_cnn_form", "pcx_autotune",
                        "pcx_sandwich_precond", "pcx_cnn_init", "pcx_cnn_gates",
                        "pcx_cnn_forward", "pcx_cnn_grad", "pcx_cnn_adam", "pcx_cnn_precond", "pcx_cnn_pairs",
                        "pcx_cg_solve", "pcx_gram", "pcx_set_gram_path", "pcx_get_gram_path", "pcx_gram_mixed", "pcx_combine", "pcx_residual", "pcx_rr_eig", "pcx_solve")]


def _check(status, ctx=None):
    if status != PCX_OK:
        msg = lib().pcx_last_error(ctx)
        raise PcxError(status, msg.decode() if msg else "")


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _kvec(k):
    k = np.ascontiguousarray(np.asarray(k, dtype=np.float64).reshape(3))
    return k, _dptr(k)


def _stream(stream):
    if stream is not None:
        return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _prec_of(t):
    import torch
    if t.dtype == torch.complex64:
        return PCX_FP32
    if t.dtype == torch.complex128:
        return PCX_FP64
    raise TypeError(f"expected complex64 or complex128, got {t.dtype}")


def _devptr(t):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


class Context:
    """Owns a pcx_ctx (device M, symbol and twiddle tables)."""

    def __init__(self, handle, n, keep=None):
        self.handle = handle
        self.n = n
        self._keep = keep

    @property
    def vector_length(self):
        return int(lib().pcx_vector_length(self.handle))

    def close(self):
        if self.handle:
            lib().pcx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PCX_M_TRIVIAL, PCX_M_CROSSDOF = 0, 1


def _desc(n, lattice, eps, background, shapes, stencil_m, ct_reading, cell_blocks, m_kind=PCX_M_TRIVIAL,
          crossdof_unchecked=False):
    d = pcx_setup_desc()
    d.n = n
    d.m_kind = m_kind
    d.crossdof_unchecked = int(bool(crossdof_unchecked))
    d.stencil_m = stencil_m
    d.ct_reading = ct_reading
    lat = np.eye(3) if lattice is None else np.asarray(lattice, dtype=np.float64)
    for i, v in enumerate(lat.reshape(9)):
        d.lattice[i] = v
    keep = []
    if cell_blocks is not None:
        cb = np.ascontiguousarray(np.asarray(cell_blocks, dtype=np.float64).reshape(-1))
        keep.append(cb)
        d.cell_blocks = _dptr(cb)
    else:
        e = np.asarray(eps, dtype=np.complex128)
        epsf = np.ascontiguousarray(np.stack([e.real, e.imag], axis=-1).reshape(-1))
        keep.append(epsf)
        d.n_mat = e.shape[0]
        d.eps = _dptr(epsf)
        d.background = background
        arr = (pcx_shape * max(1, len(shapes)))()
        for i, s in enumerate(shapes):
            arr[i].kind = int(s.kind)
            arr[i].material = int(s.material)
            for j, v in enumerate(s.params):
                arr[i].p[j] = float(v)
        keep.append(arr)
        d.n_shape = len(shapes)
        d.shapes = C.cast(arr, C.POINTER(pcx_shape))
    return d, keep


def pcx_setup(n, lattice=None, eps=None, background=0, shapes=(), stencil_m=1, ct_reading=PCX_CT_SUMMED,
              cell_blocks=None, m_kind=PCX_M_TRIVIAL, crossdof_unchecked=False):
    """Create a context.  ``eps``: (n_mat, 3, 3) complex permittivities;
    ``shapes``: objects with .kind, .material, .params; ``cell_blocks``:
    optional (N^3, 9) float64 packed blocks overriding the structure."""
    d, keep = _desc(n, lattice, eps, background, shapes, stencil_m, ct_reading, cell_blocks, m_kind,
                    crossdof_unchecked)
    h = C.c_void_p()
    st = lib().pcx_setup(C.byref(d), C.byref(h))
    if st != PCX_OK:
        msg = lib().pcx_last_error(h if h.value else None)
        if h.value:
            lib().pcx_destroy(h)
        raise PcxError(st, msg.decode() if msg else "")
    return Context(h, n)


def setup_structure(structure, n, stencil_m=1, ct_reading=PCX_CT_SUMMED, m_kind=PCX_M_TRIVIAL,
                    crossdof_unchecked=False):
    """pcx_setup from a ``workloads.Structure``."""
    return pcx_setup(n, structure.lattice, structure.eps, structure.background, structure.shapes,
                     stencil_m=stencil_m, ct_reading=ct_reading, m_kind=m_kind,
                     crossdof_unchecked=crossdof_unchecked)


def pcx_sample_host(structure, n, stencil_m=1, ct_reading=PCX_CT_SUMMED, m_kind=PCX_M_TRIVIAL, cell_blocks=None):
    """Host sampling (no GPU): (blocks (N^3, 9), ids (4, N^3) int32, first_bad)."""
    d, keep = _desc(n, structure.lattice, structure.eps, structure.background, structure.shapes, stencil_m,
                    ct_reading, cell_blocks, m_kind)
    n3 = n ** 3
    blocks = np.zeros((n3, 9))
    ids = np.zeros((4, n3), dtype=np.int32)
    bad = C.c_longlong()
    _check(lib().pcx_sample_host(C.byref(d), _dptr(blocks), ids.ctypes.data_as(C.POINTER(C.c_int32)),
                                 C.byref(bad)))
    return blocks, ids, bad.value


def pcx_cell_blocks(ctx):
    n3 = ctx.n ** 3
    out = np.zeros((n3, 9), dtype=np.float64)
    lmin = np.zeros(1)
    _check(lib().pcx_cell_blocks(ctx.handle, _dptr(out), _dptr(lmin)), ctx.handle)
    return out, float(lmin[0])


def pcx_symbols(ctx, k, gamma=0.0):
    n = ctx.n
    s = np.zeros((3, n, 2))
    q = np.zeros((3, n, 2))
    b = np.zeros(9)
    g = np.zeros(1)
    kk, kp = _kvec(k)
    _check(lib().pcx_symbols(ctx.handle, kp, float(gamma), _dptr(s), _dptr(q), _dptr(b), _dptr(g)), ctx.handle)
    return s[..., 0] + 1j * s[..., 1], q[..., 0] + 1j * q[..., 1], b.reshape(3, 3), float(g[0])


def pcx_set_apply_chunk(ctx, chunk):
    _check(lib().pcx_set_apply_chunk(ctx.handle, int(chunk)), ctx.handle)


def pcx_get_apply_chunk(ctx, precision):
    return int(lib().pcx_get_apply_chunk(ctx.handle, int(precision)))


def pcx_apply(ctx, k, X, Y, gamma=0.0, stream=None):
    kk, kp = _kvec(k)
    prec = _prec_of(X)
    if Y.dtype != X.dtype or Y.shape != X.shape:
        raise ValueError("X and Y must have the same dtype and shape")
    nvec = X.shape[0] if X.dim() == 5 else X.numel() // ctx.vector_length
    _check(lib().pcx_apply(ctx.handle, kp, float(gamma), _devptr(X), _devptr(Y), nvec, prec, _stream(stream)),
           ctx.handle)
    return Y


def pcx_apply_noalloc(ctx, k, X, Y, gamma=0.0, stream=None):
    """pcx_apply without any device allocation (static 32 MiB scratch)."""
    kk, kp = _kvec(k)
    prec = _prec_of(X)
    if Y.dtype != X.dtype or Y.shape != X.shape:
        raise ValueError("X and Y must have the same dtype and shape")
    nvec = X.shape[0] if X.dim() == 5 else X.numel() // ctx.vector_length
    _check(lib().pcx_apply_noalloc(ctx.handle, kp, float(gamma), _devptr(X), _devptr(Y), nvec, prec,
                                   _stream(stream)), ctx.handle)
    return Y


def pcx_apply_host(ctx, k, X, Y, gamma=0.0, stream=None):
    """X, Y: host arrays (numpy or CPU torch; pinned memory copies fastest)."""
    kk, kp = _kvec(k)
    if isinstance(X, np.ndarray):
        prec = PCX_FP32 if X.dtype == np.complex64 else PCX_FP64
        xp, yp = X.ctypes.data, Y.ctypes.data
        nvec = X.size // ctx.vector_length
    else:
        prec = _prec_of(X)
        xp, yp = X.data_ptr(), Y.data_ptr()
        nvec = X.numel() // ctx.vector_length
    _check(lib().pcx_apply_host(ctx.handle, kp, float(gamma), C.c_void_p(xp), C.c_void_p(yp), nvec, prec,
                                _stream(stream)), ctx.handle)
    return Y


def pcx_precond(ctx, k, R, W, gamma=0.0, stream=None):
    kk, kp = _kvec(k)
    nvec = R.numel() // ctx.vector_length
    _check(lib().pcx_precond(ctx.handle, kp, float(gamma), _devptr(R), _devptr(W), nvec, _prec_of(R),
                             _stream(stream)), ctx.handle)
    return W


def pcx_gram(A, B, G, L=None, ctx=None, stream=None):
    """G (complex128 CUDA tensor, na x nb) = A^H B for column blocks A (na, L), B (nb, L)."""
    na, nb = A.shape[0], B.shape[0]
    L = A[0].numel() if L is None else L
    _check(lib().pcx_gram(ctx.handle if ctx else None, _devptr(A), na, _devptr(B), nb, L, _prec_of(A), _devptr(G),
                          _stream(stream)), ctx.handle if ctx else None)
    return G


PCX_GRAM_AUTO, PCX_GRAM_TENSOR, PCX_GRAM_FP32 = 0, 1, 2


def pcx_set_gram_path(path):
    """Process-wide complex64 Gram kernel: PCX_GRAM_AUTO, PCX_GRAM_TENSOR or PCX_GRAM_FP32."""
    _check(lib().pcx_set_gram_path(int(path)), None)


def pcx_get_gram_path():
    return int(lib().pcx_get_gram_path())


def pcx_div_norms(ctx, k, X, out, stream=None):
    """out (float64 CUDA, 2 nvec) = [x_j^H K_B x_j, ||x_j||^2] per column of X."""
    kk = np.ascontiguousarray(np.asarray(k, dtype=np.float64).reshape(3))
    _check(lib().pcx_div_norms(ctx.handle, _dptr(kk), _devptr(X), X.shape[0], _prec_of(X), _devptr(out),
                               _stream(stream)), ctx.handle)
    return out


PCX_CNN_HIDDEN = 8
PCX_CNN_HERMITIAN, PCX_CNN_BF16 = 1, 2


PCX_CNN_NPARAMS = (PCX_CNN_HIDDEN * 3 * 27 + PCX_CNN_HIDDEN * PCX_CNN_HIDDEN * 27 + 3 * PCX_CNN_HIDDEN * 27
                   + 2 * (PCX_CNN_HIDDEN * 9 * 27 + PCX_CNN_HIDDEN))


def pcx_apply_kbatch(ctx, kpts, X, Y, gamma=0.0, stream=None):
    """Y[i, j] = Op(k_i) X[i, j] for X, Y shaped (nk, vec_per_k, 3, N, N, N)."""
    kp = np.ascontiguousarray(np.asarray(kpts, dtype=np.float64).reshape(-1, 3))
    nk, vpk = X.shape[0], X.shape[1]
    if kp.shape[0] != nk:
        raise ValueError("pcx_apply_kbatch: one k per group")
    _check(lib().pcx_apply_kbatch(ctx.handle, _dptr(kp), nk, float(gamma), _devptr(X), _devptr(Y), vpk, _prec_of(X),
                                  _stream(stream)), ctx.handle)
    return Y


def pcx_apply_kbatch_host(ctx, kpts, X, Y, vec_per_k, x_stride=None, y_stride=None, gamma=0.0, stream=None):
    """Host-buffer k-batched apply: group i (vec_per_k vectors) at vector
    i * x_stride of X is applied with kpts[i] and written at vector
    i * y_stride of Y (strides in vectors, default vec_per_k; 0 reuses one
    block).  X, Y: host numpy arrays or CPU torch tensors (pinned memory
    copies fastest)."""
    kp = np.ascontiguousarray(np.asarray(kpts, dtype=np.float64).reshape(-1, 3))
    nk = kp.shape[0]
    xs = vec_per_k if x_stride is None else x_stride
    ys = vec_per_k if y_stride is None else y_stride
    if isinstance(X, np.ndarray):
        prec = PCX_FP32 if X.dtype == np.complex64 else PCX_FP64
        xp, yp = X.ctypes.data, Y.ctypes.data
        nx, ny = X.size // ctx.vector_length, Y.size // ctx.vector_length
    else:
        prec = _prec_of(X)
        xp, yp = X.data_ptr(), Y.data_ptr()
        nx, ny = X.numel() // ctx.vector_length, Y.numel() // ctx.vector_length
    if nk > 0 and ((nk - 1) * xs + vec_per_k > nx or (nk - 1) * ys + vec_per_k > ny):
        raise ValueError("pcx_apply_kbatch_host: X or Y too small for the strides")
    _check(lib().pcx_apply_kbatch_host(ctx.handle, _dptr(kp), nk, float(gamma), C.c_void_p(xp), int(xs),
                                       C.c_void_p(yp), int(ys), int(vec_per_k), prec, _stream(stream)), ctx.handle)
    return Y


def pcx_set_apply_graphs(ctx, enable):
    _check(lib().pcx_set_apply_graphs(ctx.handle, int(bool(enable))), ctx.handle)


def pcx_set_cnn_form(ctx, flags):
    _check(lib().pcx_set_cnn_form(ctx.handle, int(flags)), ctx.handle)


def pcx_set_apply_path(ctx, path):
    _check(lib().pcx_set_apply_path(ctx.handle, int(path)), ctx.handle)


def pcx_get_apply_path(ctx, precision):
    return int(lib().pcx_get_apply_path(ctx.handle, int(precision)))


def pcx_set_apply_variant(ctx, x_variant=-1, z_variant=-1):
    _check(lib().pcx_set_apply_variant(ctx.handle, int(x_variant), int(z_variant)), ctx.handle)


def pcx_get_apply_variant(ctx):
    xv, zv = C.c_int(), C.c_int()
    _check(lib().pcx_get_apply_variant(ctx.handle, C.byref(xv), C.byref(zv)), ctx.handle)
    return xv.value, zv.value


def pcx_set_penalty_form(ctx, form):
    _check(lib().pcx_set_penalty_form(ctx.handle, int(form)), ctx.handle)


def pcx_get_penalty_form(ctx):
    return int(lib().pcx_get_penalty_form(ctx.handle))


def pcx_autotune(ctx, precision, nvec, stream=None):
    """Tunes the apply launch configuration; returns the pcx_tune_result as a dict."""
    r = pcx_tune_result()
    _check(lib().pcx_autotune(ctx.handle, int(precision), int(nvec), _stream(stream), C.byref(r)), ctx.handle)
    return r.as_dict()


def pcx_sandwich_precond(ctx, k, R, W, gamma=0.0, stream=None):
    """W = T0 R, the curl-sandwich approximate inverse (complex64 or complex128)."""
    kk, kp = _kvec(k)
    _check(lib().pcx_sandwich_precond(ctx.handle, kp, float(gamma), _devptr(R), _devptr(W), R.shape[0], _prec_of(R),
                                      _stream(stream)), ctx.handle)
    return W


def pcx_cnn_init(seed, params, stream=None):
    """params (float32 CUDA, PCX_CNN_NPARAMS): seeded initial parameters."""
    _check(lib().pcx_cnn_init(int(seed), _devptr(params), _stream(stream)))
    return params


def pcx_cnn_gates(ctx, params, gates, stream=None):
    """gates (float32 CUDA, 2 * 8 * N^3): the gate fields of the structure."""
    _check(lib().pcx_cnn_gates(ctx.handle, _devptr(params), _devptr(gates), _stream(stream)), ctx.handle)
    return gates


def pcx_cnn_forward(ctx, params, gates, U, Y, stream=None):
    """Y = g(Re U) + i g(Im U) (complex64 real-space fields)."""
    _check(lib().pcx_cnn_forward(ctx.handle, _devptr(params), _devptr(gates), _devptr(U), _devptr(Y), U.shape[0],
                                 _stream(stream)), ctx.handle)
    return Y


def pcx_cnn_grad(ctx, params, U, T, w, grad, accumulate=False, stream=None):
    """Returns L = sum_v w_v ||g(U_v) - T_v||^2; grad (float32 CUDA) receives (or accumulates) dL/dparams."""
    wv = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    loss = np.zeros(1)
    _check(lib().pcx_cnn_grad(ctx.handle, _devptr(params), _devptr(U), _devptr(T), _dptr(wv), U.shape[0],
                              _devptr(grad), int(bool(accumulate)), _dptr(loss), _stream(stream)), ctx.handle)
    return float(loss[0])


def pcx_cnn_adam(params, grad, m, v, step, lr, stream=None):
    _check(lib().pcx_cnn_adam(_devptr(params), _devptr(grad), _devptr(m), _devptr(v), int(step), float(lr),
                              _stream(stream)))
    return params


def pcx_cnn_precond(ctx, k, params, gates, R, W, gamma=0.0, stream=None):
    """W = K_P^{-1} R + F3^H g(F3 K_P^{-1} R) (complex64, Fourier basis)."""
    kk, kp = _kvec(k)
    _check(lib().pcx_cnn_precond(ctx.handle, kp, float(gamma), _devptr(params), _devptr(gates), _devptr(R),
                                 _devptr(W), R.shape[0], _stream(stream)), ctx.handle)
    return W


def pcx_cnn_pairs(ctx, k, R, E, U, T, gamma=0.0, stream=None):
    """U = F3 K_P^{-1} R, T = F3 (E - K_P^{-1} R); returns ||E_v||^2 (numpy)."""
    kk, kp = _kvec(k)
    en2 = np.zeros(R.shape[0])
    _check(lib().pcx_cnn_pairs(ctx.handle, kp, float(gamma), _devptr(R), _devptr(E), _devptr(U), _devptr(T),
                               _dptr(en2), R.shape[0], _stream(stream)), ctx.handle)
    return en2


def pcx_cg_solve(ctx, k, R, E, tol=1e-4, maxit=200, gamma=0.0, stream=None):
    """E = Op^{-1} R by PCG; returns (iterations, relative residuals)."""
    kk, kp = _kvec(k)
    its = np.zeros(1, dtype=np.int32)
    rel = np.zeros(R.shape[0])
    _check(lib().pcx_cg_solve(ctx.handle, kp, float(gamma), _devptr(R), _devptr(E), R.shape[0], float(tol),
                              int(maxit), its.ctypes.data_as(C.POINTER(C.c_int)), _dptr(rel), _stream(stream)),
           ctx.handle)
    return int(its[0]), rel


def pcx_gram_mixed(A, B, G, ctx=None, stream=None):
    """G (complex128 CUDA tensor, na x nb) = A^H B with A complex128 (na, L) and B complex64 (nb, L)."""
    import torch
    na, nb = A.shape[0], B.shape[0]
    L = A[0].numel()
    if A.dtype != torch.complex128 or B.dtype != torch.complex64 or B[0].numel() != L:
        raise ValueError("pcx_gram_mixed: A complex128 and B complex64 with equal column lengths")
    _check(lib().pcx_gram_mixed(ctx.handle if ctx else None, _devptr(A), na, _devptr(B), nb, L, _devptr(G),
                                _stream(stream)), ctx.handle if ctx else None)
    return G


def pcx_combine(S, Cm, Y, beta=0.0, ctx=None, stream=None):
    """Y_j = sum_i S_i C[i, j] (+ beta Y_j); Cm: complex128 CUDA tensor (ns, ny)."""
    ns, ny = S.shape[0], Y.shape[0]
    L = S[0].numel()
    _check(lib().pcx_combine(ctx.handle if ctx else None, _devptr(S), ns, _devptr(Cm), ny, float(beta), _devptr(Y),
                             L, _prec_of(S), _stream(stream)), ctx.handle if ctx else None)
    return Y


def pcx_residual(X, AX, theta, R, norms, ctx=None, stream=None):
    """R = AX - X diag(theta); norms (float64 CUDA, 2 nvec) = [|R_j|^2, |X_j|^2]."""
    nvec = X.shape[0]
    L = X[0].numel()
    _check(lib().pcx_residual(ctx.handle if ctx else None, _devptr(X), _devptr(AX), _devptr(theta), _devptr(R),
                              _devptr(norms), nvec, L, _prec_of(X), _stream(stream)), ctx.handle if ctx else None)
    return R, norms


def pcx_rr_eig(ga, gb, drop_tol=1e-13):
    """Host Rayleigh-Ritz: returns (theta[r], C (m, r)) for ga c = theta gb c."""
    ga = np.ascontiguousarray(ga, dtype=np.complex128)
    gb = np.ascontiguousarray(gb, dtype=np.complex128)
    m = ga.shape[0]
    th = np.zeros(m)
    cm = np.zeros((m, m), dtype=np.complex128)
    rank = C.c_int()
    st = lib().pcx_rr_eig(m, ga.ctypes.data_as(C.POINTER(C.c_double)), gb.ctypes.data_as(C.POINTER(C.c_double)),
                          float(drop_tol), _dptr(th), cm.ctypes.data_as(C.POINTER(C.c_double)), C.byref(rank))
    _check(st)
    r = rank.value
    return th[:r], cm.reshape(-1)[: m * r].reshape(m, r)


def pcx_solve(ctx, kpts, nev, tol, block=0, maxit=0, precision=PCX_FP64, switch_tol=0.0, seed=0, verbose=0,
              vec_out=None, stream=None, raise_on_noconv=True, stats=None, gamma=0.0, penalty_tol=0.0,
              cnn_params=None, dump_R=None, dump_every=0, precond_kind=0, learned_patience=0, fp32_floor=0.0,
              x0=None, k_concurrency=0, res_history=None):
    """Returns (eig (nk, nev), res (nk, nev), iters (nk,), status).  Pass a
    pcx_solve_stats instance as ``stats`` to receive counters and timings,
    and a float64 numpy array as ``res_history`` to receive the worst wanted
    residual of every iteration (count in stats.history_len)."""
    kp = np.ascontiguousarray(np.asarray(kpts, dtype=np.float64).reshape(-1, 3))
    nk = kp.shape[0]
    o = pcx_solve_opts(block, maxit, precision, switch_tol, seed, verbose,
                       C.pointer(stats) if stats is not None else None, float(gamma), float(penalty_tol),
                       _devptr(cnn_params) if cnn_params is not None else None,
                       _devptr(dump_R) if dump_R is not None else None,
                       int(dump_R.shape[0]) if dump_R is not None else 0, int(dump_every), int(precond_kind),
                       int(learned_patience), float(fp32_floor), _devptr(x0) if x0 is not None else None,
                       int(k_concurrency))
    if res_history is not None:
        if res_history.dtype != np.float64 or not res_history.flags["C_CONTIGUOUS"]:
            raise ValueError("res_history must be a contiguous float64 array")
        o.res_history = _dptr(res_history)
        o.res_history_cap = int(res_history.size)
    eig = np.zeros((nk, nev))
    res = np.zeros((nk, nev))
    its = np.zeros(nk, dtype=np.int32)
    vptr = _devptr(vec_out) if vec_out is not None else None
    st = lib().pcx_solve(ctx.handle, _dptr(kp), nk, nev, float(tol), C.byref(o), _dptr(eig), _dptr(res),
                         its.ctypes.data_as(C.POINTER(C.c_int)), vptr, _stream(stream))
    if st != PCX_OK and not (st == PCX_ENOCONV and not raise_on_noconv):
        _check(st, ctx.handle)
    return eig, res, its, st
