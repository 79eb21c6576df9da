"""ctypes binding of libpcx_baselines.so: the cuFFT / cuBLAS versions of the
apply and of the Gram products that the benchmark times beside libpcx.

Nothing in libpcx or in paper_2511_17107_gb300.pcx loads this library; it
exists only to be timed.  The per-mode symbol kappa and the cell blocks come
from libpcx's own host outputs (pcx_symbols, pcx_cell_blocks), so both
sides apply the same operator.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .. import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build_baselines()
        L = C.CDLL(path)
        vp, dp = C.c_void_p, C.POINTER(C.c_double)
        L.pcxb_create.restype = C.c_int
        L.pcxb_create.argtypes = [C.c_int, C.c_int, dp, dp, C.c_double, C.c_int, C.POINTER(vp)]
        L.pcxb_apply.restype = C.c_int
        L.pcxb_apply.argtypes = [vp, vp, vp, C.c_int, vp]
        L.pcxb_destroy.restype = None
        L.pcxb_destroy.argtypes = [vp]
        L.pcxb_gram.restype = C.c_int
        L.pcxb_gram.argtypes = [vp, C.c_int, vp, C.c_int, C.c_size_t, C.c_int, vp, vp]
        _lib = L
    return _lib


def kappa_field(pcx, ctx, k, gamma=0.0):
    """[3][N^3] complex128 kappa_i(p) = sum_j b_ji S_j(p_j) + Q_i(p_i) from the
    tables of pcx_symbols, and the gamma in use."""
    s_tab, q_tab, b, g = pcx.pcx_symbols(ctx, k, gamma)
    n = ctx.n
    idx = np.arange(n)
    kap = np.zeros((3, n, n, n), dtype=np.complex128)   # [i][p3][p2][p1]
    for i in range(3):
        kap[i] += b[0, i] * s_tab[0][idx][None, None, :]
        kap[i] += b[1, i] * s_tab[1][idx][None, :, None]
        kap[i] += b[2, i] * s_tab[2][idx][:, None, None]
    kap[0] += q_tab[0][None, None, :]
    kap[1] += q_tab[1][None, :, None]
    kap[2] += q_tab[2][:, None, None]
    return kap.reshape(3, -1), g


class CufftApply:
    """Baseline apply of one context at one k: batched cuFFT transforms and
    elementwise kernels over stored kappa and M arrays."""

    def __init__(self, pcx, ctx, k, precision, chunk):
        kap, g = kappa_field(pcx, ctx, k)
        blocks, _ = pcx.pcx_cell_blocks(ctx)
        kv = np.ascontiguousarray(np.stack([kap.real, kap.imag], axis=-1)).ravel()
        bv = np.ascontiguousarray(blocks, dtype=np.float64).ravel()
        h = C.c_void_p()
        st = lib().pcxb_create(ctx.n, 0 if precision == pcx.PCX_FP64 else 1,
                               kv.ctypes.data_as(C.POINTER(C.c_double)), bv.ctypes.data_as(C.POINTER(C.c_double)),
                               float(g), int(chunk), C.byref(h))
        if st != 0:
            raise RuntimeError(f"pcxb_create failed ({st})")
        self.h = h
        self.chunk = chunk

    def __call__(self, X, Y, stream=None):
        nvec = X.shape[0]
        st = lib().pcxb_apply(self.h, C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()), int(nvec),
                              C.c_void_p(stream.cuda_stream if stream is not None else 0))
        if st != 0:
            raise RuntimeError(f"pcxb_apply failed ({st})")

    def close(self):
        if self.h:
            lib().pcxb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cublas_gram(A, B, G, stream=None):
    """G = A^H B with cublasCgemm (complex64) / cublasZgemm (complex128); A,
    B are [n][L] column blocks, G an (na, nb) tensor of A's dtype whose
    column-major data receive the product."""
    import torch
    prec = 0 if A.dtype == torch.complex128 else 1
    na, L = A.shape
    nb = B.shape[0]
    st = lib().pcxb_gram(C.c_void_p(A.data_ptr()), na, C.c_void_p(B.data_ptr()), nb, L, prec,
                         C.c_void_p(G.data_ptr()), C.c_void_p(stream.cuda_stream if stream is not None else 0))
    if st != 0:
        raise RuntimeError(f"pcxb_gram failed ({st})")
