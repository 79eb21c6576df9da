"""Learned preconditioner correction (oracle; test infrastructure only).

The paper has no learned component.  This module defines the preconditioner
that the learned part corrects and the correction, in plain numpy FP64.

Base: the curl-sandwich approximate inverse of the compensated operator
(Johnson and Joannopoulos, Opt. Express 8 (2001) 173, Sec. 3.1, restated for
the Fourier basis of Sec. 2.4 and the symbols of Prop. 2.8):

    T0 r = K_A F3_3^H eps F3_3 (K_A^H r / |k|^2) / |k|^2 + K_B r / (gamma |k|^4)

with eps = M^{-1} cell by cell (the inverse of the 3x3 block of Sec. 3.2.1)
and |k|^2 = sum_i |kappa_i|^2 per mode.  Because K_A K_A^H + K_B = |k|^2 I
per mode, T0 is the exact inverse of Op = K_A F3_3^H M F3_3 K_A^H + gamma K_B
for a homogeneous isotropic medium; it differs from K_P^{-1} (eq.
matrixfree_finalform) only in carrying eps through real space.  Modes with
|k| = 0 (k = 0, p = 0: the null space H of Prop. 2.5) map to 0.

Correction: a three-layer circular 3D convolution net g acts next to eps on
the real-space field e = F3_3 (K_A^H r / |k|^2):

    T(r) = T0 r + K_A F3_3^H g(e) / |k|^2,

    f      = the 9 reals of the cell block of M: d1, d2, d3,
             Re/Im M_12, Re/Im M_13, Re/Im M_23            (9 x N^3)
    g1     = sigmoid(conv(f, V1) + c1)                      (C x N^3)
    g2     = sigmoid(conv(f, V2) + c2)
    a1     = conv(u, W1),  h1 = a1 * g1                     (3 -> C)
    a2     = conv(h1, W2), h2 = a2 * g2                     (C -> C)
    y      = conv(h2, W3)                                   (C -> 3)

g is linear in u for a fixed structure and acts on the real and imaginary
parts of the complex field with the same weights, so T is complex-linear.

Hermitian form (symmetric=True): g_s = (g + g^T) / 2 with the transpose

    g^T(u) = conv^T(g1 * conv^T(g2 * conv^T(u, W3), W2), W1)

(conv^T the adjoint of conv).  g_s is a symmetric real map, so T(r) =
T0 r + B^H g_s B r with B = F3_3 K_A^H / |k|^2 is Hermitian like T0 (F3_3 is
unitary): the form a conjugate-gradient-type eigensolver expects of its
preconditioner.

conv is a cross-correlation with 3 x 3 x 3 taps and periodic wrap-around:
conv(x, w)[o, z, y, x] = sum_{i, dz, dy, dx} w[o, i, dz+1, dy+1, dx+1]
x[i, z+dz, y+dy, x+dx].

Training target: e_r = Op^{-1} r (Op of eq. matrixfree_kcform).  If g(U) = T
with U = F3_3 (K_A^H r / |k|^2) and T = F3_3 K_A^H (e_r - T0 r), then
T(r) = T0 r + P (e_r - T0 r) with P = K_A K_A^H / |k|^2 the projector on the
range of K_A, whose complement T0 already inverts exactly; the loss is
sum_v w_v ||g(U_v) - T_v||^2 with w_v = 1 / (count ||K_A^H e_v||^2).

Parameters are one flat vector in the order W1, W2, W3, V1, c1, V2, c2, each
in C order (param_shapes).  The BF16 form evaluates the network with every
convolution weight rounded to bfloat16 (rounded(p)); its gradient is the
gradient of that network, applied to the unrounded parameters.
"""
from __future__ import annotations

import numpy as np

from . import fourier

HIDDEN = 8
OFFSETS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def param_shapes(c: int = HIDDEN):
    return [("W1", (c, 3, 3, 3, 3)), ("W2", (c, c, 3, 3, 3)), ("W3", (3, c, 3, 3, 3)),
            ("V1", (c, 9, 3, 3, 3)), ("c1", (c,)), ("V2", (c, 9, 3, 3, 3)), ("c2", (c,))]


def param_count(c: int = HIDDEN) -> int:
    return int(sum(np.prod(s) for _, s in param_shapes(c)))


def unpack(flat: np.ndarray, c: int = HIDDEN) -> dict:
    out, o = {}, 0
    for name, shape in param_shapes(c):
        size = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + size], dtype=np.float64).reshape(shape)
        o += size
    return out


def pack(p: dict, c: int = HIDDEN) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in param_shapes(c)])


def features(blocks: np.ndarray) -> np.ndarray:
    """(9, N, N, N) channels of the cell blocks (N, N, N, 3, 3) of M."""
    return np.stack([blocks[..., 0, 0].real, blocks[..., 1, 1].real, blocks[..., 2, 2].real,
                     blocks[..., 0, 1].real, blocks[..., 0, 1].imag,
                     blocks[..., 0, 2].real, blocks[..., 0, 2].imag,
                     blocks[..., 1, 2].real, blocks[..., 1, 2].imag])


def _shift(x: np.ndarray, dz: int, dy: int, dx: int) -> np.ndarray:
    """s[..., z, y, x] = x[..., z+dz, y+dy, x+dx] (periodic)."""
    return np.roll(x, (-dz, -dy, -dx), axis=(-3, -2, -1))


def conv(x: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Circular cross-correlation, x (Cin, N, N, N), w (Cout, Cin, 3, 3, 3)."""
    out = np.zeros((w.shape[0],) + x.shape[1:])
    for dz, dy, dx in OFFSETS:
        xs = _shift(x, dz, dy, dx)
        out += np.einsum("oi,izyx->ozyx", w[:, :, dz + 1, dy + 1, dx + 1], xs)
    return out


def conv_adjoint(dy: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Adjoint of conv(., w) applied to dy (Cout, N, N, N) -> (Cin, N, N, N)."""
    out = np.zeros((w.shape[1],) + dy.shape[1:])
    for dz, dy_, dx in OFFSETS:
        out += _shift(np.einsum("oi,ozyx->izyx", w[:, :, dz + 1, dy_ + 1, dx + 1], dy), -dz, -dy_, -dx)
    return out


def conv_weight_grad(dy: np.ndarray, x: np.ndarray) -> np.ndarray:
    """d/dw of <dy, conv(x, w)>: (Cout, Cin, 3, 3, 3)."""
    g = np.zeros((dy.shape[0], x.shape[0], 3, 3, 3))
    for dz, dy_, dx in OFFSETS:
        g[:, :, dz + 1, dy_ + 1, dx + 1] = np.einsum("ozyx,izyx->oi", dy, _shift(x, dz, dy_, dx))
    return g


def to_bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (8 exponent, 7 fraction bits), ties to
    even, from the float32 value of x: keep the top 16 bits of the float32
    encoding after adding 0x7FFF plus the lowest kept bit."""
    b = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def rounded(p: dict) -> dict:
    """The parameters with every convolution weight rounded to bfloat16 (the
    biases c1, c2 stay as they are): the network the BF16 form evaluates."""
    return {k: (to_bf16(v) if k[0] in "WV" else v) for k, v in p.items()}


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def gates(p: dict, f: np.ndarray):
    g1 = sigmoid(conv(f, p["V1"]) + p["c1"][:, None, None, None])
    g2 = sigmoid(conv(f, p["V2"]) + p["c2"][:, None, None, None])
    return g1, g2


def forward_real(p: dict, f: np.ndarray, u: np.ndarray, g=None):
    """g(u) for one real (3, N, N, N) sample; returns (y, cache)."""
    g1, g2 = gates(p, f) if g is None else g
    a1 = conv(u, p["W1"])
    h1 = a1 * g1
    a2 = conv(h1, p["W2"])
    h2 = a2 * g2
    y = conv(h2, p["W3"])
    return y, dict(u=u, g1=g1, g2=g2, a1=a1, h1=h1, a2=a2, h2=h2)


def transpose_real(p: dict, f: np.ndarray, u: np.ndarray, g=None):
    """g^T(u) for one real (3, N, N, N) sample; returns (y, cache)."""
    g1, g2 = gates(p, f) if g is None else g
    b3 = conv_adjoint(u, p["W3"])
    k2 = b3 * g2
    b2 = conv_adjoint(k2, p["W2"])
    k1 = b2 * g1
    y = conv_adjoint(k1, p["W1"])
    return y, dict(u=u, b3=b3, k2=k2, b2=b2, k1=k1)


def forward(p: dict, f: np.ndarray, U: np.ndarray, symmetric: bool = False) -> np.ndarray:
    """Complex field U (..., 3, N, N, N): g(Re U) + i g(Im U), or with
    symmetric=True the same with g_s = (g + g^T) / 2."""
    g = gates(p, f)
    flat = U.reshape((-1,) + U.shape[-4:])
    out = np.empty(flat.shape, dtype=np.complex128)

    def one(u):
        y, _ = forward_real(p, f, u, g)
        if symmetric:
            y = 0.5 * (y + transpose_real(p, f, u, g)[0])
        return y

    for v in range(flat.shape[0]):
        out[v] = one(flat[v].real) + 1j * one(flat[v].imag)
    return out.reshape(U.shape)


def loss_and_grad(p: dict, f: np.ndarray, U: np.ndarray, T: np.ndarray, w: np.ndarray, symmetric: bool = False):
    """L = sum_v w_v ||g(U_v) - T_v||^2 over complex samples (nvec, 3, N, N, N)
    (g_s in place of g with symmetric=True) and dL/dparams (dict), by the
    chain rule through every layer of both paths."""
    g1, g2 = gates(p, f)
    grads = {name: np.zeros(shape) for name, shape in param_shapes(p["W1"].shape[0])}
    dg1 = np.zeros_like(g1)
    dg2 = np.zeros_like(g2)
    loss = 0.0
    for v in range(U.shape[0]):
        for part in (np.real, np.imag):
            y, cch = forward_real(p, f, part(U[v]), (g1, g2))
            if symmetric:
                yt, cct = transpose_real(p, f, part(U[v]), (g1, g2))
                y = 0.5 * (y + yt)
            diff = y - part(T[v])
            loss += w[v] * np.sum(diff ** 2)
            dy = 2.0 * w[v] * diff * (0.5 if symmetric else 1.0)
            grads["W3"] += conv_weight_grad(dy, cch["h2"])
            dh2 = conv_adjoint(dy, p["W3"])
            da2 = dh2 * g2
            dg2 += dh2 * cch["a2"]
            grads["W2"] += conv_weight_grad(da2, cch["h1"])
            dh1 = conv_adjoint(da2, p["W2"])
            da1 = dh1 * g1
            dg1 += dh1 * cch["a1"]
            grads["W1"] += conv_weight_grad(da1, cch["u"])
            if symmetric:
                # the transpose path y' = conv^T(k1, W1): <dy, conv^T(k1, W1)>
                # = <conv(dy, W1), k1>, so dW1 = conv_weight_grad(k1, dy)
                grads["W1"] += conv_weight_grad(cct["k1"], dy)
                dk1 = conv(dy, p["W1"])
                db2 = dk1 * g1
                dg1 += dk1 * cct["b2"]
                grads["W2"] += conv_weight_grad(cct["k2"], db2)
                dk2 = conv(db2, p["W2"])
                db3 = dk2 * g2
                dg2 += dk2 * cct["b3"]
                grads["W3"] += conv_weight_grad(cct["u"], db3)
    dz1 = dg1 * g1 * (1.0 - g1)
    dz2 = dg2 * g2 * (1.0 - g2)
    grads["V1"] = conv_weight_grad(dz1, f)
    grads["c1"] = dz1.sum(axis=(1, 2, 3))
    grads["V2"] = conv_weight_grad(dz2, f)
    grads["c2"] = dz2.sum(axis=(1, 2, 3))
    return loss, grads


def _k2(kap):
    k2 = np.sum(np.abs(kap) ** 2, axis=0)
    return np.where(k2 > 0, k2, np.inf)   # 1 / inf = 0 on the null mode


def curl_h_scaled(r, kap):
    """K_A^H r / |k|^2 per mode."""
    ka = fourier.ka_matrix(kap)
    return fourier._per_mode(np.conj(np.swapaxes(ka, -1, -2)), r) / _k2(kap)


def curl_scaled(w, kap):
    """K_A w / |k|^2 per mode."""
    return fourier._per_mode(fourier.ka_matrix(kap), w) / _k2(kap)


def sandwich_precondition(r, kap, blocks, gamma):
    """T0 r (the curl-sandwich approximate inverse, module docstring); gamma a
    scalar or per-mode (N, N, N) coefficients."""
    eps = np.linalg.inv(blocks)
    e = fourier.f3(curl_h_scaled(r, kap))
    m = np.einsum("zyxij,...jzyx->...izyx", eps, e)
    longi = fourier._per_mode(fourier.kb_matrix(kap), r) / (gamma * _k2(kap) ** 2)
    return curl_scaled(fourier.f3h(m), kap) + longi


def precondition(p: dict, f: np.ndarray, r: np.ndarray, kap, gamma, blocks, symmetric: bool = False) -> np.ndarray:
    """T(r) = T0 r + K_A F3_3^H g(F3_3 K_A^H r / |k|^2) / |k|^2 (g_s with
    symmetric=True)."""
    e = fourier.f3(curl_h_scaled(r, kap))
    return sandwich_precondition(r, kap, blocks, gamma) + curl_scaled(fourier.f3h(forward(p, f, e, symmetric)), kap)


def training_pair(r: np.ndarray, e: np.ndarray, kap, gamma, blocks):
    """Network input U = F3_3 (K_A^H r / |k|^2), target T = F3_3 K_A^H (e - T0 r)
    and ||K_A^H e||^2 per vector."""
    ka = fourier.ka_matrix(kap)
    kah = np.conj(np.swapaxes(ka, -1, -2))
    U = fourier.f3(curl_h_scaled(r, kap))
    T = fourier.f3(fourier._per_mode(kah, e - sandwich_precondition(r, kap, blocks, gamma)))
    ce = fourier._per_mode(kah, e)
    en2 = np.sum(np.abs(ce) ** 2, axis=tuple(range(1, e.ndim)))
    return U, T, en2
