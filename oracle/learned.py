"""Learned preconditioner correction (oracle; test infrastructure only).

The paper has no learned component.  This module defines the small network
that corrects the FFT-diagonal preconditioner K_P^{-1} (Sec. 2.4, eqs.
matrixfree_diagP / matrixfree_finalform), in plain numpy FP64:

    T(r) = K_P^{-1} r + F3_3^H g(F3_3 K_P^{-1} r)

with F3_3 the unitary 3D DFT of every component (Sec. 2.4; x = F3_3^H H is
the Fourier basis, so F3_3 maps back to the real-space grid) and g a
three-layer circular 3D convolution net on the real-space field whose hidden
channels are gated by the per-cell permittivity blocks M (Sec. 3.2.1):

    f      = the 9 reals of the cell block of M: d1, d2, d3,
             Re/Im M_12, Re/Im M_13, Re/Im M_23            (9 x N^3)
    g1     = sigmoid(conv(f, V1) + c1)                      (C x N^3)
    g2     = sigmoid(conv(f, V2) + c2)
    a1     = conv(u, W1),  h1 = a1 * g1                     (3 -> C)
    a2     = conv(h1, W2), h2 = a2 * g2                     (C -> C)
    y      = conv(h2, W3)                                   (C -> 3)

The net is linear in u for a fixed structure, and it acts on the real and
imaginary parts of the complex field with the same weights, so T is a
complex-linear map.  conv is a cross-correlation with 3 x 3 x 3 taps and
periodic wrap-around:  conv(x, w)[o, z, y, x] =
sum_{i, dz, dy, dx} w[o, i, dz+1, dy+1, dx+1] x[i, z+dz, y+dy, x+dx].

Training target: e = Op^{-1} r (Op the compensated operator of eq.
matrixfree_kcform), the ideal preconditioner for the smallest eigenvalues;
loss = sum_v w_v ||T(r_v) - e_v||^2, evaluated in real space (F3_3 is
unitary) as sum_v w_v ||y_v - F3_3 (e_v - K_P^{-1} r_v)||^2.

Parameters are one flat vector in the order W1, W2, W3, V1, c1, V2, c2, each
in C order (param_shapes).
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


def forward(p: dict, f: np.ndarray, U: np.ndarray) -> np.ndarray:
    """Complex field U (..., 3, N, N, N): g(Re U) + i g(Im U)."""
    g = gates(p, f)
    flat = U.reshape((-1,) + U.shape[-4:])
    out = np.empty(flat.shape, dtype=np.complex128)
    for v in range(flat.shape[0]):
        yr, _ = forward_real(p, f, flat[v].real, g)
        yi, _ = forward_real(p, f, flat[v].imag, g)
        out[v] = yr + 1j * yi
    return out.reshape(U.shape)


def loss_and_grad(p: dict, f: np.ndarray, U: np.ndarray, T: np.ndarray, w: np.ndarray):
    """L = sum_v w_v ||g(U_v) - T_v||^2 over complex samples (nvec, 3, N, N, N)
    and dL/dparams (dict), by the chain rule through every layer."""
    g1, g2 = gates(p, f)
    grads = {name: np.zeros(shape) for name, shape in param_shapes(p["W1"].shape[0])}
    dg1 = np.zeros_like(g1)
    dg2 = np.zeros_like(g2)
    loss = 0.0
    for v in range(U.shape[0]):
        for part in (np.real, np.imag):
            y, cch = forward_real(p, f, part(U[v]), (g1, g2))
            diff = y - part(T[v])
            loss += w[v] * np.sum(diff ** 2)
            dy = 2.0 * w[v] * diff
            grads["W3"] += conv_weight_grad(dy, cch["h2"])
            dh2 = conv_adjoint(dy, p["W3"])
            da2 = dh2 * g2
            dg2 += dh2 * cch["a2"]
            grads["W2"] += conv_weight_grad(da2, cch["h1"])
            dh1 = conv_adjoint(da2, p["W2"])
            da1 = dh1 * g1
            dg1 += dh1 * cch["a1"]
            grads["W1"] += conv_weight_grad(da1, cch["u"])
    dz1 = dg1 * g1 * (1.0 - g1)
    dz2 = dg2 * g2 * (1.0 - g2)
    grads["V1"] = conv_weight_grad(dz1, f)
    grads["c1"] = dz1.sum(axis=(1, 2, 3))
    grads["V2"] = conv_weight_grad(dz2, f)
    grads["c2"] = dz2.sum(axis=(1, 2, 3))
    return loss, grads


def precondition(p: dict, f: np.ndarray, r: np.ndarray, kap, gamma) -> np.ndarray:
    """T(r) = K_P^{-1} r + F3_3^H g(F3_3 K_P^{-1} r), r in the Fourier basis."""
    base = fourier.precondition(r, kap, gamma)
    return base + fourier.f3h(forward(p, f, fourier.f3(base)))


def training_pair(r: np.ndarray, e: np.ndarray, kap, gamma):
    """Real-space network input U = F3_3 K_P^{-1} r, target T = F3_3 (e - K_P^{-1} r)
    and ||e||^2 per vector."""
    base = fourier.precondition(r, kap, gamma)
    U = fourier.f3(base)
    T = fourier.f3(e - base)
    en2 = np.sum(np.abs(e) ** 2, axis=tuple(range(1, e.ndim)))
    return U, T, en2
