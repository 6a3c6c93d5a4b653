"""FP64 CPU oracle of the learned surrogate (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg may
import this module.  It shares no code with the CUDA path.

The surrogate is not part of arXiv 1910.01031's method: the paper forecasts
with the numerical scheme of Sec. 2.  It replaces k model steps of that
scheme in the drift forecast of Sec. 5.2, so what it computes is defined
here from its own specification:

* network f: `depth` periodic 3x3 convolutions, 3 -> width -> ... -> width
  -> 3 channels, SiLU(z) = z / (1 + exp(-z)) after every layer but the last;
* input  x = in_scale * U(t) per field (eta, hu, hv);
* output U(t + k dt) = U(t) + out_scale * f(x);
* training loss: mean over pixels and the 3 fields of
  (f(x) - (Y - X) / out_scale)^2 for a pair (X, Y);
* Adam (Kingma & Ba 2015) with bias correction, beta1 0.9, beta2 0.999,
  eps 1e-8.

Parameters are one flat FP32 vector, per layer l: weights [3][3][cout][cin]
with cin padded to 16 at l = 0 and cout padded to 16 at the last layer
(padding entries are zero and stay zero), then bias[cout].  Convolutions are
written as sums of shifted copies of the input (np.roll for the periodic
shift); the gradients are the adjoint of each step, written out by hand.
"""
from __future__ import annotations

import numpy as np


def layer_shapes(width: int, depth: int):
    """(cin, cout) per layer as stored (padded) and as used (real)."""
    stored = [(16 if l == 0 else width, 16 if l == depth - 1 else width) for l in range(depth)]
    real = [(3 if l == 0 else width, 3 if l == depth - 1 else width) for l in range(depth)]
    return stored, real


def n_params(width: int, depth: int) -> int:
    stored, _ = layer_shapes(width, depth)
    return sum(9 * ci * co + co for ci, co in stored)


def unpack(p, width: int, depth: int):
    """Flat parameters -> list of (W [3][3][cout][cin], b [cout]) restricted to
    the real channels (FP64)."""
    p = np.asarray(p, np.float64)
    stored, real = layer_shapes(width, depth)
    out, off = [], 0
    for (ci, co), (ri, ro) in zip(stored, real):
        W = p[off:off + 9 * ci * co].reshape(3, 3, co, ci)
        off += 9 * ci * co
        b = p[off:off + co]
        off += co
        out.append((W[:, :, :ro, :ri].copy(), b[:ro].copy()))
    assert off == p.size
    return out


def pack(layers, width: int, depth: int):
    """Inverse of unpack (zeros in the padding)."""
    stored, real = layer_shapes(width, depth)
    parts = []
    for (W, b), (ci, co), (ri, ro) in zip(layers, stored, real):
        Wp = np.zeros((3, 3, co, ci))
        Wp[:, :, :ro, :ri] = W
        bp = np.zeros(co)
        bp[:ro] = b
        parts += [Wp.ravel(), bp]
    return np.concatenate(parts)


def shift(x, dy: int, dx: int):
    """s[..., y, x] = x[..., (y + dy) mod ny, (x + dx) mod nx]."""
    return np.roll(x, (-dy, -dx), axis=(-2, -1))


def conv3x3(x, W, b):
    """out[n, co, y, x] = b[co] + sum_{ky, kx, ci} W[ky, kx, co, ci]
    x[n, ci, y + ky - 1, x + kx - 1] (indices periodic); x [n][ci][ny][nx]."""
    out = np.zeros((x.shape[0], W.shape[2]) + x.shape[2:])
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("oc,ncyx->noyx", W[ky, kx], shift(x, ky - 1, kx - 1))
    return out + b[None, :, None, None]


def conv3x3_adjoint(g, W):
    """Adjoint of conv3x3 in its input: dx[n, ci, q] = sum_{ky, kx, co}
    W[ky, kx, co, ci] g[n, co, q - (ky - 1, kx - 1)]."""
    out = np.zeros((g.shape[0], W.shape[3]) + g.shape[2:])
    for ky in range(3):
        for kx in range(3):
            out += np.einsum("oc,noyx->ncyx", W[ky, kx], shift(g, 1 - ky, 1 - kx))
    return out


def conv3x3_wgrad(g, x):
    """dW[ky, kx, co, ci] = sum_{n, y, x} g[n, co, y, x] x[n, ci, y + ky - 1, x + kx - 1]."""
    dW = np.zeros((3, 3, g.shape[1], x.shape[1]))
    for ky in range(3):
        for kx in range(3):
            dW[ky, kx] = np.einsum("noyx,ncyx->oc", g, shift(x, ky - 1, kx - 1))
    return dW


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def net(p, x, width: int, depth: int, keep=False):
    """f(x) for x [n][3][ny][nx] (already scaled); with keep, also the
    pre-activations z_l and inputs a_l of every layer."""
    layers = unpack(p, width, depth)
    a, zs, ins = np.asarray(x, np.float64), [], []
    for l, (W, b) in enumerate(layers):
        ins.append(a)
        z = conv3x3(a, W, b)
        zs.append(z)
        a = silu(z) if l + 1 < depth else z
    return (a, zs, ins) if keep else a


def apply(p, U, in_scale, out_scale, width: int, depth: int):
    """U(t + k dt) = U + out_scale f(in_scale U) for U [n][3][ny][nx]."""
    U = np.asarray(U, np.float64)
    si = np.asarray(in_scale, np.float64)[None, :, None, None]
    so = np.asarray(out_scale, np.float64)[None, :, None, None]
    return U + so * net(p, si * U, width, depth)


def loss(p, X, Y, in_scale, out_scale, width: int, depth: int) -> float:
    X, Y = np.asarray(X, np.float64), np.asarray(Y, np.float64)
    si = np.asarray(in_scale, np.float64)[None, :, None, None]
    so = np.asarray(out_scale, np.float64)[None, :, None, None]
    r = net(p, si * X, width, depth) - (Y - X) / so
    return float(np.mean(r * r))


def loss_grad(p, X, Y, in_scale, out_scale, width: int, depth: int):
    """(loss, dloss/dp in the flat padded layout) by reverse-mode steps."""
    X, Y = np.asarray(X, np.float64), np.asarray(Y, np.float64)
    si = np.asarray(in_scale, np.float64)[None, :, None, None]
    so = np.asarray(out_scale, np.float64)[None, :, None, None]
    layers = unpack(p, width, depth)
    out, zs, ins = net(p, si * X, width, depth, keep=True)
    r = out - (Y - X) / so
    L = float(np.mean(r * r))
    g = 2.0 * r / r.size                 # dL/dout
    grads = [None] * depth
    for l in range(depth - 1, -1, -1):
        if l + 1 < depth:
            g = g * dsilu(zs[l])         # through the activation of layer l
        W, _ = layers[l]
        grads[l] = (conv3x3_wgrad(g, ins[l]), g.sum(axis=(0, 2, 3)))
        if l > 0:
            g = conv3x3_adjoint(g, W)
    return L, pack(grads, width, depth)


def adam(p, g, m, v, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1): returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
