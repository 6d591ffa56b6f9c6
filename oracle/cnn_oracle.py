"""Plain FP64 NumPy oracle of the learned preconditioner (TEST INFRASTRUCTURE
ONLY: imported by tests/ and bench.py's baseline leg, never by the product).

The network is the one the C ABI documents for bsc_cnn_*: four 3x3
convolutions with zero padding on the nu x nv control grid (channels
16 -> 32 -> 32 -> 32 -> 16), ReLU after the first three, input features

    r / s,  (D^-1 r) d / s,  diagonal 3x3 block of K / d (6 entries),  pin,  1

with s = RMS of r and d = mean diagonal entry of K over unpinned points, and
the preconditioned vector z = D^-1 r + (s / d) y (y = output channels 0..2,
zero at pinned points).  The loss is the energy-norm error of z against the
exact solve x* = K^-1 r, L = (z - x*)^T K (z - x*) / (x*^T K x*).  The
backward pass below is written out by hand (chain rule through the combine,
the convolutions and the ReLUs); the tests pin it against central finite
differences of the loss.

Arrays: r, z, x* are (N, 3) (control point alpha = j nu + i); K is the
oracle's stencil (N, 25, 3, 3); parameters are one flat float vector in the
C ABI's order (per layer W[dy][dx][ci][co], then b[co]).

With bf16=True every tensor the GPU stores in BF16 (features, layer outputs,
back-propagated gradients) is rounded to BF16 (round to nearest even) at the
same point, so that GPU and oracle differ only by FP32 accumulation order.
"""
from __future__ import annotations

import numpy as np

CH_IN = (16, 32, 32, 32)
CH_OUT = (32, 32, 32, 16)


def param_layout():
    """[(W slice, W shape, b slice)] per layer in the flat parameter vector."""
    out, o = [], 0
    for ci, co in zip(CH_IN, CH_OUT):
        nw = 9 * ci * co
        out.append((slice(o, o + nw), (3, 3, ci, co), slice(o + nw, o + nw + co)))
        o += nw + co
    return out


def param_count():
    return sum(9 * ci * co + co for ci, co in zip(CH_IN, CH_OUT))


def unpack(params):
    params = np.asarray(params, dtype=np.float64)
    return [(params[ws].reshape(shape), params[bs]) for ws, shape, bs in param_layout()]


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return (u.astype(np.uint32)).view(np.float32).astype(np.float64)


def _maybe(x, on):
    return bf16(x) if on else x


def conv3x3(X, W, b=None):
    """Y[j, i, co] = b[co] + sum_{dy, dx, ci} X[j + dy, i + dx, ci] W[dy + 1, dx + 1, ci, co],
    X outside the grid = 0.  X: (nv, nu, ci)."""
    nv, nu, _ = X.shape
    Xp = np.zeros((nv + 2, nu + 2, X.shape[2]))
    Xp[1:-1, 1:-1] = X
    Y = np.zeros((nv, nu, W.shape[3]))
    for dy in range(3):
        for dx in range(3):
            Y += np.einsum("jic,cd->jid", Xp[dy:dy + nv, dx:dx + nu], W[dy, dx])
    if b is not None:
        Y += b
    return Y


def conv3x3_adjoint(G, W):
    """Adjoint of conv3x3 (without bias) w.r.t. its input: dX[j, i, ci] =
    sum_{dy, dx, co} G[j - dy, i - dx, co] W[dy + 1, dx + 1, ci, co]."""
    nv, nu, _ = G.shape
    Gp = np.zeros((nv + 2, nu + 2, G.shape[2]))
    Gp[1:-1, 1:-1] = G
    dX = np.zeros((nv, nu, W.shape[2]))
    for dy in range(3):
        for dx in range(3):
            # output pixel (j, i) received X[j + dy - 1, i + dx - 1]: the input
            # pixel (j, i) feeds the outputs (j - dy + 1, i - dx + 1)
            dX += np.einsum("jid,cd->jic", Gp[2 - dy:2 - dy + nv, 2 - dx:2 - dx + nu], W[dy, dx])
    return dX


def conv3x3_wgrad(X, G):
    """dW[dy, dx, ci, co] = sum_{j, i} X[j + dy - 1, i + dx - 1, ci] G[j, i, co]; db = sum G."""
    nv, nu, _ = X.shape
    Xp = np.zeros((nv + 2, nu + 2, X.shape[2]))
    Xp[1:-1, 1:-1] = X
    dW = np.zeros((3, 3, X.shape[2], G.shape[2]))
    for dy in range(3):
        for dx in range(3):
            dW[dy, dx] = np.einsum("jic,jid->cd", Xp[dy:dy + nv, dx:dx + nu], G)
    return dW, G.sum(axis=(0, 1))


class Prepared:
    """The matrix-dependent part: diagonal blocks, their inverses, the scale d."""

    def __init__(self, nu, nv, K, pinned_mask):
        self.nu, self.nv = nu, nv
        K = np.asarray(K, dtype=np.float64).reshape(nu * nv, 25, 3, 3)
        self.K = K
        self.diag = K[:, 12]
        self.Dinv = np.linalg.inv(self.diag)
        self.pin = np.asarray(pinned_mask, dtype=bool).reshape(-1)
        tr = np.trace(self.diag, axis1=1, axis2=2)[~self.pin]
        self.d = float(tr.sum() / (3 * tr.size)) if tr.size else 1.0

    def features(self, r):
        r = np.asarray(r, dtype=np.float64).reshape(-1, 3)
        s = float(np.sqrt((r * r).sum() / r.size))
        iS = 1.0 / s if s > 0 else 0.0
        Dr = np.einsum("nab,nb->na", self.Dinv, r)
        f = np.zeros((r.shape[0], 16))
        f[:, 0:3] = r * iS
        f[:, 3:6] = Dr * self.d * iS
        g = self.diag / self.d
        f[:, 6], f[:, 7], f[:, 8] = g[:, 0, 0], g[:, 0, 1], g[:, 0, 2]
        f[:, 9], f[:, 10], f[:, 11] = g[:, 1, 1], g[:, 1, 2], g[:, 2, 2]
        f[:, 12] = self.pin.astype(np.float64)
        f[:, 13] = 1.0
        return f, s, Dr

    def matvec(self, x):
        from oracle import stencil_matvec
        return stencil_matvec(self.nu, self.nv, self.K, x)


def forward(params, prep: Prepared, r, bf16_like=False):
    """z = P(r) and the cache of the forward pass."""
    layers = unpack(params)
    f, s, Dr = prep.features(r)
    X = _maybe(f, bf16_like).reshape(prep.nv, prep.nu, 16)
    acts = [X]
    for l, (W, b) in enumerate(layers):
        Wl = _maybe(W, bf16_like)
        Y = conv3x3(acts[-1], Wl, b)
        if l < 3:
            Y = _maybe(np.maximum(Y, 0.0), bf16_like)
        acts.append(Y)
    y = acts[-1].reshape(-1, 16)[:, :3]
    z = Dr + (s / prep.d) * y
    z[prep.pin] = 0.0
    return z, {"acts": acts, "s": s, "Dr": Dr, "layers": layers}


def loss(params, prep: Prepared, r, xstar, bf16_like=False):
    z, _ = forward(params, prep, r, bf16_like)
    xs = np.asarray(xstar, dtype=np.float64).reshape(-1, 3)
    e = z - xs
    return float(np.sum(e * prep.matvec(e)) / np.sum(xs * prep.matvec(xs)))


def loss_and_grad(params, prep: Prepared, r, xstar, bf16_like=False):
    """L and dL/dparams (flat, the C ABI's order), by hand-written backprop."""
    z, cache = forward(params, prep, r, bf16_like)
    xs = np.asarray(xstar, dtype=np.float64).reshape(-1, 3)
    e = z - xs
    Ke = prep.matvec(e)
    xKx = float(np.sum(xs * prep.matvec(xs)))
    L = float(np.sum(e * Ke) / xKx)
    dz = 2.0 * Ke / xKx                       # dL/dz (K symmetric)
    dz[prep.pin] = 0.0
    dy = np.zeros((prep.nu * prep.nv, 16))
    dy[:, :3] = (cache["s"] / prep.d) * dz    # z = Dr + (s/d) y
    G = _maybe(dy, bf16_like).reshape(prep.nv, prep.nu, 16)
    acts, layers = cache["acts"], cache["layers"]
    grads = [None] * 4
    for l in range(3, -1, -1):
        dW, db = conv3x3_wgrad(acts[l], G)
        grads[l] = (dW, db)
        if l > 0:
            Wl = _maybe(layers[l][0], bf16_like)
            G = conv3x3_adjoint(G, Wl) * (acts[l] > 0.0)   # through the ReLU of layer l's input
            G = _maybe(G, bf16_like)
    flat = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])
    return L, flat


def fd_grad(params, prep, r, xstar, idx, h=1e-6):
    """Central finite differences of the loss at parameter indices idx."""
    out = []
    for k in idx:
        p1 = np.array(params, dtype=np.float64)
        p2 = p1.copy()
        p1[k] += h
        p2[k] -= h
        out.append((loss(p1, prep, r, xstar) - loss(p2, prep, r, xstar)) / (2 * h))
    return np.array(out)
