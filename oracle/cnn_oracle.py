"""Plain FP64 NumPy oracle of the learned preconditioner (TEST INFRASTRUCTURE
ONLY: imported by tests/ and bench.py's baseline leg, never by the product).

What it computes (the C ABI documents the same for bsc_cnn_*):

* Matrix features per control point alpha (32 channels): the diagonal 3x3
  block K_aa / d (six entries: 00 01 02 11 12 22), the traces of the 24
  off-diagonal blocks K_a,a+(du,dv) / d in slot order, the pin mask and 1,
  with d = mean diagonal entry of K over unpinned points.
* A network of four 3x3 convolutions with zero padding on the nu x nv grid
  (channels 32 -> 32 -> 32 -> 32 -> 16), ReLU after the first three; its
  first nine output channels o_t give the tap coefficients
      a_t(alpha) = RHO o_t / (1 + sum_s |o_s|),   RHO = 1/2,
  t = 3 (dy+1) + (dx+1) for the neighbour (i + dx, j + dy).  The bound
  sum_t |a_t| < RHO keeps B within RHO of the identity in the infinity norm,
  so B is invertible and cond(B^T B) <= ((1 + RHO) / (1 - RHO))^2 = 9 for any
  weights: training cannot reach a nearly singular preconditioner.
* The preconditioner M = P L^-T B^T B L^-1 P with D_aa = L_a L_a^T the
  Cholesky factor of every diagonal block, (B y)(alpha) = y(alpha) + sum_t
  a_t(alpha) y(alpha + off_t) (the same for the three components, zero
  outside the grid) and P zeroing the pinned entries; z = M r.  M is
  symmetric positive semidefinite for every a, and a = 0 gives the
  block-Jacobi preconditioner D^-1 (on the unpinned entries).
* The loss of a pair (r = K x, x): L = (z - x)^T K (z - x) / (x^T K x).
* Its gradient by hand-written backpropagation through M and the network;
  the tests pin it against central finite differences.

Arrays: vectors are (N, 3) (alpha = j nu + i), K is the oracle's stencil
(N, 25, 3, 3), parameters one flat float vector in the C ABI's order (per
layer W[dy][dx][ci][co], then b[co]).  With bf16_like=True every tensor the
GPU stores in BF16 (features, layer outputs, back-propagated gradients) is
rounded to BF16 at the same point.
"""
from __future__ import annotations

import numpy as np

CH_IN = (32, 32, 32, 32)
CH_OUT = (32, 32, 32, 16)
TAPS = 9
RHO = 0.5


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
            # the input pixel (j, i) feeds the outputs (j - dy + 1, i - dx + 1)
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


def shift(y, nu, nv, dx, dy):
    """(S y)(j, i) = y(j + dy, i + dx), zero outside.  y: (N, c)."""
    Y = y.reshape(nv, nu, -1)
    out = np.zeros_like(Y)
    js, je = max(0, -dy), nv - max(0, dy)
    is_, ie = max(0, -dx), nu - max(0, dx)
    out[js:je, is_:ie] = Y[js + dy:je + dy, is_ + dx:ie + dx]
    return out.reshape(y.shape)


def taps():
    return [(t % 3 - 1, t // 3 - 1) for t in range(TAPS)]   # (dx, dy) of tap t


class Prepared:
    """The matrix-dependent part: features, block Cholesky factors, the scale d."""

    def __init__(self, nu, nv, K, pinned_mask):
        self.nu, self.nv = nu, nv
        K = np.asarray(K, dtype=np.float64).reshape(nu * nv, 25, 3, 3)
        self.K = K
        self.diag = K[:, 12]
        self.pin = np.asarray(pinned_mask, dtype=bool).reshape(-1)
        tr = np.trace(self.diag, axis1=1, axis2=2)[~self.pin]
        self.d = float(tr.sum() / (3 * tr.size)) if tr.size else 1.0
        self.L = np.linalg.cholesky(self.diag)
        self.Linv = np.linalg.inv(self.L)

    def features(self):
        N = self.nu * self.nv
        f = np.zeros((N, 32))
        g = self.diag / self.d
        f[:, 0], f[:, 1], f[:, 2] = g[:, 0, 0], g[:, 0, 1], g[:, 0, 2]
        f[:, 3], f[:, 4], f[:, 5] = g[:, 1, 1], g[:, 1, 2], g[:, 2, 2]
        k = 6
        for slot in range(25):
            if slot == 12:
                continue
            f[:, k] = np.trace(self.K[:, slot], axis1=1, axis2=2) / self.d
            k += 1
        f[:, 30] = self.pin.astype(np.float64)
        f[:, 31] = 1.0
        return f

    def matvec(self, x):
        from oracle import stencil_matvec
        return stencil_matvec(self.nu, self.nv, self.K, x)


def network(params, prep: Prepared, bf16_like=False):
    """Tap coefficients a (N, 9) and the cache of the forward pass."""
    layers = unpack(params)
    X = _maybe(prep.features(), bf16_like).reshape(prep.nv, prep.nu, 32)
    acts = [X]
    for l, (W, b) in enumerate(layers):
        Y = conv3x3(acts[-1], _maybe(W, bf16_like), b)
        if l < 3:
            Y = _maybe(np.maximum(Y, 0.0), bf16_like)
        acts.append(Y)
    o = acts[-1].reshape(-1, 16)[:, :TAPS]
    a = bound_taps(o)
    return a, {"acts": acts, "layers": layers, "o": o}


def bound_taps(o):
    return RHO * o / (1.0 + np.abs(o).sum(axis=1, keepdims=True))


def bound_taps_backward(o, da):
    """d/do of sum_t da_t a_t(o) with a_t = RHO o_t / S, S = 1 + sum |o|."""
    S = 1.0 + np.abs(o).sum(axis=1, keepdims=True)
    return RHO * (da / S - np.sign(o) * np.sum(da * o, axis=1, keepdims=True) / S ** 2)


def apply_B(a, y, nu, nv):
    u = y.copy()
    for t, (dx, dy) in enumerate(taps()):
        u += a[:, t:t + 1] * shift(y, nu, nv, dx, dy)
    return u


def apply_BT(a, u, nu, nv):
    v = u.copy()
    for t, (dx, dy) in enumerate(taps()):
        v += shift(a[:, t:t + 1] * u, nu, nv, -dx, -dy)
    return v


def precondition(a, prep: Prepared, r):
    """z = M r with M = P L^-T B^T B L^-1 P, P zeroing the pinned entries; also (y, u, v)."""
    r = np.array(r, dtype=np.float64).reshape(-1, 3)
    r[prep.pin] = 0.0
    y = np.einsum("nab,nb->na", prep.Linv, r)
    u = apply_B(a, y, prep.nu, prep.nv)
    v = apply_BT(a, u, prep.nu, prep.nv)
    z = np.einsum("nba,nb->na", prep.Linv, v)
    z[prep.pin] = 0.0
    return z, (y, u, v)


def forward(params, prep: Prepared, r, bf16_like=False):
    a, cache = network(params, prep, bf16_like)
    z, yuv = precondition(a, prep, r)
    cache["a"], cache["yuv"] = a, yuv
    return z, cache


def loss(params, prep: Prepared, r, xstar, bf16_like=False):
    z, _ = forward(params, prep, r, bf16_like)
    xs = np.asarray(xstar, dtype=np.float64).reshape(-1, 3)
    e = z - xs
    return float(np.sum(e * prep.matvec(e)) / np.sum(xs * prep.matvec(xs)))


def tap_gradient(a, prep, yuv, g):
    """dL/da (N, 9) from dL/dz = g through z = L^-T B^T B L^-1 r."""
    y, u, _ = yuv
    nu, nv = prep.nu, prep.nv
    g = g.copy()
    g[prep.pin] = 0.0
    gv = np.einsum("nab,nb->na", prep.Linv, g)        # v -> z = L^-T v
    gu = apply_B(a, gv, nu, nv)                        # u -> v = B^T u
    da = np.zeros((nu * nv, TAPS))
    for t, (dx, dy) in enumerate(taps()):
        # u = y + sum a_t S_t y  and  v = u + sum S_-t (a_t u)
        da[:, t] = np.sum(gu * shift(y, nu, nv, dx, dy), axis=1) + np.sum(u * shift(gv, nu, nv, dx, dy), axis=1)
    return da


def loss_and_grad(params, prep: Prepared, r, xstar, bf16_like=False):
    """L and dL/dparams (flat, the C ABI's order), by hand-written backprop."""
    z, cache = forward(params, prep, r, bf16_like)
    xs = np.asarray(xstar, dtype=np.float64).reshape(-1, 3)
    e = z - xs
    Ke = prep.matvec(e)
    xKx = float(np.sum(xs * prep.matvec(xs)))
    L = float(np.sum(e * Ke) / xKx)
    g = 2.0 * Ke / xKx                                  # dL/dz (K symmetric)
    da = tap_gradient(cache["a"], prep, cache["yuv"], g)
    dy = np.zeros((prep.nu * prep.nv, 16))
    dy[:, :TAPS] = bound_taps_backward(cache["o"], da)
    G = _maybe(dy, bf16_like).reshape(prep.nv, prep.nu, 16)
    acts, layers = cache["acts"], cache["layers"]
    grads = [None] * 4
    for l in range(3, -1, -1):
        grads[l] = conv3x3_wgrad(acts[l], G)
        if l > 0:
            G = conv3x3_adjoint(G, _maybe(layers[l][0], bf16_like)) * (acts[l] > 0.0)
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
