"""Pins of the learned preconditioner's oracle (oracle/cnn_oracle.py) against
what does not come from it: an independent 2-D correlation (scipy), the
adjoint identity, central finite differences of the loss, the block-Jacobi
limit of zero weights, symmetry, positive semidefiniteness and linearity of
the preconditioner, and BF16 rounding of exactly representable halfway
cases."""
import numpy as np
import pytest

import oracle
from oracle import cnn_oracle as co
from paper_2506_18867_gb300 import inputs


def test_conv_matches_scipy_correlation():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(1)
    X = rng.standard_normal((6, 9, 3))
    W = rng.standard_normal((3, 3, 3, 4))
    b = rng.standard_normal(4)
    Y = co.conv3x3(X, W, b)
    for d in range(4):
        ref = b[d] + sum(signal.correlate2d(X[:, :, c], W[:, :, c, d], mode="same", boundary="fill")
                         for c in range(3))
        np.testing.assert_allclose(Y[:, :, d], ref, rtol=1e-13, atol=1e-13)


def test_adjoint_and_weight_gradient_identities():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((5, 7, 4))
    W = rng.standard_normal((3, 3, 4, 6))
    G = rng.standard_normal((5, 7, 6))
    V = rng.standard_normal(W.shape)
    lhs = np.sum(co.conv3x3(X, W) * G)
    assert lhs == pytest.approx(np.sum(X * co.conv3x3_adjoint(G, W)), rel=1e-13)
    dW, db = co.conv3x3_wgrad(X, G)
    # <conv(X, V), G> is linear in V: its derivative is the weight gradient
    assert np.sum(co.conv3x3(X, V) * G) == pytest.approx(np.sum(dW * V), rel=1e-13)
    np.testing.assert_allclose(db, G.sum(axis=(0, 1)))


def small_system(seed=3, nu=7, nv=6, noise=0.05):
    pat = inputs.config_random_small(seed, nu, nv, noise=noise)
    prob = oracle.Problem.from_patch(pat)
    sc = oracle.Scene.from_patch(pat, project=True)
    _, g, K = oracle.evaluate(prob, sc, pat.C, pat.Chat)
    pin = np.zeros(pat.n_cp, dtype=bool)
    pin[pat.pinned] = True
    prep = co.Prepared(pat.nu, pat.nv, K, pin)
    r = -g
    xs = oracle.solve_banded(pat.nu, pat.nv, K, r)
    return pat, prep, r, xs


def random_params(seed, scale=0.1):
    rng = np.random.default_rng(seed)
    p = np.zeros(co.param_count())
    for ws, shape, bs in co.param_layout():
        fan_in = 9 * shape[2]
        p[ws] = rng.standard_normal(int(np.prod(shape))) * scale * np.sqrt(2.0 / fan_in)
        p[bs] = rng.standard_normal(bs.stop - bs.start) * 0.01
    return p


def test_backprop_matches_finite_differences():
    _, prep, r, xs = small_system()
    params = random_params(4, scale=0.5)
    L, g = co.loss_and_grad(params, prep, r, xs)
    rng = np.random.default_rng(5)
    idx = []
    for ws, _, bs in co.param_layout():
        idx += list(rng.integers(ws.start, ws.stop, 6)) + [bs.start, bs.stop - 1]
    fd = co.fd_grad(params, prep, r, xs, idx, h=1e-6)
    np.testing.assert_allclose(g[idx], fd, rtol=2e-6, atol=1e-9 * np.abs(g).max())
    assert L > 0


def test_zero_weights_give_block_jacobi_and_pins():
    pat, prep, r, _ = small_system(6)
    z, _ = co.forward(np.zeros(co.param_count()), prep, r)
    ref = np.einsum("nab,nb->na", np.linalg.inv(prep.diag), r)
    ref[prep.pin] = 0.0
    np.testing.assert_allclose(z, ref, rtol=1e-12, atol=1e-300)
    assert np.all(z[pat.pinned] == 0.0)


def test_preconditioner_is_symmetric_psd_and_linear():
    """For arbitrary tap coefficients M = L^-T B^T B L^-1 (pins projected out)
    is symmetric and positive semidefinite, and z depends linearly on r."""
    pat, prep, r, _ = small_system(7)
    rng = np.random.default_rng(11)
    a = rng.standard_normal((pat.n_cp, co.TAPS)) * 0.4
    x = rng.standard_normal((pat.n_cp, 3))
    y = rng.standard_normal((pat.n_cp, 3))
    x[prep.pin] = 0.0
    y[prep.pin] = 0.0
    Mx, _ = co.precondition(a, prep, x)
    My, _ = co.precondition(a, prep, y)
    assert np.sum(y * Mx) == pytest.approx(np.sum(x * My), rel=1e-12)
    assert np.sum(x * Mx) > 0.0
    Mxy, _ = co.precondition(a, prep, 2.5 * x - 3.0 * y)
    np.testing.assert_allclose(Mxy, 2.5 * Mx - 3.0 * My, rtol=1e-12, atol=1e-12 * np.abs(Mxy).max())
    # dense check on this small grid: M assembled column by column is SPD-semidefinite
    N3 = 3 * pat.n_cp
    cols = []
    for k in range(N3):
        e = np.zeros(N3)
        e[k] = 1.0
        cols.append(co.precondition(a, prep, e.reshape(-1, 3))[0].ravel())
    M = np.array(cols).T
    np.testing.assert_allclose(M, M.T, atol=1e-12 * np.abs(M).max())
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > -1e-12 * np.abs(M).max()


def test_tap_gradient_matches_finite_differences():
    """dL/da through z = M(a) r (the first stage of the backward pass)."""
    pat, prep, r, xs = small_system(12)
    rng = np.random.default_rng(13)
    a = rng.standard_normal((pat.n_cp, co.TAPS)) * 0.2
    x = xs
    Kx = prep.matvec(x)

    def L_of(aa):
        z, _ = co.precondition(aa, prep, Kx)
        e = z - x
        return np.sum(e * prep.matvec(e)) / np.sum(x * Kx)

    z, yuv = co.precondition(a, prep, Kx)
    g = 2.0 * prep.matvec(z - x) / np.sum(x * Kx)
    da = co.tap_gradient(a, prep, yuv, g)
    h = 1e-6
    for p, t in [(0, 4), (5, 0), (17, 8), (pat.n_cp - 1, 3), (20, 5)]:
        a1, a2 = a.copy(), a.copy()
        a1[p, t] += h
        a2[p, t] -= h
        fd = (L_of(a1) - L_of(a2)) / (2 * h)
        assert da[p, t] == pytest.approx(fd, rel=1e-5, abs=1e-10)


def test_tap_bound():
    """sum_t |a_t| < 1/2 for any network output, and the bound's derivative
    matches finite differences."""
    rng = np.random.default_rng(14)
    o = rng.standard_normal((50, co.TAPS)) * 10.0
    assert np.all(np.abs(co.bound_taps(o)).sum(axis=1) < co.RHO)
    da = rng.standard_normal((50, co.TAPS))
    g = co.bound_taps_backward(o, da)
    h = 1e-6
    for p, t in [(0, 0), (7, 4), (49, 8)]:
        o1, o2 = o.copy(), o.copy()
        o1[p, t] += h
        o2[p, t] -= h
        fd = (np.sum(da * co.bound_taps(o1)) - np.sum(da * co.bound_taps(o2))) / (2 * h)
        assert g[p, t] == pytest.approx(fd, rel=1e-6)


def test_loss_is_one_for_zero_preconditioner_output():
    """z = 0 gives L = 1 (from the definition)."""
    _, prep, r, xs = small_system(9)
    e = -xs
    assert np.sum(e * prep.matvec(e)) / np.sum(xs * prep.matvec(xs)) == pytest.approx(1.0)


def test_bf16_rounding_halfway_cases():
    one = 1.0
    assert co.bf16(one) == 1.0
    assert co.bf16(one + 2.0 ** -8) == 1.0                      # halfway, ties to even (down)
    assert co.bf16(one + 3 * 2.0 ** -8) == one + 2.0 ** -6      # halfway, ties to even (up)
    assert co.bf16(one + 2.0 ** -8 + 2.0 ** -20) == one + 2.0 ** -7
    assert co.bf16(-3.0) == -3.0
    x = np.random.default_rng(0).standard_normal(1000)
    assert np.all(np.abs(co.bf16(x) - x) <= 2.0 ** -8 * np.abs(x) + 1e-300)
