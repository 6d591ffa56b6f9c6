"""Learned preconditioner on the GPU against the FP64 NumPy oracle
(oracle/cnn_oracle.py), through the C ABI.

The GPU keeps features, activations and back-propagated gradients in BF16
and accumulates in FP32 on the tensor cores; the oracle is run with the same
BF16 rounding points (bf16_like=True), so the two differ only by FP32
accumulation order and the BF16 rounding flips it causes (2^-8 relative on
a flipped element), and the ReLU masks those flips can change.  Measured
norm-wise errors on the 40 x 23 system: at most 2e-5 on layer outputs, taps
and z, 2e-5 on the loss, 4e-5 on the weight and bias gradients of layers 3
and 4 and 5.5e-4 on those of layers 1 and 2, which sit two and three BF16
back-propagation steps deep.  Bounds: 3e-3 on layers, taps and z, 1e-3 on
the loss and on the gradients of layers 3 and 4, 2e-3 on those of layers 1
and 2.

The systems are seeded synthetic SPD matrices in the stencil layout
(inputs.synthetic_stencil), x* seeded normal and r = K x* from the oracle's
stencil product: no input of the oracle comes from the GPU.  Grids: 40 x 23
(920 pixels: seven full 128-pixel tiles and a ragged tail of 24) and the
training size 512 x 512 (2048 tiles).
"""
import numpy as np
import pytest

import oracle
from oracle import cnn_oracle as co
from paper_2506_18867_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2506_18867_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2506_18867_gb300 import bsc  # noqa: E402

B_LAYER, B_GRAD = 3e-3, 1e-3
B_GRAD_LAYER = (2e-3, 2e-3, 1e-3, 1e-3)   # per layer: the first two are deeper in the BF16 backward pass


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def random_params(seed, scale=1.0, last_scale=1.0):
    rng = np.random.default_rng(seed)
    p = np.zeros(co.param_count())
    for l, (ws, shape, bs) in enumerate(co.param_layout()):
        fan_in = 9 * shape[2]
        s = scale * (last_scale if l == 3 else 1.0)
        p[ws] = rng.standard_normal(int(np.prod(shape))) * s * np.sqrt(2.0 / fan_in)
        p[bs] = rng.standard_normal(bs.stop - bs.start) * 0.05 * s
    return p.astype(np.float32).astype(np.float64)   # the GPU's FP32 master values


def make_system(pat, seed):
    """Context of the patch's grid and pins (FP32), a synthetic SPD stencil
    matrix with the same pins, x* and r = K x* (oracle product)."""
    nu, nv = pat.nu, pat.nv
    Kh = inputs.synthetic_stencil(seed, nu, nv, pinned=pat.pinned)
    pin = np.zeros(nu * nv, dtype=bool)
    pin[pat.pinned] = True
    xs_h = inputs.normal(seed + 1, 3 * nu * nv).reshape(nu * nv, 3)
    xs_h[pin] = 0.0
    r_h = oracle.stencil_matvec(nu, nv, Kh, xs_h)
    ctx = bsc.context_for_patch(pat, precision=bsc.FP32, pcg_rel_tol=1e-10)
    K = torch.as_tensor(np.ascontiguousarray(Kh.reshape(nu * nv, 225).T), dtype=torch.float32, device="cuda")
    r, xs = ctx.to_device(r_h), ctx.to_device(xs_h)
    prep = co.Prepared(nu, nv, Kh, pin)
    return ctx, K, r, xs, prep


@pytest.fixture(scope="module")
def system():
    pat = inputs.config_random_small(21, 40, 23, noise=0.05)
    ctx, K, r, xs, prep = make_system(pat, 5)
    net = bsc.Cnn(ctx)
    yield pat, ctx, net, K, r, xs, prep
    net.close()
    ctx.close()


def n3(t):
    return t.double().cpu().numpy().reshape(3, -1).T.copy()


def test_network_and_preconditioner_match_oracle(system):
    pat, ctx, net, K, r, xs, prep = system
    params = random_params(1, last_scale=0.3)
    net.set_params(params)
    net.prepare(K)
    z = net.apply(r)
    zo, cache = co.forward(params, prep, n3(r), bf16_like=True)
    f_gpu = net.activations(0)
    f_or = cache["acts"][0].reshape(-1, 32)
    ef = rel(f_gpu, f_or)
    errs = [rel(net.activations(l), cache["acts"][l].reshape(-1, 32)) for l in (1, 2, 3)]
    ea = rel(net.activations(4)[:, :9], cache["o"])
    ez = rel(n3(z), zo)
    print("features", ef, "layers", errs, "taps", ea, "z", ez)
    assert ef < 1e-3 and max(errs) < B_LAYER and ea < B_LAYER and ez < B_LAYER


def test_preconditioner_is_symmetric_on_the_gpu(system):
    pat, ctx, net, K, r, xs, prep = system
    net.set_params(random_params(5, last_scale=0.3))
    net.prepare(K)
    g = torch.Generator("cuda").manual_seed(9)
    x = torch.randn((3, ctx.N), device="cuda", generator=g)
    y = torch.randn((3, ctx.N), device="cuda", generator=g)
    pins = torch.as_tensor(pat.pinned, device="cuda", dtype=torch.long)
    x[:, pins] = 0.0
    y[:, pins] = 0.0
    Mx, My = net.apply(x.contiguous()), net.apply(y.contiguous())
    a, b = float((y * Mx).double().sum()), float((x * My).double().sum())
    assert abs(a - b) <= 1e-5 * max(abs(a), abs(b))
    assert float((x * Mx).double().sum()) > 0.0


def test_gradients_match_oracle(system):
    pat, ctx, net, K, r, xs, prep = system
    params = random_params(2, last_scale=0.3)
    net.set_params(params)
    net.prepare(K)
    L = net.loss_grad(r, xs)
    g = net.get_params(which=1).astype(np.float64)
    Lo, go = co.loss_and_grad(params, prep, n3(r), n3(xs), bf16_like=True)
    print(f"loss {L:.6e} vs oracle {Lo:.6e}: rel err {abs(L - Lo) / abs(Lo):.2e}")
    assert abs(L - Lo) <= B_GRAD * abs(Lo)
    for l, (ws, _, bs) in enumerate(co.param_layout()):
        ew, eb = rel(g[ws], go[ws]), rel(g[bs], go[bs])
        print(f"layer {l + 1}: weight-gradient rel err {ew:.2e}, bias {eb:.2e}")
        assert ew < B_GRAD_LAYER[l] and eb < B_GRAD_LAYER[l], l


def test_zero_weights_reproduce_block_jacobi(system):
    pat, ctx, net, K, r, xs, prep = system
    net.set_params(np.zeros(co.param_count()))
    net.prepare(K)
    z = n3(net.apply(r))
    ref = np.einsum("nab,nb->na", np.linalg.inv(prep.diag), n3(r))
    ref[prep.pin] = 0.0
    assert rel(z, ref) < 1e-6
    x, rep = net.solve(r, K, rel_tol=1e-8)
    _, it, _ = ctx.solve(r, K=K, rel_tol=1e-8)
    assert rep["fell_back"] == 0 and rep["rel_res"] <= 1e-8
    assert abs(rep["fcg_iters"] - it) <= 2, (rep, it)


def test_fcg_converges_with_a_random_network(system):
    pat, ctx, net, K, r, xs, prep = system
    net.set_params(random_params(3, last_scale=0.3))
    x, rep = net.solve(r, K, rel_tol=1e-8)
    assert rep["rel_res"] <= 1e-8
    res = n3(ctx.spmv(x, K=K)) - n3(r)
    assert np.linalg.norm(res) <= 1e-6 * np.linalg.norm(n3(r))
    print("random network:", rep)


def test_forced_stall_falls_back_to_pcg(system):
    """A stall window of one iteration makes the flexible CG hand over to
    block-Jacobi PCG as soon as r.r fails to drop by 4x in one iteration, on
    the patch's own Newton system (projected K, r = -g), which needs tens of
    iterations: the fallback must finish the solve to the same tolerance and
    the same solution as PCG alone."""
    pat, ctx, net, _, _, _, _ = system
    C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
    K = ctx.assemble_hessian(C, project=True)
    r = -ctx.gradient(C, Ch)
    x_pcg, it_pcg, _ = ctx.solve(r, K=K, rel_tol=1e-8)
    net.set_params(random_params(3, last_scale=0.3))
    net.set_stall_window(1)
    try:
        x, rep = net.solve(r, K, rel_tol=1e-8)
    finally:
        net.set_stall_window(24)
    print("forced stall:", rep, "PCG alone:", it_pcg)
    assert rep["fell_back"] == 1 and rep["pcg_iters"] > 0 and rep["fcg_iters"] >= 1
    assert rep["rel_res"] <= 1e-8
    res = n3(ctx.spmv(x, K=K)) - n3(r)
    assert np.linalg.norm(res) <= 1e-6 * np.linalg.norm(n3(r))
    assert rel(n3(x), n3(x_pcg)) < 1e-5


def test_cnn_parity_at_training_size():
    """512 x 512 (the training size): features, every layer output, the taps
    and z, the loss and every layer's weight and bias gradients against the
    oracle over all 262,144 pixels."""
    pat = inputs.config_learned(1, 512)
    ctx, K, r, xs, prep = make_system(pat, 11)
    net = bsc.Cnn(ctx)
    try:
        params = random_params(7, last_scale=0.3)
        net.set_params(params)
        net.prepare(K)
        z = net.apply(r)
        zo, cache = co.forward(params, prep, n3(r), bf16_like=True)
        ef = rel(net.activations(0), cache["acts"][0].reshape(-1, 32))
        errs = [rel(net.activations(l), cache["acts"][l].reshape(-1, 32)) for l in (1, 2, 3)]
        ea = rel(net.activations(4)[:, :9], cache["o"])
        ez = rel(n3(z), zo)
        L = net.loss_grad(r, xs)
        g = net.get_params(which=1).astype(np.float64)
        Lo, go = co.loss_and_grad(params, prep, n3(r), n3(xs), bf16_like=True)
        eL = abs(L - Lo) / abs(Lo)
        eg = [(rel(g[ws], go[ws]), rel(g[bs], go[bs])) for ws, _, bs in co.param_layout()]
        print(f"512x512: features {ef:.2e}, layers {[f'{e:.2e}' for e in errs]}, taps {ea:.2e}, z {ez:.2e}, "
              f"loss {eL:.2e}, gradients {[(f'{a:.2e}', f'{b:.2e}') for a, b in eg]}")
        assert ef < 1e-3 and max(errs) < B_LAYER and ea < B_LAYER and ez < B_LAYER
        assert eL < B_GRAD
        for l, (ew, eb) in enumerate(eg):
            assert ew < B_GRAD_LAYER[l] and eb < B_GRAD_LAYER[l], l
    finally:
        net.close()
        ctx.close()


def test_adam_steps_reduce_the_loss(system):
    pat, ctx, net, K, r, xs, prep = system
    params = random_params(4, scale=0.5, last_scale=0.0)
    net.set_params(params)
    net.prepare(K)
    L0 = net.loss_grad(r, xs)
    for _ in range(40):
        net.loss_grad(r, xs)
        net.adam_step(1e-3)
    L1 = net.loss_grad(r, xs)
    print("loss", L0, "->", L1)
    assert L1 < L0


WEIGHTS = __import__("os").path.join(__import__("os").path.dirname(__import__("os").path.dirname(
    __import__("os").path.abspath(__file__))), "paper_2506_18867_gb300", "weights", "cnn_learned512.npz")


@pytest.mark.skipif(not __import__("os").path.exists(WEIGHTS), reason="no trained weights")
def test_trained_network_gains_over_block_jacobi():
    """The committed network (trained on 512 x 512 Newton systems by
    paper_2506_18867_gb300.train_cnn) against the method without it, on two
    held-out systems: fewer CG iterations to 1e-8, same solution."""
    from paper_2506_18867_gb300 import train_cnn
    sy = train_cnn.Systems(512)
    net = bsc.Cnn(sy.ctx)
    net.set_params(np.load(WEIGHTS)["params"])
    tot_p = tot_f = 0
    for seed in (1_000_050, 1_000_051):
        pat, r = sy.load(seed)
        x0, it, rr = sy.ctx.solve(r, K=sy.K, rel_tol=1e-8)
        x1, rep = net.solve(r, sy.K, rel_tol=1e-8)
        assert rep["rel_res"] <= 1e-8 and rep["fell_back"] == 0
        res = (sy.ctx.spmv(x1, K=sy.K) - r).double().norm() / r.double().norm()
        assert float(res) < 1e-6
        assert float((x1 - x0).double().norm() / x0.double().norm()) < 1e-5
        print(f"seed {seed} (ratio {pat.meta['ratio']:.3g}): PCG {it} iterations, learned FCG {rep['fcg_iters']}")
        tot_p += it
        tot_f += rep["fcg_iters"]
    assert tot_f < tot_p
    net.close()
    sy.ctx.close()
