"""Strip windows of one patch on the GPU (bsc_create_window and the strip
PCG calls, include/bsc.h) against the single-domain context and the oracle.

- The gradient and Hessian rows a window owns, its energy share and its
  product rows equal the whole-patch context's bit for bit (FP64 and FP32):
  same spans, same gather order, same kernels.
- One projected Newton iteration (Sec. 5.1) run by 1, 2 and 3 host-thread
  ranks on one device (strip.ThreadComm: halo rows copied between the
  ranks' window tensors, per-row partial sums gathered on the host) gives
  the same positions bit for bit for every split, and within 1e-10 of the
  width of the oracle's Newton step on the whole patch (FP64).
- The calls reject what a window cannot do (Newton step, solve, autotune).
"""
import math

import numpy as np
import pytest

from paper_2506_18867_gb300 import inputs, partition, strip

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2506_18867_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2506_18867_gb300 import bsc  # noqa: E402


def patch():
    # 40 x 37 control points: strips of several rows, the two pinned top corners in the last strip
    p = inputs.config_wrinkle(2, 64, 1.0, crop=None)
    return inputs.Patch("wrinkle40x37", 40, 37, p.rest.reshape(64, 64, 2)[:37, :40].reshape(-1, 2).copy(),
                        p.C.reshape(64, 64, 3)[:37, :40].reshape(-1, 3).copy(),
                        p.Chat.reshape(64, 64, 3)[:37, :40].reshape(-1, 3).copy(), p.material, p.dt, p.gravity,
                        np.array([36 * 40, 36 * 40 + 39], dtype=np.int32), {})


def windows(nv, world):
    strips = partition.strip_rows(nv, world)
    return strips, [partition.window_rows(strips, r, nv) + strips[r] for r in range(world)]


def win_tensor(full, nu, w):
    """Window rows of a (3, nu * nv) tensor."""
    return full.view(3, -1, nu)[:, w[0]:w[1]].reshape(3, -1).contiguous()


def owned(t, nu, w):
    """The owned rows of a window tensor."""
    return t.view(t.shape[0], -1, nu)[:, w[2] - w[0]:w[3] - w[0]]


def rows_of(t, nu, w):
    """The same rows of a whole-patch tensor."""
    return t.view(t.shape[0], -1, nu)[:, w[2]:w[3]]


@pytest.fixture(scope="module")
def pat():
    return patch()


@pytest.mark.parametrize("precision", [bsc.FP64, bsc.FP32], ids=["fp64", "fp32"])
@pytest.mark.parametrize("world", [2, 3])
def test_window_rows_equal_whole_patch(pat, precision, world):
    nu = pat.nu
    with bsc.context_for_patch(pat, precision=precision) as full:
        C, Ch = full.to_device(pat.C), full.to_device(pat.Chat)
        g = full.gradient(C, Ch)
        K = full.assemble_hessian(C, project=True)
        x = full.to_device(np.random.default_rng(4).standard_normal((pat.n_cp, 3)))
        y = full.spmv(x, K=K)
        E = full.energy(C, Ch)
        strips, wins = windows(pat.nv, world)
        parts = []
        for w in wins:
            with bsc.context_for_patch(pat, precision=precision, window=w) as ctx:
                Cw, Chw = win_tensor(C, nu, w), win_tensor(Ch, nu, w)
                gw = ctx.gradient(Cw, Chw)
                Kw = ctx.assemble_hessian(Cw, project=True)
                yw = ctx.spmv(win_tensor(x, nu, w), K=Kw)
                assert torch.equal(owned(gw, nu, w), rows_of(g, nu, w))
                assert torch.equal(owned(Kw, nu, w), rows_of(K, nu, w))
                assert torch.equal(owned(yw, nu, w), rows_of(y, nu, w))
                sr, cr = ctx.energy_rows(Cw, Chw)
                parts.extend(list(sr) + list(cr))
                assert abs(ctx.energy(Cw, Chw) - math.fsum(list(sr) + list(cr))) <= 1e-13 * abs(E)
        Es = math.fsum(parts)
        print(f"{world} windows: energy {Es!r} vs whole patch {E!r}")
        assert abs(Es - E) <= 1e-13 * abs(E)


def strip_step(pat, world, precision=bsc.FP64, tol=1e-12):
    nu = pat.nu
    strips, wins = windows(pat.nv, world)
    C0 = torch.from_numpy(np.ascontiguousarray(pat.C.T))
    Ch0 = torch.from_numpy(np.ascontiguousarray(pat.Chat.T))
    dt = torch.float64 if precision == bsc.FP64 else torch.float32

    def rank(r, comm):
        w = wins[r]
        with bsc.context_for_patch(pat, precision=precision, window=w) as ctx:
            C = win_tensor(C0, nu, w).to(device="cuda", dtype=dt)
            Ch = win_tensor(Ch0, nu, w).to(device="cuda", dtype=dt)
            rep = strip.newton_step(ctx, comm, strips, pat.nv, C, Ch, tol=tol)
            return rep, owned(C, nu, w).reshape(3, -1).cpu()

    out = strip.run_threads(world, rank)
    return [o[0] for o in out], torch.cat([o[1] for o in out], dim=1).double().numpy().T


@pytest.fixture(scope="module")
def one_rank(pat):
    return strip_step(pat, 1)


@pytest.mark.parametrize("world", [2, 3])
def test_strip_newton_step_bit_identical(pat, one_rank, world):
    reps1, C1 = one_rank
    reps, C = strip_step(pat, world)
    for rep in reps:
        assert rep == reps1[0]
    assert np.array_equal(C, C1)


def test_strip_newton_step_matches_oracle(orc, pat, one_rank):
    reps1, C1 = one_rank
    prob = orc.Problem.from_patch(pat)
    sc = orc.Scene.from_patch(pat, project=True)
    oC, orep = orc.newton_step(prob, sc, pat.C, pat.Chat, solver=0)
    rep = reps1[0]
    width = np.ptp(pat.rest, axis=0).max()
    with bsc.context_for_patch(pat, precision=bsc.FP64, pcg_rel_tol=1e-12) as full:
        C = full.to_device(pat.C)
        frep = full.newton_step(C, full.to_device(pat.Chat))
        Cf = C.double().cpu().numpy().T
    print(f"strip: {rep['pcg_iters']} iterations, alpha {rep['alpha']}; whole-patch context "
          f"{frep.pcg_iters}; max |dC| vs oracle {np.abs(C1 - oC).max():.2e}, vs context "
          f"{np.abs(C1 - Cf).max():.2e}")
    assert rep["status"] == "ok" and rep["alpha"] == orep.alpha
    assert abs(rep["E0"] - orep.E0) <= 1e-12 * abs(orep.E0)
    assert np.abs(C1 - oC).max() <= 1e-10 * width
    assert np.abs(C1 - Cf).max() <= 1e-10 * width


def test_strip_fp32_ranks_agree(pat):
    """FP32 windows: the same bit-identity across splits (the same kernels
    and partial sums), and the step within FP32 reach of the FP64 one."""
    reps1, C1 = strip_step(pat, 1, bsc.FP32, tol=1e-6)
    reps2, C2 = strip_step(pat, 3, bsc.FP32, tol=1e-6)
    assert reps2[0] == reps1[0] and np.array_equal(C1, C2)
    _, C64 = strip_step(pat, 1, bsc.FP64, tol=1e-12)
    width = np.ptp(pat.rest, axis=0).max()
    assert np.abs(C1 - C64).max() <= 1e-5 * width


def test_window_rejects_whole_patch_calls(pat):
    w = windows(pat.nv, 2)[1][0]
    with bsc.context_for_patch(pat, precision=bsc.FP64, window=w) as ctx:
        C = win_tensor(torch.from_numpy(np.ascontiguousarray(pat.C.T)), pat.nu, w).cuda()
        for call in (lambda: ctx.newton_step(C, C.clone()), lambda: ctx.solve(ctx.new_vec()),
                     lambda: ctx.autotune(C, C.clone())):
            with pytest.raises(bsc.BscError) as e:
                call()
            assert e.value.status == bsc.ERR_INVALID_ARG
    # halos of other than two rows (clipped to the grid), owned rows outside the grid
    for bad in ((0, 5, 0, 4), (2, 9, 3, 7), (0, 3, 0, 2), (1, 8, 3, 7), (30, 37, 32, 38)):
        with pytest.raises(bsc.BscError):
            bsc.context_for_patch(pat, precision=bsc.FP64, window=bad)
