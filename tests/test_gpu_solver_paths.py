"""The Newton step with the learned solver, and the failure paths of the
solvers and of the line search, through the C ABI.

- Learned Newton step (Sec. 5.1 projected Newton with the flexible CG of the
  learned preconditioner, PCG as fallback): FP32 learned-preconditioned
  Newton iterations reach the FP64 oracle's converged positions within 1e-6
  of the cloth width; one learned step matches the plain PCG step to the
  solver tolerance; graph replay changes nothing.
- Bounded waits: with a short spin limit and one block more than launched
  expected at every barrier, the persistent PCG, the learned flexible CG and
  the Newton step return BSC_ERR_TIMEOUT instead of hanging, and the context
  solves correctly afterwards.  No wait is unbounded and nothing faults.
- Line search: a state whose Newton step needs three halvings fails with
  BSC_ERR_LINESEARCH when only two are allowed, as the oracle does, and
  leaves C unchanged.
"""
import os

import numpy as np
import pytest

from paper_2506_18867_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2506_18867_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2506_18867_gb300 import bsc  # noqa: E402

WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2506_18867_gb300",
                       "weights", "cnn_learned512.npz")


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def host(t):
    return t.double().cpu().numpy().reshape(3, -1).T.copy()


def trained_params():
    if not os.path.exists(WEIGHTS):
        pytest.skip("no trained weights")
    return np.load(WEIGHTS)["params"]


def test_learned_newton_reaches_oracle_positions(orc):
    """FP32 bulk with the learned flexible CG as the Newton step's solver
    converges to the FP64 oracle's converged positions within 1e-6 of the
    cloth width (drape physics, 64 x 64)."""
    pat = inputs.config_drape(2, 64, 1e-5)
    prob = orc.Problem.from_patch(pat)
    scene = orc.Scene.from_patch(pat, project=True)
    C_or = pat.C.copy()
    for _ in range(12):
        C_or, rep = orc.newton_step(prob, scene, C_or, pat.Chat, solver=0)
        assert rep.status == 0
        if rep.dir_inf < 1e-10:
            break
    width = 2.0
    with bsc.context_for_patch(pat, precision=bsc.FP32, pcg_rel_tol=1e-8) as ctx:
        net = bsc.Cnn(ctx)
        net.set_params(trained_params())
        ctx.set_learned_solver(net)
        C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
        steps, fcg = 0, 0
        for _ in range(15):
            st, rep = ctx.newton_step_status(C, Ch)
            steps += 1
            fcg += rep.fcg_iters
            if st == bsc.ERR_LINESEARCH or rep.dir_inf / pat.dt < 1e-6:
                break
            assert st == bsc.OK, st
            assert rep.fcg_iters > 0 and rep.pcg_rel_res <= 1e-8
        Cg = host(C)
        net.close()
    err = np.abs(Cg - C_or).max()
    print(f"FP32 learned Newton ({steps} steps, {fcg} flexible-CG iterations) vs FP64 oracle: "
          f"max |dC| = {err:.3e} m = {err / width:.2e} of the width")
    assert fcg > 0
    assert err <= 1e-6 * width


def test_learned_step_matches_pcg_step():
    """One Newton step from the same state with the learned solver and with
    plain PCG: same energies, step length and positions to the solver
    tolerance; graph replay of the learned step is bitwise the direct launch."""
    pat = inputs.config_drape(3, 96, 1e-5)
    with bsc.context_for_patch(pat, precision=bsc.FP32, pcg_rel_tol=1e-8) as ctx:
        C0 = ctx.to_device(pat.C)
        Ch = ctx.to_device(pat.Chat)
        C1 = C0.clone()
        r1 = ctx.newton_step(C1, Ch)
        net = bsc.Cnn(ctx)
        net.set_params(trained_params())
        ctx.set_learned_solver(net)
        C2 = C0.clone()
        r2 = ctx.newton_step(C2, Ch)
        ctx.set_graph(False)
        C3 = C0.clone()
        r3 = ctx.newton_step(C3, Ch)
        ctx.set_graph(True)
        print(f"PCG step: {r1.pcg_iters} iterations; learned step: {r2.fcg_iters} flexible-CG + "
              f"{r2.pcg_iters - r2.fcg_iters} PCG, fell back {r2.fell_back}")
        assert r2.fcg_iters > 0 and r2.pcg_rel_res <= 1e-8
        assert r1.E0 == r2.E0 and r1.alpha == r2.alpha
        assert abs(r1.E1 - r2.E1) <= 1e-7 * abs(r1.E0)
        width = 2.0
        assert float((C1 - C2).abs().max()) <= 1e-6 * width
        assert torch.equal(C2, C3) and r2.fcg_iters == r3.fcg_iters
        ctx.set_learned_solver(None)
        C4 = C0.clone()
        r4 = ctx.newton_step(C4, Ch)
        assert r4.fcg_iters == 0 and torch.equal(C4, C1)
        net.close()


def test_barrier_timeouts_return_and_context_recovers():
    """Every barrier expects one block more than was launched, with a spin
    limit of 2^12 sleeps: PCG, learned flexible CG and the Newton step return
    BSC_ERR_TIMEOUT; with the limit restored the same solves succeed."""
    pat = inputs.config_random_small(3, 24, 20, noise=0.05)
    with bsc.context_for_patch(pat, precision=bsc.FP32, pcg_rel_tol=1e-8) as ctx:
        C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
        K = ctx.assemble_hessian(C, project=True)
        b = -ctx.gradient(C, Ch)
        x_ref, it_ref, _ = ctx.solve(b, K=K)
        net = bsc.Cnn(ctx)
        net.set_params(trained_params())
        x_fcg_ref, _ = net.solve(b, K)
        ctx.set_wait_limit(1 << 12, 1)
        x = ctx.new_vec()
        st = ctx._lib.bsc_solve(ctx._h, bsc._ptr(K), bsc._ptr(b), bsc._ptr(x), 1e-8, 1000, None, None)
        assert st == bsc.ERR_TIMEOUT, st
        st, _, rep = net.solve_status(b, K)
        assert st == bsc.ERR_TIMEOUT, (st, rep)
        ctx.set_learned_solver(net)
        Ct = C.clone()
        st, rep = ctx.newton_step_status(Ct, Ch)
        assert st == bsc.ERR_TIMEOUT, st
        ctx.set_learned_solver(None)
        st, rep = ctx.newton_step_status(Ct, Ch)
        assert st == bsc.ERR_TIMEOUT, st
        # the default limit and no phantom block: everything works again
        ctx.set_wait_limit(1 << 25, 0)
        x2, it2, rr2 = ctx.solve(b, K=K)
        assert it2 == it_ref and torch.equal(x2, x_ref)
        x3, rep3 = net.solve(b, K)
        assert torch.equal(x3, x_fcg_ref) and rep3["rel_res"] <= 1e-8
        Cn = C.clone()
        rep = ctx.newton_step(Cn, Ch)
        assert rep.status == bsc.OK and rep.E1 <= rep.E0
        net.close()


def test_line_search_exhaustion(orc):
    """The noisy patch's Newton step needs three halvings (oracle and GPU
    agree); allowing two makes both report the line-search failure, and the
    GPU leaves C unchanged."""
    pat = inputs.config_random_small(16, 14, 12, noise=0.3)
    prob = orc.Problem.from_patch(pat)
    sc = orc.Scene.from_patch(pat, project=True)
    _, orep = orc.newton_step(prob, sc, pat.C, pat.Chat, solver=0)
    assert orep.status == 0 and orep.ls_halvings == 3
    oC2, orep2 = orc.newton_step(prob, sc, pat.C, pat.Chat, solver=0, max_halvings=2)
    assert orep2.status == -3 and np.array_equal(oC2, pat.C)
    with bsc.context_for_patch(pat, precision=bsc.FP64, pcg_rel_tol=1e-13) as ctx:
        C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
        rep = ctx.newton_step(C.clone(), Ch)
        assert rep.ls_halvings == 3
    with bsc.context_for_patch(pat, precision=bsc.FP64, pcg_rel_tol=1e-13, max_line_search=2) as ctx:
        C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
        C0 = C.clone()
        st, rep = ctx.newton_step_status(C, Ch)
        print("line search with 2 halvings:", bsc.STATUS_NAMES[st], rep.as_dict())
        assert st == bsc.ERR_LINESEARCH and rep.status == bsc.ERR_LINESEARCH
        assert rep.ls_halvings == 2 and rep.alpha == 0.0
        assert torch.equal(C, C0)
