"""Full-size parity in the bench's launch configuration (drape 256 x 256, FP32
bulk, the same context options), plus the FP64 path at the same size, on
sampled outputs the oracle computes one by one (selected spans, selected
stencil rows), and properties that hold at any size (PCG residual, energy
decrease).  Also the converged-position target: FP32 Newton iterations reach
the FP64 oracle's converged positions within 1e-6 of the cloth width.
"""
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


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def drape(orc):
    pat = inputs.config_drape(1, 256, 1e-5)
    return pat, orc.Problem.from_patch(pat), orc.Scene.from_patch(pat, project=True)


def sample_spans(Su, Sv, seed=3):
    rng = np.random.default_rng(seed)
    pick = [(0, 0), (Su - 1, Sv - 1), (0, Sv - 1), (Su - 1, 0)]                     # corners
    pick += [(0, int(b)) for b in rng.integers(1, Sv - 1, 6)]                        # u-side
    pick += [(int(a), Sv - 1) for a in rng.integers(1, Su - 1, 6)]                   # v-side
    pick += [(1, int(b)) for b in rng.integers(1, Sv - 1, 4)]                        # next to the border
    pick += [(Su - 2, int(b)) for b in rng.integers(1, Sv - 1, 4)]
    pick += [(int(a), int(b)) for a, b in rng.integers(2, min(Su, Sv) - 2, (60, 2))]  # interior
    return np.array(sorted({b * Su + a for a, b in pick}), dtype=np.int32)


def sample_rows(nu, nv, seed=4):
    rng = np.random.default_rng(seed)
    rows = [0, nu - 1, (nv - 1) * nu, nv * nu - 1, nu, 2 * nu + 1, 5 * nu + 2]     # corners, pinned edge
    rows += [int(j) * nu + int(i) for i, j in rng.integers(0, nu, (40, 2))]
    return np.array(sorted(set(rows)), dtype=np.int32)


@pytest.mark.parametrize("precision", [bsc.FP32, bsc.FP64])
def test_span_terms_full_size(orc, drape, precision):
    pat, prob, _ = drape
    idx = sample_spans(pat.nu - 2, pat.nv - 2)
    with bsc.context_for_patch(pat, precision=precision, pcg_rel_tol=1e-8) as ctx:
        E, g, H = ctx.span_terms(ctx.to_device(pat.C), project=True)
        ii = torch.as_tensor(idx, device="cuda", dtype=torch.long)
        Eg, gg, Hg = E[ii].cpu().numpy(), g[ii].double().cpu().numpy(), H[ii].double().cpu().numpy()
        del E, g, H
    oE, og, oH = orc.span_terms_subset(prob, pat.C, idx, project=True)
    per_span = [rel(Hg[k], oH[k]) for k in range(len(idx))]
    print(f"precision {precision}: {len(idx)} spans, span Hessian rel err max {max(per_span):.2e}, "
          f"gradient {rel(gg, og):.2e}, energy {rel(Eg, oE):.2e}")
    bound = 1e-12 if precision == bsc.FP64 else 2e-5
    assert max(per_span) < 10 * bound and rel(Hg, oH) < bound
    assert rel(gg, og) < (1e-12 if precision == bsc.FP64 else 1e-4)


@pytest.mark.parametrize("precision", [bsc.FP32, bsc.FP64])
def test_energy_gradient_rows_full_size(orc, drape, precision):
    pat, prob, scene = drape
    rows = sample_rows(pat.nu, pat.nv)
    with bsc.context_for_patch(pat, precision=precision, pcg_rel_tol=1e-8) as ctx:
        C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
        E = ctx.energy(C, Ch)
        g = ctx.gradient(C, Ch).double().cpu().numpy().reshape(3, -1).T
        K = ctx.assemble_hessian(C, project=True)
        Kr = K[:, torch.as_tensor(rows, device="cuda", dtype=torch.long)].double().cpu().numpy()
        Kr = Kr.reshape(25, 3, 3, -1).transpose(3, 0, 1, 2)
    oE = orc.energy(prob, scene, pat.C, pat.Chat)
    _, og, _ = orc.evaluate(prob, scene, pat.C, pat.Chat, want_K=False)
    ogr, oKr = orc.eval_rows(prob, scene, pat.C, pat.Chat, rows)
    eE, eg, eK = abs(E - oE) / abs(oE), rel(g, og), rel(Kr, oKr)
    print(f"precision {precision}: energy {eE:.2e}, gradient {eg:.2e}, {len(rows)} K rows {eK:.2e}")
    if precision == bsc.FP64:
        assert eE < 1e-12 and eg < 1e-12 and eK < 1e-12
    else:
        assert eE < 1e-6 and eg < 1e-4 and eK < 2e-5


def _np_stencil_matvec(nu, nv, K, x):
    """y = K x from the (225, N) planes, in FP64 on the host."""
    N = nu * nv
    K = K.reshape(25, 3, 3, nv, nu)
    X = x.reshape(3, nv, nu)
    y = np.zeros((3, nv, nu))
    for dv in range(-2, 3):
        for du in range(-2, 3):
            s = (dv + 2) * 5 + (du + 2)
            jy = slice(max(0, -dv), nv - max(0, dv))
            iy = slice(max(0, -du), nu - max(0, du))
            jx = slice(max(0, dv), nv - max(0, -dv))
            ix = slice(max(0, du), nu - max(0, -du))
            for r in range(3):
                for c in range(3):
                    y[r, jy, iy] += K[s, r, c, jy, iy] * X[c, jx, ix]
    return y.reshape(3, N)


def test_spmv_pcg_newton_full_size(drape):
    pat, _, _ = drape
    with bsc.context_for_patch(pat, precision=bsc.FP32, pcg_rel_tol=1e-8) as ctx:
        C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
        K = ctx.assemble_hessian(C, project=True)
        Kh = K.double().cpu().numpy()
        x = torch.randn((3, ctx.N), dtype=torch.float32, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
        y = ctx.spmv(x, K=K).double().cpu().numpy()
        yr = _np_stencil_matvec(pat.nu, pat.nv, Kh, x.double().cpu().numpy())
        assert rel(y, yr) < 1e-6
        b = -ctx.gradient(C, Ch)
        d, it, rr = ctx.solve(b, K=K, rel_tol=1e-8)
        true_res = rel(_np_stencil_matvec(pat.nu, pat.nv, Kh, d.double().cpu().numpy()), b.double().cpu().numpy())
        print(f"PCG: {it} iterations, recursive residual {rr:.2e}, true residual (FP64 host) {true_res:.2e}")
        assert rr <= 1e-8 and true_res < 1e-6
        rep = ctx.newton_step(C, Ch)
        assert rep.status == 0 and rep.E1 <= rep.E0 and rep.alpha > 0


def test_fp32_newton_reaches_oracle_positions(orc):
    """FP32 bulk Newton iterations converge to the FP64 oracle's converged
    positions within 1e-6 of the cloth width (drape physics, 64 x 64)."""
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
        C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
        steps = 0
        for _ in range(15):
            st, rep = ctx.newton_step_status(C, Ch)
            steps += 1
            if st == bsc.ERR_LINESEARCH or rep.dir_inf / pat.dt < 1e-6:
                break
            assert st == bsc.OK, st
        Cg = C.double().cpu().numpy().reshape(3, -1).T
    err = np.abs(Cg - C_or).max()
    print(f"FP32 Newton ({steps} steps) vs FP64 oracle: max |dC| = {err:.3e} m = {err / width:.2e} of the width")
    assert err <= 1e-6 * width
