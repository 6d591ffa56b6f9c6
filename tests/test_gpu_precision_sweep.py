"""Precision sweep at 1024 x 1024 control points (1,044,484 spans, 4 m x 4 m,
multi-frequency wrinkle field): energy, gradient, the assembled Hessian and
50 SpMVs on the GPU in FP64 and in FP32, each against the FP64 oracle.

The energy and the gradient are compared over the whole patch; the Hessian,
raw and with the per-span SPD projection the Newton step uses, on sampled
stencil rows (corners, edges, interior), which the oracle computes one by
one; each SpMV y = K x (random x) on the same rows, against
the oracle's rows of K applied to x in FP64.  The errors are printed per
result; the bounds are 1e-12 relative for FP64 and, for FP32, the bounds of
the drape parity tests, except the FP32 gradient: at this near-equilibrium
wrinkle state (C = C^, no inertia term) the gradient is a small sum of
large point terms, so its FP32 error relative to its own norm is larger
(about 1e-4 measured); it is bounded by 5e-4.
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

N_SIDE = 1024
N_SPMV = 50


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def sweep(orc):
    pat = inputs.config_wrinkle(1, N_SIDE)
    prob = orc.Problem.from_patch(pat)
    scene = orc.Scene.from_patch(pat, project=False)
    rng = np.random.default_rng(8)
    n = N_SIDE
    rows = [0, n - 1, (n - 1) * n, n * n - 1, 1, n + 1, 2 * n + 2, n * (n // 2)]
    rows += [int(j) * n + int(i) for i, j in rng.integers(0, n, (64, 2))]
    rows = np.array(sorted(set(rows)), dtype=np.int32)
    oE = orc.energy(prob, scene, pat.C, pat.Chat)
    _, og, _ = orc.evaluate(prob, scene, pat.C, pat.Chat, want_K=False)
    _, oK = orc.eval_rows(prob, scene, pat.C, pat.Chat, rows)
    _, oKp = orc.eval_rows(prob, orc.Scene.from_patch(pat, project=True), pat.C, pat.Chat, rows)
    return pat, rows, oE, og, oK, oKp


def neighbour_index(n, rows):
    """(len(rows), 25) control-point index of each stencil slot, -1 outside."""
    i, j = rows % n, rows // n
    out = np.full((rows.size, 25), -1, dtype=np.int64)
    for dv in range(-2, 3):
        for du in range(-2, 3):
            s = (dv + 2) * 5 + (du + 2)
            ii, jj = i + du, j + dv
            ok = (ii >= 0) & (ii < n) & (jj >= 0) & (jj < n)
            out[ok, s] = (jj * n + ii)[ok]
    return out


@pytest.mark.parametrize("precision", [bsc.FP64, bsc.FP32], ids=["fp64", "fp32"])
def test_precision_sweep_1024(sweep, precision):
    pat, rows, oE, og, oK, oKp = sweep
    nb = neighbour_index(N_SIDE, rows.astype(np.int64))
    valid = nb >= 0
    dt = torch.float64 if precision == bsc.FP64 else torch.float32
    with bsc.context_for_patch(pat, precision=precision, pcg_rel_tol=1e-8) as ctx:
        C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
        E = ctx.energy(C, Ch)
        g = ctx.gradient(C, Ch).double().cpu().numpy().reshape(3, -1).T
        K = ctx.assemble_hessian(C, project=False)
        ri = torch.as_tensor(rows, device="cuda", dtype=torch.long)
        Kr = K[:, ri].double().cpu().numpy().reshape(25, 3, 3, -1).transpose(3, 0, 1, 2)
        gen = torch.Generator("cuda").manual_seed(11)
        e_spmv = []
        for _ in range(N_SPMV):
            x = torch.randn((3, ctx.N), dtype=dt, device="cuda", generator=gen)
            y = ctx.spmv(x, K=K)[:, ri].double().cpu().numpy().T            # (rows, 3)
            xh = x.double().cpu().numpy().T                                   # (N, 3)
            xn = np.where(valid[..., None], xh[np.where(valid, nb, 0)], 0.0)  # (rows, 25, 3)
            yo = np.einsum("rsab,rsb->ra", oK, xn)
            e_spmv.append(rel(y, yo))
        del K
        Kp = ctx.assemble_hessian(C, project=True)
        Kpr = Kp[:, ri].double().cpu().numpy().reshape(25, 3, 3, -1).transpose(3, 0, 1, 2)
        del Kp
    eE, eg, eK, eKp = abs(E - oE) / abs(oE), rel(g, og), rel(Kr, oK), rel(Kpr, oKp)
    name = "FP64" if precision == bsc.FP64 else "FP32"
    print(f"{name} 1024x1024: energy {eE:.2e}, gradient {eg:.2e}, {rows.size} Hessian rows {eK:.2e} "
          f"(projected {eKp:.2e}), {N_SPMV} SpMVs max {max(e_spmv):.2e} (mean {np.mean(e_spmv):.2e})")
    if precision == bsc.FP64:
        assert eE < 1e-12 and eg < 1e-12 and eK < 1e-12 and eKp < 1e-12 and max(e_spmv) < 1e-12
    else:
        assert eE < 1e-6 and eg < 5e-4 and eK < 2e-5 and eKp < 2e-5 and max(e_spmv) < 2e-5
