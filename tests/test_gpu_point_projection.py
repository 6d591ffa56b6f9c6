"""Per-point projection of the FBW membrane Hessian (BSC_PROJECT_POINT)
against the FP64 CPU oracle, through the C ABI.

The GPU projects each FBW term's 6x6 Hessian w.r.t. (f_1, f_2) in closed form
inside the span evaluation; the oracle projects the same 6x6 matrices with its
cyclic Jacobi eigensolver.  FP64 bar 1e-12 relative (norm-wise), as for the
unprojected terms; FP32 bulk held to the FP32 bounds of the span path.
States: noisy, strongly compressed (every stretch term clamped), sheared
(both signs of I6), curved rests, and the drape at full size.
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

POINT = bsc.PROJECT_POINT


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def to_n3(t):
    return t.detach().double().cpu().numpy().reshape(3, -1).T.copy()


def _compressed(seed, nu, nv):
    pat = inputs.config_random_small(seed, nu, nv, noise=0.05)
    c = pat.C.mean(axis=0)
    pat.C = c + 0.6 * (pat.C - c)
    return pat


def _sheared(seed, nu, nv, gamma):
    pat = inputs.config_random_small(seed, nu, nv, angle=0.0, noise=0.02)
    pat.C = pat.C.copy()
    pat.C[:, 0] += gamma * pat.rest[:, 1]
    return pat


CASES = [
    ("rand5x5", lambda: inputs.config_random_small(2, 5, 5)),
    ("rand6x9_noisy", lambda: inputs.config_random_small(3, 6, 9, noise=0.3)),
    ("rand13x7_curved", lambda: inputs.config_random_small(4, 13, 7, curved=0.6, noise=0.1)),
    ("compressed11x10", lambda: _compressed(6, 11, 10)),
    ("shear+9x8", lambda: _sheared(7, 9, 8, 0.4)),
    ("shear-9x8", lambda: _sheared(8, 9, 8, -0.6)),
    ("rand40x23", lambda: inputs.config_random_small(5, 40, 23, noise=0.05)),
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request, orc):
    pat = request.param[1]()
    prob = orc.Problem.from_patch(pat)
    ctx = bsc.context_for_patch(pat, precision=bsc.FP64, project=POINT, pcg_rel_tol=1e-13)
    yield pat, prob, ctx
    ctx.close()


def test_span_terms_point_fp64(case, orc):
    pat, prob, ctx = case
    E, g, H = ctx.span_terms(ctx.to_device(pat.C), project=POINT)
    oE, og, oH = prob.span_eval_projected(pat.C, orc.PROJECT_POINT)
    assert rel(E.cpu().numpy(), oE) < 1e-12
    assert rel(g.cpu().numpy(), og) < 1e-12
    assert rel(H.cpu().numpy(), oH) < 1e-12
    Hg = H.cpu().numpy()
    assert np.abs(Hg - Hg.transpose(0, 2, 1)).max() == 0.0


def test_assembled_hessian_point_fp64(case, orc):
    pat, prob, ctx = case
    sc = orc.Scene.from_patch(pat, project=orc.PROJECT_POINT)
    _, _, oK = orc.evaluate(prob, sc, pat.C, pat.Chat, want_g=False)
    K = ctx.assemble_hessian(ctx.to_device(pat.C), project=POINT)
    Kg = K.detach().double().cpu().numpy().reshape(25, 3, 3, pat.n_cp).transpose(3, 0, 1, 2)
    assert rel(Kg, oK) < 1e-12


def test_newton_step_point_fp64(case, orc):
    pat, prob, ctx = case
    sc = orc.Scene.from_patch(pat, project=orc.PROJECT_POINT)
    oC, orep = orc.newton_step(prob, sc, pat.C, pat.Chat, solver=0 if pat.n_cp <= 4096 else 1, pcg_tol=1e-14)
    C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
    rep = ctx.newton_step(C, Ch)
    assert rep.status == 0 and orep.status == 0
    assert rep.alpha == orep.alpha and rep.spans_projected == 0
    assert abs(rep.E0 - orep.E0) <= 1e-11 * abs(orep.E0)
    width = np.ptp(pat.rest, axis=0).max()
    assert np.abs(to_n3(C) - oC).max() <= 1e-10 * width
    assert rel(to_n3(C) - pat.C, oC - pat.C) < 1e-9


@pytest.mark.parametrize("name", ["compressed11x10", "shear-9x8", "rand40x23"])
def test_span_terms_point_fp32(orc, name):
    pat = dict(CASES)[name]()
    prob = orc.Problem.from_patch(pat)
    with bsc.context_for_patch(pat, precision=bsc.FP32, project=POINT) as ctx:
        _, g, H = ctx.span_terms(ctx.to_device(pat.C), project=POINT)
        g, H = g.double().cpu().numpy(), H.double().cpu().numpy()
    _, og, oH = prob.span_eval_projected(pat.C, orc.PROJECT_POINT)
    eg, eH = rel(g, og), rel(H, oH)
    print(f"{name} FP32 per-point projection vs oracle: gradient {eg:.2e} span Hessian {eH:.2e}")
    assert eg < 1e-4 and eH < 2e-5


def test_bad_project_value():
    pat = inputs.config_random_small(2, 6, 6)
    with bsc.context_for_patch(pat, precision=bsc.FP64) as ctx:
        C = ctx.to_device(pat.C)
        with pytest.raises(bsc.BscError) as ei:
            ctx._check(ctx._lib.bsc_assemble_hessian(ctx._h, bsc._ptr(C), 3, None))
        assert ei.value.status == bsc.ERR_INVALID_ARG
        ctx.assemble_hessian(C, project=POINT)  # the context stays usable


def _sample_spans(Su, Sv, seed=3):
    rng = np.random.default_rng(seed)
    pick = [(0, 0), (Su - 1, Sv - 1), (0, Sv - 1), (Su - 1, 0)]
    pick += [(0, int(b)) for b in rng.integers(1, Sv - 1, 6)]
    pick += [(int(a), Sv - 1) for a in rng.integers(1, Su - 1, 6)]
    pick += [(int(a), int(b)) for a, b in rng.integers(1, min(Su, Sv) - 1, (60, 2))]
    return np.array(sorted({b * Su + a for a, b in pick}), dtype=np.int32)


@pytest.mark.parametrize("precision", [bsc.FP32, bsc.FP64])
def test_drape_full_size_point(orc, precision):
    """The 256 x 256 drape in the bench's options with the per-point
    projection: sampled span Hessians and stencil rows against the oracle,
    then one Newton step (PCG residual, energy decrease)."""
    pat = inputs.config_drape(1, 256, 1e-5)
    prob = orc.Problem.from_patch(pat)
    scene = orc.Scene.from_patch(pat, project=orc.PROJECT_POINT)
    idx = _sample_spans(pat.nu - 2, pat.nv - 2)
    rows = np.array(sorted({0, 255, 256 * 255, 65535, 256, 513} |
                           {int(j) * 256 + int(i) for i, j in np.random.default_rng(4).integers(0, 256, (40, 2))}),
                    dtype=np.int32)
    with bsc.context_for_patch(pat, precision=precision, project=POINT, pcg_rel_tol=1e-8) as ctx:
        C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
        _, _, H = ctx.span_terms(C, project=POINT)
        Hg = H[torch.as_tensor(idx, device="cuda", dtype=torch.long)].double().cpu().numpy()
        del H
        K = ctx.assemble_hessian(C, project=POINT)
        Kr = K[:, torch.as_tensor(rows, device="cuda", dtype=torch.long)].double().cpu().numpy()
        Kr = Kr.reshape(25, 3, 3, -1).transpose(3, 0, 1, 2)
        rep = ctx.newton_step(C, Ch)
    _, _, oH = orc.span_terms_subset(prob, pat.C, idx, project=orc.PROJECT_POINT)
    _, oKr = orc.eval_rows(prob, scene, pat.C, pat.Chat, rows)
    eH, eK = rel(Hg, oH), rel(Kr, oKr)
    print(f"precision {precision}: {len(idx)} spans {eH:.2e}, {len(rows)} K rows {eK:.2e}, "
          f"PCG {rep.pcg_iters} iterations, alpha {rep.alpha}")
    bound = 1e-12 if precision == bsc.FP64 else 2e-5
    assert eH < bound and eK < bound
    assert rep.status == 0 and rep.E1 <= rep.E0 and rep.pcg_rel_res <= 1e-8 and rep.spans_projected == 0


def test_batch_point_projection_bitwise(orc):
    """A batch of uneven patches under the per-point projection: span terms
    and K bitwise equal to one context per patch; every patch's Newton step
    succeeds."""
    pats = [inputs.config_random_small(11 + k, nu, nv, noise=0.2)
            for k, (nu, nv) in enumerate([(7, 9), (12, 6), (5, 5), (20, 14)])]
    batch = bsc.batch_for_patches(pats, precision=bsc.FP64, project=POINT)
    try:
        out = np.zeros((3, batch.N))
        for p, pat in enumerate(pats):
            out[:, batch.cp_offset[p]:batch.cp_offset[p + 1]] = pat.C.T
        C = torch.from_numpy(out).to(device="cuda", dtype=batch.dtype).contiguous()
        _, _, H = batch.span_terms(C, project=POINT)
        K = batch.assemble_hessian(C, project=POINT)
        for p, pat in enumerate(pats):
            with bsc.context_for_patch(pat, precision=bsc.FP64, project=POINT) as one:
                C1 = one.to_device(pat.C)
                _, _, H1 = one.span_terms(C1, project=POINT)
                K1 = one.assemble_hessian(C1, project=POINT)
                a, b = int(batch.span_offset[p]), int(batch.span_offset[p + 1])
                assert torch.equal(H[a:b], H1), p
                assert torch.equal(batch.patch_slice(K, p), K1), p
        rep = batch.newton_step(C, C.clone())
        assert rep.status == 0 and rep.spans_projected == 0
        assert all(r.status == 0 for r in batch.patch_reports())
    finally:
        batch.close()
