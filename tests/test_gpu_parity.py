"""GPU path (through the C ABI) against the FP64 CPU oracle.

FP64 parity bar: 1e-12 relative, norm-wise, on gradients, span Hessians and
the assembled stencil Hessian (the tolerance the method's FP64 path is held
to); tables and masses 1e-13.  FP32 results state their error against the
oracle and are held to bounds derived from FP32 rounding (about 1e-7 per
operation, amplified by the span-level cancellation of the strain).
"""
import numpy as np
import pytest

from paper_2506_18867_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - the gpu marker deselects these on CPU hosts
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2506_18867_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2506_18867_gb300 import bsc  # noqa: E402


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def to_n3(t):
    return t.detach().double().cpu().numpy().reshape(3, -1).T.copy()


def gpu_K_to_oracle(K, N):
    """(225, N) planes -> (N, 25, 3, 3)."""
    return K.detach().double().cpu().numpy().reshape(25, 3, 3, N).transpose(3, 0, 1, 2).copy()


CASES = [
    ("square32", lambda: inputs.config_square(1, 32)),
    ("rand5x5", lambda: inputs.config_random_small(2, 5, 5)),
    ("rand6x9", lambda: inputs.config_random_small(3, 6, 9, noise=0.2)),
    ("rand13x7_curved", lambda: inputs.config_random_small(4, 13, 7, curved=0.6, noise=0.1)),
    ("rand40x23", lambda: inputs.config_random_small(5, 40, 23, noise=0.05)),
    # non-rectangular rest domains (Sec. 6): the most distorted case of each family
    ("aspect10", lambda: inputs.config_distorted("aspect", 10, 24, 24)),
    ("skew30", lambda: inputs.config_distorted("skew", 30, 24, 24)),
    ("bend105", lambda: inputs.config_distorted("bend", 105, 24, 24)),
]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request, orc):
    pat = request.param[1]()
    prob = orc.Problem.from_patch(pat)
    ctx = bsc.context_for_patch(pat, precision=bsc.FP64, pcg_rel_tol=1e-13)
    yield pat, prob, ctx
    ctx.close()


def _sorted_records(rec):
    key = np.lexsort((np.round(rec[:, 0], 9), np.round(rec[:, 1], 9), rec[:, 3], rec[:, 4]))
    return rec[key]


@pytest.mark.parametrize("which", [0, 1])
def test_quadrature_tables(case, which):
    pat, prob, ctx = case
    g = _sorted_records(ctx.quadrature_tables(which))
    o_pts = prob.quad_points(which)
    o_tab = prob.point_tables(which)
    o = _sorted_records(np.concatenate([o_pts, o_tab], axis=1))
    assert g.shape[0] == o.shape[0]
    np.testing.assert_array_equal(g[:, 3:5], o[:, 3:5])          # owner spans, exact
    np.testing.assert_array_equal(g[:, 24], g[:, 4] * (pat.nu - 2) + g[:, 3])  # context-wide span index
    np.testing.assert_allclose(g[:, 0:3], o[:, 0:3], rtol=0, atol=1e-14)
    np.testing.assert_allclose(g[:, 5], o[:, 5], rtol=1e-13)     # W = w |det J|
    ncol = 18 if which == 0 else 9
    assert rel(g[:, 6:6 + ncol], o[:, 6:6 + ncol]) < 1e-13


def test_lumped_mass(case):
    pat, prob, ctx = case
    assert rel(ctx.lumped_mass(), prob.lumped_mass()) < 1e-13


@pytest.mark.parametrize("project,border_path", [(False, 0), (True, 0), (True, 1), (True, 2), (True, 3)],
                         ids=["raw", "proj-warp", "proj-thread", "proj-warp-items", "proj-warp-two-pass"])
def test_span_terms_fp64(case, project, border_path):
    """Span terms against the oracle; projected by every path of the border
    spans (one warp per span; one thread per span; one warp per span to the
    tridiagonal form, then one thread per eigenpair; one warp per span for
    the PSD test, then one warp per failing span)."""
    pat, prob, ctx = case
    C = ctx.to_device(pat.C)
    ctx.set_border_path(border_path)
    E, g, H = ctx.span_terms(C, project=project)
    ctx.set_border_path(0)
    oE, og, oH = prob.span_eval(pat.C)
    if project:
        from oracle import project_psd
        oH = np.stack([project_psd(h)[0] for h in oH])
    assert rel(E.cpu().numpy(), oE) < 1e-12
    assert rel(g.cpu().numpy(), og) < 1e-12
    assert rel(H.cpu().numpy(), oH) < 1e-12
    Hg = H.cpu().numpy()
    assert np.abs(Hg - Hg.transpose(0, 2, 1)).max() == 0.0


def test_energy_gradient_hessian_fp64(case, orc):
    pat, prob, ctx = case
    sc = orc.Scene.from_patch(pat, project=True)
    oE, og, oK = orc.evaluate(prob, sc, pat.C, pat.Chat)
    C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
    E = ctx.energy(C, Ch)
    assert abs(E - oE) <= 1e-12 * max(abs(oE), 1e-30) * 10
    g = to_n3(ctx.gradient(C, Ch))
    assert rel(g, og) < 1e-12
    K = gpu_K_to_oracle(ctx.assemble_hessian(C, project=True), pat.n_cp)
    assert rel(K, oK) < 1e-12
    sc0 = orc.Scene.from_patch(pat, project=False)
    _, _, oK0 = orc.evaluate(prob, sc0, pat.C, pat.Chat, want_g=False)
    K0 = gpu_K_to_oracle(ctx.assemble_hessian(C, project=False), pat.n_cp)
    assert rel(K0, oK0) < 1e-12


def test_spmv_and_solve_fp64(case, orc):
    pat, prob, ctx = case
    sc = orc.Scene.from_patch(pat, project=True)
    _, og, oK = orc.evaluate(prob, sc, pat.C, pat.Chat)
    C = ctx.to_device(pat.C)
    Kd = ctx.assemble_hessian(C, project=True)
    x = np.random.default_rng(7).standard_normal((pat.n_cp, 3))
    y = to_n3(ctx.spmv(ctx.to_device(x), K=Kd))
    assert rel(y, orc.stencil_matvec(pat.nu, pat.nv, oK, x)) < 1e-13
    b = -og
    xs, it, rr = ctx.solve(ctx.to_device(b), K=Kd, rel_tol=1e-13)
    assert rr <= 1e-13 and it > 0
    want = orc.solve_banded(pat.nu, pat.nv, oK, b) if pat.n_cp <= 4096 else orc.solve_pcg(
        pat.nu, pat.nv, oK, b, 1e-14)[0]
    assert rel(to_n3(xs), want) < 1e-10


def test_psd_test_changes_nothing(case, orc):
    """The FP64 LDL^T PSD test before the eigendecomposition skips the spans
    with no eigenvalue below -1e-14 ||H_r||: projected span Hessians with and
    without it agree to 1e-13 and both match the oracle's Jacobi projection;
    the spans it lets through are those without a projected eigenvalue (up
    to spans whose smallest eigenvalue lies within the thresholds' band).
    The FP32 certificate in front of it changes nothing, bit for bit."""
    pat, prob, ctx = case
    C = ctx.to_device(pat.C)
    try:
        ctx.set_psd_test(0)
        E0, g0, H0 = ctx.span_terms(C, project=True)
        nneg0, _ = ctx.projection_stats()
        ctx.set_psd_test(1)
        E1, g1, H1 = ctx.span_terms(C, project=True)
        nneg1, _ = ctx.projection_stats()
        cnt1 = ctx.psd_counts()
        ctx.set_psd_test(2)
        E2, g2, H2 = ctx.span_terms(C, project=True)
        nneg2, _ = ctx.projection_stats()
        cnt2 = ctx.psd_counts()
    finally:
        ctx.set_psd_test(2)
    _, _, oH = prob.span_eval_projected(pat.C, True)
    H0h, H1h = H0.double().cpu().numpy(), H1.double().cpu().numpy()
    print(f"{pat.name}: {int((nneg0 > 0).sum())} of {pat.n_spans} spans projected; with / without the test "
          f"{rel(H1h, H0h):.1e}; interior spans {cnt2[0]}, FP64-tested after the FP32 certificate {cnt2[1]}, "
          f"eigendecomposed {cnt2[2]}")
    assert rel(H1h, H0h) < 1e-13 and rel(H1h, oH) < 1e-12
    # the FP32 certificate only skips spans the FP64 test would pass: bitwise the same
    assert torch.equal(H1, H2) and np.array_equal(nneg1, nneg2)
    assert cnt1[0] == cnt2[0] and cnt1[1] == cnt1[0] and cnt1[2] == cnt2[2] and cnt2[2] <= cnt2[1] <= cnt2[0]
    # the two decisions use thresholds of the same size on different norms:
    # only spans whose smallest eigenvalue sits within that band may differ
    assert int(((nneg0 > 0) != (nneg1 > 0)).sum()) <= max(1, pat.n_spans // 1000)


@pytest.mark.parametrize("path", [0, 1, 2, 3], ids=["warp", "thread", "warp_items", "warp_two_pass"])
def test_border_psd_test_changes_nothing(case, orc, path):
    """Every border path with the FP64 PSD test in front (the phase kernels'
    thread-per-span test on path 1, the warp's own LDL^T on paths 0, 2 and
    3): the projected span Hessians agree with the path without it to 1e-13
    and with the oracle's Jacobi projection to 1e-12.  The warp paths' FP32
    certificate in front of the test (mode 2) changes nothing, bit for bit,
    and leaves at least the failing spans to the FP64 test."""
    pat, prob, ctx = case
    C = ctx.to_device(pat.C)
    out, raw, cnt = {}, {}, {}
    try:
        ctx.set_border_path(path)
        for mode in (0, 1, 2):
            ctx.set_psd_test(mode)
            raw[mode] = ctx.span_terms(C, project=True)[2]
            out[mode] = raw[mode].double().cpu().numpy()
            cnt[mode] = ctx.psd_counts()
    finally:
        ctx.set_psd_test(2)
        ctx.set_border_path(0)
    _, _, oH = prob.span_eval_projected(pat.C, True)
    print(f"{pat.name}: border path {path} with / without the test {rel(out[1], out[0]):.1e}, vs oracle "
          f"{rel(out[1], oH):.1e}; border spans {cnt[2][3]}, FP64-tested after the certificate {cnt[2][5]}, "
          f"eigendecomposed {cnt[2][4]}")
    assert rel(out[1], out[0]) < 1e-13 and rel(out[1], oH) < 1e-12
    assert torch.equal(raw[1], raw[2])
    assert cnt[1][5] == cnt[1][3] and cnt[1][4] == cnt[2][4] and cnt[2][4] <= cnt[2][5] <= cnt[2][3]
    if path == 1:
        assert cnt[2][5] == cnt[2][3]


@pytest.mark.parametrize("form", [1, 2], ids=["pipelined", "two_pass"])
def test_pcg_forms_fp64(case, orc, form):
    """The pipelined PCG form (one group barrier per iteration) and the
    two-pass form (q = K z + beta q) reach the same solution as the oracle's
    direct solve, and their Newton steps the oracle's positions, at the
    bounds of the three-barrier form."""
    pat, prob, ctx = case
    sc = orc.Scene.from_patch(pat, project=True)
    _, og, oK = orc.evaluate(prob, sc, pat.C, pat.Chat)
    C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
    Kd = ctx.assemble_hessian(C, project=True)
    b = -og
    _, it0, _ = ctx.solve(ctx.to_device(b), K=Kd, rel_tol=1e-13)
    ctx.set_pcg_form(form)
    try:
        xs, it, rr = ctx.solve(ctx.to_device(b), K=Kd, rel_tol=1e-13)
        assert rr <= 1e-13 and it > 0
        want = orc.solve_banded(pat.nu, pat.nv, oK, b) if pat.n_cp <= 4096 else orc.solve_pcg(
            pat.nu, pat.nv, oK, b, 1e-14)[0]
        e = rel(to_n3(xs), want)
        true_res = rel(orc.stencil_matvec(pat.nu, pat.nv, oK, to_n3(xs)), b)
        print(f"{pat.name}: PCG form {form} {it} iterations (three-barrier form {it0}), solution {e:.2e}, "
              f"true residual {true_res:.2e}")
        assert e < 1e-10 and true_res < 1e-11
        oC, orep = orc.newton_step(prob, sc, pat.C, pat.Chat, solver=0 if pat.n_cp <= 4096 else 1, pcg_tol=1e-14)
        rep = ctx.newton_step(C, Ch)
        assert rep.status == 0 and rep.alpha == orep.alpha
        width = np.ptp(pat.rest, axis=0).max()
        assert np.abs(to_n3(C) - oC).max() <= 1e-10 * width
    finally:
        ctx.set_pcg_form(0)


def test_symmetric_storage_same_newton_step(case):
    """The Newton step's matrix in the symmetric layout (13 slots, the
    default) and in the full one (25) give the same step bit for bit: the
    product reads the same entries in the same order.  After the step, a
    product with the step's own matrix (K = None) equals one with the full
    matrix assembled at the same state, up to the stand-alone full-layout
    product's own accumulation order (three FMA chains per row)."""
    pat, prob, ctx = case
    out = {}
    try:
        for sym in (False, True):
            ctx.set_k_storage(sym)
            C = ctx.to_device(pat.C)
            rep = ctx.newton_step(C, ctx.to_device(pat.Chat))
            out[sym] = (C, rep.as_dict())
        x = ctx.to_device(np.random.default_rng(7).standard_normal((pat.n_cp, 3)))
        y_sym = ctx.spmv(x)            # the last Newton step's matrix (symmetric layout)
        Kf = ctx.assemble_hessian(ctx.to_device(pat.C), project=True)
        y_full = ctx.spmv(x, K=Kf)
    finally:
        ctx.set_k_storage(True)
    assert torch.equal(out[False][0], out[True][0])
    assert out[False][1] == out[True][1]
    e = (torch.linalg.norm(y_sym - y_full) / torch.linalg.norm(y_full)).item()
    print(f"{pat.name}: product with the step's symmetric matrix vs the full one: {e:.1e}")
    assert e < 1e-14


def test_newton_step_matrix_equals_assembled(case):
    """The Newton step's own matrix (full layout; its assembly also writes the
    block-Jacobi inverses) equals the one bsc_assemble_hessian builds at the
    same state, bit for bit (compared through a product with each)."""
    pat, prob, ctx = case
    try:
        ctx.set_k_storage(False)
        C = ctx.to_device(pat.C)
        ctx.newton_step(C, ctx.to_device(pat.Chat))
        x = ctx.to_device(np.random.default_rng(11).standard_normal((pat.n_cp, 3)))
        y_step = ctx.spmv(x)
        Kf = ctx.assemble_hessian(ctx.to_device(pat.C), project=True)
        y_sep = ctx.spmv(x, K=Kf)
    finally:
        ctx.set_k_storage(True)
    assert torch.equal(y_step, y_sep)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_energy_kernel_matches_full_evaluation(case, precision):
    """bsc_energy runs the thread-per-span energy kernel; the Newton step's E0
    comes from the full span evaluation (gradient and Hessian) at the same
    state through the same reductions: the two are equal bit for bit."""
    pat, prob, ctx64 = case
    ctx = ctx64 if precision == "fp64" else bsc.context_for_patch(pat, precision=bsc.FP32)
    try:
        C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
        E = ctx.energy(C, Ch)
        rep = ctx.newton_step(C, Ch)
        assert E == rep.E0
    finally:
        if ctx is not ctx64:
            ctx.close()


def test_newton_step_fp64(case, orc):
    pat, prob, ctx = case
    sc = orc.Scene.from_patch(pat, project=True)
    oC, orep = orc.newton_step(prob, sc, pat.C, pat.Chat, solver=0 if pat.n_cp <= 4096 else 1, pcg_tol=1e-14)
    C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
    rep = ctx.newton_step(C, Ch)
    assert rep.status == 0 and orep.status == 0
    assert rep.alpha == orep.alpha
    assert abs(rep.E0 - orep.E0) <= 1e-12 * abs(orep.E0) * 10
    width = np.ptp(pat.rest, axis=0).max()
    assert np.abs(to_n3(C) - oC).max() <= 1e-10 * width
    assert rel(to_n3(C) - pat.C, oC - pat.C) < 1e-9


@pytest.mark.parametrize("border_path", [0, 1], ids=["warp", "thread"])
def test_double_float_projection_fp64(case, orc, border_path):
    """The projection's PSD test and phase 1 in double-float arithmetic (pairs
    of FP32 numbers, about 48 bits) in an FP64 context: with and without the
    PSD test, the projected span Hessians match the oracle's Jacobi
    projection to 1e-12 and the FP64 arithmetic's result to 1e-12 (border
    path 1 runs the border class through the same thread-per-span phases
    with D = 8), and the Newton step reaches the oracle's positions at the
    FP64 step's bounds."""
    pat, prob, ctx = case
    C = ctx.to_device(pat.C)
    out = {}
    try:
        ctx.set_border_path(border_path)
        for df in (0, 1):
            ctx.set_proj_arith(df)
            for mode in (0, 2):
                ctx.set_psd_test(mode)
                out[df, mode] = ctx.span_terms(C, project=True)[2].double().cpu().numpy()
        ctx.set_psd_test(2)
        ctx.set_proj_arith(1)
        sc = orc.Scene.from_patch(pat, project=True)
        oC, orep = orc.newton_step(prob, sc, pat.C, pat.Chat, solver=0 if pat.n_cp <= 4096 else 1, pcg_tol=1e-14)
        Cs = ctx.to_device(pat.C)
        rep = ctx.newton_step(Cs, ctx.to_device(pat.Chat))
    finally:
        ctx.set_proj_arith(0)
        ctx.set_psd_test(2)
        ctx.set_border_path(0)
    _, _, oH = prob.span_eval_projected(pat.C, True)
    errs = {k: rel(v, oH) for k, v in out.items()}
    print(f"{pat.name}: border path {border_path}, vs oracle (arith, psd mode): "
          + ", ".join(f"{k}: {e:.1e}" for k, e in errs.items())
          + f"; double-float vs FP64 {rel(out[1, 2], out[0, 2]):.1e}")
    assert max(errs.values()) < 1e-12
    assert rel(out[1, 2], out[0, 2]) < 1e-12 and rel(out[1, 0], out[0, 0]) < 1e-12
    assert rep.status == 0 and rep.alpha == orep.alpha
    width = np.ptp(pat.rest, axis=0).max()
    assert np.abs(to_n3(Cs) - oC).max() <= 1e-10 * width


def test_double_float_projection_fp32():
    """In an FP32 context (double-float by default) the FP32 certificate in
    front of the double-float PSD test changes nothing, bit for bit; against
    the FP64 arithmetic the projected span Hessians differ at the FP32
    storage's rounding only, on a state with many indefinite spans."""
    pat = inputs.config_wrinkle(1, 64, 0.25)
    with bsc.context_for_patch(pat, precision=bsc.FP32) as ctx:
        C = ctx.to_device(pat.C)
        H = {}
        for df in (1, 0):
            ctx.set_proj_arith(df)
            for mode in (1, 2):
                ctx.set_psd_test(mode)
                H[df, mode] = ctx.span_terms(C, project=True)[2]
                if df == 1 and mode == 2:
                    nneg = ctx.projection_stats()[0]
        assert torch.equal(H[1, 1], H[1, 2]) and torch.equal(H[0, 1], H[0, 2])
        e = rel(H[1, 2].double().cpu().numpy(), H[0, 2].double().cpu().numpy())
        print(f"wrinkle 64x64 FP32: {int((nneg > 0).sum())} of {pat.n_spans} spans projected; "
              f"double-float vs FP64 arithmetic {e:.1e}")
        assert int((nneg > 0).sum()) > pat.n_spans // 50
        assert e < 1e-6


def test_deterministic_bitwise(case):
    pat, prob, ctx = case
    C = ctx.to_device(pat.C)
    K1 = ctx.assemble_hessian(C, project=True).clone()
    K2 = ctx.assemble_hessian(C, project=True)
    assert torch.equal(K1, K2)
    g1 = ctx.gradient(C, ctx.to_device(pat.Chat)).clone()
    assert torch.equal(g1, ctx.gradient(C, ctx.to_device(pat.Chat)))


@pytest.mark.parametrize("rule", [2, 3, 4])
def test_full_gauss_rules(orc, rule):
    pat = inputs.config_random_small(8, 9, 11, noise=0.1)
    prob = orc.Problem.from_patch(pat, mem_rule=rule, bend_rule=rule)
    with bsc.context_for_patch(pat, precision=bsc.FP64, quadrature=(rule, rule)) as ctx:
        E, g, H = ctx.span_terms(ctx.to_device(pat.C), project=False)
        oE, og, oH = prob.span_eval(pat.C)
        assert rel(g.cpu().numpy(), og) < 1e-12 and rel(H.cpu().numpy(), oH) < 1e-12


@pytest.mark.parametrize("rule", [3, 4])
def test_gauss_rules_projected(orc, rule):
    """Projected span terms under the full 3x3 Gauss rule and the ablation rule
    (2x2 Gauss on interior spans): every interior span then falls in the 24x24
    class; both projections against the oracle."""
    from oracle import project_psd
    pat = inputs.config_random_small(9, 9, 8, noise=0.2)
    prob = orc.Problem.from_patch(pat, mem_rule=rule, bend_rule=rule)
    _, _, oH = prob.span_eval(pat.C)
    oHs = np.stack([project_psd(h)[0] for h in oH])
    _, _, oHp = prob.span_eval_projected(pat.C, orc.PROJECT_POINT)
    with bsc.context_for_patch(pat, precision=bsc.FP64, quadrature=(rule, rule)) as ctx:
        C = ctx.to_device(pat.C)
        for path in (0, 1, 2, 3):
            ctx.set_border_path(path)
            _, _, H = ctx.span_terms(C, project=bsc.PROJECT_SPAN)
            assert rel(H.cpu().numpy(), oHs) < 1e-12, path
        _, _, H = ctx.span_terms(C, project=bsc.PROJECT_POINT)
        assert rel(H.cpu().numpy(), oHp) < 1e-12


def test_fp32_errors_against_oracle(orc):
    """FP32 span evaluation / assembly with the FP64 projection: error stated."""
    pat = inputs.config_square(1, 32)
    prob = orc.Problem.from_patch(pat)
    sc = orc.Scene.from_patch(pat, project=True)
    oE, og, oK = orc.evaluate(prob, sc, pat.C, pat.Chat)
    with bsc.context_for_patch(pat, precision=bsc.FP32) as ctx:
        C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
        E = ctx.energy(C, Ch)
        g = to_n3(ctx.gradient(C, Ch))
        K = gpu_K_to_oracle(ctx.assemble_hessian(C, project=True), pat.n_cp)
        eg, eK = rel(g, og), rel(K, oK)
        print(f"FP32 vs oracle: energy {abs(E - oE) / abs(oE):.2e} gradient {eg:.2e} hessian {eK:.2e}")
        assert abs(E - oE) / abs(oE) < 1e-5 and eg < 1e-4 and eK < 1e-5


def test_bad_device_arguments():
    pat = inputs.config_random_small(2, 6, 6)
    with bsc.context_for_patch(pat, precision=bsc.FP64) as ctx:
        x = ctx.new_vec()
        with pytest.raises(bsc.BscError) as ei:
            ctx._check(ctx._lib.bsc_spmv(ctx._h, None, bsc._ptr(x), bsc._ptr(x)))
        assert ei.value.status == bsc.ERR_INVALID_ARG
        with pytest.raises(bsc.BscError) as ei:
            ctx._check(ctx._lib.bsc_energy(ctx._h, bsc._ptr(x), None, None))
        assert ei.value.status == bsc.ERR_INVALID_ARG
        C = ctx.to_device(pat.C)
        C[0, 3] = float("nan")
        with pytest.raises(bsc.BscError) as ei:
            ctx.energy(C, ctx.to_device(pat.Chat))
        assert ei.value.status == bsc.ERR_NUMERIC
        # the context stays usable after a reported error
        assert np.isfinite(ctx.energy(ctx.to_device(pat.C), ctx.to_device(pat.Chat)))
