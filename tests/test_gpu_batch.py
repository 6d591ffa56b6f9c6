"""Batched patches (many garments in one context): every phase runs once over
all patches, the PCG as one persistent launch split into per-patch block
groups, the Newton iteration under a captured CUDA graph.

- Batch vs one context per patch: span terms, gradient, assembled K, SpMV
  and energies are bitwise identical (the same per-element arithmetic, only
  the launch shape differs); PCG solutions and Newton positions agree to the
  solver tolerance (the reduction grouping of the block groups differs).
- Batch vs the FP64 oracle per patch: one projected Newton step, including a
  patch whose line search must halve alpha.
- Tile widths and the graph change nothing: bitwise.
- The 64-garment workload the bench times (FP32, autotuned): sampled spans
  and stencil rows of several patches against the oracle, and every patch's
  step report.
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
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def small_batch():
    """Four uneven patches across two tile classes: rotated, curved, different
    materials, pins and time steps; the last one is noisy enough that its
    line search rejects alpha = 1."""
    pats = [inputs.config_random_small(11, 9, 7),
            inputs.config_random_small(12, 12, 16, noise=0.1),
            inputs.config_random_small(13, 21, 11, curved=0.5, noise=0.05),
            inputs.config_random_small(14, 36, 40, noise=0.05)]
    pats[1].dt = 0.02
    pats[2].gravity = (0.0, 0.0, -9.81)
    return pats


def patch_vec(ctx, t, p):
    return ctx.patch_slice(t, p).detach().double().cpu().numpy()


def batch_tensor(ctx, arrays):
    """Concatenate per-patch (N_p, 3) arrays into the batch's (3, N) layout."""
    out = np.zeros((3, ctx.N))
    for p, a in enumerate(arrays):
        out[:, ctx.cp_offset[p]:ctx.cp_offset[p + 1]] = np.asarray(a).T
    return torch.from_numpy(out).to(device="cuda", dtype=ctx.dtype).contiguous()


@pytest.fixture(scope="module", params=[bsc.FP64, bsc.FP32], ids=["fp64", "fp32"])
def pair(request):
    prec = request.param
    pats = small_batch()
    batch = bsc.batch_for_patches(pats, precision=prec, pcg_rel_tol=1e-12 if prec == bsc.FP64 else 1e-6)
    singles = [bsc.context_for_patch(p, precision=prec, pcg_rel_tol=1e-12 if prec == bsc.FP64 else 1e-6)
               for p in pats]
    yield pats, batch, singles
    batch.close()
    for s in singles:
        s.close()


def test_layout(pair):
    pats, batch, _ = pair
    assert batch.P == len(pats)
    assert list(np.diff(batch.cp_offset)) == [p.n_cp for p in pats]
    assert list(np.diff(batch.span_offset)) == [p.n_spans for p in pats]
    assert batch.sizes()[0] == sum(p.n_cp for p in pats)


def test_span_terms_bitwise(pair):
    pats, batch, singles = pair
    C = batch_tensor(batch, [p.C for p in pats])
    E, g, H = batch.span_terms(C, project=True)
    for p, (pat, s) in enumerate(zip(pats, singles)):
        Es, gs, Hs = s.span_terms(s.to_device(pat.C), project=True)
        a, b = int(batch.span_offset[p]), int(batch.span_offset[p + 1])
        assert torch.equal(E[a:b], Es) and torch.equal(g[a:b], gs) and torch.equal(H[a:b], Hs), p


def test_gradient_hessian_spmv_energy_bitwise(pair):
    pats, batch, singles = pair
    C = batch_tensor(batch, [p.C for p in pats])
    Ch = batch_tensor(batch, [p.Chat for p in pats])
    g = batch.gradient(C, Ch)
    K = batch.assemble_hessian(C, project=True)
    x = torch.randn((3, batch.N), dtype=batch.dtype, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    y = batch.spmv(x, K=K)
    Eb = batch.patch_energies(C, Ch)
    assert abs(batch.energy(C, Ch) - sum(Eb)) <= 1e-15 * abs(sum(Eb)) + 1e-300
    for p, (pat, s) in enumerate(zip(pats, singles)):
        Cs, Chs = s.to_device(pat.C), s.to_device(pat.Chat)
        assert torch.equal(batch.patch_slice(g, p), s.gradient(Cs, Chs)), p
        Ks = s.assemble_hessian(Cs, project=True)
        assert torch.equal(batch.patch_slice(K, p), Ks), p
        xs = batch.patch_slice(x, p).contiguous()
        assert torch.equal(batch.patch_slice(y, p), s.spmv(xs, K=Ks)), p
        assert Eb[p] == s.energy(Cs, Chs), p


def test_solve_and_newton_match_single(pair):
    pats, batch, singles = pair
    tol = 1e-12 if batch.precision == bsc.FP64 else 1e-6
    C = batch_tensor(batch, [p.C for p in pats])
    Ch = batch_tensor(batch, [p.Chat for p in pats])
    K = batch.assemble_hessian(C, project=True)
    b = -batch.gradient(C, Ch)
    x, it, rr = batch.solve(b, K=K, rel_tol=tol)
    assert rr <= tol
    rep = batch.newton_step(C, Ch)
    reps = batch.patch_reports()
    for p, (pat, s) in enumerate(zip(pats, singles)):
        Cs, Chs = s.to_device(pat.C), s.to_device(pat.Chat)
        Ks = s.assemble_hessian(Cs, project=True)
        bs = -s.gradient(Cs, Chs)
        xs, _, _ = s.solve(bs, K=Ks, rel_tol=tol)
        assert rel(patch_vec(batch, x, p), xs.double().cpu().numpy()) < (1e-9 if tol < 1e-9 else 1e-4), p
        rs = s.newton_step(Cs, Chs)
        assert reps[p].E0 == rs.E0, p
        assert reps[p].alpha == rs.alpha and reps[p].ls_halvings == rs.ls_halvings, p
        width = np.ptp(pat.rest, axis=0).max()
        d = np.abs(patch_vec(batch, C, p) - Cs.double().cpu().numpy()).max()
        assert d <= (1e-10 if batch.precision == bsc.FP64 else 1e-5) * width, (p, d)
    assert rep.E0 == sum(r.E0 for r in reps)


def test_pipelined_pcg_batch_matches_three_barrier_form(pair):
    """Both PCG forms on the uneven batch (one block group per patch), FP64:
    every patch reaches the tolerance, and the solutions agree to it.  In
    FP32 the pipelined recurrences (u and w carried instead of recomputed)
    drift until (r, u) > 0 fails on the batch's slowest patch before 1e-6,
    and the solve reports BSC_ERR_NUMERIC; the autotuner then keeps the
    three-barrier form."""
    pats, batch, _ = pair
    if batch.precision == bsc.FP32:
        pytest.skip("the pipelined form is not used in FP32 on this batch (see the docstring)")
    tol = 1e-12
    C = batch_tensor(batch, [p.C for p in pats])
    Ch = batch_tensor(batch, [p.Chat for p in pats])
    K = batch.assemble_hessian(C, project=True)
    b = -batch.gradient(C, Ch)
    x0, it0, rr0 = batch.solve(b, K=K, rel_tol=tol)
    batch.set_pcg_form(1)
    try:
        x1, it1, rr1 = batch.solve(b, K=K, rel_tol=tol)
    finally:
        batch.set_pcg_form(0)
    print(f"batch solve: three-barrier {it0} iterations, pipelined {it1}")
    assert rr1 <= tol
    for p in range(len(pats)):
        assert rel(patch_vec(batch, x1, p), patch_vec(batch, x0, p)) < (1e-9 if tol < 1e-9 else 1e-4), p


def test_two_pass_pcg_batch_matches_three_barrier_form(pair):
    """The two-pass PCG form (q = K z + beta q carried by a recurrence) on the
    uneven batch, FP64 and FP32: every patch reaches the tolerance and the
    solutions agree with the three-barrier form's to it."""
    pats, batch, _ = pair
    tol = 1e-12 if batch.precision == bsc.FP64 else 1e-6
    C = batch_tensor(batch, [p.C for p in pats])
    Ch = batch_tensor(batch, [p.Chat for p in pats])
    K = batch.assemble_hessian(C, project=True)
    b = -batch.gradient(C, Ch)
    x0, it0, rr0 = batch.solve(b, K=K, rel_tol=tol)
    batch.set_pcg_form(2)
    try:
        x2, it2, rr2 = batch.solve(b, K=K, rel_tol=tol)
    finally:
        batch.set_pcg_form(0)
    worst = max(rel(patch_vec(batch, x2, p), patch_vec(batch, x0, p)) for p in range(len(pats)))
    print(f"batch solve: three-barrier {it0} iterations, two-pass {it2}; largest relative difference {worst:.2e}")
    assert rr2 <= tol
    assert worst < (1e-9 if batch.precision == bsc.FP64 else 1e-4)


def test_symmetric_storage_same_batch_step(pair):
    """The batch's Newton step with the symmetric and with the full matrix
    layout: bitwise the same positions and per-patch reports (FP64, FP32)."""
    pats, batch, _ = pair
    res = []
    try:
        for sym in (False, True):
            batch.set_k_storage(sym)
            C = batch_tensor(batch, [p.C for p in pats])
            batch.newton_step(C, batch_tensor(batch, [p.Chat for p in pats]))
            res.append((C, [r.as_dict() for r in batch.patch_reports()]))
    finally:
        batch.set_k_storage(True)
    assert torch.equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1]


def test_newton_step_against_oracle(orc):
    """FP64 batch: every patch's Newton step against the oracle's (banded
    Cholesky solve), including the line-search halvings."""
    pats = small_batch()
    pats[3] = inputs.config_random_small(16, 14, 12, noise=0.3)  # the oracle halves alpha 3 times
    batch = bsc.batch_for_patches(pats, precision=bsc.FP64, pcg_rel_tol=1e-13)
    C = batch_tensor(batch, [p.C for p in pats])
    Ch = batch_tensor(batch, [p.Chat for p in pats])
    st, rep = batch.newton_step_status(C, Ch)
    reps = batch.patch_reports()
    halved = 0
    for p, pat in enumerate(pats):
        prob = orc.Problem.from_patch(pat)
        sc = orc.Scene.from_patch(pat, project=True)
        oC, orep = orc.newton_step(prob, sc, pat.C, pat.Chat, solver=0)
        assert orep.status == 0 and reps[p].status == 0, (p, reps[p].status)
        assert reps[p].alpha == orep.alpha and reps[p].ls_halvings == orep.ls_halvings, p
        assert abs(reps[p].E0 - orep.E0) <= 1e-11 * abs(orep.E0)
        width = np.ptp(pat.rest, axis=0).max()
        assert np.abs(patch_vec(batch, C, p).T - oC).max() <= 1e-10 * width, p
        halved += reps[p].ls_halvings > 0
    assert st == bsc.OK
    assert halved >= 1, "the noisy patch should exercise a second line-search round"
    batch.close()


@pytest.mark.parametrize("tiles", [(8, 8, 8, 8), (16, 32, 16, 32), (32, 16, 0, 8)])
def test_tile_widths_bitwise(pair, tiles):
    pats, batch, _ = pair
    C = batch_tensor(batch, [p.C for p in pats])
    batch.set_tiles((0, 0, 0, 0))
    E0, g0, H0 = batch.span_terms(C, project=True)
    batch.set_tiles(tiles)
    E1, g1, H1 = batch.span_terms(C, project=True)
    batch.set_tiles((0, 0, 0, 0))
    assert torch.equal(E0, E1) and torch.equal(g0, g1) and torch.equal(H0, H1)


def test_graph_replay_matches_direct():
    pats = small_batch()
    a = bsc.batch_for_patches(pats, precision=bsc.FP32)
    b = bsc.batch_for_patches(pats, precision=bsc.FP32)
    b.set_graph(False)
    Ca, Cb = batch_tensor(a, [p.C for p in pats]), batch_tensor(b, [p.C for p in pats])
    Ch = batch_tensor(a, [p.Chat for p in pats])
    for _ in range(3):
        ra = a.newton_step(Ca, Ch)
        rb = b.newton_step(Cb, Ch)
        assert ra.E0 == rb.E0 and ra.E1 == rb.E1
    assert torch.equal(Ca, Cb)
    gs = a.graph_state()
    assert gs["on"] == 1 and gs["captured"] == 1 and gs["replays"] == 3
    assert b.graph_state()["captured"] == 0
    a.close()
    b.close()


@pytest.mark.parametrize("graph", [True, False])
def test_phase_times_under_graph(graph):
    pats = small_batch()
    ctx = bsc.batch_for_patches(pats, precision=bsc.FP32)
    ctx.set_graph(graph)
    ctx.set_profiling(True)
    C = batch_tensor(ctx, [p.C for p in pats])
    Ch = batch_tensor(ctx, [p.Chat for p in pats])
    for _ in range(2):
        ctx.newton_step(C, Ch)
        ph = ctx.phase_times()
        assert all(v > 0.0 for v in ph.values()), ph
        parts = sum(v for k, v in ph.items() if k != "total")
        assert abs(parts - ph["total"]) <= 1e-3 * ph["total"] + 2e-3, ph
    assert ctx.graph_state()["captured"] == int(graph)
    ctx.close()


def test_autotune_choices(pair):
    pats, batch, _ = pair
    C = batch_tensor(batch, [p.C for p in pats])
    Ch = batch_tensor(batch, [p.Chat for p in pats])
    t = batch.autotune(C, Ch)
    classes = {0 if p.nu - 2 < 32 else (1 if p.nu - 2 < 64 else 2) for p in pats}
    for k in range(4):
        if k in classes:
            assert t["tile_tu"][k] in bsc.TILE_CANDIDATES
            assert all(ms > 0 for ms in t["tile_ms"][k])
        else:
            assert t["tile_tu"][k] == -1
    split = batch.pcg_split()
    assert sum(split) == t["pcg_grid"] and min(split) >= 1
    assert t["p2_variant"] in (0, 1) and all(ms > 0 for ms in t["p2_ms"])
    assert t["psd_test"] in (0, 1, 2) and all(ms > 0 for ms in t["psd_ms"])
    assert t["pcg_form"] in (0, 1, 2) and min(t["pcg_form_ms"]) == t["pcg_form_ms"][t["pcg_form"]]
    # both occupancy variants of the projection's eigenpair phase: bitwise the same
    outs = []
    for v in (0, 1):
        batch.set_p2_variant(v)
        E, g, H = batch.span_terms(C, project=True)
        outs.append(H.cpu())
    assert torch.equal(outs[0], outs[1])
    batch.set_p2_variant(t["p2_variant"])
    batch.set_tiles((0, 0, 0, 0))
    # PCG grid: the chosen candidate is the fastest measured one; every grid
    # solves the same system to the same tolerance
    ms = [m for m in t["pcg_ms"] if m >= 0]
    assert t["pcg_grid"] in t["pcg_grid_cand"] and min(ms) == t["pcg_ms"][t["pcg_grid_cand"].index(t["pcg_grid"])]
    K = batch.assemble_hessian(C, project=True)
    b = -batch.gradient(C, Ch)
    fp64 = batch.dtype == torch.float64
    tol = 1e-10 if fp64 else 1e-6
    sols = []
    for gsz in sorted(set(t["pcg_grid_cand"])):
        batch.set_pcg_grid(gsz)
        assert sum(batch.pcg_split()) == gsz
        x, it, rr = batch.solve(b, K=K, rel_tol=tol)
        assert rr <= tol
        sols.append(x.double().cpu())
    for x in sols[1:]:
        assert float((x - sols[0]).norm() / sols[0].norm()) < (1e-7 if fp64 else 1e-3)
    with pytest.raises(bsc.BscError):
        batch.set_pcg_grid(len(pats) - 1)
    batch.set_pcg_grid(t["pcg_grid"])


def test_batch64_workload(orc):
    """The 64-garment workload in the bench's configuration (FP32, autotuned,
    graph): a Newton step succeeds for every patch, and sampled span terms and
    stencil rows of four patches match the oracle."""
    pats = inputs.config_batch(1)
    ctx = bsc.batch_for_patches(pats, precision=bsc.FP32, pcg_rel_tol=1e-8)
    C = batch_tensor(ctx, [p.C for p in pats])
    Ch = batch_tensor(ctx, [p.Chat for p in pats])
    ctx.autotune(C, Ch)
    rng = np.random.default_rng(7)
    for p in (0, 1, 17, 63):
        pat = pats[p]
        prob = orc.Problem.from_patch(pat)
        scene = orc.Scene.from_patch(pat, project=True)
        Su, Sv = pat.nu - 2, pat.nv - 2
        spans = np.unique(np.concatenate([[0, Su - 1, Su * Sv - 1], rng.integers(0, Su * Sv, 20)])).astype(np.int32)
        E, g, H = ctx.span_terms(C, project=True)
        sp = torch.as_tensor(spans + int(ctx.span_offset[p]), device="cuda", dtype=torch.long)
        oE, og, oH = orc.span_terms_subset(prob, pat.C, spans, project=True)
        assert rel(H[sp].double().cpu().numpy(), oH) < 2e-5, p
        assert rel(g[sp].double().cpu().numpy(), og) < 1e-4, p
        rows = np.unique(np.concatenate([pat.pinned, rng.integers(0, pat.n_cp, 20)])).astype(np.int32)
        K = ctx.assemble_hessian(C, project=True)
        Kr = K[:, torch.as_tensor(rows + int(ctx.cp_offset[p]), device="cuda", dtype=torch.long)]
        Kr = Kr.double().cpu().numpy().reshape(25, 3, 3, -1).transpose(3, 0, 1, 2)
        _, oKr = orc.eval_rows(prob, scene, pat.C, pat.Chat, rows)
        assert rel(Kr, oKr) < 2e-5, p
        del E, g, H, K
    rep = ctx.newton_step(C, Ch)
    reps = ctx.patch_reports()
    assert rep.status == 0
    assert all(r.status == 0 and r.E1 <= r.E0 and r.pcg_rel_res <= 1e-8 for r in reps)
    assert ctx.graph_state()["captured"] == 1
    ctx.close()
