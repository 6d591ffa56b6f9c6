"""Pins of the oracle's per-point projection of the FBW membrane Hessian.

The per-point variant projects, at every membrane quadrature point, the
Hessian of each FBW term (the two stretch terms and the shear term of
Eq. FBW stretching and shearing energy) w.r.t. (f_1, f_2) to PSD before the
chain rule (projected Newton, Sec. 5.1, with the eigenanalysis FBW admits,
Sec. 4.1); the bending Hessian is PSD by construction.

Pinned here: each term's raw 6x6 against central finite differences of its
energy density; each term's projection against LAPACK's eigensystem; the sum
over terms; the closed-form spectrum of the shear term; and at span level,
states where every term is PSD (no change), compression without shear (the
stretch term's projection is its Hessian at unit length), PSD-ness and
P - H >= 0 on random states.
"""
import numpy as np
import pytest

from paper_2506_18867_gb300 import inputs

MAT = (3.0, 5.0, 2.0, 0.0, 1.0)
TERMS = {"stretch1": (3.0, 0.0, 0.0, 0.0, 1.0), "stretch2": (0.0, 5.0, 0.0, 0.0, 1.0),
         "shear": (0.0, 0.0, 2.0, 0.0, 1.0)}


def _psi(f6, mat):
    f1, f2 = f6[:3], f6[3:]
    mu1, mu2, mush = mat[:3]
    return (mu1 * (np.linalg.norm(f1) - 1) ** 2 + mu2 * (np.linalg.norm(f2) - 1) ** 2
            + mush * (f1 @ f2) ** 2)


def _problem(orc, mat, rule=0):
    rest = inputs.flat_rest(7, 6, 0.5, 0.4, angle=0.3)
    return orc.Problem(7, 6, rest, mat, mem_rule=rule, bend_rule=rule)


def _clamp(H):
    lam, V = np.linalg.eigh(H)
    return (V * np.maximum(lam, 0.0)) @ V.T


def _states(rng, n=12):
    out = [np.array([1.2, 0.1, 0.0, -0.2, 0.9, 0.1]),      # f_2 compressed, sheared
           np.array([0.7, 0.0, 0.0, 0.0, 0.6, 0.0]),       # both compressed, I6 = 0
           np.array([1.0, 0.0, 0.0, -1.0, 0.0, 0.0])]      # f_1 + f_2 = 0
    out += [rng.standard_normal(6) * 0.6 + np.array([1, 0, 0, 0, 1, 0]) for _ in range(n)]
    return out


@pytest.mark.parametrize("term", sorted(TERMS))
def test_term_hessian_matches_finite_differences(orc, term):
    mat = TERMS[term]
    p = _problem(orc, mat)
    h = 1e-4
    for f6 in _states(np.random.default_rng(11), 4):
        A = p.fbw_hessian6(f6[:3], f6[3:])
        fd = np.zeros((6, 6))
        for i in range(6):
            for j in range(6):
                e_i, e_j = np.eye(6)[i] * h, np.eye(6)[j] * h
                fd[i, j] = (_psi(f6 + e_i + e_j, mat) - _psi(f6 + e_i - e_j, mat)
                            - _psi(f6 - e_i + e_j, mat) + _psi(f6 - e_i - e_j, mat)) / (4 * h * h)
        assert np.abs(A - fd).max() < 1e-6 * max(1.0, np.abs(A).max())


@pytest.mark.parametrize("term", sorted(TERMS))
def test_term_projection_matches_lapack(orc, term):
    p = _problem(orc, TERMS[term])
    for f6 in _states(np.random.default_rng(12)):
        A = p.fbw_hessian6(f6[:3], f6[3:])
        P = p.fbw_hessian6(f6[:3], f6[3:], point_project=True)
        assert np.abs(P - _clamp(A)).max() < 1e-12 * max(1.0, np.abs(A).max())


def test_projection_is_per_term(orc):
    """The full density's projected Hessian is the sum of the terms' projections,
    which differs from projecting the summed Hessian."""
    p = _problem(orc, MAT)
    per_term = [_problem(orc, m) for m in TERMS.values()]
    differs = 0
    for f6 in _states(np.random.default_rng(13)):
        P = p.fbw_hessian6(f6[:3], f6[3:], point_project=True)
        S = sum(q.fbw_hessian6(f6[:3], f6[3:], point_project=True) for q in per_term)
        assert np.abs(P - S).max() < 1e-12 * max(1.0, np.abs(S).max())
        differs += np.abs(P - _clamp(p.fbw_hessian6(f6[:3], f6[3:]))).max() > 1e-8
    assert differs > 0


@pytest.mark.parametrize("gamma", [0.3, -0.7, 1.5])
def test_shear_spectrum_closed_form(orc, gamma):
    """f_1 = e_1, f_2 = (gamma, 1, 0): the shear Hessian 2 mu_sh [g g^T + I6 A]
    has eigenvalues +-I6 (twice each) and (tr +- sqrt(tr^2 + 12 I6^2)) / 2 with
    tr = |f_1|^2 + |f_2|^2; its projection keeps the non-negative ones."""
    mush = TERMS["shear"][2]
    p = _problem(orc, TERMS["shear"])
    f1, f2 = np.array([1.0, 0.0, 0.0]), np.array([gamma, 1.0, 0.0])
    I6, tr = gamma, 2.0 + gamma * gamma
    sq = np.sqrt(tr * tr + 12 * I6 * I6)
    want = np.sort(2 * mush * np.array([I6, I6, -I6, -I6, (tr + sq) / 2, (tr - sq) / 2]))
    got = np.linalg.eigvalsh(p.fbw_hessian6(f1, f2))
    assert np.allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())
    gotp = np.linalg.eigvalsh(p.fbw_hessian6(f1, f2, point_project=True))
    assert np.allclose(gotp, np.sort(np.maximum(want, 0)), rtol=0, atol=1e-12 * np.abs(want).max())


def test_stretched_state_unchanged(orc):
    """Affine stretch s_b >= 1 along the material axes (I6 = 0): every term is
    PSD, so the per-point projection changes nothing."""
    rest = inputs.flat_rest(8, 7, 0.7, 0.6)
    p = orc.Problem(8, 7, rest, (30.0, 50.0, 20.0, 1e-3, 1.0))
    C = np.stack([1.1 * rest[:, 0], 1.05 * rest[:, 1], np.zeros(len(rest))], axis=1)
    _, _, H = p.span_eval(C)
    _, _, Hp = p.span_eval_projected(C, orc.PROJECT_POINT)
    assert np.abs(Hp - H).max() < 1e-12 * np.abs(H).max()


def test_compression_without_shear(orc):
    """mu_sh = 0, C = s X with s < 1: each stretch term's projected Hessian is
    2 mu f^ f^T, which is its raw Hessian at unit length along the same axis,
    so the projected span Hessians equal the raw ones of the rest state."""
    rest = inputs.flat_rest(8, 7, 0.7, 0.6, angle=0.5)
    p = orc.Problem(8, 7, rest, (30.0, 50.0, 0.0, 1e-3, 1.0))
    X = np.concatenate([rest, np.zeros((len(rest), 1))], axis=1)
    _, _, H_rest = p.span_eval(X)
    for s in (0.5, 0.9):
        _, _, Hp = p.span_eval_projected(s * X, orc.PROJECT_POINT)
        assert np.abs(Hp - H_rest).max() < 1e-12 * np.abs(H_rest).max()
        _, _, Hraw = p.span_eval(s * X)
        assert np.abs(Hraw - H_rest).max() > 1e-3 * np.abs(H_rest).max()


@pytest.mark.parametrize("rule", [0, 3])
def test_random_state_psd_and_above_raw(orc, rule):
    """P >= 0 and P - H >= 0 for every span; energy and gradient untouched."""
    pat = inputs.config_random_small(5, 8, 7, noise=0.3)
    p = orc.Problem.from_patch(pat, mem_rule=rule, bend_rule=rule)
    E, g, H = p.span_eval(pat.C)
    Ep, gp, Hp = p.span_eval_projected(pat.C, orc.PROJECT_POINT)
    assert np.array_equal(E, Ep) and np.array_equal(g, gp)
    neg = 0
    for s in range(p.n_spans):
        scale = np.abs(H[s]).max()
        assert np.linalg.eigvalsh(Hp[s]).min() > -1e-12 * scale
        assert np.linalg.eigvalsh(Hp[s] - H[s]).min() > -1e-12 * scale
        neg += np.linalg.eigvalsh(H[s]).min() < -1e-9 * scale
    assert neg > 0  # the state is compressed somewhere, so the test has teeth


def test_scene_modes_agree_with_span_terms(orc):
    """evaluate() with the per-point scene assembles the per-point span terms;
    the per-span mode projects the raw span Hessians."""
    pat = inputs.config_random_small(6, 7, 7, noise=0.2)
    p = orc.Problem.from_patch(pat)
    E1, g1, K1 = orc.evaluate(p, orc.Scene.from_patch(pat, project=orc.PROJECT_POINT), pat.C, pat.Chat)
    E0, g0, _ = orc.evaluate(p, orc.Scene.from_patch(pat, project=False), pat.C, pat.Chat)
    assert E1 == E0 and np.array_equal(g1, g0)
    rows = np.arange(pat.n_cp)
    gr, Kr = orc.eval_rows(p, orc.Scene.from_patch(pat, project=orc.PROJECT_POINT), pat.C, pat.Chat, rows)
    assert np.abs(Kr - K1).max() < 1e-12 * np.abs(K1).max()
    sp = np.arange(p.n_spans)
    _, _, Hs = orc.span_terms_subset(p, pat.C, sp, project=orc.PROJECT_POINT)
    _, _, Hp = p.span_eval_projected(pat.C, orc.PROJECT_POINT)
    assert np.abs(Hs - Hp).max() == 0.0
    _, _, Hsp = p.span_eval_projected(pat.C, orc.PROJECT_SPAN)
    _, _, Hsub = orc.span_terms_subset(p, pat.C, sp, project=True)
    assert np.abs(Hsp - Hsub).max() == 0.0
