"""Pins of the oracle's energies, derivatives, projection, assembly and Newton step.

Closed forms: affine deformations integrate the FBW density exactly
(Eq. FBW stretching and shearing energy), quadratic height fields give a
constant Laplacian (Eq. mean curvature), the flat rest state is stress free.
Derivatives are checked by central finite differences, the projection against
LAPACK, the stencil against a dense scatter written here, the Newton step on a
quadratic problem and on the paper's simply supported plate (Sec. 6.2).
"""
import math

import numpy as np
import pytest

from conftest import read_golden_sections
from paper_2506_18867_gb300 import inputs


def _fbw(A, mu1, mu2, mush):
    f1, f2 = A[:, 0], A[:, 1]
    return (mu1 * (np.linalg.norm(f1) - 1) ** 2 + mu2 * (np.linalg.norm(f2) - 1) ** 2
            + mush * (f1 @ f2) ** 2)


def _rot(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


@pytest.mark.parametrize("rule", [0, 2, 3, 4])
def test_affine_deformation_exact_energy(orc, rule):
    """phi = A X + b is reproduced exactly; energy = Psi(A) * area for any rule."""
    rng = np.random.default_rng(3)
    nu, nv, Lu, Lv = 9, 8, 0.9, 0.6
    rest = inputs.flat_rest(nu, nv, Lu, Lv, angle=0.4)
    mat = (3.0, 5.0, 2.0, 0.0, 1.0)
    p = orc.Problem(nu, nv, rest, mat, mem_rule=rule, bend_rule=rule)
    for A in [np.array([[1.1, 0], [0, 1.0], [0, 0]]),       # uniaxial stretch
              np.array([[1.0, 0.3], [0, 1.0], [0, 0]]),     # shear
              rng.standard_normal((3, 2)) * 0.5 + np.eye(3, 2)]:
        C = rest @ A.T + np.array([0.1, -0.2, 0.3])
        E, g, H = p.span_eval(C, want_g=False, want_H=False)
        assert abs(E.sum() - _fbw(A, *mat[:3]) * Lu * Lv) < 1e-12 * max(1, E.sum())


def test_rigid_motion_zero_energy_and_invariance(orc):
    rng = np.random.default_rng(4)
    pat = inputs.config_random_small(11, 7, 9, curved=0.5)
    p = orc.Problem.from_patch(pat)
    R = _rot(rng)
    C_rigid = inputs.lift(pat.rest) @ R.T + rng.standard_normal(3)
    E, g, _ = p.span_eval(C_rigid, want_H=False)
    assert np.abs(E).max() < 1e-20 and np.abs(g).max() < 1e-12
    E1, g1, H1 = p.span_eval(pat.C)
    C2 = pat.C @ R.T + rng.standard_normal(3)
    E2, g2, H2 = p.span_eval(C2)
    np.testing.assert_allclose(E2, E1, rtol=1e-12, atol=1e-14)
    # gradient rotates with the motion: g2_l = R g1_l
    g1r = (g1.reshape(-1, 9, 3) @ R.T).reshape(g1.shape)
    np.testing.assert_allclose(g2, g1r, atol=1e-9 * np.abs(g1).max())


def _poly_control(nu, nv, coeffs):
    """Control values of p(u,v) = sum c_ab u^a v^b (a, b <= 2) via blossoms."""
    ku = np.array([min(max(k - 2, 0), nu - 2) for k in range(nu + 3)], float)
    kv = np.array([min(max(k - 2, 0), nv - 2) for k in range(nv + 3)], float)
    bu = {0: np.ones(nu), 1: np.array([(ku[i + 1] + ku[i + 2]) / 2 for i in range(nu)]),
          2: np.array([ku[i + 1] * ku[i + 2] for i in range(nu)])}
    bv = {0: np.ones(nv), 1: np.array([(kv[j + 1] + kv[j + 2]) / 2 for j in range(nv)]),
          2: np.array([kv[j + 1] * kv[j + 2] for j in range(nv)])}
    out = np.zeros((nv, nu))
    for (a, b), c in coeffs.items():
        out += c * np.outer(bv[b], bu[a])
    return out.reshape(-1)


@pytest.mark.parametrize("angle", [0.0, 0.7])
def test_quadratic_height_field_bending_energy(orc, angle):
    """phi = (X, Y, a X^2 + b Y^2): Laplacian (0, 0, 2a + 2b) everywhere, so the
    bending energy is mu_bd/2 (2a+2b)^2 * area exactly, independent of the owner
    convention at knots (Eq. general bending energy, Eq. mean curvature)."""
    nu, nv, Lu, Lv = 10, 8, 0.8, 0.5
    rest = inputs.flat_rest(nu, nv, Lu, Lv, angle=angle)
    mu_bd, a, b = 0.37, 1.3, -0.4
    p = orc.Problem(nu, nv, rest, (0.0, 0.0, 0.0, mu_bd, 1.0))
    # X = c + Ru (Lu/Su) u + Rv (Lv/Sv) v with rotation columns Ru, Rv
    c, s = math.cos(angle), math.sin(angle)
    su, sv = Lu / (nu - 2), Lv / (nv - 2)
    ex = np.array([c * su, -s * sv])                          # X = ex . (u, v)
    ey = np.array([s * su, c * sv])                           # Y = ey . (u, v)
    # z = a X^2 + b Y^2 as a polynomial in u, v
    coeffs = {(2, 0): a * ex[0] ** 2 + b * ey[0] ** 2, (0, 2): a * ex[1] ** 2 + b * ey[1] ** 2,
              (1, 1): 2 * (a * ex[0] * ex[1] + b * ey[0] * ey[1])}
    z = _poly_control(nu, nv, coeffs)
    C = inputs.lift(rest)
    C[:, 2] = z
    E, g, H = p.span_eval(C, want_H=False)
    assert abs(E.sum() - 0.5 * mu_bd * (2 * a + 2 * b) ** 2 * Lu * Lv) < 1e-11
    # the flat rest state is free of bending and membrane energy and gradient
    pm = orc.Problem(nu, nv, rest, (5.0, 6.0, 7.0, mu_bd, 1.0))
    E0, g0, _ = pm.span_eval(inputs.lift(rest), want_H=False)
    assert np.abs(E0).max() < 1e-25 and np.abs(g0).max() < 1e-12


def test_gradient_and_hessian_by_central_differences(orc):
    pat = inputs.config_random_small(21, 6, 7, curved=0.6, noise=0.2)
    p = orc.Problem.from_patch(pat)
    E, g, H = p.span_eval(pat.C)
    rng = np.random.default_rng(5)
    h = 1e-6 * pat.meta["span_m"]
    Su = pat.nu - 2
    for s in rng.choice(p.n_spans, 6, replace=False):
        a, b = s % Su, s // Su
        for dof in rng.choice(27, 5, replace=False):
            l, c = divmod(int(dof), 3)
            al = (b + l // 3) * pat.nu + a + l % 3
            Cp, Cm = pat.C.copy(), pat.C.copy()
            Cp[al, c] += h
            Cm[al, c] -= h
            Ep, gp, _ = p.span_eval(Cp, want_H=False)
            Em, gm, _ = p.span_eval(Cm, want_H=False)
            fd = (Ep[s] - Em[s]) / (2 * h)
            assert abs(fd - g[s, dof]) <= 1e-6 * (np.abs(g[s]).max() + 1e-12)
            fdH = (gp[s] - gm[s]) / (2 * h)
            assert np.abs(fdH - H[s, :, dof]).max() <= 1e-6 * np.abs(H[s]).max()
    assert np.abs(H - H.transpose(0, 2, 1)).max() <= 1e-13 * np.abs(H).max()


def test_projection_against_lapack_and_invariants(orc):
    pat = inputs.config_square(2, 12)
    p = orc.Problem.from_patch(pat)
    _, _, H = p.span_eval(pat.C, want_g=False)
    for s in [0, 5, 37, 99]:
        P, lam, sweeps = orc.project_psd(H[s])
        w, V = np.linalg.eigh(H[s])
        Pl = (V * np.maximum(w, 0)) @ V.T
        nrm = np.linalg.norm(H[s])
        assert np.linalg.norm(P - Pl) <= 1e-13 * nrm
        assert np.linalg.eigvalsh(P).min() >= -1e-13 * nrm       # P is PSD
        # H = H+ - H- with H+ = P, so P - H = H- is PSD as well
        assert np.linalg.eigvalsh(P - H[s]).min() >= -1e-13 * nrm
        assert np.linalg.norm(P @ (P - H[s])) <= 1e-12 * nrm ** 2  # complementary
        np.testing.assert_allclose(np.sort(lam), w, atol=1e-13 * nrm)


def _dense_reference(orc, pat, project):
    """Dense 3N x 3N Hessian by plain scatter of the oracle's span Hessians."""
    p = orc.Problem.from_patch(pat)
    nu, nv, N = pat.nu, pat.nv, pat.n_cp
    _, _, H = p.span_eval(pat.C, want_g=False)
    D = np.zeros((3 * N, 3 * N))
    Su = nu - 2
    for s in range(p.n_spans):
        a, b = s % Su, s // Su
        Hs = orc.project_psd(H[s])[0] if project else H[s]
        dofs = [3 * ((b + l // 3) * nu + a + l % 3) + c for l in range(9) for c in range(3)]
        D[np.ix_(dofs, dofs)] += Hs
    m = p.lumped_mass()
    D[np.arange(3 * N), np.arange(3 * N)] += np.repeat(m, 3) / pat.dt ** 2
    for al in pat.pinned:
        D[3 * al:3 * al + 3, :] = 0
        D[:, 3 * al:3 * al + 3] = 0
        D[3 * al:3 * al + 3, 3 * al:3 * al + 3] = np.eye(3)
    return D


@pytest.mark.parametrize("shape,project", [((5, 5), True), ((6, 7), False), ((6, 7), True)])
def test_stencil_equals_dense_scatter(orc, shape, project):
    pat = inputs.config_random_small(7, *shape, noise=0.3)
    p = orc.Problem.from_patch(pat)
    sc = orc.Scene.from_patch(pat, project=project)
    E, g, K = orc.evaluate(p, sc, pat.C, pat.Chat)
    D = orc.stencil_to_dense(pat.nu, pat.nv, K)
    Dr = _dense_reference(orc, pat, project)
    assert np.abs(D - Dr).max() <= 1e-12 * np.abs(Dr).max()
    assert np.abs(D - D.T).max() <= 1e-12 * np.abs(D).max()
    x = np.random.default_rng(2).standard_normal((pat.n_cp, 3))
    np.testing.assert_allclose(orc.stencil_matvec(pat.nu, pat.nv, K, x).ravel(), D @ x.ravel(),
                               atol=1e-12 * np.abs(D).max() * np.abs(x).max() * 25)
    if project:
        assert np.linalg.eigvalsh(D).min() > 0


def test_incremental_potential_gradient_fd(orc):
    pat = inputs.config_random_small(9, 6, 6, noise=0.2)
    p = orc.Problem.from_patch(pat)
    sc = orc.Scene.from_patch(pat)
    sc_free = orc.Scene(pat.dt, pat.gravity, [], True)
    E, g, _ = orc.evaluate(p, sc_free, pat.C, pat.Chat, want_K=False)
    h = 1e-7
    for al, c in [(3, 0), (10, 2), (20, 1), (35, 2)]:
        Cp, Cm = pat.C.copy(), pat.C.copy()
        Cp[al, c] += h
        Cm[al, c] -= h
        fd = (orc.energy(p, sc_free, Cp, pat.Chat) - orc.energy(p, sc_free, Cm, pat.Chat)) / (2 * h)
        assert abs(fd - g[al, c]) <= 1e-6 * np.abs(g).max()
    _, gp, _ = orc.evaluate(p, sc, pat.C, pat.Chat, want_K=False)
    assert np.abs(gp[pat.pinned]).max() == 0.0


def test_solvers_agree_with_lapack(orc):
    pat = inputs.config_random_small(3, 6, 8)
    p = orc.Problem.from_patch(pat)
    sc = orc.Scene.from_patch(pat)
    E, g, K = orc.evaluate(p, sc, pat.C, pat.Chat)
    D = orc.stencil_to_dense(pat.nu, pat.nv, K)
    want = np.linalg.solve(D, -g.ravel())
    xb = orc.solve_banded(pat.nu, pat.nv, K, -g)
    xp, it = orc.solve_pcg(pat.nu, pat.nv, K, -g, 1e-13)
    assert it > 0
    np.testing.assert_allclose(xb.ravel(), want, atol=1e-12 * np.abs(want).max())
    np.testing.assert_allclose(xp.ravel(), want, atol=1e-10 * np.abs(want).max())


def test_newton_on_quadratic_problem_converges_in_one_step(orc):
    """Bending-only static problem is quadratic in C: one exact Newton step
    zeroes the gradient (Sec. 5.1 projected Newton; projection is a no-op on
    the PSD bending Hessian)."""
    pat = inputs.config_random_small(13, 7, 7, noise=0.3)
    mat = (0.0, 0.0, 0.0, 0.05, 0.3)
    p = orc.Problem(pat.nu, pat.nv, pat.rest, mat)
    # pin the whole boundary ring so the quadratic form is definite
    ring = [al for al in range(pat.n_cp) if al % pat.nu in (0, pat.nu - 1) or al // pat.nu in (0, pat.nv - 1)]
    sc = orc.Scene(0.0, (0.0, 0.0, -9.81), ring, True)
    C1, rep = orc.newton_step(p, sc, pat.C)
    assert rep.status == 0 and rep.alpha == 1.0 and rep.E1 <= rep.E0
    _, g1, _ = orc.evaluate(p, sc, C1, want_K=False)
    assert np.abs(g1).max() <= 1e-10 * rep.grad_inf


def test_line_search_backtracking_branch(orc):
    """Sec. 5.1 backtracking (plain decrease, no Armijo constant): on a noisy
    state whose full Newton step increases the incremental potential, the
    oracle takes the first alpha in 1, 1/2, 1/4, ... at which the energy has
    not increased, with the energies evaluated here step by step; along an
    uphill direction (d = +g, so E(C + alpha d) > E(C) for every small alpha)
    it gives up after 30 halvings and leaves C unchanged; and it stops at
    the halving limit it is given."""
    pat = inputs.config_random_small(16, 14, 12, noise=0.3)
    prob = orc.Problem.from_patch(pat)
    sc = orc.Scene.from_patch(pat, project=True)
    E0, g, K = orc.evaluate(prob, sc, pat.C, pat.Chat)
    d = orc.solve_banded(pat.nu, pat.nv, K, -g)
    alphas = [0.5 ** k for k in range(31)]
    Es = [orc.energy(prob, sc, pat.C + a * d, pat.Chat) for a in alphas]
    first = next(k for k, E in enumerate(Es) if E <= E0)
    assert first >= 1 and Es[0] > E0            # the full step overshoots here
    assert all(E > E0 for E in Es[:first])
    C1, st, rep = orc.line_search(prob, sc, pat.C, pat.Chat, d)
    assert st == 0 and rep.ls_halvings == first and rep.alpha == alphas[first]
    assert rep.E1 == Es[first] and rep.E1 <= E0
    np.testing.assert_array_equal(C1, pat.C + alphas[first] * d)
    Cn, rn = orc.newton_step(prob, sc, pat.C, pat.Chat, solver=0)
    assert rn.status == 0 and rn.ls_halvings == first and rn.alpha == alphas[first]
    np.testing.assert_array_equal(Cn, C1)
    # a non-descent direction: uphill along the gradient
    assert all(orc.energy(prob, sc, pat.C + a * g, pat.Chat) > E0 for a in alphas)
    C2, st2, rep2 = orc.line_search(prob, sc, pat.C, pat.Chat, g)
    assert st2 == -3 and rep2.ls_halvings == 30 and rep2.alpha == 0.0
    np.testing.assert_array_equal(C2, pat.C)
    _, rep3 = orc.newton_step(prob, sc, pat.C, pat.Chat, solver=0, max_halvings=first - 1)
    assert rep3.status == -3 and rep3.ls_halvings == first - 1


def test_plate_deflection_converges_to_navier_solution(orc):
    """Sec. 6.2 bending benchmark: simply supported plate, bending only, uniform
    load B; the maximum deflection approaches 0.048744 B a^4 (1-nu^2)/(E h^3)
    under refinement."""
    gd = {r[0]: r[1] for r in read_golden_sections("plate_navier.txt")["main"]}
    E, nu_p, h, B = gd["E"], gd["nu"], gd["h"], gd["B"]
    w_exact = gd["coefficient"] * B * 1.0 ** 4 * (1 - nu_p ** 2) / (E * h ** 3)
    D = E * h ** 3 / (12 * (1 - nu_p ** 2))
    errs = []
    for n in (10, 18, 34):
        rest = inputs.flat_rest(n, n, 1.0, 1.0)
        p = orc.Problem(n, n, rest, (0.0, 0.0, 0.0, D, 1.0))  # load B = rho_area * g
        ring = [al for al in range(n * n) if al % n in (0, n - 1) or al // n in (0, n - 1)]
        sc = orc.Scene(0.0, (0.0, 0.0, -B), ring, True)
        C0 = inputs.lift(rest)
        C1, rep = orc.newton_step(p, sc, C0)
        assert rep.status == 0
        # deflection at the plate centre: evaluate the surface at (u, v) = (S/2, S/2)
        S = n - 2
        a = S // 2 if S % 2 else S // 2 - 1
        Bs = p.basis9(S / 2, S / 2, a, a)
        z = sum(Bs[0, l] * C1[(a + l // 3) * n + a + l % 3, 2] for l in range(9))
        errs.append(abs(-z - w_exact) / w_exact)
    assert errs[-1] < 0.02, errs
    assert errs[0] > errs[1] > errs[2], errs


def test_subset_drivers_match_full_evaluation(orc):
    """The selected-span and selected-row drivers reproduce the full evaluation."""
    pat = inputs.config_random_small(17, 9, 8, noise=0.2)
    p = orc.Problem.from_patch(pat)
    sc = orc.Scene.from_patch(pat, project=True)
    E, g, H = p.span_eval(pat.C)
    spans = [0, 5, 17, 30, 41]
    Es, gs, Hs = orc.span_terms_subset(p, pat.C, spans, project=False)
    np.testing.assert_array_equal(Es, E[spans])
    np.testing.assert_array_equal(Hs, H[spans])
    _, _, Hp = orc.span_terms_subset(p, pat.C, spans, project=True)
    assert np.abs(Hp[2] - orc.project_psd(H[17])[0]).max() == 0.0
    Ef, gf, Kf = orc.evaluate(p, sc, pat.C, pat.Chat)
    rows = [0, 3, 8, 20, 40, 71]
    gr, Kr = orc.eval_rows(p, sc, pat.C, pat.Chat, rows)
    np.testing.assert_allclose(gr, gf[rows], rtol=1e-13, atol=1e-13 * np.abs(gf).max())
    np.testing.assert_allclose(Kr, Kf[rows], rtol=1e-13, atol=1e-13 * np.abs(Kf).max())
