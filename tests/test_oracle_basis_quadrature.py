"""Pins of the oracle's basis functions, quadrature rules, rest geometry and mass.

Each test pins the oracle to something other than itself: textbook closed forms
of open uniform quadratic B-splines, the paper's own figure of the reduced
rules (Fig. 3), the stencil sizes the paper states (Sec. 4.1, Sec. 4.2),
exact reproduction of linear and quadratic fields, and finite differences.
"""
import math

import numpy as np
import pytest

from conftest import read_golden_sections
from paper_2506_18867_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore")


def _prob(orc, nu, nv, rest=None, mat=(1.0, 1.0, 1.0, 1.0, 1.0), **kw):
    if rest is None:
        rest = inputs.flat_rest(nu, nv, float(nu - 2), float(nv - 2))
    return orc.Problem(nu, nv, rest, mat, **kw)


def _knots(n):
    S = n - 2
    return np.array([min(max(k - 2, 0), S) for k in range(n + 3)], dtype=float)


# --------------------------------------------------------------------- basis

def test_basis_closed_forms_interior_and_boundary(orc):
    """Textbook pieces: uniform interior span (1-t)^2/2, (-2t^2+2t+1)/2, t^2/2;
    first span of an open knot vector (1-t)^2, 2t - 3t^2/2, t^2/2 (Eq. B-spline basis)."""
    p = _prob(orc, 9, 9)
    for t in [0.0, 0.13, 0.5, 0.77, 0.999]:
        # u in interior span a = 3, v in first span b = 0: tensor product rows factor
        B = p.basis9(3 + t, 0.0 + t, 3, 0)
        Nu = B[0, 0:3] / B[0, 0:3].sum()  # v-factor cancels in the ratio of row lj=0
        Nv_first = np.array([B[0, 0] + B[0, 1] + B[0, 2], B[0, 3] + B[0, 4] + B[0, 5],
                             B[0, 6] + B[0, 7] + B[0, 8]])
        np.testing.assert_allclose(Nu, [(1 - t) ** 2 / 2, (-2 * t * t + 2 * t + 1) / 2, t * t / 2],
                                   atol=1e-14)
        np.testing.assert_allclose(Nv_first, [(1 - t) ** 2, 2 * t - 1.5 * t * t, t * t / 2], atol=1e-14)
        # derivatives: interior d/du, boundary d/dv (sum over the other index)
        dNu = B[1, 0:3] + B[1, 3:6] + B[1, 6:9]
        np.testing.assert_allclose(dNu, [-(1 - t), -2 * t + 1, t], atol=1e-13)
        dNv = np.array([B[2, 0:3].sum(), B[2, 3:6].sum(), B[2, 6:9].sum()])
        np.testing.assert_allclose(dNv, [-2 * (1 - t), 2 - 3 * t, t], atol=1e-13)
        d2u = B[3, 0:3] + B[3, 3:6] + B[3, 6:9]
        np.testing.assert_allclose(d2u, [1.0, -2.0, 1.0], atol=1e-13)
        d2v = np.array([B[5, 0:3].sum(), B[5, 3:6].sum(), B[5, 6:9].sum()])
        np.testing.assert_allclose(d2v, [2.0, -3.0, 1.0], atol=1e-13)


def test_partition_of_unity_everywhere(orc):
    rng = np.random.default_rng(0)
    for nu, nv in [(5, 5), (6, 9), (12, 7)]:
        p = _prob(orc, nu, nv)
        for _ in range(40):
            a, b = rng.integers(0, nu - 2), rng.integers(0, nv - 2)
            u, v = a + rng.random(), b + rng.random()
            B = p.basis9(u, v, a, b)
            assert abs(B[0].sum() - 1.0) < 1e-14
            assert np.all(B[0] >= -1e-15)
            for r in range(1, 6):
                assert abs(B[r].sum()) < 1e-12


def test_exact_reproduction_linear_and_quadratic(orc):
    """Blossoms: control values (xi_{i+1}+xi_{i+2})/2 reproduce u, xi_{i+1} xi_{i+2} reproduce u^2."""
    rng = np.random.default_rng(1)
    nu, nv = 8, 6
    p = _prob(orc, nu, nv)
    ku, kv = _knots(nu), _knots(nv)
    cu_lin = np.array([(ku[i + 1] + ku[i + 2]) / 2 for i in range(nu)])
    cu_sq = np.array([ku[i + 1] * ku[i + 2] for i in range(nu)])
    cv_sq = np.array([kv[j + 1] * kv[j + 2] for j in range(nv)])
    for _ in range(50):
        a, b = rng.integers(0, nu - 2), rng.integers(0, nv - 2)
        u, v = a + rng.random(), b + rng.random()
        B = p.basis9(u, v, a, b)
        lin = np.array([cu_lin[a + l % 3] for l in range(9)])
        usq = np.array([cu_sq[a + l % 3] for l in range(9)])
        uv = np.array([cu_lin[a + l % 3] * ((kv[b + l // 3 + 1] + kv[b + l // 3 + 2]) / 2) for l in range(9)])
        vsq = np.array([cv_sq[b + l // 3] for l in range(9)])
        assert abs(B[0] @ lin - u) < 1e-13 and abs(B[1] @ lin - 1) < 1e-13 and abs(B[3] @ lin) < 1e-12
        assert abs(B[0] @ usq - u * u) < 1e-12 and abs(B[1] @ usq - 2 * u) < 1e-12
        assert abs(B[3] @ usq - 2.0) < 1e-12 and abs(B[2] @ usq) < 1e-12
        assert abs(B[0] @ uv - u * v) < 1e-12 and abs(B[4] @ uv - 1.0) < 1e-12
        assert abs(B[5] @ vsq - 2.0) < 1e-12 and abs(B[0] @ vsq - v * v) < 1e-12


def test_c1_continuity_and_one_sided_second_derivatives(orc):
    """Quadratic B-splines on simple knots are C1: values and first derivatives
    agree from both neighbouring spans; second derivatives jump (reading R3)."""
    p = _prob(orc, 9, 9)
    for k in [1, 2, 3, 4, 5, 6]:
        left = p.basis9(k, 3.5, k - 1, 3)   # u = k evaluated in span k-1
        right = p.basis9(k, 3.5, k, 3)      # and in span k
        # map local indices: global i = a + li
        gl = {(k - 1 + l % 3, l // 3): l for l in range(9)}
        gr = {(k + l % 3, l // 3): l for l in range(9)}
        for key in set(gl) | set(gr):
            for row in (0, 1, 2):
                vl = left[row, gl[key]] if key in gl else 0.0
                vr = right[row, gr[key]] if key in gr else 0.0
                assert abs(vl - vr) < 1e-13
    jump = p.basis9(4, 3.5, 3, 3)[3].sum(), p.basis9(4, 3.5, 4, 3)[3].sum()
    assert abs(jump[0]) < 1e-12 and abs(jump[1]) < 1e-12  # sum stays zero on both sides


# ---------------------------------------------------------------- quadrature

def _as_set(pts, nd=3):
    return sorted((round(float(u), nd), round(float(v), nd)) for u, v in pts)


def test_fig3_membrane_rule_S5(orc):
    """Oracle's reduced membrane rule on 5x5 spans equals the points drawn in Fig. 3."""
    g = read_golden_sections("fig3_membrane_S5.txt")
    p = _prob(orc, 7, 7)
    q = p.quad_points(0)
    S = 5
    ring = (q[:, 3] == 0) | (q[:, 3] == S - 1) | (q[:, 4] == 0) | (q[:, 4] == S - 1)
    inner = q[~ring]
    # interior-region points lie on the interior region [1, S-1]^2
    assert np.all((inner[:, :2] >= 1) & (inner[:, :2] <= S - 1))
    assert _as_set(inner[:, :2]) == _as_set(np.array(g["interior"]))
    cells = {"corner": g["cell corner"], "vside": g["cell vside"], "uside": g["cell uside"]}
    for a in range(S):
        for b in range(S):
            ru, rv = a in (0, S - 1), b in (0, S - 1)
            if not (ru or rv):
                continue
            cls = "corner" if (ru and rv) else ("uside" if ru else "vside")
            sel = q[(q[:, 3] == a) & (q[:, 4] == b)]
            loc = sel[:, :2] - np.array([a, b])
            got = sorted((round(u, 2), round(v, 2)) for u, v in loc)
            want = sorted((round(u, 2), round(v, 2)) for u, v in cells[cls])
            assert got == want, (a, b, cls)


def test_fig3_bending_rule_S5(orc):
    g = read_golden_sections("fig3_bending_S5.txt")
    p = _prob(orc, 7, 7)
    q = p.quad_points(1)
    assert _as_set(q[:, :2]) == _as_set(np.array(g["main"]))


@pytest.mark.parametrize("nu,nv", [(5, 5), (5, 9), (7, 7), (10, 13), (32, 32)])
def test_rule_weights_cover_parametric_area(orc, nu, nv):
    """Weights sum to the parametric area S_u S_v for both rules; points lie in
    their owner span; the interior region carries (S_u-2)(S_v-2)."""
    p = _prob(orc, nu, nv)
    Su, Sv = nu - 2, nv - 2
    for which in (0, 1):
        q = p.quad_points(which)
        assert abs(q[:, 2].sum() - Su * Sv) < 1e-10
        assert np.all(q[:, 0] >= q[:, 3] - 1e-12) and np.all(q[:, 0] <= q[:, 3] + 1 + 1e-12)
        assert np.all(q[:, 1] >= q[:, 4] - 1e-12) and np.all(q[:, 1] <= q[:, 4] + 1 + 1e-12)
        ring = (q[:, 3] == 0) | (q[:, 3] == Su - 1) | (q[:, 4] == 0) | (q[:, 4] == Sv - 1)
        assert abs(q[~ring, 2].sum() - (Su - 2) * (Sv - 2)) < 1e-10


def test_point_counts_32x32(orc):
    p = _prob(orc, 32, 32)
    assert len(p.quad_points(0)) == 2386
    assert len(p.quad_points(1)) == 957


def test_reduced_stencil_sizes(orc):
    """Sec. 4.1: every interior membrane point touches 2x3 = 6 control points;
    Sec. 4.2: values and first derivatives at an interior bending point touch
    only the 2x2 control points of its dual cell."""
    p = _prob(orc, 11, 9)
    Su, Sv = 9, 7
    q = p.quad_points(0)
    for u, v, w, a, b in q:
        B = p.basis9(u, v, int(a), int(b))
        support = np.abs(B[0]) + np.abs(B[1]) + np.abs(B[2]) > 1e-14
        ring = a in (0, Su - 1) or b in (0, Sv - 1)
        if not ring:
            on_corner = float(u).is_integer() and float(v).is_integer()
            assert support.sum() == (4 if on_corner else 6)
    qb = p.quad_points(1)
    for u, v, w, a, b in qb:
        if float(u).is_integer() and float(v).is_integer():
            B = p.basis9(u, v, int(a), int(b))
            support = np.abs(B[0]) + np.abs(B[1]) + np.abs(B[2]) > 1e-14
            assert support.sum() == 4


def test_gauss_rules(orc):
    p = _prob(orc, 6, 6, mem_rule=orc.RULE_GAUSS3, bend_rule=orc.RULE_GAUSS2)
    q3, q2 = p.quad_points(0), p.quad_points(1)
    assert len(q3) == 16 * 9 and len(q2) == 16 * 4
    # 3-point rule integrates t^4 on [0,1] exactly, 2-point integrates t^3
    loc3 = q3[q3[:, 3] + q3[:, 4] == 0]
    assert abs((loc3[:, 2] * loc3[:, 0] ** 4).sum() - 0.2) < 1e-14
    loc2 = q2[q2[:, 3] + q2[:, 4] == 0]
    assert abs((loc2[:, 2] * loc2[:, 0] ** 3).sum() - 0.25) < 1e-14


@pytest.mark.parametrize("nu,nv", [(5, 5), (7, 9), (12, 10)])
def test_standard_rule_of_the_ablation(orc, nu, nv):
    """Sec. 6.5 case A: 2x2 Gauss on every interior span for both energies,
    the reduced rules' placements on the boundary spans."""
    Su, Sv = nu - 2, nv - 2
    red = _prob(orc, nu, nv)
    std = _prob(orc, nu, nv, mem_rule=orc.RULE_STANDARD, bend_rule=orc.RULE_STANDARD)
    for which in (0, 1):
        qr, qs = red.quad_points(which), std.quad_points(which)
        ring_r = (qr[:, 3] == 0) | (qr[:, 3] == Su - 1) | (qr[:, 4] == 0) | (qr[:, 4] == Sv - 1)
        ring_s = (qs[:, 3] == 0) | (qs[:, 3] == Su - 1) | (qs[:, 4] == 0) | (qs[:, 4] == Sv - 1)
        key = lambda q: sorted(tuple(round(float(x), 12) for x in row) for row in q[:, :5])  # noqa: E731
        assert key(qs[ring_s]) == key(qr[ring_r])
        inner = qs[~ring_s]
        assert len(inner) == 4 * (Su - 2) * (Sv - 2)
        assert abs(qs[:, 2].sum() - Su * Sv) < 1e-10
        for a in range(1, Su - 1):
            for b in range(1, Sv - 1):
                loc = inner[(inner[:, 3] == a) & (inner[:, 4] == b)]
                t, r = loc[:, 0] - a, loc[:, 1] - b
                assert len(loc) == 4 and abs(loc[:, 2].sum() - 1.0) < 1e-14
                # the 2-point rule integrates t^3 and t^3 r^3 exactly, not t^4
                assert abs((loc[:, 2] * t ** 3).sum() - 0.25) < 1e-14
                assert abs((loc[:, 2] * t ** 3 * r ** 3).sum() - 1 / 16) < 1e-14
                assert abs((loc[:, 2] * t ** 4).sum() - 0.2) > 1e-3


# ---------------------------------------------------------------- geometry

def test_affine_rest_geometry(orc):
    """Greville rest placement is affine in (u, v): J = R diag(Lu/Su, Lv/Sv),
    the inverse-map second derivatives vanish (c_u = c_v = 0) and the
    Laplacian coefficients are c_uu = (Su/Lu)^2, c_vv = (Sv/Lv)^2, c_uv = 0."""
    nu, nv, Lu, Lv, th = 9, 7, 0.7, 0.4, 0.6
    rest = inputs.flat_rest(nu, nv, Lu, Lv, angle=th)
    p = _prob(orc, nu, nv, rest=rest)
    Su, Sv = nu - 2, nv - 2
    tb = p.point_tables(1)
    np.testing.assert_allclose(tb[:, 15], (Lu / Su) * (Lv / Sv), rtol=1e-13)
    np.testing.assert_allclose(tb[:, 10], (Su / Lu) ** 2, rtol=1e-12)
    np.testing.assert_allclose(tb[:, 11], (Sv / Lv) ** 2, rtol=1e-12)
    assert np.abs(tb[:, 12:15]).max() < 1e-9
    tm = p.point_tables(0)
    assert abs(tm[:, 0].sum() - Lu * Lv) < 1e-12  # sum W = physical area


def _xmap(p, rest, nu, u, v):
    a, b = min(int(u), nu - 3), min(int(v), p.nv - 3)
    B = p.basis9(u, v, a, b)
    X = np.zeros(2)
    for l in range(9):
        X += B[0, l] * rest[(b + l // 3) * nu + a + l % 3]
    return X


def test_curved_rest_inverse_map_derivatives(orc):
    """Inverse function theorem terms (Sec. 4.1, 4.2) against finite differences
    of the numerically inverted rest map u(X) on a curved rest shape."""
    nu, nv = 8, 8
    pat = inputs.config_random_small(5, nu, nv, angle=0.3, curved=0.8)
    rest = pat.rest
    p = _prob(orc, nu, nv, rest=rest)
    tb = p.point_tables(1)
    q = p.quad_points(1)

    def inv(X, uv0):
        uv = np.array(uv0, dtype=float)
        for _ in range(50):
            h = 1e-7
            F = _xmap(p, rest, nu, *uv) - X
            J = np.zeros((2, 2))
            J[:, 0] = (_xmap(p, rest, nu, uv[0] + h, uv[1]) - _xmap(p, rest, nu, uv[0] - h, uv[1])) / (2 * h)
            J[:, 1] = (_xmap(p, rest, nu, uv[0], uv[1] + h) - _xmap(p, rest, nu, uv[0], uv[1] - h)) / (2 * h)
            uv -= np.linalg.solve(J, F)
            if np.abs(F).max() < 1e-15:
                break
        return uv

    # span-centre points of boundary spans: the map is smooth there
    rows = [k for k in range(len(q)) if not float(q[k, 0]).is_integer()][:6]
    for k in rows:
        u0, v0 = q[k, :2]
        X0 = _xmap(p, rest, nu, u0, v0)
        h = 1e-3 * 0.05
        f = lambda dx, dy: inv(X0 + np.array([dx, dy]), (u0, v0))
        c = f(0, 0)
        lap = (f(h, 0) + f(-h, 0) + f(0, h) + f(0, -h) - 4 * c) / (h * h)
        gx = (f(h, 0) - f(-h, 0)) / (2 * h)
        gy = (f(0, h) - f(0, -h)) / (2 * h)
        np.testing.assert_allclose([gx[0] ** 2 + gy[0] ** 2, gx[1] ** 2 + gy[1] ** 2,
                                    2 * (gx[0] * gx[1] + gy[0] * gy[1])],
                                   [tb[k, 10], tb[k, 11], tb[k, 14]], rtol=1e-6, atol=1e-6)
        np.testing.assert_allclose(lap, [tb[k, 12], tb[k, 13]], rtol=2e-3, atol=2e-3 * np.abs(tb[k, 10]))


def test_lumped_mass_closed_form(orc):
    """int N_i = (xi_{i+3} - xi_i) / 3 on an affine rest: m = rho (Lu/Su)(Lv/Sv)
    (xi_{i+3}-xi_i)(eta_{j+3}-eta_j)/9; the masses sum to rho * area."""
    nu, nv, Lu, Lv, rho = 9, 6, 1.3, 0.8, 3.7
    p = _prob(orc, nu, nv, rest=inputs.flat_rest(nu, nv, Lu, Lv, angle=1.1), mat=(1, 1, 1, 1, rho))
    m = p.lumped_mass()
    ku, kv = _knots(nu), _knots(nv)
    want = np.array([rho * (Lu / (nu - 2)) * (Lv / (nv - 2)) * (ku[i + 3] - ku[i]) * (kv[j + 3] - kv[j]) / 9
                     for j in range(nv) for i in range(nu)])
    np.testing.assert_allclose(m, want, rtol=1e-13)
    assert abs(m.sum() - rho * Lu * Lv) < 1e-12
