"""Reduced quadrature on non-rectangular rest domains (Sec. 6, "Support of
Non-Rectangular Domains", and its figure on integration error).

The paper distorts the rest domain in three ways - aspect ratios 1:1 to
1:10, parallelograms with interior angle 75 down to 30 degrees, and a sharp
mid-edge bend with interior angle 165 down to 105 degrees - and reports that
the mass-matrix and elastic-energy quadrature errors stay below 1e-3.  Here
the same three families (inputs.distorted_rest) carry a smooth deformed
state (inputs.config_distorted without its noise); the reference is the
same discrete field integrated with 3x3 Gauss points per span, so the
difference is the reduced rules' quadrature error alone:

- the area the membrane rule integrates, sum of W_q = w_q |det J|, against
  the 3x3 Gauss area;
- the membrane + bending energy of the reduced rules against 3x3 Gauss;
- the lumped masses (3x3 Gauss per span, the oracle's reading of the mass
  integral) against a 5x5 Gauss integration of rho N_alpha |det J| written
  here from the basis and the rest control points: |det J| of a biquadratic
  map is a polynomial of degree <= 3 per variable, so both are exact and
  the mass carries no quadrature error at all.

Each stays below 1e-3 on a 48 x 48 control grid, falls by at least 3x from
24 x 24 to 48 x 48 (the O(h^2) of a quadrature error), and the bend family's
error grows with the sharpness of the bend.
"""
import numpy as np
import pytest

from paper_2506_18867_gb300 import inputs

FAMILIES = [("aspect", (1, 2, 5, 10)), ("skew", (75, 60, 45, 30)), ("bend", (165, 150, 135, 120, 105))]
CASES = [(k, p) for k, ps in FAMILIES for p in ps]


def smooth_state(kind, param, n):
    pat = inputs.config_distorted(kind, param, n, n)
    lo, hi = pat.rest.min(axis=0), pat.rest.max(axis=0)
    span = min((hi[0] - lo[0]) / (n - 2), (hi[1] - lo[1]) / (n - 2))
    pat.C -= 1e-3 * span * inputs.normal(pat.meta["seed"], pat.C.size).reshape(pat.C.shape)  # noise off
    return pat


GL5 = np.polynomial.legendre.leggauss(5)


def lumped_mass_gauss5(orc, pat):
    """m_alpha = rho int N_alpha |det J| du dv, 5x5 Gauss-Legendre per span;
    J = sum_l X_l (N_l,u, N_l,v) over the span's 9 control points."""
    prob = orc.Problem.from_patch(pat)
    x, w = (GL5[0] + 1.0) / 2.0, GL5[1] / 2.0
    m = np.zeros(pat.n_cp)
    for b in range(pat.nv - 2):
        for a in range(pat.nu - 2):
            idx = [(b + lj) * pat.nu + a + li for lj in range(3) for li in range(3)]
            X = pat.rest[idx]                                   # (9, 2)
            for xu, wu in zip(x, w):
                for xv, wv in zip(x, w):
                    B = prob.basis9(a + xu, b + xv, a, b)
                    J = np.stack([X.T @ B[1], X.T @ B[2]], axis=1)
                    m[idx] += wu * wv * abs(np.linalg.det(J)) * B[0]
    return m * pat.material.rho_area


def quadrature_errors(orc, kind, param, n):
    pat = smooth_state(kind, param, n)
    out, E, A = {}, {}, {}
    for rule in (orc.RULE_REDUCED, orc.RULE_GAUSS3):
        prob = orc.Problem(pat.nu, pat.nv, pat.rest, pat.material, mem_rule=rule, bend_rule=rule)
        E[rule] = prob.span_eval(pat.C, want_g=False, want_H=False)[0].sum()
        A[rule] = prob.point_tables(0)[:, 0].sum()
    out["energy"] = abs(E[orc.RULE_REDUCED] - E[orc.RULE_GAUSS3]) / abs(E[orc.RULE_GAUSS3])
    out["area"] = abs(A[orc.RULE_REDUCED] - A[orc.RULE_GAUSS3]) / A[orc.RULE_GAUSS3]
    if n == 24:
        m = orc.Problem.from_patch(pat).lumped_mass()
        m5 = lumped_mass_gauss5(orc, pat)
        out["mass"] = float(np.linalg.norm(m - m5) / np.linalg.norm(m5))
        out["area_exact"] = abs(A[orc.RULE_GAUSS3] * pat.material.rho_area - m5.sum()) / m5.sum()
    return out


@pytest.fixture(scope="module")
def errors(orc):
    return {(k, p, n): quadrature_errors(orc, k, p, n) for k, p in CASES for n in (24, 48)}


@pytest.mark.parametrize("kind,param", CASES, ids=[f"{k}{p}" for k, p in CASES])
def test_quadrature_error_below_1e3(errors, kind, param):
    e48, e24 = errors[(kind, param, 48)], errors[(kind, param, 24)]
    print(f"{kind} {param}: 48x48 energy {e48['energy']:.1e} area {e48['area']:.1e}; 24x24 energy "
          f"{e24['energy']:.1e} area {e24['area']:.1e}; lumped mass vs 5x5 Gauss {e24['mass']:.1e}")
    assert e48["energy"] < 1e-3 and e48["area"] < 1e-3
    # a quadrature error of a smooth field falls like h^2 under refinement
    assert e48["energy"] < e24["energy"] / 3.0
    assert e48["area"] < e24["area"] / 3.0 or e48["area"] < 1e-13
    # the mass integral is exact (and the 3x3 Gauss area is the domain's)
    assert e24["mass"] < 1e-13 and e24["area_exact"] < 1e-13


def test_affine_domains_integrate_mass_exactly(errors):
    """Rectangles and parallelograms are affine images of the parameter
    square: |det J| is constant, so the reduced rule integrates the area
    exactly; the bend is not affine and shows a (small) error."""
    for k, p in CASES:
        if k in ("aspect", "skew"):
            assert errors[(k, p, 48)]["area"] < 1e-13, (k, p)
    assert errors[("bend", 105, 48)]["area"] > 1e-8


def test_bend_error_grows_with_sharpness(errors):
    """The paper: the error grows with distortion.  Along the bend family
    (165 -> 105 degrees) the energy and area errors increase monotonically."""
    for q in ("energy", "area"):
        v = [errors[("bend", p, 48)][q] for p in (165, 150, 135, 120, 105)]
        assert all(b > a for a, b in zip(v, v[1:])), (q, v)
