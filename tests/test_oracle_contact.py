"""Pins of the contact oracle (oracle/contact_oracle.py; Sec. 4.3 with the
IPC log barrier).

- Closest point on a triangle against brute-force sampling, and the
  reported feature carrying the point.
- A flat cloth at height h over a plane: B = kappa beta(h / dhat) area, the
  z-gradient summed over control points kappa beta'(h / dhat) / dhat area,
  the zz-Hessian summed over all blocks kappa beta'' / dhat^2 area (partition
  of unity of the embedding weights).
- Each point-edge / point-corner distance counted once (a vertex over the
  shared edge of two triangles).
- Central differences of the energy (gradient) and of the gradient (full
  Hessian) near a pyramid whose faces, edges and apex are all active.
- The projected pair Hessian is PSD and differs from the full one by a
  negative semidefinite matrix.
- The step bound of a vertex falling onto the plane: 0.9 h / |dz|.
"""
import math

import numpy as np
import pytest

from oracle import contact_oracle as co
from paper_2506_18867_gb300 import inputs

DHAT, KAPPA = 0.02, 1e3


def plane(z=0.0, half=10.0):
    """One large triangle (no interior edges: near a shared edge both of its
    triangles would contribute, the point-edge term of one and the
    point-face term of the other, as in IPC's constraint set)."""
    V = [(-half, -half, z), (3 * half, -half, z), (-half, 3 * half, z)]
    return co.Obstacle(V, [(0, 1, 2)])


def pyramid(apex_z=-0.004, base_z=-0.03, half=0.2, cx=0.25, cy=0.25):
    V = [(cx - half, cy - half, base_z), (cx + half, cy - half, base_z), (cx + half, cy + half, base_z),
         (cx - half, cy + half, base_z), (cx, cy, apex_z)]
    T = [(0, 1, 4), (1, 2, 4), (2, 3, 4), (3, 0, 4)]
    return co.Obstacle(V, T)


def flat_patch(n=9, size=0.5, h=0.01):
    rest = inputs.flat_rest(n, n, size, size)
    C = inputs.lift(rest)
    C[:, 2] = h
    return rest, C


def test_closest_point_against_sampling():
    rng = np.random.default_rng(3)
    a, b, c = rng.standard_normal((3, 3))
    s = np.linspace(0.0, 1.0, 201)
    U, W = np.meshgrid(s, s)
    keep = U + W <= 1.0
    pts = a + U[keep, None] * (b - a) + W[keep, None] * (c - a)
    for _ in range(200):
        p = rng.standard_normal(3) * 1.5
        q, feat = co.closest_point(p, a, b, c)
        dmin = np.min(np.linalg.norm(pts - p, axis=1))
        d = np.linalg.norm(p - q)
        assert d <= dmin + 1e-12 and dmin - d < 2e-2
        tri = (a, b, c)
        if feat[0] == "vertex":
            assert np.allclose(q, tri[feat[1]])
        elif feat[0] == "edge":
            e0, e1 = tri[feat[1]], tri[feat[2]]
            assert np.linalg.norm(np.cross(q - e0, e1 - e0)) < 1e-10
        else:  # interior: p - q is normal to the triangle
            n = np.cross(b - a, c - a)
            assert np.linalg.norm(np.cross(p - q, n)) < 1e-10 * max(1.0, np.linalg.norm(p - q) * np.linalg.norm(n))


def test_flat_cloth_over_plane_closed_form(orc):
    rest, C = flat_patch(h=0.01)
    prob = orc.Problem(9, 9, rest, (1.0, 1.0, 0.5, 0.0, 1.0))
    cm = co.ContactMesh(prob, 12, 11)
    area = 0.5 * 0.5
    assert abs(cm.area.sum() - area) < 1e-14
    x = 0.01 / DHAT
    E, G, K = co.contact_terms(cm, plane(), C, DHAT, KAPPA)
    assert abs(E - KAPPA * co.beta(x) * area) < 1e-12 * abs(E)
    assert abs(G[:, 2].sum() - KAPPA * co.beta_d1(x) / DHAT * area) < 1e-10 * abs(G[:, 2].sum())
    assert np.abs(G[:, :2]).max() < 1e-12 * np.abs(G).max()
    assert abs(K[:, :, 2, 2].sum() - KAPPA * co.beta_d2(x) / DHAT ** 2 * area) < 1e-10 * abs(K[:, :, 2, 2].sum())
    # beyond dhat nothing is active
    C2 = C.copy()
    C2[:, 2] = 1.5 * DHAT
    E2, G2, _ = co.contact_terms(cm, plane(), C2, DHAT, KAPPA)
    assert E2 == 0.0 and not G2.any()


def test_shared_edge_counted_once():
    obs = co.Obstacle([(-1, -1, 0), (1, -1, 0), (1, 1, 0), (-1, 1, 0)], [(0, 1, 2), (0, 2, 3)])
    # the diagonal (0, 2) is shared; a point straight above it, beside the plane's z = 0 face
    x = np.array([0.3, 0.3, 0.005])
    e, _, _ = co.vertex_terms(x, obs, DHAT)
    # both triangles see the point over their face or over the diagonal; in
    # every case the distance is 0.005 and one term enters per distinct feature
    q0, f0 = co.closest_point(x, *obs.V[obs.T[0]])
    q1, f1 = co.closest_point(x, *obs.V[obs.T[1]])
    n_terms = sum(obs.counts(t, f) for t, f in ((0, f0), (1, f1)))
    assert n_terms == 1
    assert abs(e - co.beta(0.005 / DHAT)) < 1e-15


def _wavy_state(n=11, seed=2):
    rest = inputs.flat_rest(n, n, 0.5, 0.5)
    C = inputs.lift(rest)
    X = rest
    C[:, 2] = 0.006 + 0.004 * np.sin(2 * math.pi * X[:, 0] / 0.5) * np.cos(2 * math.pi * X[:, 1] / 0.5)
    C += 1e-3 * inputs.normal(seed, C.size).reshape(C.shape)
    return rest, C


def test_derivatives_by_central_differences(orc):
    rest, C = _wavy_state()
    prob = orc.Problem(11, 11, rest, (1.0, 1.0, 0.5, 0.0, 1.0))
    cm = co.ContactMesh(prob, 31, 31)   # a vertex right above the apex at (0.25, 0.25)
    obs = pyramid()
    kinds = set()
    for x in cm.positions(C):
        for t in range(len(obs.T)):
            q, f = co.closest_point(x, *obs.V[obs.T[t]])
            if np.linalg.norm(x - q) < DHAT and obs.counts(t, f):
                kinds.add(f[0])
    assert kinds == {"face", "edge", "vertex"}, kinds
    E, G, Kf = co.contact_terms(cm, obs, C, DHAT, KAPPA, hessian="full")
    rng = np.random.default_rng(1)
    h = 1e-7
    active = np.nonzero(np.abs(G).sum(axis=1))[0]
    for al in rng.choice(active, 8, replace=False):
        for c in range(3):
            Cp, Cm = C.copy(), C.copy()
            Cp[al, c] += h
            Cm[al, c] -= h
            Ep, Gp, _ = co.contact_terms(cm, obs, Cp, DHAT, KAPPA)
            Em, Gm, _ = co.contact_terms(cm, obs, Cm, DHAT, KAPPA)
            fd = (Ep - Em) / (2 * h)
            assert abs(fd - G[al, c]) <= 1e-5 * np.abs(G).max(), (al, c)
            # column (al, c) of the full Hessian against the gradient's differences
            dG = (Gp - Gm) / (2 * h)
            col = np.zeros_like(G)
            nu = 11
            for be in range(prob.n_cp):
                du, dv = al % nu - be % nu, al // nu - be // nu
                if abs(du) <= 2 and abs(dv) <= 2:
                    col[be] = Kf[be, (dv + 2) * 5 + du + 2][:, c]
            assert np.abs(dG - col).max() <= 1e-4 * np.abs(Kf).max(), (al, c)


def test_projected_pair_hessian_is_psd_and_below_full():
    obs = pyramid()
    rng = np.random.default_rng(5)
    seen = 0
    for _ in range(400):
        x = np.array([0.25, 0.25, 0.0]) + rng.uniform(-0.14, 0.14, 3) * np.array([1, 1, 0.2])
        _, _, Hp = co.vertex_terms(x, obs, DHAT, "projected")
        _, _, Hf = co.vertex_terms(x, obs, DHAT, "full")
        if not Hp.any():
            continue
        seen += 1
        assert np.linalg.eigvalsh(Hp).min() >= -1e-9 * np.abs(Hp).max()
        assert np.linalg.eigvalsh(Hf - Hp).max() <= 1e-9 * np.abs(Hp).max()
    assert seen > 20


def test_step_bound_falling_vertex(orc):
    rest, C = flat_patch(h=0.01)
    prob = orc.Problem(9, 9, rest, (1.0, 1.0, 0.5, 0.0, 1.0))
    cm = co.ContactMesh(prob, 9, 9)
    D = np.zeros_like(C)
    D[:, 2] = -0.05
    assert abs(co.step_bound(cm, plane(), C, D) - 0.9 * 0.01 / 0.05) < 1e-14
    D[:, 2] = +0.05
    assert co.step_bound(cm, plane(), C, D) == 1.0
