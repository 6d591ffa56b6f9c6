"""Plain FP64 NumPy oracle of the contact term (TEST INFRASTRUCTURE ONLY:
imported by tests/, never by the product).

What it computes (Sec. 4.3, with the barrier of incremental potential
contact):

* The contact mesh: a regular triangle mesh embedded in the B-spline
  surface.  Its mu x mv vertices sit at fixed parametric coordinates
  u_i = S_u i / (mu - 1), v_j = S_v j / (mv - 1); vertex k = j mu + i belongs
  to the span (clamp(floor(u), 0, S_u - 1), clamp(floor(v), 0, S_v - 1)) and
  its world position is x_k = sum_l N_l(u, v) C_l over that span's nine
  control points (Eq. trig mesh node from control points).  Cells are split
  into two triangles along alternating diagonals.  Each vertex carries the
  area weight A_k = one third of the rest areas of its triangles (rest
  positions X_k = sum_l N_l X_l).
* The obstacle: a static triangle mesh.  For a vertex x and an obstacle
  triangle t, d = distance from x to t, attained at the closest point q on a
  feature of t (its interior, an edge or a corner).  The pair counts when
  d < dhat and, for an edge or a corner, t is the lowest-index triangle
  containing that feature (each point-edge and point-corner distance enters
  once, as in IPC's constraint set).
* Barrier (dimensionless, in x = d / dhat): beta(x) = -(x - 1)^2 ln x for
  0 < x < 1, else 0.  Contact potential B(C) = kappa sum_k A_k sum_pairs
  beta(d / dhat), kappa in Pa.
* Gradient w.r.t. the vertex: kappa A beta'(x) / dhat * u, u = (x - q) / d.
  Hessian w.r.t. the vertex: kappa A (beta''(x) / dhat^2 u u^T + beta'(x) /
  dhat * grad^2 d), grad^2 d = 0 (interior), (I - e e^T - u u^T) / d (edge of
  direction e), (I - u u^T) / d (corner).  beta' < 0 and grad^2 d is PSD and
  orthogonal to u, so the PSD projection of the pair Hessian is
  kappa A beta''(x) / dhat^2 u u^T.
* Chain rule to the control points (Eq. gradient and hessian of contact
  barrier): dB/dC_l = sum_k N_l(k) dB/dx_k, d2B/dC_l dC_m = sum_k N_l(k)
  N_m(k) d2B/dx_k^2 (x_k is linear in C, so no second term).
* Conservative step bound for the line search: the distance from a moving
  point x + a dx to a convex triangle is convex in a, hence at least
  d + a (u . dx); the point stays at least 0.1 d away from t for
  a <= 0.9 d / (-u . dx) when u . dx < 0.  The bound of a step is the
  smallest over all vertices and obstacle triangles, and at most 1.
"""
from __future__ import annotations

import math

import numpy as np


# ---- barrier -------------------------------------------------------------

def beta(x):
    return -(x - 1.0) ** 2 * math.log(x) if 0.0 < x < 1.0 else 0.0


def beta_d1(x):
    return (-2.0 * (x - 1.0) * math.log(x) - (x - 1.0) ** 2 / x) if 0.0 < x < 1.0 else 0.0


def beta_d2(x):
    if not 0.0 < x < 1.0:
        return 0.0
    return -2.0 * math.log(x) - 4.0 * (x - 1.0) / x + (x - 1.0) ** 2 / (x * x)


# ---- closest point on a triangle ------------------------------------------

FEATURE_TOL = 1e-10


def closest_point(p, a, b, c):
    """Closest point q of triangle (a, b, c) to p and its feature: ("face",),
    ("edge", i, j) with corner indices i < j, or ("vertex", i).  q from the
    seven Voronoi regions of the triangle (barycentric sign tests); the
    feature from q's barycentric coordinates, a coordinate at most
    FEATURE_TOL counting as zero, so that a point over a shared edge is on
    that edge for both of its triangles whatever the rounding."""
    q = _closest(p, a, b, c)
    a, b, c = (np.asarray(v, dtype=np.float64) for v in (a, b, c))
    ab, ac, aq = b - a, c - a, q - a
    g00, g01, g11 = ab @ ab, ab @ ac, ac @ ac
    r0, r1 = ab @ aq, ac @ aq
    det = g00 * g11 - g01 * g01
    lam1 = (g11 * r0 - g01 * r1) / det
    lam2 = (g00 * r1 - g01 * r0) / det
    lam = (1.0 - lam1 - lam2, lam1, lam2)
    nz = [k for k in range(3) if lam[k] > FEATURE_TOL]
    if len(nz) == 3:
        return q, ("face",)
    if len(nz) == 2:
        return q, ("edge", nz[0], nz[1])
    return q, ("vertex", nz[0] if nz else int(np.argmax(lam)))


def _closest(p, a, b, c):
    p, a, b, c = (np.asarray(v, dtype=np.float64) for v in (p, a, b, c))
    ab, ac, ap = b - a, c - a, p - a
    d1, d2 = ab @ ap, ac @ ap
    if d1 <= 0.0 and d2 <= 0.0:
        return a
    bp = p - b
    d3, d4 = ab @ bp, ac @ bp
    if d3 >= 0.0 and d4 <= d3:
        return b
    vc = d1 * d4 - d3 * d2
    if vc <= 0.0 and d1 >= 0.0 and d3 <= 0.0:
        return a + (d1 / (d1 - d3)) * ab
    cp = p - c
    d5, d6 = ab @ cp, ac @ cp
    if d6 >= 0.0 and d5 <= d6:
        return c
    vb = d5 * d2 - d1 * d6
    if vb <= 0.0 and d2 >= 0.0 and d6 <= 0.0:
        return a + (d2 / (d2 - d6)) * ac
    va = d3 * d6 - d5 * d4
    if va <= 0.0 and (d4 - d3) >= 0.0 and (d5 - d6) >= 0.0:
        w = (d4 - d3) / ((d4 - d3) + (d5 - d6))
        return b + w * (c - b)
    denom = 1.0 / (va + vb + vc)
    v, w = vb * denom, vc * denom
    return a + ab * v + ac * w


class Obstacle:
    """Static triangle mesh with the owner (lowest-index incident triangle) of
    every edge and corner."""

    def __init__(self, V, T):
        self.V = np.asarray(V, dtype=np.float64).reshape(-1, 3)
        self.T = np.asarray(T, dtype=np.int64).reshape(-1, 3)
        self.edge_owner, self.vert_owner = {}, {}
        for t, tri in enumerate(self.T):
            for i in range(3):
                self.vert_owner.setdefault(int(tri[i]), t)
                for j in range(i + 1, 3):
                    e = tuple(sorted((int(tri[i]), int(tri[j]))))
                    self.edge_owner.setdefault(e, t)

    def counts(self, t, feature):
        tri = self.T[t]
        if feature[0] == "face":
            return True
        if feature[0] == "edge":
            e = tuple(sorted((int(tri[feature[1]]), int(tri[feature[2]]))))
            return self.edge_owner[e] == t
        return self.vert_owner[int(tri[feature[1]])] == t


# ---- contact mesh -----------------------------------------------------------

class ContactMesh:
    """Vertices at fixed parametric points of a patch (oracle.Problem)."""

    def __init__(self, prob, mu, mv):
        self.prob, self.mu, self.mv = prob, mu, mv
        Su, Sv = prob.nu - 2, prob.nv - 2
        self.uv, self.owner, self.W = [], [], []
        for j in range(mv):
            for i in range(mu):
                u, v = Su * i / (mu - 1), Sv * j / (mv - 1)
                a, b = min(max(int(math.floor(u)), 0), Su - 1), min(max(int(math.floor(v)), 0), Sv - 1)
                N = prob.basis9(u, v, a, b)[0]
                self.uv.append((u, v))
                self.owner.append((a, b))
                self.W.append(N)
        self.W = np.array(self.W)
        self.tris = []
        for j in range(mv - 1):
            for i in range(mu - 1):
                k = j * mu + i
                if (i + j) % 2 == 0:
                    self.tris += [(k, k + 1, k + mu + 1), (k, k + mu + 1, k + mu)]
                else:
                    self.tris += [(k, k + 1, k + mu), (k + 1, k + mu + 1, k + mu)]
        Xr = self.positions(np.concatenate([prob.rest, np.zeros((prob.n_cp, 1))], axis=1))
        self.area = np.zeros(mu * mv)
        for (p, q, r) in self.tris:
            A = 0.5 * np.linalg.norm(np.cross(Xr[q] - Xr[p], Xr[r] - Xr[p]))
            for k in (p, q, r):
                self.area[k] += A / 3.0

    def cps(self, k):
        """Control-point indices of vertex k's span, in basis9 order (l = 3 lj + li)."""
        a, b = self.owner[k]
        nu = self.prob.nu
        return [(b + lj) * nu + a + li for lj in range(3) for li in range(3)]

    def positions(self, C):
        C = np.asarray(C, dtype=np.float64).reshape(-1, 3)
        return np.array([self.W[k] @ C[self.cps(k)] for k in range(len(self.W))])


# ---- contact potential ------------------------------------------------------

def vertex_terms(x, obs: Obstacle, dhat, hessian="projected"):
    """Sum over the counted pairs of one vertex: beta, its gradient and its
    Hessian w.r.t. x (per unit kappa A).  hessian: "projected" or "full"."""
    e, g, H = 0.0, np.zeros(3), np.zeros((3, 3))
    for t in range(len(obs.T)):
        a, b, c = obs.V[obs.T[t]]
        q, feat = closest_point(x, a, b, c)
        d = float(np.linalg.norm(x - q))
        if not d < dhat or not obs.counts(t, feat):
            continue
        if d <= 0.0:
            raise FloatingPointError("a contact vertex touches the obstacle")
        u = (x - q) / d
        s = d / dhat
        e += beta(s)
        g += beta_d1(s) / dhat * u
        H += beta_d2(s) / dhat ** 2 * np.outer(u, u)
        if hessian == "full":
            if feat[0] == "edge":
                ed = obs.V[obs.T[t][feat[2]]] - obs.V[obs.T[t][feat[1]]]
                ed /= np.linalg.norm(ed)
                H += beta_d1(s) / dhat * (np.eye(3) - np.outer(ed, ed) - np.outer(u, u)) / d
            elif feat[0] == "vertex":
                H += beta_d1(s) / dhat * (np.eye(3) - np.outer(u, u)) / d
    return e, g, H


def contact_terms(cm: ContactMesh, obs: Obstacle, C, dhat, kappa, hessian="projected"):
    """B(C), dB/dC (N, 3) and the stencil Hessian (N, 25, 3, 3) of the contact
    potential; pinned rows are not eliminated here."""
    N, nu = cm.prob.n_cp, cm.prob.nu
    X = cm.positions(C)
    E, G, K = 0.0, np.zeros((N, 3)), np.zeros((N, 25, 3, 3))
    for k, x in enumerate(X):
        e, g, H = vertex_terms(x, obs, dhat, hessian)
        if e == 0.0 and not g.any():
            continue
        w = kappa * cm.area[k]
        E += w * e
        idx = cm.cps(k)
        for l, al in enumerate(idx):
            G[al] += w * cm.W[k][l] * g
            for m, be in enumerate(idx):
                du, dv = be % nu - al % nu, be // nu - al // nu
                K[al, (dv + 2) * 5 + du + 2] += w * cm.W[k][l] * cm.W[k][m] * H
    return E, G, K


def step_bound(cm: ContactMesh, obs: Obstacle, C, D):
    """Largest a <= 1 with every vertex kept at least 0.1 of its distance
    from every obstacle triangle along C + a D (convexity bound)."""
    X, DX = cm.positions(C), cm.positions(D)
    amax = 1.0
    for x, dx in zip(X, DX):
        for t in range(len(obs.T)):
            a, b, c = obs.V[obs.T[t]]
            q, _ = closest_point(x, a, b, c)
            d = float(np.linalg.norm(x - q))
            rate = float((x - q) @ dx) / d
            if rate < 0.0:
                amax = min(amax, 0.9 * d / -rate)
    return amax


def eliminate(K, G, pinned, nu, nv):
    """Dirichlet elimination of a contact term: rows and columns of pinned
    control points zeroed (the elastic term already holds their identity)."""
    K, G = K.copy(), G.copy()
    pins = set(int(p) for p in pinned)
    for al in range(nu * nv):
        i, j = al % nu, al // nu
        for dv in range(-2, 3):
            for du in range(-2, 3):
                be = (j + dv) * nu + i + du
                if 0 <= i + du < nu and 0 <= j + dv < nv and (al in pins or be in pins):
                    K[al, (dv + 2) * 5 + du + 2] = 0.0
    G[list(pins)] = 0.0
    return K, G


def newton_step(orc, prob, scene, cm, obs, C, Chat, dhat, kappa, max_halvings=30):
    """One projected Newton iteration of the incremental potential plus the
    contact potential: K = elastic (projected, Dirichlet-eliminated) + contact
    (projected pair Hessians), d from the banded Cholesky, the line search
    started at min(1, step bound) and halved until the total energy does not
    increase.  Returns (C_new, status, info)."""
    C = np.asarray(C, dtype=np.float64).reshape(-1, 3)
    E_el, g_el, K_el = orc.evaluate(prob, scene, C, Chat)
    E_c, G_c, K_c = contact_terms(cm, obs, C, dhat, kappa)
    K_c, G_c = eliminate(K_c, G_c, scene.pinned, prob.nu, prob.nv)
    g, K = g_el + G_c, K_el + K_c
    d = orc.solve_banded(prob.nu, prob.nv, K, -g)
    E0 = E_el + E_c
    a0 = min(1.0, step_bound(cm, obs, C, d))
    alpha, h = a0, 0
    while True:
        Ct = C + alpha * d
        E1 = orc.energy(prob, scene, Ct, Chat) + contact_terms(cm, obs, Ct, dhat, kappa)[0]
        if E1 <= E0:
            return Ct, 0, {"E0": E0, "E1": E1, "alpha": alpha, "alpha0": a0, "halvings": h, "d": d}
        if h == max_halvings:
            return C, -3, {"E0": E0, "E1": E1, "alpha": 0.0, "alpha0": a0, "halvings": h, "d": d}
        alpha *= 0.5
        h += 1
