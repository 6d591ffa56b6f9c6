"""Seeded synthetic cloth states shaped like the paper's scenes.

This module is the only code shared by the CUDA path, the CPU oracle and the
bench: it draws inputs and holds none of the method's arithmetic (no basis
functions, quadrature, energies or derivatives).  Random numbers come from
splitmix64 (Steele, Lea & Flood 2014, as published by Vigna) driven by a
counter, turned into uniforms with the top 53 bits and into normals with the
Box-Muller transform, so every array is reproducible on any machine and any
numpy version.

Geometry conventions
--------------------
* A patch has ``nu x nv`` control points (``nu, nv >= 5``) on open uniform
  quadratic knot vectors ``(0,0,0,1,...,S,S,S)`` with ``S = n - 2`` spans per
  axis (integer lattice starting at 0, Sec. 3.1.2).
* Control point ``alpha = j * nu + i`` (``i`` along u, ``j`` along v).
* ``rest`` is ``(nu*nv, 2)`` float64 material coordinates; ``C`` is
  ``(nu*nv, 3)`` float64 world positions.
* Flat rest states place control point ``(i, j)`` at the Greville abscissae
  ``gamma = (0, 1/2, 3/2, ..., S-1/2, S)`` scaled to the patch size, the layout
  drawn in the paper's reduced-quadrature figure (Fig. 3).

Material mapping (a reading; the paper defers it to its supplement)
--------------------------------------------------------------------
``mu_st1 = mu_st2 = E h / 2``, ``mu_sh = G h / 2`` with ``G = E / (2 (1 + nu))``,
``mu_bd = E h^3 / (12 (1 - nu^2))`` and ``rho_area`` in kg/m^2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """``n`` outputs of splitmix64 for counters ``offset+1 .. offset+n``."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m, 2 * offset)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * math.pi * u2)
    z[1::2] = r * np.sin(2.0 * math.pi * u2)
    return z[:n]


@dataclass
class Material:
    mu_st1: float
    mu_st2: float
    mu_sh: float
    mu_bd: float
    rho_area: float

    @staticmethod
    def from_engineering(E: float, nu: float, h: float, rho_area: float) -> "Material":
        G = E / (2.0 * (1.0 + nu))
        return Material(E * h / 2.0, E * h / 2.0, G * h / 2.0,
                        E * h ** 3 / (12.0 * (1.0 - nu * nu)), rho_area)

    def as_tuple(self):
        return (self.mu_st1, self.mu_st2, self.mu_sh, self.mu_bd, self.rho_area)


@dataclass
class Patch:
    """One synthetic cloth state: geometry, material, scene and current state."""
    name: str
    nu: int
    nv: int
    rest: np.ndarray            # (N, 2) float64
    C: np.ndarray               # (N, 3) float64, current positions
    Chat: np.ndarray            # (N, 3) float64, C^n + dt v^n
    material: Material
    dt: float
    gravity: tuple
    pinned: np.ndarray          # int32 control-point indices
    meta: dict = field(default_factory=dict)

    @property
    def n_cp(self) -> int:
        return self.nu * self.nv

    @property
    def n_spans(self) -> int:
        return (self.nu - 2) * (self.nv - 2)


def greville(n: int) -> np.ndarray:
    """Greville abscissae of the open uniform quadratic knot vector with n-2 spans."""
    S = n - 2
    g = np.empty(n)
    g[0] = 0.0
    g[-1] = float(S)
    g[1:-1] = np.arange(n - 2) + 0.5
    return g


def flat_rest(nu: int, nv: int, Lu: float, Lv: float, angle: float = 0.0,
              origin=(0.0, 0.0)) -> np.ndarray:
    """Greville-placed flat rest control points, optionally rotated in the plane."""
    gu = greville(nu) * (Lu / (nu - 2))
    gv = greville(nv) * (Lv / (nv - 2))
    X = np.empty((nv, nu, 2))
    X[:, :, 0] = gu[None, :]
    X[:, :, 1] = gv[:, None]
    X = X.reshape(-1, 2)
    if angle != 0.0:
        c, s = math.cos(angle), math.sin(angle)
        X = X @ np.array([[c, s], [-s, c]])
    return X + np.asarray(origin)[None, :]


def corner_pins_top(nu: int, nv: int) -> np.ndarray:
    """The two control points at the v = max corners (the top corners)."""
    return np.array([(nv - 1) * nu, (nv - 1) * nu + nu - 1], dtype=np.int32)


def edge_pins_u0(nu: int, nv: int) -> np.ndarray:
    """Every control point on the u = 0 edge (the x = 0 edge of a flat rest)."""
    return (np.arange(nv, dtype=np.int32) * nu)


def lift(rest: np.ndarray) -> np.ndarray:
    C = np.zeros((rest.shape[0], 3))
    C[:, :2] = rest
    return C


def config_square(seed: int = 1, n: int = 32) -> Patch:
    """Square patch, 1 m x 1 m, seeded noise of 0.01 span + 2 mm wrinkle along x.

    E = 1e5 Pa, nu = 0.3, h = 1 mm, 200 kg/m^2; dt = 0.01 s; gravity -y; the two
    top corners pinned.  The wrinkle wavelength (8 spans) is a reading.
    """
    span = 1.0 / (n - 2)
    rest = flat_rest(n, n, 1.0, 1.0)
    C = lift(rest)
    C += (0.01 * span) * normal(seed, C.size).reshape(C.shape)
    lam = 8 * span
    C[:, 2] += 0.002 * np.sin(2.0 * math.pi * rest[:, 0] / lam)
    mat = Material.from_engineering(1e5, 0.3, 1e-3, 200.0)
    return Patch(f"square{n}", n, n, rest, C, C.copy(), mat, 0.01, (0.0, -9.81, 0.0),
                 corner_pins_top(n, n), {"seed": seed, "span_m": span})


def config_drape(seed: int = 1, n: int = 256, mu_bd: float = 1e-5, size_m: float = 2.0) -> Patch:
    """Drape: n x n patch, size_m square, sigma = 1 mm noise, u = 0 edge pinned, gravity -z."""
    rest = flat_rest(n, n, size_m, size_m)
    C = lift(rest)
    C += 1e-3 * normal(seed, C.size).reshape(C.shape)
    mat = Material.from_engineering(1e5, 0.3, 1e-3, 200.0)
    mat.mu_bd = mu_bd
    return Patch(f"drape{n}", n, n, rest, C, C.copy(), mat, 0.01, (0.0, 0.0, -9.81),
                 edge_pins_u0(n, n), {"seed": seed, "mu_bd": mu_bd, "size_m": size_m})


def wrinkle_field(seed: int, X: np.ndarray, span: float, k: int = 8) -> np.ndarray:
    """Sum of k sinusoids: direction U[0, 2 pi), wavelength log-U[4, 64] spans,
    amplitude U[1, 5] mm, phase U[0, 2 pi)."""
    u = uniform(seed ^ 0x5EED, 4 * k)
    z = np.zeros(X.shape[0])
    for m in range(k):
        th = 2.0 * math.pi * u[4 * m]
        lam = span * math.exp(math.log(4.0) + u[4 * m + 1] * (math.log(64.0) - math.log(4.0)))
        amp = 1e-3 + 4e-3 * u[4 * m + 2]
        ph = 2.0 * math.pi * u[4 * m + 3]
        z += amp * np.sin(2.0 * math.pi * (X[:, 0] * math.cos(th) + X[:, 1] * math.sin(th)) / lam + ph)
    return z


def config_wrinkle(seed: int = 1, n: int = 1024, size_m: float = 4.0, crop: int | None = None) -> Patch:
    """Precision-sweep patch: n x n, size_m square, multi-frequency wrinkle field.

    ``crop`` returns the leading ``crop x crop`` control points of the same
    field (same span length), the oracle's sample of the full patch.
    """
    span = size_m / (n - 2)
    m = n if crop is None else crop
    rest = flat_rest(m, m, span * (m - 2), span * (m - 2))
    C = lift(rest)
    C[:, 2] += wrinkle_field(seed, rest, span)
    mat = Material.from_engineering(1e5, 0.3, 1e-3, 200.0)
    return Patch(f"wrinkle{n}" + (f"_crop{m}" if crop else ""), m, m, rest, C, C.copy(), mat, 0.01,
                 (0.0, 0.0, -9.81), corner_pins_top(m, m), {"seed": seed, "span_m": span})


def config_random_small(seed: int, nu: int, nv: int, angle: float | None = None,
                        noise: float = 0.05, curved: float = 0.0) -> Patch:
    """Small generic patch for parity tests: rotated (optionally curved) rest,
    noisy world state, random material, a few pins."""
    u = uniform(seed, 8)
    if angle is None:
        angle = 2.0 * math.pi * u[0]
    Lu, Lv = 0.3 + 0.4 * u[1], 0.3 + 0.4 * u[2]
    rest = flat_rest(nu, nv, Lu, Lv, angle=angle)
    if curved != 0.0:
        # smooth in-plane bend of the rest map: a curved, non-affine X(u, v)
        g = rest - rest.mean(axis=0)
        rest = rest + curved * np.stack([g[:, 1] ** 2, 0.5 * g[:, 0] ** 2], axis=1)
    C = lift(rest)
    span = min(Lu / (nu - 2), Lv / (nv - 2))
    C += noise * span * normal(seed + 17, C.size).reshape(C.shape)
    E = math.exp(math.log(1e4) + u[3] * (math.log(1e6) - math.log(1e4)))
    mat = Material.from_engineering(E, 0.2 + 0.25 * u[4], 1e-3, 0.2 + u[5])
    pins = np.array([0, nu - 1], dtype=np.int32)
    Chat = C + 0.01 * span * normal(seed + 31, C.size).reshape(C.shape)
    return Patch(f"rand{nu}x{nv}", nu, nv, rest, C, Chat, mat, 0.01, (0.0, -9.81, 0.0), pins,
                 {"seed": seed, "span_m": span})


def config_batch(seed: int = 1, count: int = 64, lo: int = 16, hi: int = 192, span_m: float = 0.01,
                 sigma: float = 1e-3) -> list:
    """Batched garments: `count` independent patches.  Per patch: nu and nv
    independently uniform in [lo, hi] (non-square), E log-uniform in
    [1e4, 1e6] Pa, Poisson ratio uniform in [0.2, 0.45], h = 1 mm,
    200 kg/m^2, a rest map rotated by a uniform angle in the plane with 1 cm
    spans, the drape's perturbation law (sigma = 1 mm per component), the two
    top corners pinned, gravity -y, dt = 0.01 s."""
    u = uniform(seed ^ 0xBA7C4, 5 * count)
    out = []
    for p in range(count):
        up = u[5 * p:5 * p + 5]
        nu = lo + min(int(up[0] * (hi - lo + 1)), hi - lo)
        nv = lo + min(int(up[1] * (hi - lo + 1)), hi - lo)
        E = math.exp(math.log(1e4) + up[2] * (math.log(1e6) - math.log(1e4)))
        pr = 0.2 + 0.25 * up[3]
        angle = 2.0 * math.pi * up[4]
        rest = flat_rest(nu, nv, span_m * (nu - 2), span_m * (nv - 2), angle=angle)
        C = lift(rest)
        C += sigma * normal(seed * 7919 + 101 + p, C.size).reshape(C.shape)
        mat = Material.from_engineering(E, pr, 1e-3, 200.0)
        out.append(Patch(f"garment{p}_{nu}x{nv}", nu, nv, rest, C, C.copy(), mat, 0.01, (0.0, -9.81, 0.0),
                         corner_pins_top(nu, nv), {"seed": seed, "index": p, "E": E, "poisson": pr,
                                                   "angle": angle}))
    return out


def config_learned(seed: int = 1, n: int = 512, size_m: float = 1.0) -> Patch:
    """Newton system for the learned preconditioner: n x n patch, size_m
    square, E = 1e5 Pa, nu = 0.3, h = 1 mm, 200 kg/m^2, dt = 0.01 s, gravity
    -y, the two top corners pinned.  The membrane / bending stiffness ratio
    mu_st h_span^2 / mu_bd is log-uniform in [1e3, 1e5] (h_span the span
    length); the state is the rest plus sigma = 1 mm noise and a seeded
    multi-frequency wrinkle field."""
    u = uniform(seed ^ 0x1EA4, 2)
    ratio = math.exp(math.log(1e3) + u[0] * (math.log(1e5) - math.log(1e3)))
    span = size_m / (n - 2)
    rest = flat_rest(n, n, size_m, size_m)
    C = lift(rest)
    C += 1e-3 * normal(seed * 104729 + 7, C.size).reshape(C.shape)
    C[:, 2] += wrinkle_field(seed, rest, span, k=6)
    mat = Material.from_engineering(1e5, 0.3, 1e-3, 200.0)
    mat.mu_bd = mat.mu_st1 * span * span / ratio
    return Patch(f"learned{n}", n, n, rest, C, C.copy(), mat, 0.01, (0.0, -9.81, 0.0), corner_pins_top(n, n),
                 {"seed": seed, "ratio": ratio, "span_m": span})


def distorted_rest(kind: str, param: float, nu: int, nv: int, size_m: float = 1.0) -> np.ndarray:
    """Rest control points of the three distortion families of the paper's
    non-rectangular-domain study (Sec. 6): Greville-placed control points of
    the unit square mapped to
      "aspect"  a size x (param * size) rectangle (aspect ratio 1:param);
      "skew"    a parallelogram with interior angle param degrees at the
                origin (sides of length size);
      "bend"    the unit square whose v = max edge is pulled inwards at its
                middle so that the control polygon of that edge turns with
                interior angle param degrees (v scaled linearly between the
                straight bottom edge and the bent top edge)."""
    gu, gv = greville(nu) / (nu - 2), greville(nv) / (nv - 2)
    U, V = np.meshgrid(gu, gv)          # (nv, nu): control point (i, j) at [j, i]
    if kind == "aspect":
        X, Y = U * size_m, V * size_m * param
    elif kind == "skew":
        th = math.radians(param)
        X, Y = (U + V * math.cos(th)) * size_m, V * math.sin(th) * size_m
    elif kind == "bend":
        h = 0.5 * math.tan(math.radians(180.0 - param) / 2.0)
        top = 1.0 - h * (1.0 - np.abs(2.0 * U - 1.0))
        X, Y = U * size_m, V * top * size_m
    else:
        raise ValueError(kind)
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def config_distorted(kind: str, param: float, nu: int = 24, nv: int = 24, seed: int = 1) -> Patch:
    """A cloth state on a distorted rest domain (distorted_rest): a smooth,
    non-affine deformation of it (2 % stretch along X1, 1 % shear, an in-plane
    ripple and an out-of-plane bulge of 3 % of the extent) plus seeded noise
    of 1e-3 span; E = 1e5 Pa, nu = 0.3, h = 1 mm, 200 kg/m^2, dt = 0.01 s,
    gravity -z, corners of the v = 0 edge pinned."""
    rest = distorted_rest(kind, param, nu, nv)
    lo, hi = rest.min(axis=0), rest.max(axis=0)
    L = hi - lo
    Xn = (rest - lo) / L
    C = np.zeros((rest.shape[0], 3))
    C[:, 0] = 1.02 * rest[:, 0] + 0.01 * rest[:, 1]
    C[:, 1] = 0.99 * rest[:, 1] + 0.005 * L.min() * np.sin(2.0 * math.pi * Xn[:, 0])
    C[:, 2] = 0.03 * L.min() * np.sin(math.pi * Xn[:, 0]) * np.sin(math.pi * Xn[:, 1])
    span = min(L[0] / (nu - 2), L[1] / (nv - 2))
    C += 1e-3 * span * normal(seed, C.size).reshape(C.shape)
    mat = Material.from_engineering(1e5, 0.3, 1e-3, 200.0)
    pins = np.array([0, nu - 1], dtype=np.int32)
    return Patch(f"{kind}{param:g}", nu, nv, rest, C, C.copy(), mat, 0.01, (0.0, 0.0, -9.81), pins,
                 {"seed": seed, "kind": kind, "param": param, "span_m": span})


def pyramid_obstacle(cx=0.25, cy=0.25, apex_z=-0.004, base_z=-0.03, half=0.2):
    """A square pyramid (apex up) as a static obstacle triangle mesh: 5
    vertices, the 4 side faces.  Returns (vertices (5, 3), triangles (4, 3))."""
    V = np.array([(cx - half, cy - half, base_z), (cx + half, cy - half, base_z), (cx + half, cy + half, base_z),
                  (cx - half, cy + half, base_z), (cx, cy, apex_z)])
    T = np.array([(0, 1, 4), (1, 2, 4), (2, 3, 4), (3, 0, 4)], dtype=np.int32)
    return V, T


def sphere_obstacle(center, radius, n_lat=24, n_lon=48):
    """A UV sphere as a static obstacle triangle mesh (vertices, triangles)."""
    cx, cy, cz = center
    V = [(cx, cy, cz + radius)]
    for i in range(1, n_lat):
        th = math.pi * i / n_lat
        for j in range(n_lon):
            ph = 2.0 * math.pi * j / n_lon
            V.append((cx + radius * math.sin(th) * math.cos(ph), cy + radius * math.sin(th) * math.sin(ph),
                      cz + radius * math.cos(th)))
    V.append((cx, cy, cz - radius))
    T = []
    for j in range(n_lon):
        T.append((0, 1 + j, 1 + (j + 1) % n_lon))
    for i in range(n_lat - 2):
        r0, r1 = 1 + i * n_lon, 1 + (i + 1) * n_lon
        for j in range(n_lon):
            a, b = r0 + j, r0 + (j + 1) % n_lon
            c, d = r1 + j, r1 + (j + 1) % n_lon
            T += [(a, c, b), (b, c, d)]
    last = len(V) - 1
    r0 = 1 + (n_lat - 2) * n_lon
    for j in range(n_lon):
        T.append((r0 + j, last, r0 + (j + 1) % n_lon))
    return np.array(V), np.array(T, dtype=np.int32)


def config_contact(seed: int = 2, n: int = 11, size_m: float = 0.5) -> Patch:
    """A cloth patch just above the apex of a pyramid obstacle
    (pyramid_obstacle): n x n control points, size_m square, height 6 mm
    with a 4 mm standing wave and seeded 1 mm noise, E = 1e5 Pa, nu = 0.3,
    h = 1 mm, 200 kg/m^2, dt = 0.01 s, gravity -z, corners of the v = 0 edge
    pinned.  Contact parameters in meta: dhat = 0.02 m, kappa = 1e3 Pa."""
    rest = flat_rest(n, n, size_m, size_m)
    C = lift(rest)
    X = rest
    C[:, 2] = 0.006 + 0.004 * np.sin(2 * math.pi * X[:, 0] / size_m) * np.cos(2 * math.pi * X[:, 1] / size_m)
    C += 1e-3 * normal(seed, C.size).reshape(C.shape)
    mat = Material.from_engineering(1e5, 0.3, 1e-3, 200.0)
    pins = np.array([0, n - 1], dtype=np.int32)
    return Patch(f"contact{n}", n, n, rest, C, C.copy(), mat, 0.01, (0.0, 0.0, -9.81), pins,
                 {"seed": seed, "dhat": 0.02, "kappa": 1e3})


def synthetic_stencil(seed: int, nu: int, nv: int, pinned=(), coupling: float = 0.15) -> np.ndarray:
    """A seeded symmetric positive definite matrix in the 5 x 5 block-stencil
    shape of the global Hessian, (N, 25, 3, 3) with slot = (dv + 2) * 5 + (du + 2):
    normal off-diagonal 3 x 3 blocks of scale `coupling` for every neighbour pair
    (block (beta, alpha) the transpose of block (alpha, beta)), diagonal blocks
    A A^T / 3 + (1 + the row's absolute off-diagonal sum) I, so the matrix is
    strictly diagonally dominant; rows and columns of pinned control points
    are replaced by the identity.  Input for tests of solvers and of the
    learned preconditioner that need no cloth state."""
    N = nu * nv
    K = np.zeros((N, 25, 3, 3))
    j, i = np.divmod(np.arange(N), nu)
    k = 0
    for dv in range(-2, 3):
        for du in range(-2, 3):
            s = (dv + 2) * 5 + (du + 2)
            if s <= 12:
                continue
            B = coupling * normal(seed, 9 * N, offset=9 * N * k).reshape(N, 3, 3)
            k += 1
            ok = (i + du >= 0) & (i + du < nu) & (j + dv >= 0) & (j + dv < nv)
            a = np.nonzero(ok)[0]
            b = a + dv * nu + du
            K[a, s] = B[a]
            K[b, 24 - s] = np.transpose(B[a], (0, 2, 1))
    A = normal(seed ^ 0xD1A6, 9 * N).reshape(N, 3, 3)
    off = np.abs(K).sum(axis=(1, 3)) - np.abs(K[:, 12]).sum(axis=2)   # (N, 3) row sums
    D = np.einsum("nab,ncb->nac", A, A) / 3.0
    D += (1.0 + off.max(axis=1))[:, None, None] * np.eye(3)[None]
    K[:, 12] = D
    pins = np.asarray(pinned, dtype=np.int64).ravel()
    if pins.size:
        pj, pi = np.divmod(pins, nu)
        for dv in range(-2, 3):
            for du in range(-2, 3):
                s = (dv + 2) * 5 + (du + 2)
                ok = (pi + du >= 0) & (pi + du < nu) & (pj + dv >= 0) & (pj + dv < nv)
                q = pins[ok] + dv * nu + du
                K[pins[ok], s] = 0.0
                K[q, 24 - s] = 0.0
        K[pins, 12] = np.eye(3)[None]
    return K


def crop(patch: Patch, mu: int, mv: int | None = None) -> Patch:
    """The leading mu x mv control points of a patch (same span length, same
    state, pins restricted to the crop): a bounded sample of a large workload."""
    mv = mu if mv is None else mv
    idx = np.array([j * patch.nu + i for j in range(mv) for i in range(mu)])
    remap = {int(a): k for k, a in enumerate(idx)}
    pins = np.array([remap[int(p)] for p in patch.pinned if int(p) in remap], dtype=np.int32)
    return Patch(f"{patch.name}_crop{mu}x{mv}", mu, mv, patch.rest[idx].copy(), patch.C[idx].copy(),
                 patch.Chat[idx].copy(), patch.material, patch.dt, patch.gravity, pins,
                 dict(patch.meta, crop=(mu, mv)))
