"""ctypes wrapper of the plain FP64 CPU oracle (``bsc_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product package never imports it.  Arrays use the oracle's AoS layout:
``rest (N, 2)``, ``C (N, 3)``, stencil ``K (N, 25, 3, 3)`` with
``slot = (dv + 2) * 5 + (du + 2)``.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bsc_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

RULE_REDUCED, RULE_GAUSS2, RULE_GAUSS3, RULE_STANDARD = 0, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no fast-math)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "bsc_oracle.h"))):
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"])
    return _LIB


class _Problem(ct.Structure):
    _fields_ = [("nu", ct.c_int), ("nv", ct.c_int), ("rest", ct.POINTER(ct.c_double)),
                ("mu_st1", ct.c_double), ("mu_st2", ct.c_double), ("mu_sh", ct.c_double),
                ("mu_bd", ct.c_double), ("rho", ct.c_double),
                ("mem_rule", ct.c_int), ("bend_rule", ct.c_int)]


class _Scene(ct.Structure):
    _fields_ = [("dt", ct.c_double), ("gravity", ct.c_double * 3),
                ("pinned", ct.POINTER(ct.c_int)), ("n_pinned", ct.c_int), ("project", ct.c_int)]


class NewtonReport(ct.Structure):
    _fields_ = [("E0", ct.c_double), ("E1", ct.c_double), ("alpha", ct.c_double),
                ("dir_inf", ct.c_double), ("grad_inf", ct.c_double),
                ("ls_halvings", ct.c_int), ("solver_iters", ct.c_int), ("status", ct.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ct.CDLL(build())
        P, D, I = ct.POINTER(_Problem), ct.POINTER(ct.c_double), ct.c_int
        S = ct.POINTER(_Scene)
        _lib.or_quad_points.argtypes = [P, I, D, I]
        _lib.or_quad_points.restype = I
        _lib.or_point_tables.argtypes = [P, I, D, I]
        _lib.or_point_tables.restype = I
        _lib.or_basis9.argtypes = [P, ct.c_double, ct.c_double, I, I, D]
        _lib.or_lumped_mass.argtypes = [P, D]
        _lib.or_span_eval.argtypes = [P, D, D, D, D]
        _lib.or_span_eval_projected.argtypes = [P, D, ct.c_int, D, D, D]
        _lib.or_fbw_hessian6.argtypes = [P, D, I, D]
        _lib.or_span_terms_subset.argtypes = [P, D, I, ct.POINTER(I), I, D, D, D]
        _lib.or_eval_rows.argtypes = [P, S, D, D, I, ct.POINTER(I), D, D]
        _lib.or_project_psd.argtypes = [I, D, D, D]
        _lib.or_project_psd.restype = I
        _lib.or_eval.argtypes = [P, S, D, D, D, D]
        _lib.or_eval.restype = ct.c_double
        _lib.or_energy.argtypes = [P, S, D, D]
        _lib.or_energy.restype = ct.c_double
        _lib.or_stencil_matvec.argtypes = [I, I, D, D, D]
        _lib.or_solve_banded.argtypes = [I, I, D, D, D]
        _lib.or_solve_banded.restype = I
        _lib.or_solve_pcg.argtypes = [I, I, D, D, D, ct.c_double, I]
        _lib.or_solve_pcg.restype = I
        _lib.or_newton_step.argtypes = [P, S, D, D, I, ct.c_double, I, ct.POINTER(NewtonReport)]
        _lib.or_newton_step.restype = I
        _lib.or_line_search.argtypes = [P, S, D, D, D, ct.c_double, I, D, ct.POINTER(NewtonReport)]
        _lib.or_line_search.restype = I
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ct.POINTER(ct.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Problem:
    """Geometry + material + quadrature rules of one patch."""

    def __init__(self, nu, nv, rest, material, mem_rule=RULE_REDUCED, bend_rule=RULE_REDUCED):
        self.nu, self.nv = int(nu), int(nv)
        self.rest = _f64(rest).reshape(self.nu * self.nv, 2)
        mu1, mu2, mush, mubd, rho = (material.as_tuple() if hasattr(material, "as_tuple")
                                     else tuple(material))
        self._p = _Problem(self.nu, self.nv, _dp(self.rest), mu1, mu2, mush, mubd, rho,
                           int(mem_rule), int(bend_rule))

    @classmethod
    def from_patch(cls, patch, **kw):
        return cls(patch.nu, patch.nv, patch.rest, patch.material, **kw)

    @property
    def n_cp(self):
        return self.nu * self.nv

    @property
    def n_spans(self):
        return (self.nu - 2) * (self.nv - 2)

    def quad_points(self, which: int) -> np.ndarray:
        n = lib().or_quad_points(ct.byref(self._p), which, None, 0)
        out = np.zeros((n, 5))
        lib().or_quad_points(ct.byref(self._p), which, _dp(out), n)
        return out

    def point_tables(self, which: int) -> np.ndarray:
        n = lib().or_quad_points(ct.byref(self._p), which, None, 0)
        w = 20 if which == 0 else 16
        out = np.zeros((n, w))
        lib().or_point_tables(ct.byref(self._p), which, _dp(out), n)
        return out

    def basis9(self, u, v, a, b) -> np.ndarray:
        out = np.zeros((6, 9))
        lib().or_basis9(ct.byref(self._p), float(u), float(v), int(a), int(b), _dp(out))
        return out

    def lumped_mass(self) -> np.ndarray:
        m = np.zeros(self.n_cp)
        lib().or_lumped_mass(ct.byref(self._p), _dp(m))
        return m

    def span_eval(self, C, want_g=True, want_H=True):
        C = _f64(C).reshape(self.n_cp, 3)
        E = np.zeros(self.n_spans)
        g = np.zeros((self.n_spans, 27)) if want_g else None
        H = np.zeros((self.n_spans, 27, 27)) if want_H else None
        lib().or_span_eval(ct.byref(self._p), _dp(C), _dp(E), _dp(g), _dp(H))
        return E, g, H

    def fbw_hessian6(self, f1, f2, point_project=False):
        """6x6 d^2 Psi / d(f_1, f_2)^2 of the FBW density with this problem's
        material; with point_project each term's Hessian is projected first."""
        f6 = np.ascontiguousarray(np.concatenate([_f64(f1).ravel(), _f64(f2).ravel()]))
        A6 = np.zeros((6, 6))
        lib().or_fbw_hessian6(ct.byref(self._p), _dp(f6), int(bool(point_project)), _dp(A6))
        return A6

    def span_eval_projected(self, C, project, want_g=True, want_H=True):
        """span_eval with the Hessians projected per project (see _project_mode)."""
        C = _f64(C).reshape(self.n_cp, 3)
        E = np.zeros(self.n_spans)
        g = np.zeros((self.n_spans, 27)) if want_g else None
        H = np.zeros((self.n_spans, 27, 27)) if want_H else None
        lib().or_span_eval_projected(ct.byref(self._p), _dp(C), _project_mode(project), _dp(E), _dp(g), _dp(H))
        return E, g, H


PROJECT_NONE, PROJECT_SPAN, PROJECT_POINT = 0, 1, 2


def _project_mode(project):
    """True/False or one of PROJECT_*: True means the per-span projection."""
    if project is True or project is False:
        return int(project)
    if project not in (PROJECT_NONE, PROJECT_SPAN, PROJECT_POINT):
        raise ValueError(f"project must be a bool or one of PROJECT_*, got {project!r}")
    return int(project)


def span_terms_subset(prob, C, spans, project=True):
    """E, g, H (projected per project, see _project_mode) of the selected spans only."""
    C = _f64(C).reshape(prob.n_cp, 3)
    sp = np.ascontiguousarray(np.asarray(spans, dtype=np.int32))
    n = sp.size
    E, g, H = np.zeros(n), np.zeros((n, 27)), np.zeros((n, 27, 27))
    lib().or_span_terms_subset(ct.byref(prob._p), _dp(C), n, sp.ctypes.data_as(ct.POINTER(ct.c_int)),
                               _project_mode(project), _dp(E), _dp(g), _dp(H))
    return E, g, H


def eval_rows(prob, scene, C, Chat, rows):
    """Gradient entries (n, 3) and stencil rows (n, 25, 3, 3) of selected control points."""
    C = _f64(C).reshape(prob.n_cp, 3)
    Chat = C if Chat is None else _f64(Chat).reshape(prob.n_cp, 3)
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int32))
    n = r.size
    g, K = np.zeros((n, 3)), np.zeros((n, 25, 3, 3))
    lib().or_eval_rows(ct.byref(prob._p), ct.byref(scene._s), _dp(C), _dp(Chat), n,
                       r.ctypes.data_as(ct.POINTER(ct.c_int)), _dp(g), _dp(K))
    return g, K


class Scene:
    def __init__(self, dt, gravity, pinned=(), project=True):
        self.pinned = np.ascontiguousarray(np.asarray(pinned, dtype=np.int32).ravel())
        self._s = _Scene(float(dt), (ct.c_double * 3)(*gravity),
                         self.pinned.ctypes.data_as(ct.POINTER(ct.c_int)), int(self.pinned.size),
                         _project_mode(project))

    @classmethod
    def from_patch(cls, patch, project=True, static=False):
        return cls(0.0 if static else patch.dt, patch.gravity, patch.pinned, project)


def project_psd(H):
    H = _f64(H)
    n = H.shape[0]
    P = np.zeros_like(H)
    lam = np.zeros(n)
    sweeps = lib().or_project_psd(n, _dp(H), _dp(P), _dp(lam))
    return P, lam, sweeps


def evaluate(prob: Problem, scene: Scene, C, Chat=None, want_g=True, want_K=True):
    C = _f64(C).reshape(prob.n_cp, 3)
    Chat = C if Chat is None else _f64(Chat).reshape(prob.n_cp, 3)
    g = np.zeros((prob.n_cp, 3)) if want_g else None
    K = np.zeros((prob.n_cp, 25, 3, 3)) if want_K else None
    E = lib().or_eval(ct.byref(prob._p), ct.byref(scene._s), _dp(C), _dp(Chat), _dp(g), _dp(K))
    return E, g, K


def energy(prob: Problem, scene: Scene, C, Chat=None) -> float:
    C = _f64(C).reshape(prob.n_cp, 3)
    Chat = C if Chat is None else _f64(Chat).reshape(prob.n_cp, 3)
    return lib().or_energy(ct.byref(prob._p), ct.byref(scene._s), _dp(C), _dp(Chat))


def stencil_matvec(nu, nv, K, x):
    K = _f64(K)
    x = _f64(x).reshape(nu * nv, 3)
    y = np.zeros_like(x)
    lib().or_stencil_matvec(nu, nv, _dp(K), _dp(x), _dp(y))
    return y


def solve_banded(nu, nv, K, b):
    K = _f64(K)
    b = _f64(b).reshape(-1)
    x = np.zeros_like(b)
    st = lib().or_solve_banded(nu, nv, _dp(K), _dp(b), _dp(x))
    if st != 0:
        raise RuntimeError(f"banded Cholesky failed ({st})")
    return x.reshape(nu * nv, 3)


def solve_pcg(nu, nv, K, b, rel_tol=1e-12, max_iter=100000):
    K = _f64(K)
    b = _f64(b).reshape(-1)
    x = np.zeros_like(b)
    it = lib().or_solve_pcg(nu, nv, _dp(K), _dp(b), _dp(x), float(rel_tol), int(max_iter))
    return x.reshape(nu * nv, 3), it


def newton_step(prob: Problem, scene: Scene, C, Chat=None, solver=0, pcg_tol=1e-12, max_halvings=30):
    """One projected Newton iteration; returns (C_new, report)."""
    C = _f64(C).reshape(prob.n_cp, 3).copy()
    Chat = C.copy() if Chat is None else _f64(Chat).reshape(prob.n_cp, 3)
    rep = NewtonReport()
    lib().or_newton_step(ct.byref(prob._p), ct.byref(scene._s), _dp(C), _dp(Chat), int(solver),
                         float(pcg_tol), int(max_halvings), ct.byref(rep))
    return C, rep


def line_search(prob: Problem, scene: Scene, C, Chat, d, max_halvings=30):
    """The oracle's backtracking along direction d from C; returns (C_new, status, report)."""
    C = _f64(C).reshape(prob.n_cp, 3).copy()
    Chat = C.copy() if Chat is None else _f64(Chat).reshape(prob.n_cp, 3)
    d = _f64(d).reshape(prob.n_cp, 3)
    E0 = energy(prob, scene, C, Chat)
    work = np.zeros_like(C)
    rep = NewtonReport()
    st = lib().or_line_search(ct.byref(prob._p), ct.byref(scene._s), _dp(C), _dp(Chat), _dp(d), float(E0),
                              int(max_halvings), _dp(work), ct.byref(rep))
    rep.E0 = E0
    return C, st, rep


def stencil_to_dense(nu, nv, K) -> np.ndarray:
    """Expand the stencil Hessian into a dense (3N, 3N) matrix (small grids)."""
    N = nu * nv
    D = np.zeros((3 * N, 3 * N))
    K = np.asarray(K).reshape(N, 25, 3, 3)
    for al in range(N):
        i, j = al % nu, al // nu
        for dv in range(-2, 3):
            for du in range(-2, 3):
                ii, jj = i + du, j + dv
                if 0 <= ii < nu and 0 <= jj < nv:
                    be = jj * nu + ii
                    D[3 * al:3 * al + 3, 3 * be:3 * be + 3] = K[al, (dv + 2) * 5 + du + 2]
    return D
