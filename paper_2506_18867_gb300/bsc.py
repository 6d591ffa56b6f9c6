"""Thin ctypes binding of the C ABI in include/bsc.h (argument marshalling only).

Every step of the hot path runs in the CUDA kernels of ``libbsc.so``; this
module only converts torch tensors to device pointers and structs.  Loading
fails loudly when the library is missing: there is no CPU fallback.

Layouts (see include/bsc.h): per-control-point vectors are ``(3, N)`` tensors
(x, y, z planes), the stencil Hessian is ``(225, N)`` with plane index
``slot * 9 + 3 * r + c`` and ``slot = (dv + 2) * 5 + (du + 2)``.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbsc.so")

OK, ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_NUMERIC, ERR_NOT_CONVERGED, ERR_LINESEARCH, ERR_TIMEOUT = range(8)
FP64, FP32 = 0, 1
QUAD_REDUCED, QUAD_GAUSS2, QUAD_GAUSS3, QUAD_STANDARD = 0, 2, 3, 4
PROJECT_NONE, PROJECT_SPAN, PROJECT_POINT = 0, 1, 2


def _project(project):
    """True / False (per-span projection or none) or one of PROJECT_*."""
    if project is True or project is False:
        return int(project)
    if project not in (PROJECT_NONE, PROJECT_SPAN, PROJECT_POINT):
        raise ValueError(f"project must be a bool or one of PROJECT_*, got {project!r}")
    return int(project)

STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "OOM", 4: "NUMERIC", 5: "NOT_CONVERGED",
                6: "LINESEARCH", 7: "TIMEOUT"}

# Every entry point declared in include/bsc.h.
EXPORTS = ("bsc_create", "bsc_destroy", "bsc_last_error", "bsc_set_stream", "bsc_energy", "bsc_gradient",
           "bsc_assemble_hessian", "bsc_spmv", "bsc_solve", "bsc_newton_step", "bsc_create_batch",
           "bsc_batch_layout", "bsc_patch_reports", "bsc_patch_energies", "bsc_autotune", "bsc_set_tiles",
           "bsc_set_border_path", "bsc_set_p2_variant", "bsc_set_pcg_grid", "bsc_set_material",
           "bsc_pcg_split", "bsc_plan_blocks", "bsc_set_graph", "bsc_graph_state", "bsc_span_terms",
           "bsc_quadrature_tables", "bsc_lumped_mass", "bsc_sizes", "bsc_set_profiling", "bsc_phase_times",
           "bsc_launch_count", "bsc_projection_stats", "bsc_solve_static", "bsc_cnn_param_count",
           "bsc_cnn_create", "bsc_cnn_destroy", "bsc_cnn_set_params", "bsc_cnn_get_params", "bsc_cnn_prepare",
           "bsc_cnn_apply", "bsc_cnn_loss_grad", "bsc_cnn_adam_step", "bsc_cnn_activations", "bsc_solve_fcg",
           "bsc_set_learned_solver", "bsc_cnn_set_stall_window", "bsc_set_wait_limit", "bsc_set_pcg_form",
           "bsc_set_psd_test", "bsc_set_proj_arith", "bsc_contact_attach", "bsc_contact_detach", "bsc_contact_vertices",
           "bsc_contact_step_bound", "bsc_contact_stats", "bsc_create_window", "bsc_window_energy_rows",
           "bsc_window_pcg_begin", "bsc_window_pcg_product", "bsc_window_pcg_update", "bsc_window_pcg_direction",
           "bsc_axpy", "bsc_set_k_storage", "bsc_psd_counts")

TILE_CANDIDATES = (0, 8, 16, 32)

STATIC_SOLVE_MAX_CP = 16384  # BSC_STATIC_SOLVE_MAX_CP in include/bsc.h


class Window(ct.Structure):
    _fields_ = [("row0", ct.c_int), ("row1", ct.c_int), ("own0", ct.c_int), ("own1", ct.c_int)]


class KnotGrid(ct.Structure):
    _fields_ = [("nu", ct.c_int), ("nv", ct.c_int), ("knots_u", ct.POINTER(ct.c_double)),
                ("knots_v", ct.POINTER(ct.c_double))]


class Material(ct.Structure):
    _fields_ = [("mu_st1", ct.c_double), ("mu_st2", ct.c_double), ("mu_sh", ct.c_double),
                ("mu_bd", ct.c_double), ("rho_area", ct.c_double)]


class Quadrature(ct.Structure):
    _fields_ = [("membrane", ct.c_int), ("bending", ct.c_int)]


class Options(ct.Structure):
    _fields_ = [("precision", ct.c_int), ("dt", ct.c_double), ("gravity", ct.c_double * 3),
                ("pinned", ct.POINTER(ct.c_int32)), ("n_pinned", ct.c_int), ("project", ct.c_int),
                ("pcg_rel_tol", ct.c_double), ("pcg_max_iter", ct.c_int), ("max_line_search", ct.c_int)]


class NewtonReport(ct.Structure):
    _fields_ = [("E0", ct.c_double), ("E1", ct.c_double), ("alpha", ct.c_double), ("dir_inf", ct.c_double),
                ("pcg_rel_res", ct.c_double), ("pcg_iters", ct.c_int), ("ls_halvings", ct.c_int),
                ("status", ct.c_int), ("spans_projected", ct.c_int), ("fcg_iters", ct.c_int),
                ("fell_back", ct.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(ct.Structure):
    _fields_ = [("tile_tu", ct.c_int * 4), ("tile_ms", (ct.c_double * 4) * 4), ("pcg_grid", ct.c_int),
                ("border_path", ct.c_int), ("border_ms", ct.c_double * 4), ("p2_variant", ct.c_int),
                ("p2_ms", ct.c_double * 2), ("pcg_grid_cand", ct.c_int * 4), ("pcg_ms", ct.c_double * 4),
                ("pcg_form", ct.c_int), ("pcg_form_ms", ct.c_double * 3), ("psd_test", ct.c_int),
                ("psd_ms", ct.c_double * 3)]

    def as_dict(self):
        return {"tile_tu": list(self.tile_tu), "tile_ms": [list(r) for r in self.tile_ms],
                "pcg_grid": self.pcg_grid, "border_path": self.border_path, "border_ms": list(self.border_ms),
                "p2_variant": self.p2_variant, "p2_ms": list(self.p2_ms),
                "pcg_grid_cand": list(self.pcg_grid_cand), "pcg_ms": list(self.pcg_ms),
                "pcg_form": self.pcg_form, "pcg_form_ms": list(self.pcg_form_ms),
                "psd_test": self.psd_test, "psd_ms": list(self.psd_ms)}


class FcgReport(ct.Structure):
    _fields_ = [("fcg_iters", ct.c_int), ("pcg_iters", ct.c_int), ("fell_back", ct.c_int), ("rel_res", ct.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BscError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libbsc.so (built by ``paper_2506_18867_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2506_18867_gb300.build` "
                          "(there is no CPU fallback for the CUDA path)")
    lib = ct.CDLL(path)
    P, I, D, V = ct.c_void_p, ct.c_int, ct.c_double, ct.c_void_p
    lib.bsc_create.argtypes = [ct.POINTER(KnotGrid), ct.POINTER(ct.c_double), ct.POINTER(Material),
                               ct.POINTER(Quadrature), ct.POINTER(Options), V, ct.POINTER(P)]
    lib.bsc_destroy.argtypes = [P]
    lib.bsc_destroy.restype = None
    lib.bsc_last_error.argtypes = [P]
    lib.bsc_last_error.restype = ct.c_char_p
    lib.bsc_set_stream.argtypes = [P, V]
    lib.bsc_energy.argtypes = [P, V, V, ct.POINTER(D)]
    lib.bsc_gradient.argtypes = [P, V, V, V]
    lib.bsc_assemble_hessian.argtypes = [P, V, I, V]
    lib.bsc_spmv.argtypes = [P, V, V, V]
    lib.bsc_solve.argtypes = [P, V, V, V, D, I, ct.POINTER(I), ct.POINTER(D)]
    lib.bsc_newton_step.argtypes = [P, V, V, ct.POINTER(NewtonReport)]
    lib.bsc_span_terms.argtypes = [P, V, I, V, V, V]
    lib.bsc_quadrature_tables.argtypes = [P, I, ct.POINTER(D), I, ct.POINTER(I)]
    lib.bsc_lumped_mass.argtypes = [P, ct.POINTER(D)]
    lib.bsc_sizes.argtypes = [P, ct.POINTER(I), ct.POINTER(I), ct.POINTER(I), ct.POINTER(I)]
    lib.bsc_set_profiling.argtypes = [P, I]
    lib.bsc_phase_times.argtypes = [P, ct.POINTER(D)]
    lib.bsc_launch_count.argtypes = [P, ct.POINTER(ct.c_ulonglong)]
    lib.bsc_projection_stats.argtypes = [P, ct.POINTER(I), ct.POINTER(I)]
    lib.bsc_solve_static.argtypes = [I, I, I, V, V, V, D, I, V, ct.POINTER(I), ct.POINTER(D)]
    lib.bsc_create_batch.argtypes = [I, ct.POINTER(KnotGrid), ct.POINTER(ct.POINTER(ct.c_double)),
                                     ct.POINTER(Material), ct.POINTER(Quadrature), ct.POINTER(Options), V,
                                     ct.POINTER(P)]
    lib.bsc_batch_layout.argtypes = [P, ct.POINTER(I), ct.POINTER(I), ct.POINTER(I)]
    lib.bsc_patch_reports.argtypes = [P, ct.POINTER(NewtonReport)]
    lib.bsc_patch_energies.argtypes = [P, V, V, ct.POINTER(D)]
    lib.bsc_autotune.argtypes = [P, V, V, ct.POINTER(Tuning)]
    lib.bsc_set_tiles.argtypes = [P, ct.POINTER(I)]
    lib.bsc_pcg_split.argtypes = [P, ct.POINTER(I)]
    lib.bsc_set_border_path.argtypes = [P, I]
    lib.bsc_set_p2_variant.argtypes = [P, I]
    lib.bsc_set_pcg_grid.argtypes = [P, I]
    lib.bsc_set_material.argtypes = [P, I, ct.POINTER(Material)]
    lib.bsc_plan_blocks.argtypes = [I, ct.POINTER(I), ct.POINTER(D), I, ct.POINTER(I)]
    lib.bsc_set_graph.argtypes = [P, I]
    F = ct.POINTER(ct.c_float)
    lib.bsc_cnn_param_count.argtypes = []
    lib.bsc_cnn_create.argtypes = [P, ct.POINTER(P)]
    lib.bsc_cnn_destroy.argtypes = [P]
    lib.bsc_cnn_destroy.restype = None
    lib.bsc_cnn_set_params.argtypes = [P, F, I]
    lib.bsc_cnn_get_params.argtypes = [P, F, I, I]
    lib.bsc_cnn_prepare.argtypes = [P, V]
    lib.bsc_cnn_apply.argtypes = [P, V, V]
    lib.bsc_cnn_loss_grad.argtypes = [P, V, V, ct.POINTER(D)]
    lib.bsc_cnn_adam_step.argtypes = [P, D, D, D, D]
    lib.bsc_cnn_activations.argtypes = [P, I, F]
    lib.bsc_solve_fcg.argtypes = [P, P, V, V, V, D, I, ct.POINTER(FcgReport)]
    lib.bsc_graph_state.argtypes = [P, ct.POINTER(I), ct.POINTER(I), ct.POINTER(ct.c_longlong)]
    lib.bsc_set_learned_solver.argtypes = [P, P]
    lib.bsc_cnn_set_stall_window.argtypes = [P, I]
    lib.bsc_set_wait_limit.argtypes = [P, ct.c_longlong, I]
    lib.bsc_set_pcg_form.argtypes = [P, I]
    lib.bsc_set_psd_test.argtypes = [P, I]
    lib.bsc_set_proj_arith.argtypes = [P, I]
    lib.bsc_contact_attach.argtypes = [P, ct.POINTER(D), I, ct.POINTER(ct.c_int32), I, I, I, D, D]
    lib.bsc_contact_detach.argtypes = [P]
    lib.bsc_contact_vertices.argtypes = [P, V, ct.POINTER(D), I, ct.POINTER(I)]
    lib.bsc_contact_step_bound.argtypes = [P, V, V, ct.POINTER(D)]
    lib.bsc_contact_stats.argtypes = [P, ct.POINTER(I), ct.POINTER(I)]
    lib.bsc_create_window.argtypes = [ct.POINTER(KnotGrid), ct.POINTER(D), ct.POINTER(Material),
                                      ct.POINTER(Quadrature), ct.POINTER(Options), ct.POINTER(Window), V,
                                      ct.POINTER(P)]
    lib.bsc_window_energy_rows.argtypes = [P, V, V, ct.POINTER(D), I, ct.POINTER(I)]
    lib.bsc_window_pcg_begin.argtypes = [P, V, V, V, V, ct.POINTER(D)]
    lib.bsc_window_pcg_product.argtypes = [P, V, ct.POINTER(D)]
    lib.bsc_window_pcg_update.argtypes = [P, D, ct.POINTER(D)]
    lib.bsc_window_pcg_direction.argtypes = [P, D]
    lib.bsc_axpy.argtypes = [P, V, V, D, V]
    lib.bsc_set_k_storage.argtypes = [P, I]
    lib.bsc_psd_counts.argtypes = [P, ct.POINTER(I)]
    for name in EXPORTS:
        if name not in ("bsc_destroy", "bsc_last_error", "bsc_cnn_destroy"):
            getattr(lib, name).restype = I
    _lib = lib
    return lib


def _ptr(t):
    return None if t is None else ct.c_void_p(t.data_ptr())


class Context:
    """Patches on the GPU (wraps ``bsc_ctx``): one patch from the constructor,
    several independent patches from :meth:`batch`.  Tensors must be CUDA
    tensors of the context's dtype, contiguous, in the layouts of
    include/bsc.h (a batch concatenates its patches' control points)."""

    def __init__(self, nu, nv, rest, material, precision=FP64, dt=0.01, gravity=(0.0, -9.81, 0.0),
                 pinned=(), project=True, quadrature=(QUAD_REDUCED, QUAD_REDUCED), pcg_rel_tol=1e-8,
                 pcg_max_iter=10000, max_line_search=30, stream=None, window=None):
        """window: (row0, row1, own0, own1) for a strip window of the patch
        (bsc_create_window); nu, nv, rest and pinned then describe the whole
        patch."""
        self._create([dict(nu=nu, nv=nv, rest=rest, material=material, dt=dt, gravity=gravity, pinned=pinned)],
                     precision, project, quadrature, pcg_rel_tol, pcg_max_iter, max_line_search, stream, window)

    @classmethod
    def batch(cls, specs, precision=FP64, project=True, quadrature=(QUAD_REDUCED, QUAD_REDUCED), pcg_rel_tol=1e-8,
              pcg_max_iter=10000, max_line_search=30, stream=None):
        """Context of several patches; specs: dicts with nu, nv, rest, material,
        dt, gravity, pinned (patch-local indices)."""
        self = cls.__new__(cls)
        self._create(list(specs), precision, project, quadrature, pcg_rel_tol, pcg_max_iter, max_line_search,
                     stream)
        return self

    def _create(self, specs, precision, project, quadrature, pcg_rel_tol, pcg_max_iter, max_line_search, stream,
                window=None):
        import torch
        self.torch = torch
        lib = load()
        P = len(specs)
        self.P = P
        self.precision = precision
        self.dtype = torch.float64 if precision == FP64 else torch.float32
        self._grids = (KnotGrid * P)()
        self._mats = (Material * P)()
        self._opts = (Options * P)()
        self._rests, self._pins = [], []
        rest_ptrs = (ct.POINTER(ct.c_double) * P)()
        for p, sp in enumerate(specs):
            nu, nv = int(sp["nu"]), int(sp["nv"])
            self._grids[p] = KnotGrid(nu, nv, None, None)
            r = np.ascontiguousarray(np.asarray(sp["rest"], dtype=np.float64).reshape(nu * nv, 2))
            self._rests.append(r)
            rest_ptrs[p] = r.ctypes.data_as(ct.POINTER(ct.c_double))
            m = sp["material"]
            self._mats[p] = Material(*(m.as_tuple() if hasattr(m, "as_tuple") else tuple(m)))
            pins = np.ascontiguousarray(np.asarray(sp.get("pinned", ()), dtype=np.int32).ravel())
            self._pins.append(pins)
            self._opts[p] = Options(precision, float(sp.get("dt", 0.01)),
                                    (ct.c_double * 3)(*sp.get("gravity", (0.0, -9.81, 0.0))),
                                    pins.ctypes.data_as(ct.POINTER(ct.c_int32)), int(pins.size),
                                    _project(project), float(pcg_rel_tol), int(pcg_max_iter), int(max_line_search))
        self._quad = Quadrature(*quadrature)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        h = ct.c_void_p()
        self.window = None
        if window is not None:
            self._win = Window(*(int(v) for v in window))
            self.window = tuple(int(v) for v in window)
            st = lib.bsc_create_window(ct.byref(self._grids[0]), rest_ptrs[0], ct.byref(self._mats[0]),
                                       ct.byref(self._quad), ct.byref(self._opts[0]), ct.byref(self._win),
                                       ct.c_void_p(stream), ct.byref(h))
        elif P == 1:
            st = lib.bsc_create(ct.byref(self._grids[0]), rest_ptrs[0], ct.byref(self._mats[0]),
                                ct.byref(self._quad), ct.byref(self._opts[0]), ct.c_void_p(stream), ct.byref(h))
        else:
            st = lib.bsc_create_batch(P, self._grids, rest_ptrs, self._mats, ct.byref(self._quad), self._opts,
                                      ct.c_void_p(stream), ct.byref(h))
        if st != OK:
            raise BscError(st, lib.bsc_last_error(None).decode())
        self._h = h
        self._lib = lib
        cnt = ct.c_int()
        cpo = (ct.c_int * (P + 1))()
        spo = (ct.c_int * (P + 1))()
        self._check(lib.bsc_batch_layout(h, ct.byref(cnt), cpo, spo))
        self.cp_offset = np.array(list(cpo), dtype=np.int64)
        self.span_offset = np.array(list(spo), dtype=np.int64)
        self.N = int(self.cp_offset[-1])
        self.n_spans = int(self.span_offset[-1])
        self.nu, self.nv = int(self._grids[0].nu), int(self._grids[0].nv)
        if window is not None:
            self.nv = self.N // self.nu   # the window's rows

    # -- helpers -----------------------------------------------------------
    def _check(self, st):
        if st != OK:
            raise BscError(st, self._lib.bsc_last_error(self._h).decode())

    def _vec(self, t, name):
        if t is None:
            return None
        if not (t.is_cuda and t.dtype == self.dtype and t.is_contiguous() and t.numel() == 3 * self.N):
            raise ValueError(f"{name}: expected a contiguous CUDA {self.dtype} tensor with 3*N elements")
        return t

    def _mat(self, K):
        if not (K.is_cuda and K.dtype == self.dtype and K.is_contiguous() and K.numel() == 225 * self.N):
            raise ValueError(f"K: expected a contiguous CUDA {self.dtype} tensor with 225*N elements")
        return K

    def new_vec(self):
        return self.torch.zeros((3, self.N), dtype=self.dtype, device="cuda")

    def new_matrix(self):
        return self.torch.zeros((225, self.N), dtype=self.dtype, device="cuda")

    def to_device(self, arr_n3):
        """(N, 3) host array -> (3, N) device tensor of the context dtype."""
        a = np.ascontiguousarray(np.asarray(arr_n3, dtype=np.float64).reshape(self.N, 3).T)
        return self.torch.from_numpy(a).to(device="cuda", dtype=self.dtype).contiguous()

    # -- C ABI ---------------------------------------------------------------
    def energy(self, C, Chat=None) -> float:
        E = ct.c_double()
        self._check(self._lib.bsc_energy(self._h, _ptr(self._vec(C, "C")), _ptr(self._vec(Chat, "Chat")),
                                         ct.byref(E)))
        return E.value

    def gradient(self, C, Chat=None, out=None):
        out = self.new_vec() if out is None else out
        self._check(self._lib.bsc_gradient(self._h, _ptr(self._vec(C, "C")), _ptr(self._vec(Chat, "Chat")),
                                           _ptr(self._vec(out, "g"))))
        return out

    def assemble_hessian(self, C, project=True, out=None, internal=False):
        if internal:
            self._check(self._lib.bsc_assemble_hessian(self._h, _ptr(self._vec(C, "C")), _project(project), None))
            return None
        out = self.new_matrix() if out is None else out
        self._check(self._lib.bsc_assemble_hessian(self._h, _ptr(self._vec(C, "C")), _project(project),
                                                   _ptr(out)))
        return out

    def spmv(self, x, K=None, out=None):
        out = self.new_vec() if out is None else out
        self._check(self._lib.bsc_spmv(self._h, _ptr(K), _ptr(self._vec(x, "x")), _ptr(self._vec(out, "y"))))
        return out

    def solve(self, b, K=None, rel_tol=1e-8, max_iter=10000, out=None, allow_unconverged=False):
        """PCG solve; with allow_unconverged the iterate after max_iter is returned
        instead of raising NOT_CONVERGED."""
        out = self.new_vec() if out is None else out
        it, rr = ct.c_int(), ct.c_double()
        st = self._lib.bsc_solve(self._h, _ptr(K), _ptr(self._vec(b, "b")), _ptr(self._vec(out, "x")),
                                 float(rel_tol), int(max_iter), ct.byref(it), ct.byref(rr))
        if not (allow_unconverged and st == ERR_NOT_CONVERGED):
            self._check(st)
        return out, it.value, rr.value

    def newton_step(self, C, Chat=None):
        rep = NewtonReport()
        st = self._lib.bsc_newton_step(self._h, _ptr(self._vec(C, "C")), _ptr(self._vec(Chat, "Chat")),
                                       ct.byref(rep))
        self._check(st)
        return rep

    def newton_step_status(self, C, Chat=None):
        """Like newton_step but returns (status, report) instead of raising."""
        rep = NewtonReport()
        st = self._lib.bsc_newton_step(self._h, _ptr(self._vec(C, "C")), _ptr(self._vec(Chat, "Chat")),
                                       ct.byref(rep))
        return st, rep

    def span_terms(self, C, project=True):
        t = self.torch
        E = t.zeros(self.n_spans, dtype=t.float64, device="cuda")
        g = t.zeros((self.n_spans, 27), dtype=self.dtype, device="cuda")
        H = t.zeros((self.n_spans, 27, 27), dtype=self.dtype, device="cuda")
        self._check(self._lib.bsc_span_terms(self._h, _ptr(self._vec(C, "C")), _project(project), _ptr(E),
                                             _ptr(g), _ptr(H)))
        return E, g, H

    def quadrature_tables(self, which):
        n = ct.c_int()
        self._check(self._lib.bsc_quadrature_tables(self._h, int(which), None, 0, ct.byref(n)))
        out = np.zeros((n.value, 25))
        self._check(self._lib.bsc_quadrature_tables(self._h, int(which),
                                                    out.ctypes.data_as(ct.POINTER(ct.c_double)), n.value,
                                                    ct.byref(n)))
        return out

    def lumped_mass(self):
        m = np.zeros(self.N)
        self._check(self._lib.bsc_lumped_mass(self._h, m.ctypes.data_as(ct.POINTER(ct.c_double))))
        return m

    def sizes(self):
        a, b, c, d = ct.c_int(), ct.c_int(), ct.c_int(), ct.c_int()
        self._check(self._lib.bsc_sizes(self._h, ct.byref(a), ct.byref(b), ct.byref(c), ct.byref(d)))
        return a.value, b.value, c.value, d.value

    PHASES = ("span_eval", "project", "assemble", "solve", "line_search", "total")

    def set_profiling(self, on=True):
        self._check(self._lib.bsc_set_profiling(self._h, int(bool(on))))

    def phase_times(self):
        """Durations (ms) of the phases of the last Newton step (needs profiling)."""
        out = (ct.c_double * 6)()
        self._check(self._lib.bsc_phase_times(self._h, out))
        return dict(zip(self.PHASES, list(out)))

    def launch_count(self) -> int:
        n = ct.c_ulonglong()
        self._check(self._lib.bsc_launch_count(self._h, ct.byref(n)))
        return n.value

    def projection_stats(self):
        """Per span: negative eigenvalues projected away, reduced problem size."""
        a = np.zeros(self.n_spans, dtype=np.int32)
        b = np.zeros(self.n_spans, dtype=np.int32)
        self._check(self._lib.bsc_projection_stats(self._h, a.ctypes.data_as(ct.POINTER(ct.c_int)),
                                                   b.ctypes.data_as(ct.POINTER(ct.c_int))))
        return a, b

    # -- batches ------------------------------------------------------------
    def patch_reports(self):
        reps = (NewtonReport * self.P)()
        self._check(self._lib.bsc_patch_reports(self._h, reps))
        return [reps[p] for p in range(self.P)]

    def patch_energies(self, C, Chat=None):
        out = (ct.c_double * self.P)()
        self._check(self._lib.bsc_patch_energies(self._h, _ptr(self._vec(C, "C")), _ptr(self._vec(Chat, "Chat")),
                                                 out))
        return np.array(list(out))

    def autotune(self, C, Chat=None):
        t = Tuning()
        self._check(self._lib.bsc_autotune(self._h, _ptr(self._vec(C, "C")), _ptr(self._vec(Chat, "Chat")),
                                           ct.byref(t)))
        return t.as_dict()

    def set_tiles(self, tiles):
        arr = (ct.c_int * 4)(*[int(t) for t in tiles])
        self._check(self._lib.bsc_set_tiles(self._h, arr))

    def set_material(self, material, patch=0):
        m = Material(*(material.as_tuple() if hasattr(material, "as_tuple") else tuple(material)))
        self._check(self._lib.bsc_set_material(self._h, int(patch), ct.byref(m)))

    def set_border_path(self, path):
        self._check(self._lib.bsc_set_border_path(self._h, int(path)))

    def set_p2_variant(self, variant):
        """Occupancy variant (0 or 1) of the interior projection's eigenpair
        phase; both give bitwise the same result."""
        self._check(self._lib.bsc_set_p2_variant(self._h, int(variant)))

    def set_pcg_grid(self, grid):
        """Blocks of the persistent PCG, in [patches, usable blocks]."""
        self._check(self._lib.bsc_set_pcg_grid(self._h, int(grid)))

    # -- contact with a static obstacle ---------------------------------------
    def contact_attach(self, vertices, triangles, dhat, kappa, mu=0, mv=0):
        """Obstacle triangle mesh (vertices (n, 3), triangles (m, 3)); contact
        mesh of mu x mv vertices (0: about twice the control points)."""
        V = np.ascontiguousarray(np.asarray(vertices, dtype=np.float64).reshape(-1, 3))
        T = np.ascontiguousarray(np.asarray(triangles, dtype=np.int32).reshape(-1, 3))
        self._check(self._lib.bsc_contact_attach(self._h, V.ctypes.data_as(ct.POINTER(ct.c_double)), V.shape[0],
                                                 T.ctypes.data_as(ct.POINTER(ct.c_int32)), T.shape[0], int(mu),
                                                 int(mv), float(dhat), float(kappa)))

    def contact_detach(self):
        self._check(self._lib.bsc_contact_detach(self._h))

    def contact_vertices(self, C):
        n = ct.c_int()
        self._check(self._lib.bsc_contact_vertices(self._h, None, None, 0, ct.byref(n)))
        out = np.zeros((n.value, 3))
        self._check(self._lib.bsc_contact_vertices(self._h, _ptr(self._vec(C, "C")),
                                                   out.ctypes.data_as(ct.POINTER(ct.c_double)), n.value,
                                                   ct.byref(n)))
        return out

    def contact_step_bound(self, C, D):
        a = ct.c_double()
        self._check(self._lib.bsc_contact_step_bound(self._h, _ptr(self._vec(C, "C")), _ptr(self._vec(D, "D")),
                                                     ct.byref(a)))
        return a.value

    def contact_stats(self):
        n, p = ct.c_int(), ct.c_int()
        self._check(self._lib.bsc_contact_stats(self._h, ct.byref(n), ct.byref(p)))
        return {"vertices": n.value, "pairs": p.value}

    def set_psd_test(self, mode=2):
        """PSD test before the interior spans' eigendecomposition: 0 / False
        none, 1 / True the FP64 LDL^T test, 2 the FP32 certificate first."""
        self._check(self._lib.bsc_set_psd_test(self._h, int(mode)))

    def set_proj_arith(self, mode):
        """Arithmetic of the projection's PSD test and phase 1: 0 FP64, 1 double-float
        (pairs of FP32 numbers; the default of FP32 contexts)."""
        self._check(self._lib.bsc_set_proj_arith(self._h, int(mode)))

    def psd_counts(self):
        """(interior spans, interior spans the FP64 test ran on, interior spans eigendecomposed,
        border spans, border spans eigendecomposed, border spans the FP64 test ran on) of the last
        projection."""
        out = (ct.c_int * 6)()
        self._check(self._lib.bsc_psd_counts(self._h, out))
        return tuple(out)

    def set_pcg_form(self, form):
        """PCG form: 0 three group barriers per iteration, 1 the pipelined
        recurrences with one, 2 two passes with two (q = K z + beta q)."""
        self._check(self._lib.bsc_set_pcg_form(self._h, int(form)))

    # -- strip windows (bsc_create_window) ----------------------------------
    def _n_own(self):
        if self.window is None:
            raise ValueError("not a strip window context")
        return self.window[3] - self.window[2]

    def energy_rows(self, C, Chat=None):
        """Per-row partial energies of a strip window: (owned span rows, owned
        control-point rows), host float64 arrays."""
        own = self._n_own()
        n = ct.c_int()
        self._check(self._lib.bsc_window_energy_rows(self._h, None, None, None, 0, ct.byref(n)))
        out = np.zeros(n.value)
        self._check(self._lib.bsc_window_energy_rows(self._h, _ptr(self._vec(C, "C")), _ptr(self._vec(Chat, "Chat")),
                                                     out.ctypes.data_as(ct.POINTER(ct.c_double)), n.value,
                                                     ct.byref(n)))
        return out[:n.value - own], out[n.value - own:]

    def pcg_begin(self, K, g, x, p):
        """Strip PCG of K d = -g: x = 0, p = z = M^-1 r; returns the owned rows'
        partial sums (r.z, r.r) as a (2, rows) array.  x and p stay in use
        until the solve ends."""
        rows = np.zeros((2, self._n_own()))
        self._win_xp = (x, p)
        self._check(self._lib.bsc_window_pcg_begin(self._h, _ptr(self._mat(K)), _ptr(self._vec(g, "g")),
                                                   _ptr(self._vec(x, "x")), _ptr(self._vec(p, "p")),
                                                   rows.ctypes.data_as(ct.POINTER(ct.c_double))))
        return rows

    def pcg_product(self, K):
        """q = K p on the owned rows (p's halo rows current); partial sums p.q."""
        rows = np.zeros(self._n_own())
        self._check(self._lib.bsc_window_pcg_product(self._h, _ptr(self._mat(K)),
                                                     rows.ctypes.data_as(ct.POINTER(ct.c_double))))
        return rows

    def pcg_update(self, alpha):
        """x += alpha p, r -= alpha q, z = M^-1 r; partial sums (r.z, r.r)."""
        rows = np.zeros((2, self._n_own()))
        self._check(self._lib.bsc_window_pcg_update(self._h, float(alpha),
                                                    rows.ctypes.data_as(ct.POINTER(ct.c_double))))
        return rows

    def pcg_direction(self, beta):
        """p = z + beta p on the owned rows."""
        self._check(self._lib.bsc_window_pcg_direction(self._h, float(beta)))

    def axpy(self, a, d, alpha, out=None):
        """out = a + alpha d (a new tensor unless out is given)."""
        if out is None:
            out = self.new_vec()
        self._check(self._lib.bsc_axpy(self._h, _ptr(self._vec(a, "a")), _ptr(self._vec(d, "d")), float(alpha),
                                       _ptr(self._vec(out, "out"))))
        return out

    def set_k_storage(self, symmetric):
        """Layout of the Newton step's matrix: symmetric (13 slots, the default) or full (25)."""
        self._check(self._lib.bsc_set_k_storage(self._h, int(bool(symmetric))))

    def pcg_split(self):
        out = (ct.c_int * self.P)()
        self._check(self._lib.bsc_pcg_split(self._h, out))
        return list(out)

    def set_graph(self, on=True):
        self._check(self._lib.bsc_set_graph(self._h, int(bool(on))))

    def graph_state(self):
        on, cap, rep = ct.c_int(), ct.c_int(), ct.c_longlong()
        self._check(self._lib.bsc_graph_state(self._h, ct.byref(on), ct.byref(cap), ct.byref(rep)))
        return {"on": on.value, "captured": cap.value, "replays": rep.value}

    def set_learned_solver(self, cnn):
        """Newton steps solve with the learned flexible CG of `cnn` (a Cnn of this
        context), PCG as fallback; None returns to plain PCG."""
        self._check(self._lib.bsc_set_learned_solver(self._h, None if cnn is None else cnn._h))

    def set_wait_limit(self, spins, extra_blocks=0):
        """Spin limit of the persistent solvers' bounded barriers; extra_blocks > 0
        makes every barrier wait out its limit (tests of the timeout path)."""
        self._check(self._lib.bsc_set_wait_limit(self._h, int(spins), int(extra_blocks)))

    def patch_slice(self, t, p):
        """Patch p's columns of a (k, N) tensor (a view)."""
        return t[..., int(self.cp_offset[p]):int(self.cp_offset[p + 1])]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.bsc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def solve_static(nu, nv, precision, K, b, x, rel_tol=1e-8, max_iter=10000, stream=None):
    """K x = b without any device allocation (bsc_solve_static): the working set
    lives in a fixed device array sized for STATIC_SOLVE_MAX_CP control points.
    Returns (iterations, relative residual); raises BscError on failure."""
    lib = load()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    it, rr = ct.c_int(), ct.c_double()
    st = lib.bsc_solve_static(int(nu), int(nv), int(precision), _ptr(K), _ptr(b), _ptr(x), float(rel_tol),
                              int(max_iter), ct.c_void_p(stream), ct.byref(it), ct.byref(rr))
    if st != OK:
        raise BscError(st, lib.bsc_last_error(None).decode())
    return it.value, rr.value


class Cnn:
    """The learned preconditioner of a single-patch FP32 context (wraps bsc_cnn)."""

    def __init__(self, ctx: Context):
        self.ctx = ctx
        self._lib = ctx._lib
        h = ct.c_void_p()
        ctx._check(self._lib.bsc_cnn_create(ctx._h, ct.byref(h)))
        self._h = h
        self.n_params = self._lib.bsc_cnn_param_count()

    def set_params(self, params):
        a = np.ascontiguousarray(np.asarray(params, dtype=np.float32).ravel())
        assert a.size == self.n_params
        self.ctx._check(self._lib.bsc_cnn_set_params(self._h, a.ctypes.data_as(ct.POINTER(ct.c_float)), a.size))

    def get_params(self, which=0):
        a = np.zeros(self.n_params, dtype=np.float32)
        self.ctx._check(self._lib.bsc_cnn_get_params(self._h, a.ctypes.data_as(ct.POINTER(ct.c_float)), a.size,
                                                     int(which)))
        return a

    def prepare(self, K):
        self.ctx._check(self._lib.bsc_cnn_prepare(self._h, _ptr(K)))

    def apply(self, r, out=None):
        out = self.ctx.new_vec() if out is None else out
        self.ctx._check(self._lib.bsc_cnn_apply(self._h, _ptr(self.ctx._vec(r, "r")), _ptr(self.ctx._vec(out, "z"))))
        return out

    def loss_grad(self, r, xstar):
        L = ct.c_double()
        self.ctx._check(self._lib.bsc_cnn_loss_grad(self._h, _ptr(self.ctx._vec(r, "r")),
                                                    _ptr(self.ctx._vec(xstar, "x*")), ct.byref(L)))
        return L.value

    def adam_step(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.ctx._check(self._lib.bsc_cnn_adam_step(self._h, float(lr), float(beta1), float(beta2), float(eps)))

    def activations(self, which):
        ch = {0: 32, 1: 32, 2: 32, 3: 32, 4: 16}[which]
        a = np.zeros((self.ctx.N, ch), dtype=np.float32)
        self.ctx._check(self._lib.bsc_cnn_activations(self._h, int(which), a.ctypes.data_as(ct.POINTER(ct.c_float))))
        return a

    def set_stall_window(self, window):
        """Iterations in which r.r must drop by 4x before the flexible CG falls back to PCG."""
        self.ctx._check(self._lib.bsc_cnn_set_stall_window(self._h, int(window)))

    def solve_status(self, b, K, rel_tol=1e-8, max_iter=10000, out=None):
        """Like solve but returns (status, x, report) instead of raising."""
        out = self.ctx.new_vec() if out is None else out
        rep = FcgReport()
        st = self._lib.bsc_solve_fcg(self.ctx._h, self._h, _ptr(K), _ptr(self.ctx._vec(b, "b")),
                                     _ptr(self.ctx._vec(out, "x")), float(rel_tol), int(max_iter), ct.byref(rep))
        return st, out, rep.as_dict()

    def solve(self, b, K, rel_tol=1e-8, max_iter=10000, out=None):
        out = self.ctx.new_vec() if out is None else out
        rep = FcgReport()
        st = self._lib.bsc_solve_fcg(self.ctx._h, self._h, _ptr(K), _ptr(self.ctx._vec(b, "b")),
                                     _ptr(self.ctx._vec(out, "x")), float(rel_tol), int(max_iter), ct.byref(rep))
        self.ctx._check(st)
        return out, rep.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            self._lib.bsc_cnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_blocks(n_cp, work, total):
    """bsc_plan_blocks: split `total` PCG blocks over patches (pure host code)."""
    lib = load()
    n = len(n_cp)
    a = (ct.c_int * n)(*[int(v) for v in n_cp])
    w = (ct.c_double * n)(*[float(v) for v in work])
    out = (ct.c_int * n)()
    used = lib.bsc_plan_blocks(n, a, w, int(total), out)
    return used, list(out)


def batch_for_patches(patches, precision=FP64, **kw):
    """Batched context for a list of ``inputs.Patch``."""
    specs = [dict(nu=p.nu, nv=p.nv, rest=p.rest, material=p.material, dt=p.dt, gravity=p.gravity,
                  pinned=p.pinned) for p in patches]
    return Context.batch(specs, precision=precision, **kw)


def context_for_patch(patch, precision=FP64, **kw):
    """Context for an ``inputs.Patch`` (rest, material, scene); window=(row0,
    row1, own0, own1) gives a strip window of it."""
    kw.setdefault("dt", patch.dt)
    kw.setdefault("gravity", patch.gravity)
    kw.setdefault("pinned", patch.pinned)
    return Context(patch.nu, patch.nv, patch.rest, patch.material, precision=precision, **kw)
