"""bsc_solve_static: the CG solve for callers that cannot allocate device memory.

Some callers own all device memory through their own manager or cannot
afford the device-wide synchronisation of cudaMalloc / cudaFree; the entry
point serves them from a fixed device array.  These tests call it through the
C ABI and compare it with bsc_solve, whose working set the context allocates,
on two calls in a row (the second call finds the first call's leftovers in
the shared array).  The file is named to be collected last.
"""
import ctypes as ct

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


def _system(precision, nu=41, nv=37):
    pat = inputs.config_random_small(23, nu, nv, noise=0.05)
    ctx = bsc.context_for_patch(pat, precision=precision)
    C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
    K = ctx.assemble_hessian(C, project=True)
    b = -ctx.gradient(C, Ch)
    return pat, ctx, K, b


@pytest.mark.parametrize("precision,tol,agree", [(bsc.FP64, 1e-12, 1e-9), (bsc.FP32, 1e-6, 1e-4)])
def test_static_solve_matches_context_solve(precision, tol, agree):
    pat, ctx, K, b = _system(precision)
    with ctx:
        x_ref, it_ref, rr_ref = ctx.solve(b, K=K, rel_tol=tol)
        for call in range(2):
            x = torch.full_like(b, float("nan"))
            it, rr = bsc.solve_static(pat.nu, pat.nv, precision, K, b, x, rel_tol=tol)
            torch.cuda.synchronize()
            assert rr <= tol and it > 0, (call, it, rr)
            d = (x.double() - x_ref.double()).norm() / x_ref.double().norm()
            assert float(d) < agree, (call, float(d))
            # K x = b to the requested tolerance, checked with the context's SpMV
            r = ctx.spmv(x, K=K) - b
            assert float(r.double().norm() / b.double().norm()) < 10 * tol


def test_static_solve_rejects_oversized_grids():
    nu = nv = int(np.sqrt(bsc.STATIC_SOLVE_MAX_CP)) + 2
    lib = bsc.load()
    x = torch.zeros((3, 8), dtype=torch.float64, device="cuda")
    it, rr = ct.c_int(), ct.c_double()
    st = lib.bsc_solve_static(nu, nv, bsc.FP64, bsc._ptr(x), bsc._ptr(x), bsc._ptr(x), 1e-8, 10, None,
                              ct.byref(it), ct.byref(rr))
    assert st == bsc.ERR_INVALID_ARG
    assert b"exceed" in lib.bsc_last_error(None)
