"""Contact with a static obstacle on the GPU (Sec. 4.3, IPC log barrier,
Eq. gradient and hessian of contact barrier) against the contact oracle
(oracle/contact_oracle.py) and the elastic oracle, through the C ABI.

A 11 x 11 patch just above the apex of a pyramid (inputs.config_contact),
contact mesh 31 x 31 (a vertex right above the apex), dhat = 2 cm: pairs of
every feature type (face, edge, corner) are active.

- FP64: contact-mesh vertex positions, the total energy, the gradient and the
  stencil Hessian (elastic + contact, Dirichlet-eliminated) within 1e-12;
  the line search's step bound of a falling and a rising direction; one
  Newton step (positions within 1e-10 of the width, the same step length
  and start of the line search).
- FP32: the same quantities, errors stated, bounds of the FP32 parity tests.
- A cloth dropped onto a sphere for 15 time steps keeps every contact vertex
  outside the (convex) obstacle and every Newton step decreases the total
  energy.
"""
import numpy as np
import pytest

from oracle import contact_oracle as co
from paper_2506_18867_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2506_18867_gb300 import build as _build  # noqa: E402

_build.build()
from paper_2506_18867_gb300 import bsc  # noqa: E402

MU = MV = 31


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_n3(t):
    return t.detach().double().cpu().numpy().reshape(3, -1).T.copy()


def gpu_K(K, N):
    return K.detach().double().cpu().numpy().reshape(25, 3, 3, N).transpose(3, 0, 1, 2).copy()


@pytest.fixture(scope="module")
def scene(orc):
    pat = inputs.config_contact()
    V, T = inputs.pyramid_obstacle()
    prob = orc.Problem.from_patch(pat)
    sc = orc.Scene.from_patch(pat, project=True)
    cm = co.ContactMesh(prob, MU, MV)
    obs = co.Obstacle(V, T)
    return pat, V, T, prob, sc, cm, obs


def oracle_terms(orc, pat, prob, sc, cm, obs, C):
    E_el, g_el, K_el = orc.evaluate(prob, sc, C, pat.Chat)
    E_c, G_c, K_c = co.contact_terms(cm, obs, C, pat.meta["dhat"], pat.meta["kappa"])
    K_c, G_c = co.eliminate(K_c, G_c, pat.pinned, pat.nu, pat.nv)
    return E_el + E_c, g_el + G_c, K_el + K_c


@pytest.mark.parametrize("precision", [bsc.FP64, bsc.FP32], ids=["fp64", "fp32"])
def test_contact_terms_match_oracle(orc, scene, precision):
    pat, V, T, prob, sc, cm, obs = scene
    E, g, K = oracle_terms(orc, pat, prob, sc, cm, obs, pat.C)
    with bsc.context_for_patch(pat, precision=precision, pcg_rel_tol=1e-13) as ctx:
        ctx.contact_attach(V, T, pat.meta["dhat"], pat.meta["kappa"], MU, MV)
        C, Ch = ctx.to_device(pat.C), ctx.to_device(pat.Chat)
        X = ctx.contact_vertices(C)
        Eg = ctx.energy(C, Ch)
        gg = to_n3(ctx.gradient(C, Ch))
        Kg = gpu_K(ctx.assemble_hessian(C, project=True), pat.n_cp)
        pairs = ctx.contact_stats()["pairs"]
    eX = np.abs(X - cm.positions(pat.C)).max()
    eE, eg, eK = abs(Eg - E) / abs(E), rel(gg, g), rel(Kg, K)
    print(f"precision {precision}: {pairs} pairs; vertices {eX:.1e} m, energy {eE:.1e}, gradient {eg:.1e}, "
          f"Hessian {eK:.1e}")
    assert pairs > 50
    if precision == bsc.FP64:
        assert eX < 1e-15 and eE < 1e-12 and eg < 1e-12 and eK < 1e-12
    else:
        assert eX < 1e-7 and eE < 1e-6 and eg < 1e-4 and eK < 2e-5


def test_contact_step_bound_matches_oracle(scene):
    pat, V, T, prob, sc, cm, obs = scene
    with bsc.context_for_patch(pat, precision=bsc.FP64) as ctx:
        ctx.contact_attach(V, T, pat.meta["dhat"], pat.meta["kappa"], MU, MV)
        C = ctx.to_device(pat.C)
        D = np.zeros_like(pat.C)
        D[:, 2] = -0.01
        D[:, 0] = 0.002
        a_down = ctx.contact_step_bound(C, ctx.to_device(D))
        a_up = ctx.contact_step_bound(C, ctx.to_device(-D))
    o_down = co.step_bound(cm, obs, pat.C, D)
    print(f"step bound falling {a_down:.6f} (oracle {o_down:.6f}), rising {a_up}")
    assert o_down < 1.0 and abs(a_down - o_down) <= 1e-14 * o_down
    assert a_up == 1.0 and co.step_bound(cm, obs, pat.C, -D) == 1.0


@pytest.mark.parametrize("push", [0.0, 0.03], ids=["at_rest", "pushed_down"])
def test_contact_newton_step_fp64(orc, scene, push):
    """push: the inertial target C^ lies that far below C, so the Newton step
    heads into the obstacle and the step bound starts the line search below 1."""
    pat, V, T, prob, sc, cm, obs = scene
    Chat = pat.Chat.copy()
    Chat[:, 2] -= push
    oC, st, info = co.newton_step(orc, prob, sc, cm, obs, pat.C, Chat, pat.meta["dhat"], pat.meta["kappa"])
    assert st == 0
    if push:
        assert info["alpha0"] < 1.0
    with bsc.context_for_patch(pat, precision=bsc.FP64, pcg_rel_tol=1e-14) as ctx:
        ctx.contact_attach(V, T, pat.meta["dhat"], pat.meta["kappa"], MU, MV)
        C, Ch = ctx.to_device(pat.C), ctx.to_device(Chat)
        rep = ctx.newton_step(C, Ch)
        Cg = to_n3(C)
    width = np.ptp(pat.rest, axis=0).max()
    print(f"Newton step with contact: alpha {rep.alpha} (oracle {info['alpha']}, bound {info['alpha0']:.4f}), "
          f"halvings {rep.ls_halvings}, max |dC| {np.abs(Cg - oC).max():.2e}")
    # the step bound is a quotient of distances summed in different orders
    assert rep.status == 0 and rep.ls_halvings == info["halvings"]
    assert abs(rep.alpha - info["alpha"]) <= 1e-12 * info["alpha"]
    assert abs(rep.E0 - info["E0"]) <= 1e-12 * abs(info["E0"])
    assert np.abs(Cg - oC).max() <= 1e-10 * width


def test_drop_onto_sphere_stays_penetration_free(orc):
    """15 implicit-Euler steps of a 17 x 17 patch falling onto a sphere: every
    Newton step decreases the energy and every contact vertex stays outside
    the obstacle (a positive signed distance to the convex mesh)."""
    n = 17
    rest = inputs.flat_rest(n, n, 0.6, 0.6)
    C0 = inputs.lift(rest)
    C0[:, 0] -= 0.3
    C0[:, 1] -= 0.3
    C0[:, 2] = 0.215
    mat = inputs.Material.from_engineering(1e5, 0.3, 1e-3, 0.2)
    pat = inputs.Patch("drop17", n, n, rest, C0, C0.copy(), mat, 0.01, (0.0, 0.0, -9.81),
                       np.zeros(0, dtype=np.int32), {})
    V, T = inputs.sphere_obstacle((0.0, 0.0, 0.0), 0.2, 16, 32)
    obs = co.Obstacle(V, T)
    with bsc.context_for_patch(pat, precision=bsc.FP64, pcg_rel_tol=1e-10) as ctx:
        ctx.contact_attach(V, T, 0.01, 1e3, 0, 0)
        C = ctx.to_device(pat.C)
        v = torch.zeros_like(C)
        Chat = C.clone()
        min_d, newton, touched = 1.0, 0, 0
        for step in range(15):
            C_prev = C.clone()
            Chat.copy_(C + pat.dt * v)
            for _ in range(20):
                st, rep = ctx.newton_step_status(C, Chat)
                newton += 1
                assert st == bsc.OK, (step, bsc.STATUS_NAMES[st])
                assert rep.E1 <= rep.E0
                if rep.dir_inf / pat.dt < 1e-3:
                    break
            v = (C - C_prev) / pat.dt
            # signed distance to the convex obstacle: the largest over its
            # faces of the height above the face plane (positive outside)
            X = ctx.contact_vertices(C)
            A, B, Cc = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
            nrm = np.cross(B - A, Cc - A)
            nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
            out = np.sign(np.einsum("ij,ij->i", nrm, A))[:, None] * nrm     # outward normals
            sd = np.max(np.einsum("kj,tj->kt", X, out) - np.einsum("tj,tj->t", out, A)[None, :], axis=1)
            min_d = min(min_d, float(sd.min()))
            touched = max(touched, ctx.contact_stats()["pairs"])
    print(f"drop: {newton} Newton steps, smallest signed distance {min_d:.3e} m, most pairs {touched}")
    assert touched > 0 and min_d > 0.0
