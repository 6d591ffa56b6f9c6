"""Strip decomposition of one patch (paper_2506_18867_gb300/strip.py) on CPU:
the driver's halo plans, and one projected Newton iteration (Sec. 5.1)
computed strip by strip with the oracle as each rank's compute
(tests/oracle_window.py) and
  - host threads as ranks (ThreadComm), 1, 2 and 3 of them, and
  - two gloo processes (DistComm over torch.distributed),
bit-identical to the one-rank decomposition and within the solver tolerance
of the oracle's own Newton step on the whole patch.
"""
import os
import socket

import numpy as np
import pytest
import torch

from paper_2506_18867_gb300 import inputs, partition, strip

HERE = os.path.dirname(os.path.abspath(__file__))


def patch():
    return inputs.config_square(3, 14)


def windows(nv, world):
    strips = partition.strip_rows(nv, world)
    out = []
    for r, (j0, j1) in enumerate(strips):
        w0, w1 = partition.window_rows(strips, r, nv)
        out.append((w0, w1, j0, j1))
    return strips, out


@pytest.mark.parametrize("nv,world", [(9, 2), (14, 3), (7, 7), (30, 4)])
def test_halo_plans(nv, world):
    """Every halo row comes from its owner; what a rank receives from q is
    exactly what q sends it."""
    strips = partition.strip_rows(nv, world)
    for r in range(world):
        w0, w1 = partition.window_rows(strips, r, nv)
        j0, j1 = strips[r]
        got = []
        for o, g0, g1 in strip.halo_plan(strips, r, nv):
            assert o != r and g0 < g1
            assert all(strip.owner_of_row(strips, g) == o for g in range(g0, g1))
            got.extend(range(g0, g1))
        assert sorted(got) == [g for g in range(w0, w1) if not j0 <= g < j1]
        for q in range(world):
            if q == r:
                continue
            sent = [(g0, g1) for d, g0, g1 in strip.send_plan(strips, q, nv) if d == r]
            recv = [(g0, g1) for o, g0, g1 in strip.halo_plan(strips, r, nv) if o == q]
            assert sent == recv


def window_state(pat, w):
    row0, row1 = w[0], w[1]
    sl = slice(row0 * pat.nu, row1 * pat.nu)
    return (torch.from_numpy(np.ascontiguousarray(pat.C[sl].T)),
            torch.from_numpy(np.ascontiguousarray(pat.Chat[sl].T)))


def owned_rows(pat, w, C):
    n0 = (w[2] - w[0]) * pat.nu
    n1 = (w[3] - w[0]) * pat.nu
    return C[:, n0:n1].numpy().T.copy()


def run_world(orc, pat, world, tol):
    from oracle_window import OracleWindow
    strips, wins = windows(pat.nv, world)

    def rank(r, comm):
        ctx = OracleWindow(orc, pat, wins[r])
        C, Ch = window_state(pat, wins[r])
        rep = strip.newton_step(ctx, comm, strips, pat.nv, C, Ch, tol=tol)
        return rep, owned_rows(pat, wins[r], C)

    out = strip.run_threads(world, rank)
    return [o[0] for o in out], np.concatenate([o[1] for o in out])


@pytest.fixture(scope="module")
def one_rank(orc):
    import sys
    if HERE not in sys.path:
        sys.path.insert(0, HERE)
    pat = patch()
    return pat, run_world(orc, pat, 1, 1e-12)


@pytest.mark.parametrize("world", [2, 3])
def test_thread_ranks_bit_identical(orc, one_rank, world):
    pat, (reps1, C1) = one_rank
    reps, C = run_world(orc, pat, world, 1e-12)
    for rep in reps:
        assert rep == reps1[0]
    assert np.array_equal(C, C1)


def test_one_rank_matches_oracle_newton_step(orc, one_rank):
    pat, (reps1, C1) = one_rank
    prob = orc.Problem.from_patch(pat)
    sc = orc.Scene.from_patch(pat, project=True)
    oC, orep = orc.newton_step(prob, sc, pat.C, pat.Chat, solver=0)
    rep = reps1[0]
    width = np.ptp(pat.rest, axis=0).max()
    print(f"strip step: {rep['pcg_iters']} PCG iterations, alpha {rep['alpha']}, "
          f"max |dC| {np.abs(C1 - oC).max():.2e} (width {width})")
    assert rep["status"] == "ok" and rep["alpha"] == orep.alpha
    assert abs(rep["E0"] - orep.E0) <= 1e-12 * abs(orep.E0)
    assert np.abs(C1 - oC).max() <= 1e-9 * width


def _gloo_rank(rank, world, port, out_dir):
    import sys
    root = os.path.dirname(HERE)
    for d in (root, HERE):
        if d not in sys.path:
            sys.path.insert(0, d)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import oracle
    from oracle_window import OracleWindow
    from paper_2506_18867_gb300 import strip as st
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pat = patch()
        strips, wins = windows(pat.nv, world)
        ctx = OracleWindow(oracle, pat, wins[rank])
        C, Ch = window_state(pat, wins[rank])
        rep = st.newton_step(ctx, st.DistComm(dist), strips, pat.nv, C, Ch, tol=1e-12)
        np.save(os.path.join(out_dir, f"C{rank}.npy"), owned_rows(pat, wins[rank], C))
        np.save(os.path.join(out_dir, f"rep{rank}.npy"), np.array([rep["E0"], rep["E1"], rep["alpha"],
                                                                    rep["pcg_iters"], rep["pcg_rel_res"]]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_bit_identical(orc, one_rank, tmp_path):
    import torch.multiprocessing as mp
    pat, (reps1, C1) = one_rank
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.start_processes(_gloo_rank, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    C = np.concatenate([np.load(tmp_path / f"C{r}.npy") for r in range(2)])
    assert np.array_equal(C, C1)
    r1 = reps1[0]
    for r in range(2):
        rep = np.load(tmp_path / f"rep{r}.npy")
        assert list(rep) == [r1["E0"], r1["E1"], r1["alpha"], r1["pcg_iters"], r1["pcg_rel_res"]]
