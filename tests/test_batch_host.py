"""Host-side logic of the batched workload (no GPU): the PCG block split
(bsc_plan_blocks, a pure host function of libbsc.so), the batched-garment
generator, and the cross-rank aggregation of the bench on two gloo ranks."""
import itertools
import math
import os

import numpy as np
import pytest

from paper_2506_18867_gb300 import inputs


@pytest.fixture(scope="module")
def bsc():
    from paper_2506_18867_gb300 import build as _build
    _build.build()
    from paper_2506_18867_gb300 import bsc as mod
    mod.load()
    return mod


def brute_force_split(n_cp, work, total):
    caps = [max(1, math.ceil(n / 256)) for n in n_cp]
    use = min(total, sum(caps))
    best = None
    for alloc in itertools.product(*[range(1, c + 1) for c in caps]):
        if sum(alloc) != use:
            continue
        m = max(w / b for w, b in zip(work, alloc))
        best = m if best is None else min(best, m)
    return use, best


@pytest.mark.parametrize("case", range(40))
def test_plan_blocks_is_optimal(bsc, case):
    rng = np.random.default_rng(case)
    P = int(rng.integers(1, 5))
    n_cp = [int(v) for v in rng.integers(25, 1800, P)]
    work = [float(v) for v in rng.uniform(1.0, 50.0, P) * np.array(n_cp)]
    total = int(rng.integers(P, 16))
    used, blocks = bsc.plan_blocks(n_cp, work, total)
    want_use, want_max = brute_force_split(n_cp, work, total)
    assert used == want_use == sum(blocks)
    assert all(1 <= b <= max(1, math.ceil(n / 256)) for b, n in zip(blocks, n_cp))
    assert max(w / b for w, b in zip(work, blocks)) == pytest.approx(want_max, rel=1e-12)


def test_plan_blocks_edge_cases(bsc):
    assert bsc.plan_blocks([100, 100], [1.0, 1.0], 1)[0] == -1          # fewer blocks than patches
    used, b = bsc.plan_blocks([100], [5.0], 304)                         # one small patch: one block
    assert used == 1 and b == [1]
    used, b = bsc.plan_blocks([65536], [65536.0], 304)                   # the drape: capped by the grid
    assert used == 256 and b == [256]
    used, b = bsc.plan_blocks([256] * 4, [1.0, 2.0, 3.0, 4.0], 4)        # exactly one each
    assert used == 4 and b == [1, 1, 1, 1]
    used, b = bsc.plan_blocks([10000, 10000], [1.0, 1.0], 10)             # ties go to the lower index
    assert b == [5, 5]
    used, b = bsc.plan_blocks([10000, 10000], [1.0, 1.0], 9)
    assert b == [5, 4]


def test_config_batch_distribution():
    pats = inputs.config_batch(1)
    assert len(pats) == 64
    nu = np.array([p.nu for p in pats])
    nv = np.array([p.nv for p in pats])
    assert nu.min() >= 16 and nv.min() >= 16 and nu.max() <= 192 and nv.max() <= 192
    assert (nu != nv).sum() >= 60                                        # non-square
    E = np.array([p.meta["E"] for p in pats])
    pr = np.array([p.meta["poisson"] for p in pats])
    assert E.min() >= 1e4 and E.max() <= 1e6 and 0.2 <= pr.min() and pr.max() <= 0.45
    # log-uniform E: about half the draws on each side of 1e5
    assert 20 <= (E < 1e5).sum() <= 44
    tot = sum(p.n_cp for p in pats)
    assert 4.5e5 < tot < 9.5e5                                            # 64 x E[n]^2 = 692K
    # deterministic per seed, different across seeds
    again = inputs.config_batch(1)
    assert all(np.array_equal(a.C, b.C) and a.nu == b.nu for a, b in zip(pats, again))
    other = inputs.config_batch(2)
    assert any(a.nu != b.nu or a.nv != b.nv for a, b in zip(pats, other))


def test_config_batch_rest_is_a_rotated_greville_grid():
    for p in inputs.config_batch(3, count=6):
        X = p.rest.reshape(p.nv, p.nu, 2)
        # 1 cm spans: interior Greville points are one span apart along both axes
        du = np.linalg.norm(X[:, 2:-1] - X[:, 1:-2], axis=-1)
        dv = np.linalg.norm(X[2:-1, :] - X[1:-2, :], axis=-1)
        assert np.allclose(du, 0.01, atol=1e-12) and np.allclose(dv, 0.01, atol=1e-12)
        # the two axes stay orthogonal (a rotation, no shear)
        a = X[0, 1] - X[0, 0]
        b = X[1, 0] - X[0, 0]
        assert abs(np.dot(a, b)) < 1e-15
        assert list(p.pinned) == [(p.nv - 1) * p.nu, p.nv * p.nu - 1]
        assert np.abs(p.C[:, :2] - p.rest).max() < 0.01                  # sigma = 1 mm perturbation


def _rank_main(rank, world, port, out_dir):
    import sys

    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # every rank builds its own batch (seed 1 + rank), as the bench does
    pats = inputs.config_batch(1 + rank, count=4)
    spans = sum(p.n_spans for p in pats)
    agg = bench.reduce_over_ranks(dist, {"eval": 10.0 + rank, "step": 30.0 - 5 * rank}, spans, "cpu")
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(f"{agg['eval']} {agg['step']} {agg['spans']} {spans}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_weak_scaling_aggregation_two_gloo_ranks(tmp_path):
    import socket

    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    rows = [list(map(float, open(tmp_path / f"rank{r}.txt").read().split())) for r in range(2)]
    local = [int(r[3]) for r in rows]
    assert local[0] != local[1]                       # different seeds, different batches
    for r in rows:
        assert r[0] == 11.0 and r[1] == 30.0          # max over ranks
        assert int(r[2]) == sum(local)                # work adds up
