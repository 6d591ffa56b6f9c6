"""Host logic of the multi-GPU partitions, on CPU (no GPU needed).

- The patch -> rank assignment of a garment batch (partition.assign_patches):
  every patch on exactly one rank, deterministic, balanced within one patch
  of the ideal, and computed identically by two gloo ranks that never
  exchange it (each rank derives its share from the same inputs).
- The strip partition of one patch (partition.strip_rows): owned rows tile
  the grid, spans have one owner each, the halo rows a rank needs are the
  two rows beyond its strip.
"""
import os

import numpy as np
import pytest

from paper_2506_18867_gb300 import inputs, partition


def test_assignment_covers_every_patch_once():
    pats = inputs.config_batch(1, 64)
    work = partition.patch_work(pats)
    for world in (1, 2, 3, 4, 8):
        a = partition.assign_patches(work, world)
        flat = sorted(p for v in a for p in v)
        assert flat == list(range(64)), world
        assert partition.assign_patches(work, world) == a          # deterministic
        loads = [sum(work[p] for p in v) for v in a]
        # LPT: the largest load exceeds the mean by less than the largest patch
        assert max(loads) - sum(loads) / world <= max(work), world
        print(world, "ranks: imbalance", round(partition.imbalance(work, a), 4))
    assert partition.imbalance(work, partition.assign_patches(work, 8)) < 1.05


def test_more_ranks_than_patches():
    a = partition.assign_patches([5.0, 3.0], 4)
    assert sorted(p for v in a for p in v) == [0, 1] and sum(1 for v in a if not v) == 2
    with pytest.raises(ValueError):
        partition.assign_patches([1.0], 0)


@pytest.mark.parametrize("nv,world", [(5, 1), (9, 2), (64, 3), (1024, 8), (7, 4)])
def test_strip_rows_tile_the_grid(nv, world):
    strips = partition.strip_rows(nv, world)
    assert strips[0][0] == 0 and strips[-1][1] == nv
    for (a0, a1), (b0, b1) in zip(strips, strips[1:]):
        assert a1 == b0 and a1 > a0
    sizes = [b - a for a, b in strips]
    assert max(sizes) - min(sizes) <= 1
    # every span (rows b .. b + 2) has exactly one owner: the rank of its middle row
    owners = [partition.span_owner(strips, b) for b in range(nv - 2)]
    for b, r in enumerate(owners):
        assert strips[r][0] <= b + 1 < strips[r][1]
    # a rank's span window and halo rows
    for r, (j0, j1) in enumerate(strips):
        w0, w1 = partition.window_rows(strips, r, nv)
        assert w0 == max(0, j0 - 2) and w1 == min(nv, j1 + 2)
        s0, s1 = partition.window_spans(strips, r, nv)
        assert s0 == max(0, j0 - 2) and s1 == min(nv - 2, j1)


def _rank_main(rank, world, port, out_dir):
    import sys

    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from paper_2506_18867_gb300 import inputs as inp
    from paper_2506_18867_gb300 import partition as part
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pats = inp.config_batch(1, 64)
    idx, mine = part.rank_patches(pats, rank, world)
    mask = torch.zeros(64, dtype=torch.int64)
    mask[idx] = 1
    dist.all_reduce(mask)                       # how many ranks hold each patch
    spans = torch.tensor([sum(p.n_spans for p in mine)], dtype=torch.int64)
    dist.all_reduce(spans)
    with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
        f.write(" ".join(map(str, mask.tolist())) + f"\n{spans.item()} {len(idx)}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_partition_a_batch(tmp_path):
    import socket

    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    total = sum(p.n_spans for p in inputs.config_batch(1, 64))
    for r in range(2):
        lines = open(tmp_path / f"rank{r}.txt").read().split("\n")
        assert list(map(int, lines[0].split())) == [1] * 64    # every patch on exactly one rank
        spans, npat = map(int, lines[1].split())
        assert spans == total and npat > 0
