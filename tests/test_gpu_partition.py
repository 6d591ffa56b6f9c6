"""A garment batch split over two ranks (paper_2506_18867_gb300.partition),
each rank a process with its own batched context, gloo for the host-side
gathering: the union of the ranks' FP64 span terms, gradients and stencil
rows equals one context over the whole batch bit for bit, and their Newton
steps agree with it to the solver tolerance (the PCG's reductions group by
a different block split).  Both ranks run on the one GPU this test gets;
their kernels never wait on each other (the partition has no exchange).
"""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2506_18867_gb300 import build as _build  # noqa: E402

_build.build()

COUNT = 10


def _batch():
    from paper_2506_18867_gb300 import inputs
    return inputs.config_batch(3, count=COUNT, lo=12, hi=40)


def _results(pats):
    """Per patch: E, g, H span terms, gradient, K and the Newton step's C (numpy)."""
    from paper_2506_18867_gb300 import bsc
    ctx = bsc.batch_for_patches(pats, precision=bsc.FP64, pcg_rel_tol=1e-12)
    N = ctx.N
    C = torch.zeros((3, N), dtype=torch.float64)
    Ch = torch.zeros((3, N), dtype=torch.float64)
    for p, pat in enumerate(pats):
        a, b = ctx.cp_offset[p], ctx.cp_offset[p + 1]
        C[:, a:b] = torch.from_numpy(pat.C.T)
        Ch[:, a:b] = torch.from_numpy(pat.Chat.T)
    C, Ch = C.cuda().contiguous(), Ch.cuda().contiguous()
    E, g, H = ctx.span_terms(C, project=True)
    grad = ctx.gradient(C, Ch)
    K = ctx.assemble_hessian(C, project=True)
    ctx.newton_step(C, Ch)
    out = []
    for p in range(len(pats)):
        s0, s1 = int(ctx.span_offset[p]), int(ctx.span_offset[p + 1])
        a, b = int(ctx.cp_offset[p]), int(ctx.cp_offset[p + 1])
        out.append({"E": E[s0:s1].cpu().numpy(), "g": g[s0:s1].cpu().numpy(), "H": H[s0:s1].cpu().numpy(),
                    "grad": grad[:, a:b].cpu().numpy(), "K": K[:, a:b].cpu().numpy(),
                    "C": C[:, a:b].cpu().numpy()})
    ctx.close()
    return out


def _rank_main(rank, world, port, out_dir):
    import pickle
    import sys

    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch as th
    th.cuda.set_device(0)
    from paper_2506_18867_gb300 import partition
    dist.init_process_group("gloo", rank=rank, world_size=world)
    idx, mine = partition.rank_patches(_batch(), rank, world)
    res = _results(mine)
    gathered = [None] * world
    dist.all_gather_object(gathered, (idx, res))
    if rank == 0:
        with open(os.path.join(out_dir, "gathered.pkl"), "wb") as f:
            pickle.dump(gathered, f)
    dist.barrier()
    dist.destroy_process_group()


def test_batch_split_over_two_ranks_matches_one_context(tmp_path):
    import pickle

    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    gathered = pickle.load(open(tmp_path / "gathered.pkl", "rb"))
    pats = _batch()
    whole = _results(pats)
    seen = []
    for idx, res in gathered:
        assert len(idx) > 0
        for p, r in zip(idx, res):
            seen.append(p)
            w = whole[p]
            for key in ("E", "g", "H", "grad", "K"):
                assert np.array_equal(r[key], w[key]), (p, key)
            width = np.ptp(pats[p].rest, axis=0).max()
            assert np.abs(r["C"] - w["C"]).max() <= 1e-10 * width, p
    assert sorted(seen) == list(range(COUNT))
