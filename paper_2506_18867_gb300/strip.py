"""Strip decomposition of one patch over ranks: the projected Newton
iteration (Sec. 5.1: Newton direction from the block-Jacobi PCG, then
backtracking from alpha = 1 until the incremental potential does not
increase) with each rank holding a strip window of the patch
(bsc_create_window, include/bsc.h).

Rank r owns the control-point rows strips[r] = [j0, j1) (partition.strip_rows)
and holds them plus two halo rows each side.  Per Newton iteration the ranks
exchange
  - the halo rows of the search direction p before every product K p, and
    of the solution d before the line search (from the rows' owners);
  - the per-row partial sums of the PCG's dot products and of the energy
    (an all-gather), which every rank adds up with a correctly rounded sum
    (math.fsum), so the scalars - and with them all iterates - do not depend
    on how the rows are split: every decomposition, one rank included,
    gives the same result bit for bit.
The per-rank work runs in the library's kernels; this module only orders the
calls and moves rows and scalars between ranks through a `comm` object:
  ThreadComm - host threads in one process driving contexts on one device
               (the halo copies are device-to-device copies on the default
               stream that every context uses);
  DistComm   - torch.distributed process groups (NCCL between GPUs, gloo for
               CPU tensors), point-to-point sends of the halo rows.
No kernel waits for another rank: ranks meet only on the host, between
launches.
"""
from __future__ import annotations

import math
import threading

import numpy as np

from . import partition


def owner_of_row(strips, j):
    for r, (j0, j1) in enumerate(strips):
        if j0 <= j < j1:
            return r
    raise ValueError(f"row {j} outside the strips")


def halo_plan(strips, rank, nv):
    """The halo rows of `rank` as (owner, g0, g1) global row ranges."""
    w0, w1 = partition.window_rows(strips, rank, nv)
    j0, j1 = strips[rank]
    out = []
    for a, b in ((w0, j0), (j1, w1)):
        g = a
        while g < b:
            o = owner_of_row(strips, g)
            e = min(b, strips[o][1])
            out.append((o, g, e))
            g = e
    return out


def send_plan(strips, rank, nv):
    """The rows `rank` sends: (receiver, g0, g1) for every halo range it owns."""
    out = []
    for q in range(len(strips)):
        if q != rank:
            out.extend((q, g0, g1) for o, g0, g1 in halo_plan(strips, q, nv) if o == rank)
    return out


def _rows(t, nu, row0, g0, g1):
    """View of the global rows [g0, g1) of a window tensor (3, rows * nu) starting at row0."""
    return t.view(3, -1, nu)[:, g0 - row0:g1 - row0]


class ThreadHub:
    """Meeting point of `world` host threads, one per rank."""

    def __init__(self, world):
        self.world = world
        self.barrier = threading.Barrier(world)
        self.slots = [None] * world

    def comm(self, rank):
        return ThreadComm(self, rank)


class ThreadComm:
    def __init__(self, hub, rank):
        self.hub, self.rank, self.world = hub, rank, hub.world

    def allgather(self, obj):
        h = self.hub
        h.slots[self.rank] = obj
        h.barrier.wait()
        out = list(h.slots)
        h.barrier.wait()
        return out

    def exchange(self, t, strips, nv, nu, row0):
        """Fills t's halo rows from their owners' tensors (device copies, ordered
        on the shared stream after the owners' kernels launched before)."""
        tensors = self.allgather((t, row0))
        for o, g0, g1 in halo_plan(strips, self.rank, nv):
            src, srow0 = tensors[o]
            _rows(t, nu, row0, g0, g1).copy_(_rows(src, nu, srow0, g0, g1))
        self.hub.barrier.wait()   # no rank moves on (and overwrites its rows) before all copies are issued


class DistComm:
    """torch.distributed process group (already initialised) as the transport."""

    def __init__(self, dist):
        self.dist = dist
        self.rank, self.world = dist.get_rank(), dist.get_world_size()

    def allgather(self, obj):
        out = [None] * self.world
        self.dist.all_gather_object(out, obj)
        return out

    def exchange(self, t, strips, nv, nu, row0):
        import torch
        reqs, recvs = [], []
        for q, g0, g1 in send_plan(strips, self.rank, nv):
            buf = _rows(t, nu, row0, g0, g1).contiguous()
            reqs.append((self.dist.isend(buf, q), buf))
        for o, g0, g1 in halo_plan(strips, self.rank, nv):
            buf = torch.empty((3, g1 - g0, nu), dtype=t.dtype, device=t.device)
            recvs.append((self.dist.irecv(buf, o), buf, g0, g1))
        for rq, buf, g0, g1 in recvs:
            rq.wait()
            _rows(t, nu, row0, g0, g1).copy_(buf)
        for rq, _ in reqs:
            rq.wait()


def _fsum_rows(comm, rows):
    """Sums over all ranks of per-row partials: rows (k, n_own) -> k floats."""
    parts = comm.allgather(np.asarray(rows, dtype=np.float64).reshape(-1, np.shape(rows)[-1]))
    return [math.fsum(v for part in parts for v in part[i]) for i in range(parts[0].shape[0])]


def energy(ctx, comm, C, Chat):
    """Incremental potential of the whole patch at the window states C, Chat."""
    span_rows, cp_rows = ctx.energy_rows(C, Chat)
    parts = comm.allgather((np.asarray(span_rows), np.asarray(cp_rows)))
    return math.fsum(v for sr, cr in parts for v in list(sr) + list(cr))


class StripReport(dict):
    """E0, E1, alpha, halvings, pcg_iters, pcg_rel_res, dir_inf, status ("ok",
    "not_converged", "linesearch")."""


def newton_step(ctx, comm, strips, nv, C, Chat, tol=1e-8, max_iter=10000, max_halvings=30):
    """One projected Newton iteration of the patch, this rank's share.  ctx: the
    rank's strip window context; C, Chat: its window states (3, rows * nu),
    halo rows current; C is updated in place (halo rows included: every rank
    applies the same update to the rows it shares).  Every rank must call it
    with the same arguments apart from its own window."""
    nu = ctx.nu
    row0 = ctx.window[0]
    j0, j1 = ctx.window[2], ctx.window[3]
    g = ctx.gradient(C, Chat)
    K = ctx.assemble_hessian(C, project=True)
    E0 = energy(ctx, comm, C, Chat)
    x, p = ctx.new_vec(), ctx.new_vec()
    rz, bb = _fsum_rows(comm, ctx.pcg_begin(K, g, x, p))
    stop2 = tol * tol * bb
    rr, it = bb, 0
    converged = bb == 0.0
    if bb > 0.0:
        for it in range(1, max_iter + 1):
            comm.exchange(p, strips, nv, nu, row0)
            pq, = _fsum_rows(comm, ctx.pcg_product(K)[None, :])
            if not (pq > 0.0 and math.isfinite(pq)):
                raise FloatingPointError(f"strip PCG: p.Kp = {pq} at iteration {it}")
            rz_new, rr = _fsum_rows(comm, ctx.pcg_update(rz / pq))
            if rr <= stop2:
                converged = True
                break
            ctx.pcg_direction(rz_new / rz)
            rz = rz_new
    comm.exchange(x, strips, nv, nu, row0)
    dir_inf = max(comm.allgather(float(np.abs(_rows(x, nu, row0, j0, j1).cpu().numpy()).max())))
    alpha, E1, status, h = 1.0, E0, "linesearch", 0
    trial = ctx.new_vec()
    for h in range(max_halvings + 1):
        ctx.axpy(C, x, alpha, trial)
        E1 = energy(ctx, comm, trial, Chat)
        if E1 <= E0:
            ctx.axpy(C, x, alpha, C)
            status = "ok" if converged else "not_converged"
            break
        alpha *= 0.5
    return StripReport(E0=E0, E1=E1, alpha=alpha, halvings=h, pcg_iters=it,
                       pcg_rel_res=math.sqrt(rr / bb) if bb > 0 else 0.0, dir_inf=dir_inf, status=status)


def run_threads(world, fn):
    """Runs fn(rank, comm) in `world` host threads (one rank each) and returns
    their results in rank order; the first exception is re-raised."""
    hub = ThreadHub(world)
    out, err = [None] * world, []

    def body(r):
        try:
            out[r] = fn(r, hub.comm(r))
        except BaseException as e:   # noqa: BLE001 - handed to the caller
            err.append(e)
            hub.barrier.abort()

    ts = [threading.Thread(target=body, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if err:
        raise err[0]
    return out
