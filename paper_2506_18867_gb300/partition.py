"""Work partition across ranks (one process per GPU).

A batch of independent garment patches shards with no data exchange: every
rank creates a batched context of the patches assigned to it and steps them
on its own GPU.  The assignment balances the ranks' work - the span count of
a patch, which sets the cost of span evaluation, projection and assembly,
times its expected solver work when known - by the longest-processing-time
rule: patches in decreasing order of work (ties to the lower index), each to
the rank with the least work so far (ties to the lower rank).  The rule is
deterministic, so every rank computes the same assignment from the same
inputs without communicating.

Pure host code; no GPU needed.
"""
from __future__ import annotations


def assign_patches(work, ranks):
    """Lists of patch indices per rank (each sorted ascending).  work: per-patch
    positive costs; ranks >= 1.  Every patch goes to exactly one rank; a rank
    may get none when there are fewer patches than ranks."""
    if ranks < 1:
        raise ValueError("ranks must be >= 1")
    order = sorted(range(len(work)), key=lambda p: (-float(work[p]), p))
    load = [0.0] * ranks
    out = [[] for _ in range(ranks)]
    for p in order:
        r = min(range(ranks), key=lambda k: (load[k], k))
        out[r].append(p)
        load[r] += float(work[p])
    return [sorted(v) for v in out]


def patch_work(patches):
    """Work estimate of each patch: its span count."""
    return [(p.nu - 2) * (p.nv - 2) for p in patches]


def rank_patches(patches, rank, world):
    """The patches of `rank` (and their indices in the batch) under assign_patches."""
    idx = assign_patches(patch_work(patches), world)[rank]
    return idx, [patches[i] for i in idx]


def imbalance(work, assignment):
    """Largest rank load over the mean load (1.0 = perfect balance)."""
    loads = [sum(float(work[p]) for p in v) for v in assignment]
    mean = sum(loads) / len(loads)
    return max(loads) / mean if mean > 0 else 1.0


# ---------------------------------------------------------------------------
# Strips of one large patch: rank r owns the control-point rows
# [j0, j1) = strip_rows(nv, world)[r] (v direction, whole rows).  Span b
# covers rows b .. b + 2 and is owned by the rank of its middle row b + 1, so
# every span has one owner.  The rows a rank owns need the spans that touch
# them, b in [j0 - 2, j1), whose control points are the rows
# [j0 - 2, j1 + 2): the strip and a halo of two rows on each side (clipped to
# the grid).  A product y = K x on the owned rows reads x on the same rows.
# ---------------------------------------------------------------------------

def strip_rows(nv, world):
    """Contiguous row ranges [j0, j1) per rank, sizes differing by at most one."""
    if world < 1 or nv < world:
        raise ValueError("need 1 <= world <= nv")
    q, r = divmod(nv, world)
    out, j = [], 0
    for k in range(world):
        n = q + (1 if k < r else 0)
        out.append((j, j + n))
        j += n
    return out


def span_owner(strips, b):
    """Rank owning span b (the rank of its middle row b + 1)."""
    for r, (j0, j1) in enumerate(strips):
        if j0 <= b + 1 < j1:
            return r
    raise ValueError(f"span {b} outside the strips")


def window_rows(strips, rank, nv):
    """Rows [w0, w1) of control points a rank holds: its strip and two halo rows each side."""
    j0, j1 = strips[rank]
    return max(0, j0 - 2), min(nv, j1 + 2)


def window_spans(strips, rank, nv):
    """Spans [s0, s1) that touch the rank's rows (all of them lie in its window)."""
    j0, j1 = strips[rank]
    return max(0, j0 - 2), min(nv - 2, j1)


def owned_spans(strips, rank, nv):
    """Spans [o0, o1) the rank owns (middle row in its strip)."""
    j0, j1 = strips[rank]
    return max(0, j0 - 1), min(nv - 2, j1 - 1)
