"""Work partition across ranks (one process per GPU).

The distillation path shards without any exchange during the solves: a unit of work is a source
group, i.e. one source timeslice per domain (t = g, g + e_0, ... for the tiling of the time axis),
whose full-operator and domain-operator perambulators and loops are independent of every other
group.  Units are dealt round-robin to ranks; the only collective is a gather of the per-group
loops (a few kilobytes) to the rank that forms the correlators.
"""
import numpy as np


def source_groups(Lt, extents, t_start=0):
    """Source groups of a tiling of the time axis whose domain 0 starts at t_start: group g holds
    t0(d) + g (mod Lt) for every domain d wide enough, g = 0 .. max(extents) - 1 (domains narrower
    than g + 1 drop out of group g)."""
    extents = [int(e) for e in extents]
    if sum(extents) != Lt or min(extents) < 1:
        raise ValueError("extents must tile the time axis")
    if not 0 <= int(t_start) < Lt:
        raise ValueError("t_start outside [0, Lt)")
    starts = int(t_start) + np.cumsum([0] + extents[:-1])
    return [[int((s + g) % Lt) for s, e in zip(starts, extents) if g < e] for g in range(max(extents))]


def domain_groups(t_src, Lt, extents, t_start=0):
    """Groups of the source timeslices t_src for multi-site domain solves: each group holds at
    most one timeslice per domain (level k of every domain's list, in t_src order), the grouping
    the library's domain-mode perambulators use."""
    extents = [int(e) for e in extents]
    if sum(extents) != Lt or min(extents) < 1:
        raise ValueError("extents must tile the time axis")
    dom = np.empty(Lt, dtype=np.int64)
    t = int(t_start)
    for d, e in enumerate(extents):
        for k in range(e):
            dom[(t + k) % Lt] = d
        t += e
    per = {}
    for ts in t_src:
        per.setdefault(int(dom[int(ts)]), []).append(int(ts))
    groups = []
    level = 0
    while True:
        grp = [per[d][level] for d in sorted(per) if level < len(per[d])]
        if not grp:
            return groups
        groups.append(grp)
        level += 1


def shard(units, rank, world):
    """Units of this rank: round-robin over the list."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return list(units)[rank::world]


def units_for_step(units, step, rank, world):
    """The unit a rank processes in bench step `step` (weak scaling: every rank one unit per step)."""
    return units[(step * world + rank) % len(units)]


def plan_unit(unit, n_full, n_groups, n_blocks):
    """Work of bench unit `unit` (unit = step * world + rank): the full-operator source timeslice
    index k (into t_src) with its RHS block bf, and the domain source-group index g with its RHS
    block bd (block b = source vectors b * nj .. b * nj + nj - 1, all spins).  The full work walks
    the timeslices first, then the blocks, so n_full * n_blocks consecutive units cover every
    full-operator right-hand side once; the domain work walks the groups, then the blocks, so
    n_groups * n_blocks consecutive units cover every domain right-hand side once.  Returns
    (k, bf, g, bd)."""
    if unit < 0 or min(n_full, n_groups, n_blocks) < 1:
        raise ValueError("bad unit or sizes")
    return unit % n_full, (unit // n_full) % n_blocks, unit % n_groups, (unit // n_groups) % n_blocks


def gather_loops(local, rank, world, dist=None):
    """Gather {t: loop values} dictionaries of all ranks on every rank (torch.distributed object
    gather; the identity when world == 1).  Raises if two ranks produced the same timeslice."""
    if world == 1 or dist is None:
        merged = dict(local)
    else:
        parts = [None] * world
        dist.all_gather_object(parts, dict(local))
        merged = {}
        for p in parts:
            for t, v in p.items():
                if t in merged:
                    raise RuntimeError("timeslice %d computed by two ranks" % t)
                merged[t] = v
    return dict(sorted(merged.items()))
