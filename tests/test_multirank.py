"""Multi-rank host logic with two gloo ranks on CPU: every source group is processed exactly once
across ranks, and the gathered loops equal a single-process run (units are independent)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2609_37049_b300.shard import source_groups, shard, gather_loops, units_for_step


def fake_loops(group):
    """Stand-in for the per-group GPU work: deterministic values per timeslice."""
    return {t: np.array([np.sin(t + 0.5), np.cos(3 * t)]) for t in group}


def _worker(rank, world, port, groups, out_q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = {}
    for g in shard(groups, rank, world):
        local.update(fake_loops(g))
    merged = gather_loops(local, rank, world, dist)
    if rank == 0:
        out_q.put({t: v.tolist() for t, v in merged.items()})
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_source_groups_tile_every_timeslice_once():
    for Lt, ext in ((32, [4] * 8), (48, [6, 8, 10, 6, 8, 10]), (8, [4, 4]), (8, [8])):
        groups = source_groups(Lt, ext)
        flat = sorted(t for g in groups for t in g)
        assert flat == list(range(Lt))
        starts = np.cumsum([0] + ext[:-1])
        dom = np.repeat(np.arange(len(ext)), ext)
        for g in groups:
            assert len({int(dom[t]) for t in g}) == len(g)  # at most one timeslice per domain
    with pytest.raises(ValueError):
        source_groups(8, [4, 3])


def test_source_groups_of_shifted_tiling():
    """Tiling [3, 5] starting at t = 6: domain 0 = {6, 7, 0}, domain 1 = {1, ..., 5}."""
    groups = source_groups(8, [3, 5], t_start=6)
    assert groups == [[6, 1], [7, 2], [0, 3], [4], [5]]
    assert sorted(t for g in groups for t in g) == list(range(8))
    with pytest.raises(ValueError):
        source_groups(8, [3, 5], t_start=8)


def test_units_for_step_cover_all_units_across_ranks():
    units = source_groups(32, [4] * 8)
    seen = [units_for_step(units, s, r, 2) for s in range(2) for r in range(2)]
    assert sorted(map(tuple, seen)) == sorted(map(tuple, units))


def test_two_gloo_ranks_gather_equals_single_process():
    groups = source_groups(48, [6, 8, 10, 6, 8, 10])
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, groups, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    single = {}
    for g in groups:
        single.update(fake_loops(g))
    assert sorted(int(t) for t in got) == list(range(48))
    for t, v in single.items():
        assert np.allclose(got[t], v)


def test_duplicate_timeslice_is_an_error():
    class FakeDist:
        def all_gather_object(self, parts, obj):
            parts[0] = {1: 1.0}
            parts[1] = {1: 2.0}
    with pytest.raises(RuntimeError):
        gather_loops({1: 1.0}, 0, 2, FakeDist())


def test_plan_unit_covers_every_rhs_block_once():
    from paper_2609_37049_b300.shard import plan_unit
    for n_full, n_groups, n_blocks in ((16, 1, 32), (32, 4, 8), (48, 10, 4)):
        full = [plan_unit(u, n_full, n_groups, n_blocks)[:2] for u in range(n_full * n_blocks)]
        dom = [plan_unit(u, n_full, n_groups, n_blocks)[2:] for u in range(n_groups * n_blocks)]
        assert len(set(full)) == n_full * n_blocks
        assert len(set(dom)) == n_groups * n_blocks


def _fake_unit(unit, t_src, groups, n_blocks):
    """Stand-in for one bench step's GPU work on unit `unit` (the plan of bench.py): the loops of
    the full-operator block at one source timeslice and of the domain-operator block of one group."""
    from paper_2609_37049_b300.shard import plan_unit
    k, bf, g, bd = plan_unit(unit, len(t_src), len(groups), n_blocks)
    out = {("f", t_src[k], bf): np.array([np.sin(t_src[k] + 0.1 * bf), np.cos(bf)])}
    if unit < len(groups) * n_blocks:  # the domain work repeats after every group and block was done
        for t in groups[g]:
            out[("d", t, bd)] = np.array([np.cos(t - 0.3 * bd), np.sin(2 * bd + t)])
    return out


def _bench_worker(rank, world, port, steps, t_src, groups, n_blocks, out_q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = {}
    for s in range(steps):
        for key, v in _fake_unit(s * world + rank, t_src, groups, n_blocks).items():
            assert key not in local  # a rank never repeats a unit within the run
            local[key] = v
    merged = gather_loops(local, rank, world, dist)
    if rank == 0:
        out_q.put({k: v.tolist() for k, v in merged.items()})
    dist.barrier()
    dist.destroy_process_group()


def test_bench_step_plan_gathered_over_two_ranks_equals_one_rank():
    """bench.py under torchrun: rank r runs unit s * world + r in step s (weak scaling, no exchange
    during the steps); gathering the per-rank loops afterwards gives exactly the single-rank run of
    twice the steps, and n_full * n_blocks units cover every full-operator block once."""
    from paper_2609_37049_b300.shard import domain_groups
    t_src = list(range(0, 96, 6))
    groups = domain_groups(t_src, 96, [8] * 12)
    n_blocks = 4
    steps = len(t_src) * n_blocks // 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_worker, args=(r, 2, port, steps, t_src, groups, n_blocks, q))
             for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    single = {}
    for u in range(2 * steps):
        for key, v in _fake_unit(u, t_src, groups, n_blocks).items():
            single[key] = v
    assert set(got) == set(single)
    for key, v in single.items():
        assert np.allclose(got[key], v)
    full = sorted((t, b) for (kind, t, b) in single if kind == "f")
    assert full == sorted((t, b) for t in t_src for b in range(n_blocks))
    dom = sorted((t, b) for (kind, t, b) in single if kind == "d")
    assert dom == sorted((t, b) for g in groups for t in g for b in range(n_blocks))
