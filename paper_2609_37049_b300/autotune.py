"""Autotuner for the batched solver: the dslash launch variant (register cap / resident blocks) and the RHS block
width (right-hand sides solved in lockstep per launch), persisted in a JSON cache keyed by
lattice extents, GPU name and precision.

    from paper_2609_37049_b300 import Context, autotune
    choice = autotune.tune(ctx, cache="tuning.json")     # times once, then reads the cache
    params.rhs_block = choice["rhs_block"]

The RHS block is chosen from the measured dslash time per right-hand side (the solver's cost is
dominated by the Schur-operator dslash pair; wider blocks share the link and clover loads), among
widths whose work vectors fit a memory budget.
"""
import json
import os

from . import lqcd

CANDIDATE_BLOCKS = (16, 32, 64, 128)


def _gpu_name():
    try:
        import torch
        return torch.cuda.get_device_name(0)
    except Exception:
        return "unknown"


def _key(ctx):
    return "%s|%s" % ("x".join(str(d) for d in ctx.dims), _gpu_name())


def _spinor_bytes(ctx, prec, nrhs):
    per = {lqcd.LQCD_PREC_F64: 16, lqcd.LQCD_PREC_F32: 8, lqcd.LQCD_PREC_F16: 4, lqcd.LQCD_PREC_DF: 16}[prec]
    return ctx.volume // 2 * nrhs * 12 * per


def _device_budget():
    """60% of the device memory (the work vectors of one batch must fit beside the caller's)."""
    try:
        import torch
        return int(0.6 * torch.cuda.mem_get_info()[1])
    except Exception:
        return 64 << 30


def tune(ctx, cache=None, precisions=(lqcd.LQCD_PREC_F32, lqcd.LQCD_PREC_F16, lqcd.LQCD_PREC_F64,
                                      lqcd.LQCD_PREC_DF),
         blocks=CANDIDATE_BLOCKS, memory_budget=None, retune=False):
    """Tune (or load from `cache`) and install the launch choices on ctx; returns the choice dict.
    memory_budget (bytes; default 60% of the device memory) bounds the RHS blocks tried."""
    if memory_budget is None:
        memory_budget = _device_budget()
    db = {}
    if cache and os.path.exists(cache) and not retune:
        with open(cache) as f:
            db = json.load(f)
    key = _key(ctx)
    if key in db:
        choice = db[key]
        for prec, per_n in choice["variant"].items():
            for n, v in per_n.items():
                ctx.set_dslash_variant(int(prec), int(n), int(v))
        return choice
    variants, per_rhs = {}, {}
    for prec in precisions:
        variants[str(prec)] = {}
        for n in blocks:
            # timing a variant needs two vectors of the block; choosing the block as the solver's
            # width needs its work vectors (about 20 of the inner precision plus FP64 outer ones)
            # to fit the budget.  A single requested block is tuned whatever its size.
            if 2 * _spinor_bytes(ctx, prec, n) > memory_budget:
                continue
            t, ms = ctx.tune_dslash(prec, n)
            variants[str(prec)][str(n)] = t
            need = 20 * _spinor_bytes(ctx, prec, n) + 8 * _spinor_bytes(ctx, lqcd.LQCD_PREC_F64, n)
            if prec == lqcd.LQCD_PREC_F32 and (need <= memory_budget or len(blocks) == 1):
                per_rhs[n] = ms / n
    best = min(per_rhs, key=per_rhs.get) if per_rhs else 64
    choice = {"variant": variants, "rhs_block": int(best),
              "dslash_ms_per_rhs_f32": {str(k): v for k, v in per_rhs.items()}}
    if cache:
        db[key] = choice
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1, sort_keys=True)
        os.replace(tmp, cache)
    return choice
