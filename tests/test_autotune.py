"""Autotuner cache logic (host side; the timing itself runs on the GPU)."""
import json

from paper_2609_37049_b300 import autotune, lqcd


class FakeCtx:
    dims = (8, 8, 8, 16)
    volume = 8 * 8 * 8 * 16

    def __init__(self):
        self.timed, self.installed = [], []

    def tune_dslash(self, prec, n):
        self.timed.append((prec, n))
        return (2 if n >= 64 else 0), 0.01 * n ** 0.8  # wider blocks: cheaper per RHS

    def set_dslash_variant(self, prec, n, v):
        self.installed.append((prec, n, v))


def test_tune_writes_cache_and_reload_installs_it(tmp_path):
    cache = str(tmp_path / "tune.json")
    c1 = FakeCtx()
    ch = autotune.tune(c1, cache=cache, precisions=(lqcd.LQCD_PREC_F32,), blocks=(16, 32, 64, 128))
    assert ch["rhs_block"] == 128 and len(c1.timed) == 4
    db = json.load(open(cache))
    assert len(db) == 1
    c2 = FakeCtx()
    ch2 = autotune.tune(c2, cache=cache)
    assert ch2 == ch and c2.timed == [] and (lqcd.LQCD_PREC_F32, 64, 2) in c2.installed


def test_memory_budget_excludes_wide_blocks(tmp_path):
    """Every block is timed (two vectors fit), but a block whose solver work vectors exceed the
    budget is not chosen as the RHS width."""
    c = FakeCtx()
    ch = autotune.tune(c, cache=None, precisions=(lqcd.LQCD_PREC_F32,), memory_budget=1 << 30)
    assert [n for _, n in c.timed] == [16, 32, 64, 128] and ch["rhs_block"] == 64
    assert ch["variant"][str(lqcd.LQCD_PREC_F32)]["128"] == 2


def test_single_requested_block_is_tuned_beyond_the_budget():
    """A caller that fixes the block (the 48^3 x 96 bench, 16 RHS) still gets its launch variant."""
    c = FakeCtx()
    ch = autotune.tune(c, cache=None, precisions=(lqcd.LQCD_PREC_F32,), blocks=(64,), memory_budget=200 << 20)
    assert c.timed == [(lqcd.LQCD_PREC_F32, 64)] and ch["rhs_block"] == 64
