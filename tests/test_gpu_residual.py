"""The defect correction's true residual r = b - D x.

The library computes it either in double-float arithmetic (pairs of floats on the FP32 pipe, read
from and written to the FP64 fields; the default) or in native FP64.  Either way the relative
residual it reports for each right-hand side (and domain) must equal the oracle's FP64 residual of
the solution it returns, to well below the 1e-10 tolerance: the double-float arithmetic errs by
about 2^-47 of the operands, so |reported - oracle| <= 2e-13 + 1e-3 reported.  Sources scaled by
1e-18 and 1e18 exercise the exponent handling of the FP64-to-double-float split.
"""
import numpy as np
import pytest

from lqcd_inputs import random_spinors
from oracle.dirac import WilsonClover
from tests.lattice_cases import ROUGH, gauge, per_domain_resid

pytestmark = pytest.mark.gpu

pytest.importorskip("paper_2609_37049_b300")
from paper_2609_37049_b300 import Context, Stats, default_params, lqcd  # noqa: E402


def _setup(seed):
    case = ROUGH
    U = gauge(case, seed)
    ctx = Context(case["dims"])
    ctx.gauge_upload(U, case["kappa"], case["c_sw"])
    ctx.set_domains(case["extents"])
    return case, U, ctx


@pytest.mark.parametrize("residual", [0, 1])
@pytest.mark.parametrize("scale", [1.0, 1e-18, 1e18])
@pytest.mark.parametrize("domain", [False, True])
def test_reported_true_residual_matches_oracle(domain, scale, residual):
    case, U, ctx = _setup(2301)
    ext = case["extents"] if domain else [case["dims"][3]]
    b = random_spinors(case["dims"], 4, 2302) * scale
    x = np.zeros_like(b)
    st = Stats(4, len(ext))
    ctx.solve(b, x, default_params(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F32, rhs_block=4,
                                   residual=residual), domain=domain, stats=st)
    op = WilsonClover(U, case["kappa"], case["c_sw"])
    if domain:
        op = op.restricted(case["extents"])
    res = per_domain_resid(b, b - op.apply(x), ext)
    assert res.max() <= 1.02e-10, res
    lib = st.true_resid.reshape(4, len(ext))
    assert np.abs(lib - res).max() <= 2e-13 + 1e-3 * res.max(), (lib, res)


@pytest.mark.parametrize("solver", ["plain", "mixed"])
def test_double_float_and_fp64_residual_give_the_same_solution(solver):
    case, U, ctx = _setup(2303)
    b = random_spinors(case["dims"], 4, 2304)
    kw = dict(solver=lqcd.LQCD_SOLVER_BICGSTAB64) if solver == "plain" else dict(
        solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F32)
    xs = []
    for residual in (0, 1):
        x = np.zeros_like(b)
        st = Stats(4, 1)
        ctx.solve(b, x, default_params(rhs_block=4, residual=residual, **kw), stats=st)
        assert st.max_true_resid <= 1e-10
        xs.append(x)
    assert np.linalg.norm(xs[0] - xs[1]) <= 1e-11 * np.linalg.norm(xs[1])


def test_tune_the_residual_kernel():
    case, U, ctx = _setup(2305)
    v, ms = ctx.tune_dslash(lqcd.LQCD_PREC_DF, 4)
    assert 0 <= v <= 2 and ms > 0
    ctx.set_dslash_variant(lqcd.LQCD_PREC_DF, 4, 1)
    b = random_spinors(case["dims"], 4, 2306)
    x = np.zeros_like(b)
    st = Stats(4, 1)
    ctx.solve(b, x, default_params(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F32, rhs_block=4),
              stats=st)
    assert st.max_true_resid <= 1e-10
