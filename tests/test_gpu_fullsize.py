"""Parity at the full size of the mixed-precision workload (16^3 x 32, eps 0.5, kappa 0.125,
c_sw 1.6, eight domains of 4 timeslices) in the launch configuration bench.py times: 64-RHS
blocks, the staged-links FP32 dslash (launch variant 3) and the FP64 residual variant the
autotuner picks there.  Outputs the oracle can compute one by one are sampled: a few right-hand
sides of the operator and of the solves, checked element by element (operators) or by the true
residual of the oracle's own D (solves, 1e-10 per RHS and per domain)."""
import numpy as np
import pytest

from lqcd_inputs import gauge_field, random_spinors
from oracle.dirac import WilsonClover, domain_of_t
from tests.lattice_cases import rel_max
from tests.test_gpu_dirac import oracle_schur

pytestmark = pytest.mark.gpu

pytest.importorskip("paper_2609_37049_b300")
from paper_2609_37049_b300 import Context, Stats, default_params, lqcd  # noqa: E402

DIMS = (16, 16, 16, 32)
EXT = [4] * 8
NRHS = 64
SAMPLE = [0, 37, 63]


@pytest.fixture(scope="module")
def full():
    U = gauge_field(DIMS, 0.5, 9001)
    op = WilsonClover(U, 0.125, 1.6)
    ctx = Context(DIMS)
    ctx.gauge_upload(U, 0.125, 1.6)
    ctx.set_domains(EXT)
    ctx.set_dslash_variant(lqcd.LQCD_PREC_F32, NRHS, 3)
    ctx.set_dslash_variant(lqcd.LQCD_PREC_F64, NRHS, 1)
    b = random_spinors(DIMS, NRHS, 9002)
    return dict(op=op, ctx=ctx, b=b)


def test_fullsize_operators(full):
    op, ctx, b = full["op"], full["ctx"], full["b"]
    out = np.zeros_like(b[:2])
    ctx.dirac_apply(np.ascontiguousarray(b[:2]), out)
    assert rel_max(out, op.apply(b[:2])) < 1e-14
    for prec, tol in ((lqcd.LQCD_PREC_F32, 2e-6), (lqcd.LQCD_PREC_F64, 1e-13)):
        out = np.zeros_like(b)
        ctx.schur_apply(prec, b, out)
        want = oracle_schur(op, b[SAMPLE])
        assert rel_max(out[SAMPLE], want) < tol, prec


@pytest.mark.parametrize("domain", [False, True])
def test_fullsize_mixed_solve_true_residual(full, domain):
    op, ctx, b = full["op"], full["ctx"], full["b"]
    x = np.zeros_like(b)
    st = Stats(NRHS, len(EXT) if domain else 1)
    ctx.solve(b, x, default_params(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F32, rhs_block=NRHS),
              domain=domain, stats=st)
    assert st.max_true_resid <= 1e-10
    ref = op.restricted(EXT) if domain else op
    dom = domain_of_t(EXT, DIMS[3]) if domain else np.zeros(DIMS[3], dtype=int)
    r = b[SAMPLE] - ref.apply(x[SAMPLE])
    for k in range(len(SAMPLE)):
        for d in np.unique(dom):
            m = dom == d
            assert np.linalg.norm(r[k, m]) / np.linalg.norm(b[SAMPLE[k], m]) <= 1.02e-10, (k, d)


def test_uneven_domains_24x48():
    """The batched uneven-domain configuration at full size (24^3 x 48, eps 0.5, kappa 0.125,
    domains of 6, 8, 10, 6, 8, 10 timeslices): one 16-RHS mixed domain solve, every domain of the
    sampled RHS checked by the oracle's own D_Lambda to 1e-10."""
    dims = (24, 24, 24, 48)
    ext = [6, 8, 10, 6, 8, 10]
    U = gauge_field(dims, 0.5, 9101)
    ctx = Context(dims)
    ctx.gauge_upload(U, 0.125, 1.6)
    ctx.set_domains(ext)
    b = random_spinors(dims, 16, 9102)
    x = np.zeros_like(b)
    st = Stats(16, len(ext))
    ctx.solve(b, x, default_params(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F32, rhs_block=16),
              domain=True, stats=st)
    assert st.max_true_resid <= 1e-10
    op = WilsonClover(U, 0.125, 1.6).restricted(ext)
    dom = domain_of_t(ext, dims[3])
    sample = [0, 15]
    r = b[sample] - op.apply(x[sample])
    for k in range(len(sample)):
        for d in range(len(ext)):
            m = dom == d
            assert np.linalg.norm(r[k, m]) / np.linalg.norm(b[sample[k], m]) <= 1.02e-10, (k, d)
