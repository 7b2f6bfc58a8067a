"""Device-side solver loops and two batches in flight.

With use_graph = 1 every batch's whole solve (defect-correction cycles and inner iterations) is one
CUDA graph whose loops run on the device; with pipeline = 2 two batches are in flight on two
streams.  Both change only where the host waits, not the arithmetic, so the solutions must equal
the host-driven loop's bit for bit, with the same iteration counts, for every solver, full and
domain operators, and at the max_iter / max_outer limits (NOT_CONVERGED with the same last
iterate).  Perambulators computed with two batches in flight match the oracle at 1e-9.
"""
import numpy as np
import pytest

from lqcd_inputs import random_spinors
from oracle.dirac import WilsonClover
from oracle.distill import laplace_eigs, perambulators
from tests.lattice_cases import SMALL, ROUGH, gauge, per_domain_resid

pytestmark = pytest.mark.gpu

pytest.importorskip("paper_2609_37049_b300")
from paper_2609_37049_b300 import Context, LqcdError, Stats, default_params, lqcd  # noqa: E402

SOLVERS = {
    "bicgstab64": dict(solver=lqcd.LQCD_SOLVER_BICGSTAB64),
    "mixed32": dict(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F32),
    "fgcr_mr16": dict(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F16, precond_iters=3),
}


def _ctx(case, U):
    ctx = Context(case["dims"])
    ctx.gauge_upload(U, case["kappa"], case["c_sw"])
    ctx.set_domains(case["extents"])
    return ctx


def _solve(ctx, b, domain, allow=False, **kw):
    x = np.zeros_like(b)
    nseg = len(ctx.extents) if domain else 1
    st = Stats(b.shape[0], nseg)
    rc = ctx.solve(b, x, default_params(**kw), domain=domain, stats=st, allow_not_converged=allow)
    return x, st, rc


@pytest.mark.parametrize("domain", [False, True])
@pytest.mark.parametrize("name", sorted(SOLVERS))
def test_device_loops_equal_host_loop(name, domain):
    case = ROUGH
    U = gauge(case, 1401)
    ctx = _ctx(case, U)
    b = random_spinors(case["dims"], 6, 1402)
    kw = dict(SOLVERS[name], rhs_block=2)
    xh, sh, _ = _solve(ctx, b, domain, use_graph=0, **kw)
    xd, sd, _ = _solve(ctx, b, domain, use_graph=1, **kw)
    xp, sp, _ = _solve(ctx, b, domain, use_graph=1, pipeline=2, **kw)
    assert sh.device_loops == 0 and sd.device_loops == 3 and sp.device_loops == 3
    assert np.array_equal(xh, xd) and np.array_equal(xh, xp)
    assert np.array_equal(sh.iters, sd.iters) and np.array_equal(sh.iters, sp.iters)
    assert np.array_equal(sh.true_resid, sd.true_resid) and sh.outer_cycles == sd.outer_cycles
    assert sh.dslash_calls == sd.dslash_calls
    op = WilsonClover(U, case["kappa"], case["c_sw"])
    if domain:
        op = op.restricted(case["extents"])
    r = b - op.apply(xd)
    ext = case["extents"] if domain else [case["dims"][3]]
    assert per_domain_resid(b, r, ext).max() <= 1.02e-10


@pytest.mark.parametrize("limit", [dict(max_iter=8, check_every=8), dict(max_outer=1)])
def test_device_loops_stop_at_the_limits(limit):
    case = ROUGH
    U = gauge(case, 1403)
    ctx = _ctx(case, U)
    b = random_spinors(case["dims"], 2, 1404)
    kw = dict(SOLVERS["mixed32"], rhs_block=2, **limit)
    res = {}
    for g in (0, 1):
        x = np.zeros_like(b)
        st = Stats(2, 1)
        with pytest.raises(LqcdError) as ei:
            ctx.solve(b, x, default_params(use_graph=g, **kw), stats=st)
        assert ei.value.code == lqcd.LQCD_ERR_NOT_CONVERGED
        res[g] = (x, st.iters.copy(), st.true_resid.copy(), st.device_loops)
    assert res[0][3] == 0 and res[1][3] == 1
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert np.array_equal(res[0][2], res[1][2]) and res[1][2].max() > 1e-10


def test_pipelined_perambulators_match_the_oracle():
    case = SMALL
    U = gauge(case, 1001)
    lam, V = laplace_eigs(U, case["n_ev"])
    T, n_ev = case["dims"][3], case["n_ev"]
    L3 = case["dims"][0] * case["dims"][1] * case["dims"][2]
    Vf = np.ascontiguousarray(V.reshape(T, n_ev, L3, 3))
    ctx = _ctx(case, U)
    op = WilsonClover(U, case["kappa"], case["c_sw"])
    t_src = [0, 3, 5]
    for mode, o in ((lqcd.LQCD_MODE_FULL, op), (lqcd.LQCD_MODE_DOMAIN, op.restricted(case["extents"]))):
        taus = {}
        for pipe in (1, 2):
            tau = np.zeros((len(t_src), n_ev, 4, n_ev, 4), dtype=complex)
            st = Stats(1, 1)
            ctx.perambulator(Vf, n_ev, t_src, tau, mode=mode, stats=st,
                             params=default_params(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F32,
                                                   rhs_block=4, pipeline=pipe))
            assert st.max_true_resid <= 1e-10 and st.device_loops > 0
            taus[pipe] = tau
        assert np.array_equal(taus[1], taus[2])
        want = perambulators(o, V, t_src)
        for k in range(len(t_src)):
            assert np.linalg.norm(taus[2][k] - want[k]) / np.linalg.norm(want[k]) < 1e-9


def test_release_workspace_then_solve_again():
    """lqcd_release_workspace frees the work vectors and the graphs captured on them; the next solve
    allocates and captures them again and returns the same solution bit for bit."""
    case = ROUGH
    U = gauge(case, 1405)
    ctx = _ctx(case, U)
    b = random_spinors(case["dims"], 4, 1406)
    kw = dict(SOLVERS["mixed32"], rhs_block=4, use_graph=1)
    x1, s1, _ = _solve(ctx, b, False, **kw)
    ctx.release_workspace()
    x2, s2, _ = _solve(ctx, b, False, **kw)
    assert np.array_equal(x1, x2) and np.array_equal(s1.iters, s2.iters) and s2.device_loops == s1.device_loops
