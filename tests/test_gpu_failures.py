"""Error paths injected on the host (nothing here faults, traps or hangs the GPU), the re-upload of
a gauge field with a new kappa, and the column-range / per-source-vector perambulator entry point.

* a NaN in one right-hand side of a solve returns LQCD_ERR_NAN, reports that system's true
  residual as NaN, and still solves and writes every other right-hand side to 1e-10 (checked with
  the oracle's operator);
* a NaN or Inf link makes lqcd_gauge_upload return LQCD_ERR_NAN (its clover block has no inverse)
  and leaves the context without a usable field (solves return LQCD_ERR_STATE);
* a context re-uploaded with another kappa solves exactly as a fresh context with that kappa (the
  solver graphs captured with the old kappa are dropped);
* lqcd_perambulator_cols writes the perambulator columns (Sec. 3.1) of the requested source
  vectors and leaves every other entry untouched, with the colour vectors of every timeslice or
  only of the source timeslices (LQCD_SINKS_DIAG_SRCV).
"""
import numpy as np
import pytest

from lqcd_inputs import random_spinors
from oracle.dirac import WilsonClover
from oracle.distill import laplace_eigs, perambulators
from tests.lattice_cases import SMALL, ROUGH, gauge, per_domain_resid

pytestmark = pytest.mark.gpu

pytest.importorskip("paper_2609_37049_b300")
import torch  # noqa: E402
from paper_2609_37049_b300 import Context, LqcdError, Stats, default_params, lqcd  # noqa: E402


def _ctx(case, U, kappa=None):
    ctx = Context(case["dims"])
    ctx.gauge_upload(U, case["kappa"] if kappa is None else kappa, case["c_sw"])
    ctx.set_domains(case["extents"])
    return ctx


@pytest.mark.parametrize("domain", [False, True])
@pytest.mark.parametrize("solver", [lqcd.LQCD_SOLVER_BICGSTAB64, lqcd.LQCD_SOLVER_MIXED])
def test_nan_source_reports_nan_and_keeps_the_other_rhs(domain, solver):
    case = ROUGH
    U = gauge(case, 1301)
    ctx = _ctx(case, U)
    b = random_spinors(case["dims"], 3, 1302)
    b[1, 2, 1, 0, 3, 2, 1] = np.nan  # one site of right-hand side 1 (domain 0 of the [4, 4] tiling)
    x = np.zeros_like(b)
    nseg = len(case["extents"]) if domain else 1
    st = Stats(3, nseg)
    with pytest.raises(LqcdError) as ei:
        ctx.solve(b, x, default_params(solver=solver, inner_prec=lqcd.LQCD_PREC_F32), domain=domain, stats=st)
    assert ei.value.code == lqcd.LQCD_ERR_NAN
    res = st.true_resid.reshape(3, nseg)
    assert np.isnan(res[1, 0])
    op = WilsonClover(U, case["kappa"], case["c_sw"])
    if domain:
        op = op.restricted(case["extents"])
    for r in (0, 2):
        assert np.all(np.isfinite(x[r]))
        rr = b[r] - op.apply(x[r:r + 1])[0]
        if domain:
            assert per_domain_resid(b[r:r + 1], rr[None], case["extents"]).max() <= 1.01e-10
        else:
            assert np.linalg.norm(rr) / np.linalg.norm(b[r]) <= 1.01e-10
        assert np.all(res[r] <= 1e-10)
    if domain:  # the other domain of the poisoned right-hand side is an independent system
        assert res[1, 1] <= 1e-10


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_corrupted_link_rejected_at_upload(bad):
    case = SMALL
    U = gauge(case, 1303)
    ctx = Context(case["dims"])
    ctx.gauge_upload(U, case["kappa"], case["c_sw"])
    Ub = U.copy()
    Ub[3, 1, 2, 0, 1, 0, 2] = bad  # one link entry, host side
    with pytest.raises(LqcdError) as ei:
        ctx.gauge_upload(Ub, case["kappa"], case["c_sw"])
    assert ei.value.code == lqcd.LQCD_ERR_NAN
    b = random_spinors(case["dims"], 1, 1304)
    with pytest.raises(LqcdError) as ei:
        ctx.solve(b, np.zeros_like(b))
    assert ei.value.code == lqcd.LQCD_ERR_STATE
    # a clean upload makes the context usable again
    ctx.gauge_upload(U, case["kappa"], case["c_sw"])
    ctx.solve(b, np.zeros_like(b))


@pytest.mark.parametrize("solver", [lqcd.LQCD_SOLVER_MIXED, lqcd.LQCD_SOLVER_BICGSTAB64])
def test_kappa_reupload_matches_a_fresh_context(solver):
    case = ROUGH
    U = gauge(case, 1305)
    b = random_spinors(case["dims"], 2, 1306)
    p = default_params(solver=solver, inner_prec=lqcd.LQCD_PREC_F32, use_graph=1)
    k2 = 0.118
    ctx = _ctx(case, U)
    x1 = np.zeros_like(b)
    ctx.solve(b, x1, p)  # captures graphs with the first kappa
    ctx.gauge_upload(U, k2, case["c_sw"])
    x2, st2 = np.zeros_like(b), Stats(2, 1)
    ctx.solve(b, x2, p, stats=st2)
    fresh = _ctx(case, U, kappa=k2)
    x3, st3 = np.zeros_like(b), Stats(2, 1)
    fresh.solve(b, x3, p, stats=st3)
    assert np.array_equal(st2.iters, st3.iters)
    assert np.array_equal(x2, x3)
    op = WilsonClover(U, k2, case["c_sw"])
    r = b - op.apply(x2)
    assert max(np.linalg.norm(r[k]) / np.linalg.norm(b[k]) for k in range(2)) <= 1.01e-10
    assert np.abs(x1 - x2).max() > 1e-3  # the operator did change


@pytest.fixture(scope="module")
def cols_case():
    case = SMALL
    U = gauge(case, 1001)
    lam, V = laplace_eigs(U, case["n_ev"])
    op = WilsonClover(U, case["kappa"], case["c_sw"])
    t_src = [1, 6]
    return dict(case=case, U=U, V=V, t_src=t_src, tau_f=perambulators(op, V, t_src),
                tau_d=perambulators(op.restricted(case["extents"]), V, t_src))


@pytest.mark.parametrize("where", ["host", "device"])
@pytest.mark.parametrize("mode", [lqcd.LQCD_MODE_FULL, lqcd.LQCD_MODE_DOMAIN])
@pytest.mark.parametrize("srcv", [False, True])
def test_perambulator_columns(cols_case, where, mode, srcv):
    c = cols_case
    case, t_src = c["case"], c["t_src"]
    n_ev = case["n_ev"]
    T, L3 = case["dims"][3], case["dims"][0] * case["dims"][1] * case["dims"][2]
    ctx = _ctx(case, c["U"])
    Vall = np.ascontiguousarray(c["V"].reshape(T, n_ev, L3, 3))
    Vin = np.ascontiguousarray(Vall[t_src]) if srcv else Vall
    sinks = lqcd.LQCD_SINKS_DIAG_SRCV if srcv else lqcd.LQCD_SINKS_DIAG
    ref = c["tau_f"] if mode == lqcd.LQCD_MODE_FULL else c["tau_d"]
    sentinel = 7.0 - 3.0j
    tau = np.full((len(t_src), n_ev, 4, n_ev, 4), sentinel, dtype=complex)
    j0, nj = 1, 2
    p = default_params(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F32, rhs_block=3)
    if where == "device":
        Vd, td = torch.from_numpy(Vin).cuda(), torch.from_numpy(tau).cuda()
        ctx.perambulator_cols(Vd, n_ev, t_src, td, j0, nj, mode=mode, sinks=sinks, params=p)
        tau = td.cpu().numpy()
    else:
        ctx.perambulator_cols(Vin, n_ev, t_src, tau, j0, nj, mode=mode, sinks=sinks, params=p)
    cols = tau[:, :, :, j0:j0 + nj, :]
    for k in range(len(t_src)):
        r = ref[k][:, :, j0:j0 + nj, :]
        assert np.linalg.norm(cols[k] - r) / np.linalg.norm(r) < 1e-9
    untouched = np.ones(n_ev, dtype=bool)
    untouched[j0:j0 + nj] = False
    assert np.all(tau[:, :, :, untouched, :] == sentinel)


def test_perambulator_columns_rejects_bad_ranges(cols_case):
    c = cols_case
    case = c["case"]
    n_ev = case["n_ev"]
    T, L3 = case["dims"][3], case["dims"][0] * case["dims"][1] * case["dims"][2]
    ctx = _ctx(case, c["U"])
    V = np.ascontiguousarray(c["V"].reshape(T, n_ev, L3, 3))
    tau = np.zeros((1, n_ev, 4, n_ev, 4), dtype=complex)
    for j0, nj in ((-1, 1), (0, 0), (n_ev - 1, 2)):
        with pytest.raises(LqcdError) as ei:
            ctx.perambulator_cols(V, n_ev, [0], tau, j0, nj)
        assert ei.value.code == lqcd.LQCD_ERR_INVALID_ARG
    with pytest.raises(LqcdError) as ei:  # a repeated timeslice with per-source vectors
        ctx.perambulator_cols(np.ascontiguousarray(V[[2, 2]]), n_ev, [2, 2], np.zeros((2,) + tau.shape[1:], complex),
                              0, 1, sinks=lqcd.LQCD_SINKS_DIAG_SRCV)
    assert ei.value.code == lqcd.LQCD_ERR_INVALID_ARG
