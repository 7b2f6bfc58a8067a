"""GPU parity of the distillation path against the FP64 oracle: perambulators (full and domain,
diagonal and all sinks), quark loops (Sec. 2, Sec. 3.1-3.2) and the full, completely factorised
and subtracted correlators (Eqs. Cdisc, correlator_factorised, subtracted_correlator,
corr1-corr4).  Tolerances: perambulators and loops 1e-9 relative (Frobenius per source
timeslice / max over t), correlators 1e-8 relative to max |<L Lt>|, arithmetic-only stages at
FP64 round-off."""
import numpy as np
import pytest

from lqcd_inputs import colour_vectors
from oracle.dirac import WilsonClover
from oracle.distill import (laplace_eigs, perambulators, loops, disc_correlators,
                            profile_weights, conn_correlator, nr_estimator)
from tests.lattice_cases import SMALL, ROUGH, gauge

pytestmark = pytest.mark.gpu

pytest.importorskip("paper_2609_37049_b300")
from paper_2609_37049_b300 import Context, LqcdError, Stats, default_params, lqcd  # noqa: E402

GAMMAS = [5, 1, 2, 3, 0]  # gamma_5, gamma_x, gamma_y, gamma_z, 1


def tau_rel(a, b):
    return max(np.linalg.norm(a[k] - b[k]) / np.linalg.norm(b[k]) for k in range(b.shape[0]))


def _ctx(case, U):
    ctx = Context(case["dims"])
    ctx.gauge_upload(U, case["kappa"], case["c_sw"])
    ctx.set_domains(case["extents"])
    return ctx


def _gpu_tau(ctx, V, n_ev, t_src, mode, params=None, sinks=lqcd.LQCD_SINKS_DIAG):
    n_t = len(t_src)
    shape = (n_t, n_ev, 4, n_ev, 4) if sinks == lqcd.LQCD_SINKS_DIAG else \
        (n_t, V.shape[0], n_ev, 4, n_ev, 4)
    tau = np.zeros(shape, dtype=complex)
    st = Stats(1, 1)
    ctx.perambulator(np.ascontiguousarray(V), n_ev, list(t_src), tau, mode=mode, sinks=sinks,
                     params=params or default_params(), stats=st)
    assert st.max_true_resid <= 1e-10
    return tau


@pytest.fixture(scope="module")
def small_config():
    case = SMALL
    U = gauge(case, 1001)
    lam, V = laplace_eigs(U, case["n_ev"])
    op = WilsonClover(U, case["kappa"], case["c_sw"])
    T = case["dims"][3]
    tau_f = perambulators(op, V, range(T))
    tau_d = perambulators(op.restricted(case["extents"]), V, range(T))
    return dict(case=case, U=U, V=V, lam=lam, tau_f=tau_f, tau_d=tau_d)


@pytest.mark.parametrize("solver", ["bicgstab64", "mixed32"])
def test_perambulators_full_and_domain(small_config, solver):
    c = small_config
    case = c["case"]
    kw = dict(solver=lqcd.LQCD_SOLVER_BICGSTAB64) if solver == "bicgstab64" else \
        dict(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F32)
    ctx = _ctx(case, c["U"])
    T = case["dims"][3]
    tf = _gpu_tau(ctx, c["V"], case["n_ev"], range(T), lqcd.LQCD_MODE_FULL, default_params(**kw))
    td = _gpu_tau(ctx, c["V"], case["n_ev"], range(T), lqcd.LQCD_MODE_DOMAIN, default_params(**kw))
    assert tau_rel(tf, c["tau_f"]) < 1e-9
    assert tau_rel(td, c["tau_d"]) < 1e-9
    # the domain loops differ from the full ones (the correction dL of Sec. 2 is not zero)
    assert tau_rel(td, c["tau_f"]) > 1e-6


def test_loops_end_to_end(small_config):
    c = small_config
    case = c["case"]
    ctx = _ctx(case, c["U"])
    T, n_ev = case["dims"][3], case["n_ev"]
    tf = _gpu_tau(ctx, c["V"], n_ev, range(T), lqcd.LQCD_MODE_FULL)
    L = np.zeros((len(GAMMAS), T), dtype=complex)
    Lt = np.zeros_like(L)
    ctx.loops(tf, n_ev, T, GAMMAS, L, Lt)
    Lo, Lto = loops(c["tau_f"], GAMMAS)
    assert np.abs(L - Lo).max() / np.abs(Lo).max() < 1e-9
    assert np.abs(Lt - Lto).max() / np.abs(Lto).max() < 1e-9


def test_loops_arithmetic_with_profile_weights(small_config):
    """Loop contraction alone on the oracle's perambulators, with Gaussian-profile weights."""
    c = small_config
    case = c["case"]
    ctx = _ctx(case, c["U"])
    T, n_ev = case["dims"][3], case["n_ev"]
    w = profile_weights(c["lam"], 0.287)
    gids = list(range(16))
    L = np.zeros((16, T), dtype=complex)
    Lt = np.zeros_like(L)
    ctx.loops(np.ascontiguousarray(c["tau_f"]), n_ev, T, gids, L, Lt, weights=np.ascontiguousarray(w))
    Lo, Lto = loops(c["tau_f"], gids, weights=w)
    assert np.abs(L - Lo).max() <= 1e-13 * np.abs(Lo).max()
    assert np.abs(Lt - Lto).max() <= 1e-13 * np.abs(Lto).max()


def test_all_sinks_and_ragged_batches(small_config):
    c = small_config
    case = c["case"]
    ctx = _ctx(case, c["U"])
    n_ev = case["n_ev"]
    op = WilsonClover(c["U"], case["kappa"], case["c_sw"])
    ta = _gpu_tau(ctx, c["V"], n_ev, [2, 5], lqcd.LQCD_MODE_FULL, default_params(rhs_block=5),
                  sinks=lqcd.LQCD_SINKS_ALL)
    to = perambulators(op, c["V"], [2, 5], sinks="all")
    assert tau_rel(ta.reshape(2, -1), to.reshape(2, -1)) < 1e-9


def test_connected_correlator_and_nr_estimator(small_config):
    """Connected correlator from all-sink perambulators: the GPU contraction (gamma_5-hermiticity
    form) on the oracle's perambulators at FP64 round-off, end to end from the GPU's perambulators
    at 1e-9, a subset of sources column by column; and the noise-reduced estimator exactly."""
    c = small_config
    case = c["case"]
    ctx = _ctx(case, c["U"])
    T, n_ev = case["dims"][3], case["n_ev"]
    op = WilsonClover(c["U"], case["kappa"], case["c_sw"])
    t_all = list(range(T))
    to = perambulators(op, c["V"], t_all, sinks="all")
    gids = [5, 0, 1, 4, 10]
    Co, Co_avg = conn_correlator(to, t_all, gids)
    C = np.zeros((len(gids), T, T), complex)
    C_avg = np.zeros((len(gids), T), complex)
    ctx.conn_correlator(np.ascontiguousarray(to), n_ev, t_all, gids, C, C_avg)
    scale = np.abs(Co).max()
    assert np.abs(C - Co).max() <= 1e-13 * scale and np.abs(C_avg - Co_avg).max() <= 1e-13 * scale
    sub = [6, 1]
    Cs = np.zeros((len(gids), T, 2), complex)
    ctx.conn_correlator(np.ascontiguousarray(to[sub]), n_ev, sub, gids, Cs)
    assert np.abs(Cs - Co[:, :, sub]).max() <= 1e-13 * scale
    ta = _gpu_tau(ctx, c["V"], n_ev, t_all, lqcd.LQCD_MODE_FULL, sinks=lqcd.LQCD_SINKS_ALL)
    ctx.conn_correlator(ta, n_ev, t_all, gids, C, C_avg)
    assert np.abs(C - Co).max() <= 1e-9 * scale
    # noise-reduced estimator: two block sizes, the standard estimator at the shortest separations
    rng = np.random.default_rng(9)
    cplx = lambda *sh: rng.normal(size=sh) + 1j * rng.normal(size=sh)
    disc, dC = cplx(len(gids), T), cplx(2, len(gids), T)
    sel = [-1, -1, 0, 0, 1, 1, 1, 0]
    out = np.zeros((len(gids), T), complex)
    ctx.nr_estimator(np.ascontiguousarray(Co_avg), disc, dC, sel, out)
    assert np.array_equal(out, nr_estimator(Co_avg, disc, dC, sel))


def test_domain_mode_uneven_grouping(small_config):
    """Sources in only one domain (the other domains' systems are empty) and n_ev = 1."""
    c = small_config
    case = c["case"]
    ctx = _ctx(case, c["U"])
    td = _gpu_tau(ctx, c["V"][:, :1].copy(), 1, [1, 2, 6], lqcd.LQCD_MODE_DOMAIN)
    opd = WilsonClover(c["U"], case["kappa"], case["c_sw"]).restricted(case["extents"])
    to = perambulators(opd, c["V"][:, :1], [1, 2, 6])
    assert tau_rel(td, to) < 1e-9


def test_shifted_tiling_perambulators_and_correlators(small_config):
    """A tiling starting at t = 3 (domain [3, 5] wraps as t = 7, 0): domain-mode perambulators
    against the oracle's shifted D_Lambda, and the correlator validity table and subtracted
    correlator against the oracle on the same loops."""
    c = small_config
    case = c["case"]
    ext, t0 = [4, 4], 3
    ctx = Context(case["dims"])
    ctx.gauge_upload(c["U"], case["kappa"], case["c_sw"])
    ctx.set_domains(ext, t_start=t0)
    T, n_ev = case["dims"][3], case["n_ev"]
    opd = WilsonClover(c["U"], case["kappa"], case["c_sw"]).restricted(ext, t0)
    want = perambulators(opd, c["V"], range(T))
    td = _gpu_tau(ctx, c["V"], n_ev, range(T), lqcd.LQCD_MODE_DOMAIN)
    assert tau_rel(td, want) < 1e-9
    assert tau_rel(td, c["tau_d"]) > 1e-6  # differs from the unshifted tiling's perambulators
    L, Lt, Ld, Ltd = _random_loops(2, len(GAMMAS), T, 5)
    out = _gpu_corr(ctx, L, Lt, Ld, Ltd, True)
    o = disc_correlators(L, Lt, Ld, Ltd, ext, vev=True, t_start=t0)
    assert np.array_equal(out["valid"], o["valid"]) and np.array_equal(out["n_valid"], o["n_valid"])
    assert np.abs(out["dC"] - o["dC"]).max() <= 1e-13 * np.abs(o["C"]).max()
    assert np.abs(out["dC_avg"] - o["dC_avg"]).max() <= 1e-13 * np.abs(o["C"]).max()


def test_colour_vector_sources_rough_field():
    case = ROUGH
    U = gauge(case, 3003)
    V = colour_vectors(case["dims"], 3, 3004)
    ctx = _ctx(case, U)
    kw = dict(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F16)
    td = _gpu_tau(ctx, V, 3, [0, 5], lqcd.LQCD_MODE_DOMAIN, default_params(**kw))
    opd = WilsonClover(U, case["kappa"], case["c_sw"]).restricted(case["extents"])
    assert tau_rel(td, perambulators(opd, V, [0, 5])) < 1e-9


def _random_loops(n_cfg, n_g, T, seed):
    rng = np.random.default_rng(seed)
    c = lambda: rng.normal(size=(n_cfg, n_g, T)) + 1j * rng.normal(size=(n_cfg, n_g, T))
    return c(), c(), c(), c()


def _gpu_corr(ctx, L, Lt, Ld, Ltd, vev, terms=True):
    n_g, T = L.shape[1], L.shape[2]
    out = dict(C=np.zeros((n_g, T, T), complex), Cdd=np.zeros((n_g, T, T), complex),
               dC=np.zeros((n_g, T, T), complex), C_avg=np.zeros((n_g, T), complex),
               dC_avg=np.zeros((n_g, T), complex), valid=np.zeros((T, T), np.int32),
               n_valid=np.zeros(T, np.int32))
    tm = np.zeros((4, n_g, T, T), complex) if terms else None
    ctx.disc_correlator(L, Lt, Ld, Ltd, vev, out, terms=tm)
    out["terms"] = tm
    return out


@pytest.mark.parametrize("vev", [True, False])
def test_correlator_arithmetic(vev):
    T = 8
    ctx = Context((4, 4, 4, T))
    ctx.set_domains([3, 5])
    L, Lt, Ld, Ltd = _random_loops(5, 3, T, 1)
    g = _gpu_corr(ctx, L, Lt, Ld, Ltd, vev)
    o = disc_correlators(L, Lt, Ld, Ltd, [3, 5], vev=vev)
    for k in ("C", "C_dd", "dC", "C_avg", "dC_avg", "terms"):
        gk = g["Cdd" if k == "C_dd" else k]
        assert np.abs(gk - o[k]).max() <= 1e-13 * np.abs(o["C"]).max(), k
    assert np.array_equal(g["valid"], o["valid"]) and np.array_equal(g["n_valid"], o["n_valid"])


def test_correlator_rejects_vev_with_one_config():
    ctx = Context((4, 4, 4, 8))
    L = np.zeros((1, 1, 8), complex)
    with pytest.raises(lqcd.LqcdError):
        _gpu_corr(ctx, L, L, L, L, True)


def test_full_estimator_two_configs():
    """Perambulators -> loops -> C, C_LL, dC over two gauge configurations, end to end."""
    case = SMALL
    T, n_ev, ext = case["dims"][3], case["n_ev"], case["extents"]
    gids = [5, 0]
    Lg, Ltg, Ldg, Ltdg, Lo_, Lto_, Ldo_, Ltdo_ = ([] for _ in range(8))
    for seed in (1001, 1002):
        U = gauge(case, seed)
        lam, V = laplace_eigs(U, n_ev)
        ctx = _ctx(case, U)
        for mode, outs in ((lqcd.LQCD_MODE_FULL, (Lg, Ltg)), (lqcd.LQCD_MODE_DOMAIN, (Ldg, Ltdg))):
            tau = _gpu_tau(ctx, V, n_ev, range(T), mode)
            L = np.zeros((len(gids), T), complex)
            Lt = np.zeros_like(L)
            ctx.loops(tau, n_ev, T, gids, L, Lt)
            outs[0].append(L)
            outs[1].append(Lt)
        op = WilsonClover(U, case["kappa"], case["c_sw"])
        for o, outs in ((op, (Lo_, Lto_)), (op.restricted(ext), (Ldo_, Ltdo_))):
            L, Lt = loops(perambulators(o, V, range(T)), gids)
            outs[0].append(L)
            outs[1].append(Lt)
    ctx = Context(case["dims"])
    ctx.set_domains(ext)
    arr = lambda x: np.ascontiguousarray(np.array(x))
    g = _gpu_corr(ctx, arr(Lg), arr(Ltg), arr(Ldg), arr(Ltdg), True)
    o = disc_correlators(arr(Lo_), arr(Lto_), arr(Ldo_), arr(Ltdo_), ext, vev=True)
    scale = np.abs(np.einsum("cgx,cgy->gxy", arr(Lo_), arr(Lto_)) / 2).max()
    for k, ko in (("C", "C"), ("Cdd", "C_dd"), ("dC", "dC"), ("dC_avg", "dC_avg")):
        assert np.abs(g[k] - o[ko]).max() <= 1e-8 * scale, k


def test_open_bc_shifted_tiling_window_end_to_end():
    """The paper's geometry (Sec. 3: open time boundaries, averages over source and sink in the
    bulk; regions placed around the chosen timeslices, Fig. 1): open-boundary operator, a tiling
    starting at t = 2 whose last domain wraps, perambulators (full and domain) -> loops -> C, C_LL,
    dC over two configurations -> bulk-window averages, each stage against the oracle."""
    from oracle.dirac import BC_OPEN
    from oracle.distill import window_average
    case = SMALL
    T, n_ev = case["dims"][3], case["n_ev"]
    ext, t0 = [3, 5], 2
    gids = [5, 0]
    gpu = {k: [] for k in ("L", "Lt", "Ld", "Ltd")}
    ora = {k: [] for k in ("L", "Lt", "Ld", "Ltd")}
    for seed in (1011, 1012):
        U = gauge(case, seed)
        lam, V = laplace_eigs(U, n_ev)
        ctx = Context(case["dims"], bc_t=lqcd.LQCD_BC_OPEN)
        ctx.gauge_upload(U, case["kappa"], case["c_sw"])
        ctx.set_domains(ext, t_start=t0)
        op = WilsonClover(U, case["kappa"], case["c_sw"], bc_t=BC_OPEN)
        for mode, o, (a, b) in ((lqcd.LQCD_MODE_FULL, op, ("L", "Lt")),
                                (lqcd.LQCD_MODE_DOMAIN, op.restricted(ext, t0), ("Ld", "Ltd"))):
            tau = _gpu_tau(ctx, V, n_ev, range(T), mode)
            want = perambulators(o, V, range(T))
            assert tau_rel(tau, want) < 1e-9
            L, Lt = np.zeros((len(gids), T), complex), np.zeros((len(gids), T), complex)
            ctx.loops(tau, n_ev, T, gids, L, Lt)
            Lo, Lto = loops(want, gids)
            assert np.abs(L - Lo).max() <= 1e-9 * np.abs(Lo).max()
            gpu[a].append(L)
            gpu[b].append(Lt)
            ora[a].append(Lo)
            ora[b].append(Lto)
    arr = lambda x: np.ascontiguousarray(np.array(x))
    g = _gpu_corr(ctx, arr(gpu["L"]), arr(gpu["Lt"]), arr(gpu["Ld"]), arr(gpu["Ltd"]), True)
    o = disc_correlators(arr(ora["L"]), arr(ora["Lt"]), arr(ora["Ld"]), arr(ora["Ltd"]), ext, vev=True, t_start=t0)
    scale = np.abs(np.einsum("cgx,cgy->gxy", arr(ora["L"]), arr(ora["Lt"])) / 2).max()
    for k, ko in (("C", "C"), ("Cdd", "C_dd"), ("dC", "dC")):
        assert np.abs(g[k] - o[ko]).max() <= 1e-8 * scale, k
    assert np.array_equal(g["valid"], o["valid"])
    t_lo, t_hi = 1, 6
    out = dict(C_avg=np.zeros((len(gids), T), complex), dC_avg=np.zeros((len(gids), T), complex),
               n_pairs=np.zeros(T, np.int32), n_valid=np.zeros(T, np.int32))
    ctx.window_average(g["C"], g["dC"], g["valid"], t_lo, t_hi, out)
    w = window_average(o["C"], o["dC"], o["valid"], t_lo, t_hi)
    assert np.array_equal(out["n_pairs"], w["n_pairs"]) and np.array_equal(out["n_valid"], w["n_valid"])
    for k in ("C_avg", "dC_avg"):
        assert np.abs(out[k] - w[k]).max() <= 1e-8 * scale, k
    # the arithmetic alone, on the oracle's correlators: FP64 round-off
    ctx.window_average(np.ascontiguousarray(o["C"]), np.ascontiguousarray(o["dC"]),
                       np.ascontiguousarray(o["valid"].astype(np.int32)), t_lo, t_hi, out)
    for k in ("C_avg", "dC_avg"):
        assert np.abs(out[k] - w[k]).max() <= 1e-13 * scale, k
    with pytest.raises(LqcdError):
        ctx.window_average(g["C"], g["dC"], g["valid"], 5, 4, out)


@pytest.mark.parametrize("mode", [lqcd.LQCD_MODE_FULL, lqcd.LQCD_MODE_DOMAIN])
def test_double_float_projection_matches_fp64(small_config, mode):
    """The projection tau = V^dag X in double-float arithmetic on the FP32 pipe (the default) agrees
    with the native FP64 GEMM to 1e-12 and with the oracle to 1e-9."""
    c = small_config
    case = c["case"]
    ctx = _ctx(case, c["U"])
    T, n_ev = case["dims"][3], case["n_ev"]
    kw = dict(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F32)
    t_df = _gpu_tau(ctx, c["V"], n_ev, range(T), mode, default_params(projection=0, **kw))
    t_64 = _gpu_tau(ctx, c["V"], n_ev, range(T), mode, default_params(projection=1, **kw))
    assert tau_rel(t_df, t_64) < 1e-12
    assert tau_rel(t_df, c["tau_f"] if mode == lqcd.LQCD_MODE_FULL else c["tau_d"]) < 1e-9
