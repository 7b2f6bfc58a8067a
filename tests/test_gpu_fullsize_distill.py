"""Full-size parity of the distillation path (Sec. 3.1 perambulators and loops) in the launch
configurations bench.py times.

16^3 x 32 mixed-precision workload (eps 0.5, kappa 0.125, c_sw 1.6, eight domains of 4; 64-RHS
blocks, staged-links FP32 dslash): perambulator columns of the full operator (source timeslice 0)
and of the domain operator (multi-site sources on the timeslices 0, 4, ..., 28), and the loops
they give, against the oracle's values written by tests/golden/make_fullsize_golden.py (CGNR to
true residual 1e-12; nothing there comes from the CUDA path), at 1e-9; the GPU Laplacian
eigenvalues of one timeslice against the oracle's dense eigensolve; the network forward pass and
gradients on one full-size sample against oracle/nn.py.

48^3 x 96 scale workload (eps 0.6, kappa 0.126, c_sw 1.7, 24 domains of 4, 16-RHS blocks): the
oracle cannot solve at this size, so it checks what it can compute one site at a time
(oracle.dirac.apply_at_sites): the FP64 operator and the domain operator element by element at
sampled sites, and the true residual of a mixed solve at sampled sites (each |r(x)| <= ||r||);
the bench's perambulator call is checked against the plain FP64 solver on the same columns and
by the gamma_5-hermiticity of its diagonal block.
"""
import json
import os

import numpy as np
import pytest

from lqcd_inputs import colour_vectors, gauge_field, random_spinors
from oracle import nn
from oracle.dirac import BC_ANTIPERIODIC, apply_at_sites, fermion_links
from oracle.distill import laplacian3d, loops as oracle_loops

pytestmark = pytest.mark.gpu

pytest.importorskip("paper_2609_37049_b300")
import torch  # noqa: E402
from paper_2609_37049_b300 import Context, Stats, default_params, lqcd  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "fullsize_16x16x16x32.json")
GAMMAS = [5, 0, 1]


def _golden():
    with open(GOLDEN) as f:
        g = json.load(f)
    for key in ("tau_full", "tau_dom"):
        a = np.array(g[key]["values"], dtype=float)
        g[key]["array"] = (a[:, 0] + 1j * a[:, 1]).reshape(g[key]["shape"])
    return g


@pytest.fixture(scope="module")
def mixed():
    g = _golden()
    w = g["workload"]
    dims = tuple(w["dims"])
    U = gauge_field(dims, w["eps"], w["gauge_seed"])
    ctx = Context(dims)
    ctx.gauge_upload(U, w["kappa"], w["c_sw"])
    ctx.set_domains([4] * 8)
    ctx.set_dslash_variant(lqcd.LQCD_PREC_F32, 64, 3)
    ctx.set_dslash_variant(lqcd.LQCD_PREC_F64, 64, 1)
    t_dom = g["tau_dom"]["t"]
    L3 = dims[0] * dims[1] * dims[2]
    V = colour_vectors(dims, w["n_ev"], w["cv_seed"], timeslices=t_dom).reshape(len(t_dom), w["n_ev"], L3, 3)
    return dict(g=g, U=U, ctx=ctx, V=np.ascontiguousarray(V), dims=dims, n_ev=w["n_ev"])


def _cols(m, mode):
    """GPU perambulator columns of the sampled source vectors, 64-RHS blocks (16 vectors x 4 spins)."""
    g, ctx, n_ev = m["g"], m["ctx"], m["n_ev"]
    key = "tau_full" if mode == lqcd.LQCD_MODE_FULL else "tau_dom"
    t_src = [g[key]["t"]] if mode == lqcd.LQCD_MODE_FULL else g[key]["t"]
    V = m["V"][:1] if mode == lqcd.LQCD_MODE_FULL else m["V"]
    tau = np.zeros((len(t_src), n_ev, 4, n_ev, 4), dtype=complex)
    p = default_params(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F32, rhs_block=64)
    for j in g[key]["j"]:
        st = Stats(1, 1)
        j0 = (j // 16) * 16
        ctx.perambulator_cols(V, n_ev, t_src, tau, j0, 16, mode=mode, sinks=lqcd.LQCD_SINKS_DIAG_SRCV, params=p,
                              stats=st)
        assert st.max_true_resid <= 1e-10
    return tau, g[key]


@pytest.mark.parametrize("mode", [lqcd.LQCD_MODE_FULL, lqcd.LQCD_MODE_DOMAIN])
def test_perambulator_columns_and_loops_16x32(mixed, mode):
    tau, ref = _cols(mixed, mode)
    J = ref["j"]
    want = ref["array"] if mode == lqcd.LQCD_MODE_DOMAIN else ref["array"][None]
    got = tau[:, :, :, J, :]
    for k in range(want.shape[0]):
        err = np.linalg.norm(got[k] - want[k]) / np.linalg.norm(want[k])
        assert err < 1e-9, (k, err)
    # loops of the sampled vectors: weights select i in J, so only the golden columns enter
    n_ev, n_t = mixed["n_ev"], want.shape[0]
    w = np.zeros((n_t, n_ev))
    w[:, J] = 1.0
    L, Lt = np.zeros((len(GAMMAS), n_t), complex), np.zeros((len(GAMMAS), n_t), complex)
    mixed["ctx"].loops(tau, n_ev, n_t, GAMMAS, L, Lt, weights=w)
    full_ref = np.zeros((n_t, n_ev, 4, n_ev, 4), dtype=complex)
    full_ref[:, :, :, J, :] = want
    Lo, Lto = oracle_loops(full_ref, GAMMAS, weights=w)
    assert np.abs(L - Lo).max() <= 1e-9 * np.abs(Lo).max()
    assert np.abs(Lt - Lto).max() <= 1e-9 * np.abs(Lto).max()


def test_laplace_eigenpairs_16x32(mixed):
    """The GPU eigensolver (bench sources of the 16^3 x 32 workload) on timeslice 0 against the
    oracle's dense eigensolve (eigenvalues), and its vectors against the oracle's Laplacian."""
    g, dims = mixed["g"], mixed["dims"]
    n_ev = g["eig_lambda"]["n_ev"]
    T, L3 = dims[3], dims[0] * dims[1] * dims[2]
    Vd = torch.zeros((T, n_ev, L3, 3), dtype=torch.complex128, device="cuda")
    lam = torch.zeros((T, n_ev), dtype=torch.float64, device="cuda")
    mixed["ctx"].laplace_eigs(n_ev, Vd, lam)
    lam0 = lam[0].cpu().numpy()
    lo = np.array(g["eig_lambda"]["values"])
    assert np.abs(lam0 - lo).max() < 1e-9 * max(1.0, np.abs(lo).max())
    V0 = Vd[0].cpu().numpy().reshape(n_ev, dims[2], dims[1], dims[0], 3)
    res = laplacian3d(mixed["U"], 0, V0) - lam0[:, None, None, None, None] * V0
    assert np.abs(res).max() < 1e-8
    X = V0.reshape(n_ev, -1)
    assert np.abs(X @ X.conj().T - np.eye(n_ev)).max() < 1e-12


def test_network_forward_and_gradient_16x32(mixed):
    U, dims, ctx = mixed["U"], mixed["dims"], mixed["ctx"]
    Ws = [np.asarray(W, np.complex64).astype(np.complex128) for W in nn.init_weights(6, 0.3)]
    ctx.nn_set_weights(Ws)
    rng = np.random.default_rng(5)
    shape = (1, dims[3], dims[2], dims[1], dims[0], 4, 3)
    x = (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)
    tgt = (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)
    out = np.zeros_like(x)
    ctx.nn_apply(x, out)
    Ue = fermion_links(U, BC_ANTIPERIODIC)
    ref = nn.forward(Ws, Ue, x.astype(np.complex128))[-1]
    assert np.abs(out - ref).max() / np.abs(ref).max() < 2e-5
    L, G = ctx.nn_loss_grad(x, tgt)
    Lo, Go = nn.loss_and_grad(Ws, Ue, x.astype(np.complex128), tgt.astype(np.complex128),
                              np.ones(shape[1:5]))
    assert abs(L - Lo) < 1e-5 * Lo
    for g_, go in zip(G, Go):
        assert np.abs(g_ - go).max() < 1e-4 * np.abs(go).max()


# ----------------------------------------------------------------------------- 48^3 x 96
SCALE = dict(dims=(48, 48, 48, 96), eps=0.6, kappa=0.126, c_sw=1.7, n_ev=128, extents=[4] * 24,
             gauge_seed=5001, cv_seed=5002, rhs_block=16)


def _sample_sites(dims, n, seed):
    rng = np.random.default_rng(seed)
    pts = [tuple(int(rng.integers(0, L)) for L in dims) for _ in range(n)]
    Lx, Ly, Lz, Lt = dims
    # the time boundary, domain cuts and the spatial wrap
    pts += [(0, 0, 0, 0), (Lx - 1, Ly - 1, Lz - 1, Lt - 1), (3, 5, 7, 3), (3, 5, 7, 4), (Lx - 1, 0, 5, 47)]
    return pts


@pytest.fixture(scope="module")
def scale():
    s = SCALE
    dims = s["dims"]
    U = gauge_field(dims, s["eps"], s["gauge_seed"])
    ctx = Context(dims)
    ctx.gauge_upload(U, s["kappa"], s["c_sw"])
    ctx.set_domains(s["extents"])
    from paper_2609_37049_b300 import autotune
    autotune.tune(ctx, precisions=(lqcd.LQCD_PREC_F32, lqcd.LQCD_PREC_F64, lqcd.LQCD_PREC_DF), blocks=(s["rhs_block"],))
    return dict(U=U, ctx=ctx, dims=dims)


@pytest.mark.parametrize("domain", [False, True])
def test_scale_operator_at_sampled_sites(scale, domain):
    U, ctx, dims = scale["U"], scale["ctx"], scale["dims"]
    psi = random_spinors(dims, 1, 5101)
    out = np.zeros_like(psi)
    ctx.dirac_apply(psi, out, domain_restricted=domain)
    sites = _sample_sites(dims, 64, 5102)
    ref = apply_at_sites(U, SCALE["kappa"], SCALE["c_sw"], psi[0], sites,
                         extents=SCALE["extents"] if domain else None)
    got = np.array([out[0, t, z, y, x] for (x, y, z, t) in sites])
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()


def test_scale_solve_residual_at_sampled_sites(scale):
    """A mixed solve of 8 sources (colour vectors 0, 1 of timeslice 0, four spins): at sampled
    sites the oracle's residual b(x) - (D x)(x) is below 1e-10 ||b|| (a bound on every site)."""
    U, ctx, dims = scale["U"], scale["ctx"], scale["dims"]
    Lx, Ly, Lz, Lt = dims
    V0 = colour_vectors(dims, SCALE["n_ev"], SCALE["cv_seed"], timeslices=[0])[0]
    b = torch.zeros((8, Lt, Lz, Ly, Lx, 4, 3), dtype=torch.complex128, device="cuda")
    for j in range(2):
        v = torch.from_numpy(V0[j]).cuda()
        for beta in range(4):
            b[4 * j + beta, 0, :, :, :, beta, :] = v
    x = torch.zeros_like(b)
    st = Stats(8, 1)
    ctx.solve(b, x, default_params(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F32, rhs_block=8),
              stats=st)
    assert st.max_true_resid <= 1e-10
    sites = _sample_sites(dims, 24, 5103) + [(x_, 7, 9, 0) for x_ in range(0, Lx, 6)] + [(5, 5, 5, 1), (5, 5, 5, 95)]
    for r in (0, 5):
        xr = x[r].cpu().numpy()
        br = b[r].cpu().numpy()
        Dx = apply_at_sites(U, SCALE["kappa"], SCALE["c_sw"], xr, sites)
        res = np.array([br[t, z, y, x_] for (x_, y, z, t) in sites]) - Dx
        assert np.sqrt((np.abs(res) ** 2).sum(axis=(1, 2))).max() <= 1.02e-10 * np.linalg.norm(br)
        del xr, br
    del b, x
    torch.cuda.empty_cache()  # the library allocates its own work vectors beside torch's cache


@pytest.mark.parametrize("mode", [lqcd.LQCD_MODE_FULL, lqcd.LQCD_MODE_DOMAIN])
def test_scale_perambulator_block(scale, mode):
    """The bench's call (16-RHS block of colour vectors 0..3, per-source vectors, mixed solver)
    against the plain FP64 solver on the same columns (4-RHS blocks: its FP64 work vectors for 16
    would not fit beside the rest at this size), and gamma_5-hermiticity of tau(t, t) on the
    block i, j < 4: tau^{ij}_{ab} = g5_aa conj(tau^{ji}_{ba}) g5_bb."""
    ctx, dims = scale["ctx"], scale["dims"]
    n_ev = SCALE["n_ev"]
    L3 = dims[0] * dims[1] * dims[2]
    t_src = [0] if mode == lqcd.LQCD_MODE_FULL else [0, 6, 12, 18]
    V = torch.from_numpy(colour_vectors(dims, n_ev, SCALE["cv_seed"], timeslices=t_src).reshape(
        len(t_src), n_ev, L3, 3)).cuda()
    taus = {}
    for name, p in (("mixed", default_params(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F32,
                                             rhs_block=16)),
                    ("plain", default_params(solver=lqcd.LQCD_SOLVER_BICGSTAB64, rhs_block=4))):
        tau = torch.zeros((len(t_src), n_ev, 4, n_ev, 4), dtype=torch.complex128, device="cuda")
        st = Stats(1, 1)
        ctx.perambulator_cols(V, n_ev, t_src, tau, 0, 4, mode=mode, sinks=lqcd.LQCD_SINKS_DIAG_SRCV, params=p,
                              stats=st)
        assert st.max_true_resid <= 1e-10
        taus[name] = tau.cpu().numpy()[:, :, :, :4, :]
        del tau
    for k in range(len(t_src)):
        a, b = taus["mixed"][k], taus["plain"][k]
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-9
        blk = a[:4]  # [i, alpha, j, beta], i, j < 4
        g5 = np.array([1, 1, -1, -1])
        herm = g5[None, :, None, None] * np.conj(np.transpose(blk, (2, 3, 0, 1))) * g5[None, None, None, :]
        assert np.linalg.norm(blk - herm) / np.linalg.norm(blk) < 1e-9
