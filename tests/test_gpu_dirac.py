"""GPU parity of the operator and the solvers against the FP64 oracle (Sec. 2.1, Sec. 3).

The operator is compared element by element (FP64 round-off); every solve is checked by the
ORACLE's operator: ||b - D x_gpu|| / ||b|| <= 1e-10 per right-hand side (and per domain for the
Dirichlet domain operator), and x_gpu against the oracle's own solution."""
import numpy as np
import pytest

from lqcd_inputs import gauge_field, random_spinors
from oracle.dirac import WilsonClover, BC_ANTIPERIODIC, BC_PERIODIC, BC_OPEN
from oracle.solve import cgnr
from tests.lattice_cases import ROUGH, gauge, rel_max, per_domain_resid

pytestmark = pytest.mark.gpu

lqcd_pkg = pytest.importorskip("paper_2609_37049_b300")
from paper_2609_37049_b300 import Context, Stats, default_params, lqcd  # noqa: E402


@pytest.mark.parametrize("dims,bc,ext", [
    ((4, 4, 4, 8), BC_ANTIPERIODIC, [4, 4]),
    ((6, 4, 2, 8), BC_PERIODIC, [2, 3, 3]),
    ((4, 2, 4, 6), BC_OPEN, [6]),
    ((2, 2, 2, 4), BC_ANTIPERIODIC, [1, 3]),
])
def test_dirac_apply_parity(dims, bc, ext):
    U = gauge_field(dims, 0.5, 1234)
    op = WilsonClover(U, 0.125, 1.6, bc)
    psi = random_spinors(dims, 3, 7)
    ctx = Context(dims, bc)
    ctx.gauge_upload(U, 0.125, 1.6)
    out = np.zeros_like(psi)
    ctx.dirac_apply(psi, out)
    assert rel_max(out, op.apply(psi)) < 1e-14
    ctx.set_domains(ext)
    ctx.dirac_apply(psi, out, domain_restricted=True)
    assert rel_max(out, op.restricted(ext).apply(psi)) < 1e-14


def test_dirac_apply_device_pointers():
    torch = pytest.importorskip("torch")
    dims = (4, 4, 4, 8)
    U = gauge_field(dims, 0.5, 99)
    psi = random_spinors(dims, 2, 5)
    ctx = Context(dims)
    ctx.gauge_upload(torch.from_numpy(U).cuda(), 0.125, 1.6)
    out = torch.zeros(psi.shape, dtype=torch.complex128, device="cuda")
    ctx.dirac_apply(torch.from_numpy(psi).cuda(), out)
    torch.cuda.synchronize()
    assert rel_max(out.cpu().numpy(), WilsonClover(U, 0.125, 1.6).apply(psi)) < 1e-14


SOLVERS = [
    ("bicgstab64", dict(solver=lqcd.LQCD_SOLVER_BICGSTAB64)),
    ("mixed32", dict(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F32)),
    ("mixed16", dict(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F16)),
    ("nograph", dict(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=lqcd.LQCD_PREC_F32, use_graph=0)),
]


@pytest.mark.parametrize("name,kw", SOLVERS)
@pytest.mark.parametrize("domain", [False, True])
def test_solve_true_residual(name, kw, domain):
    case = ROUGH
    U = gauge(case, 2024)
    op = WilsonClover(U, case["kappa"], case["c_sw"])
    ext = case["extents"]
    b = random_spinors(case["dims"], 5, 11)
    ctx = Context(case["dims"])
    ctx.gauge_upload(U, case["kappa"], case["c_sw"])
    ctx.set_domains(ext)
    x = np.zeros_like(b)
    st = Stats(5, len(ext) if domain else 1)
    ctx.solve(b, x, default_params(rhs_block=3, **kw), domain=domain, stats=st)
    ref_op = op.restricted(ext) if domain else op
    r = b - ref_op.apply(x)
    res = per_domain_resid(b, r, ext if domain else [case["dims"][3]])
    assert res.max() <= 1.02e-10, res
    assert st.max_true_resid <= 1e-10 and np.all(st.true_resid <= 1e-10)
    assert np.all(st.iters > 0)
    xo, _ = cgnr(ref_op, b, tol=1e-13)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) < 1e-8


def test_domain_solve_with_empty_domain_and_one_domain_equals_full():
    case = ROUGH
    U = gauge(case, 7)
    ctx = Context(case["dims"])
    ctx.gauge_upload(U, case["kappa"], case["c_sw"])
    b = random_spinors(case["dims"], 2, 3)
    b[:, 4:] = 0  # nothing in the second domain
    ctx.set_domains([4, 4])
    x = np.zeros_like(b)
    st = Stats(2, 2)
    ctx.solve(b, x, default_params(), domain=True, stats=st)
    assert np.abs(x[:, 4:]).max() == 0
    assert np.all(st.true_resid.reshape(2, 2)[:, 1] == 0)
    # a single domain covering the whole time axis is the full operator
    ctx.set_domains([8])
    xd, xf = np.zeros_like(b), np.zeros_like(b)
    ctx.solve(b, xd, default_params(), domain=True)
    ctx.solve(b, xf, default_params(), domain=False)
    assert np.array_equal(xd, xf)


def test_invalid_arguments_do_nothing():
    ctx = Context((4, 4, 4, 8))
    with pytest.raises(lqcd.LqcdError) as e:
        ctx.set_domains([4, 3])
    assert e.value.code == lqcd.LQCD_ERR_INVALID_ARG
    b = np.zeros((1, 8, 4, 4, 4, 4, 3), dtype=complex)
    with pytest.raises(lqcd.LqcdError) as e:
        ctx.solve(b, b.copy())
    assert e.value.code == lqcd.LQCD_ERR_STATE


def test_not_converged_reports_partial_result():
    case = ROUGH
    U = gauge(case, 5)
    ctx = Context(case["dims"])
    ctx.gauge_upload(U, case["kappa"], case["c_sw"])
    b = random_spinors(case["dims"], 1, 3)
    x = np.zeros_like(b)
    st = Stats(1, 1)
    rc = ctx.solve(b, x, default_params(max_iter=8, max_outer=1, check_every=4), stats=st,
                   allow_not_converged=True)
    assert rc == lqcd.LQCD_ERR_NOT_CONVERGED
    assert 1e-10 < st.max_true_resid < 1.0


@pytest.mark.parametrize("prec,nrhs", [("f32", 16), ("f32", 32), ("f16", 32)])
def test_dslash_launch_variants_agree(prec, nrhs):
    """Every dslash launch variant (register caps; links and clover staged per site in shared
    memory; neighbour spinors staged by bulk copies) computes the same operator up to FP32
    rounding (the compiler may contract the same expressions differently): each mixed solve
    reaches the oracle's true residual, takes within two iterations of variant 0 per RHS, and
    agrees with it within the solves' accuracy.  16 RHS = 8 sites per staged block; 32 RHS also
    runs the bulk-copy kernel."""
    case = ROUGH
    U = gauge(case, 77)
    op = WilsonClover(U, case["kappa"], case["c_sw"])
    ext = case["extents"]
    b = random_spinors(case["dims"], nrhs, 13)
    ctx = Context(case["dims"])
    ctx.gauge_upload(U, case["kappa"], case["c_sw"])
    ctx.set_domains(ext)
    p = lqcd.LQCD_PREC_F32 if prec == "f32" else lqcd.LQCD_PREC_F16
    params = default_params(solver=lqcd.LQCD_SOLVER_MIXED, inner_prec=p, rhs_block=nrhs)
    for domain in (False, True):
        ref_op = op.restricted(ext) if domain else op
        ref = None
        for v in range(8):
            ctx.set_dslash_variant(p, nrhs, v)
            ctx.set_dslash_variant(lqcd.LQCD_PREC_F64, nrhs, v % 3)  # the FP64 true-residual launches
            x = np.zeros_like(b)
            st = Stats(nrhs, len(ext) if domain else 1)
            ctx.solve(b, x, params, domain=domain, stats=st)
            res = per_domain_resid(b, b - ref_op.apply(x), ext if domain else [case["dims"][3]])
            assert res.max() <= 1.02e-10, (v, res.max())
            if ref is None:
                ref = (x.copy(), st.iters.copy())
            else:
                assert np.abs(st.iters - ref[1]).max() <= 2, (v, st.iters, ref[1])
                assert np.linalg.norm(x - ref[0]) / np.linalg.norm(ref[0]) < 1e-8, v


def oracle_schur(op, x):
    """M x_e = x_e - kappa^2 A_ee^-1 H_eo A_oo^-1 H_oe x_e from the oracle's pieces (even sites)."""
    from oracle.dirac import apply_site_matrix, hopping, parity_table
    Lx, Ly, Lz, Lt = op.dims
    par = parity_table(op.dims).reshape(Lt, Lz, Ly, Lx)
    even = (par == 0)[..., None, None]
    odd = (par == 1)[..., None, None]
    Ainv = np.linalg.inv(op.A)
    xe = x * even
    z = apply_site_matrix(Ainv, hopping(op.Ue, xe) * odd) * odd
    return xe - op.kappa ** 2 * apply_site_matrix(Ainv, hopping(op.Ue, z) * even) * even


# storage precision -> (launch variants, max relative error against the FP64 oracle)
SCHUR_PRECS = {"f64": (range(3), 1e-13), "f32": (range(8), 2e-6), "f16": (range(8), 4e-3)}


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("nrhs", [3, 16, 32])
@pytest.mark.parametrize("domain", [False, True])
def test_schur_operator_parity(prec, nrhs, domain):
    """The solvers' even-odd operator in each storage precision and launch variant, element by
    element against the oracle (FP32 / FP16 bounds: storage rounding of inputs, links and clover
    plus FP32 arithmetic).  nrhs 3 runs every variant as the direct kernel; 16 / 32 the staged
    kernels (8 / 4 sites per block; 32 also the bulk-copy kernel)."""
    case = ROUGH
    U = gauge(case, 555)
    op = WilsonClover(U, case["kappa"], case["c_sw"])
    ext = case["extents"]
    ref_op = op.restricted(ext) if domain else op
    x = random_spinors(case["dims"], nrhs, 21)
    ref = oracle_schur(ref_op, x)
    ctx = Context(case["dims"])
    ctx.gauge_upload(U, case["kappa"], case["c_sw"])
    ctx.set_domains(ext)
    p = {"f64": lqcd.LQCD_PREC_F64, "f32": lqcd.LQCD_PREC_F32, "f16": lqcd.LQCD_PREC_F16}[prec]
    variants, tol = SCHUR_PRECS[prec]
    for v in variants:
        ctx.set_dslash_variant(p, nrhs, v)
        out = np.zeros_like(x)
        ctx.schur_apply(p, x, out, domain_restricted=domain)
        err = rel_max(out, ref)
        assert err < tol, (prec, v, err)


@pytest.mark.parametrize("ext,t_start", [([3, 5], 6), ([2, 3, 3], 1), ([4, 4], 2)])
def test_shifted_tiling_operator_and_solve(ext, t_start):
    """Tilings whose domain 0 starts at t_start (the last domain wraps around the time boundary):
    the domain operator element by element, and a mixed domain solve to 1e-10 in every domain,
    both against the oracle's shifted D_Lambda."""
    from oracle.dirac import domain_of_t
    case = ROUGH
    U = gauge(case, 4242)
    op = WilsonClover(U, case["kappa"], case["c_sw"]).restricted(ext, t_start)
    ctx = Context(case["dims"])
    ctx.gauge_upload(U, case["kappa"], case["c_sw"])
    ctx.set_domains(ext, t_start=t_start)
    psi = random_spinors(case["dims"], 3, 8)
    out = np.zeros_like(psi)
    ctx.dirac_apply(psi, out, domain_restricted=True)
    assert rel_max(out, op.apply(psi)) < 1e-14
    b = random_spinors(case["dims"], 4, 9)
    x = np.zeros_like(b)
    st = Stats(4, len(ext))
    ctx.solve(b, x, default_params(solver=lqcd.LQCD_SOLVER_MIXED, rhs_block=4), domain=True, stats=st)
    dom = domain_of_t(ext, case["dims"][3], t_start)
    r = b - op.apply(x)
    for k in range(4):
        for d in range(len(ext)):
            m = dom == d
            assert np.linalg.norm(r[k, m]) / np.linalg.norm(b[k, m]) <= 1.02e-10
    assert st.max_true_resid <= 1e-10
