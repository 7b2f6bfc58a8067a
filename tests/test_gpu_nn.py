"""GPU network preconditioner against the oracle (oracle/nn.py): forward pass, loss and Wirtinger
gradients (FP32 kernels vs FP64 oracle, same weights), training on solver-generated pairs, and
the flexible-GCR solve it preconditions, judged by the oracle's operator at 1e-10."""
import numpy as np
import pytest

from lqcd_inputs import random_spinors
from oracle import nn
from oracle.dirac import WilsonClover, fermion_links, parity_table, BC_ANTIPERIODIC
from tests.lattice_cases import ROUGH, gauge, per_domain_resid

pytestmark = pytest.mark.gpu
pytest.importorskip("paper_2609_37049_b300")
from paper_2609_37049_b300 import Context, Stats, default_params, lqcd  # noqa: E402


def _ctx(case, U):
    ctx = Context(case["dims"])
    ctx.gauge_upload(U, case["kappa"], case["c_sw"])
    ctx.set_domains(case["extents"])
    return ctx


def _fields(case, n, seed):
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz, Lt = case["dims"]
    shape = (n, Lt, Lz, Ly, Lx, 4, 3)
    return (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)


def _bf16_safe(Ws):
    return [np.asarray(W, np.complex64).astype(np.complex128) for W in Ws]


@pytest.mark.parametrize("domain", [False, True])
def test_forward_matches_oracle(domain):
    case = ROUGH
    U = gauge(case, 77)
    ctx = _ctx(case, U)
    Ws = _bf16_safe(nn.init_weights(3, 0.3))
    ctx.nn_set_weights(Ws)
    x = _fields(case, 3, 1)
    out = np.zeros_like(x)
    ctx.nn_apply(x, out, domain=domain)
    Ue = fermion_links(U, BC_ANTIPERIODIC, case["extents"] if domain else None)
    ref = nn.forward(Ws, Ue, x.astype(np.complex128))[-1]
    assert np.abs(out - ref).max() / np.abs(ref).max() < 2e-5


@pytest.mark.parametrize("domain", [False, True])
def test_tensor_core_forward_within_bf16_bound(domain):
    """The inference path (BF16 weights and activations, tcgen05 channel mixing, FP32 accumulation)
    against the FP64 oracle with the same weights: BF16 keeps 8 significant bits, so each layer's
    inputs carry about 2^-9 relative rounding; over four layers the outputs stay within 2% of the
    largest output entry and 1% in the Frobenius norm."""
    case = ROUGH
    U = gauge(case, 81)
    ctx = _ctx(case, U)
    Ws = [np.asarray(W, np.complex64).astype(np.complex128) for W in nn.init_weights(7, 0.3)]
    ctx.nn_set_weights(Ws)
    x = _fields(case, 5, 9)
    out = np.zeros_like(x)
    ctx.nn_apply_tc(x, out, domain=domain)
    Ue = fermion_links(U, BC_ANTIPERIODIC, case["extents"] if domain else None)
    ref = nn.forward(Ws, Ue, x.astype(np.complex128))[-1]
    assert np.abs(out - ref).max() <= 2e-2 * np.abs(ref).max()
    assert np.linalg.norm(out - ref) <= 1e-2 * np.linalg.norm(ref)
    assert np.linalg.norm(out - ref) > 0  # BF16 rounding is visible: this is not the FP32 path


@pytest.mark.parametrize("even_only", [False, True])
def test_loss_and_gradient_match_oracle(even_only):
    case = ROUGH
    U = gauge(case, 78)
    ctx = _ctx(case, U)
    Ws = _bf16_safe(nn.init_weights(4, 0.3))
    ctx.nn_set_weights(Ws)
    x, tgt = _fields(case, 2, 2), _fields(case, 2, 3)
    L, G = ctx.nn_loss_grad(x, tgt, even_only=even_only)
    dims = case["dims"]
    mask = np.ones((dims[3], dims[2], dims[1], dims[0]))
    if even_only:
        mask = (parity_table(dims) == 0).reshape(mask.shape).astype(float)
    Lo, Go = nn.loss_and_grad(Ws, fermion_links(U), x.astype(np.complex128), tgt.astype(np.complex128), mask)
    assert abs(L - Lo) < 1e-5 * Lo
    for g, go in zip(G, Go):
        assert np.abs(g - go).max() < 1e-4 * np.abs(go).max()


def test_bf16_training_gradient_within_bound():
    """The BF16 training kernels (tensor-core forward / backward-data layers, BF16 transported
    activations) give the loss to BF16 rounding and a gradient within 3% (Frobenius, per layer) of
    the FP64 oracle's."""
    case = ROUGH
    U = gauge(case, 82)
    ctx = _ctx(case, U)
    Ws = _bf16_safe(nn.init_weights(8, 0.3))
    ctx.nn_set_weights(Ws)
    x, tgt = _fields(case, 2, 4), _fields(case, 2, 5)
    dims = case["dims"]
    mask = (parity_table(dims) == 0).reshape(dims[3], dims[2], dims[1], dims[0]).astype(float)
    L, G = ctx.nn_loss_grad(x, tgt, even_only=True, bf16=True)
    Lo, Go = nn.loss_and_grad(Ws, fermion_links(U), x.astype(np.complex128), tgt.astype(np.complex128), mask)
    assert abs(L - Lo) < 2e-2 * Lo
    for g, go in zip(G, Go):
        assert np.linalg.norm(g - go) < 3e-2 * np.linalg.norm(go)


def test_training_lowers_loss_and_preconditions_fgcr():
    """Training on pairs from the plain solver lowers the loss; the trained network inside FGCR
    reaches FP64 true residual 1e-10 (checked with the oracle's operator) in fewer iterations than
    FGCR without a preconditioner (the gain the network brings)."""
    case = ROUGH
    U = gauge(case, 79)
    ctx = _ctx(case, U)
    ctx.nn_set_weights(nn.init_weights(5, 0.05))
    hist = ctx.nn_train(n_pairs=32, epochs=8, batch=4, lr=3e-3, seed=11)
    assert hist[-1] < 0.7 * hist[0], hist
    b = random_spinors(case["dims"], 4, 12)
    iters = {}
    for name, kw in (("nn", dict(solver=lqcd.LQCD_SOLVER_FGCR_NN)),
                     ("none", dict(solver=lqcd.LQCD_SOLVER_FGCR_NN, precond_iters=-1))):
        x = np.zeros_like(b)
        st = Stats(4, 1)
        ctx.solve(b, x, default_params(**kw), stats=st)
        r = b - WilsonClover(U, case["kappa"], case["c_sw"]).apply(x)
        assert per_domain_resid(b, r, [case["dims"][3]]).max() <= 1.02e-10
        assert st.fallback == 0
        iters[name] = st.total_iters
    assert iters["nn"] < iters["none"], iters


def test_fgcr_nn_without_network_falls_back():
    case = ROUGH
    U = gauge(case, 80)
    ctx = _ctx(case, U)
    b = random_spinors(case["dims"], 2, 13)
    x = np.zeros_like(b)
    st = Stats(2, 1)
    ctx.solve(b, x, default_params(solver=lqcd.LQCD_SOLVER_FGCR_NN), stats=st)
    assert st.fallback == 1 and st.max_true_resid <= 1e-10
