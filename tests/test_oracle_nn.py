"""Pins of the network oracle: finite differences of its gradients, gauge covariance, the
adjoint identity and the free-field form of a layer (plane waves are eigenvectors of the paths)."""
import numpy as np

from lqcd_inputs import gauge_field, random_gauge_transform, unit_gauge_field
from oracle.dirac import fermion_links, parity_table, BC_ANTIPERIODIC
from oracle import nn

DIMS = (4, 2, 2, 4)


def _field(seed, C=4, batch=2):
    rng = np.random.default_rng(seed)
    Lx, Ly, Lz, Lt = DIMS
    return rng.normal(size=(batch, Lt, Lz, Ly, Lx, C, 3)) + 1j * rng.normal(size=(batch, Lt, Lz, Ly, Lx, C, 3))


def test_gradient_by_finite_differences():
    Ue = fermion_links(gauge_field(DIMS, 0.5, 3), BC_ANTIPERIODIC, [2, 2])
    Ws = nn.init_weights(5, 0.3)
    h, tgt = _field(1), _field(2)
    mask = (parity_table(DIMS) == 0).reshape(DIMS[3], DIMS[2], DIMS[1], DIMS[0]).astype(float)
    L, G = nn.loss_and_grad(Ws, Ue, h, tgt, mask)
    rng = np.random.default_rng(0)
    for l in range(4):
        for _ in range(3):
            p, o, c = rng.integers(9), rng.integers(Ws[l].shape[1]), rng.integers(Ws[l].shape[2])
            for part, unit in ((0, 1.0), (1, 1j)):
                eps = 1e-6
                Wp = [W.copy() for W in Ws]
                Wm = [W.copy() for W in Ws]
                Wp[l][p, o, c] += eps * unit
                Wm[l][p, o, c] -= eps * unit
                fd = (nn.loss_and_grad(Wp, Ue, h, tgt, mask)[0] - nn.loss_and_grad(Wm, Ue, h, tgt, mask)[0]) / (2 * eps)
                an = 2 * (G[l][p, o, c].real if part == 0 else G[l][p, o, c].imag)
                assert abs(fd - an) < 1e-6 * max(1.0, abs(an)), (l, p, o, c, part, fd, an)


def test_gauge_covariance():
    U = gauge_field(DIMS, 0.6, 7)
    G = random_gauge_transform(DIMS, 8)
    Gsh = {0: np.roll(G, -1, 3), 1: np.roll(G, -1, 2), 2: np.roll(G, -1, 1), 3: np.roll(G, -1, 0)}
    UG = np.stack([G @ U[:, :, :, :, mu] @ np.conj(np.swapaxes(Gsh[mu], -1, -2)) for mu in range(4)], axis=4)
    Ws = nn.init_weights(9, 0.3)
    h = _field(3, batch=1)
    rot = lambda f: np.einsum("tzyxab,ntzyxcb->ntzyxca", G, f)
    out = nn.forward(Ws, fermion_links(U), h)[-1]
    outG = nn.forward(Ws, fermion_links(UG), rot(h))[-1]
    assert np.abs(outG - rot(out)).max() < 1e-12


def test_adjoint_identity():
    Ue = fermion_links(gauge_field(DIMS, 0.5, 11))
    W = nn.init_weights(12, 0.5)[1]  # 8 -> 8
    a, b = _field(4, C=8, batch=1), _field(5, C=8, batch=1)
    lhs = np.vdot(a, nn.layer(W, Ue, b))
    rhs = np.vdot(nn.layer_adjoint(W, Ue, a), b)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_free_field_layer_is_diagonal_in_momentum():
    """U = 1, periodic fermion links: T_{+mu} e^{ipx} = e^{i p_mu} e^{ipx}, T_{-mu} -> e^{-i p_mu}."""
    Ue = fermion_links(unit_gauge_field(DIMS), bc_t=0)
    W = nn.init_weights(13, 0.5)[0]  # 4 -> 8
    Lx, Ly, Lz, Lt = DIMS
    p = np.array([2 * np.pi / Lx, 0, np.pi, 2 * np.pi * 3 / Lt])
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    u = np.arange(12).reshape(4, 3) * (0.3 + 0.1j)
    h = ph[..., None, None] * u
    fac = np.array([1] + [np.exp(1j * p[m]) for m in range(4)] + [np.exp(-1j * p[m]) for m in range(4)])
    want = ph[..., None, None] * np.einsum("p,poc,ca->oa", fac, W, u)
    assert np.abs(nn.layer(W, Ue, h) - want).max() < 1e-12
