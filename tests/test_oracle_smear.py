"""Pins of the oracle's APE smearing and SU(3) projection (Sec. 3.1 smeared distillation links)."""
import numpy as np

from lqcd_inputs import gauge_field, unit_gauge_field, random_gauge_transform
from oracle.smear import ape_smear, project_su3


def _dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def test_projection_returns_the_unitary_factor():
    """P(V H) = V for V in SU(3) and H Hermitian positive definite (polar decomposition is unique),
    and P(c V) = V for c > 0."""
    V = random_gauge_transform((2, 2, 2, 2), 11).reshape(-1, 3, 3)
    rng = np.random.default_rng(3)
    A = rng.normal(size=(V.shape[0], 3, 3)) + 1j * rng.normal(size=(V.shape[0], 3, 3))
    H = A @ _dag(A) + 0.5 * np.eye(3)
    assert np.abs(project_su3(V @ H) - V).max() < 1e-13
    assert np.abs(project_su3(2.5 * V) - V).max() < 1e-14


def test_output_in_su3_and_fixed_points():
    dims = (4, 4, 4, 2)
    U = gauge_field(dims, 0.6, 21)
    S = ape_smear(U, 0.5, 3)
    eye = np.eye(3)
    assert np.abs(_dag(S) @ S - eye).max() < 1e-13
    assert np.abs(np.linalg.det(S) - 1).max() < 1e-13
    assert np.array_equal(S[..., 3, :, :], U[..., 3, :, :])  # time links untouched
    assert np.abs(ape_smear(U, 0.0, 2) - U).max() < 1e-13  # alpha = 0: projection of SU(3) is itself
    one = unit_gauge_field(dims)
    assert np.abs(ape_smear(one, 0.5, 2) - one).max() < 1e-14
    # constant commuting fields: every staple equals the link itself
    C = unit_gauge_field(dims)
    for k, th in enumerate((0.3, -0.7, 1.1)):
        C[..., k, :, :] = np.diag(np.exp(1j * np.array([th, 2 * th, -3 * th])))
    assert np.abs(ape_smear(C, 0.4, 2) - C).max() < 1e-13


def test_gauge_covariance():
    """Smearing U^G (U_k(x) -> G(x) U_k(x) G(x+k)^dag) gives the smeared field transformed by G."""
    dims = (4, 2, 4, 2)
    U = gauge_field(dims, 0.5, 31)
    G = random_gauge_transform(dims, 32)
    axis = {0: 3, 1: 2, 2: 1, 3: 0}

    def transform(F):
        out = F.copy()
        for mu in range(4):
            Gs = np.roll(G, -1, axis=axis[mu])
            out[..., mu, :, :] = G @ F[..., mu, :, :] @ _dag(Gs)
        return out

    a = ape_smear(transform(U), 0.5, 2)
    b = transform(ape_smear(U, 0.5, 2))
    assert np.abs(a - b).max() < 1e-12
