"""GPU Laplacian eigensolver (distillation vectors, Sec. 3.1-3.2) against the oracle's dense
eigensolve, the free-field closed form, and the oracle's own Laplacian (residuals)."""
import itertools

import numpy as np
import pytest

from lqcd_inputs import gauge_field, unit_gauge_field
from oracle.distill import laplace_eigs, laplacian3d

pytestmark = pytest.mark.gpu
pytest.importorskip("paper_2609_37049_b300")
from paper_2609_37049_b300 import Context  # noqa: E402


def _gpu_eigs(U, n_ev, tol=1e-10):
    Lt, Lz, Ly, Lx = U.shape[:4]
    ctx = Context((Lx, Ly, Lz, Lt))
    ctx.gauge_upload(U, 0.12, 1.0)
    V = np.zeros((Lt, n_ev, Lx * Ly * Lz, 3), dtype=complex)
    lam = np.zeros((Lt, n_ev))
    ctx.laplace_eigs(n_ev, V, lam, tol=tol)
    return lam, V.reshape(Lt, n_ev, Lz, Ly, Lx, 3)


@pytest.mark.parametrize("dims,n_ev", [((4, 4, 4, 8), 6), ((8, 6, 4, 4), 16)])
def test_eigenpairs_match_dense_oracle(dims, n_ev):
    U = gauge_field(dims, 0.5, 4242)
    lam, V = _gpu_eigs(U, n_ev)
    lo, Vo = laplace_eigs(U, n_ev)
    assert np.abs(lam - lo).max() < 1e-10
    for t in range(dims[3]):
        ov = np.abs(np.einsum("izyxa,izyxa->i", V[t].conj(), Vo[t]))
        assert np.all(ov > 1 - 1e-8), ov
        res = laplacian3d(U, t, V[t]) - lam[t][:, None, None, None, None] * V[t]
        assert np.abs(res).max() < 1e-9
        X = V[t].reshape(n_ev, -1)
        assert np.abs(X @ X.conj().T - np.eye(n_ev)).max() < 1e-12
        k = np.argmax(np.abs(X), axis=1)
        ph = X[np.arange(n_ev), k]
        assert np.abs(ph.imag).max() < 1e-13 and ph.real.min() > 0


def test_free_field_spectrum():
    """Highly degenerate spectrum with a 21-fold cluster cut by n_ev: the eigenvector residual
    floor is ~1e-9 there, the eigenvalues (error quadratic in the residual) are exact."""
    dims = (4, 4, 2, 2)
    n_ev = 20
    lam, _ = _gpu_eigs(unit_gauge_field(dims), n_ev, tol=1e-8)
    want = sorted(sum(2 - 2 * np.cos(2 * np.pi * n[k] / dims[k]) for k in range(3))
                  for n in itertools.product(range(4), range(4), range(2)) for _ in range(3))[:n_ev]
    for t in range(2):
        assert np.abs(lam[t] - np.array(want)).max() < 1e-10


def test_ape_smeared_links_and_eigenvectors():
    """APE smearing (alpha 0.5, 3 steps) against the oracle link by link; the distillation vectors
    on the smeared links against the oracle's dense eigensolve of the oracle-smeared field; a
    smearing of 0 steps brings back the plain links' spectrum."""
    from oracle.smear import ape_smear
    dims = (4, 4, 4, 4)
    U = gauge_field(dims, 0.5, 515)
    ctx = Context(dims)
    ctx.gauge_upload(U, 0.12, 1.0)
    ctx.ape_smear(0.5, 3)
    S = np.zeros(U.shape[:4] + (3, 3, 3), dtype=complex)
    ctx.smeared_links(S)
    So = ape_smear(U, 0.5, 3)
    assert np.abs(S - So[..., :3, :, :]).max() < 1e-12
    n_ev = 6
    V = np.zeros((dims[3], n_ev, 64, 3), dtype=complex)
    lam = np.zeros((dims[3], n_ev))
    ctx.laplace_eigs(n_ev, V, lam)
    lo, Vo = laplace_eigs(So, n_ev)
    assert np.abs(lam - lo).max() < 1e-10
    V = V.reshape(dims[3], n_ev, 4, 4, 4, 3)
    for t in range(dims[3]):
        ov = np.abs(np.einsum("izyxa,izyxa->i", V[t].conj(), Vo[t]))
        assert np.all(ov > 1 - 1e-8), ov
    # smeared links spread the low spectrum less than the rough links: the lowest eigenvalues drop
    lr, _ = laplace_eigs(U, n_ev)
    assert lo[:, 0].mean() < lr[:, 0].mean()
    ctx.ape_smear(0.5, 0)
    ctx.laplace_eigs(n_ev, V.reshape(dims[3], n_ev, 64, 3), lam)
    assert np.abs(lam - lr).max() < 1e-10
