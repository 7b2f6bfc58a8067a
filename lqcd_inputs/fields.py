"""Synthetic lattice fields drawn from the Philox streams of ``philox.py``.

Recipes (index arithmetic fixed here so both sides draw identical numbers):

* gauge links: link id ``l = 4*s + mu`` (``s`` = flat site index, ``mu`` = 0..3 = x,y,z,t); the
  eight coefficients h_1..h_8 come from Philox indices ``4*l + j`` (j = 0..3, two normals each,
  h_{2j+1}, h_{2j+2}); ``H = sum_a h_a lambda_a / 2`` with the Gell-Mann matrices ``lambda_a``;
  ``U = exp(i eps H)`` through the eigendecomposition of the Hermitian ``H``.
* colour vectors: element ``(t, i, s3, a)`` (``s3`` = flat spatial index) uses Philox index
  ``((t*n_ev + i)*L^3 + s3)*3 + a``; the two normals are the real and imaginary parts (each
  scaled by 1/sqrt 2).  The ``n_ev`` vectors of each timeslice are then orthonormalised by
  Cholesky-QR applied twice (a Gram-Schmidt-equivalent, deterministic orthonormalisation).
* spinors: element ``(r, s, spin, colour)`` uses index ``((r*V + s)*4 + spin)*3 + colour``.
"""
import numpy as np

from .philox import gaussians


def _per_timeslice(fn, items):
    """fn(k, t) for every (k, t) of items, in order (the compiled generators and BLAS parallelise
    inside each timeslice)."""
    for k, t in items:
        fn(k, t)

PURPOSE_GAUGE = 1
PURPOSE_COLOUR = 2
PURPOSE_SPINOR = 3
PURPOSE_GAUGE_TRANSFORM = 4


def gell_mann():
    """The eight Gell-Mann matrices lambda_1..lambda_8 as an array (8, 3, 3) complex128."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0, 0, 1] = l[0, 1, 0] = 1
    l[1, 0, 1] = -1j
    l[1, 1, 0] = 1j
    l[2, 0, 0] = 1
    l[2, 1, 1] = -1
    l[3, 0, 2] = l[3, 2, 0] = 1
    l[4, 0, 2] = -1j
    l[4, 2, 0] = 1j
    l[5, 1, 2] = l[5, 2, 1] = 1
    l[6, 1, 2] = -1j
    l[6, 2, 1] = 1j
    l[7, 0, 0] = l[7, 1, 1] = 1 / np.sqrt(3)
    l[7, 2, 2] = -2 / np.sqrt(3)
    return l


def _su3_from_ids(seed, purpose, link_ids, eps):
    from .philox import _compiled
    lib = _compiled()
    if lib is not None and link_ids.size >= 1024:  # compiled recipe: Jacobi eigen-decomposition of H
        ids = np.ascontiguousarray(link_ids, dtype=np.uint64)
        out = np.empty((ids.size, 3, 3), dtype=np.complex128)
        lib.su3_links(ids.ctypes.data, ids.size, int(purpose) & 0xFFFFFFFF, int(seed) & 0xFFFFFFFFFFFFFFFF,
                      float(eps), out.ctypes.data)
        return out
    g = gaussians(seed, purpose, link_ids[:, None] * 4 + np.arange(4, dtype=np.uint64)[None, :])
    h = g.reshape(link_ids.shape[0], 8)
    H = np.einsum("na,aij->nij", h, gell_mann() / 2.0)
    w, Q = np.linalg.eigh(H)
    return np.einsum("nij,nj,nkj->nik", Q, np.exp(1j * eps * w), Q.conj())


def gauge_field(dims, eps, seed):
    """U[t,z,y,x,mu,3,3] = exp(i eps H) with Philox-seeded Gaussian traceless Hermitian H."""
    Lx, Ly, Lz, Lt = dims
    vol3 = Lx * Ly * Lz
    U = np.empty((Lt, Lz, Ly, Lx, 4, 3, 3), dtype=np.complex128)

    def one(k, t):  # one timeslice at a time bounds the temporary memory
        ids = (np.uint64(t * vol3 * 4) + np.arange(vol3 * 4, dtype=np.uint64))
        U[t] = _su3_from_ids(seed, PURPOSE_GAUGE, ids, eps).reshape(Lz, Ly, Lx, 4, 3, 3)

    _per_timeslice(one, enumerate(range(Lt)))
    return U


def unit_gauge_field(dims):
    """The free field U = 1."""
    Lx, Ly, Lz, Lt = dims
    U = np.zeros((Lt, Lz, Ly, Lx, 4, 3, 3), dtype=np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1.0
    return U


def random_gauge_transform(dims, seed, eps=1.0):
    """A field G[t,z,y,x,3,3] of SU(3) matrices (one per site), same recipe as the links."""
    Lx, Ly, Lz, Lt = dims
    V = Lx * Ly * Lz * Lt
    G = _su3_from_ids(seed, PURPOSE_GAUGE_TRANSFORM, np.arange(V, dtype=np.uint64), eps)
    return G.reshape(Lt, Lz, Ly, Lx, 3, 3)


def _cholqr_rows(X):
    """Orthonormalise the rows of X (n, m) by Cholesky-QR: X <- L^{-1} X with L L^H = X X^H."""
    from scipy.linalg import solve_triangular
    G = X @ X.conj().T
    L = np.linalg.cholesky(G)
    return solve_triangular(L, X, lower=True)


def colour_vectors(dims, n_ev, seed, timeslices=None):
    """V[t, i, z, y, x, a]: n_ev orthonormal complex Gaussian colour vectors per timeslice.

    ``timeslices`` selects which t to generate (default all); the draws depend only on the
    global (t, i, s3, a) so a subset reproduces the corresponding slices of the full set.
    """
    Lx, Ly, Lz, Lt = dims
    vol3 = Lx * Ly * Lz
    ts = list(range(Lt)) if timeslices is None else list(timeslices)
    out = np.empty((len(ts), n_ev, Lz, Ly, Lx, 3), dtype=np.complex128)
    n = vol3 * 3

    def one(k, t):
        ids = np.uint64(t * n_ev * n) + np.arange(n_ev * n, dtype=np.uint64)
        g = gaussians(seed, PURPOSE_COLOUR, ids)
        X = ((g[..., 0] + 1j * g[..., 1]) / np.sqrt(2.0)).reshape(n_ev, n)
        X = _cholqr_rows(_cholqr_rows(X))
        out[k] = X.reshape(n_ev, Lz, Ly, Lx, 3)

    _per_timeslice(one, enumerate(ts))
    return out


def random_spinors(dims, nrhs, seed):
    """psi[r, t, z, y, x, spin, colour]: complex Gaussian spinor fields."""
    Lx, Ly, Lz, Lt = dims
    V = Lx * Ly * Lz * Lt
    ids = np.arange(nrhs * V * 12, dtype=np.uint64)
    g = gaussians(seed, PURPOSE_SPINOR, ids)
    psi = (g[..., 0] + 1j * g[..., 1]) / np.sqrt(2.0)
    return psi.reshape(nrhs, Lt, Lz, Ly, Lx, 4, 3)
