"""Linear solves for the oracle (test infrastructure).

The paper names no solver ("inversions", Sec. 4).  The oracle uses two obviously-correct ones:

* ``cgnr``: conjugate gradients on the normal equations D^dag D x = D^dag b (Hestenes-Stiefel),
  run independently per right-hand side (vectorised over a leading batch axis), stopped on the
  recursively updated residual and accepted only when the TRUE residual ||b - D x|| / ||b||
  (recomputed from scratch) is below ``tol``; otherwise it restarts from the current iterate.
* ``dense_solve``: LU with partial pivoting (numpy.linalg.solve) on the dense 12V x 12V matrix,
  for lattices up to 4^3 x 8.

Pinned by: agreement of the two on 4^4 and 4^3x8 fields, and the free-field closed-form
propagator (tests/test_oracle_solve.py).
"""
import numpy as np


def _norm2(v):
    ax = tuple(range(1, v.ndim))
    return np.sum(np.abs(v) ** 2, axis=ax)


def _dot(a, b):
    ax = tuple(range(1, a.ndim))
    return np.sum(np.conj(a) * b, axis=ax)


def _bc(s, v):
    return s.reshape((-1,) + (1,) * (v.ndim - 1))


def cgnr(op, b, tol=1e-13, max_iter=20000, x0=None):
    """Solve op.apply(x) = b for every right-hand side in b[r, ...].

    Returns (x, info) with info = dict(iters=[...], true_resid=[...])."""
    b = np.asarray(b, dtype=np.complex128)
    nb = b.shape[0]
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    bnorm = np.sqrt(_norm2(b))
    bnorm = np.where(bnorm == 0, 1.0, bnorm)
    iters = np.zeros(nb, dtype=np.int64)
    total = 0
    while True:
        r = b - op.apply(x)
        true_res = np.sqrt(_norm2(r)) / bnorm
        active = true_res > tol
        if not active.any() or total >= max_iter:
            break
        z = op.apply_dagger(r)
        p = z.copy()
        zz = _norm2(z)
        while total < max_iter:
            w = op.apply(p)
            ww = _norm2(w)
            alpha = np.where(active, zz / np.where(ww == 0, 1, ww), 0.0)
            x = x + _bc(alpha, x) * p
            r = r - _bc(alpha, r) * w
            z = op.apply_dagger(r)
            zz_new = _norm2(z)
            beta = np.where(active, zz_new / np.where(zz == 0, 1, zz), 0.0)
            p = z + _bc(beta, p) * p
            zz = zz_new
            iters += active
            total += 1
            rel = np.sqrt(_norm2(r)) / bnorm
            active = active & (rel > 0.5 * tol)
            if not active.any():
                break
    return x, {"iters": iters, "true_resid": true_res}


def dense_solve(M, b):
    """x = M^{-1} b for b[r, ...] flattened per right-hand side (LU with partial pivoting)."""
    nb = b.shape[0]
    B = b.reshape(nb, -1).T
    X = np.linalg.solve(M, B)
    return X.T.reshape(b.shape)
