"""APE smearing of the spatial links (oracle; test infrastructure).

The paper computes its distillation vectors on APE-smeared gauge links and takes the smearing
parameters from elsewhere (Sec. 3.1); the definition followed here, with the weight alpha and the
number of steps as inputs:

    X_k(x)  = (1 - alpha) U_k(x) + (alpha / 4) sum_{j spatial, j != k} [ U_j(x) U_k(x+j) U_j(x+k)^dag
                                                        + U_j(x-j)^dag U_k(x-j) U_j(x-j+k) ]
    U'_k(x) = P(X_k(x)),   k = x, y, z  (time links are not smeared),

all links of a step updated from the previous step's field.  P projects onto SU(3): the unitary
polar factor W = X (X^dag X)^(-1/2) (the unitary matrix nearest to X in the Frobenius norm),
divided by det(W)^(1/3) with the principal cube root (arg in (-pi, pi] divided by 3).  Here
(X^dag X)^(-1/2) comes from a dense Hermitian eigendecomposition.

Pinned by (tests/test_oracle_smear.py): alpha = 0 and the unit field are fixed points, constant
commuting (diagonal) fields are fixed points, P(V H) = V for V in SU(3) and H positive definite
Hermitian, the output lies in SU(3), and gauge covariance U -> G U G^dag.
"""
import numpy as np

# numpy axis of a link array [t, z, y, x, mu, 3, 3] for a shift along mu
_AXIS = {0: 3, 1: 2, 2: 1, 3: 0}


def _shift(f, mu, n):
    """g(x) = f(x + n mu), periodic."""
    return np.roll(f, -n, axis=_AXIS[mu])


def _dag(M):
    return np.conj(np.swapaxes(M, -1, -2))


def project_su3(X):
    """P(X) for a stack of 3x3 complex matrices (unitary polar factor, det phase removed)."""
    H = _dag(X) @ X
    lam, Q = np.linalg.eigh(H)
    inv_sqrt = Q @ (lam[..., :, None] ** -0.5 * _dag(Q))
    W = X @ inv_sqrt
    d = np.linalg.det(W)
    root = np.exp(1j * np.angle(d) / 3.0) * np.abs(d) ** (1.0 / 3.0)
    return W / root[..., None, None]


def ape_smear(U, alpha, n_iter):
    """Spatial APE smearing of U[t, z, y, x, mu, 3, 3]; returns a new field (time links copied)."""
    out = U.copy()
    for _ in range(n_iter):
        prev = out.copy()
        for k in range(3):
            Uk = prev[..., k, :, :]
            stap = np.zeros_like(Uk)
            for j in range(3):
                if j == k:
                    continue
                Uj = prev[..., j, :, :]
                # forward staple: U_j(x) U_k(x+j) U_j(x+k)^dag
                stap += Uj @ _shift(Uk, j, 1) @ _dag(_shift(Uj, k, 1))
                # backward staple: U_j(x-j)^dag U_k(x-j) U_j(x-j+k)
                Ujm = _shift(Uj, j, -1)
                stap += _dag(Ujm) @ _shift(Uk, j, -1) @ _shift(_shift(Uj, j, -1), k, 1)
            out[..., k, :, :] = project_su3((1.0 - alpha) * Uk + (alpha / 4.0) * stap)
    return out
