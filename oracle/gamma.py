"""Dirac matrices for the oracle (test infrastructure; see package docstring).

Conventions (the paper names gamma_0 and gamma_5 but fixes no basis, Sec. 2):
Euclidean, Hermitian, chiral basis
    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]   (k = x, y, z)
    gamma_t = [[0, 1], [1, 0]]                     (the paper's gamma_0)
    gamma_5 = gamma_x gamma_y gamma_z gamma_t
    sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu].
The 16-element Clifford table used for Gamma masks:
    0: 1,  1-4: gamma_x, gamma_y, gamma_z, gamma_t,  5: gamma_5,
    6-9: gamma_mu gamma_5 (mu = x,y,z,t),
    10-15: sigma_{mu nu} for (mu,nu) = (x,y),(x,z),(x,t),(y,z),(y,t),(z,t).
Pinned by: Clifford algebra, Hermiticity, gamma_5 = diag(1,1,-1,-1) (tests/test_oracle_gamma.py).
"""
import numpy as np

PAULI = np.array(
    [[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=np.complex128
)


def gammas():
    """gamma_mu for mu = 0..3 = x, y, z, t as an array (4, 4, 4)."""
    g = np.zeros((4, 4, 4), dtype=np.complex128)
    z = np.zeros((2, 2), dtype=np.complex128)
    for k in range(3):
        g[k] = np.block([[z, -1j * PAULI[k]], [1j * PAULI[k], z]])
    g[3] = np.block([[z, np.eye(2)], [np.eye(2), z]])
    return g


def gamma5():
    g = gammas()
    return g[0] @ g[1] @ g[2] @ g[3]


def sigma(mu, nu):
    g = gammas()
    return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])


PLANES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def clifford_table():
    """The 16 Gamma matrices indexed as in the module docstring, shape (16, 4, 4)."""
    g = gammas()
    g5 = gamma5()
    out = [np.eye(4, dtype=np.complex128)]
    out += [g[m] for m in range(4)]
    out += [g5]
    out += [g[m] @ g5 for m in range(4)]
    out += [sigma(m, n) for (m, n) in PLANES]
    return np.array(out)


def gamma_tilde(G):
    """Gamma-tilde = gamma_0 Gamma^dagger gamma_0 with gamma_0 = gamma_t (Sec. 2, after Eq. Cdisc)."""
    gt = gammas()[3]
    return gt @ G.conj().T @ gt
