"""Pins of the oracle's Dirac matrices: Clifford algebra, Hermiticity, chiral gamma_5, the
Clifford table's trace orthogonality and Gamma-tilde of Sec. 2 (gamma_0 Gamma^dag gamma_0)."""
import numpy as np

from oracle.gamma import gammas, gamma5, sigma, clifford_table, gamma_tilde


def test_clifford_algebra_and_hermiticity():
    g = gammas()
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T)
        for n in range(4):
            assert np.allclose(g[m] @ g[n] + g[n] @ g[m], 2.0 * (m == n) * np.eye(4))


def test_gamma5_chiral():
    g5 = gamma5()
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))
    for m in range(4):
        assert np.allclose(g5 @ gammas()[m], -gammas()[m] @ g5)


def test_sigma_hermitian_block_diagonal():
    for m in range(4):
        for n in range(4):
            s = sigma(m, n)
            assert np.allclose(s, s.conj().T)
            assert np.allclose(s[:2, 2:], 0) and np.allclose(s[2:, :2], 0)


def test_clifford_table_basis():
    T = clifford_table()
    G = np.einsum("aij,bij->ab", T.conj(), T)  # Tr(T_a^dag T_b)
    assert np.allclose(G, 4 * np.eye(16))


def test_gamma_tilde_values():
    T = clifford_table()
    assert np.allclose(gamma_tilde(T[0]), T[0])
    assert np.allclose(gamma_tilde(T[5]), -T[5])  # gamma_5 -> -gamma_5
    for k in (1, 2, 3):
        assert np.allclose(gamma_tilde(T[k]), -T[k])  # gamma_i -> -gamma_i
    assert np.allclose(gamma_tilde(T[4]), T[4])
