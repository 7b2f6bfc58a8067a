"""Pins of the oracle solvers: CGNR against dense LU, and the free-field propagator
S(x,y) = (1/V) sum_p e^{ip(x-y)} D(p)^{-1} (antiperiodic p_t = (2n+1) pi / T)."""
import itertools

import numpy as np

from lqcd_inputs import gauge_field, unit_gauge_field, random_spinors
from oracle.dirac import WilsonClover
from oracle.gamma import gammas
from oracle.solve import cgnr, dense_solve


def test_cgnr_matches_dense_lu():
    dims = (4, 4, 4, 4)
    op = WilsonClover(gauge_field(dims, 0.5, 51), 0.125, 1.6)
    b = random_spinors(dims, 2, 52)
    x, info = cgnr(op, b, tol=1e-13)
    assert np.all(info["true_resid"] <= 1e-13)
    xd = dense_solve(op.dense(), b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-12


def test_cgnr_domain_operator_matches_dense_lu():
    dims = (2, 2, 2, 8)
    op = WilsonClover(gauge_field(dims, 0.5, 53), 0.125, 1.6).restricted([2, 6])
    b = random_spinors(dims, 1, 54)
    x, info = cgnr(op, b, tol=1e-13)
    assert np.linalg.norm(x - dense_solve(op.dense(), b)) / np.linalg.norm(x) < 1e-12


def test_free_propagator_closed_form():
    dims = (2, 2, 4, 6)
    Lx, Ly, Lz, Lt = dims
    kappa = 0.11
    op = WilsonClover(unit_gauge_field(dims), kappa, 1.0)
    beta = 2
    b = np.zeros((1, Lt, Lz, Ly, Lx, 4, 3), dtype=complex)
    b[0, 0, 0, 0, 0, beta, 1] = 1.0  # point source at the origin, spin beta, colour 1
    x, info = cgnr(op, b, tol=1e-13)
    g = gammas()
    S = np.zeros((Lt, Lz, Ly, Lx, 4), dtype=complex)
    t, z, y, xx = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx),
                              indexing="ij")
    for n in itertools.product(range(Lx), range(Ly), range(Lz), range(Lt)):
        p = np.array([2 * np.pi * n[0] / Lx, 2 * np.pi * n[1] / Ly, 2 * np.pi * n[2] / Lz,
                      (2 * n[3] + 1) * np.pi / Lt])
        Dp = np.eye(4) * (1 - 2 * kappa * np.cos(p).sum()) + 2j * kappa * sum(
            g[m] * np.sin(p[m]) for m in range(4))
        col = np.linalg.inv(Dp)[:, beta]
        ph = np.exp(1j * (p[0] * xx + p[1] * y + p[2] * z + p[3] * t))
        S += ph[..., None] * col / (Lx * Ly * Lz * Lt)
    assert np.abs(x[0, ..., 1] - S).max() < 1e-12
    assert np.abs(x[0, ..., 0]).max() < 1e-14  # colour is untouched by the free field
