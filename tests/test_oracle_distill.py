"""Pins of the oracle's distillation, loops and correlators (Sec. 2, Sec. 3.1-3.2, Sec. 4)."""
import itertools

import numpy as np
import pytest

from lqcd_inputs import gauge_field, unit_gauge_field, random_gauge_transform, colour_vectors
from oracle.dirac import WilsonClover
from oracle.gamma import gammas, clifford_table
from oracle.distill import (laplacian3d, laplace_eigs, perambulators, loops, point_loops,
                            disc_correlators, profile_weights, effective_mass, conn_correlator,
                            point_conn_correlator, nr_estimator)


def test_free_laplacian_spectrum():
    dims = (4, 4, 2, 2)
    lam, V = laplace_eigs(unit_gauge_field(dims), 3 * 4 * 4 * 2, timeslices=[0])
    want = sorted(
        sum(2 - 2 * np.cos(2 * np.pi * n[k] / dims[k]) for k in range(3))
        for n in itertools.product(range(4), range(4), range(2)) for _ in range(3))
    assert np.abs(lam[0] - np.array(want)).max() < 1e-12


def test_laplacian_eigvecs_random_field():
    dims = (4, 4, 4, 2)
    U = gauge_field(dims, 0.5, 61)
    lam, V = laplace_eigs(U, 8)
    for t in range(2):
        X = V[t].reshape(8, -1)
        assert np.abs(X @ X.conj().T - np.eye(8)).max() < 1e-12
        res = laplacian3d(U, t, V[t]) - lam[t][:, None, None, None, None] * V[t]
        assert np.abs(res).max() < 1e-12
        k = np.argmax(np.abs(X), axis=1)
        ph = X[np.arange(8), k]
        assert np.all(np.abs(ph.imag) < 1e-15) and np.all(ph.real > 0)
    assert np.all(np.diff(lam, axis=1) >= 0) and lam.min() > 0


def test_free_field_perambulator_closed_form():
    """Plane-wave sources v_i = e^{i p.x} e_c / sqrt(L^3) in the free field give
    tau^{ij}(t,t) = delta_ij (1/T) sum_{p_t} D(p_t, p)^{-1} (antiperiodic p_t)."""
    dims = (4, 4, 2, 6)
    Lx, Ly, Lz, Lt = dims
    kappa = 0.11
    op = WilsonClover(unit_gauge_field(dims), kappa, 1.2)
    z, y, x = np.meshgrid(np.arange(Lz), np.arange(Ly), np.arange(Lx), indexing="ij")
    modes = [((0, 0, 0), 0), ((1, 0, 1), 2), ((3, 1, 0), 1)]
    V1 = np.zeros((3, Lz, Ly, Lx, 3), dtype=complex)
    for i, (n, c) in enumerate(modes):
        V1[i, ..., c] = np.exp(2j * np.pi * (n[0] * x / Lx + n[1] * y / Ly + n[2] * z / Lz))
    V1 /= np.sqrt(Lx * Ly * Lz)
    V = np.repeat(V1[None], Lt, axis=0)
    tau = perambulators(op, V, [0, 3], tol=1e-13)
    g = gammas()
    for i, (n, c) in enumerate(modes):
        S = np.zeros((4, 4), dtype=complex)
        for nt in range(Lt):
            p = np.array([2 * np.pi * n[0] / Lx, 2 * np.pi * n[1] / Ly, 2 * np.pi * n[2] / Lz,
                          (2 * nt + 1) * np.pi / Lt])
            Dp = np.eye(4) * (1 - 2 * kappa * np.cos(p).sum()) + 2j * kappa * sum(
                g[m] * np.sin(p[m]) for m in range(4))
            S += np.linalg.inv(Dp) / Lt
        for k in range(2):
            assert np.abs(tau[k, i, :, i, :] - S).max() < 1e-12
            for j in range(3):
                if j != i:
                    assert np.abs(tau[k, i, :, j, :]).max() < 1e-12


def test_complete_basis_loops_equal_point_traces():
    """With N_ev = 3 L^3 eigenvectors the distilled loop is sum_xvec Tr[Gamma D^{-1}(x,x)]."""
    dims = (2, 2, 2, 4)
    U = gauge_field(dims, 0.5, 71)
    op = WilsonClover(U, 0.125, 1.6)
    lam, V = laplace_eigs(U, 24)
    tau = perambulators(op, V, range(4), tol=1e-13)
    gids = list(range(16))
    L, Lt = loops(tau, gids)
    Dinv = np.linalg.inv(op.dense())
    n = 12
    blocks = np.array([Dinv[s * n:(s + 1) * n, s * n:(s + 1) * n] for s in range(32)])
    P = point_loops(blocks.reshape(4, 2, 2, 2, 12, 12), gids)
    assert np.abs(L - P).max() < 1e-11 * np.abs(P).max()


def test_complete_basis_connected_correlator_equals_point_contraction():
    """With N_ev = 3 L^3 the distilled connected correlator -Tr[G tau(x0,y0) Gt tau(y0,x0)] is the
    point-source one, -sum_{xvec,yvec} Tr[G D^-1(x,y) Gt D^-1(y,x)], from dense LU; and the
    hermiticity tau(y0,x0) = g5 tau(x0,y0)^dag g5 holds between the all-sink perambulators."""
    dims = (2, 2, 2, 4)
    U = gauge_field(dims, 0.5, 73)
    op = WilsonClover(U, 0.125, 1.6)
    lam, V = laplace_eigs(U, 24)
    tau = perambulators(op, V, range(4), sinks="all", tol=1e-13)
    gids = [5, 0, 1, 13]
    C, C_avg = conn_correlator(tau, list(range(4)), gids)
    P = point_conn_correlator(np.linalg.inv(op.dense()), dims, gids)
    assert np.abs(C - P).max() < 1e-11 * np.abs(P).max()
    eps = np.array([1, 1, -1, -1])
    A = tau[0, 2]  # tau(2, 0)
    B = tau[2, 0]  # tau(0, 2)
    want = np.einsum("c,d,idjc->jcid", eps, eps, np.conj(A))
    assert np.abs(B - want).max() < 1e-11 * np.abs(B).max()
    assert np.allclose(C_avg[:, 1], np.mean([C[:, (y + 1) % 4, y] for y in range(4)], axis=0))
    # pseudoscalar: Gt(g5) = -g5, so C = +Tr[S(x,y) S(x,y)^dag] > 0
    assert np.abs(C[0].imag).max() < 1e-11 * np.abs(C[0]).max() and np.all(C[0].real > 0)


def test_nr_estimator_selects_block_size_per_separation():
    T = 6
    conn = np.arange(2 * T).reshape(2, T).astype(complex)
    disc = 100 + np.zeros((2, T), complex)
    dC = np.array([1000 + np.zeros((2, T)), 2000 + np.zeros((2, T))], dtype=complex)
    out = nr_estimator(conn, disc, dC, [-1, -1, 0, 0, 1, 1])
    assert np.array_equal(out[:, :2], conn[:, :2] + 100)
    assert np.array_equal(out[:, 2:4], conn[:, 2:4] + 1000)
    assert np.array_equal(out[:, 4:], conn[:, 4:] + 2000)


def test_loops_gauge_invariant_and_real():
    dims = (4, 2, 2, 4)
    U = gauge_field(dims, 0.5, 81)
    V = colour_vectors(dims, 3, 82)
    G = random_gauge_transform(dims, 83)
    Gsh = {0: np.roll(G, -1, 3), 1: np.roll(G, -1, 2), 2: np.roll(G, -1, 1), 3: np.roll(G, -1, 0)}
    UG = np.stack([G @ U[:, :, :, :, mu] @ np.conj(np.swapaxes(Gsh[mu], -1, -2))
                   for mu in range(4)], axis=4)
    VG = np.einsum("tzyxab,tizyxb->tizyxa", G, V)
    gids = [0, 1, 2, 3, 5]
    L, Lt = loops(perambulators(WilsonClover(U, 0.125, 1.6), V, [1, 2]), gids)
    LG, LtG = loops(perambulators(WilsonClover(UG, 0.125, 1.6), VG, [1, 2]), gids)
    assert np.abs(L - LG).max() < 1e-11
    # gamma_5-hermiticity: L_1, L_g5 real; L_gi imaginary (i = x, y, z)
    assert np.abs(L[[0, 4]].imag).max() < 1e-11 < np.abs(L[[0, 4]].real).max()
    assert np.abs(L[[1, 2, 3]].real).max() < 1e-11
    assert np.allclose(Lt[4], -L[4]) and np.allclose(Lt[0], L[0])


def test_profile_weights():
    lam = np.array([0.0, 0.05, 0.2])
    w = profile_weights(lam, 0.05)
    assert w[0] == 1.0
    assert np.isclose(w[1], np.exp(-(0.05 ** 2) / (0.8 * 0.05) ** 2))


def _random_loops(n_cfg, n_g, T, seed):
    rng = np.random.default_rng(seed)
    c = lambda: rng.normal(size=(n_cfg, n_g, T)) + 1j * rng.normal(size=(n_cfg, n_g, T))
    return c(), c(), c(), c()


def test_correlators_against_numpy_covariance():
    L, Lt, Ld, Ltd = _random_loops(7, 2, 8, 0)
    r = disc_correlators(L, Lt, Ld, Ltd, [4, 4], vev=True)
    for g in range(2):
        for x0, y0 in [(0, 5), (3, 3), (7, 1)]:
            cov = np.cov(L[:, g, x0], np.conj(Lt[:, g, y0]), bias=True)[0, 1]
            assert np.isclose(r["C"][g, x0, y0], cov, rtol=1e-13)
            covd = np.cov(Ld[:, g, x0], np.conj(Ltd[:, g, y0]), bias=True)[0, 1]
            assert np.isclose(r["dC"][g, x0, y0], cov - covd, rtol=1e-12)
    assert r["valid"][0, 5] == 1 and r["valid"][0, 3] == 0
    # the four pieces of Eqs. corr1-corr4 add up to the full correlator (L = L_Lambda + dL)
    assert np.abs(r["terms"].sum(0) - r["C"]).max() < 1e-13
    assert np.abs(r["terms"][0] - r["C_dd"]).max() < 1e-15


def test_subtracted_correlator_vanishes_without_domains():
    L, Lt, _, _ = _random_loops(5, 1, 6, 1)
    r = disc_correlators(L, Lt, L, Lt, [6], vev=True)
    assert np.abs(r["dC"]).max() == 0
    assert r["n_valid"].sum() == 0


def test_source_average_of_translation_invariant_correlator():
    """C(x0,y0) = f(x0 - y0) -> the y0-average returns f; VEV subtraction removes constants."""
    T, n_cfg = 6, 4
    rng = np.random.default_rng(2)
    a = rng.normal(size=n_cfg)
    f = rng.normal(size=T)
    # L(x0) = a_c e^{i k x0}, Lt(y0) = a_c e^{-i k y0}: <L Lt> - <L><Lt> = var(a) e^{i k (x0-y0)}
    k = 2 * np.pi / T
    L = (a[:, None] * np.exp(1j * k * np.arange(T)))[:, None, :] + 3.0
    Lt = (a[:, None] * np.exp(-1j * k * np.arange(T)))[:, None, :] - 1.0
    r = disc_correlators(L, Lt, L, Lt, [3, 3], vev=True)
    want = np.var(a) * np.exp(1j * k * np.arange(T))
    assert np.abs(r["C_avg"][0] - want).max() < 1e-13
    del f


def test_effective_mass_of_exponential():
    C = 3.0 * np.exp(-0.7 * np.arange(6))
    assert np.allclose(effective_mass(C), 0.7)


def test_window_average_closed_forms():
    """Bulk-window averages (Sec. 3 / Sec. 4 restrict x0, y0 to the bulk): a translation-invariant
    correlator f(x0 - y0) averages to f(dt) with t_hi - t_lo + 1 - dt pairs; pairs in one domain
    are excluded from dC only; the full window with a periodic f reproduces the non-wrapping part
    of the all-y0 average."""
    from oracle.distill import window_average
    T, lo, hi = 16, 3, 12
    f = np.exp(-0.3 * np.arange(T)) + 0.1j * np.arange(T)
    x0, y0 = np.meshgrid(np.arange(T), np.arange(T), indexing="ij")
    C = f[(x0 - y0) % T][None].repeat(2, axis=0)
    C[1] *= 2.0
    dC = 3.0 * C
    dom = np.repeat(np.arange(4), 4)
    valid = (dom[:, None] != dom[None, :]).astype(np.int32)
    w = window_average(C, dC, valid, lo, hi)
    n = hi - lo + 1
    for dt in range(T):
        assert w["n_pairs"][dt] == max(0, n - dt)
        if dt < n:
            assert np.allclose(w["C_avg"][:, dt], [f[dt], 2 * f[dt]])
        else:
            assert np.all(w["C_avg"][:, dt] == 0)
        brute = sum(1 for y in range(lo, hi + 1) if y + dt <= hi and dom[y + dt] != dom[y])
        assert w["n_valid"][dt] == brute
        if brute:
            assert np.allclose(w["dC_avg"][:, dt], [3 * f[dt], 6 * f[dt]])
    # a pair inside one domain never enters dC: make those entries huge
    dC2 = dC.copy()
    dC2[:, valid == 0] = 1e30
    assert np.allclose(window_average(C, dC2, valid, lo, hi)["dC_avg"], w["dC_avg"])
    with pytest.raises(ValueError):
        window_average(C, dC, valid, 5, 4)
