"""Pins of the oracle's Wilson-clover operator (Sec. 2.1, Sec. 3) and its domain restriction.

Each test checks the oracle against something it does not compute itself: momentum-space closed
forms for free and constant-U(1) fields, the abelian clover closed form evaluated by explicit
coordinate loops, gauge covariance, the independently coded adjoint, and the dense block
structure required of D_Lambda."""
import itertools

import numpy as np
import pytest

from lqcd_inputs import gauge_field, unit_gauge_field, random_spinors, random_gauge_transform
from oracle.dirac import (WilsonClover, BC_ANTIPERIODIC, BC_PERIODIC, BC_OPEN, eo_order,
                          parity_table, domain_of_t, cut_after, coords)
from oracle.gamma import gammas, gamma5, sigma, PLANES

KAPPA, CSW = 0.12, 1.5


def _plane_wave(dims, p):
    Lx, Ly, Lz, Lt = dims
    t, z, y, x = np.meshgrid(np.arange(Lt), np.arange(Lz), np.arange(Ly), np.arange(Lx),
                             indexing="ij")
    return np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))


def _Dp(p, kappa):
    """Free Wilson operator in momentum space: 1 - 2 kappa sum cos p + 2 i kappa sum gamma sin p."""
    g = gammas()
    return np.eye(4) * (1 - 2 * kappa * np.cos(p).sum()) + 2j * kappa * sum(
        g[m] * np.sin(p[m]) for m in range(4))


@pytest.mark.parametrize("bc", [BC_ANTIPERIODIC, BC_PERIODIC])
def test_free_field_plane_waves(bc):
    dims = (4, 2, 4, 6)
    op = WilsonClover(unit_gauge_field(dims), KAPPA, CSW, bc)
    rng = np.random.default_rng(0)
    for n in [(0, 0, 0, 0), (1, 1, 2, 1), (3, 0, 1, 5)]:
        p = np.array([2 * np.pi * n[0] / 4, 2 * np.pi * n[1] / 2, 2 * np.pi * n[2] / 4,
                      (2 * n[3] + (1 if bc == BC_ANTIPERIODIC else 0) * 1.0) * np.pi / 6
                      if bc == BC_ANTIPERIODIC else 2 * np.pi * n[3] / 6])
        u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
        f = _plane_wave(dims, p)[..., None, None] * u
        want = _plane_wave(dims, p)[..., None, None] * (_Dp(p, KAPPA) @ u)
        assert np.abs(op.apply(f) - want).max() < 1e-13


def test_open_bc_removes_wrap_hop():
    dims = (2, 2, 2, 4)
    U = gauge_field(dims, 0.4, 3)
    D = WilsonClover(U, KAPPA, CSW, BC_OPEN).dense()
    t = coords(dims)[3]
    rows = np.repeat(t, 12)
    assert np.abs(D[np.ix_(rows == 3, rows == 0)]).max() == 0
    assert np.abs(D[np.ix_(rows == 0, rows == 3)]).max() == 0


def test_constant_u1_twist():
    """U_mu = exp(i theta_mu) (constant): D e^{ipx} u = e^{ipx} D(p + theta) u; F = 0."""
    dims = (4, 4, 2, 4)
    theta = np.array([0.3, -0.7, 1.1, 0.25])
    U = unit_gauge_field(dims) * np.exp(1j * theta)[None, None, None, None, :, None, None]
    op = WilsonClover(U, KAPPA, CSW, BC_ANTIPERIODIC)
    p = np.array([2 * np.pi / 4, 0.0, np.pi, 3 * np.pi / 4])
    u = np.arange(12).reshape(4, 3) * (1 + 0.5j)
    f = _plane_wave(dims, p)[..., None, None] * u
    want = _plane_wave(dims, p)[..., None, None] * (_Dp(p + theta, KAPPA) @ u)
    assert np.abs(op.apply(f) - want).max() < 1e-12


def test_abelian_clover_closed_form():
    """For U_mu(x) = exp(i phi_mu(x)) 1_3 the clover term is
    A = 1 - (kappa c_sw / 4) sum_{mu<nu} sigma_{mu nu} sum_{4 plaquettes} sin(theta_{mu nu}),
    plaquettes based at x, x-mu, x-mu-nu, x-nu; evaluated here with explicit coordinates."""
    dims = (4, 2, 2, 4)
    Lx, Ly, Lz, Lt = dims
    L = np.array(dims)
    rng = np.random.default_rng(1)
    phi = rng.uniform(-np.pi, np.pi, size=(Lt, Lz, Ly, Lx, 4))
    U = np.exp(1j * phi)[..., None, None] * np.eye(3)
    A = WilsonClover(U, KAPPA, CSW).A

    def ph(c, mu):
        c = np.mod(c, L)
        return phi[c[3], c[2], c[1], c[0], mu]

    e = np.eye(4, dtype=int)
    for c in itertools.product(range(Lx), range(Ly), range(Lz), range(Lt)):
        c = np.array(c)
        want = np.eye(12, dtype=complex)
        for (mu, nu) in PLANES:
            s = 0.0
            for base in (c, c - e[mu], c - e[mu] - e[nu], c - e[nu]):
                th = ph(base, mu) + ph(base + e[mu], nu) - ph(base + e[nu], mu) - ph(base, nu)
                s += np.sin(th)
            want += -(KAPPA * CSW / 4.0) * s * np.kron(sigma(mu, nu), np.eye(3))
        assert np.abs(A[c[3], c[2], c[1], c[0]] - want).max() < 1e-13


def test_adjoint_and_gamma5_hermiticity():
    dims = (4, 4, 4, 4)
    op = WilsonClover(gauge_field(dims, 0.5, 5), 0.125, 1.6)
    x = random_spinors(dims, 1, 1)[0]
    y = random_spinors(dims, 1, 2)[0]
    lhs = np.vdot(y, op.apply(x))
    assert abs(lhs - np.vdot(op.apply_dagger(y), x)) < 1e-12 * abs(lhs)
    g5 = lambda p: np.matmul(gamma5(), p)
    assert np.abs(g5(op.apply(g5(x))) - op.apply_dagger(x)).max() < 1e-13


def test_clover_hermitian_chiral():
    op = WilsonClover(gauge_field((4, 4, 2, 4), 0.6, 9), 0.126, 1.7)
    A = op.A
    assert np.abs(A - np.conj(np.swapaxes(A, -1, -2))).max() < 1e-15
    G5 = np.kron(gamma5(), np.eye(3))
    assert np.abs(A @ G5 - G5 @ A).max() < 1e-15
    assert np.abs(A - np.eye(12)).max() > 1e-2  # a rough field gives a non-trivial clover term


@pytest.mark.parametrize("bc", [BC_ANTIPERIODIC, BC_OPEN])
def test_gauge_covariance(bc):
    dims = (4, 2, 4, 4)
    U = gauge_field(dims, 0.5, 21)
    G = random_gauge_transform(dims, 22)
    Gsh = {0: np.roll(G, -1, 3), 1: np.roll(G, -1, 2), 2: np.roll(G, -1, 1), 3: np.roll(G, -1, 0)}
    UG = np.stack([G @ U[:, :, :, :, mu] @ np.conj(np.swapaxes(Gsh[mu], -1, -2))
                   for mu in range(4)], axis=4)
    psi = random_spinors(dims, 1, 3)[0]
    rot = lambda p: np.matmul(p, np.swapaxes(G, -1, -2))  # (G psi)_{s a} = G_ab psi_{s b}
    for ext in (None, [2, 2]):
        op = WilsonClover(U, 0.125, 1.6, bc, ext)
        opG = WilsonClover(UG, 0.125, 1.6, bc, ext)
        assert np.abs(opG.apply(rot(psi)) - rot(op.apply(psi))).max() < 1e-13


def test_geometry_tables():
    dims = (4, 2, 4, 6)
    par = parity_table(dims)
    perm, cb = eo_order(dims)
    V = 4 * 2 * 4 * 6
    assert sorted(perm) == list(range(V))
    assert np.all(par[perm[: V // 2]] == 0) and np.all(par[perm[V // 2:]] == 1)
    assert np.array_equal(cb, np.arange(V) >> 1)  # checkerboard index is s >> 1 for even Lx
    assert list(domain_of_t([2, 4, 2, 4], 12)) == [0, 0, 1, 1, 1, 1, 2, 2, 3, 3, 3, 3]
    assert list(np.nonzero(cut_after([2, 4, 2, 4], 12))[0]) == [1, 5, 7, 11]
    assert not cut_after([12], 12).any()
    with pytest.raises(ValueError):
        domain_of_t([4, 4], 12)
    # shifted tilings (regions placed around chosen x0, y0): the last domain wraps around
    assert list(domain_of_t([3, 5], 8, t_start=6)) == [0, 1, 1, 1, 1, 1, 0, 0]
    assert list(np.nonzero(cut_after([3, 5], 8, t_start=6))[0]) == [0, 5]
    assert list(domain_of_t([2, 4, 2, 4], 12, 3)) == [3, 3, 3, 0, 0, 1, 1, 1, 1, 2, 2, 3]
    assert list(np.nonzero(cut_after([2, 4, 2, 4], 12, 3))[0]) == [2, 4, 8, 10]
    with pytest.raises(ValueError):
        domain_of_t([4, 4], 8, t_start=8)


def test_domain_operator_block_structure():
    """D_Lambda = D with every matrix element between different domains removed; one domain = D."""
    dims = (2, 2, 2, 8)
    U = gauge_field(dims, 0.5, 31)
    op = WilsonClover(U, 0.125, 1.6)
    D = op.dense()
    t = np.repeat(coords(dims)[3], 12)
    for ext, t0 in (([2, 4, 2], 0), ([3, 5], 0), ([1, 7], 0), ([3, 5], 6), ([2, 4, 2], 7), ([1, 7], 3)):
        dom = domain_of_t(ext, 8, t0)[t]
        want = np.where(dom[:, None] == dom[None, :], D, 0)
        assert np.abs(op.restricted(ext, t0).dense() - want).max() == 0
    assert np.abs(op.restricted([8]).dense() - D).max() == 0
    assert np.abs(op.restricted([8], 5).dense() - D).max() == 0


@pytest.mark.parametrize("shift", [1, 3, 6])
def test_shifted_tiling_translation_covariance(shift):
    """With periodic time boundary conditions, translating the gauge field, the spinor and the
    tiling by the same number of timeslices commutes with D_Lambda: D_Lambda[T U, t_start = s]
    (T psi) = T (D_Lambda[U, t_start = 0] psi), (T f)(t) = f(t - s)."""
    dims = (2, 2, 4, 8)
    U = gauge_field(dims, 0.5, 57)
    psi = random_spinors(dims, 2, 58)
    ext = [3, 5]
    ref = WilsonClover(U, KAPPA, CSW, BC_PERIODIC, ext).apply(psi)
    Us = np.roll(U, shift, axis=0)
    got = WilsonClover(Us, KAPPA, CSW, BC_PERIODIC, ext, t_start=shift).apply(np.roll(psi, shift, axis=1))
    assert np.abs(got - np.roll(ref, shift, axis=1)).max() < 1e-13


def test_schur_factorisation_of_propagator():
    """Eq. (factorisation), read as the Schur complement: for x0 in Lambda,
    (D^-1)_LL = D_L^-1 + D_L^-1 D_{L L*} (D^-1)_{L* L*} D_{L* L} D_L^-1."""
    dims = (2, 2, 2, 8)
    op = WilsonClover(gauge_field(dims, 0.5, 41), 0.125, 1.6)
    D = op.dense()
    Dinv = np.linalg.inv(D)
    t = np.repeat(coords(dims)[3], 12)
    lam = t < 3
    DL = op.restricted([3, 5]).dense()[np.ix_(lam, lam)]
    DLi = np.linalg.inv(DL)
    B = D[np.ix_(lam, ~lam)]
    C = D[np.ix_(~lam, lam)]
    rhs = DLi + DLi @ B @ Dinv[np.ix_(~lam, ~lam)] @ C @ DLi
    assert np.abs(Dinv[np.ix_(lam, lam)] - rhs).max() < 1e-11
    # the correction term is what the domain loop leaves out; it is not negligible here
    assert np.abs(Dinv[np.ix_(lam, lam)] - DLi).max() > 1e-6


def test_single_site_operator_equals_the_lattice_operator():
    """apply_at_sites (per-site leaves and hops from explicit coordinates, for lattices too large
    for the whole-lattice oracle) agrees with WilsonClover on a ragged lattice, for every time
    boundary condition, with and without a shifted domain tiling."""
    from lqcd_inputs import gauge_field, random_spinors
    from oracle.dirac import WilsonClover, apply_at_sites
    dims = (4, 6, 2, 8)
    U = gauge_field(dims, 0.4, 11)
    psi = random_spinors(dims, 1, 12)[0]
    sites = [(x, y, z, t) for t in range(8) for z in range(2) for y in range(6) for x in range(4)][::5]
    for bc in (0, 1, 2):
        for ext, ts in ((None, 0), ([3, 5], 2)):
            op = WilsonClover(U, 0.13, 1.7, bc, ext, ts)
            full = op.apply(psi[None])[0]
            loc = apply_at_sites(U, 0.13, 1.7, psi, sites, bc, ext, ts)
            ref = np.array([full[t, z, y, x] for (x, y, z, t) in sites])
            assert np.abs(loc - ref).max() <= 1e-14 * np.abs(ref).max()
