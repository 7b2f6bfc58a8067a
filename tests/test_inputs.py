"""Seeded input generators: Philox known answers, SU(3) links, orthonormal colour vectors."""
import os

import numpy as np

from lqcd_inputs import (philox4x32_10, gauge_field, colour_vectors, random_spinors,
                         random_gauge_transform, gell_mann)

HERE = os.path.dirname(__file__)


def test_philox_known_answers():
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        out = philox4x32_10(w[0], w[1], w[2], w[3], w[4], w[5])
        assert [int(o) for o in out] == w[6:10]


def test_gell_mann_algebra():
    l = gell_mann()
    for a in range(8):
        assert np.allclose(l[a], l[a].conj().T)
        assert abs(np.trace(l[a])) < 1e-15
        for b in range(8):
            assert np.isclose(np.trace(l[a] @ l[b]).real, 2.0 * (a == b))


def test_gauge_field_su3_and_deterministic():
    dims = (4, 4, 2, 4)
    U = gauge_field(dims, 0.5, 7)
    I = np.einsum("...ab,...cb->...ac", U, U.conj())
    assert np.abs(I - np.eye(3)).max() < 1e-13
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-13
    assert np.array_equal(U, gauge_field(dims, 0.5, 7))
    assert not np.allclose(U, gauge_field(dims, 0.5, 8))
    # eps -> 0 approaches the unit field
    assert np.abs(gauge_field(dims, 1e-9, 7) - np.eye(3)).max() < 1e-8


def test_colour_vectors_orthonormal_and_subset_consistent():
    dims = (4, 4, 4, 4)
    V = colour_vectors(dims, 6, 11)
    for t in range(4):
        X = V[t].reshape(6, -1)
        assert np.abs(X @ X.conj().T - np.eye(6)).max() < 1e-13
    Vs = colour_vectors(dims, 6, 11, timeslices=[2])
    assert np.array_equal(Vs[0], V[2])


def test_random_fields_shapes():
    psi = random_spinors((2, 2, 2, 4), 3, 1)
    assert psi.shape == (3, 4, 2, 2, 2, 4, 3)
    G = random_gauge_transform((2, 2, 2, 4), 3)
    assert np.abs(np.einsum("...ab,...cb->...ac", G, G.conj()) - np.eye(3)).max() < 1e-13


def test_compiled_philox_words_equal_the_numpy_rounds():
    """The compiled generator used for large lattices gives the numpy version's words bit for bit."""
    import subprocess
    import sys
    from lqcd_inputs import philox
    subprocess.run([sys.executable, os.path.join(os.path.dirname(HERE), "lqcd_inputs", "build.py")], check=True)
    philox._LIB = None
    assert philox._compiled() is not None
    idx = (np.arange(20000, dtype=np.uint64) * np.uint64(2654435761)) ^ np.uint64(0xDEADBEEF12345)
    for seed, purpose in ((7, 1), (2 ** 40 + 3, 2), (5001, 4)):
        a = philox.philox_words(seed, purpose, idx)
        b = philox4x32_10(idx & np.uint64(0xFFFFFFFF), idx >> np.uint64(32), np.uint64(purpose), 0,
                          seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)


def test_compiled_generators_follow_the_numpy_recipe():
    """The compiled Box-Muller normals and SU(3) links (Jacobi eigen-decomposition of H) agree with
    the numpy recipe to round-off, so inputs do not depend on which path drew them."""
    from lqcd_inputs import philox
    from lqcd_inputs.fields import _su3_from_ids
    assert philox._compiled() is not None
    ids = np.arange(50000, dtype=np.uint64) * np.uint64(3) + np.uint64(77)
    a = philox.gaussians(91, 2, ids)
    lib, philox._LIB = philox._LIB, False
    try:
        b = philox.gaussians(91, 2, ids)
        Un = _su3_from_ids(91, 1, ids, 0.6)
    finally:
        philox._LIB = lib
    assert np.abs(a - b).max() < 1e-13
    Uc = _su3_from_ids(91, 1, ids, 0.6)
    assert np.abs(Uc - Un).max() < 1e-13
