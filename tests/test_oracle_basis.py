"""Pins of the oracle's 1D bases, Gauss rules and SplitMix64 (no GPU)."""
import os

import numpy as np
import pytest

from oracle.basis import gauss01, h1, leg, legendre_xi
from oracle.splitmix import splitmix64, uniform01

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_gauss_exact_up_to_degree_2n_minus_1(n):
    x, w = gauss01(n)
    for k in range(2 * n):
        assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14
    # and not beyond: degree 2n is integrated with an error
    if n <= 5:
        assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-10


def test_legendre_closed_forms():
    xi = np.linspace(-1, 1, 7)
    P, dP = legendre_xi(4, xi)
    assert np.allclose(P[2], (3 * xi ** 2 - 1) / 2, atol=1e-15)
    assert np.allclose(P[3], (5 * xi ** 3 - 3 * xi) / 2, atol=1e-15)
    assert np.allclose(P[4], (35 * xi ** 4 - 30 * xi ** 2 + 3) / 8, atol=1e-15)
    assert np.allclose(dP[3], (15 * xi ** 2 - 3) / 2, atol=1e-14)
    assert np.allclose(dP[4], (140 * xi ** 3 - 60 * xi) / 8, atol=1e-14)


def test_legendre_orthogonality_on_unit_interval():
    x, w = gauss01(10)
    L, _ = leg(7, x)
    M = (L * w) @ L.T
    assert np.allclose(M, np.diag(1.0 / (2 * np.arange(8) + 1)), atol=1e-14)
    L1, _ = leg(7, np.array([0.0, 1.0]))
    assert np.allclose(L1[:, 1], 1.0)
    assert np.allclose(L1[:, 0], (-1.0) ** np.arange(8))


@pytest.mark.parametrize("p", [1, 2, 3, 5])
def test_h1_family(p):
    ends, _ = h1(p, np.array([0.0, 1.0]))
    assert np.allclose(ends[0], [1, 0]) and (p < 1 or np.allclose(ends[1], [0, 1]))
    assert np.allclose(ends[2:], 0.0, atol=1e-15)       # bubbles vanish at both ends
    x = np.linspace(0.013, 0.987, 9)
    V, D = h1(p, x)
    # derivative by central differences
    eps = 1e-6
    Vp, _ = h1(p, x + eps)
    Vm, _ = h1(p, x - eps)
    assert np.allclose(D, (Vp - Vm) / (2 * eps), atol=1e-7)
    # integrated Legendre: phi_k' = 2 (2k-1) P_{k-1}(2x-1) / sqrt(2(2k-1))
    P, _ = legendre_xi(p, 2 * x - 1)
    for k in range(2, p + 1):
        assert np.allclose(D[k], 2 * (2 * k - 1) * P[k - 1] / np.sqrt(2 * (2 * k - 1)), atol=1e-12)
    # the family is a basis of polynomials of degree <= p: Vandermonde is regular
    xs = np.linspace(0, 1, p + 1)
    Vs, _ = h1(p, xs)
    assert abs(np.linalg.det(Vs)) > 1e-6


def test_splitmix64_reference_vectors():
    with open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) as f:
        ref = [int(l) for l in f if l.strip() and not l.startswith("#")]
    assert [splitmix64(1234567, k) for k in range(5)] == ref
    u = [uniform01(7, k) for k in range(1000)]
    assert 0.0 <= min(u) and max(u) < 1.0 and abs(np.mean(u) - 0.5) < 0.05


def test_workload_sign_generator_matches_reference_vectors():
    # the vectorised sign rows of the shared input module take the sign bit of
    # the same SplitMix64 outputs (counter k = row * n + column)
    from paper_2304_01728_gb300.workloads import rademacher_rows
    with open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) as f:
        ref = [int(l) for l in f if l.strip() and not l.startswith("#")]
    signs = rademacher_rows(1234567, 0, 1, 5)[0]
    assert signs.tolist() == [-1.0 if v >> 63 else 1.0 for v in ref]
    rows = rademacher_rows(99, 2, 4, 1000)
    assert rows.shape == (2, 1000) and set(np.unique(rows)) == {-1.0, 1.0}
    assert np.array_equal(rows, rademacher_rows(99, 0, 4, 1000)[2:])
    assert abs(rows.mean()) < 0.1
