"""Pins of oracle.basis against closed forms (GLL points, Gauss exactness, Lagrange identities)."""
import math

import numpy as np
import pytest

from oracle.basis import CellTables, gauss_rule, gll_nodes, lagrange
from oracle.rng import splitmix64_uniform


def test_gll_closed_forms():
    np.testing.assert_allclose(gll_nodes(1), [0.0, 1.0], atol=0)
    np.testing.assert_allclose(gll_nodes(2), [0.0, 0.5, 1.0], atol=1e-15)
    a = 1 / math.sqrt(5)
    np.testing.assert_allclose(gll_nodes(3), [0, (1 - a) / 2, (1 + a) / 2, 1], atol=1e-15)
    b = math.sqrt(3 / 7)
    np.testing.assert_allclose(gll_nodes(4), [0, (1 - b) / 2, 0.5, (1 + b) / 2, 1], atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_gauss_exactness(n):
    x, w = gauss_rule(n)
    for p in range(2 * n):
        assert abs(np.sum(w * x**p) - 1.0 / (p + 1)) < 1e-14
    # degree 2n is not integrated exactly
    assert abs(np.sum(w * x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-6


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_lagrange_identities(k):
    nodes = gll_nodes(k)
    V, D = lagrange(nodes, nodes)
    np.testing.assert_allclose(V, np.eye(k + 1), atol=1e-14)
    xs = np.linspace(-0.3, 1.2, 17)
    V, D = lagrange(nodes, xs)
    np.testing.assert_allclose(V.sum(1), 1.0, atol=1e-12)
    np.testing.assert_allclose(D.sum(1), 0.0, atol=1e-10)
    for p in range(k + 1):  # x^p is reproduced with its derivative
        np.testing.assert_allclose(V @ nodes**p, xs**p, atol=1e-12)
        np.testing.assert_allclose(D @ nodes**p, p * xs ** max(p - 1, 0) if p else 0 * xs, atol=1e-11)


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (2, 4), (3, 1), (3, 2), (3, 3)])
def test_cell_tables(dim, k):
    t = CellTables(dim, k)
    np.testing.assert_allclose(t.N.sum(1), 1.0, atol=1e-13)
    np.testing.assert_allclose(t.dN.sum(1), 0.0, atol=1e-11)
    assert abs(t.w.sum() - 1.0) < 1e-14
    # interpolate f = prod_i x_i^{p_i} (p_i <= k) at the nodes; integrate f and df/dx_0 exactly
    nodes = gll_nodes(k)
    grids = np.meshgrid(*([nodes] * dim), indexing="ij")
    coords = [g.transpose(tuple(range(dim))[::-1]).reshape(-1) for g in grids]
    p = [min(k, i + 1) for i in range(dim)]
    f = np.prod([coords[i] ** p[i] for i in range(dim)], axis=0)
    exact = np.prod([1.0 / (pi + 1) for pi in p])
    assert abs(t.w @ (t.N @ f) - exact) < 1e-14
    dexact = np.prod([1.0 / (p[i] + 1) if i else 1.0 for i in range(dim)])  # int d/dx0 x0^p0 = 1
    assert abs(t.w @ (t.dN[:, :, 0] @ f) - dexact) < 1e-12


def test_splitmix64_published_vector():
    # SplitMix64 seeded with 0: first outputs 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4
    u = splitmix64_uniform(0, 2)
    for val, ref in zip(u, (0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4)):
        assert val == 2.0 * ((ref >> 11) * 2.0**-53) - 1.0
