"""Q_k Lagrange basis on GLL nodes with the (k+1)-point Gauss rule (Sec. 5, Tables 1-2: q = p + 1).

Test infrastructure (see oracle/__init__.py). Built directly from the definitions:
Lagrange polynomials by their product formula, tensor-product tables by explicit
products over all (quadrature point, node) multi-index pairs -- no sum factorisation.
"""
from __future__ import annotations

import itertools

import numpy as np
from numpy.polynomial import legendre


def gll_nodes(k: int) -> np.ndarray:
    """k+1 Gauss-Lobatto-Legendre points on [0,1]: the end points and the roots of P_k'."""
    if k < 1:
        raise ValueError("degree must be >= 1")
    inner = np.zeros(0) if k == 1 else np.sort(np.real(legendre.Legendre.basis(k).deriv().roots()))
    return 0.5 * (np.concatenate(([-1.0], inner, [1.0])) + 1.0)


def gauss_rule(n: int):
    """n-point Gauss-Legendre rule on [0,1] (points, weights)."""
    x, w = legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange(nodes: np.ndarray, x: np.ndarray):
    """V[p, j] = l_j(x_p) and D[p, j] = l_j'(x_p) for the Lagrange polynomials l_j on `nodes`."""
    nodes = np.asarray(nodes, dtype=float)
    x = np.atleast_1d(np.asarray(x, dtype=float))
    n = len(nodes)
    V = np.ones((len(x), n))
    D = np.zeros((len(x), n))
    for j in range(n):
        for mm in range(n):
            if mm != j:
                V[:, j] *= (x - nodes[mm]) / (nodes[j] - nodes[mm])
        for mm in range(n):
            if mm == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[mm]))
            for ll in range(n):
                if ll != j and ll != mm:
                    term *= (x - nodes[ll]) / (nodes[j] - nodes[ll])
            D[:, j] += term
    return V, D


class CellTables:
    """Full tensor-product tables on the unit cell [0,1]^dim.

    N[q, a]      value of node a's shape function at quadrature point q
    dN[q, a, J]  derivative of that shape function along reference axis J
    w[q]         quadrature weight (sum = 1)
    Multi-indices are flattened with axis 0 (x) fastest, for nodes and points alike.
    """

    def __init__(self, dim: int, k: int):
        self.dim, self.k, self.n = dim, k, k + 1
        nodes = gll_nodes(k)
        xq, wq = gauss_rule(k + 1)
        V, D = lagrange(nodes, xq)
        n = k + 1
        nq = n**dim
        self.N = np.zeros((nq, nq))
        self.dN = np.zeros((nq, nq, dim))
        self.w = np.zeros(nq)
        multi = list(itertools.product(range(n), repeat=dim))
        flat = lambda t: sum(t[i] * n**i for i in range(dim))  # noqa: E731  (x fastest)
        for qt in multi:
            q = flat(qt)
            self.w[q] = np.prod([wq[qt[i]] for i in range(dim)])
            for at in multi:
                a = flat(at)
                self.N[q, a] = np.prod([V[qt[i], at[i]] for i in range(dim)])
                for J in range(dim):
                    self.dN[q, a, J] = np.prod(
                        [D[qt[i], at[i]] if i == J else V[qt[i], at[i]] for i in range(dim)])
        self.nodes_1d, self.xq_1d, self.wq_1d = nodes, xq, wq
