"""Values the paper prints (tests/golden/, each file citing its source).

Tables 1-2 (Sec. 7) list the benchmark's degree p, quadrature points q, refinements and the element and
DoF counts of the paper's own mesh (its geometry is not available). What they fix, and what is checked:
* q = p + 1 Gauss points per direction (reading O5), which the oracle's element tables use;
* uniform refinement: N_el = N_el,0 * 2^(dim * N_gref) with one coarse-mesh size per dimension;
* the DoF count of a continuous Q_p vector field depends only on p * 2^N_gref (a Q_p space on a mesh equals
  the Q_1 space on that mesh refined p times, node for node), which the lattice count of this repository
  obeys too: n_dofs(dim, p, m) = n_dofs(dim, 1, p m).
"""
import os

import numpy as np
import pytest

from oracle.basis import CellTables
from paper_1904_13131_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def table_rows():
    rows = []
    with open(os.path.join(GOLDEN, "paper_tables_1_2.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(v) for v in line.split()))
    return rows


def test_quadrature_points_per_degree():
    rows = table_rows()
    assert len(rows) == 12
    for dim, p, q, _, _, _ in rows:
        assert q == p + 1
        if p <= 4:
            t = CellTables(dim, p)
            assert t.n == q and len(t.wq_1d) == q and t.w.shape == (q**dim,)
            # a q-point Gauss rule integrates x^(2q-1) exactly on [0, 1]
            assert np.dot(t.wq_1d, t.xq_1d ** (2 * q - 1)) == pytest.approx(1.0 / (2 * q), rel=1e-14)


def test_uniform_refinement_of_one_coarse_mesh():
    for dim in (2, 3):
        coarse = {n_el // 2 ** (dim * g) for d, _, _, g, n_el, _ in table_rows() if d == dim}
        assert len(coarse) == 1  # 88 quadrilaterals in 2D, 352 hexahedra in 3D
        for d, _, _, g, n_el, _ in table_rows():
            if d == dim:
                assert n_el % 2 ** (dim * g) == 0


def test_dofs_depend_on_degree_times_refinement_only():
    by_level = {}
    for dim, p, _, g, _, n_dof in table_rows():
        by_level.setdefault((dim, p * 2**g), set()).add(n_dof)
    assert all(len(v) == 1 for v in by_level.values())
    assert len([k for k in by_level if k[0] == 2]) < 8  # the table does repeat levels (128, 96)
    for dim in (2, 3):
        for p in (1, 2, 3, 4):
            for m in (1, 2, 3, 5):
                assert inputs.n_dofs(dim, p, m) == inputs.n_dofs(dim, 1, p * m)
