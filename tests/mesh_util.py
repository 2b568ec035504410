"""Lattice helpers shared by tests (no arithmetic of the method)."""


def cells_of_node(k, m, idx):
    """Cells (x-fastest index) whose closure holds the lattice node with multi-index idx (3D, Q_k on m^3)."""
    per_axis = []
    for i in idx:
        cs = {min(i // k, m - 1)}
        if i % k == 0 and i > 0:
            cs.add(i // k - 1)
        per_axis.append(sorted(cs))
    return [c0 + m * (c1 + m * c2) for c2 in per_axis[2] for c1 in per_axis[1] for c0 in per_axis[0]]
