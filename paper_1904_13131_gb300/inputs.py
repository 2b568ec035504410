"""Seeded synthetic inputs for the heterogeneous-inclusion hyperelastic problems.

This module is shared by the CUDA path's callers (tests, bench) and by the CPU
oracle. It holds problem *data* only -- lattice node coordinates, per-cell
material ids of the inclusion geometry, smooth random displacement fields,
Gaussian vectors and Dirichlet face masks -- and none of the method's
arithmetic (no kinematics, stress, tangent, quadrature or sum factorisation).

Workload recipe (stands in for the paper's Miehe-2007 benchmark of Sec. 7,
whose geometry exists only as a missing figure):
  * unit square / cube, uniform m^d mesh of Q_k cells, nodes at the
    Gauss-Lobatto-Legendre (GLL) points of each cell;
  * one circular / spherical inclusion, centre 0.5, radius r (default 0.25),
    a cell belongs to the inclusion iff its centroid lies strictly inside;
  * matrix mu = 1, nu = 0.3, lambda = 2 mu nu / (1 - 2 nu); the inclusion scales
    mu and lambda together by the stiffness ratio (default 10);
  * bottom face clamped; top face either free or with its normal component
    prescribed.

Vector layout (the canonical layout of the whole library): nodes of the
(k m + 1)^d lattice in lexicographic order, x fastest; the d displacement
components of a node are interleaved, so dof = node * d + component.
"""
from __future__ import annotations

import numpy as np

# Face numbering used by every Dirichlet mask: (-x, +x, -y, +y, -z, +z).
FACE_NAMES = ("-x", "+x", "-y", "+y", "-z", "+z")


def lame_lambda(mu: float, nu: float) -> float:
    """Lame's first parameter from shear modulus and Poisson ratio (3D / plane strain)."""
    return 2.0 * mu * nu / (1.0 - 2.0 * nu)


def gll_unit(k: int) -> np.ndarray:
    """The k+1 Gauss-Lobatto-Legendre points on [0, 1] (end points plus roots of P_k')."""
    if k < 1:
        raise ValueError("degree must be >= 1")
    if k == 1:
        inner = np.zeros(0)
    else:
        inner = np.sort(np.real(np.polynomial.legendre.Legendre.basis(k).deriv().roots()))
    return 0.5 * (np.concatenate(([-1.0], inner, [1.0])) + 1.0)


def lattice_1d(k: int, m: int) -> np.ndarray:
    """Coordinates of the k*m+1 lattice nodes along one axis of the unit interval."""
    g = gll_unit(k)
    x = np.empty(k * m + 1)
    for c in range(m):
        x[k * c : k * c + k] = (c + g[:k]) / m
    x[-1] = 1.0
    return x


def node_coords(dim: int, k: int, m: int) -> np.ndarray:
    """(n_nodes, dim) coordinates in lattice order (x fastest)."""
    x = lattice_1d(k, m)
    grids = np.meshgrid(*([x] * dim), indexing="ij")  # grids[a][i0, i1, ...]
    # lattice order has x fastest, so flatten with axis order reversed
    cols = [g.transpose(tuple(range(dim))[::-1]).reshape(-1) for g in grids]
    return np.stack(cols, axis=1)


def n_dofs(dim: int, k: int, m: int) -> int:
    return dim * (k * m + 1) ** dim


def inclusion_ids(dim: int, m: int, radius: float = 0.25, center: float = 0.5) -> np.ndarray:
    """uint8 material id per cell (x fastest): 1 iff the centroid is strictly inside the inclusion."""
    c = (np.arange(m) + 0.5) / m
    grids = np.meshgrid(*([c] * dim), indexing="ij")
    r2 = sum((g - center) ** 2 for g in grids)
    ids = (r2 < radius * radius).astype(np.uint8)
    return ids.transpose(tuple(range(dim))[::-1]).reshape(-1).copy()


def material_table(ratio: float = 10.0, mu: float = 1.0, nu: float = 0.3):
    """(mu[2], lambda[2]) for matrix (id 0) and inclusion (id 1)."""
    lam = lame_lambda(mu, nu)
    return np.array([mu, ratio * mu]), np.array([lam, ratio * lam])


def level_sizes(m_fine: int, n_levels: int) -> list[int]:
    """Cells per direction from the coarsest (index 0) to the finest level; each level halves m."""
    ms = [m_fine]
    for _ in range(n_levels - 1):
        if ms[-1] % 2:
            raise ValueError("cells per direction must stay even while coarsening")
        ms.append(ms[-1] // 2)
    return ms[::-1]


def face_masks(dim: int, bottom: int | None = None, top: int = 0) -> list[int]:
    """Per-face component bitmasks; bottom (x_d = 0) fully clamped unless given, top as given."""
    masks = [0] * (2 * dim)
    masks[2 * (dim - 1)] = (1 << dim) - 1 if bottom is None else bottom
    masks[2 * (dim - 1) + 1] = top
    return masks


def normal_top_mask(dim: int) -> int:
    """Bitmask selecting the normal (last) component on the top face."""
    return 1 << (dim - 1)


def smooth_field(dim: int, k: int, m: int, seed: int, amplitude: float = 0.05) -> np.ndarray:
    """Seeded smooth displacement field, zero on the clamped face x_d = 0.

    phi_c(X) = X_d * sum_{mode in {1,2}^d} a_{c,mode} prod_i cos(pi mode_i X_i), a ~ N(0,1) from
    numpy's default_rng(seed); normalised to max nodal |phi| = 1, then scaled by `amplitude`.
    Returned in the canonical interleaved lattice layout.
    """
    rng = np.random.default_rng(seed)
    X = node_coords(dim, k, m)
    modes = np.array(np.meshgrid(*([[1, 2]] * dim), indexing="ij")).reshape(dim, -1).T
    a = rng.standard_normal((dim, len(modes)))
    basis = np.ones((X.shape[0], len(modes)))
    for i in range(dim):
        basis *= np.cos(np.pi * modes[None, :, i] * X[:, i : i + 1])
    phi = X[:, dim - 1 : dim] * (basis @ a.T)
    phi /= np.max(np.abs(phi))
    return (amplitude * phi).reshape(-1).copy()


def curved_coords(dim: int, k: int, m: int, delta=(0.06, 0.045, 0.03)) -> np.ndarray:
    """(n_nodes, dim) nodal coordinates of a curved geometry of the unit square / cube: lattice node xi moved
    to X = xi + delta * prod_j sin(pi xi_j) (component-wise delta). The bump vanishes on every face, so the
    faces stay where they are and keep their in-face metric; the interior cells are curved."""
    xi = node_coords(dim, k, m)
    bump = np.prod(np.sin(np.pi * xi), axis=1)
    return xi + bump[:, None] * np.asarray(delta[:dim], dtype=float)[None, :]


def gaussian_vector(n: int, seed: int) -> np.ndarray:
    """N(0,1) vector from numpy's default_rng(seed)."""
    return np.random.default_rng(seed).standard_normal(n)


def constrained_mask(dim: int, k: int, m: int, masks) -> np.ndarray:
    """Boolean per dof: True where some face mask constrains that node's component."""
    L = k * m + 1
    idx = np.indices((L,) * dim).reshape(dim, -1)[::-1]  # idx[a] = lattice index along axis a, x fastest
    out = np.zeros((L**dim, dim), dtype=bool)
    for a in range(dim):
        for side, val in ((0, 0), (1, L - 1)):
            fm = masks[2 * a + side]
            on = idx[a] == val
            for c in range(dim):
                if fm >> c & 1:
                    out[on, c] = True
    return out.reshape(-1)


def problem(dim: int, k: int, m: int, *, ratio: float = 10.0, radius: float = 0.25, n_levels: int = 1,
            top: int = 0):
    """Convenience bundle of one inclusion problem's data on every level (coarsest first)."""
    ms = level_sizes(m, n_levels)
    mu, lam = material_table(ratio)
    return {
        "dim": dim, "k": k, "m": m, "levels_m": ms,
        "ids": [inclusion_ids(dim, ml, radius) for ml in ms],
        "mu": mu, "lam": lam,
        "masks": face_masks(dim, top=top),
    }


def levels_for(m: int) -> int:
    """Hierarchy depth for a mesh of m cells per direction: halve while m stays even and m/2 >= 2."""
    L = 1
    while m % 2 == 0 and m // 2 >= 2:
        m //= 2
        L += 1
    return L


def serving_requests(n: int, seed: int = 0, rate: float = 1.0):
    """Seeded stream of solve requests shaped like the heterogeneous-inclusion workload: dim 2 or 3
    (equal odds), degree 1-3, 2D meshes 32^2..256^2 and 3D 8^3..48^3, stiffness ratio log-uniform on
    [2, 100], inclusion radius uniform on [0.1, 0.35], top compression uniform on [2, 15] %, and
    exponential inter-arrival times of the given mean rate (requests per second)."""
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for i in range(n):
        dim = int(rng.choice([2, 3]))
        k = int(rng.integers(1, 4))
        m = int(rng.choice([32, 64, 128, 256] if dim == 2 else [8, 16, 24, 32, 48]))
        ratio = float(np.exp(rng.uniform(np.log(2.0), np.log(100.0))))
        radius = float(rng.uniform(0.1, 0.35))
        compression = float(rng.uniform(0.02, 0.15))
        t += float(rng.exponential(1.0 / rate))
        out.append({"id": i, "dim": dim, "k": k, "m": m, "levels": levels_for(m), "ratio": ratio, "radius": radius,
                    "compression": compression, "arrival": t})
    return out
