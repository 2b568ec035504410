"""The workload configurations as parity cases.

* 3D 32^3 Q2 tangent application (823,875 dofs) in the launch configuration the benchmark times: every
  output of every variant against the oracle's element-by-element application (FP64 1e-12, FP32 2e-6).
* The largest mesh of the degree sweep, 128^3 Q2 (50,923,779 dofs): the tangent action (T4 and NC in FP64, T4
  in FP32, tuned kernel forms) against the oracle at seeded sample dofs, each evaluated by the oracle from
  the cells that contain its node (1e-12 / 2e-6).
* Degree sweep Q1-Q4 of the 3D Newton solve under 10 % compression in 5 load steps: against the oracle's
  Newton on reduced meshes (1e-8), and at 64^3 Q2 (6.4M dofs) by properties that hold at any size: the FP64,
  mixed-precision and exact-coarse solves converge to the same displacement (1e-8).
* Mixed precision per load step: the FP32 V-cycle inside FP64 CG/Newton against the FP64 path and the oracle
  after every load step (1e-8), with the iteration counts of both.
"""
import numpy as np
import pytest

from oracle.fem import Problem
from oracle.newton import newton_solve
from paper_1904_13131_gb300 import inputs

from .gpu_util import context, rel, require_gpu
from .mesh_util import cells_of_node

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def face_values(dim, disp):
    fv = [[0.0] * 3 for _ in range(6)]
    fv[2 * (dim - 1) + 1][dim - 1] = disp
    return fv


def oracle_bc(P, dim, k, m, disp):
    X = inputs.node_coords(dim, k, m)
    ubc = np.zeros((P.n_nodes, dim))
    ubc[np.isclose(X[:, dim - 1], 1.0), dim - 1] = disp
    return ubc.reshape(-1)


def test_config2_full_size_apply_every_output(torch):
    dim, k, m = 3, 2, 32
    pr = inputs.problem(dim, k, m, top=0)
    P = Problem(dim, k, m, pr["ids"][0], pr["mu"], pr["lam"], pr["masks"], chunk=2048)
    u = inputs.smooth_field(dim, k, m, seed=0)
    x = inputs.gaussian_vector(P.n_dofs, seed=1)
    y_ref = P.apply(u, x)
    ud, xd = torch.tensor(u, device="cuda"), torch.tensor(x, device="cuda")
    with context(pr) as ctx:
        ctx.set_solver_params(coarse_eig_iters=5)
        for var in ("T4", "T2", "FC", "SC", "NC"):
            ctx.set_displacement(ud, var, level_dtype=1)
            assert rel(ctx.apply_tangent(xd).cpu().numpy(), y_ref) < 1e-12, var
            assert rel(ctx.apply_tangent(xd.float(), dtype=1).cpu().numpy(), y_ref) < 2e-6, var


def test_config3_largest_mesh_sampled_outputs(torch):
    dim, k, m = 3, 2, 128
    pr = inputs.problem(dim, k, m, top=0)
    P = Problem(dim, k, m, pr["ids"][0], pr["mu"], pr["lam"], pr["masks"])
    assert P.n_dofs == 50_923_779
    u = inputs.smooth_field(dim, k, m, seed=0)
    x = inputs.gaussian_vector(P.n_dofs, seed=1)
    L = k * m + 1
    rng = np.random.default_rng(7)
    # random dofs plus dofs on the clamped bottom face, a cell corner and the last node
    dofs = np.concatenate([rng.choice(P.n_dofs, 300, replace=False), [0, 5, dim * (L * L + L + 1) * 2 + 2,
                                                                       P.n_dofs - 1]])
    cells = sorted({c for d in dofs for c in cells_of_node(k, m, ((d // dim) % L, (d // dim // L) % L,
                                                                   d // dim // (L * L)))})
    y_ref = np.zeros(P.n_dofs)
    P.apply_cells(u, np.where(P.constrained, 0.0, x), np.array(cells), y_ref)
    ref = np.where(P.constrained[dofs], x[dofs], y_ref[dofs])
    assert P.constrained[dofs].any() and not P.constrained[dofs].all()
    ud, xd = torch.tensor(u, device="cuda"), torch.tensor(x, device="cuda")
    del u, y_ref
    with context(pr) as ctx:
        ctx.set_solver_params(coarse_eig_iters=5)
        for var in ("T4", "NC"):
            ctx.set_displacement(ud, var, level_dtype=1 if var == "T4" else 0)
            y = ctx.apply_tangent(xd)[torch.tensor(dofs, device="cuda")].cpu().numpy()
            assert rel(y, ref) < 1e-12, (var, rel(y, ref))
            if var == "T4":
                y32 = ctx.apply_tangent(xd.float(), dtype=1)[torch.tensor(dofs, device="cuda")].cpu().numpy()
                assert rel(y32, ref) < 2e-6, rel(y32, ref)


@pytest.mark.parametrize("k,m,L", [(1, 8, 3), (2, 4, 2), (3, 4, 2), (4, 2, 2)])
def test_config3_degree_sweep_newton_matches_oracle(torch, k, m, L):
    dim = 3
    pr = inputs.problem(dim, k, m, n_levels=L, top=inputs.normal_top_mask(dim))
    P = Problem(dim, k, m, pr["ids"][-1], pr["mu"], pr["lam"], pr["masks"])
    u_ref, _ = newton_solve(P, oracle_bc(P, dim, k, m, -0.1), load_steps=5)
    from paper_1904_13131_gb300.api import Context
    runs = [(0, 0, 0), (1, 1, 0)]
    if k <= 2 or k == 4:
        # double-float coarse inverse and finest-level action in the outer CG, T2 level operators
        runs.append((1, 2, 2))
    with context(pr) as ctx:
        for ldt, coarse, fine in runs:
            ctx.set_solver_params(coarse_solver=coarse, fine_dtype=fine, level_variant=1 if fine == 2 else -1)
            u = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda")
            rep = ctx.newton_solve(u, Context.newton_params(level_dtype=ldt, face_values=face_values(dim, -0.1)))
            assert rep["load_steps_done"] == 5
            assert rel(u.cpu().numpy(), u_ref) < 1e-8, (k, ldt, coarse, fine)


def test_config3_64cube_q2_paths_agree(torch):
    """6.4M dofs, 5 levels (64 -> 4): FP64 V-cycle with Chebyshev coarse solve, mixed precision, mixed
    precision with the exact coarse solve, and that with the double-float finest-level action reach the same
    equilibrium."""
    dim, k, m, L = 3, 2, 64, 5
    pr = inputs.problem(dim, k, m, n_levels=L, top=inputs.normal_top_mask(dim))
    from paper_1904_13131_gb300.api import Context
    sols = []
    with context(pr) as ctx:
        for ldt, coarse, fine in ((0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 2, 2)):
            ctx.set_solver_params(coarse_solver=coarse, fine_dtype=fine)
            u = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda")
            rep = ctx.newton_solve(u, Context.newton_params(level_dtype=ldt, face_values=face_values(dim, -0.1)))
            assert rep["load_steps_done"] == 5 and rep["cg_iterations_max"] < 60
            sols.append(u.cpu().numpy())
            r = ctx.residual(u)
            assert torch.isfinite(r).all()
    assert rel(sols[1], sols[0]) < 1e-8 and rel(sols[2], sols[0]) < 1e-8 and rel(sols[3], sols[0]) < 1e-8


def test_config4_mixed_precision_per_load_step(torch):
    """After every load step the mixed-precision state equals the FP64 one and the oracle's (8^3 Q2)."""
    dim, k, m, L, steps = 3, 2, 8, 3, 5
    pr = inputs.problem(dim, k, m, n_levels=L, top=inputs.normal_top_mask(dim))
    P = Problem(dim, k, m, pr["ids"][-1], pr["mu"], pr["lam"], pr["masks"])
    final = oracle_bc(P, dim, k, m, -0.1)
    from paper_1904_13131_gb300.api import Context
    u_or = np.zeros(P.n_dofs)
    with context(pr) as ctx:
        u64 = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda")
        u32 = torch.zeros_like(u64)
        its64, its32 = [], []
        for s in range(1, steps + 1):
            fv = face_values(dim, -0.1 * s / steps)
            u_or, _ = newton_solve(P, final * s / steps, load_steps=1, u0=u_or)
            r64 = ctx.newton_solve(u64, Context.newton_params(load_steps=1, level_dtype=0, face_values=fv))
            r32 = ctx.newton_solve(u32, Context.newton_params(load_steps=1, level_dtype=1, face_values=fv))
            its64.append(r64["cg_iterations_total"])
            its32.append(r32["cg_iterations_total"])
            a64, a32 = u64.cpu().numpy(), u32.cpu().numpy()
            assert rel(a32, a64) < 1e-8 and rel(a64, u_or) < 1e-8 and rel(a32, u_or) < 1e-8, s
    # the FP32 V-cycle is as good a preconditioner as the FP64 one (within two CG iterations per solve)
    assert sum(its32) <= sum(its64) + 2 * 3 * steps
