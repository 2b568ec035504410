"""Curved (isoparametric) cells through every variant.

Parity with the oracle's isoparametric Problem on the seeded curved geometry (inputs.curved_coords): the
tangent action of all five variants in FP64 (1e-12) and FP32 (2e-6), both kernel forms -- T4 and T2 fold
the map into their cached state, FC, SC (the paper's Algorithm 1) and NC run their general build, which
reads the inverse Jacobian and weight of each Gauss point from the cache -- and of T4/T2 in double-float
(1e-12); the residual and the diagonal (1e-12); Newton with FP64 and mixed V-cycles and the exact coarse
inverse (1e-8), through T4 and SC. The curved result differs from the lattice one (checked). A V-cycle
with the exact coarse inverse matches the oracle's hierarchy with the coordinates carried down by nodal
interpolation (1e-10), which pins the coarse-level geometry and the dense coarse assembly on curved cells.
The double-float action has no general build of FC/SC/NC and refuses them.
"""
import numpy as np
import pytest

from oracle.fem import Problem
from oracle.gmg import Hierarchy
from oracle.newton import newton_solve
from paper_1904_13131_gb300 import inputs

from .gpu_util import context, problem, rel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def oracle(pr, X=None):
    return Problem(pr["dim"], pr["k"], pr["m"], pr["ids"][-1], pr["mu"], pr["lam"], pr["masks"], X=X)


@pytest.mark.parametrize("dim,k,m", [(2, 2, 6), (2, 3, 3), (3, 1, 4), (3, 2, 3)])
def test_apply_residual_diagonal_on_curved_cells(torch, dim, k, m):
    from paper_1904_13131_gb300.api import FF
    pr = problem(dim, k, m)
    X = inputs.curved_coords(dim, k, m)
    P = oracle(pr, X)
    u = inputs.smooth_field(dim, k, m, seed=41, amplitude=0.03)
    x = inputs.gaussian_vector(P.n_dofs, seed=42)
    y_ref = P.apply(u, x)
    assert rel(oracle(pr).apply(u, x), y_ref) > 1e-3
    ud, xd = torch.tensor(u, device="cuda"), torch.tensor(x, device="cuda")
    with context(pr) as ctx:
        ctx.set_geometry(torch.tensor(X.reshape(-1), device="cuda"))
        assert rel(ctx.residual(ud).cpu().numpy(), P.residual(u)) < 1e-12
        for var in ("T4", "T2", "FC", "SC", "NC"):
            for form in (0, 1):
                ff = k <= 2 and var in ("T4", "T2")
                ctx.set_solver_params(coarse_eig_iters=5, fine_dtype=FF if ff else 0, kernel_form=form)
                ctx.set_displacement(ud, var, level_dtype=1)
                assert rel(ctx.apply_tangent(xd).cpu().numpy(), y_ref) < 1e-12, (var, form)
                assert rel(ctx.apply_tangent(xd.float(), dtype=1).cpu().numpy(), y_ref) < 2e-6, (var, form)
                if ff:
                    assert rel(ctx.apply_tangent(xd, dtype=FF).cpu().numpy(), y_ref) < 1e-12, (var, form)
        assert rel(ctx.diagonal().cpu().numpy(), P.diagonal(u)) < 1e-12
        ctx.set_solver_params(kernel_form=-1)
        ctx.set_geometry(None)  # back to the lattice
        ctx.set_displacement(ud, "T4")
        assert rel(ctx.apply_tangent(xd).cpu().numpy(), oracle(pr).apply(u, x)) < 1e-12


@pytest.mark.parametrize("dim,k,m,L", [(2, 2, 8, 3), (3, 2, 4, 2), (3, 1, 8, 3)])
def test_vcycle_on_curved_cells(torch, dim, k, m, L):
    pr = problem(dim, k, m, n_levels=L)
    X = inputs.curved_coords(dim, k, m)
    H = Hierarchy(pr["dim"], pr["k"], pr["levels_m"], pr["ids"], pr["mu"], pr["lam"], pr["masks"],
                  coarse_solver="direct", X=X)
    u = inputs.smooth_field(dim, k, m, seed=5, amplitude=0.02)
    b = inputs.gaussian_vector(inputs.n_dofs(dim, k, m), 8)
    with context(pr) as ctx:
        ctx.set_geometry(torch.tensor(X.reshape(-1), device="cuda"))
        ctx.set_solver_params(coarse_solver=1)
        ctx.set_displacement(torch.tensor(u, device="cuda"), "T4")
        info = [ctx.level_info(l) for l in range(L)]
        H.set_displacement(u, lmax=[i["lmax"] for i in info])
        bb = b.copy()
        bb[H.levels[-1].constrained] = 0.0
        z = ctx.gmg_vcycle(torch.tensor(bb, device="cuda")).cpu().numpy()
    assert rel(z, H.vcycle(bb)) < 1e-10


@pytest.mark.parametrize("variant", ["T4", "SC"])
@pytest.mark.parametrize("dim,k,m,L", [(2, 2, 8, 3), (3, 2, 4, 2)])
def test_newton_on_curved_cells(torch, dim, k, m, L, variant):
    from paper_1904_13131_gb300.api import Context
    pr = problem(dim, k, m, n_levels=L)
    X = inputs.curved_coords(dim, k, m)
    P = oracle(pr, X)
    lat = inputs.node_coords(dim, k, m)
    ubc = np.zeros((P.n_nodes, dim))
    ubc[np.isclose(lat[:, dim - 1], 1.0), dim - 1] = -0.1
    u_ref, _ = newton_solve(P, ubc.reshape(-1), load_steps=3)
    fv = [[0.0] * 3 for _ in range(6)]
    fv[2 * (dim - 1) + 1][dim - 1] = -0.1
    with context(pr) as ctx:
        ctx.set_geometry(torch.tensor(X.reshape(-1), device="cuda"))
        for ldt, coarse in ((0, 0), (1, 1)):
            ctx.set_solver_params(coarse_solver=coarse)
            u = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda")
            rep = ctx.newton_solve(u, Context.newton_params(load_steps=3, level_dtype=ldt, face_values=fv,
                                                            variant=variant))
            assert rep["load_steps_done"] == 3
            assert rel(u.cpu().numpy(), u_ref) < 1e-8, (ldt, coarse)


def test_double_float_refuses_the_general_builds(torch):
    from paper_1904_13131_gb300.api import FF, HyError
    dim, k, m = 2, 1, 2
    pr = problem(dim, k, m)
    with context(pr) as ctx:
        ctx.set_geometry(torch.tensor(inputs.curved_coords(dim, k, m).reshape(-1), device="cuda"))
        u = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda")
        ctx.set_solver_params(fine_dtype=FF)
        for var in ("FC", "SC", "NC"):
            with pytest.raises(HyError) as e:
                ctx.set_displacement(u, var)
            assert e.value.status == "HY_ERR_UNSUPPORTED"
        ctx.set_solver_params(fine_dtype=0)
        for var in ("FC", "SC", "NC"):
            ctx.set_displacement(u, var)
