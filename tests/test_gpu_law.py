"""The second volumetric function, U = lambda/4 (J^2 - 1 - 2 ln J), through every variant.

Parity with the oracle's law 1 on the same seeded inputs: the tangent action of all five variants in FP64
(1e-12) and FP32 (2e-6), both kernel forms (FC, SC, NC by their general build, which evaluates the law
chosen at run time), and of T4/T2 in double-float (1e-12, degrees 1-2); the residual and the diagonal
(1e-12); a Newton solve with FP64 and mixed-precision V-cycles and the exact coarse inverse (1e-8), through
T4 and NC. The two laws give different tangents (checked), so a kernel that ignored the law would fail. The
double-float action of FC/SC/NC refuses the second law (HY_ERR_UNSUPPORTED).
"""
import numpy as np
import pytest

from oracle.fem import Problem
from oracle.newton import newton_solve
from paper_1904_13131_gb300 import inputs

from .gpu_util import context, problem, rel, require_gpu

pytestmark = pytest.mark.gpu

VARIANTS = ["T4", "T2", "FC", "SC", "NC"]


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def oracle(pr, law, level=-1):
    return Problem(pr["dim"], pr["k"], pr["levels_m"][level], pr["ids"][level], pr["mu"], pr["lam"], pr["masks"],
                   law=law)


@pytest.mark.parametrize("dim,k,m", [(2, 2, 7), (3, 2, 3), (3, 1, 5), (3, 3, 2)])
def test_apply_residual_diagonal_second_law(torch, dim, k, m):
    from paper_1904_13131_gb300.api import FF, LAW_J2
    pr = problem(dim, k, m)
    P, P0 = oracle(pr, 1), oracle(pr, 0)
    u = inputs.smooth_field(dim, k, m, seed=31, amplitude=0.05)
    x = inputs.gaussian_vector(P.n_dofs, seed=32)
    y_ref = P.apply(u, x)
    assert rel(P0.apply(u, x), y_ref) > 1e-3  # the laws differ at this state
    ud, xd = torch.tensor(u, device="cuda"), torch.tensor(x, device="cuda")
    with context(pr) as ctx:
        ctx.set_material_law(LAW_J2)
        assert rel(ctx.residual(ud).cpu().numpy(), P.residual(u)) < 1e-12
        for var in VARIANTS:
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


@pytest.mark.parametrize("variant", ["T4", "NC"])
@pytest.mark.parametrize("dim,k,m,L", [(2, 2, 8, 3), (3, 2, 4, 2)])
def test_newton_second_law(torch, dim, k, m, L, variant):
    from paper_1904_13131_gb300.api import Context, LAW_J2
    pr = problem(dim, k, m, n_levels=L)
    P = oracle(pr, 1)
    X = inputs.node_coords(dim, k, m)
    ubc = np.zeros((P.n_nodes, dim))
    ubc[np.isclose(X[:, dim - 1], 1.0), dim - 1] = -0.1
    u_ref, _ = newton_solve(P, ubc.reshape(-1), load_steps=3)
    u0, _ = newton_solve(oracle(pr, 0), ubc.reshape(-1), load_steps=3)
    assert rel(u0, u_ref) > 1e-4
    fv = [[0.0] * 3 for _ in range(6)]
    fv[2 * (dim - 1) + 1][dim - 1] = -0.1
    with context(pr) as ctx:
        ctx.set_material_law(LAW_J2)
        for ldt, coarse in ((0, 0), (1, 1)):
            ctx.set_solver_params(coarse_solver=coarse)
            u = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda")
            rep = ctx.newton_solve(u, Context.newton_params(load_steps=3, level_dtype=ldt, face_values=fv,
                                                            variant=variant))
            assert rep["load_steps_done"] == 3
            assert rel(u.cpu().numpy(), u_ref) < 1e-8, (ldt, coarse)


def test_law_argument_checked(torch):
    from paper_1904_13131_gb300.api import FF, HyError, LAW_J2
    pr = problem(2, 1, 2)
    with context(pr) as ctx:
        with pytest.raises(HyError):
            ctx.set_material_law(7)
        ctx.set_material_law(LAW_J2)
        u = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda")
        ctx.set_solver_params(fine_dtype=FF)
        for var in ("FC", "SC", "NC"):
            with pytest.raises(HyError) as e:
                ctx.set_displacement(u, var)
            assert e.value.status == "HY_ERR_UNSUPPORTED"
        ctx.set_solver_params(fine_dtype=0, level_variant="NC")
        ctx.set_displacement(u, "T4")  # NC level operators under the second law: the general build
