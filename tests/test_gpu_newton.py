"""Newton solves on the GPU (GMG-preconditioned CG) against the oracle's Newton with direct solves.
Tolerance: displacement relative L2 1e-8."""
import numpy as np
import pytest

from oracle.newton import newton_solve
from paper_1904_13131_gb300 import inputs

from .gpu_util import context, oracle_level, problem, rel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def face_values(dim, top_disp):
    fv = [[0.0] * 3 for _ in range(6)]
    fv[2 * (dim - 1) + 1][dim - 1] = top_disp
    return fv


def oracle_bc(P, dim, k, m, top_disp):
    X = inputs.node_coords(dim, k, m)
    ubc = np.zeros((P.n_nodes, dim))
    ubc[np.isclose(X[:, dim - 1], 1.0), dim - 1] = top_disp
    return ubc.reshape(-1)


@pytest.fixture(scope="module")
def config1_reference():
    dim, k, m = 2, 2, 16
    pr = problem(dim, k, m, n_levels=3)
    P = oracle_level(pr)
    u_ref, rep = newton_solve(P, oracle_bc(P, dim, k, m, -0.1), load_steps=5)
    return pr, u_ref, rep


@pytest.mark.parametrize("variant,level_dtype", [("T4", 0), ("NC", 0), ("FC", 1), ("T4", 1)])
def test_config1_newton_matches_oracle(torch, config1_reference, variant, level_dtype):
    """2D 16x16 Q2 inclusion, top displaced by -0.1 in 5 load steps, GMG with 3 levels."""
    pr, u_ref, rep_ref = config1_reference
    from paper_1904_13131_gb300.api import Context
    with context(pr) as ctx:
        u = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda")
        params = Context.newton_params(variant=variant, level_dtype=level_dtype, face_values=face_values(2, -0.1))
        rep = ctx.newton_solve(u, params)
    assert rep["load_steps_done"] == 5
    assert rel(u.cpu().numpy(), u_ref) < 1e-8
    assert max(rep["newton_iterations"]) <= max(rep_ref["iterations"]) + 2


def test_3d_newton_matches_oracle(torch):
    dim, k, m = 3, 2, 4
    pr = problem(dim, k, m, n_levels=2)
    P = oracle_level(pr)
    u_ref, _ = newton_solve(P, oracle_bc(P, dim, k, m, -0.1), load_steps=2)
    from paper_1904_13131_gb300.api import Context
    with context(pr) as ctx:
        u = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda")
        rep = ctx.newton_solve(u, Context.newton_params(load_steps=2, face_values=face_values(3, -0.1)))
    assert rep["load_steps_done"] == 2
    assert rel(u.cpu().numpy(), u_ref) < 1e-8


def test_config1_newton_exact_coarse_matches_oracle(torch, config1_reference):
    pr, u_ref, _ = config1_reference
    from paper_1904_13131_gb300.api import Context
    with context(pr) as ctx:
        ctx.set_solver_params(coarse_solver=1)
        u = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda")
        rep = ctx.newton_solve(u, Context.newton_params(level_dtype=1, face_values=face_values(2, -0.1)))
    assert rep["load_steps_done"] == 5
    assert rel(u.cpu().numpy(), u_ref) < 1e-8


def test_checkpoint_and_resume_continue_the_load_path(torch):
    """Checkpoint / resume at load-step granularity: load steps 1-2 in one context, the displacement saved to
    the host, steps 3-5 from it in a fresh context (and through the solve server) reach the one-shot
    solution (1e-10); the reports count absolute steps."""
    from paper_1904_13131_gb300.api import Context, HyError, Server, SolverParams
    dim, k, m, L = 3, 2, 4, 2
    pr = inputs.problem(dim, k, m, n_levels=L, top=inputs.normal_top_mask(dim))
    fv = [[0.0] * 3 for _ in range(6)]
    fv[5][2] = -0.1
    n = inputs.n_dofs(dim, k, m)
    with context(pr) as c:
        u_full = torch.zeros(n, dtype=torch.float64, device="cuda")
        c.newton_solve(u_full, Context.newton_params(level_dtype=1, face_values=fv))
        with pytest.raises(HyError) as e:
            c.newton_solve(torch.zeros_like(u_full), Context.newton_params(face_values=fv, first_step=4, last_step=3))
        assert e.value.status == "HY_ERR_ARG"
        u = torch.zeros_like(u_full)
        rep = c.newton_solve(u, Context.newton_params(level_dtype=1, face_values=fv, last_step=2))
        assert rep["load_steps_done"] == 2 and rep["newton_iterations"][2:] == [0, 0, 0]
    checkpoint = u.cpu().numpy()
    with context(pr) as c:
        u = torch.tensor(checkpoint, device="cuda")
        rep = c.newton_solve(u, Context.newton_params(level_dtype=1, face_values=fv, first_step=3))
        assert rep["load_steps_done"] == 5 and rep["newton_iterations"][:2] == [0, 0]
        assert min(rep["newton_iterations"][2:]) > 0
    ref = u_full.cpu().numpy()
    assert rel(u.cpu().numpy(), ref) < 1e-10
    solver = SolverParams(4, 1, 0.6, 1.2, 30, 0, 1e-3, 1, -1, 0, -1)
    with Server(0, budget_bytes=4 << 30, max_active=2) as sv:
        t1 = sv.submit(pr, Context.newton_params(level_dtype=1, face_values=fv, last_step=2), solver)
        sv.wait(t1, 600.0)
        r1 = sv.poll(t1, want_u=True)
        assert r1["state"] == 2 and r1["report"]["load_steps_done"] == 2
        t2 = sv.submit(pr, Context.newton_params(level_dtype=1, face_values=fv, first_step=3), solver,
                       u_start=r1["u"])
        sv.wait(t2, 600.0)
        r2 = sv.poll(t2, want_u=True)
        assert r2["state"] == 2 and r2["report"]["load_steps_done"] == 5
    assert rel(r2["u"], ref) < 1e-10


def uniaxial_setup(dim, k, m, L):
    """Homogeneous body (mu = 1, nu = 0.3), bottom clamped, side faces held in their normal component, the top
    face held laterally (free along its normal): uniaxial strain, with a positive definite tangent along the
    whole compressed path, as CG and the Chebyshev coarse solve need."""
    masks = [0] * (2 * dim)
    for a in range(dim - 1):
        masks[2 * a] = masks[2 * a + 1] = 1 << a
    masks[2 * (dim - 1)] = (1 << dim) - 1
    masks[2 * (dim - 1) + 1] = (1 << (dim - 1)) - 1
    mu, lam = inputs.material_table(1.0)
    ms = inputs.level_sizes(m, L)
    pr = {"dim": dim, "k": k, "m": m, "levels_m": ms, "ids": [np.zeros(ml**dim, np.uint8) for ml in ms],
          "mu": mu, "lam": lam, "masks": masks}
    return pr


def traction_top(dim, t):
    tr = np.zeros((6, 3))
    tr[2 * dim - 1][dim - 1] = -t
    return tr


@pytest.mark.parametrize("dim,k,m,L", [(2, 1, 4, 2), (2, 2, 4, 2), (3, 1, 4, 2), (3, 2, 4, 2)])
@pytest.mark.parametrize("t", [7.5, 12.0])
def test_newton_step_halving_matches_oracle(torch, dim, k, m, L, t):
    """Reading O15 (J > 0, Sec. 2.1) on the GPU: one load step of a compressive dead traction whose first
    Newton update would fold every cell. The GMG-CG Newton halves it as often as the oracle does (one
    halving for t = 7.5, two for t = 12; counted in the report's backtracks) and converges to the oracle's
    solution (1e-8)."""
    from paper_1904_13131_gb300.api import Context
    pr = uniaxial_setup(dim, k, m, L)
    P = oracle_level(pr)
    tr = traction_top(dim, t)
    u_ref, rep_ref = newton_solve(P, np.zeros(P.n_dofs), load_steps=1, f_ext=P.face_load(tr[: 2 * dim, :dim]))
    with context(pr) as ctx:
        for ldt in (0, 1):
            u = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda")
            rep = ctx.newton_solve(u, Context.newton_params(load_steps=1, level_dtype=ldt, face_traction=tr))
            assert rep["load_steps_done"] == 1
            assert rep["backtracks"] == sum(rep_ref["halvings"][0]) == (1 if t == 7.5 else 2)
            assert abs(rep["newton_iterations"][0] - rep_ref["iterations"][0]) <= 1
            assert rel(u.cpu().numpy(), u_ref) < 1e-8, (ldt, rel(u.cpu().numpy(), u_ref))


@pytest.mark.parametrize("dim", [2, 3])
def test_newton_reports_jneg_after_five_halvings(torch, dim):
    """t = 200: every halving down to 1/32 of the first update still folds the cells. The solve returns
    HY_ERR_JNEG (the oracle raises), leaves u at the last accepted iterate (zero), and the context stays
    usable: the next solve on it succeeds."""
    from paper_1904_13131_gb300.api import Context, HyError
    pr = uniaxial_setup(dim, 1, 4, 2)
    P = oracle_level(pr)
    with pytest.raises(FloatingPointError):
        newton_solve(P, np.zeros(P.n_dofs), load_steps=1, f_ext=P.face_load(traction_top(dim, 200.0)[: 2 * dim, :dim]))
    with context(pr) as ctx:
        u = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda")
        with pytest.raises(HyError) as e:
            ctx.newton_solve(u, Context.newton_params(load_steps=1, face_traction=traction_top(dim, 200.0)))
        assert e.value.status == "HY_ERR_JNEG"
        assert float(u.abs().max()) == 0.0
        rep = ctx.newton_solve(u, Context.newton_params(load_steps=1, face_traction=traction_top(dim, 7.5)))
        assert rep["load_steps_done"] == 1 and rep["backtracks"] == 1


@pytest.mark.parametrize("coarse", [0, 1])
def test_setup_reuse_keeps_the_solution(torch, config1_reference, coarse):
    """Solver parameter setup_reuse: linearisations whose coarsest-level displacement moved little since the
    last full setup keep its eigenvalue estimates and coarse solve. The preconditioner changes, the Newton
    solution does not (1e-8 against the oracle), and some setups were reused."""
    pr, u_ref, rep_ref = config1_reference
    from paper_1904_13131_gb300.api import Context
    with context(pr) as ctx:
        ctx.set_solver_params(coarse_solver=coarse)
        u0 = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda")
        rep0 = ctx.newton_solve(u0, Context.newton_params(level_dtype=1, face_values=face_values(2, -0.1)))
        ctx.set_solver_params(coarse_solver=coarse, setup_reuse=0.05)
        u = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda")
        rep = ctx.newton_solve(u, Context.newton_params(level_dtype=1, face_values=face_values(2, -0.1)))
    assert rep0["setups_reused"] == 0 and rep["setups_reused"] > 0
    assert rep["load_steps_done"] == 5
    assert rel(u.cpu().numpy(), u_ref) < 1e-8
    assert rep["newton_iterations"] == rep0["newton_iterations"]
    assert rep["cg_iterations_max"] <= rep0["cg_iterations_max"] + 5
