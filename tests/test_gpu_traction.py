"""Dead tractions (the surface term of Eq. weak_form), as the paper loads its benchmark (Sec. 7).

* The face load vector equals the oracle's (1e-14) on every face, 2D and 3D, degrees 1-3.
* Newton under a shear traction on the free top face (bottom clamped) in 5 load steps matches the oracle's
  Newton (1e-8) with FP64 and mixed-precision V-cycles, and a traction combined with a prescribed
  normal displacement as well.
"""
import numpy as np
import pytest

from oracle.fem import Problem
from oracle.newton import newton_solve
from paper_1904_13131_gb300 import inputs

from .gpu_util import context, problem, rel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def oracle(pr, level=-1):
    return Problem(pr["dim"], pr["k"], pr["levels_m"][level], pr["ids"][level], pr["mu"], pr["lam"], pr["masks"])


@pytest.mark.parametrize("dim,k,m", [(2, 1, 5), (2, 2, 4), (2, 3, 3), (3, 1, 3), (3, 2, 2), (3, 3, 2)])
def test_face_load_matches_oracle(torch, dim, k, m):
    pr = problem(dim, k, m, top=0)
    P = oracle(pr)
    rng = np.random.default_rng(dim * 10 + k)
    t = np.zeros((6, 3))
    t[: 2 * dim, :dim] = rng.standard_normal((2 * dim, dim))
    with context(pr) as ctx:
        f = ctx.face_load(t).cpu().numpy()
    ref = P.face_load(t[: 2 * dim, :dim])
    np.testing.assert_allclose(f, ref, atol=1e-14 * np.abs(ref).max())


@pytest.mark.parametrize("dim,k,m,L,top", [(2, 2, 8, 3, 0), (3, 2, 4, 2, 0), (2, 2, 8, 3, 2)])
def test_newton_under_traction_matches_oracle(torch, dim, k, m, L, top):
    from paper_1904_13131_gb300.api import Context
    pr = problem(dim, k, m, n_levels=L, top=top)
    P = oracle(pr)
    t = np.zeros((6, 3))
    t[2 * (dim - 1) + 1][0] = 0.05  # shear on the top face along x
    ubc = np.zeros(P.n_dofs)
    fv = [[0.0] * 3 for _ in range(6)]
    if top:  # also prescribe the normal displacement of the top face
        X = inputs.node_coords(dim, k, m)
        ub = ubc.reshape(-1, dim)
        ub[np.isclose(X[:, dim - 1], 1.0), dim - 1] = -0.05
        fv[2 * (dim - 1) + 1][dim - 1] = -0.05
    u_ref, _ = newton_solve(P, ubc, load_steps=5, f_ext=P.face_load(t[: 2 * dim, :dim]))
    with context(pr) as ctx:
        for ldt in (0, 1):
            u = torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda")
            rep = ctx.newton_solve(u, Context.newton_params(load_steps=5, level_dtype=ldt, face_values=fv,
                                                            face_traction=t))
            assert rep["load_steps_done"] == 5
            assert rel(u.cpu().numpy(), u_ref) < 1e-8, (ldt, rel(u.cpu().numpy(), u_ref))
