"""Parity of the multigrid pieces with the oracle: transfers, carried-down displacement,
eigenvalue estimates, the V-cycle (FP64 and mixed precision) and PCG."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.gmg import Hierarchy
from paper_1904_13131_gb300 import inputs

from .gpu_util import context, problem, rel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def hierarchy(pr):
    return Hierarchy(pr["dim"], pr["k"], pr["levels_m"], pr["ids"], pr["mu"], pr["lam"], pr["masks"])


@pytest.mark.parametrize("dim,k,m,L", [(2, 2, 8, 3), (2, 3, 4, 2), (3, 1, 8, 3), (3, 2, 4, 2), (3, 4, 2, 2)])
def test_transfers_and_level_displacement(torch, dim, k, m, L):
    pr = problem(dim, k, m, n_levels=L)
    H = hierarchy(pr)
    u = inputs.smooth_field(dim, k, m, seed=4)
    H.set_displacement(u, lmax=[1.0] * L, coarse_bounds=(0.1, 1.0))
    with context(pr) as ctx:
        ctx.set_displacement(torch.tensor(u, device="cuda"), "T4")
        for l in range(1, L):
            nc, nf = ctx.num_dofs(l - 1), ctx.num_dofs(l)
            c = inputs.gaussian_vector(nc, l)
            f = inputs.gaussian_vector(nf, l + 7)
            fine0 = inputs.gaussian_vector(nf, l + 9)
            fd = torch.tensor(fine0, device="cuda")
            ctx.prolongate_add(l, torch.tensor(c, device="cuda"), fd)
            assert rel(fd.cpu().numpy(), fine0 + H.P[l] @ c) < 1e-14
            rc = ctx.restrict(l, torch.tensor(f, device="cuda")).cpu().numpy()
            assert rel(rc, H.P[l].T @ f) < 1e-14
            # FP32 transfers
            fd32 = torch.tensor(fine0, device="cuda").float()
            ctx.prolongate_add(l, torch.tensor(c, device="cuda").float(), fd32, dtype=1)
            assert rel(fd32.cpu().numpy(), fine0 + H.P[l] @ c) < 1e-6
        for l in range(L):
            np.testing.assert_allclose(ctx.level_displacement(l).cpu().numpy(), H.u[l], rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim,k,m,L", [(2, 2, 8, 3), (3, 2, 4, 2)])
def test_eigen_estimates_and_vcycle(torch, dim, k, m, L):
    pr = problem(dim, k, m, n_levels=L)
    H = hierarchy(pr)
    u = inputs.smooth_field(dim, k, m, seed=5)
    b = inputs.gaussian_vector(inputs.n_dofs(dim, k, m), 8)
    with context(pr) as ctx:
        ud = torch.tensor(u, device="cuda")
        ctx.set_displacement(ud, "T4")
        info = [ctx.level_info(l) for l in range(L)]
        H.set_displacement(u)  # oracle's own estimates
        for l in range(1, L):
            assert abs(info[l]["lmax"] - H.lmax[l]) < 1e-8 * H.lmax[l]
        assert abs(info[0]["coarse_hi"] - H.coarse_hi) < 1e-8 * H.coarse_hi
        assert abs(info[0]["coarse_lo"] - H.coarse_lo) < 1e-6 * H.coarse_lo
        # the V-cycle with identical parameters
        H.set_displacement(u, lmax=[i["lmax"] for i in info], coarse_bounds=(info[0]["coarse_lo"], info[0]["coarse_hi"]))
        assert H.coarse_deg == info[0]["coarse_degree"]
        bb = b.copy()
        bb[H.levels[-1].constrained] = 0.0
        z = ctx.gmg_vcycle(torch.tensor(bb, device="cuda")).cpu().numpy()
        z_ref = H.vcycle(bb)
        assert rel(z, z_ref) < 1e-10
        # mixed precision: FP32 V-cycle, FP64 coarse level
        ctx.set_displacement(ud, "T4", level_dtype=1)
        info32 = [ctx.level_info(l) for l in range(L)]
        H.set_displacement(u, lmax=[i["lmax"] for i in info32],
                           coarse_bounds=(info32[0]["coarse_lo"], info32[0]["coarse_hi"]))
        z32 = ctx.gmg_vcycle(torch.tensor(bb, device="cuda")).cpu().numpy()
        assert rel(z32, H.vcycle(bb)) < 1e-4


@pytest.mark.parametrize("variant,level_dtype", [("T4", 0), ("NC", 0), ("T4", 1), ("FC", 1)])
def test_pcg_solves_tangent_system(torch, variant, level_dtype):
    dim, k, m, L = 2, 2, 16, 3
    pr = problem(dim, k, m, n_levels=L)
    H = hierarchy(pr)
    u = inputs.smooth_field(dim, k, m, seed=6)
    P = H.levels[-1]
    A = P.tangent(u)
    b = inputs.gaussian_vector(P.n_dofs, 9)
    b[P.constrained] = 0.0
    x_ref = spla.spsolve(A.tocsc(), b)
    with context(pr) as ctx:
        ctx.set_displacement(torch.tensor(u, device="cuda"), variant, level_dtype=level_dtype)
        x, its = ctx.pcg(torch.tensor(b, device="cuda"), rtol=1e-10, max_iter=200)
    x = x.cpu().numpy()
    assert its < 60
    assert np.linalg.norm(A @ x - b) <= 1.01e-10 * np.linalg.norm(b)
    assert rel(x, x_ref) < 1e-7


def test_indefinite_coarse_level_is_reported_by_the_vcycle(torch):
    """u = 0.05 * smooth field with the top face free linearises about an unstable state: the 4^3
    coarsest tangent is indefinite (the oracle's dense eigenvalues agree). Applications still work;
    the V-cycle returns HY_ERR_NOCONV instead of running an unstable Chebyshev solve."""
    from paper_1904_13131_gb300.api import HyError
    dim, k, m = 3, 2, 8
    pr = problem(dim, k, m, n_levels=2, top=0)
    u = inputs.smooth_field(dim, k, m, seed=0)
    H = hierarchy(pr)
    H.set_displacement(u)
    assert not H.coarse_spd
    with context(pr) as ctx:
        ud = torch.tensor(u, device="cuda")
        ctx.set_displacement(ud, "T4")
        assert ctx.level_info(0)["coarse_lo"] < 0 and ctx.level_info(0)["coarse_degree"] == 0
        y = ctx.apply_tangent(ud)
        assert torch.isfinite(y).all()
        with pytest.raises(HyError) as e:
            ctx.gmg_vcycle(torch.zeros_like(ud))
        assert e.value.status == "HY_ERR_NOCONV"


@pytest.mark.parametrize("coarse", [1, 2])
@pytest.mark.parametrize("dim,k,m,L", [(2, 2, 8, 3), (3, 2, 4, 2), (3, 1, 8, 3), (3, 4, 4, 2), (3, 3, 4, 2)])
def test_exact_coarse_vcycle(torch, dim, k, m, L, coarse):
    """Option: the coarsest level solved exactly (dense inverse; coarse = 2 inverts in double-float)
    instead of by Chebyshev."""
    pr = problem(dim, k, m, n_levels=L)
    H = Hierarchy(pr["dim"], pr["k"], pr["levels_m"], pr["ids"], pr["mu"], pr["lam"], pr["masks"],
                  coarse_solver="direct")
    u = inputs.smooth_field(dim, k, m, seed=5, amplitude=0.02)
    b = inputs.gaussian_vector(inputs.n_dofs(dim, k, m), 8)
    with context(pr) as ctx:
        ctx.set_solver_params(coarse_solver=coarse)
        ctx.set_displacement(torch.tensor(u, device="cuda"), "T4")
        info = [ctx.level_info(l) for l in range(L)]
        H.set_displacement(u, lmax=[i["lmax"] for i in info])
        bb = b.copy()
        bb[H.levels[-1].constrained] = 0.0
        z = ctx.gmg_vcycle(torch.tensor(bb, device="cuda")).cpu().numpy()
    assert rel(z, H.vcycle(bb)) < 1e-10


@pytest.mark.parametrize("coarse,tol", [(1, 1e-11), (2, 1e-9)])
def test_exact_coarse_single_level_is_the_inverse(torch, coarse, tol):
    """The inverse applied on a one-level hierarchy is the sparse direct solve; the double-float inverse
    carries about 48 significant bits times the condition number of the coarse tangent."""
    dim, k, m = 3, 2, 3
    pr = problem(dim, k, m, n_levels=1)
    H = hierarchy(pr)
    u = inputs.smooth_field(dim, k, m, seed=2, amplitude=0.02)
    H.set_displacement(u)
    A = H.A[0]
    b = inputs.gaussian_vector(A.shape[0], 3)
    b[H.levels[0].constrained] = 0.0
    with context(pr) as ctx:
        ctx.set_solver_params(coarse_solver=coarse)
        ctx.set_displacement(torch.tensor(u, device="cuda"), "T4")
        z = ctx.gmg_vcycle(torch.tensor(b, device="cuda")).cpu().numpy()
        x, its = ctx.pcg(torch.tensor(b, device="cuda"), rtol=1e-12)
    assert rel(z, spla.spsolve(A.tocsc(), b)) < tol
    assert its <= 2 if coarse == 1 else its <= 4
