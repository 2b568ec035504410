"""Work-list batches: several problems of one dim and degree advanced together.

* One list launch applies every problem's tangent: equal to the oracle's element-by-element action of each
  problem (FP64 1e-12, FP32 2e-6) for both kernel forms, with problems of different mesh sizes, materials
  and linearisation points in the same launch (ragged block counts, one-cell problems).
* The batched PCG (one graph replay per iteration for all resident problems) solves each problem's
  tangent system like the single-problem PCG: the same iteration counts within 5 % (the order of atomic
  sums differs between runs), solutions within the
  solver tolerance of the oracle's sparse direct solve, mixed-precision V-cycles included; a problem that
  hits its iteration cap fails alone.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from paper_1904_13131_gb300 import inputs

from .gpu_util import context, oracle_level, problem, rel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


def members(dim, k, ms, n_levels=1, ratios=None):
    """Problem bundles of one dim and degree with different sizes and stiffness ratios."""
    ratios = ratios or [10.0] * len(ms)
    return [problem(dim, k, m, n_levels=n_levels, ratio=r) for m, r in zip(ms, ratios)]


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("dim,k,ms,var", [(3, 2, [3, 1, 4, 2], "NC"), (3, 1, [5, 2, 3], "T4"),
                                           (2, 3, [5, 1, 7, 3, 2], "FC"), (2, 2, [6, 4], "T2"),
                                           (3, 3, [2, 1], "SC")])
def test_batch_apply_matches_oracle(torch, form, dim, k, ms, var):
    from paper_1904_13131_gb300.api import Batch
    prs = members(dim, k, ms, ratios=[2.0 + 7.0 * i for i in range(len(ms))])
    ctxs, us, xs, refs = [], [], [], []
    try:
        for i, pr in enumerate(prs):
            P = oracle_level(pr)
            u = inputs.smooth_field(dim, k, pr["m"], seed=20 + i, amplitude=0.03)
            x = inputs.gaussian_vector(P.n_dofs, seed=40 + i)
            refs.append(P.apply(u, x))
            c = context(pr)
            c.set_solver_params(kernel_form=form)
            c.set_displacement(torch.tensor(u, device="cuda"), var, level_dtype=1)
            ctxs.append(c)
            xs.append(torch.tensor(x, device="cuda"))
        with Batch(ctxs) as b:
            y64 = b.apply(xs)
            y32 = b.apply([x.float() for x in xs], dtype=1)
            assert b.kernel_form(0) == form and b.kernel_form(1) == form
            assert b.kernel_launches() > 0
        for i in range(len(prs)):
            assert rel(y64[i].cpu().numpy(), refs[i]) < 1e-12, (i, rel(y64[i].cpu().numpy(), refs[i]))
            assert rel(y32[i].cpu().numpy(), refs[i]) < 2e-6, i
    finally:
        for c in ctxs:
            c.close()


def test_batch_apply_tuned_and_repeated(torch):
    """Autotuned list form; repeated calls with the same and with new vectors agree with single applies."""
    from paper_1904_13131_gb300.api import Batch
    dim, k = 3, 2
    prs = members(dim, k, [4, 2, 6])
    ctxs = []
    try:
        for i, pr in enumerate(prs):
            c = context(pr)
            c.set_displacement(torch.tensor(inputs.smooth_field(dim, k, pr["m"], seed=i), device="cuda"), "T4")
            ctxs.append(c)
        with Batch(ctxs) as b:
            for seed in (1, 1, 2):
                xs = [torch.tensor(inputs.gaussian_vector(c.num_dofs(), seed + 10 * i), device="cuda")
                      for i, c in enumerate(ctxs)]
                ys = b.apply(xs)
                for c, x, y in zip(ctxs, xs, ys):
                    assert rel(y.cpu().numpy(), c.apply_tangent(x).cpu().numpy()) < 1e-13
            assert b.kernel_form(0) in (0, 1)
    finally:
        for c in ctxs:
            c.close()


@pytest.mark.parametrize("level_dtype,coarse,fine", [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 2), (0, 0, 2)])
def test_batch_pcg_matches_single_and_direct_solve(torch, level_dtype, coarse, fine):
    from paper_1904_13131_gb300.api import Batch
    dim, k = 2, 2
    prs = [problem(dim, k, m, n_levels=L, ratio=r) for m, L, r in ((16, 3, 10.0), (8, 2, 3.0), (12, 2, 30.0),
                                                                    (4, 1, 5.0))]
    ctxs, bs, refs, As = [], [], [], []
    try:
        for i, pr in enumerate(prs):
            P = oracle_level(pr)
            u = inputs.smooth_field(dim, k, pr["m"], seed=60 + i, amplitude=0.005)
            A = P.tangent(u)
            b = inputs.gaussian_vector(P.n_dofs, 70 + i)
            b[P.constrained] = 0.0
            refs.append(spla.spsolve(A.tocsc(), b))
            As.append(A)
            c = context(pr)
            c.set_solver_params(coarse_solver=coarse, fine_dtype=fine)
            c.set_displacement(torch.tensor(u, device="cuda"), "T4", level_dtype=level_dtype)
            ctxs.append(c)
            bs.append(torch.tensor(b, device="cuda"))
        single = [c.pcg(b, rtol=1e-10, max_iter=300) for c, b in zip(ctxs, bs)]
        with Batch(ctxs) as bt:
            xs, its, sts = bt.pcg(bs, rtol=1e-10, max_iter=300)
            launches = bt.kernel_launches()
        assert sts == [0] * len(prs)
        assert launches > 0
        for i in range(len(prs)):
            x = xs[i].cpu().numpy()
            b = bs[i].cpu().numpy()
            # the same arithmetic up to the order of the atomic sums, which moves a long FP32-preconditioned
            # run by a few iterations at most
            assert abs(its[i] - single[i][1]) <= max(1, 0.05 * single[i][1]), (i, its[i], single[i][1])
            assert np.linalg.norm(As[i] @ x - b) <= 1.01e-10 * np.linalg.norm(b), i
            assert rel(x, refs[i]) < 1e-7, i
            assert rel(x, single[i][0].cpu().numpy()) < 1e-7, i
    finally:
        for c in ctxs:
            c.close()


def test_batch_pcg_3d_members_and_iteration_cap(torch):
    """3D Q2 members of 2-3 levels; a cap of 3 iterations fails every member alone (status NOCONV) and a
    zero right-hand side converges at once."""
    from paper_1904_13131_gb300.api import Batch
    dim, k = 3, 2
    prs = [problem(dim, k, m, n_levels=L) for m, L in ((8, 3), (4, 2), (6, 2))]
    ctxs, bs = [], []
    try:
        for i, pr in enumerate(prs):
            c = context(pr)
            c.set_displacement(torch.tensor(inputs.smooth_field(dim, k, pr["m"], seed=i, amplitude=0.005),
                                            device="cuda"), "NC")
            ctxs.append(c)
            bs.append(torch.tensor(inputs.gaussian_vector(c.num_dofs(), 80 + i), device="cuda"))
        bs[1].zero_()
        with Batch(ctxs) as bt:
            xs, its, sts = bt.pcg(bs, rtol=1e-9, max_iter=200)
            assert sts == [0, 0, 0] and its[1] == 0 and its[0] > 0 and its[2] > 0
            for c, x, b, n in zip(ctxs, xs, bs, its):
                r = c.apply_tangent(x) - b
                assert float(r.norm()) <= 1.01e-9 * max(float(b.norm()), 1e-300) or n == 0
            _, its2, sts2 = bt.pcg(bs, rtol=1e-12, max_iter=3)
            assert sts2[0] != 0 and sts2[2] != 0 and sts2[1] == 0 and its2 == [3, 0, 3]
    finally:
        for c in ctxs:
            c.close()


def test_batch_argument_errors(torch):
    from paper_1904_13131_gb300.api import Batch, HyError
    a = context(problem(2, 2, 4))
    b = context(problem(2, 3, 4))
    c = context(problem(2, 2, 6))
    try:
        with pytest.raises(HyError):
            Batch([a, b])          # degrees differ
        with pytest.raises(HyError):
            Batch([a, a])          # repeated context
        with Batch([a, c]) as bt:
            xs = [torch.zeros(a.num_dofs(), dtype=torch.float64, device="cuda"),
                  torch.zeros(c.num_dofs(), dtype=torch.float64, device="cuda")]
            with pytest.raises(HyError):
                bt.apply(xs)       # no linearisation yet
            a.set_displacement(torch.zeros(a.num_dofs(), dtype=torch.float64, device="cuda"), "T4")
            c.set_displacement(torch.zeros(c.num_dofs(), dtype=torch.float64, device="cuda"), "NC")
            with pytest.raises(HyError):
                bt.apply(xs)       # variants differ
            c.set_displacement(torch.zeros(c.num_dofs(), dtype=torch.float64, device="cuda"), "T4")
            with pytest.raises(HyError):
                bt.apply([x.float() for x in xs], dtype=1)  # no FP32 cache on the finest level
            ys = bt.apply(xs)
            assert all(float(y.abs().max()) == 0.0 for y in ys)
    finally:
        for x in (a, b, c):
            x.close()
