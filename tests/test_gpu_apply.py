"""Parity of the cell kernels with the CPU oracle on the same seeded inputs.

Tolerances (relative L2): tangent action 1e-12 in FP64 and 2e-6 in FP32; residual and diagonal 1e-12.
Sizes span several thread blocks with a ragged last block (cells not a multiple of the cells per
block) and degrees 1-4 in 2D and 3D.
"""
import numpy as np
import pytest

from paper_1904_13131_gb300 import inputs

from .gpu_util import context, oracle_level, problem, rel, require_gpu

pytestmark = pytest.mark.gpu

VARIANTS = ["T4", "T2", "FC", "SC", "NC"]
CASES = [(2, 1, 13), (2, 2, 7), (2, 3, 5), (2, 4, 4), (3, 1, 5), (3, 2, 3), (3, 3, 3), (3, 4, 2)]


@pytest.fixture(scope="module")
def torch():
    return require_gpu()


@pytest.mark.parametrize("dim,k,m", CASES)
def test_apply_all_variants_fp64_fp32(torch, dim, k, m):
    pr = problem(dim, k, m)
    P = oracle_level(pr)
    u = inputs.smooth_field(dim, k, m, seed=dim * 10 + k)
    x = inputs.gaussian_vector(P.n_dofs, seed=k)
    y_ref = P.apply(u, x)
    ud = torch.tensor(u, device="cuda")
    xd = torch.tensor(x, device="cuda")
    xf = xd.float()
    with context(pr) as ctx:
        # one thread per (cell, Gauss point); one thread per x-line of a cell; the persistent line form (FP32;
        # the line form elsewhere); one thread per z-plane of a cell (FP32 in 3D; the line form elsewhere)
        for form in (0, 1, 2, 3):
            ctx.set_solver_params(kernel_form=form)
            for var in VARIANTS:
                ctx.set_displacement(ud, var, level_dtype=1)  # builds the FP64 and the FP32 fine cache
                assert ctx.kernel_form(-1, 0) == form and ctx.kernel_form(-1, 1) == form
                y64 = ctx.apply_tangent(xd).cpu().numpy()
                y32 = ctx.apply_tangent(xf, dtype=1).cpu().numpy()
                assert rel(y64, y_ref) < 1e-12, (form, var, rel(y64, y_ref))
                assert rel(y32, y_ref) < 2e-6, (form, var, rel(y32, y_ref))
                # constrained rows are the identity
                np.testing.assert_array_equal(y64[P.constrained], x[P.constrained])


@pytest.mark.parametrize("dim,k,m", [(2, 1, 13), (2, 2, 7), (2, 3, 5), (2, 4, 3), (3, 1, 5), (3, 2, 3), (3, 2, 4),
                                     (3, 3, 3), (3, 4, 2)])
def test_apply_double_float(torch, dim, k, m):
    """The double-float action (FP64 vectors, FP32-pipe arithmetic) meets the FP64 bar against the oracle,
    in both kernel forms and every variant; the finest level only."""
    from paper_1904_13131_gb300.api import FF
    pr = problem(dim, k, m)
    P = oracle_level(pr)
    u = inputs.smooth_field(dim, k, m, seed=dim * 10 + k + 5)
    x = inputs.gaussian_vector(P.n_dofs, seed=k + 7)
    y_ref = P.apply(u, x)
    ud, xd = torch.tensor(u, device="cuda"), torch.tensor(x, device="cuda")
    with context(pr) as ctx:
        for form in (0, 1, -1):
            ctx.set_solver_params(kernel_form=form, fine_dtype=FF, coarse_eig_iters=5)
            for var in VARIANTS:
                ctx.set_displacement(ud, var)
                yff = ctx.apply_tangent(xd, dtype=FF).cpu().numpy()
                assert rel(yff, y_ref) < 1e-12, (form, var, rel(yff, y_ref))
                np.testing.assert_array_equal(yff[P.constrained], x[P.constrained])
                assert ctx.kernel_form(-1, FF) in ((0, 1) if form < 0 else (form,))


def test_double_float_needs_its_cache(torch):
    from paper_1904_13131_gb300.api import FF, HyError
    pr = problem(3, 3, 2)
    u = torch.zeros(inputs.n_dofs(3, 3, 2), dtype=torch.float64, device="cuda")
    with context(pr) as ctx:
        ctx.set_displacement(u, "T4")
        with pytest.raises(HyError):
            ctx.apply_tangent(u, dtype=FF)  # no double-float cache without fine_dtype = FF
        ctx.set_solver_params(fine_dtype=FF)
        ctx.set_displacement(u, "T4")  # degree 3: built
        assert float(ctx.apply_tangent(u, dtype=FF).abs().max()) == 0.0


def test_autotuned_form_is_recorded_and_reused(torch):
    """kernel_form = -1 picks one of the two forms per level and precision (-1 where a level has no cache
    of that precision); a second context with the same shapes reuses the process-wide decisions."""
    dim, k, m = 3, 2, 6
    pr = problem(dim, k, m, n_levels=2)
    u = inputs.smooth_field(dim, k, m, seed=4)
    ud = torch.tensor(u, device="cuda")
    forms = []
    for _ in range(2):
        with context(pr) as ctx:
            ctx.set_solver_params(kernel_form=-1)
            ctx.set_displacement(ud, "NC", level_dtype=1)
            f = [(ctx.kernel_form(l, 0), ctx.kernel_form(l, 1)) for l in range(2)]
            forms.append(f)
            assert f[1][0] in (0, 1) and f[1][1] in (0, 1, 2) and f[0][0] in (0, 1) and f[0][1] in (-1, 0, 1, 2)
    assert forms[0] == forms[1]


@pytest.mark.parametrize("dim,k,m", [(2, 2, 7), (3, 2, 3), (3, 3, 2), (2, 4, 3), (3, 4, 2)])
def test_residual_and_diagonal(torch, dim, k, m):
    """Residual in FP64; the sum-factorised diagonal (per (J, L) pair and component, one 1D contraction per
    direction) in FP64 and, with fine_dtype = FF, in double-float, its state read from the T4 or T2 cache or
    (NC) evaluated from the displacement."""
    from paper_1904_13131_gb300.api import FF
    pr = problem(dim, k, m)
    P = oracle_level(pr)
    u = inputs.smooth_field(dim, k, m, seed=3)
    ud = torch.tensor(u, device="cuda")
    d_ref = P.diagonal(u)
    with context(pr) as ctx:
        r = ctx.residual(ud).cpu().numpy()
        for fine in (0, FF):
            ctx.set_solver_params(fine_dtype=fine)
            for var in ("T4", "T2", "NC"):
                ctx.set_displacement(ud, var)
                d = ctx.diagonal().cpu().numpy()
                assert rel(d, d_ref) < 1e-12, (fine, var, rel(d, d_ref))
    assert rel(r, P.residual(u)) < 1e-12


def test_deferred_fp64_cache_under_double_float(torch):
    """With a double-float finest action the finest FP64 cache is built at its first FP64 use (no kernel
    form before it), and that action then matches the oracle; the double-float action needs no FP64 cache."""
    from paper_1904_13131_gb300.api import F64, FF
    dim, k, m = 3, 2, 4
    pr = problem(dim, k, m, n_levels=2)
    P = oracle_level(pr)
    u = inputs.smooth_field(dim, k, m, seed=12)
    x = inputs.gaussian_vector(P.n_dofs, seed=13)
    y_ref = P.apply(u, x)
    ud, xd = torch.tensor(u, device="cuda"), torch.tensor(x, device="cuda")
    with context(pr) as ctx:
        ctx.set_solver_params(fine_dtype=FF)
        for var in ("T4", "NC"):
            ctx.set_displacement(ud, var)
            assert ctx.kernel_form(-1, F64) == -1 and ctx.kernel_form(-1, FF) >= 0
            assert rel(ctx.apply_tangent(xd, dtype=FF).cpu().numpy(), y_ref) < 1e-12
            assert ctx.kernel_form(-1, F64) == -1
            assert rel(ctx.apply_tangent(xd, dtype=F64).cpu().numpy(), y_ref) < 1e-12
            assert ctx.kernel_form(-1, F64) >= 0


@pytest.mark.parametrize("dim,k,m", [(2, 3, 6), (3, 2, 4)])
def test_finest_fp32_cache_from_the_high_precision_cache(torch, dim, k, m):
    """The finest level's FP32 cache of a mixed-precision hierarchy is taken from its FP64 or double-float
    cache of the same state (the same variant rounded, or T2 from T4); its FP32 action matches the oracle."""
    from paper_1904_13131_gb300.api import F32, F64, FF
    pr = problem(dim, k, m, n_levels=2)
    P = oracle_level(pr)
    u = inputs.smooth_field(dim, k, m, seed=21)
    x = inputs.gaussian_vector(P.n_dofs, seed=22)
    y_ref = P.apply(u, x)
    ud, xd = torch.tensor(u, device="cuda"), torch.tensor(x, device="cuda").float()
    with context(pr) as ctx:
        for fine, var, lvar in ((F64, "T4", -1), (FF, "T4", -1), (FF, "T4", "T2"), (F64, "T4", "T2"),
                                (FF, "T2", -1), (F64, "SC", -1), (FF, "NC", -1), (F64, "FC", "FC")):
            ctx.set_solver_params(fine_dtype=fine, level_variant=lvar)
            ctx.set_displacement(ud, var, level_dtype=1)
            y = ctx.apply_tangent(xd, dtype=F32).double().cpu().numpy()
            assert rel(y, y_ref) < 2e-6, (fine, var, lvar, rel(y, y_ref))


def test_zero_state_and_zero_vector(torch):
    """u = 0 gives R = 0 exactly; x = 0 gives y = 0 exactly (degenerate inputs)."""
    pr = problem(3, 2, 3)
    with context(pr) as ctx:
        n = ctx.num_dofs()
        z = torch.zeros(n, dtype=torch.float64, device="cuda")
        assert torch.count_nonzero(ctx.residual(z)).item() == 0
        ctx.set_displacement(z, "NC")
        assert torch.count_nonzero(ctx.apply_tangent(z)).item() == 0


def test_single_cell_and_fully_constrained(torch):
    dim, k, m = 3, 4, 1
    pr = problem(dim, k, m)
    pr["masks"] = [7] * 6  # every boundary dof constrained
    P = oracle_level(pr)
    u = inputs.smooth_field(dim, k, m, seed=1, amplitude=0.02)
    x = inputs.gaussian_vector(P.n_dofs, 2)
    with context(pr) as ctx:
        ctx.set_displacement(torch.tensor(u, device="cuda"), "T4")
        y = ctx.apply_tangent(torch.tensor(x, device="cuda")).cpu().numpy()
    assert rel(y, P.apply(u, x)) < 1e-12


def test_inverted_element_reports_jneg(torch):
    """A displacement that folds a cell (J <= 0) is reported as HY_ERR_JNEG, device stays usable."""
    from paper_1904_13131_gb300.api import HyError
    pr = problem(2, 1, 4)
    u = np.zeros(inputs.n_dofs(2, 1, 4))
    u[1::2] = -2.0 * inputs.node_coords(2, 1, 4)[:, 1]  # y -> -y: J = -1 everywhere
    with context(pr) as ctx:
        with pytest.raises(HyError) as e:
            ctx.residual(torch.tensor(u, device="cuda"))
        assert e.value.status == "HY_ERR_JNEG"
        with pytest.raises(HyError) as e:
            ctx.set_displacement(torch.tensor(u, device="cuda"), "T4")
        assert e.value.status == "HY_ERR_JNEG"
        ok = ctx.residual(torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda"))
        assert torch.count_nonzero(ok).item() == 0


def test_bounded_wait_gives_up_and_context_stays_usable(torch):
    """A bulk-copy wait that can never complete (nothing arrives on the barrier) gives up by itself after its
    wall-time bound: HY_ERR_TIMEOUT, then the same context applies the tangent correctly."""
    import time
    from paper_1904_13131_gb300.api import HyError
    dim, k, m = 3, 2, 3
    pr = problem(dim, k, m)
    P = oracle_level(pr)
    u = inputs.smooth_field(dim, k, m, seed=3)
    x = inputs.gaussian_vector(P.n_dofs, seed=4)
    with context(pr) as ctx:
        for limit in (0.05, 0.3):
            t0 = time.perf_counter()
            with pytest.raises(HyError) as e:
                ctx.check_bounded_wait(limit)
            assert e.value.status == "HY_ERR_TIMEOUT"
            assert time.perf_counter() - t0 < 5.0
        with pytest.raises(HyError) as e:
            ctx.check_bounded_wait(60.0)
        assert e.value.status == "HY_ERR_ARG"
        ctx.set_displacement(torch.tensor(u, device="cuda"), "T4")
        y = ctx.apply_tangent(torch.tensor(x, device="cuda")).cpu().numpy()
        assert rel(y, P.apply(u, x)) < 1e-12


def test_argument_errors(torch):
    from paper_1904_13131_gb300.api import Context, HyError
    with Context(0) as ctx:
        with pytest.raises(HyError) as e:
            ctx.mesh_setup(3, 5, 4, 1, [1, 0, 0, 0, 0, 0])
        assert e.value.status == "HY_ERR_UNSUPPORTED"
        with pytest.raises(HyError) as e:
            ctx.mesh_setup(3, 2, 6, 3, [1, 0, 0, 0, 0, 0])  # 6 -> 3 -> odd
        assert e.value.status == "HY_ERR_ARG"
        ctx.mesh_setup(2, 2, 4, 1, [0, 0, 3, 0])
        with pytest.raises(HyError) as e:
            ctx.set_displacement(torch.zeros(ctx.num_dofs(), dtype=torch.float64, device="cuda"))
        assert e.value.status == "HY_ERR_STATE"  # material not set
        with pytest.raises(HyError) as e:
            ctx.set_material(0, np.full(16, 3, np.uint8), [1.0, 2.0], [1.0, 2.0])
        assert e.value.status == "HY_ERR_ARG"


def test_deterministic_dot(torch):
    pr = problem(3, 2, 4)
    with context(pr) as ctx:
        n = ctx.num_dofs()
        a = torch.tensor(inputs.gaussian_vector(n, 5), device="cuda")
        b = torch.tensor(inputs.gaussian_vector(n, 6), device="cuda")
        vals = {ctx.dot(a, b) for _ in range(5)}
        assert len(vals) == 1
        assert abs(vals.pop() - float(a.cpu().numpy() @ b.cpu().numpy())) < 1e-10 * n


_TUNE_SCRIPT = """
import json, sys, torch
from paper_1904_13131_gb300 import api, inputs
pr = inputs.problem(3, 2, 4, n_levels=2, top=inputs.normal_top_mask(3))
with api.Context(0) as c:
    c.setup_problem(pr)
    c.set_displacement(torch.tensor(inputs.smooth_field(3, 2, 4, seed=1), device="cuda"), "FC", level_dtype=1)
    print(json.dumps([c.kernel_form(1, 0), c.kernel_form(1, 1)]))
"""


def test_tuning_file_is_json_and_reused(torch, tmp_path):
    """A fresh process tunes and writes HY_TUNE_FILE (a JSON array of decisions); a second process reads
    the decisions back instead of timing again (HY_VERBOSE prints a line per timing)."""
    import json
    import os
    import subprocess
    import sys
    path = tmp_path / "tune.json"
    env = dict(os.environ, HY_TUNE_FILE=str(path), HY_VERBOSE="1")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    runs = [subprocess.run([sys.executable, "-c", _TUNE_SCRIPT], env=env, cwd=root, capture_output=True, text=True,
                           timeout=600) for _ in range(2)]
    for r in runs:
        assert r.returncode == 0, r.stderr[-2000:]
    entries = json.loads(path.read_text())
    assert entries and all(set(e) == {"dim", "degree", "variant", "precision", "cells_log2", "threads_per_cell"}
                           for e in entries)
    assert {(e["variant"], e["precision"], e["cells_log2"]) for e in entries} >= {("FC", "f64", 6), ("FC", "f32", 6)}
    assert "[hy] autotune dim" in runs[0].stderr and "[hy] autotune dim" not in runs[1].stderr
    f1, f2 = (json.loads(r.stdout.strip().splitlines()[-1]) for r in runs)
    assert f1 == f2 and f1[0] in (0, 1) and f1[1] in (0, 1, 2)
