"""Shared helpers of the GPU tests: build the library once, set up problems on both sides."""
import numpy as np
import pytest

from oracle.fem import Problem
from paper_1904_13131_gb300 import inputs


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_13131_gb300 import build
    build.build()
    return torch


def rel(a, b):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def problem(dim, k, m, n_levels=1, top=None, ratio=10.0, radius=0.25):
    top = inputs.normal_top_mask(dim) if top is None else top
    return inputs.problem(dim, k, m, n_levels=n_levels, top=top, ratio=ratio, radius=radius)


def oracle_level(pr, level=-1):
    ml = pr["levels_m"][level]
    return Problem(pr["dim"], pr["k"], ml, pr["ids"][level], pr["mu"], pr["lam"], pr["masks"])


def context(pr, n_levels=None):
    from paper_1904_13131_gb300 import api
    ctx = api.Context(0)
    ctx.setup_problem(pr, n_levels)
    return ctx
