"""hy_dot_noalloc: the dot product for callers that must not allocate device memory while running.

Collected last on purpose (file name): it must pass both alone in a fresh process and after the rest
of the GPU suite. It calls the C ABI directly and checks the result against hy_dot, the context-based
entry point, within the relative tolerance of the other FP64 tests (1e-12), on two calls in a row --
the second call reuses the library's fixed scratch array that the first one left filled. It also checks
what the entry point exists for: after a warm-up call (which looks up the array's address), repeated calls
leave the device's free memory exactly where it was, so nothing was allocated, and the calling thread's
current device is unchanged.
"""
import ctypes

import pytest

from paper_1904_13131_gb300 import inputs

from .gpu_util import context, problem, require_gpu

pytestmark = pytest.mark.gpu


def test_dot_noalloc_matches_context_dot_twice():
    torch = require_gpu()
    from paper_1904_13131_gb300 import api
    lib = api.load_library()
    pr = problem(3, 2, 8)
    with context(pr) as ctx:
        n = ctx.num_dofs()
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for seed in (3, 4):  # two calls in a row on different data
            a = torch.tensor(inputs.gaussian_vector(n, seed), device="cuda")
            b = torch.tensor(inputs.gaussian_vector(n, seed + 10), device="cuda")
            ref = ctx.dot(a, b)
            out = ctypes.c_double()
            st = lib.hy_dot_noalloc(0, stream, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), n,
                                    ctypes.byref(out))
            assert st == 0
            assert abs(out.value - ref) <= 1e-12 * abs(ref)
        # a length spanning many blocks with a ragged tail, and the empty case
        m = 3 * 4096 * 7 + 123
        a = torch.tensor(inputs.gaussian_vector(m, 7), device="cuda")
        b = torch.tensor(inputs.gaussian_vector(m, 8), device="cuda")
        v1 = api.dot_noalloc(a, b)
        v2 = api.dot_noalloc(a, b)
        assert v1 == v2  # fixed summation order
        assert abs(v1 - float(a.cpu().numpy() @ b.cpu().numpy())) <= 1e-12 * abs(v1) * 10
        out = ctypes.c_double(1.0)
        assert lib.hy_dot_noalloc(0, stream, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), 0,
                                  ctypes.byref(out)) == 0
        assert out.value == 0.0


def test_dot_noalloc_allocates_nothing():
    torch = require_gpu()
    from paper_1904_13131_gb300 import api
    n = 3 * 4096 * 5 + 17
    a = torch.tensor(inputs.gaussian_vector(n, 21), device="cuda")
    b = torch.tensor(inputs.gaussian_vector(n, 22), device="cuda")
    ref = api.dot_noalloc(a, b)  # warm-up: the first call on the device looks up the scratch address
    torch.cuda.synchronize()
    dev_before = torch.cuda.current_device()
    free_before, _ = torch.cuda.mem_get_info()
    for _ in range(20):
        assert api.dot_noalloc(a, b) == ref
    torch.cuda.synchronize()
    free_after, _ = torch.cuda.mem_get_info()
    assert free_after == free_before
    assert torch.cuda.current_device() == dev_before


def test_dot_noalloc_rejects_oversize():
    require_gpu()
    from paper_1904_13131_gb300 import api
    lib = api.load_library()
    out = ctypes.c_double()
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    st = lib.hy_dot_noalloc(0, None, dummy, dummy, api.DOT_NOALLOC_MAX_N + 1, ctypes.byref(out))
    assert api.STATUS[st] == "HY_ERR_ARG"
