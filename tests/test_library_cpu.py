"""CPU-side checks of the C ABI: the library builds, loads and exports every declared symbol;
argument errors are reported without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1904_13131_gb300 import api, build
    build.build()
    return api.load_library()


def test_header_symbols_exported(lib):
    from paper_1904_13131_gb300 import api
    header = open(os.path.join(ROOT, "include", "hyperelastic.h")).read()
    declared = set(re.findall(r"\b(hy_[a-z_0-9]+)\s*\(", header))
    assert declared == set(api.EXPORTED), declared ^ set(api.EXPORTED)
    for name in declared:
        assert hasattr(lib, name), name


def test_status_strings_and_null_args(lib):
    assert lib.hy_status_str(0) == b"HY_OK"
    assert lib.hy_status_str(5) == b"HY_ERR_JNEG"
    assert lib.hy_last_error(None) == b"null context"
    # a null output pointer is an argument error, decided before any CUDA call
    assert lib.hy_create(None, 0, None) == 1
    assert lib.hy_num_dofs(None, 0, None) == 1
    assert lib.hy_apply_tangent(None, None, None, 0) == 1
    lib.hy_destroy(None)


def test_no_oracle_in_product_package():
    pkg = os.path.join(ROOT, "paper_1904_13131_gb300")
    for dp, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".inc")):
                src = open(os.path.join(dp, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", src, re.M), f


def test_footprint_is_host_arithmetic(lib):
    """hy_footprint needs no GPU; it grows with the mesh and with the mixed-precision / exact-coarse extras."""
    from paper_1904_13131_gb300 import api
    b64 = api.footprint(3, 2, 32, 4)
    bmx = api.footprint(3, 2, 32, 4, level_dtype=api.F32)
    bex = api.footprint(3, 2, 32, 4, level_dtype=api.F32, coarse_solver=1)
    assert 0 < b64 < bmx < bex
    n0 = 3 * 9**3  # 4^3 Q2 coarsest level: without masks the exact coarse solve is bounded by all its dofs
    # exact coarse: dense pair + pivots + index maps, and the eigen history shrinks to the smoother's 2*30
    assert bex - bmx == 2 * 8 * n0 * n0 + 8 * (1024 + 64 * n0) + 4 * n0 + 4 * n0 + 8 * (60 - 2 * n0)
    masks = [0, 0, 0, 0, 7, 4]  # bottom clamped, top normal: 9*9*3 + 9*9 constrained coarse dofs
    nf = n0 - 9 * 9 * 4
    bmm = api.footprint(3, 2, 32, 4, level_dtype=api.F32, face_masks=masks)
    bfm = api.footprint(3, 2, 32, 4, level_dtype=api.F32, coarse_solver=1, face_masks=masks)
    assert bfm - bmm == 2 * 8 * nf * nf + 8 * (1024 + 64 * nf) + 4 * nf + 4 * n0 + 8 * (60 - 2 * nf)
    assert api.footprint(3, 2, 64, 5) > 7 * b64
    # double-float finest-level cache: the FP64 layout again (T4, 36 values per Gauss point, 9 cells per block)
    blocks = -(-32**3 // 9)
    assert api.footprint(3, 2, 32, 4, fine_dtype=api.FF) - b64 == 8 * 36 * ((9 * 27 + 3) // 4 * 4) * blocks
    # T2 level operators (17 values per Gauss point instead of 36) on the three levels below the finest
    cells = [4**3, 8**3, 16**3]
    saved = sum(8 * (36 - 17) * ((9 * 27 + 3) // 4 * 4) * -(-c // 9) for c in cells)
    assert b64 - api.footprint(3, 2, 32, 4, level_variant="T2") == saved
    with pytest.raises(api.HyError):
        api.footprint(3, 5, 32, 4)


def test_dot_noalloc_checks_its_inputs_before_the_gpu():
    """The binding of the allocation-free dot product refuses a second vector of another length, another
    dtype, a non-contiguous view or a tensor off the device before anything is launched (the kernel
    itself would read past the end of the shorter vector)."""
    torch = pytest.importorskip("torch")
    from paper_1904_13131_gb300 import api
    a = torch.zeros(10, dtype=torch.float64)
    with pytest.raises(ValueError, match="length"):
        api.dot_noalloc(a, torch.zeros(9, dtype=torch.float64))
    with pytest.raises(ValueError, match="float64"):
        api.dot_noalloc(a, torch.zeros(10, dtype=torch.float32))
    with pytest.raises(ValueError, match="contiguous"):
        api.dot_noalloc(a, torch.zeros(20, dtype=torch.float64)[::2])
    with pytest.raises(ValueError, match="not on cuda:0"):
        api.dot_noalloc(a, torch.zeros(10, dtype=torch.float64))
