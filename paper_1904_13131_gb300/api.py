"""Thin ctypes binding of libhyperelastic (include/hyperelastic.h), same names as the C ABI.

Argument marshalling only: torch tensors provide device memory and the CUDA stream; every step of
the computation runs in the library's kernels. The library must be built (see build.py); loading
fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhyperelastic.so")

STATUS = {0: "HY_OK", 1: "HY_ERR_ARG", 2: "HY_ERR_STATE", 3: "HY_ERR_OOM", 4: "HY_ERR_CUDA", 5: "HY_ERR_JNEG",
          6: "HY_ERR_NOCONV", 7: "HY_ERR_TIMEOUT", 8: "HY_ERR_UNSUPPORTED"}
VARIANTS = {"T4": 0, "T2": 1, "FC": 2, "SC": 3, "NC": 4}
LAW_LOG2, LAW_J2 = 0, 1  # hy_law
# the linearisation phases of hy_newton_report.setup_phase_ms
SETUP_PHASES = ("carry_down", "state_and_diagonal", "autotune", "smoother_eigenvalues", "coarse_setup_wait",
                "coarse_inverse_side_stream")
F64, F32, FF = 0, 1, 2  # hy_dtype; FF: double-float action on FP64 vectors

# every symbol the header declares (checked by the CPU test suite)
EXPORTED = ("hy_create", "hy_destroy", "hy_status_str", "hy_last_error", "hy_mesh_setup", "hy_num_dofs",
            "hy_set_material", "hy_set_displacement", "hy_apply_tangent", "hy_vmult", "hy_residual", "hy_diagonal",
            "hy_gmg_vcycle", "hy_set_solver_params", "hy_get_solver_params", "hy_level_info", "hy_set_level_info",
            "hy_level_displacement", "hy_prolongate_add", "hy_restrict", "hy_pcg", "hy_newton_default_params",
            "hy_newton_solve", "hy_dot", "hy_dot_noalloc", "hy_kernel_launches", "hy_footprint", "hy_ctx_bytes",
            "hy_server_create", "hy_server_destroy", "hy_server_submit", "hy_server_poll", "hy_server_wait",
            "hy_server_release", "hy_server_stats_get", "hy_kernel_form", "hy_batch_create", "hy_batch_destroy",
            "hy_batch_last_error", "hy_batch_apply", "hy_batch_pcg", "hy_batch_kernel_launches",
            "hy_batch_kernel_form", "hy_set_material_law", "hy_face_load", "hy_set_geometry",
            "hy_check_bounded_wait", "hy_server_set_batching")


class HyError(RuntimeError):
    """A failed C-ABI call: .status is the hy_status name ("HY_ERR_ARG", ...), the message the library's."""
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = STATUS.get(status, str(status))


class SolverParams(ctypes.Structure):
    """ctypes mirror of hy_solver_params (include/hyperelastic.h)."""
    _fields_ = [("cheb_degree", ctypes.c_int), ("cheb_sweeps", ctypes.c_int), ("cheb_lo", ctypes.c_double),
                ("cheb_hi", ctypes.c_double), ("eig_iters", ctypes.c_int), ("coarse_eig_iters", ctypes.c_int),
                ("coarse_reduction", ctypes.c_double), ("coarse_solver", ctypes.c_int), ("kernel_form", ctypes.c_int),
                ("fine_dtype", ctypes.c_int), ("level_variant", ctypes.c_int), ("setup_reuse", ctypes.c_double)]


class NewtonParams(ctypes.Structure):
    """ctypes mirror of hy_newton_params (include/hyperelastic.h)."""
    _fields_ = [("load_steps", ctypes.c_int), ("max_newton", ctypes.c_int), ("newton_rtol", ctypes.c_double),
                ("newton_atol", ctypes.c_double), ("cg_rtol", ctypes.c_double), ("cg_max_iter", ctypes.c_int),
                ("variant", ctypes.c_int), ("level_dtype", ctypes.c_int),
                ("face_values", (ctypes.c_double * 3) * 6), ("face_traction", (ctypes.c_double * 3) * 6),
                ("first_step", ctypes.c_int), ("last_step", ctypes.c_int)]


class NewtonReport(ctypes.Structure):
    """ctypes mirror of hy_newton_report (include/hyperelastic.h)."""
    _fields_ = [("load_steps_done", ctypes.c_int), ("newton_iterations", ctypes.c_int * 64),
                ("cg_iterations_total", ctypes.c_int), ("cg_iterations_max", ctypes.c_int),
                ("final_residual", ctypes.c_double), ("backtracks", ctypes.c_int), ("n_solves", ctypes.c_int),
                ("solve_cg_iterations", ctypes.c_int * 256), ("solve_ms", ctypes.c_double * 256),
                ("setup_ms_total", ctypes.c_double), ("total_ms", ctypes.c_double), ("setups_reused", ctypes.c_int),
                ("setup_phase_ms", ctypes.c_double * 6)]


class Request(ctypes.Structure):
    """ctypes mirror of hy_request (include/hyperelastic.h)."""
    _fields_ = [("dim", ctypes.c_int), ("degree", ctypes.c_int), ("cells_per_dir", ctypes.c_int),
                ("n_levels", ctypes.c_int), ("face_masks", ctypes.c_uint32 * 6), ("cell_mat_levels", ctypes.c_void_p),
                ("mu", ctypes.POINTER(ctypes.c_double)), ("lambda_", ctypes.POINTER(ctypes.c_double)),
                ("n_mat", ctypes.c_int), ("newton", NewtonParams), ("solver", SolverParams), ("law", ctypes.c_int),
                ("u_start", ctypes.POINTER(ctypes.c_double))]


class ServerStats(ctypes.Structure):
    """ctypes mirror of hy_server_stats (include/hyperelastic.h)."""
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "failed", "active", "queued", "bytes_in_use",
                                              "bytes_peak", "budget", "retried", "batched_solves", "batch_runs")]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libhyperelastic.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_1904_13131_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "hy_create": [ctypes.POINTER(vp), i32, vp],
        "hy_destroy": [vp],
        "hy_status_str": [i32],
        "hy_last_error": [vp],
        "hy_mesh_setup": [vp, i32, i32, i32, i32, ctypes.POINTER(ctypes.c_uint32)],
        "hy_num_dofs": [vp, i32, ctypes.POINTER(i64)],
        "hy_set_material": [vp, i32, vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl), i32],
        "hy_set_displacement": [vp, vp, i32, i32],
        "hy_apply_tangent": [vp, vp, vp, i32],
        "hy_vmult": [vp, i32, vp, vp, i32],
        "hy_residual": [vp, vp, vp],
        "hy_diagonal": [vp, i32, vp, i32],
        "hy_gmg_vcycle": [vp, vp, vp],
        "hy_set_solver_params": [vp, ctypes.POINTER(SolverParams)],
        "hy_get_solver_params": [vp, ctypes.POINTER(SolverParams)],
        "hy_level_info": [vp, i32, ctypes.POINTER(dbl), ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                          ctypes.POINTER(i32)],
        "hy_set_level_info": [vp, i32, dbl, dbl, dbl],
        "hy_level_displacement": [vp, i32, vp],
        "hy_prolongate_add": [vp, i32, vp, vp, i32],
        "hy_restrict": [vp, i32, vp, vp, i32],
        "hy_pcg": [vp, vp, vp, dbl, i32, ctypes.POINTER(i32)],
        "hy_newton_default_params": [ctypes.POINTER(NewtonParams)],
        "hy_newton_solve": [vp, ctypes.POINTER(NewtonParams), vp, ctypes.POINTER(NewtonReport)],
        "hy_dot": [vp, vp, vp, i64, ctypes.POINTER(dbl)],
        "hy_kernel_launches": [vp, ctypes.POINTER(i64)],
        "hy_dot_noalloc": [i32, vp, vp, vp, i64, ctypes.POINTER(dbl)],
        "hy_footprint": [i32, i32, i32, i32, i32, i32, ctypes.POINTER(SolverParams), ctypes.POINTER(ctypes.c_uint32),
                         ctypes.POINTER(i64)],
        "hy_kernel_form": [vp, i32, i32, ctypes.POINTER(i32)],
        "hy_set_material_law": [vp, i32],
        "hy_face_load": [vp, ctypes.c_void_p, vp],
        "hy_set_geometry": [vp, vp],
        "hy_check_bounded_wait": [vp, ctypes.c_double],
        "hy_ctx_bytes": [vp, ctypes.POINTER(i64)],
        "hy_batch_create": [ctypes.POINTER(vp), ctypes.POINTER(vp), i32],
        "hy_batch_destroy": [vp],
        "hy_batch_last_error": [vp],
        "hy_batch_apply": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), i32],
        "hy_batch_pcg": [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), dbl, i32, ctypes.POINTER(i32),
                         ctypes.POINTER(i32)],
        "hy_batch_kernel_launches": [vp, ctypes.POINTER(i64)],
        "hy_batch_kernel_form": [vp, i32, ctypes.POINTER(i32)],
        "hy_server_create": [ctypes.POINTER(vp), i32, i64, i32],
        "hy_server_destroy": [vp],
        "hy_server_submit": [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)],
        "hy_server_poll": [vp, ctypes.c_uint64, ctypes.POINTER(i32), ctypes.POINTER(NewtonReport),
                           ctypes.POINTER(dbl), i64, ctypes.POINTER(dbl)],
        "hy_server_wait": [vp, ctypes.c_uint64, dbl],
        "hy_server_release": [vp, ctypes.c_uint64],
        "hy_server_stats_get": [vp, ctypes.POINTER(ServerStats)],
        "hy_server_set_batching": [vp, i32, dbl],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = None if name in ("hy_destroy", "hy_newton_default_params", "hy_server_destroy",
                                     "hy_batch_destroy") else ctypes.c_int
    lib.hy_status_str.restype = ctypes.c_char_p
    lib.hy_last_error.restype = ctypes.c_char_p
    lib.hy_batch_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


class Context:
    """One hy_ctx on a CUDA device, enqueuing on the given torch stream (default: the current one)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self._torch = torch
        self.lib = load_library()
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        h = ctypes.c_void_p()
        st = self.lib.hy_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream))
        if st != 0:
            raise HyError(st, "hy_create failed")
        self.h = h
        self.dim = self.degree = self.m = self.n_levels = None

    def close(self):
        """hy_destroy; idempotent."""
        if getattr(self, "h", None):
            self.lib.hy_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _ck(self, st):
        if st != 0:
            raise HyError(st, self.lib.hy_last_error(self.h).decode())

    def _vec(self, t, n, dtype):
        torch = self._torch
        want = torch.float32 if dtype == F32 else torch.float64
        if t.device != self.device or t.dtype != want or not t.is_contiguous() or t.numel() != n:
            raise ValueError(f"expected a contiguous {want} tensor of {n} elements on {self.device}")
        return _ptr(t)

    def empty(self, level=-1, dtype=F64):
        """An uninitialised device vector of a level's dofs (FP64; FP32 for dtype=F32)."""
        torch = self._torch
        return torch.empty(self.num_dofs(level), dtype=torch.float32 if dtype == F32 else torch.float64,
                           device=self.device)

    # ---- mesh / material -------------------------------------------------------------------------
    def mesh_setup(self, dim, degree, cells_per_dir, n_levels, face_masks):
        """hy_mesh_setup: dim 2|3, degree 1-4, cells per direction, levels; face_masks[2*dim] per face."""
        fm = (ctypes.c_uint32 * (2 * dim))(*[int(x) for x in face_masks[: 2 * dim]])
        self._ck(self.lib.hy_mesh_setup(self.h, dim, degree, cells_per_dir, n_levels, fm))
        self.dim, self.degree, self.m, self.n_levels = dim, degree, cells_per_dir, n_levels

    def num_dofs(self, level=-1):
        """hy_num_dofs of a level (-1 = finest)."""
        n = ctypes.c_int64()
        self._ck(self.lib.hy_num_dofs(self.h, level, ctypes.byref(n)))
        return n.value

    def set_geometry(self, X=None):
        """Curved cells: X the finest level's nodal coordinates (n_dofs FP64 values on the device, interleaved
        like a displacement), or None for the uniform lattice."""
        self._ck(self.lib.hy_set_geometry(self.h, None if X is None else self._vec(X, self.num_dofs(), F64)))

    def check_bounded_wait(self, limit_s=0.2):
        """Runs the failure-path check of the bounded device waits; raises HyError (HY_ERR_TIMEOUT) once the
        never-completing wait has given up, as it must."""
        self._ck(self.lib.hy_check_bounded_wait(self.h, float(limit_s)))

    def set_material_law(self, law):
        """0 (LAW_LOG2): the paper's lambda ln^2 J; 1 (LAW_J2): lambda/4 (J^2 - 1 - 2 ln J)."""
        self._ck(self.lib.hy_set_material_law(self.h, int(law)))

    def set_material(self, level, cell_mat, mu, lam):
        """hy_set_material of one level: per-cell material ids (uint8, x fastest), per-id mu and lambda."""
        ids = np.ascontiguousarray(cell_mat, dtype=np.uint8)
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        self._ck(self.lib.hy_set_material(self.h, level, ids.ctypes.data_as(ctypes.c_void_p),
                                          mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                          lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(mu)))

    def setup_problem(self, problem: dict, n_levels: int | None = None):
        """mesh_setup + set_material on every level from an inputs.problem(...) bundle; n_levels (at most the
        bundle's) keeps the finest n_levels of its hierarchy."""
        nb = len(problem["levels_m"])
        L = nb if n_levels is None else n_levels
        if not 1 <= L <= nb:
            raise ValueError(f"n_levels must lie in [1, {nb}]")
        self.mesh_setup(problem["dim"], problem["k"], problem["m"], L, problem["masks"])
        for l in range(L):
            self.set_material(l, problem["ids"][nb - L + l], problem["mu"], problem["lam"])

    # ---- state / operators ----------------------------------------------------------------------
    def set_displacement(self, u, variant="T4", level_dtype=F64):
        """hy_set_displacement: linearise every level about u (finest, FP64 on the device) in the given
        variant; level_dtype=F32 builds the mixed-precision V-cycle."""
        self._ck(self.lib.hy_set_displacement(self.h, self._vec(u, self.num_dofs(), F64), VARIANTS[variant],
                                              level_dtype))

    def apply_tangent(self, x, y=None, dtype=F64):
        """hy_apply_tangent: y = A(u) x on the finest level in dtype (F64, F32 or FF); returns y."""
        n = self.num_dofs()
        if y is None:
            y = self.empty(-1, dtype)
        self._ck(self.lib.hy_apply_tangent(self.h, self._vec(x, n, dtype), self._vec(y, n, dtype), dtype))
        return y

    def vmult(self, level, x, y=None, dtype=F64):
        """hy_vmult: y = A_l x on level `level`; returns y."""
        n = self.num_dofs(level)
        if y is None:
            y = self.empty(level, dtype)
        self._ck(self.lib.hy_vmult(self.h, level, self._vec(x, n, dtype), self._vec(y, n, dtype), dtype))
        return y

    def residual(self, u, r=None):
        """hy_residual: r = R(u) in FP64, zero on constrained dofs; returns r."""
        n = self.num_dofs()
        if r is None:
            r = self.empty()
        self._ck(self.lib.hy_residual(self.h, self._vec(u, n, F64), self._vec(r, n, F64)))
        return r

    def diagonal(self, level=-1, dtype=F64):
        """hy_diagonal: the diagonal of a level's tangent (1 on constrained dofs)."""
        d = self.empty(level, dtype)
        self._ck(self.lib.hy_diagonal(self.h, level, self._vec(d, self.num_dofs(level), dtype), dtype))
        return d

    def gmg_vcycle(self, r, z=None):
        """hy_gmg_vcycle: z = V r, one V-cycle on the finest level; returns z."""
        n = self.num_dofs()
        if z is None:
            z = self.empty()
        self._ck(self.lib.hy_gmg_vcycle(self.h, self._vec(r, n, F64), self._vec(z, n, F64)))
        return z

    def set_solver_params(self, **kw):
        """hy_set_solver_params with the named hy_solver_params fields changed (level_variant also by
        variant name)."""
        p = self.get_solver_params()
        for k, v in kw.items():
            if k == "level_variant" and isinstance(v, str):
                v = VARIANTS[v]
            setattr(p, k, v)
        self._ck(self.lib.hy_set_solver_params(self.h, ctypes.byref(p)))

    def get_solver_params(self):
        """hy_get_solver_params as a SolverParams structure."""
        p = SolverParams()
        self._ck(self.lib.hy_get_solver_params(self.h, ctypes.byref(p)))
        return p

    def level_info(self, level):
        """hy_level_info: lmax of a level and, for the coarsest, its Chebyshev interval and degree."""
        lm, lo, hi, dg = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
        self._ck(self.lib.hy_level_info(self.h, level, ctypes.byref(lm), ctypes.byref(lo), ctypes.byref(hi),
                                        ctypes.byref(dg)))
        return {"lmax": lm.value, "coarse_lo": lo.value, "coarse_hi": hi.value, "coarse_degree": dg.value}

    def set_level_info(self, level, lmax=0.0, coarse_lo=0.0, coarse_hi=0.0):
        """hy_set_level_info: impose the eigenvalue estimates of a level instead of computing them."""
        self._ck(self.lib.hy_set_level_info(self.h, level, lmax, coarse_lo, coarse_hi))

    def kernel_form(self, level=-1, dtype=F64):
        """hy_kernel_form: the tangent-action kernel form of a level and precision (-1: no cache)."""
        f = ctypes.c_int()
        self._ck(self.lib.hy_kernel_form(self.h, level, dtype, ctypes.byref(f)))
        return f.value

    def level_displacement(self, level):
        """hy_level_displacement: the displacement carried down to a level (FP64)."""
        u = self.empty(level)
        self._ck(self.lib.hy_level_displacement(self.h, level, self._vec(u, self.num_dofs(level), F64)))
        return u

    def prolongate_add(self, fine_level, coarse, fine, dtype=F64):
        """hy_prolongate_add: fine += P coarse (levels fine_level - 1 -> fine_level); returns fine."""
        fl = fine_level if fine_level >= 0 else self.n_levels + fine_level
        self._ck(self.lib.hy_prolongate_add(self.h, fl, self._vec(coarse, self.num_dofs(fl - 1), dtype),
                                            self._vec(fine, self.num_dofs(fl), dtype), dtype))
        return fine

    def restrict(self, fine_level, fine, coarse=None, dtype=F64):
        """hy_restrict: coarse = P^T fine; returns coarse."""
        fl = fine_level if fine_level >= 0 else self.n_levels + fine_level
        if coarse is None:
            coarse = self.empty(fl - 1, dtype)
        self._ck(self.lib.hy_restrict(self.h, fl, self._vec(fine, self.num_dofs(fl), dtype),
                                      self._vec(coarse, self.num_dofs(fl - 1), dtype), dtype))
        return coarse

    def pcg(self, b, x=None, rtol=1e-8, max_iter=1000):
        """hy_pcg: V-cycle-preconditioned CG from zero to ||r|| <= rtol ||b||; returns (x, iterations)."""
        n = self.num_dofs()
        if x is None:
            x = self.empty()
        its = ctypes.c_int()
        self._ck(self.lib.hy_pcg(self.h, self._vec(b, n, F64), self._vec(x, n, F64), rtol, max_iter,
                                 ctypes.byref(its)))
        return x, its.value

    @staticmethod
    def newton_params(**kw):
        """hy_newton_default_params with the named fields changed: face_values and face_traction as
        [face][component] lists, variant by name."""
        p = NewtonParams()
        load_library().hy_newton_default_params(ctypes.byref(p))
        face_values = kw.pop("face_values", None)
        face_traction = kw.pop("face_traction", None)
        for k, v in kw.items():
            if k == "variant":
                v = VARIANTS[v]
            setattr(p, k, v)
        for arr, dst in ((face_values, p.face_values), (face_traction, p.face_traction)):
            if arr is not None:
                for f in range(6):
                    for c in range(3):
                        dst[f][c] = float(arr[f][c]) if f < len(arr) and c < len(arr[f]) else 0.0
        return p

    def face_load(self, traction, f=None):
        """External force of dead tractions traction[face][component] on the finest level (device FP64)."""
        if f is None:
            f = self.empty()
        t = ((ctypes.c_double * 3) * 6)()
        for i in range(min(6, len(traction))):
            for c in range(min(3, len(traction[i]))):
                t[i][c] = float(traction[i][c])
        self._ck(self.lib.hy_face_load(self.h, t, self._vec(f, self.num_dofs(), F64)))
        return f

    def newton_solve(self, u, params: NewtonParams):
        """hy_newton_solve: u (finest, FP64 on the device) in and out; returns the report as a dict and
        raises HyError on failure (u then holds the last accepted iterate)."""
        rep = NewtonReport()
        st = self.lib.hy_newton_solve(self.h, ctypes.byref(params), self._vec(u, self.num_dofs(), F64),
                                      ctypes.byref(rep))
        report = {"load_steps_done": rep.load_steps_done,
                  "newton_iterations": list(rep.newton_iterations[: max(rep.load_steps_done, params.load_steps)]),
                  "cg_iterations_total": rep.cg_iterations_total, "cg_iterations_max": rep.cg_iterations_max,
                  "final_residual": rep.final_residual, "backtracks": rep.backtracks,
                  "n_solves": rep.n_solves, "solve_cg_iterations": list(rep.solve_cg_iterations[: min(rep.n_solves, 256)]),
                  "solve_ms": list(rep.solve_ms[: min(rep.n_solves, 256)]), "setup_ms_total": rep.setup_ms_total,
                  "total_ms": rep.total_ms, "setups_reused": rep.setups_reused,
                  "setup_phase_ms": dict(zip(SETUP_PHASES, rep.setup_phase_ms))}
        self._ck(st)
        return report

    def dot(self, a, b):
        """hy_dot: FP64 dot product of two finest-level vectors in a fixed summation order."""
        n = a.numel()
        out = ctypes.c_double()
        self._ck(self.lib.hy_dot(self.h, self._vec(a, n, F64), self._vec(b, n, F64), n, ctypes.byref(out)))
        return out.value

    def bytes(self):
        """hy_ctx_bytes: device bytes the context owns."""
        b = ctypes.c_int64()
        self._ck(self.lib.hy_ctx_bytes(self.h, ctypes.byref(b)))
        return b.value

    def kernel_launches(self):
        """hy_kernel_launches: kernels the context has launched so far."""
        c = ctypes.c_int64()
        self._ck(self.lib.hy_kernel_launches(self.h, ctypes.byref(c)))
        return c.value


DOT_NOALLOC_MAX_N = 16384 * 4096


def dot_noalloc(a, b, device: int = 0, stream=None) -> float:
    """a . b through hy_dot_noalloc: no context and no device allocation (see include/hyperelastic.h).
    a and b must be contiguous float64 tensors of equal length on cuda:device (ValueError otherwise,
    before anything reaches the GPU)."""
    import torch
    dev = torch.device("cuda", device)
    for name, t in (("a", a), ("b", b)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous torch.float64 tensor")
    if a.numel() != b.numel():
        raise ValueError(f"a and b differ in length ({a.numel()} vs {b.numel()})")
    for name, t in (("a", a), ("b", b)):
        if t.device != dev:
            raise ValueError(f"{name} is on {t.device}, not on {dev}")
    lib = load_library()
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    out = ctypes.c_double()
    st = lib.hy_dot_noalloc(device, ctypes.c_void_p(stream.cuda_stream), _ptr(a), _ptr(b), a.numel(), ctypes.byref(out))
    if st != 0:
        raise HyError(st, "hy_dot_noalloc failed")
    return out.value


def footprint(dim, degree, cells_per_dir, n_levels, variant="T4", level_dtype=F64, coarse_solver=0,
              face_masks=None, fine_dtype=None, level_variant=None) -> int:
    """Device bytes a context needs for this problem (host arithmetic, no GPU)."""
    b = ctypes.c_int64()
    fm = None if face_masks is None else (ctypes.c_uint32 * 6)(*[int(x) for x in list(face_masks) + [0] * 6][:6])
    lv = -1 if level_variant is None else (VARIANTS[level_variant] if isinstance(level_variant, str) else level_variant)
    sp = SolverParams(4, 1, 0.6, 1.2, 30, 0, 1e-3, coarse_solver, -1, F64 if fine_dtype is None else fine_dtype, lv)
    st = load_library().hy_footprint(dim, degree, cells_per_dir, n_levels, VARIANTS[variant], level_dtype,
                                     ctypes.byref(sp), fm, ctypes.byref(b))
    if st != 0:
        raise HyError(st, "hy_footprint")
    return b.value


def _report_dict(rep, steps):
    return {"load_steps_done": rep.load_steps_done, "newton_iterations": list(rep.newton_iterations[:steps]),
            "cg_iterations_total": rep.cg_iterations_total, "cg_iterations_max": rep.cg_iterations_max,
            "final_residual": rep.final_residual, "n_solves": rep.n_solves, "total_ms": rep.total_ms,
            "setup_ms_total": rep.setup_ms_total, "setups_reused": rep.setups_reused}


class Batch:
    """hy_batch: work-list batch of contexts of the same dim and degree (see include/hyperelastic.h).
    Enqueues after, and makes each context's stream wait for, the batch's own stream."""

    def __init__(self, contexts):
        self.lib = load_library()
        self.contexts = list(contexts)
        arr = (ctypes.c_void_p * len(self.contexts))(*[c.h.value for c in self.contexts])
        h = ctypes.c_void_p()
        st = self.lib.hy_batch_create(ctypes.byref(h), arr, len(self.contexts))
        if st != 0:
            raise HyError(st, "hy_batch_create")
        self.h = h

    def close(self):
        """hy_batch_destroy; idempotent (the contexts stay)."""
        if getattr(self, "h", None):
            self.lib.hy_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _ck(self, st):
        if st != 0:
            raise HyError(st, self.lib.hy_batch_last_error(self.h).decode())

    def _vecs(self, ts, dtype):
        if len(ts) != len(self.contexts):
            raise ValueError("one vector per context")
        return (ctypes.c_void_p * len(ts))(*[c._vec(t, c.num_dofs(), dtype).value for c, t in zip(self.contexts, ts)])

    def apply(self, xs, ys=None, dtype=F64):
        """hy_batch_apply: ys[i] = A_i xs[i] for every context in one list launch; returns ys."""
        if ys is None:
            ys = [c.empty(-1, dtype) for c in self.contexts]
        self._ck(self.lib.hy_batch_apply(self.h, self._vecs(xs, dtype), self._vecs(ys, dtype), dtype))
        return ys

    def pcg(self, bs, xs=None, rtol=1e-8, max_iter=1000):
        """Returns (xs, iterations, statuses); statuses are hy_status codes per problem."""
        if xs is None:
            xs = [c.empty() for c in self.contexts]
        n = len(self.contexts)
        its = (ctypes.c_int * n)()
        sts = (ctypes.c_int * n)()
        self._ck(self.lib.hy_batch_pcg(self.h, self._vecs(bs, F64), self._vecs(xs, F64), rtol, max_iter, its, sts))
        return xs, list(its), list(sts)

    def kernel_launches(self):
        """hy_batch_kernel_launches: kernels the batch has launched so far."""
        v = ctypes.c_int64()
        self._ck(self.lib.hy_batch_kernel_launches(self.h, ctypes.byref(v)))
        return v.value

    def kernel_form(self, dtype=F64):
        """hy_batch_kernel_form: the list launch's kernel form for a precision (-1: not chosen yet)."""
        v = ctypes.c_int()
        self._ck(self.lib.hy_batch_kernel_form(self.h, dtype, ctypes.byref(v)))
        return v.value


class Server:
    """hy_server: continuous batching of independent Newton solves on one GPU (see include/hyperelastic.h)."""

    def __init__(self, device=0, budget_bytes=64 << 30, max_active=4, batching=False, window_ms=2.0):
        """hy_server_create, then hy_server_set_batching when batching (fused outer CG solves)."""
        self.lib = load_library()
        h = ctypes.c_void_p()
        st = self.lib.hy_server_create(ctypes.byref(h), device, int(budget_bytes), max_active)
        if st != 0:
            raise HyError(st, "hy_server_create")
        self.h = h
        self._steps = {}
        if batching:
            st = self.lib.hy_server_set_batching(self.h, 1, float(window_ms))
            if st != 0:
                self.close()
                raise HyError(st, "hy_server_set_batching")

    def close(self):
        """hy_server_destroy: running requests finish, queued ones are dropped; idempotent."""
        if getattr(self, "h", None):
            self.lib.hy_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, problem: dict, newton: NewtonParams, solver: SolverParams | None = None, law: int = 0,
               u_start=None) -> int:
        """problem: an inputs.problem(...) bundle (ids of every level, coarsest first); law: a hy_law; u_start:
        host start state (a checkpoint, with newton.first_step > 1), None = zero."""
        if solver is None:
            solver = SolverParams(4, 1, 0.6, 1.2, 30, 0, 1e-3, 0, -1, 0, -1)
        ids = np.ascontiguousarray(np.concatenate([np.asarray(i, dtype=np.uint8) for i in problem["ids"]]))
        mu = np.ascontiguousarray(problem["mu"], dtype=np.float64)
        lam = np.ascontiguousarray(problem["lam"], dtype=np.float64)
        r = Request()
        r.dim, r.degree, r.cells_per_dir, r.n_levels = problem["dim"], problem["k"], problem["m"], len(problem["ids"])
        for i, fm in enumerate(problem["masks"]):
            r.face_masks[i] = int(fm)
        r.cell_mat_levels = ids.ctypes.data_as(ctypes.c_void_p)
        r.mu = mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        r.lambda_ = lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        r.n_mat = len(mu)
        r.newton = newton
        r.solver = solver
        r.law = int(law)
        if u_start is not None:
            u_start = np.ascontiguousarray(u_start, dtype=np.float64)
            if u_start.size != r.dim * (r.degree * r.cells_per_dir + 1) ** r.dim:
                raise ValueError("u_start has the wrong length")
            r.u_start = u_start.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        t = ctypes.c_uint64()
        st = self.lib.hy_server_submit(self.h, ctypes.byref(r), ctypes.byref(t))
        if st != 0:
            raise HyError(st, "hy_server_submit")
        self._steps[t.value] = (newton.load_steps, r.dim * (r.degree * r.cells_per_dir + 1) ** r.dim)
        return t.value

    def poll(self, ticket, want_u=False):
        """hy_server_poll: {"state": 0 queued | 1 running | 2 done | 3 failed, "status"} plus, once finished,
        the report, the latency and (want_u, done) the solution on the host."""
        state, rep, lat = ctypes.c_int(), NewtonReport(), ctypes.c_double()
        steps, n = self._steps[ticket]
        u = np.empty(n) if want_u else None
        st = self.lib.hy_server_poll(self.h, ticket, ctypes.byref(state), ctypes.byref(rep),
                                     u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if want_u else None,
                                     n if want_u else 0, ctypes.byref(lat))
        out = {"state": state.value, "status": STATUS.get(st, st)}
        if state.value >= 2:
            out.update(report=_report_dict(rep, steps), latency_ms=lat.value, u=u if state.value == 2 else None)
        return out

    def wait(self, ticket, timeout_s=600.0):
        """hy_server_wait: block until the request has finished; HyError (HY_ERR_TIMEOUT) after timeout_s."""
        st = self.lib.hy_server_wait(self.h, ticket, timeout_s)
        if st != 0:
            raise HyError(st, "hy_server_wait")

    def release(self, ticket):
        """hy_server_release: forget a finished request."""
        self.lib.hy_server_release(self.h, ticket)

    def stats(self):
        """hy_server_stats_get as a dict."""
        s = ServerStats()
        st = self.lib.hy_server_stats_get(self.h, ctypes.byref(s))
        if st != 0:
            raise HyError(st, "hy_server_stats_get")
        return {n: getattr(s, n) for n, _ in ServerStats._fields_}
