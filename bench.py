"""Benchmark: matrix-free finite-strain tangent application on one GB300 (and GMG-CG solve latency).

Workload (one step): the 3D compressible neo-Hookean unit cube with a spherical inclusion (r = 0.25,
10x stiffer, mu = 1, nu = 0.3), uniform 32^3 Q2 hexahedra (823,875 dofs), 3^3 Gauss points, bottom
face clamped, displacement state u = 0.05 * seeded smooth random field, source vector N(0,1). One
step applies the FP64 tangent once in each of the three caching variants -- fourth-order tangent
cached (T4, Algorithm 3), F cached with the stress recomputed (FC), nothing cached (NC).
value = dofs processed / device time = 3 * 823,875 * K / sum of the K*3 kernel-event durations.
Before every application the L2 cache is flushed by writing a 256 MB buffer and then reading another
256 MB one (outside the timed events): the read evicts the dirty lines of the write, so that their
write-back does not land inside the timed application. Extra keys report every variant in FP64 and FP32 and the GMG-preconditioned CG solve
latency (p50/p99) of the same problem with a 4-level hierarchy (32 -> 4), FP64 and mixed precision.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-solve]

--impl reference times the CPU oracle (the test oracle of this repository, FP64 numpy) on the
host cores on a bounded sample of the same workload (the same problem on a 16^3 Q2 mesh).
"""
import os

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

import argparse  # noqa: E402
import json  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import time  # noqa: E402

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tangent-apply GDoF/s (FP64 vs mixed) & GMG-CG solve p50/p99 latency, 1 GB300"
UNIT = "GDoF/s"
DIM, K, M = 3, 2, 32
VARIANTS = ("T4", "FC", "NC")
ALL_VARIANTS = ("T4", "T2", "FC", "SC", "NC")
WORKLOAD = "3D neo-Hookean unit cube, spherical inclusion r=0.25 10x, 32^3 Q2 (823,875 dofs), FP64 tangent apply x {T4, FC, NC}"


FORMS = {-1: None, 0: "point", 1: "line", 2: "line_persistent", 3: "plane"}


def flops_per_qp(var, dim=3, n=3):
    """Algorithmic FP64 flops per Gauss point of one application, counted from the kernel's arithmetic
    (FMA = 2): sum factorisation 4 d^2 (2n-1) + d(d-1); quadrature work per variant."""
    sf = 4 * dim * dim * (2 * n - 1) + dim * (dim - 1)
    g = dim * dim * (2 * dim - 1)          # g = G M
    q = dim * dim * 2 * dim                # Q = S + g tau
    p = dim * dim * (2 * dim - 1)          # P = Q M^T
    ns = 6 if dim == 3 else 3
    mat4 = ns * (2 * ns - 1) + 3           # Voigt J*C action
    nh = 16                                # neo-Hooke action c1 sym(g) + c2 tr(g) I
    state = 88                             # J, F^{-1}, ln J (counted as 1), b, tau, c1, c2 from F
    ubar = 2 * dim * dim * (2 * n - 1) + 2 * dim * dim  # gradient of the displacement, F = I + Grad u
    return {
        "T4": sf + g + mat4 + q + p,
        "T2": sf + g + nh + q + p,
        "FC": sf + state + g + nh + q + p,
        "SC": sf + ubar + state + g + nh + q + p,
        "NC": sf + ubar + state + g + nh + q + p,
    }[var]


def bytes_per_apply(var, dtype_bytes, nqp, ndofs, dim=3):
    """Algorithmic HBM bytes of one application: the cache once, x and the displacement once, y written once."""
    nvals = {"T4": dim * dim + 6 + 21, "T2": dim * dim + 6 + 2, "FC": dim * dim, "SC": 1, "NC": 0}[var]
    vec = 2 * ndofs * dtype_bytes + (ndofs * dtype_bytes if var in ("SC", "NC") else 0)
    return nvals * nqp * dtype_bytes + vec


# Algorithmic FP64 flops per dof of one 3D Q2 application, the per-unit figures of the scope table's
# measurement row: sum factorisation 8 d^2 n^(d+1) per cell, about 250 flops per Gauss point of
# quadrature work for the caching variants, and for NC in addition the gradient of the displacement
# (4 d^2 n^(d+1) per cell) and about 150 flops per Gauss point of kinematics.
SCOPE_FLOPS_PER_DOF = {"T4": 530.0, "NC": 830.0}


def kernel_source_sha():
    """sha256 of the tangent-action kernel source; a capture taken on other source no longer applies."""
    import hashlib
    with open(os.path.join(ROOT, "paper_1904_13131_gb300", "csrc", "cell_kernels.cuh"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def captured_traffic(kernel):
    """DRAM bytes (read + write) per launch of `kernel` from a committed ncu summary under profiles/ that
    names it on a 'traffic:' line together with the sha256 of the kernel source it was captured on:
        traffic: <kernel> <bytes per launch> <source sha256>
    None when no summary has it for the current source."""
    import glob
    sha = kernel_source_sha()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*"))):
        try:
            lines = open(path).read().splitlines()
        except (OSError, UnicodeDecodeError):
            continue
        for line in lines:
            parts = line.strip().strip("`").split()
            if len(parts) == 4 and parts[0] == "traffic:" and parts[1] == kernel and parts[3] == sha:
                return int(parts[2])
    return None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm, src = 6800.0, "fallback"
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        hbm, src = float(d.get("hbm_gbs", hbm)), "measured"
    # FP64 pipe: 2 DFMA per clock per SM x 152 SMs x 2.07 GHz (nominal 1.25 TFLOP/s)
    fp64 = 2 * 2 * 152 * 2.07e9 / 1e12
    return hbm, src, fp64


class Clocks:
    """Samples nvidia-smi clocks / throttle reasons while running (start before, stop after)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(os.environ.get("HY_CLOCKS_DIR", "/tmp"), f"hy_clocks_{os.getpid()}_{index}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def setup_contexts(torch, api, inputs, dev):
    pr = inputs.problem(DIM, K, M, n_levels=1, top=0)  # bottom clamped, top free
    u = torch.tensor(inputs.smooth_field(DIM, K, M, seed=0), device=dev)
    x = torch.tensor(inputs.gaussian_vector(inputs.n_dofs(DIM, K, M), seed=1), device=dev)
    ctxs = {}
    for var in ALL_VARIANTS:
        c = api.Context(dev.index)
        c.setup_problem(pr)
        # one-level hierarchy: the coarse estimate is not used here; FP64, FP32 and double-float caches
        c.set_solver_params(coarse_eig_iters=5, fine_dtype=api.FF)
        c.set_displacement(u, var, level_dtype=1)
        ctxs[var] = c
    return pr, u, x, ctxs


class L2Flush:
    """Write a 256 MB buffer (twice the 129 MB L2), then read a second 256 MB buffer: the read evicts the
    dirty lines the write left, so no write-back of the flush lands in the next timed kernel."""

    def __init__(self, torch, dev):
        self.w = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.r = torch.zeros(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def __call__(self):
        self.w.zero_()
        return self.r.sum()


def time_applies(torch, ctxs, variants, x, dtype, steps, warmup, flush, stream):
    """Per-(step, variant) CUDA-event durations in ms, L2 flushed before every application."""
    xin = x.float() if dtype == 1 else x
    ys = {v: torch.empty_like(xin) for v in variants}
    for _ in range(warmup):
        for v in variants:
            ctxs[v].apply_tangent(xin, ys[v], dtype=dtype)
    torch.cuda.synchronize()
    launches0 = sum(ctxs[v].kernel_launches() for v in variants)
    ev = []
    for _ in range(steps):
        row = []
        for v in variants:
            flush()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctxs[v].apply_tangent(xin, ys[v], dtype=dtype)
            e1.record(stream)
            row.append((e0, e1))
        ev.append(row)
    torch.cuda.synchronize()
    launches = sum(ctxs[v].kernel_launches() for v in variants) - launches0
    return np.array([[a.elapsed_time(b) for a, b in row] for row in ev]), ys, launches


def solve_latency(torch, api, inputs, dev):
    """GMG-preconditioned CG inside Newton: the 32^3 Q2 inclusion cube under 10% compression (bottom clamped,
    top normal displacement -0.1) in 5 load steps, 4 levels (32 -> 4, FP64 Chebyshev coarse solve on 4^3),
    CG rtol 1e-8; FP64 V-cycle and mixed precision (FP32 V-cycle). Latency of every linear solve."""
    pr = inputs.problem(DIM, K, M, n_levels=4, top=inputs.normal_top_mask(DIM))
    fv = [[0.0] * 3 for _ in range(6)]
    fv[5][2] = -0.1
    out, sols = {}, {}
    with api.Context(dev.index) as c:
        c.setup_problem(pr)
        t2 = api.VARIANTS["T2"]
        for name, ldt, coarse, fine, lvar, reuse, var in (
                ("fp64", 0, 0, 0, -1, 0.0, "T4"), ("mixed", 1, 0, 0, -1, 0.0, "T4"),
                ("mixed_exact_coarse", 1, 1, 0, -1, 0.0, "T4"),
                ("mixed_exact_coarse_fp64_inverse_t2_levels", 1, 1, 0, t2, 0.0, "T4"),
                ("mixed_exact_coarse_ff", 1, 2, 2, -1, 0.0, "T4"),
                ("mixed_exact_coarse_ff_t2_levels", 1, 2, 2, t2, 0.0, "T4"),
                ("mixed_exact_coarse_ff_t2_levels_setup_reuse", 1, 2, 2, t2, 0.05, "T4"),
                ("mixed_fp64_coarse_inverse_ff_t2_levels_setup_reuse", 1, 1, 2, t2, 0.05, "T4"),
                ("mixed_exact_coarse_ff_t2_everywhere", 1, 2, 2, t2, 0.0, "T2")):
            c.set_solver_params(coarse_solver=coarse, fine_dtype=fine, level_variant=lvar, setup_reuse=reuse)
            u = torch.zeros(inputs.n_dofs(DIM, K, M), dtype=torch.float64, device=dev)
            rep = c.newton_solve(u, api.Context.newton_params(level_dtype=ldt, face_values=fv, variant=var))
            lat = np.array(rep["solve_ms"])
            out[name] = {"solve_p50_ms": float(np.percentile(lat, 50)), "solve_p99_ms": float(np.percentile(lat, 99)),
                         "solves": rep["n_solves"], "cg_iterations_median": int(np.median(rep["solve_cg_iterations"])),
                         "cg_iterations_max": rep["cg_iterations_max"], "newton_iterations": rep["newton_iterations"],
                         "newton_total_ms": rep["total_ms"], "setup_ms_total": rep["setup_ms_total"],
                         "setup_fraction": rep["setup_ms_total"] / rep["total_ms"],
                         "setups_reused": rep["setups_reused"], "setup_phase_ms": rep["setup_phase_ms"],
                         "coarse_degree": c.level_info(0)["coarse_degree"]}
            sols[name] = u.cpu().numpy()
    for name in sols:
        if name != "fp64":
            out[f"{name}_vs_fp64_rel_l2"] = float(np.linalg.norm(sols[name] - sols["fp64"]) / np.linalg.norm(sols["fp64"]))
    # the paper's loading: a dead traction on the free top face along (1, 1, 0) (bottom clamped)
    prt = inputs.problem(DIM, K, M, n_levels=4, top=0)
    tr = [[0.0] * 3 for _ in range(6)]
    tr[5][0] = tr[5][1] = 0.05 / np.sqrt(2.0)
    with api.Context(dev.index) as c:
        c.setup_problem(prt)
        c.set_solver_params(coarse_solver=2, fine_dtype=api.FF, level_variant=api.VARIANTS["T2"])
        u = torch.zeros(inputs.n_dofs(DIM, K, M), dtype=torch.float64, device=dev)
        rep = c.newton_solve(u, api.Context.newton_params(level_dtype=1, face_traction=tr))
        lat = np.array(rep["solve_ms"])
        out["traction_mixed_exact_coarse_ff_t2_levels"] = {
            "solve_p50_ms": float(np.percentile(lat, 50)), "solve_p99_ms": float(np.percentile(lat, 99)),
            "solves": rep["n_solves"], "cg_iterations_max": rep["cg_iterations_max"],
            "newton_iterations": rep["newton_iterations"], "newton_total_ms": rep["total_ms"],
            "setup_ms_total": rep["setup_ms_total"], "max_abs_u": float(u.abs().max()),
            "load": "dead traction 0.05 along (1,1,0)/sqrt(2) on the free top face, 5 load steps"}
    # the same compression on curved cells (the seeded isoparametric perturbation of the cube), best mode
    Xc = torch.tensor(inputs.curved_coords(DIM, K, M).reshape(-1), device=dev)
    with api.Context(dev.index) as c:
        c.setup_problem(pr)
        c.set_geometry(Xc)
        c.set_solver_params(coarse_solver=2, fine_dtype=api.FF, level_variant=api.VARIANTS["T2"])
        u = torch.zeros(inputs.n_dofs(DIM, K, M), dtype=torch.float64, device=dev)
        rep = c.newton_solve(u, api.Context.newton_params(level_dtype=1, face_values=fv))
        lat = np.array(rep["solve_ms"])
        out["curved_mixed_exact_coarse_ff_t2_levels"] = {
            "solve_p50_ms": float(np.percentile(lat, 50)), "solve_p99_ms": float(np.percentile(lat, 99)),
            "solves": rep["n_solves"], "cg_iterations_max": rep["cg_iterations_max"],
            "newton_iterations": rep["newton_iterations"], "newton_total_ms": rep["total_ms"],
            "setup_ms_total": rep["setup_ms_total"],
            "geometry": "lattice nodes moved by the seeded smooth perturbation (amplitudes 0.06, 0.045, 0.03)"}
    out["coarse_solvers"] = ("fp64/mixed: Chebyshev to 1e-3 on 4^3 (Sec. 7); mixed_exact_coarse: dense inverse "
                             "(FP64 Gauss-Jordan, the FP64 coarse solve); _ff: coarse inverse computed in "
                             "double-float (about 48 bits) and double-float finest-level action in the outer CG; "
                             "_t2_levels: the V-cycle's level operators in the T2 variant; _setup_reuse: "
                             "eigenvalue estimates and coarse inverse kept while the coarse displacement moved "
                             "less than 5 % since the last full setup; mixed_fp64_coarse_inverse_*: the fastest "
                             "mode with the coarse inverse in FP64 (the FP64 coarse solve of the mixed-precision "
                             "pattern) instead of double-float; _t2_everywhere: the outer CG's finest-level action "
                             "in T2 as well (Algorithm 2)")
    out["workload"] = ("32^3 Q2 (823,875 dofs), 10% compression in 5 load steps, 4 levels, CG rtol 1e-8, T4 for "
                       "the outer CG unless the mode says otherwise")
    return out


def f32_steady_state(torch, api, inputs, dev, hbm):
    """The FP32 action in steady state: 64^3 Q2 (6.4M dofs; caches of 0.5-1 GB, far larger than L2), ten
    back-to-back applications per timing, best of three; T4 and T2 with the tuned kernel form."""
    k, m = 2, 64
    pr = inputs.problem(3, k, m, n_levels=1, top=0)
    n = inputs.n_dofs(3, k, m)
    nqp = m**3 * (k + 1) ** 3
    u = torch.tensor(inputs.smooth_field(3, k, m, seed=0), device=dev)
    x = torch.tensor(inputs.gaussian_vector(n, seed=1), device=dev).float()
    y = torch.empty_like(x)
    out = {"workload": "64^3 Q2 inclusion cube (6,440,067 dofs), u = 0.05 smooth field, FP32 cache and vectors"}
    for var in ("T4", "T2"):
        with api.Context(dev.index) as c:
            c.setup_problem(pr)
            c.set_solver_params(coarse_eig_iters=5)
            c.set_displacement(u, var, level_dtype=1)
            for _ in range(3):
                c.apply_tangent(x, y, dtype=1)
            best = 1e30
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(10):
                    c.apply_tangent(x, y, dtype=1)
                e1.record()
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1) / 10)
            gbs = bytes_per_apply(var, 4, nqp, n) / (best * 1e-3) / 1e9
            out[var] = {"ms": best, "gdofs": n / (best * 1e-3) / 1e9, "gbs": gbs, "hbm_frac": gbs / hbm,
                        "form": FORMS[c.kernel_form(-1, 1)], "algorithmic_bytes": bytes_per_apply(var, 4, nqp, n)}
    return out


def whole_job_rate(torch, dist, local_ms, units_per_rank, device):
    """Whole-job throughput of N replicas: the units all ranks processed over the slowest rank's timed region
    (max over ranks), in units per second; returns (rate, slowest ms). dist: torch.distributed or None."""
    t = float(local_ms)
    world = 1
    if dist is not None:
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
        world = dist.get_world_size()
    return units_per_rank * world / (t * 1e-3), t


def newton_summary(rep):
    lat = np.array(rep["solve_ms"])
    return {"solve_p50_ms": float(np.percentile(lat, 50)), "solve_p99_ms": float(np.percentile(lat, 99)),
            "solves": rep["n_solves"], "cg_iterations_median": int(np.median(rep["solve_cg_iterations"])),
            "cg_iterations_max": rep["cg_iterations_max"], "newton_iterations": rep["newton_iterations"],
            "newton_total_ms": rep["total_ms"], "setup_ms_total": rep["setup_ms_total"],
            "setups_reused": rep["setups_reused"]}


DEFAULT_SWEEP = [(1, 128, 6), (1, 256, 7), (2, 64, 5), (2, 128, 6), (3, 48, 5), (3, 64, 5), (4, 32, 4), (4, 64, 5)]


def config_study(torch, api, inputs, dev, sweep=None, paper_max_dofs=60_000_000, mixed_study=True):
    """The large workloads: (a) the 3D degree sweep Q1-Q4 at 6.4M-51M dofs, full Newton solve under 10%
    compression in 5 load steps, CG rtol 1e-8, in the paper's mode (FP64 V-cycle down to a 3^3-4^3 coarse
    level, Chebyshev coarse solve) and in the fastest mode (FP32 V-cycle with T2 level operators, coarsened
    further where needed to a level of at most 6000 dofs that is inverted exactly in double-float,
    double-float finest-level action, setup reuse at 5 %); (b) mixed precision on the 64^3 Q2 inclusion cube, load step by load step: displacement
    difference between the FP64 and the mixed-precision Newton states, and the CG iterations of both."""
    out = {}
    for k, m, L in (sweep or DEFAULT_SWEEP):
        n = inputs.n_dofs(3, k, m)
        fv = [[0.0] * 3 for _ in range(6)]
        fv[5][2] = -0.1
        # the fastest mode coarsens further (halving an even cell count) until its coarsest level can be
        # inverted exactly (at most 6000 dofs): 2^3 for Q3 64^3 and Q4
        Lf = L
        while inputs.n_dofs(3, k, m >> (Lf - 1)) > 6000 and (m >> (Lf - 1)) % 2 == 0 and (m >> (Lf - 1)) >= 4:
            Lf += 1
        coarse_exact = inputs.n_dofs(3, k, m >> (Lf - 1)) <= 6000
        modes = [("fastest", Lf, 1, 2 if coarse_exact else 0, api.FF, api.VARIANTS["T2"], 0.05)]
        if n <= paper_max_dofs:
            modes.insert(0, ("paper_fp64", L, 0, 0, api.F64, -1, 0.0))
        row = {"dofs": n, "levels": L, "coarse_m": m >> (L - 1)}
        sols = {}
        for name, levels, ldt, coarse, fine, lvar, reuse in modes:
            pr = inputs.problem(3, k, m, n_levels=levels, top=inputs.normal_top_mask(3))
            with api.Context(dev.index) as c:
                c.setup_problem(pr)
                c.set_solver_params(coarse_solver=coarse, fine_dtype=fine, level_variant=lvar, setup_reuse=reuse)
                u = torch.zeros(n, dtype=torch.float64, device=dev)
                rep = c.newton_solve(u, api.Context.newton_params(level_dtype=ldt, face_values=fv))
                row[name] = newton_summary(rep)
                row[name]["levels"] = levels
                row[name]["coarse_m"] = m >> (levels - 1)
                row[name]["coarse_solver"] = ["chebyshev", "exact_fp64", "exact_ff"][coarse]
                row[name]["fine_dtype"] = "ff" if fine == api.FF else "f64"
                row[name]["setup_reuse"] = reuse
                row[name]["solves_per_s"] = 1e3 / row[name]["solve_p50_ms"]
                sols[name] = u
        if len(sols) == 2:
            row["fastest_vs_paper_rel_l2"] = float(torch.linalg.norm(sols["fastest"] - sols["paper_fp64"]) /
                                                   torch.linalg.norm(sols["paper_fp64"]))
        del sols
        out[f"Q{k}_{m}^3"] = row
        print(json.dumps({"config_progress": f"Q{k}_{m}^3"}), file=sys.stderr, flush=True)
    if not mixed_study:
        return out
    # (b) mixed precision per load step on 64^3 Q2 (5 levels, FP64 Chebyshev coarse solve in both)
    k, m, L, steps = 2, 64, 5, 5
    pr = inputs.problem(3, k, m, n_levels=L, top=inputs.normal_top_mask(3))
    n = inputs.n_dofs(3, k, m)
    per_step = []
    with api.Context(dev.index) as c:
        c.setup_problem(pr)
        u64 = torch.zeros(n, dtype=torch.float64, device=dev)
        u32 = torch.zeros_like(u64)
        for s in range(1, steps + 1):
            fv = [[0.0] * 3 for _ in range(6)]
            fv[5][2] = -0.1 * s / steps
            r64 = c.newton_solve(u64, api.Context.newton_params(load_steps=1, level_dtype=0, face_values=fv))
            r32 = c.newton_solve(u32, api.Context.newton_params(load_steps=1, level_dtype=1, face_values=fv))
            per_step.append({"step": s, "mixed_vs_fp64_rel_l2": float(torch.linalg.norm(u32 - u64) / torch.linalg.norm(u64)),
                             "cg_iterations_fp64": r64["cg_iterations_total"], "cg_iterations_mixed": r32["cg_iterations_total"],
                             "newton_iterations_fp64": r64["newton_iterations"][0],
                             "newton_iterations_mixed": r32["newton_iterations"][0],
                             "solve_p50_ms_fp64": float(np.percentile(r64["solve_ms"], 50)),
                             "solve_p50_ms_mixed": float(np.percentile(r32["solve_ms"], 50))})
    out["mixed_per_load_step_64^3_Q2"] = per_step
    out["note"] = ("paper_fp64: FP64 V-cycle, Chebyshev coarse to 1e-3 (Sec. 7); fastest: FP32 V-cycle with T2 level "
                   "operators, exact coarse inverse (double-float Gauss-Jordan) where the coarsest level allows, "
                   "double-float finest-level action, setup reuse at 5 %; Newton under 10% compression in 5 load steps")
    return out


def serve_bench(api, inputs, dev, n_req, seed=0, max_active=8, budget_gb=160, seq_every=1, poisson=True,
                rate=None):
    """Serving (continuous batching): a seeded stream of uneven solve requests (2D 32^2-256^2 and 3D 8^3-48^3,
    Q1-Q3, stiffness ratio 2-100, radius 0.1-0.35, compression 2-15 %, 5 load steps). Baseline: the same
    requests solved one at a time with plain FP64 (FP64 V-cycle, Chebyshev coarse solve); with seq_every > 1
    only every seq_every-th request is solved that way and the baseline rate is that subset's (stated in the
    result). Served: up to `max_active` resident solves, mixed-precision V-cycle, exact coarse solve with the
    double-float inverse, double-float finest-level action and diagonals; closed loop (all at
    t=0) for peak solves/s, once with independent per-request solves and once with the outer CG solves fused
    across requests (hy_server_set_batching); Poisson arrivals at twice the baseline rate (or `rate` per
    second) for p50/p99."""
    reqs = inputs.serving_requests(n_req, seed)

    def problem(q):
        return inputs.problem(q["dim"], q["k"], q["m"], n_levels=q["levels"], ratio=q["ratio"], radius=q["radius"],
                              top=inputs.normal_top_mask(q["dim"]))

    def params(q, ldt):
        fv = [[0.0] * 3 for _ in range(6)]
        fv[2 * (q["dim"] - 1) + 1][q["dim"] - 1] = -q["compression"]
        return api.Context.newton_params(face_values=fv, level_dtype=ldt)

    def solver(q, coarse, ff):
        # ff: double-float coarse inverse and double-float finest-level action
        fine = api.FF if ff else api.F64
        return api.SolverParams(4, 1, 0.6, 1.2, 30, 0, 1e-3, 2 if (ff and coarse) else coarse, -1, fine,
                               api.VARIANTS["T2"] if ff else -1)

    def run(subset, max_act, ldt, coarse, arrivals=None, ff=False, batching=False):
        out = {}
        with api.Server(dev.index, budget_bytes=budget_gb << 30, max_active=max_act, batching=batching) as sv:
            t0 = time.perf_counter()
            tickets = []
            for q in subset:
                if arrivals is not None:
                    delay = arrivals[q["id"]] - (time.perf_counter() - t0)
                    if delay > 0:
                        time.sleep(delay)
                tickets.append(sv.submit(problem(q), params(q, ldt), solver(q, coarse, ff)))
            for t in tickets:
                sv.wait(t, 3600.0)
            makespan = time.perf_counter() - t0
            res = [sv.poll(t, want_u=True) for t in tickets]
            stats = sv.stats()
        lat = np.array([r["latency_ms"] for r in res])
        failed = sum(r["state"] != 2 for r in res)
        out = {"requests": len(subset), "solves_per_s": (len(subset) - failed) / makespan,
               "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
               "makespan_s": makespan, "failed": failed,
               "failed_requests": [dict(id=q["id"], status=r["status"], dim=q["dim"], k=q["k"], m=q["m"],
                                        ratio=q["ratio"], compression=q["compression"])
                                   for q, r in zip(subset, res) if r["state"] != 2],
               "bytes_peak_gb": stats["bytes_peak"] / 1e9, "max_active": max_act, "retried": stats["retried"]}
        if batching:
            out.update(batched_solves=stats["batched_solves"], batch_runs=stats["batch_runs"],
                       mean_solves_per_batch=stats["batched_solves"] / max(1, stats["batch_runs"]))
        return out, {q["id"]: r["u"] for q, r in zip(subset, res)}

    sub = reqs[::seq_every]
    seq, u_seq = run(sub, 1, 0, 0)
    if seq_every > 1:
        seq["subset"] = f"every {seq_every}th request ({len(sub)} of {n_req}); the baseline rate is this subset's"
    rate = 2.0 * seq["solves_per_s"] if rate is None else rate
    peak, u_peak = run(reqs, max_active, 1, 1, ff=True)
    fused, u_fused = run(reqs, max_active, 1, 1, ff=True, batching=True)
    out = {"requests": n_req, "seed": seed, "sequential_fp64": seq, "served_closed_loop": peak,
           "served_closed_loop_batched": fused,
           "speedup_solves_per_s": peak["solves_per_s"] / seq["solves_per_s"],
           "speedup_solves_per_s_batched": fused["solves_per_s"] / seq["solves_per_s"],
           "mix": [(q["dim"], q["k"], q["m"]) for q in reqs]}

    def max_err(us):
        errs = [float(np.linalg.norm(us[i] - u_seq[i]) / np.linalg.norm(u_seq[i])) for i in u_seq
                if us.get(i) is not None and u_seq[i] is not None]
        return max(errs) if errs else None

    out["max_rel_l2_served_vs_fp64"] = max_err(u_peak)
    out["max_rel_l2_batched_vs_fp64"] = max_err(u_fused)
    if poisson:
        rng = np.random.default_rng(seed + 1)
        arr, t = {}, 0.0
        for q in reqs:
            t += float(rng.exponential(1.0 / rate))
            arr[q["id"]] = t
        best_batched = fused["solves_per_s"] > peak["solves_per_s"]
        poi, _ = run(reqs, max_active, 1, 1, arrivals=arr, ff=True, batching=best_batched)
        out["served_poisson"] = dict(poi, arrival_rate_per_s=rate, batching=best_batched)
    return out


def batch_bench(torch, api, inputs, dev, stream, n_apply=64, n_solve=16, reps=20):
    """Work-list batches of many small problems (the serving regime): 3D Q2 inclusion cubes of 8^3 cells
    (14,739 dofs each) with stiffness ratios 2-17. (a) NC FP64 tangent actions of n_apply problems
    (943k dofs in all, about the size of the 32^3 workload): one list launch against one launch per
    problem, both L2-resident. (b) GMG-PCG (3 levels 8 -> 2, mixed precision, T4, rtol 1e-8) of n_solve
    problems, exact coarse solve: the batched solve (one graph replay and one host synchronisation per
    iteration for all) against the single-problem solve called once per problem."""
    m, k = 8, 2
    out = {}
    ctxs = []
    try:
        for i in range(n_apply):
            pr = inputs.problem(3, k, m, n_levels=1, top=0, ratio=2.0 + i % 16)
            c = api.Context(dev.index)
            c.setup_problem(pr)
            c.set_solver_params(coarse_eig_iters=5)
            c.set_displacement(torch.tensor(inputs.smooth_field(3, k, m, seed=i), device=dev), "NC")
            ctxs.append(c)
        n = ctxs[0].num_dofs()
        xs = [torch.tensor(inputs.gaussian_vector(n, 100 + i), device=dev) for i in range(n_apply)]
        ys = [torch.empty_like(x) for x in xs]
        with api.Batch(ctxs) as b:
            for _ in range(3):
                b.apply(xs, ys)
                for c, x, y in zip(ctxs, xs, ys):
                    c.apply_tangent(x, y)
            t_seq, t_bat = [], []
            for _ in range(reps):
                e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                e0.record(stream)
                for c, x, y in zip(ctxs, xs, ys):
                    c.apply_tangent(x, y)
                e1.record(stream)
                b.apply(xs, ys)
                e2.record(stream)
                e2.synchronize()
                t_seq.append(e0.elapsed_time(e1))
                t_bat.append(e1.elapsed_time(e2))
            form = b.kernel_form(0)
        ts, tb = float(np.median(t_seq)), float(np.median(t_bat))
        out["apply"] = {"problems": n_apply, "dofs_total": n * n_apply, "variant": "NC", "dtype": "f64",
                        "one_launch_per_problem_ms": ts, "list_launch_ms": tb,
                        "one_launch_per_problem_gdofs": n * n_apply / (ts * 1e-3) / 1e9,
                        "list_launch_gdofs": n * n_apply / (tb * 1e-3) / 1e9, "speedup": ts / tb,
                        "list_form": FORMS[form], "l2": "resident (same for both)"}
    finally:
        for c in ctxs:
            c.close()
    ctxs = []
    try:
        for i in range(n_solve):
            pr = inputs.problem(3, k, m, n_levels=3, top=inputs.normal_top_mask(3), ratio=2.0 + i)
            c = api.Context(dev.index)
            c.setup_problem(pr)
            c.set_solver_params(coarse_solver=1)
            c.set_displacement(torch.tensor(inputs.smooth_field(3, k, m, seed=i, amplitude=0.005), device=dev), "T4",
                               level_dtype=1)
            ctxs.append(c)
        n = ctxs[0].num_dofs()
        bs = [torch.tensor(inputs.gaussian_vector(n, 200 + i), device=dev) for i in range(n_solve)]
        xs = [torch.empty_like(v) for v in bs]
        with api.Batch(ctxs) as b:
            b.pcg(bs, xs, rtol=1e-8, max_iter=200)  # warm-up (graph capture, list-form choice)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            its_single = [c.pcg(v, x, rtol=1e-8, max_iter=200)[1] for c, v, x in zip(ctxs, bs, xs)]
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            _, its_batch, sts = b.pcg(bs, xs, rtol=1e-8, max_iter=200)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
        out["pcg"] = {"problems": n_solve, "dofs_each": n, "levels": 3, "variant": "T4", "level_dtype": "f32 (mixed)",
                      "coarse_solver": "exact (dense inverse)",
                      "one_solve_per_problem_ms": (t1 - t0) * 1e3, "batched_ms": (t2 - t1) * 1e3,
                      "speedup": (t1 - t0) / (t2 - t1), "cg_iterations_single": its_single,
                      "cg_iterations_batched": its_batch, "statuses": sts}
    finally:
        for c in ctxs:
            c.close()
    return out


# ---- the CPU oracle on the host cores (cpu_baseline and the reference arm) -----------------------------
# The oracle's element-by-element action (oracle.fem.Problem.apply, Eq. mf_vmult) as it stands, spread over
# a pool of host processes: each process runs the oracle's own per-chunk loop body (Problem.apply_cells)
# over a contiguous range of cells into its own slot of a shared result array, and the parent adds the
# slots and applies the Dirichlet rows exactly as Problem.apply does. The pool is started with "spawn"
# (never forked from a process that has touched the GPU).
_W = {}


def _oracle_worker_init(m, x_name, y_name, slots):
    from multiprocessing import shared_memory

    from oracle.fem import Problem
    from paper_1904_13131_gb300 import inputs
    pr = inputs.problem(DIM, K, m, n_levels=1, top=0)
    P = Problem(DIM, K, m, pr["ids"][0], pr["mu"], pr["lam"], pr["masks"])
    _W["P"], _W["u"] = P, inputs.smooth_field(DIM, K, m, seed=0)
    _W["shx"] = shared_memory.SharedMemory(name=x_name)
    _W["shy"] = shared_memory.SharedMemory(name=y_name)
    _W["x"] = np.ndarray((P.n_dofs,), dtype=np.float64, buffer=_W["shx"].buf)
    _W["y"] = np.ndarray((slots, P.n_dofs), dtype=np.float64, buffer=_W["shy"].buf)


def _oracle_worker_apply(task):
    slot, lo, hi = task
    P, y = _W["P"], _W["y"][slot]
    y[:] = 0.0
    for c in range(lo, hi, P.chunk):
        P.apply_cells(_W["u"], _W["x"], np.arange(c, min(c + P.chunk, hi)), y)
    return hi - lo


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


class OraclePool:
    """The oracle's tangent action on the m^3 Q2 inclusion cube (the apply workload's problem) over
    `workers` spawned host processes."""

    def __init__(self, m=M, workers=None):
        import multiprocessing as mp
        from multiprocessing import shared_memory

        from oracle.fem import Problem
        from paper_1904_13131_gb300 import inputs
        self.workers = workers or host_cores()
        pr = inputs.problem(DIM, K, m, n_levels=1, top=0)
        self.P = Problem(DIM, K, m, pr["ids"][0], pr["mu"], pr["lam"], pr["masks"])
        self.n, self.ncells = self.P.n_dofs, m**DIM
        self.shx = shared_memory.SharedMemory(create=True, size=8 * self.n)
        self.shy = shared_memory.SharedMemory(create=True, size=8 * self.n * self.workers)
        self.x = np.ndarray((self.n,), dtype=np.float64, buffer=self.shx.buf)
        self.y = np.ndarray((self.workers, self.n), dtype=np.float64, buffer=self.shy.buf)
        self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_oracle_worker_init,
                                                 initargs=(m, self.shx.name, self.shy.name, self.workers))

    def apply(self, x, n_cells=None):
        """y = A(u) x over the first n_cells cells (default all), Dirichlet rows as Problem.apply."""
        nc = self.ncells if n_cells is None else n_cells
        cons = self.P.constrained
        self.x[:] = np.where(cons, 0.0, x)
        bounds = np.linspace(0, nc, self.workers + 1).astype(int)
        self.pool.map(_oracle_worker_apply, [(i, int(bounds[i]), int(bounds[i + 1])) for i in range(self.workers)])
        y = self.y.sum(axis=0)
        if nc == self.ncells:
            y[cons] = np.asarray(x)[cons]
        return y

    def close(self):
        self.pool.terminate()
        self.pool.join()
        for sh in (self.shx, self.shy):
            sh.close()
            sh.unlink()


def cpu_matrix_based(m=12):
    """The paper's matrix-based comparator (Sec. 4) with the oracle on one host core: assembly of the
    sparse tangent (Problem.tangent_raw) and its CSR SpMV (scipy), on an m^3 Q2 sample of the problem."""
    from oracle.fem import Problem
    from paper_1904_13131_gb300 import inputs
    pr = inputs.problem(DIM, K, m, n_levels=1, top=0)
    P = Problem(DIM, K, m, pr["ids"][0], pr["mu"], pr["lam"], pr["masks"])
    u = inputs.smooth_field(DIM, K, m, seed=0)
    x = inputs.gaussian_vector(P.n_dofs, seed=1)
    t0 = time.perf_counter()
    A = P.tangent_raw(u)
    t_asm = time.perf_counter() - t0
    ts = []
    for _ in range(10):
        t0 = time.perf_counter()
        A @ x
        ts.append(time.perf_counter() - t0)
    t_spmv = float(np.median(ts))
    return {"sample": f"{m}^3 Q2 ({P.n_dofs} dofs, {A.nnz} nonzeros), one core",
            "assembly_s": t_asm, "assembly_s_per_cell": t_asm / m**DIM,
            "csr_spmv_ms": t_spmv * 1e3, "csr_spmv_gdofs": P.n_dofs / t_spmv / 1e9,
            "csr_bytes_per_spmv": int(A.nnz * 12 + (A.shape[0] + 1) * 4 + 2 * A.shape[0] * 8)}


def cpu_newton_config1():
    """The oracle's Newton (sparse direct solves) on the 2D 16^2 Q2 inclusion problem, 5 load steps."""
    from oracle.fem import Problem
    from oracle.newton import newton_solve
    from paper_1904_13131_gb300 import inputs
    dim, k, m = 2, 2, 16
    pr = inputs.problem(dim, k, m, top=inputs.normal_top_mask(dim))
    P = Problem(dim, k, m, pr["ids"][0], pr["mu"], pr["lam"], pr["masks"])
    X = inputs.node_coords(dim, k, m)
    ubc = np.zeros((P.n_nodes, dim))
    ubc[np.isclose(X[:, 1], 1.0), 1] = -0.1
    t0 = time.perf_counter()
    _, rep = newton_solve(P, ubc.reshape(-1), load_steps=5)
    return {"problem": "2D 16^2 Q2 inclusion, top -0.1 in 5 load steps (2,178 dofs), one core",
            "seconds": time.perf_counter() - t0, "newton_iterations": rep["iterations"]}


def cpu_baseline(x):
    """cpu_baseline of the GPU arm: the oracle's action on the full apply workload over all host cores
    (one warm-up application, then one step = the three variants' applications, which the oracle computes
    alike), plus the matrix-based comparator and a Newton solve of the oracle on one core each."""
    pool = OraclePool(M)
    try:
        pool.apply(x)
        t0 = time.perf_counter()
        for _ in VARIANTS:
            pool.apply(x)
        el = time.perf_counter() - t0
    finally:
        pool.close()
    rate = 3 * inputs_ndofs() / el / 1e9
    return {"value": rate, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
            "sample": f"the full workload (32^3 Q2, {inputs_ndofs()} dofs), one step = {len(VARIANTS)} "
                      f"element-by-element applications of the oracle in {el:.1f} s, after one warm-up "
                      f"application; {pool.workers} spawned host processes",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "matrix_based": cpu_matrix_based(), "newton": cpu_newton_config1()}


def run_reference(args, rank, world, budget_s=150.0):
    """The reference arm: the oracle as it stands, on the host cores, stepping through the same workload
    (one step = the three applications). If full steps would not fit the time budget, every step applies
    the oracle to the same leading fraction of the cells and counts only those cells' dofs."""
    if rank != 0:
        return
    from paper_1904_13131_gb300 import inputs
    x = inputs.gaussian_vector(inputs_ndofs(), seed=1)
    pool = OraclePool(M)
    try:
        t0 = time.perf_counter()
        for _ in VARIANTS:
            pool.apply(x)
        t_full = time.perf_counter() - t0
        n_cells = pool.ncells
        if (args.steps + args.warmup - 1) * t_full > budget_s:
            frac = max(budget_s / ((args.steps + args.warmup - 1) * t_full), 1.0 / 64)
            n_cells = max(1, int(pool.ncells * frac))
        for _ in range(args.warmup - 1):
            for _ in VARIANTS:
                pool.apply(x, n_cells)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for _ in VARIANTS:
                pool.apply(x, n_cells)
        el = time.perf_counter() - t0
    finally:
        pool.close()
    units = len(VARIANTS) * inputs_ndofs() * n_cells / pool.ncells * args.steps
    rate = units / el / 1e9
    sample = (f"{args.steps} steps of {len(VARIANTS)} element-by-element applications of the oracle over "
              f"{n_cells} of the {pool.ncells} cells of the 32^3 Q2 workload ({n_cells / pool.ncells:.3f} of it; "
              f"dofs counted in proportion) in {el:.1f} s after {args.warmup} warm-up steps; "
              f"{pool.workers} spawned host processes")
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)", "cells_per_step": n_cells},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": pool.workers, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model()},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def inputs_ndofs():
    return DIM * (K * M + 1) ** DIM


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--only", default=None, help="profile mode: VARIANT:f64|f32, a few applications of one kernel")
    ap.add_argument("--form", type=int, default=-1, help="profile mode: kernel form (0 point, 1 line, -1 tuned)")
    ap.add_argument("--m", type=int, default=M, help="profile mode: cells per direction of the Q2 cube")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--serve-requests", type=int, default=12, help="requests in the serving section (0 = skip)")
    ap.add_argument("--serve-only", action="store_true")
    ap.add_argument("--serve-seq-every", type=int, default=1,
                    help="sequential FP64 baseline on every n-th request only (long streams)")
    ap.add_argument("--no-serve-poisson", dest="serve_poisson", action="store_false")
    ap.add_argument("--serve-rate", type=float, default=None,
                    help="Poisson arrival rate per second (default: twice the sequential baseline's solves/s)")
    ap.add_argument("--no-batch", dest="batch", action="store_false", help="skip the work-list batch section")
    ap.add_argument("--batch-only", action="store_true")
    ap.add_argument("--solve-only", action="store_true")
    ap.add_argument("--vcycle", action="store_true", help="profile mode: V-cycles of the 32^3 Q2 hierarchy")
    ap.add_argument("--profile-all", action="store_true",
                    help="profile mode: one application of every variant in FP64, then FP32, tuned forms, inside "
                         "the NVTX range 'measure' (ncu --nvtx --nvtx-include measure/)")
    ap.add_argument("--configs", action="store_true", help="the degree sweep at 6-51M dofs and the 64^3 mixed study")
    ap.add_argument("--sweep", default=None,
                    help="--configs: meshes as degree:cells:levels,... (default: all eight), no mixed study")
    ap.add_argument("--fastest-only", action="store_true", help="--configs: the fastest mode alone")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    from paper_1904_13131_gb300 import api, build, inputs
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream(dev)
    if args.only:
        var, dt = args.only.split(":")
        mo = args.m
        pr = inputs.problem(DIM, K, mo, n_levels=1, top=0)
        u = torch.tensor(inputs.smooth_field(DIM, K, mo, seed=0), device=dev)
        x = torch.tensor(inputs.gaussian_vector(inputs.n_dofs(DIM, K, mo), seed=1), device=dev)
        code = {"f64": 0, "f32": 1, "ff": 2}[dt]
        with api.Context(dev.index) as c:
            c.setup_problem(pr)
            c.set_solver_params(coarse_eig_iters=5, kernel_form=args.form, fine_dtype=api.FF if code == 2 else api.F64)
            c.set_displacement(u, var, level_dtype=1 if code == 1 else 0)
            xin = x.float() if code == 1 else x
            y = torch.empty_like(xin)
            for _ in range(args.reps):
                c.apply_tangent(xin, y, dtype=code)
            torch.cuda.synchronize()
        print(json.dumps({"only": args.only, "reps": args.reps}))
        return
    if args.profile_all:
        # profile mode: the workload's contexts (caches of every precision, tuned kernel forms), then one
        # application per (precision, variant) inside an NVTX range that ncu can select
        _, _, x, ctxs = setup_contexts(torch, api, inputs, dev)
        x32 = x.float()
        y64, y32 = torch.empty_like(x), torch.empty_like(x32)
        torch.cuda.synchronize()
        forms = {}
        torch.cuda.nvtx.range_push("measure")
        for dt, xin, y in ((0, x, y64), (1, x32, y32)):
            for v in ALL_VARIANTS:
                ctxs[v].apply_tangent(xin, y, dtype=dt)
                forms[f"{v}:{'f64' if dt == 0 else 'f32'}"] = FORMS[ctxs[v].kernel_form(-1, dt)]
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        for c in ctxs.values():
            c.close()
        print(json.dumps({"profile_all": forms}))
        return
    if args.vcycle:
        # profile mode: V-cycles of the 32^3 Q2 hierarchy (4 levels) in the fastest mode; the first call
        # captures the graph, then args.reps timed replays
        pr = inputs.problem(DIM, K, M, n_levels=4, top=inputs.normal_top_mask(DIM))
        with api.Context(dev.index) as c:
            c.setup_problem(pr)
            c.set_solver_params(coarse_solver=2, fine_dtype=api.FF, level_variant=api.VARIANTS["T2"])
            c.set_displacement(torch.tensor(inputs.smooth_field(DIM, K, M, seed=0, amplitude=0.02), device=dev),
                               "T4", level_dtype=1)
            b = torch.tensor(inputs.gaussian_vector(c.num_dofs(), seed=1), device=dev)
            z = torch.empty_like(b)
            n0 = c.kernel_launches()
            c.gmg_vcycle(b, z)
            torch.cuda.synchronize()
            per = c.kernel_launches() - n0
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.reps):
                c.gmg_vcycle(b, z)
            e1.record(stream)
            e1.synchronize()
            print(json.dumps({"vcycle_ms": e0.elapsed_time(e1) / args.reps, "reps": args.reps,
                              "kernels_per_vcycle": per,
                              "forms_f32": [c.kernel_form(level, 1) for level in range(4)]}))
        return
    if args.configs:
        sweep = [tuple(int(v) for v in item.split(":")) for item in args.sweep.split(",")] if args.sweep else None
        print(json.dumps({"configs": config_study(torch, api, inputs, dev, sweep=sweep, mixed_study=sweep is None,
                                                   paper_max_dofs=0 if args.fastest_only else 60_000_000)}),
              flush=True)
        return
    if args.solve_only:
        print(json.dumps({"solve": solve_latency(torch, api, inputs, dev)}), flush=True)
        return
    if args.batch_only:
        print(json.dumps({"batch": batch_bench(torch, api, inputs, dev, stream)}), flush=True)
        return
    if args.serve_only:
        print(json.dumps({"serve": serve_bench(api, inputs, dev, args.serve_requests, seq_every=args.serve_seq_every,
                                               poisson=args.serve_poisson, rate=args.serve_rate)}), flush=True)
        return
    pr, u, x, ctxs = setup_contexts(torch, api, inputs, dev)
    n = inputs.n_dofs(DIM, K, M)
    ncells = M**DIM
    nqp = ncells * (K + 1) ** DIM
    flush = L2Flush(torch, dev)

    # ---- timed region: K steps of {T4, FC, NC} FP64 applications --------------------------------
    clk = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    t_wall = time.perf_counter()
    ms, ys, launches_timed = time_applies(torch, ctxs, VARIANTS, x, 0, args.steps, args.warmup, flush, stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - t_wall
    clocks = clk.stop()
    rate, total_ms = whole_job_rate(torch, dist, float(ms.sum()), 3 * n * args.steps, dev)
    value = rate / 1e9
    per_var_ms = {v: float(np.median(ms[:, i])) for i, v in enumerate(VARIANTS)}

    # ---- per-variant FP64 / FP32 throughput (untimed for the headline) ---------------------------
    ms64, _, _ = time_applies(torch, ctxs, ALL_VARIANTS, x, 0, 5, 2, flush, stream)
    ms32, _, _ = time_applies(torch, ctxs, ALL_VARIANTS, x, 1, 5, 2, flush, stream)
    msff, _, _ = time_applies(torch, ctxs, ALL_VARIANTS, x, 2, 5, 2, flush, stream)
    hbm, hbm_src, fp64_peak = peaks()
    variants = {}
    for i, v in enumerate(ALL_VARIANTS):
        t64, t32, tff = float(np.median(ms64[:, i])), float(np.median(ms32[:, i])), float(np.median(msff[:, i]))
        variants[v] = {
            "f64_gdofs": n / (t64 * 1e-3) / 1e9, "f64_ms": t64,
            "f64_tflops": flops_per_qp(v) * nqp / (t64 * 1e-3) / 1e12,
            "f32_gdofs": n / (t32 * 1e-3) / 1e9, "f32_ms": t32,
            "f32_gbs": bytes_per_apply(v, 4, nqp, n) / (t32 * 1e-3) / 1e9,
            "f32_hbm_frac": bytes_per_apply(v, 4, nqp, n) / (t32 * 1e-3) / 1e9 / hbm,
            "ff_gdofs": n / (tff * 1e-3) / 1e9, "ff_ms": tff,
            "ff_tflops_fp64_equiv": flops_per_qp(v) * nqp / (tff * 1e-3) / 1e12,
            "f64_form": FORMS[ctxs[v].kernel_form(-1, 0)], "f32_form": FORMS[ctxs[v].kernel_form(-1, 1)],
            "ff_form": FORMS[ctxs[v].kernel_form(-1, 2)],
        }
    # the second volumetric function (law 1) and curved (isoparametric) cells through every variant in FP64
    # and FP32: T4 and T2 fold both into their cached state, so their applies should cost what they cost on
    # the lattice; FC, SC and NC run their general build (the reference map of every Gauss point read from
    # the cache, the law chosen at run time), which has no double-float action
    def relinearise(v, law=None, X=None, restore=False):
        general_ff = v in ("FC", "SC", "NC")
        if law is not None:
            ctxs[v].set_material_law(law)
        if X is not None or restore:
            ctxs[v].set_geometry(X)
        ctxs[v].set_solver_params(fine_dtype=api.FF if (restore or not general_ff) else api.F64)
        ctxs[v].set_displacement(u, v, level_dtype=1)

    steady = f32_steady_state(torch, api, inputs, dev, hbm)
    second_law, curved = {}, {}
    for v in ALL_VARIANTS:
        relinearise(v, law=api.LAW_J2)
    msl64, _, _ = time_applies(torch, ctxs, ALL_VARIANTS, x, 0, 5, 2, flush, stream)
    msl32, _, _ = time_applies(torch, ctxs, ALL_VARIANTS, x, 1, 5, 2, flush, stream)
    for i, v in enumerate(ALL_VARIANTS):
        t64, t32 = float(np.median(msl64[:, i])), float(np.median(msl32[:, i]))
        second_law[v] = {"f64_ms": t64, "f64_gdofs": n / (t64 * 1e-3) / 1e9, "f32_ms": t32,
                         "f32_gdofs": n / (t32 * 1e-3) / 1e9}
        relinearise(v, law=api.LAW_LOG2, restore=True)
    Xc = torch.tensor(inputs.curved_coords(DIM, K, M).reshape(-1), device=dev)
    for v in ALL_VARIANTS:
        relinearise(v, X=Xc)
    msc64, _, _ = time_applies(torch, ctxs, ALL_VARIANTS, x, 0, 5, 2, flush, stream)
    msc32, _, _ = time_applies(torch, ctxs, ALL_VARIANTS, x, 1, 5, 2, flush, stream)
    for i, v in enumerate(ALL_VARIANTS):
        t64, t32 = float(np.median(msc64[:, i])), float(np.median(msc32[:, i]))
        curved[v] = {"f64_ms": t64, "f64_gdofs": n / (t64 * 1e-3) / 1e9, "f32_ms": t32,
                     "f32_gdofs": n / (t32 * 1e-3) / 1e9}
        relinearise(v, restore=True)
    del Xc
    # dominant kernel of the step: the slowest variant's FP64 apply (FP64-pipe bound). achieved = the scope
    # table's algorithmic flops per dof x dofs per launch / event time; the count of the kernel's own
    # arithmetic (flops_per_qp, FMA = 2) is reported beside it
    dom = max(per_var_ms, key=per_var_ms.get)
    t_dom = per_var_ms[dom] * 1e-3
    kname = "apply_line_kernel" if ctxs[dom].kernel_form(-1, 0) == 1 else "apply_kernel"
    kfull = f"{kname}<3,3,{dom},double>"
    scope = SCOPE_FLOPS_PER_DOF.get(dom)
    alg = scope * n if scope else flops_per_qp(dom) * nqp
    ach = alg / t_dom / 1e12
    roofline = {"bound": "alu", "kernel": kfull, "achieved": ach, "peak": fp64_peak,
                "unit": "TFLOP/s", "frac": ach / fp64_peak, "traffic": captured_traffic(kfull),
                "traffic_unit": "bytes per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
                "peak_source": "FP64 pipe: 2 DFMA/clk/SM x 152 SMs x 2.07 GHz (derived, nominal 1.25 TFLOP/s)",
                "algorithmic_flops_per_launch": alg,
                "flops_per_dof": scope if scope else flops_per_qp(dom) * nqp / n,
                "kernel_count_flops_per_launch": flops_per_qp(dom) * nqp,
                "kernel_count_frac": flops_per_qp(dom) * nqp / t_dom / 1e12 / fp64_peak,
                "algorithmic_bytes_per_launch": bytes_per_apply(dom, 8, nqp, n),
                "kernel_source_sha256": kernel_source_sha()}

    # ---- end to end through the public API: pinned host x -> device, 3 applies, results -> host ----
    # each result goes to the host on a copy stream while the next variant computes
    xh = x.cpu().pin_memory()
    yh = {v: torch.empty(n, dtype=torch.float64).pin_memory() for v in VARIANTS}
    xd = torch.empty_like(x)
    copy_stream = torch.cuda.Stream(dev)
    e2e_ms = []
    for it in range(args.warmup + args.steps):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xd.copy_(xh, non_blocking=True)
        for v in VARIANTS:
            ctxs[v].apply_tangent(xd, ys[v])
            done = torch.cuda.Event()
            done.record(stream)
            copy_stream.wait_event(done)
            with torch.cuda.stream(copy_stream):
                yh[v].copy_(ys[v], non_blocking=True)
        stream.wait_stream(copy_stream)
        e1.record(stream)
        e1.synchronize()
        if it >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_rate, _ = whole_job_rate(torch, dist, float(np.sum(e2e_ms)), 3 * n * len(e2e_ms), dev)
    e2e = {"value": e2e_rate / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": int(x.numel() * 8), "d2h_bytes_per_step": int(3 * n * 8)}

    solve = None
    if not args.no_solve and rank == 0:
        for c in ctxs.values():
            c.close()
        try:
            solve = solve_latency(torch, api, inputs, dev)
        except api.HyError as e:
            solve = {"error": str(e)}

    serve = None
    if args.serve_requests > 0 and rank == 0:
        try:
            serve = serve_bench(api, inputs, dev, args.serve_requests)
        except api.HyError as e:
            serve = {"error": str(e)}

    batch = None
    if args.batch and rank == 0:
        try:
            batch = batch_bench(torch, api, inputs, dev, stream)
        except api.HyError as e:
            batch = {"error": str(e)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(x.cpu().numpy())

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "dofs": n, "cells": ncells, "degree": K, "dim": DIM,
                           "variants_per_step": list(VARIANTS), "l2": "flushed before every application (256 MB write, then 256 MB read)",
                           "parallelism": f"replicas x{world}"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": int(launches_timed),
                "per_variant_ms_f64": per_var_ms, "variants": variants, "second_law": second_law, "curved": curved,
                "f32_steady_state_64cube": steady, "solve": solve,
                "serve": serve, "batch": batch,
                "wall_s_timed_region": wall, "hbm_peak_gbs": hbm, "hbm_peak_source": hbm_src}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
