"""Newton-Raphson with load steps for prescribed boundary displacements and dead tractions (Sec. 3, Sec. 7).

Test infrastructure (see oracle/__init__.py). Each Newton iteration solves Eq. linear_system,
A(u) du = -F(u), on the free dofs with scipy's sparse direct solver. Readings of the paper where it is
silent: displacement-driven loading in S equal steps; the prescribed increment of a
step is lifted into the first linear solve (du_c given, A_ff du_f = -R_f - A_fc du_c); the step
converges when ||R_free|| <= max(rtol * ||first right-hand side||, atol); a step that makes J <= 0
at a Gauss point (Sec. 2.1 requires J > 0) is halved up to 5 times before the solve reports failure
(reading O15). The report lists, per load step, how many halvings each accepted Newton update took.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .fem import Problem


def newton_solve(prob: Problem, u_final_bc, load_steps=5, rtol=1e-10, atol=1e-14, max_iter=25, u0=None,
                 linear_solve=None, f_ext=None):
    """Return (u, report). u_final_bc holds the final prescribed values on constrained dofs; f_ext (optional)
    the final external force of dead loads (Problem.face_load), applied in the same equal increments.

    linear_solve(prob, u, rhs) -> du (free part) overrides the direct solve (used to mirror a GMG-CG).
    """
    u = np.zeros(prob.n_dofs) if u0 is None else np.array(u0, dtype=float)
    cons = prob.constrained
    free = prob.free
    report = {"iterations": [], "residuals": [], "halvings": []}
    for s in range(1, load_steps + 1):
        target = np.where(cons, (s / load_steps) * np.asarray(u_final_bc, dtype=float), 0.0)
        ref = None
        its = 0
        res_hist = []
        halv = []
        while True:
            du0 = np.where(cons, target - u, 0.0)
            R = prob.residual_raw(u)
            if f_ext is not None:
                R = R - (s / load_steps) * np.asarray(f_ext, dtype=float)
            A = prob.tangent_raw(u)
            rhs = -(R + A @ du0)
            rhs[cons] = 0.0
            nr = np.linalg.norm(rhs[free])
            if ref is None:
                ref = nr
            res_hist.append(nr)
            if its > 0 and not np.any(du0) and nr <= max(rtol * ref, atol):
                break
            if its >= max_iter:
                raise RuntimeError(f"Newton did not converge in load step {s}")
            if linear_solve is None:
                Aff = A[free][:, free]
                du = du0.copy()
                du[free] = spla.spsolve(Aff.tocsc(), rhs[free])
            else:
                du = du0 + linear_solve(prob, u, rhs)
            step = 1.0
            for h in range(6):
                trial = u + step * du
                if prob.min_jacobian(trial) > 0:
                    break
                step *= 0.5
            else:
                raise FloatingPointError("J <= 0 after 5 halvings")
            halv.append(h)
            u = trial
            its += 1
        report["iterations"].append(its)
        report["residuals"].append(res_hist)
        report["halvings"].append(halv)
    return u, report
