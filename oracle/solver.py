"""The whole pCGMG solve, wired from the oracle's pieces (test infrastructure only).

Paper passages: Alg. 2 (PCG) preconditioned by one V-cycle of Alg. 1 on the
Q4 system of Eqs. 5-9; compliance and sensitivities after it (Eq. 6, Sec. 4).
Also the plain definition it must agree with: u = K_ff^-1 f_f.
"""

import time

import numpy as np

from . import fem, multigrid, pcg, sensitivity


def solve_direct(nelx, nely, x, E_phase, penal, f, nu=0.3, fixed_edges=fem.BOTTOM):
    """u = K_ff^-1 f_f by a sparse direct solve; returns u as [nely+1][nelx+1][2]."""
    E = fem.simp_moduli(x, E_phase, penal)
    KE = fem.element_stiffness(nu)
    K = fem.assemble(nelx, nely, E, KE)
    free = fem.free_dofs(nelx, nely, fixed_edges)
    return fem.direct_solve(K, f, free).reshape(nely + 1, nelx + 1, 2)


def solve_pcgmg(nelx, nely, x, E_phase, penal, f, nu=0.3, fixed_edges=fem.BOTTOM,
                n_coarsen=3, omega=0.6, nu1=2, nu2=2, tol=1e-10, max_it=1000,
                coarse_kind="galerkin", u0=None, flexible=False, rr_every=0,
                vcycle_E=None, gamma=1, timings=None):
    """PCG (Alg. 2) preconditioned by one cycle of Alg. 1 (gamma = 1: V-cycle,
    2: W-cycle).

    vcycle_E, when given, replaces the element moduli inside the preconditioner
    only (the mixed-precision path builds its V-cycle from bfloat16 moduli while
    the outer operator keeps the float64 ones).

    Returns a dict: u ([nely+1][nelx+1][2], zero on clamped DOFs), iters,
    converged, history (||r||/||f|| per iteration), E, KE, levels.

    timings, when a dict, receives wall-clock times (observation only):
    "setup_s" (moduli, hierarchy, coarsest factor), "start_s" (from then to
    the first preconditioner call: the initial residual) and "iter_s" (one
    entry per PCG iteration, from one preconditioner call to the next, the
    last one to the end of the loop).
    """
    t0 = time.perf_counter()
    E = fem.simp_moduli(x, E_phase, penal)
    KE = fem.element_stiffness(nu)
    E_pre = E if vcycle_E is None else np.asarray(vcycle_E, dtype=np.float64)
    levels = multigrid.build_hierarchy(nelx, nely, E_pre, KE, fixed_edges, n_coarsen, coarse_kind)
    free = levels[-1].free
    if vcycle_E is None:
        K = levels[-1].K
    else:
        K = fem.assemble(nelx, nely, E, KE)[free][:, free]
    f_full = np.asarray(f, dtype=np.float64).ravel()
    x0 = None if u0 is None else np.asarray(u0, dtype=np.float64).ravel()[free]
    M = multigrid.vcycle_preconditioner(levels, omega, nu1, nu2, gamma)
    if timings is not None:
        stamps = [time.perf_counter()]
        M_untimed = M

        def M(r):
            stamps.append(time.perf_counter())
            return M_untimed(r)

    uf, iters, conv, hist = pcg.pcg(lambda v: K @ v, f_full[free], M, x0=x0, tol=tol,
                                    max_it=max_it, flexible=flexible, rr_every=rr_every)
    if timings is not None:
        stamps.append(time.perf_counter())
        timings["setup_s"] = stamps[0] - t0
        timings["start_s"] = stamps[1] - stamps[0] if len(stamps) > 2 else stamps[-1] - stamps[0]
        timings["iter_s"] = [b - a for a, b in zip(stamps[1:-1], stamps[2:])]
    u = np.zeros_like(f_full)
    u[free] = uf
    return dict(u=u.reshape(nely + 1, nelx + 1, 2), iters=iters, converged=conv,
                history=hist, E=E, KE=KE, levels=levels)


def compliance_and_gradient(nelx, nely, x, E_phase, penal, f, u, nu=0.3):
    """C = f.u and dC/dx [n_phase][nely][nelx] for one load case."""
    KE = fem.element_stiffness(nu)
    w = sensitivity.element_energy(nelx, nely, KE, u)
    return sensitivity.compliance(f, u), sensitivity.compliance_gradient(x, E_phase, penal, w)


def true_relative_residual(nelx, nely, E, f, u, nu=0.3, fixed_edges=fem.BOTTOM):
    """||f - K u|| / ||f|| over the free DOFs, by the element-by-element product."""
    KE = fem.element_stiffness(nu)
    free = fem.free_dofs(nelx, nely, fixed_edges)
    r = np.asarray(f, dtype=np.float64).ravel() - fem.apply_K(nelx, nely, E, KE, u)
    fn = np.linalg.norm(np.asarray(f, dtype=np.float64).ravel()[free])
    return float(np.linalg.norm(r[free]) / fn)
