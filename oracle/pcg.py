"""Preconditioned conjugate gradient (test infrastructure only).

Paper passage: Sec. 2.2, Alg. 2.

Readings:
  * Alg. 2 computes z_i before testing r_i = 0.  Here the test comes first and
    is relative: stop when ||r_i||_2 <= tol * ||b||_2 (no preconditioner call is
    spent on a converged residual).  `iters` counts completed x updates.
  * beta_{i-1} = z_i^T r_i / z_{i-1}^T r_{i-1} (Fletcher-Reeves form, as
    printed).  flexible=True uses z_i^T (r_i - r_{i-1}) / z_{i-1}^T r_{i-1}
    instead, the form that tolerates a preconditioner computed in lower
    precision.
  * rr_every = k > 0 replaces the recursive residual by b - A x after every k-th
    update (residual replacement); it is not in the paper.

`trace`, when a list, receives one (p_i, q_i = A p_i, beta used for p_i) tuple
per step; it only records, the arithmetic is the same with or without it.
"""

import numpy as np


def pcg(apply_A, b, apply_M, x0=None, tol=1e-10, max_it=1000, flexible=False, rr_every=0,
        trace=None):
    """Solve A x = b.  Returns (x, iters, converged, history of ||r||/||b||)."""
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    bnorm = np.linalg.norm(b)
    r = b - apply_A(x)
    history = []
    if bnorm == 0.0:
        return np.zeros_like(b), 0, True, history
    p = None
    rho_prev = None
    r_prev = None
    it = 0
    while True:
        rel = np.linalg.norm(r) / bnorm
        history.append(rel)
        if rel <= tol:
            return x, it, True, history
        if it >= max_it:
            return x, it, False, history
        z = apply_M(r)
        rho = z @ r
        if p is None:
            beta = 0.0
            p = z.copy()
        else:
            num = z @ (r - r_prev) if flexible else rho
            beta = num / rho_prev
            p = z + beta * p
        q = apply_A(p)
        if trace is not None:
            trace.append((p.copy(), q.copy(), beta))
        alpha = rho / (p @ q)
        x = x + alpha * p
        r_prev = r
        r = r - alpha * q
        rho_prev = rho
        it += 1
        if rr_every and it % rr_every == 0:
            r = b - apply_A(x)
