"""Compliance and its sensitivities (test infrastructure only).

Paper passages: Eq. 6 (the compliance objective, with K(alpha) U = F), Eq. 5
(the multi-material interpolation it differentiates) and Sec. 4 (sensitivity
analysis follows the solve).  The paper does not print the sensitivity
formula; it is the standard self-adjoint result: with K u = f and f fixed,
dC/dtheta = -u^T (dK/dtheta) u, and dK/dx_{e,i} = p x_{e,i}^{p-1} E_i KE on
element e.
"""

import numpy as np

from . import fem


def compliance(f, u):
    """C = f . u (equal to u^T K u at the solution, Eq. 6)."""
    return float(np.dot(np.asarray(f).ravel(), np.asarray(u).ravel()))


def element_energy(nelx, nely, KE, u):
    """w_e = u_e^T KE u_e for the unit-modulus element matrix, [nely][nelx]."""
    ue = np.asarray(u, dtype=np.float64).ravel()[fem.element_dofs(nelx, nely)]
    return np.einsum("ea,ab,eb->e", ue, KE, ue).reshape(nely, nelx)


def compliance_gradient(x, E_phase, penal, w):
    """dC/dx_{e,i} = -p x_{e,i}^{p-1} E_i w_e, [n_phase][nely][nelx]."""
    x = np.asarray(x, dtype=np.float64)
    E_phase = np.asarray(E_phase, dtype=np.float64)
    return -penal * x ** (penal - 1) * E_phase[:, None, None] * np.asarray(w)[None]


def energy_sum(E, w):
    """sum_e E_e w_e, which equals f . u at the exact solution (energy identity)."""
    return float(np.sum(np.asarray(E) * np.asarray(w)))
