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


def element_energy_relative(nelx, nely, KE, u):
    """w_e = u_e^T KE u_e evaluated on the nodal differences u_e - t_e, where t_e
    is the displacement of the element's first node repeated at its four nodes.

    The exact element matrix annihilates rigid translations (Eq. 7: a uniform
    displacement has no strain), so this is the same quantity as
    element_energy.  In floating point it is far more accurate on large
    displacement fields: the differences are of the size of the strains rather
    than of the displacements, and for neighbouring nodes of the same sign
    they are formed exactly.  [nely][nelx].
    """
    ue = np.asarray(u, dtype=np.float64).ravel()[fem.element_dofs(nelx, nely)]
    d = ue - np.tile(ue[:, 0:2], (1, 4))
    return np.einsum("ea,ab,eb->e", d, KE, d).reshape(nely, nelx)


def variational_energy_terms(nelx, nely, E, KE, f, u):
    """Terms whose exact sum is Pi(u) = 2 f.u - u^T K u (K of Eq. 7 with moduli E).

    Pi is stationary (a maximum) at the solution of K u = f, where it equals the
    compliance f.u of Eq. 6: a solve error delta changes it only by
    -delta^T K delta.  Returned unsummed so that a caller can sum the terms of
    two energies together (energy_difference) without rounding either total.
    """
    w = element_energy_relative(nelx, nely, KE, u)
    fu = np.asarray(f, dtype=np.float64).ravel() * np.asarray(u, dtype=np.float64).ravel()
    return np.concatenate([2.0 * fu, -(np.asarray(E, dtype=np.float64) * w).ravel()])


def energy_difference(terms_a, terms_b):
    """Pi_a - Pi_b from their terms, with one rounding (math.fsum is exact)."""
    import math
    return math.fsum(np.concatenate([np.asarray(terms_a), -np.asarray(terms_b)]).tolist())
