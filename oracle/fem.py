"""Finite-element pieces of the oracle (test infrastructure only).

Paper passages: Sec. 3.1 Eq. 5 (multi-material SIMP), Eqs. 6-9 (compliance
problem, element stiffness, plane-stress material matrix, strain-displacement
matrix).

Mesh conventions: nelx x nely unit-square Q4 elements; node (i, j) has index
n = j*(nelx+1) + i (x fastest); DOF 2n is u_x and 2n+1 is u_y; element
e = j*nelx + i has its local nodes counter-clockwise from the bottom-left:
(i,j), (i+1,j), (i+1,j+1), (i,j+1).  The paper fixes none of these (Fig. 3 is
missing); they are the project's reading.
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

BOTTOM, LEFT, RIGHT, TOP = 1, 2, 4, 8

# Reference-square corner coordinates (xi_a, eta_a) in the local node order.
_CORNERS = ((-1.0, -1.0), (1.0, -1.0), (1.0, 1.0), (-1.0, 1.0))


def plane_stress_matrix(E, nu):
    """Eq. 8: D = E / (1 - nu^2) [[1, nu, 0], [nu, 1, 0], [0, 0, (1 - nu)/2]]."""
    return E / (1.0 - nu * nu) * np.array(
        [[1.0, nu, 0.0], [nu, 1.0, 0.0], [0.0, 0.0, 0.5 * (1.0 - nu)]]
    )


def strain_displacement(xi, eta):
    """Eq. 9 evaluated for the unit-square element at reference point (xi, eta).

    N_a = (1 + xi xi_a)(1 + eta eta_a) / 4.  The element maps [-1,1]^2 onto
    [0,1]^2 by x = (xi + 1)/2, y = (eta + 1)/2, so d/dx = 2 d/dxi and the
    Jacobian determinant is 1/4.  Rows: eps_xx, eps_yy, gamma_xy.
    """
    B = np.zeros((3, 8))
    for a, (xa, ea) in enumerate(_CORNERS):
        dN_dxi = 0.25 * xa * (1.0 + eta * ea)
        dN_deta = 0.25 * ea * (1.0 + xi * xa)
        dN_dx, dN_dy = 2.0 * dN_dxi, 2.0 * dN_deta
        B[0, 2 * a] = dN_dx
        B[1, 2 * a + 1] = dN_dy
        B[2, 2 * a] = dN_dy
        B[2, 2 * a + 1] = dN_dx
    return B


def element_stiffness(nu, E=1.0):
    """Eq. 7: KE = integral over the element of B^T D B, by 2x2 Gauss quadrature.

    The integrand is at most quadratic in each of xi and eta, so the two-point
    rule (points +-1/sqrt(3), weights 1) is exact.
    """
    D = plane_stress_matrix(E, nu)
    g = 1.0 / np.sqrt(3.0)
    KE = np.zeros((8, 8))
    for xi in (-g, g):
        for eta in (-g, g):
            B = strain_displacement(xi, eta)
            KE += B.T @ D @ B * 0.25  # weight 1 x 1, det J = 1/4
    return KE


def simp_moduli(x, E_phase, penal):
    """Eq. 5: E_e = sum_i x_{e,i}^p E_i^0 over all phases (void included).

    x is [n_phase][nely][nelx]; returns [nely][nelx].  No extra floor is added:
    the void phase carries its own small modulus.
    """
    x = np.asarray(x, dtype=np.float64)
    E_phase = np.asarray(E_phase, dtype=np.float64)
    return np.einsum("i,ijk->jk", E_phase, x ** penal)


def element_nodes(nelx, nely):
    """[n_el, 4] node indices, counter-clockwise from the bottom-left."""
    j, i = np.meshgrid(np.arange(nely), np.arange(nelx), indexing="ij")
    n0 = (j * (nelx + 1) + i).ravel()
    return np.stack([n0, n0 + 1, n0 + nelx + 2, n0 + nelx + 1], axis=1)


def element_dofs(nelx, nely):
    """[n_el, 8] DOF indices in the element's local order (u_x, u_y per node)."""
    nodes = element_nodes(nelx, nely)
    dofs = np.empty((nodes.shape[0], 8), dtype=np.int64)
    dofs[:, 0::2] = 2 * nodes
    dofs[:, 1::2] = 2 * nodes + 1
    return dofs


def fixed_node_mask(nelx, nely, fixed_edges):
    """Boolean [nely+1][nelx+1]: nodes on a clamped edge (both DOFs fixed)."""
    m = np.zeros((nely + 1, nelx + 1), dtype=bool)
    if fixed_edges & BOTTOM:
        m[0, :] = True
    if fixed_edges & TOP:
        m[nely, :] = True
    if fixed_edges & LEFT:
        m[:, 0] = True
    if fixed_edges & RIGHT:
        m[:, nelx] = True
    return m


def free_dofs(nelx, nely, fixed_edges):
    """Sorted global indices of the unconstrained DOFs."""
    fixed = np.repeat(fixed_node_mask(nelx, nely, fixed_edges).ravel(), 2)
    return np.flatnonzero(~fixed)


def assemble(nelx, nely, E, KE):
    """Global K = sum_e E_e KE scattered onto the element DOFs (Eq. 7), CSR."""
    dofs = element_dofs(nelx, nely)
    n_dof = 2 * (nelx + 1) * (nely + 1)
    rows = np.repeat(dofs, 8, axis=1).ravel()
    cols = np.tile(dofs, (1, 8)).ravel()
    vals = (np.asarray(E, dtype=np.float64).ravel()[:, None, None] * KE[None]).ravel()
    return sp.coo_matrix((vals, (rows, cols)), shape=(n_dof, n_dof)).tocsr()


def apply_K(nelx, nely, E, KE, v):
    """Element-by-element K v = sum_e E_e KE v_e, without assembling K.

    The same product as assemble(...) @ v; used where an assembled matrix would
    not fit (full-size residual checks).  v is any array of 2(nelx+1)(nely+1)
    values in the node-interleaved layout.
    """
    dofs = element_dofs(nelx, nely)
    v = np.asarray(v, dtype=np.float64).ravel()
    ve = v[dofs]  # [n_el, 8]
    ye = (np.asarray(E, dtype=np.float64).ravel()[:, None]) * (ve @ KE.T)
    return np.bincount(dofs.ravel(), weights=ye.ravel(), minlength=v.size)


def direct_solve(K, f, free):
    """u = K_ff^-1 f_f with u = 0 on the fixed DOFs (the plain definition)."""
    f = np.asarray(f, dtype=np.float64).ravel()
    Kff = K[free][:, free].tocsc()
    u = np.zeros_like(f)
    u[free] = spla.spsolve(Kff, f[free])
    return u
