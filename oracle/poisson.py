"""Scalar Poisson problem of Sec. 5.1 (test infrastructure only).

Paper passage: Sec. 5.1 solves -Laplace(u) = f on a square with u = 0 on the
boundary by the same pCGMG (Alg. 2 preconditioned by Alg. 1), on 16 x 16 to
256 x 256 meshes coarsened down to a 2 x 2 grid (Table 1).  The paper gives
the problem, the meshes and the levels, not the discretisation; the reading
here is the one its elasticity problem uses: unit-square Q4 (bilinear)
elements, one DOF per node, element matrix KE = integral of grad N_a . grad N_b
(Eq. 7 with the strain-displacement matrix replaced by the gradient of the
shape functions and D by the identity), 2 x 2 Gauss quadrature.

Readings (the paper does not fix these):
  * every node of the four edges is fixed (u = 0 on the boundary);
  * nodes (nelx+1) x (nely+1), x fastest; vectors are [nely+1][nelx+1];
  * the right-hand side is the nodal load vector of the caller (the bench
    uses f = 1 at every node, i.e. a uniform unit source on unit elements);
  * the coarse operators are Galerkin, K_c = P^T K P with bilinear P; for the
    constant-coefficient Q4 Laplacian this equals the operator rediscretised
    on the coarse mesh (the 2-D element matrix does not depend on the
    element size);
  * smoothing, cycle and Krylov method as for elasticity (damped Jacobi,
    Alg. 1, Alg. 2, coarsest solve by Alg. 3).
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import cholesky, multigrid, pcg

_CORNERS = ((-1.0, -1.0), (1.0, -1.0), (1.0, 1.0), (-1.0, 1.0))


def gradient_matrix(xi, eta):
    """Rows d/dx and d/dy of the four bilinear shape functions at (xi, eta),
    for the unit square mapped from [-1, 1]^2 (d/dx = 2 d/dxi)."""
    G = np.zeros((2, 4))
    for a, (xa, ea) in enumerate(_CORNERS):
        G[0, a] = 2.0 * 0.25 * xa * (1.0 + eta * ea)
        G[1, a] = 2.0 * 0.25 * ea * (1.0 + xi * xa)
    return G


def element_matrix():
    """KE = integral over the unit element of G^T G, 2 x 2 Gauss (exact here)."""
    g = 1.0 / np.sqrt(3.0)
    KE = np.zeros((4, 4))
    for xi in (-g, g):
        for eta in (-g, g):
            G = gradient_matrix(xi, eta)
            KE += G.T @ G * 0.25  # weights 1 x 1, det J = 1/4
    return KE


def element_nodes(nelx, nely):
    """[n_el, 4] node indices of every element, counter-clockwise from the bottom-left."""
    j, i = np.meshgrid(np.arange(nely), np.arange(nelx), indexing="ij")
    n0 = (j * (nelx + 1) + i).ravel()
    return np.stack([n0, n0 + 1, n0 + nelx + 2, n0 + nelx + 1], axis=1)


def assemble(nelx, nely, KE, k=None):
    """K = sum_e k_e KE over the element nodes (k = 1 when None), CSR."""
    nodes = element_nodes(nelx, nely)
    n = (nelx + 1) * (nely + 1)
    kk = np.ones(nelx * nely) if k is None else np.asarray(k, dtype=np.float64).ravel()
    rows = np.repeat(nodes, 4, axis=1).ravel()
    cols = np.tile(nodes, (1, 4)).ravel()
    vals = (kk[:, None, None] * KE[None]).ravel()
    return sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()


def free_nodes(nelx, nely):
    """Indices of the interior nodes (every boundary node is fixed)."""
    j, i = np.meshgrid(np.arange(nely + 1), np.arange(nelx + 1), indexing="ij")
    interior = (i > 0) & (i < nelx) & (j > 0) & (j < nely)
    return np.flatnonzero(interior.ravel())


def prolongation(nelx_c, nely_c):
    """Scalar bilinear interpolation from the coarse to the twice finer mesh."""
    return sp.kron(multigrid.prolongation_1d(nely_c), multigrid.prolongation_1d(nelx_c)).tocsr()


def build_hierarchy(nelx, nely, n_coarsen, factor_coarsest=True):
    """[level_0 (coarsest), ..., level_L (finest)] as multigrid.Level objects
    (free nodes, K on them, its diagonal, P from the next coarser level), so
    that the oracle's Alg. 1 (multigrid.mg_cycle) runs on them unchanged."""
    if nelx % (1 << n_coarsen) or nely % (1 << n_coarsen):
        raise ValueError("mesh must be divisible by 2**n_coarsen")
    KE = element_matrix()
    free = free_nodes(nelx, nely)
    levels = [multigrid.Level(nelx, nely, free, assemble(nelx, nely, KE)[free][:, free])]
    for _ in range(n_coarsen):
        fine = levels[-1]
        ncx, ncy = fine.nelx // 2, fine.nely // 2
        free_c = free_nodes(ncx, ncy)
        P = prolongation(ncx, ncy)[fine.free][:, free_c].tocsr()
        fine.P = P
        levels.append(multigrid.Level(ncx, ncy, free_c, (P.T @ fine.K @ P).tocsr()))
    levels.reverse()
    if factor_coarsest and levels[0].n_free > 0:
        levels[0].chol = cholesky.cholesky(levels[0].K.toarray())
    return levels


def solve_direct(nelx, nely, f):
    """u = K_ff^-1 f_f with u = 0 on the boundary, [nely+1][nelx+1]."""
    K = assemble(nelx, nely, element_matrix())
    free = free_nodes(nelx, nely)
    f = np.asarray(f, dtype=np.float64).ravel()
    u = np.zeros_like(f)
    u[free] = spla.spsolve(K[free][:, free].tocsc(), f[free])
    return u.reshape(nely + 1, nelx + 1)


def solve_pcgmg(nelx, nely, f, n_coarsen, omega=0.6, nu1=2, nu2=2, tol=1e-10, max_it=1000,
                gamma=1, u0=None):
    """Alg. 2 preconditioned by one cycle of Alg. 1 on the scalar problem.
    Returns a dict: u [nely+1][nelx+1] (zero on the boundary), iters,
    converged, history, levels."""
    levels = build_hierarchy(nelx, nely, n_coarsen)
    free = levels[-1].free
    K = levels[-1].K
    f = np.asarray(f, dtype=np.float64).ravel()
    x0 = None if u0 is None else np.asarray(u0, dtype=np.float64).ravel()[free]
    M = multigrid.vcycle_preconditioner(levels, omega, nu1, nu2, gamma)
    uf, iters, conv, hist = pcg.pcg(lambda v: K @ v, f[free], M, x0=x0, tol=tol, max_it=max_it)
    u = np.zeros_like(f)
    u[free] = uf
    return dict(u=u.reshape(nely + 1, nelx + 1), iters=iters, converged=conv, history=hist,
                levels=levels)


def sine_mode(nelx, nely, k, l):
    """Nodal values sin(k pi i / nelx) sin(l pi j / nely), [nely+1][nelx+1]."""
    i = np.arange(nelx + 1)
    j = np.arange(nely + 1)
    return np.outer(np.sin(l * np.pi * j / nely), np.sin(k * np.pi * i / nelx))
