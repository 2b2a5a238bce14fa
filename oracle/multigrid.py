"""Multigrid pieces of the oracle (test infrastructure only).

Paper passages: Sec. 2.1 (nested grids Omega_0 ... Omega_m, transfer operators
R_l and P_l, the two-level formula Eq. 1, the gamma-cycle of Alg. 1) and
Sec. 2.3 (the damped Jacobi iteration x <- (I - w D^-1 A) x + w D^-1 b).

Levels are numbered as in Alg. 1: level 0 is the coarsest grid, level L the
finest.  Each coarser grid halves nelx and nely.

Readings (the paper does not fix these):
  * P_l is bilinear interpolation of both displacement components from the
    coarse nodes to the fine nodes; R_l = P_l^T.
  * The coarse operator is either Galerkin, K_{l-1} = P_l^T K_l P_l, or
    rediscretised: the same Q4 element matrix scaled by the arithmetic mean of
    the four child moduli (Sec. 2.1 speaks of a discretisation on each mesh).
  * A coarse node is clamped exactly when it lies on a clamped edge; all
    operators act on the free DOFs only.
  * The finest level calls the next coarser grid once and every other level
    calls it gamma times (Alg. 1 sets gamma = 1 on the finest grid): gamma = 1
    is the V-cycle, gamma = 2 the W-cycle.  Each repeated call starts from the
    coarse iterate that the previous one returned.  The smoother is damped
    Jacobi with nu1 pre- and nu2 post-sweeps; the coarsest system is solved by
    the dense Cholesky factorisation of Alg. 3.
"""

import numpy as np
import scipy.sparse as sp

from . import cholesky, fem


def prolongation_1d(n_c):
    """1-D linear interpolation from n_c + 1 coarse nodes to 2 n_c + 1 fine nodes.

    A fine node at an even index coincides with a coarse node (weight 1); at an
    odd index it sits midway between two coarse nodes (weights 1/2 each).
    """
    rows, cols, vals = [], [], []
    for I in range(n_c + 1):
        rows.append(2 * I)
        cols.append(I)
        vals.append(1.0)
    for I in range(n_c):
        rows += [2 * I + 1, 2 * I + 1]
        cols += [I, I + 1]
        vals += [0.5, 0.5]
    return sp.coo_matrix((vals, (rows, cols)), shape=(2 * n_c + 1, n_c + 1)).tocsr()


def prolongation(nelx_c, nely_c):
    """Bilinear P from the coarse mesh (nelx_c x nely_c) to the mesh twice as fine.

    Full-DOF matrix of shape (2 n_fine_nodes, 2 n_coarse_nodes).  Bilinear
    interpolation is the tensor product of the 1-D rule in y (slow node index)
    and x (fast node index), applied to each displacement component alike
    (the trailing 2x2 identity keeps u_x and u_y interleaved).
    """
    Pn = sp.kron(prolongation_1d(nely_c), prolongation_1d(nelx_c))
    return sp.kron(Pn, sp.identity(2)).tocsr()


class Level:
    """One grid of the hierarchy: mesh size, free DOFs and operators on them.

    K    -- stiffness restricted to the free DOFs (CSR).
    diag -- diag(K), the Jacobi diagonal D of Sec. 2.3.
    P    -- prolongation from the next coarser level, free rows and free
            columns only (None on level 0).
    E    -- element moduli used to build K (None for Galerkin coarse levels).
    """

    def __init__(self, nelx, nely, free, K, E=None):
        self.nelx, self.nely = nelx, nely
        self.free = free
        self.K = K.tocsr()
        self.diag = self.K.diagonal().copy()
        self.P = None
        self.E = E
        self.chol = None

    @property
    def n_free(self):
        return self.free.size


def build_hierarchy(nelx, nely, E, KE, fixed_edges, n_coarsen, coarse_kind="galerkin",
                    factor_coarsest=True):
    """Return [level_0 (coarsest), ..., level_L (finest)].

    The finest operator is the assembled K of Eq. 7 restricted to the free DOFs.
    coarse_kind: "galerkin" (K_c = P^T K P) or "rediscretize" (mean child E).
    factor_coarsest=False skips the dense Cholesky factor of level 0 (Alg. 3,
    cubic in its size) for callers that only need the operators.
    """
    if nelx % (1 << n_coarsen) or nely % (1 << n_coarsen):
        raise ValueError("mesh must be divisible by 2**n_coarsen")
    E = np.asarray(E, dtype=np.float64).reshape(nely, nelx)
    free = fem.free_dofs(nelx, nely, fixed_edges)
    K = fem.assemble(nelx, nely, E, KE)[free][:, free]
    levels = [Level(nelx, nely, free, K, E)]
    for _ in range(n_coarsen):
        fine = levels[-1]
        ncx, ncy = fine.nelx // 2, fine.nely // 2
        free_c = fem.free_dofs(ncx, ncy, fixed_edges)
        P = prolongation(ncx, ncy)[fine.free][:, free_c].tocsr()
        if coarse_kind == "galerkin":
            Kc = (P.T @ fine.K @ P).tocsr()
            Ec = None
        elif coarse_kind == "rediscretize":
            Ef = fine.E
            Ec = 0.25 * (Ef[0::2, 0::2] + Ef[0::2, 1::2] + Ef[1::2, 0::2] + Ef[1::2, 1::2])
            Kc = fem.assemble(ncx, ncy, Ec, KE)[free_c][:, free_c]
        else:
            raise ValueError(coarse_kind)
        fine.P = P
        levels.append(Level(ncx, ncy, free_c, Kc, Ec))
    levels.reverse()
    levels[0].chol = cholesky.cholesky(levels[0].K.toarray()) if factor_coarsest else None
    return levels


def damped_jacobi(K, diag, x, b, omega, sweeps):
    """Sec. 2.3: x_{k+1} = (I - w D^-1 K) x_k + w D^-1 b, applied `sweeps` times."""
    for _ in range(sweeps):
        x = x + omega * (b - K @ x) / diag
    return x


def mg_cycle(levels, l, U, F, omega, nu1, nu2, gamma=1):
    """Alg. 1, MG_gamma^l(U_l, F_l), returning the new U_l.

    l == 0: U = K_0^-1 F (Cholesky, Alg. 3).  Otherwise: pre-smooth nu1 times,
    restrict the residual F_{l-1} = R_l (F_l - K_l U_l), start the coarse
    iterate at zero, call the scheme on level l-1 (once when l is the finest
    level, gamma times otherwise), correct with U_l += P_l U_{l-1},
    post-smooth nu2 times.
    """
    lev = levels[l]
    if l == 0:
        return cholesky.cholesky_solve(lev.chol, F)
    U = damped_jacobi(lev.K, lev.diag, U, F, omega, nu1)
    Fc = lev.P.T @ (F - lev.K @ U)
    Uc = np.zeros(levels[l - 1].n_free)
    calls = 1 if l == len(levels) - 1 else gamma
    for _ in range(calls):
        Uc = mg_cycle(levels, l - 1, Uc, Fc, omega, nu1, nu2, gamma)
    U = U + lev.P @ Uc
    return damped_jacobi(lev.K, lev.diag, U, F, omega, nu2)


def vcycle_preconditioner(levels, omega=0.6, nu1=2, nu2=2, gamma=1):
    """z = M^-1 r: one cycle of Alg. 1 on the finest level started from U = 0
    (Sec. 2.2); a V-cycle for gamma = 1, a W-cycle for gamma = 2."""
    L = len(levels) - 1

    def apply(r):
        return mg_cycle(levels, L, np.zeros_like(r), r, omega, nu1, nu2, gamma)

    return apply


def two_level_correction(K, P, Kc, U, F):
    """Eq. 1: U_new = U - P K_c^-1 R (K U - F), with R = P^T and a dense solve."""
    Kc = Kc.toarray() if sp.issparse(Kc) else Kc
    return U - P @ np.linalg.solve(Kc, P.T @ (K @ U - F))
