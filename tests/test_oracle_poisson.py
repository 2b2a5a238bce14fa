"""Pins of the scalar Poisson oracle (Sec. 5.1) against mathematics.

None of these tests calls the CUDA library.  Closed forms used:
  * the bilinear unit-square Laplace element matrix
    KE = (1/6) [[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]];
  * on an nelx x nely mesh with u = 0 on the boundary, K = K1 (x) M1 + M1 (x) K1
    (1-D stiffness tridiag(-1, 2, -1), 1-D mass tridiag(1, 4, 1) / 6), so the
    discrete sine modes sin(k pi i / nelx) sin(l pi j / nely) are eigenvectors
    with eigenvalue
    [(2 - 2 cos a)(4 + 2 cos b) + (4 + 2 cos a)(2 - 2 cos b)] / 6,
    a = k pi / nelx, b = l pi / nely.
"""

import numpy as np
import pytest

from oracle import multigrid, poisson


def test_element_matrix_closed_form():
    KE = poisson.element_matrix()
    ref = np.array([[4, -1, -2, -1], [-1, 4, -1, -2], [-2, -1, 4, -1], [-1, -2, -1, 4]]) / 6.0
    np.testing.assert_allclose(KE, ref, rtol=0, atol=1e-15)


def eigenvalue(nelx, nely, k, l):
    a, b = k * np.pi / nelx, l * np.pi / nely
    return ((2 - 2 * np.cos(a)) * (4 + 2 * np.cos(b)) + (4 + 2 * np.cos(a)) * (2 - 2 * np.cos(b))) / 6.0


@pytest.mark.parametrize("nelx,nely", [(8, 8), (12, 6)])
def test_sine_modes_are_eigenvectors(nelx, nely):
    K = poisson.assemble(nelx, nely, poisson.element_matrix())
    free = poisson.free_nodes(nelx, nely)
    Kff = K[free][:, free]
    for k, l in ((1, 1), (2, 1), (nelx - 1, 1), (3, nely - 1)):
        v = poisson.sine_mode(nelx, nely, k, l).ravel()[free]
        np.testing.assert_allclose(Kff @ v, eigenvalue(nelx, nely, k, l) * v, atol=1e-13)


def test_linear_fields_are_discrete_harmonic():
    # Interior rows of the full K annihilate linear fields (patch test).
    nelx, nely = 7, 5
    K = poisson.assemble(nelx, nely, poisson.element_matrix())
    J, I = np.meshgrid(np.arange(nely + 1), np.arange(nelx + 1), indexing="ij")
    free = poisson.free_nodes(nelx, nely)
    for u in (1.0 + 0 * I, I.astype(float), 2.0 * J - 0.5 * I + 3.0):
        np.testing.assert_allclose((K @ u.ravel())[free], 0.0, atol=1e-13)
    # A quadratic is not harmonic: x^2 gives the stencil's second difference.
    y = (K @ (I.astype(float) ** 2).ravel())[free]
    np.testing.assert_allclose(y, -2.0, atol=1e-12)


def test_galerkin_coarse_operator_is_the_rediscretised_stencil():
    # Sec. 5.1 coarsens to 2 x 2; the 2-D Q4 Laplacian does not depend on the
    # element size, so P^T K P equals the coarse-mesh assembly on every level.
    lv = poisson.build_hierarchy(16, 16, 3, factor_coarsest=False)
    KE = poisson.element_matrix()
    for L in lv:
        free = poisson.free_nodes(L.nelx, L.nely)
        Kr = poisson.assemble(L.nelx, L.nely, KE)[free][:, free]
        assert abs(L.K - Kr).max() < 1e-13
    assert lv[0].nelx == 2 and lv[0].n_free == 1
    assert lv[0].K[0, 0] == pytest.approx(8.0 / 3.0)


def test_direct_solve_recovers_a_sine_mode():
    nelx, nely = 16, 8
    mode = poisson.sine_mode(nelx, nely, 3, 2)
    f = eigenvalue(nelx, nely, 3, 2) * mode
    np.testing.assert_allclose(poisson.solve_direct(nelx, nely, f), mode, atol=1e-12)


def test_vcycle_is_symmetric_positive_definite():
    lv = poisson.build_hierarchy(32, 32, 4)
    M = multigrid.vcycle_preconditioner(lv)
    rng = np.random.default_rng(0)
    n = lv[-1].n_free
    for _ in range(3):
        a, b = rng.standard_normal(n), rng.standard_normal(n)
        assert a @ M(b) == pytest.approx(b @ M(a), rel=1e-12)
        assert a @ M(a) > 0


@pytest.mark.parametrize("n,nc", [(16, 3), (32, 4), (64, 2)])
def test_pcgmg_converges_to_direct_solution(n, nc):
    f = np.random.default_rng(n).standard_normal((n + 1, n + 1))
    ud = poisson.solve_direct(n, n, f)
    r = poisson.solve_pcgmg(n, n, f, nc, tol=1e-12)
    assert r["converged"]
    assert np.linalg.norm(r["u"] - ud) / np.linalg.norm(ud) < 1e-10
    assert np.all(r["u"][0] == 0) and np.all(r["u"][:, -1] == 0)


def test_iterations_nearly_mesh_independent():
    # Sec. 5.1: the multigrid-preconditioned iteration count hardly grows with
    # the mesh (meshes 16^2 ... 128^2, each coarsened to 2 x 2).
    its = []
    for n in (16, 32, 64, 128):
        r = poisson.solve_pcgmg(n, n, np.ones((n + 1, n + 1)), n.bit_length() - 2, tol=1e-8)
        its.append(r["iters"])
    assert max(its) - min(its) <= 2, its
    # Two grids (one coarsening, exact coarse solve) need no more iterations.
    r0 = poisson.solve_pcgmg(64, 64, np.ones((65, 65)), 1, tol=1e-8)
    assert r0["iters"] <= max(its)


def test_unsupported_mesh_rejected():
    with pytest.raises(ValueError):
        poisson.build_hierarchy(12, 8, 3)
