"""Pins of the oracle's finite-element pieces against closed forms and invariants.

Paper passages: Eqs. 5, 7-9 (Sec. 3.1), Eq. 6 (compliance).  None of these
tests calls the CUDA library.
"""

import numpy as np
import pytest

from oracle import fem
from synth import BOTTOM, LEFT, RIGHT, TOP, dirichlet_design


def hadamard_energy(u, nu, E=1.0):
    """u^T KE u of a bilinear field on the unit square, from the continuum.

    With u_x = c0 + c1 xi + c2 eta + c3 xi eta and u_y = d0 + d1 xi + d2 eta +
    d3 xi eta on [-1,1]^2 (x = (xi+1)/2), the strains are eps_xx = 2(c1 + c3 eta),
    eps_yy = 2(d2 + d3 xi), gamma = 2(c2 + d1 + c3 xi + d3 eta).  Averaging
    eps^T D eps (Eq. 8) over the square (<xi^2> = 1/3, odd moments 0) gives
        4E/(1-nu^2) [c1^2 + d2^2 + 2 nu c1 d2 + (c3^2 + d3^2)/3
                     + (1-nu)/2 ((c2 + d1)^2 + (c3^2 + d3^2)/3)].
    Derived by hand from the energy, independently of Eq. 9's B matrix.
    """
    ux, uy = u[0::2], u[1::2]  # nodes BL, BR, TR, TL

    def coeffs(v):
        c1 = (-v[0] + v[1] + v[2] - v[3]) / 4
        c2 = (-v[0] - v[1] + v[2] + v[3]) / 4
        c3 = (v[0] - v[1] + v[2] - v[3]) / 4
        return c1, c2, c3

    c1, c2, c3 = coeffs(ux)
    d1, d2, d3 = coeffs(uy)
    return 4 * E / (1 - nu**2) * (
        c1**2 + d2**2 + 2 * nu * c1 * d2 + (c3**2 + d3**2) / 3
        + (1 - nu) / 2 * ((c2 + d1) ** 2 + (c3**2 + d3**2) / 3))


@pytest.mark.parametrize("nu", [0.0, 0.25, 0.3, 0.45])
def test_ke_matches_continuum_energy(nu):
    KE = fem.element_stiffness(nu)
    rng = np.random.default_rng(1)
    # A symmetric matrix is fixed by its quadratic form: check on a basis of
    # sums e_a + e_b, which determines every entry.
    for a in range(8):
        for b in range(8):
            u = np.zeros(8)
            u[a] += 1.0
            u[b] += 1.0
            assert u @ KE @ u == pytest.approx(hadamard_energy(u, nu), rel=1e-13, abs=1e-14)
    for _ in range(20):
        u = rng.standard_normal(8)
        assert u @ KE @ u == pytest.approx(hadamard_energy(u, nu), rel=1e-12)


def test_ke_exact_symbolic():
    sympy = pytest.importorskip("sympy")
    x, y, nu = sympy.symbols("x y nu")
    # Bilinear shape functions on [0,1]^2, counter-clockwise from the bottom-left.
    N = [(1 - x) * (1 - y), x * (1 - y), x * y, (1 - x) * y]
    B = sympy.zeros(3, 8)
    for a, Na in enumerate(N):
        B[0, 2 * a] = sympy.diff(Na, x)
        B[1, 2 * a + 1] = sympy.diff(Na, y)
        B[2, 2 * a] = sympy.diff(Na, y)
        B[2, 2 * a + 1] = sympy.diff(Na, x)
    D = 1 / (1 - nu**2) * sympy.Matrix([[1, nu, 0], [nu, 1, 0], [0, 0, (1 - nu) / 2]])
    K = (B.T * D * B).applyfunc(lambda t: sympy.integrate(t, (x, 0, 1), (y, 0, 1)))
    for nv in (0.3, 0.2):
        exact = np.array(K.subs(nu, nv).evalf(), dtype=np.float64)
        np.testing.assert_allclose(fem.element_stiffness(nv), exact, rtol=1e-13, atol=1e-15)


def test_ke_spectrum_closed_form():
    nu = 0.3
    ev = np.sort(np.linalg.eigvalsh(fem.element_stiffness(nu)))
    expected = np.sort([0, 0, 0,
                        (3 - nu) / (6 * (1 - nu**2)), (3 - nu) / (6 * (1 - nu**2)),
                        1 / (1 + nu), 1 / (1 + nu), 1 / (1 - nu)])
    np.testing.assert_allclose(ev, expected, atol=1e-13)


def test_plane_stress_matrix():
    D = fem.plane_stress_matrix(2.0, 0.3)
    # Uniaxial stress: strain (1, -nu, 0) gives stress (E, 0, 0).
    np.testing.assert_allclose(D @ np.array([1.0, -0.3, 0.0]), [2.0, 0.0, 0.0], atol=1e-14)
    # Pure shear: G = E / (2(1+nu)).
    assert D[2, 2] == pytest.approx(2.0 / (2 * 1.3))


def test_simp_moduli():
    x = np.array([[[0.5]], [[0.25]], [[0.25]]])
    E = fem.simp_moduli(x, [1.0, 0.5, 1e-9], 3.0)
    assert E[0, 0] == pytest.approx(0.125 + 0.5 * 0.015625 + 1e-9 * 0.015625, rel=1e-15)
    x2 = dirichlet_design(5, 3, 4, seed=0)
    E2 = fem.simp_moduli(x2, [1.0, 0.5, 0.25, 1e-9], 3.0)
    brute = sum(Ei * x2[i] ** 3 for i, Ei in enumerate([1.0, 0.5, 0.25, 1e-9]))
    np.testing.assert_allclose(E2, brute, rtol=1e-15)


def test_element_numbering():
    nodes = fem.element_nodes(3, 2)
    # Element (i=2, j=1) -> e = 1*3 + 2 = 5; node (i, j) index j*4 + i.
    assert list(nodes[5]) == [1 * 4 + 2, 1 * 4 + 3, 2 * 4 + 3, 2 * 4 + 2]
    dofs = fem.element_dofs(3, 2)
    assert list(dofs[0]) == [0, 1, 2, 3, 10, 11, 8, 9]


def rigid_modes(nelx, nely):
    j, i = np.meshgrid(np.arange(nely + 1), np.arange(nelx + 1), indexing="ij")
    X, Y = i.ravel().astype(float), j.ravel().astype(float)
    tx = np.zeros(2 * X.size); tx[0::2] = 1
    ty = np.zeros(2 * X.size); ty[1::2] = 1
    rot = np.zeros(2 * X.size); rot[0::2] = -Y; rot[1::2] = X
    return tx, ty, rot


def test_global_K_symmetry_and_rigid_null_space():
    nelx, nely = 7, 5
    x = dirichlet_design(nelx, nely, 4, seed=3)
    E = fem.simp_moduli(x, [1.0, 0.5, 0.25, 1e-9], 3.0)
    K = fem.assemble(nelx, nely, E, fem.element_stiffness(0.3))
    assert abs(K - K.T).max() < 1e-15
    for m in rigid_modes(nelx, nely):
        assert np.abs(K @ m).max() < 1e-13 * max(1.0, np.abs(m).max())
    # Exactly three zero eigenvalues (the rigid modes), the rest positive.
    ev = np.linalg.eigvalsh(K.toarray())
    assert np.sum(np.abs(ev) < 1e-10) == 3
    assert ev.min() > -1e-12


def test_patch_test_linear_field():
    nelx, nely = 6, 4
    K = fem.assemble(nelx, nely, np.full((nely, nelx), 2.5), fem.element_stiffness(0.3))
    j, i = np.meshgrid(np.arange(nely + 1), np.arange(nelx + 1), indexing="ij")
    u = np.zeros((nely + 1, nelx + 1, 2))
    u[..., 0] = 0.3 + 0.7 * i - 0.2 * j
    u[..., 1] = -0.1 + 0.4 * i + 0.9 * j
    r = (K @ u.ravel()).reshape(nely + 1, nelx + 1, 2)
    # Constant stress: internal forces cancel at every interior node.
    assert np.abs(r[1:-1, 1:-1]).max() < 1e-13


def test_element_by_element_product_matches_assembled():
    nelx, nely = 9, 6
    x = dirichlet_design(nelx, nely, 4, seed=5)
    E = fem.simp_moduli(x, [1.0, 0.5, 0.25, 1e-9], 3.0)
    KE = fem.element_stiffness(0.3)
    v = np.random.default_rng(0).standard_normal(2 * (nelx + 1) * (nely + 1))
    np.testing.assert_allclose(fem.apply_K(nelx, nely, E, KE, v),
                               fem.assemble(nelx, nely, E, KE) @ v, rtol=1e-13, atol=1e-14)


def test_fixed_edges():
    m = fem.fixed_node_mask(3, 2, BOTTOM | RIGHT)
    assert m[0].all() and m[:, 3].all() and m.sum() == 4 + 3 - 1
    free = fem.free_dofs(3, 2, BOTTOM)
    assert free[0] == 8 and free.size == 2 * 4 * 2
    assert fem.fixed_node_mask(2, 2, LEFT | TOP)[:, 0].all()


def test_direct_solve_dense_and_mirror_symmetry():
    nelx, nely = 8, 6
    E = np.ones((nely, nelx))
    KE = fem.element_stiffness(0.3)
    K = fem.assemble(nelx, nely, E, KE)
    free = fem.free_dofs(nelx, nely, BOTTOM)
    f = np.zeros((nely + 1, nelx + 1, 2)); f[nely, :, 1] = -1.0
    u = fem.direct_solve(K, f, free)
    ud = np.zeros_like(u)
    ud[free] = np.linalg.solve(K.toarray()[np.ix_(free, free)], f.ravel()[free])
    np.testing.assert_allclose(u, ud, rtol=1e-11, atol=1e-13)
    U = u.reshape(nely + 1, nelx + 1, 2)
    # Uniform E, symmetric load: u_x odd and u_y even about x = nelx/2.
    np.testing.assert_allclose(U[..., 0], -U[:, ::-1, 0], atol=1e-12)
    np.testing.assert_allclose(U[..., 1], U[:, ::-1, 1], atol=1e-12)
    # Loads push down: every free top node moves down.
    assert (U[nely, :, 1] < 0).all()
    # Scaling: u(cE) = u(E) / c.
    u3 = fem.direct_solve(fem.assemble(nelx, nely, 3.0 * E, KE), f, free)
    np.testing.assert_allclose(u3, u / 3.0, rtol=1e-12, atol=1e-13 * np.abs(u).max())
