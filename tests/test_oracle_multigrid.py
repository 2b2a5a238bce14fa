"""Pins of the oracle's multigrid, Cholesky and PCG against mathematics.

Paper passages: Sec. 2.1 (Eq. 1, Alg. 1), Sec. 2.2 (Alg. 2), Sec. 2.3 (Alg. 3,
damped Jacobi).  None of these tests calls the CUDA library.
"""

import numpy as np
import pytest

from oracle import cholesky, fem, multigrid, pcg, solver
from synth import BOTTOM, LEFT, dirichlet_design, load_top_edge

EP = [1.0, 0.5, 0.25, 1e-9]


def design_E(nelx, nely, seed=0):
    return fem.simp_moduli(dirichlet_design(nelx, nely, 4, seed), EP, 3.0)


def test_cholesky_matches_lapack():
    rng = np.random.default_rng(0)
    for n in (1, 2, 5, 17, 60):
        A = rng.standard_normal((n, n))
        A = A @ A.T + n * np.eye(n)
        L = cholesky.cholesky(A)
        np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=1e-12, atol=1e-12)
        assert np.allclose(np.triu(L, 1), 0.0)
        b = rng.standard_normal(n)
        np.testing.assert_allclose(cholesky.cholesky_solve(L, b), np.linalg.solve(A, b),
                                   rtol=1e-10, atol=1e-12)
    with pytest.raises(np.linalg.LinAlgError):
        cholesky.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))


def test_cholesky_on_stiffness_matches_lapack():
    for n in (1, 2, 4, 8):
        E = design_E(n, n, seed=n)
        K = fem.assemble(n, n, E, fem.element_stiffness(0.3))
        free = fem.free_dofs(n, n, BOTTOM)
        A = K.toarray()[np.ix_(free, free)]
        np.testing.assert_allclose(cholesky.cholesky(A), np.linalg.cholesky(A),
                                   rtol=1e-9, atol=1e-12 * np.abs(A).max())


def test_prolongation_reproduces_bilinear_fields():
    ncx, ncy = 3, 2
    P = multigrid.prolongation(ncx, ncy)
    Jc, Ic = np.meshgrid(np.arange(ncy + 1), np.arange(ncx + 1), indexing="ij")
    Jf, If = np.meshgrid(np.arange(2 * ncy + 1) / 2, np.arange(2 * ncx + 1) / 2, indexing="ij")
    for fun in (lambda x, y: 1 + 0 * x, lambda x, y: x, lambda x, y: y,
                lambda x, y: 2 * x * y - 0.5 * x + 3):
        vc = np.zeros((ncy + 1, ncx + 1, 2))
        vc[..., 0] = fun(Ic, Jc)
        vc[..., 1] = -fun(Ic, Jc)
        vf = (P @ vc.ravel()).reshape(2 * ncy + 1, 2 * ncx + 1, 2)
        np.testing.assert_allclose(vf[..., 0], fun(If, Jf), atol=1e-14)
        np.testing.assert_allclose(vf[..., 1], -fun(If, Jf), atol=1e-14)
    # A quadratic is not reproduced (the interpolation is only bilinear).
    vc = np.zeros((ncy + 1, ncx + 1, 2)); vc[..., 0] = Ic**2
    vf = (P @ vc.ravel()).reshape(2 * ncy + 1, 2 * ncx + 1, 2)
    assert np.abs(vf[..., 0] - If**2).max() > 0.2
    # Columns of P sum to the 1-D weights (1 + 1/2 + 1/2)^2 in the interior.
    colsum = np.asarray(P.sum(axis=0)).ravel().reshape(ncy + 1, ncx + 1, 2)
    assert colsum[1, 1, 0] == pytest.approx(4.0)


def test_galerkin_equals_rediscretised_for_constant_modulus():
    # 2-D Q4 stiffness is invariant under scaling of the element size, so
    # P^T K_h P (Galerkin) must equal the stiffness assembled on the 2h mesh.
    for fixed in (BOTTOM, BOTTOM | LEFT):
        lv_g = multigrid.build_hierarchy(8, 4, np.full((4, 8), 1.7), fem.element_stiffness(0.3),
                                         fixed, 2, "galerkin")
        lv_r = multigrid.build_hierarchy(8, 4, np.full((4, 8), 1.7), fem.element_stiffness(0.3),
                                         fixed, 2, "rediscretize")
        for a, b in zip(lv_g, lv_r):
            assert abs(a.K - b.K).max() < 1e-13


def test_galerkin_coarse_operator_is_energy_of_coarse_field():
    # u_c^T K_c u_c = (P u_c)^T K (P u_c): the coarse operator measures the fine
    # energy of the interpolated field.  Checked against a fresh assembly.
    nelx, nely = 8, 8
    E = design_E(nelx, nely, 2)
    KE = fem.element_stiffness(0.3)
    lv = multigrid.build_hierarchy(nelx, nely, E, KE, BOTTOM, 1, "galerkin")
    Kf = fem.assemble(nelx, nely, E, KE)
    Pfull = multigrid.prolongation(4, 4)
    rng = np.random.default_rng(0)
    for _ in range(3):
        uc_full = rng.standard_normal(2 * 25)
        uc_full.reshape(5, 5, 2)[0] = 0.0  # clamped coarse row
        uf = Pfull @ uc_full
        uc = uc_full[lv[0].free]
        assert uc @ (lv[0].K @ uc) == pytest.approx(uf @ (Kf @ uf), rel=1e-12)


def test_two_grid_correction_is_K_orthogonal_projector():
    nelx, nely = 8, 8
    E = design_E(nelx, nely, 4)
    lv = multigrid.build_hierarchy(nelx, nely, E, fem.element_stiffness(0.3), BOTTOM, 1)
    K, P, Kc = lv[1].K.toarray(), lv[1].P.toarray(), lv[0].K.toarray()
    n = K.shape[0]
    T = np.eye(n) - P @ np.linalg.solve(Kc, P.T @ K)
    np.testing.assert_allclose(T @ T, T, atol=1e-9)
    np.testing.assert_allclose(K @ T, (K @ T).T, atol=1e-9 * np.abs(K).max())
    # Eq. 1 from U = 0 with F gives exactly the coarse-space Galerkin solution.
    F = np.random.default_rng(1).standard_normal(n)
    U = multigrid.two_level_correction(lv[1].K, lv[1].P, lv[0].K, np.zeros(n), F)
    np.testing.assert_allclose(P.T @ (K @ U), P.T @ F, atol=1e-10)


def test_two_grid_without_smoothing_equals_eq1():
    nelx, nely = 8, 8
    E = design_E(nelx, nely, 6)
    lv = multigrid.build_hierarchy(nelx, nely, E, fem.element_stiffness(0.3), BOTTOM, 1)
    rng = np.random.default_rng(2)
    U0 = rng.standard_normal(lv[1].n_free)
    F = rng.standard_normal(lv[1].n_free)
    mg = multigrid.mg_cycle(lv, 1, U0, F, 0.6, 0, 0)
    eq1 = multigrid.two_level_correction(lv[1].K, lv[1].P, lv[0].K, U0, F)
    np.testing.assert_allclose(mg, eq1, rtol=1e-10, atol=1e-12)


def test_damped_jacobi_error_propagation():
    nelx, nely = 4, 4
    E = design_E(nelx, nely, 7)
    lv = multigrid.build_hierarchy(nelx, nely, E, fem.element_stiffness(0.3), BOTTOM, 0)
    K = lv[0].K.toarray()
    D = np.diag(K)
    rng = np.random.default_rng(3)
    x0, b = rng.standard_normal(K.shape[0]), rng.standard_normal(K.shape[0])
    xs = np.linalg.solve(K, b)
    x2 = multigrid.damped_jacobi(lv[0].K, lv[0].diag, x0, b, 0.6, 2)
    G = np.eye(K.shape[0]) - 0.6 * K / D[:, None]
    np.testing.assert_allclose(x2 - xs, G @ G @ (x0 - xs), atol=1e-9)


def test_vcycle_is_symmetric_positive_definite():
    nelx, nely = 16, 16
    E = design_E(nelx, nely, 8)
    lv = multigrid.build_hierarchy(nelx, nely, E, fem.element_stiffness(0.3), BOTTOM, 2)
    M = multigrid.vcycle_preconditioner(lv)
    rng = np.random.default_rng(4)
    n = lv[-1].n_free
    for _ in range(3):
        a, b = rng.standard_normal(n), rng.standard_normal(n)
        assert a @ M(b) == pytest.approx(b @ M(a), rel=1e-11)
        assert a @ M(a) > 0
    # Linear in its argument.
    a, b = rng.standard_normal(n), rng.standard_normal(n)
    np.testing.assert_allclose(M(2 * a - b), 2 * M(a) - M(b), rtol=1e-10, atol=1e-12)


def test_vcycle_unsymmetric_smoothing_breaks_symmetry():
    # Symmetry needs nu1 = nu2 (Sec. 2.2): the check above would catch a
    # V-cycle that dropped its post-smoothing.
    nelx, nely = 16, 16
    E = design_E(nelx, nely, 8)
    lv = multigrid.build_hierarchy(nelx, nely, E, fem.element_stiffness(0.3), BOTTOM, 2)
    M = multigrid.vcycle_preconditioner(lv, nu1=2, nu2=0)
    rng = np.random.default_rng(4)
    n = lv[-1].n_free
    a, b = rng.standard_normal(n), rng.standard_normal(n)
    assert abs(a @ M(b) - b @ M(a)) > 1e-6 * abs(a @ M(b))


def _cycle_error_operator(lv, omega, nu1, nu2, gamma):
    """Error propagation of Alg. 1, built from matrices level by level:
    E_0 = 0 and E_l = S_l^nu2 (I - P_l (I - E_{l-1}^c) K_{l-1}^-1 P_l^T K_l) S_l^nu1,
    S_l = I - omega D_l^-1 K_l, with c = 1 on the finest level and gamma below
    it (gamma calls on level l-1, each continuing from the last iterate)."""
    E_prev = np.zeros((lv[0].n_free, lv[0].n_free))
    for l in range(1, len(lv)):
        K, P, Kc = lv[l].K.toarray(), lv[l].P.toarray(), lv[l - 1].K.toarray()
        n = K.shape[0]
        S = np.eye(n) - omega * K / np.diag(K)[:, None]
        c = 1 if l == len(lv) - 1 else gamma
        inner = np.eye(Kc.shape[0]) - np.linalg.matrix_power(E_prev, c)
        T = np.eye(n) - P @ inner @ np.linalg.solve(Kc, P.T @ K)
        E_prev = np.linalg.matrix_power(S, nu2) @ T @ np.linalg.matrix_power(S, nu1)
    return E_prev


@pytest.mark.parametrize("gamma", [1, 2, 3])
def test_gamma_cycle_matches_error_propagation(gamma):
    # Four grids (16^2 down to 2^2): the W-cycle visits the 4^2 grid twice
    # and the coarsest four times, each visit from the last coarse iterate.
    nelx, nely = 16, 16
    E = design_E(nelx, nely, 12)
    lv = multigrid.build_hierarchy(nelx, nely, E, fem.element_stiffness(0.3), BOTTOM, 3)
    rng = np.random.default_rng(13)
    n = lv[-1].n_free
    U0, F = rng.standard_normal(n), rng.standard_normal(n)
    Us = np.linalg.solve(lv[-1].K.toarray(), F)
    Em = _cycle_error_operator(lv, 0.6, 2, 1, gamma)
    U = multigrid.mg_cycle(lv, len(lv) - 1, U0, F, 0.6, 2, 1, gamma)
    np.testing.assert_allclose(U - Us, Em @ (U0 - Us), atol=1e-9 * np.abs(Us).max())


def test_w_cycle_equals_v_cycle_on_three_grids_only():
    # Alg. 1 calls the next grid once from the finest grid, and a repeated
    # exact coarsest solve returns the same iterate: with two or three grids
    # the W-cycle is the V-cycle; from four grids on it is not.
    nelx, nely = 16, 16
    E = design_E(nelx, nely, 14)
    KE = fem.element_stiffness(0.3)
    r = np.random.default_rng(15).standard_normal
    for nc in (1, 2):
        lv = multigrid.build_hierarchy(nelx, nely, E, KE, BOTTOM, nc)
        b = r(lv[-1].n_free)
        np.testing.assert_array_equal(multigrid.vcycle_preconditioner(lv, gamma=2)(b),
                                      multigrid.vcycle_preconditioner(lv)(b))
    lv = multigrid.build_hierarchy(nelx, nely, E, KE, BOTTOM, 3)
    b = r(lv[-1].n_free)
    zv = multigrid.vcycle_preconditioner(lv)(b)
    zw = multigrid.vcycle_preconditioner(lv, gamma=2)(b)
    assert np.linalg.norm(zw - zv) > 1e-3 * np.linalg.norm(zv)


def test_w_cycle_is_symmetric_positive_definite():
    nelx, nely = 16, 16
    E = design_E(nelx, nely, 16)
    lv = multigrid.build_hierarchy(nelx, nely, E, fem.element_stiffness(0.3), BOTTOM, 3)
    M = multigrid.vcycle_preconditioner(lv, gamma=2)
    rng = np.random.default_rng(17)
    n = lv[-1].n_free
    for _ in range(3):
        a, b = rng.standard_normal(n), rng.standard_normal(n)
        assert a @ M(b) == pytest.approx(b @ M(a), rel=1e-11)
        assert a @ M(a) > 0


def test_pcg_without_preconditioner_matches_textbook_cg():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((30, 30)); A = A @ A.T + 30 * np.eye(30)
    b = rng.standard_normal(30)
    x, it, conv, hist = pcg.pcg(lambda v: A @ v, b, lambda r: r.copy(), tol=1e-12)
    assert conv and it <= 30
    xs = np.linalg.solve(A, b)
    np.testing.assert_allclose(x, xs, rtol=1e-9, atol=1e-11 * np.abs(xs).max())
    # Exact preconditioner: one iteration.
    x1, it1, conv1, _ = pcg.pcg(lambda v: A @ v, b, lambda r: np.linalg.solve(A, r), tol=1e-12)
    assert conv1 and it1 == 1


@pytest.mark.parametrize("n_coarsen,kind", [(1, "galerkin"), (2, "galerkin"), (3, "galerkin"),
                                            (2, "rediscretize")])
def test_pcgmg_converges_to_direct_solution(n_coarsen, kind):
    nelx, nely = 16, 16
    x = dirichlet_design(nelx, nely, 4, seed=0)
    f = load_top_edge(nelx, nely)
    ud = solver.solve_direct(nelx, nely, x, EP, 3.0, f)
    res = solver.solve_pcgmg(nelx, nely, x, EP, 3.0, f, n_coarsen=n_coarsen, tol=1e-12,
                             coarse_kind=kind)
    assert res["converged"]
    err = np.linalg.norm(res["u"] - ud) / np.linalg.norm(ud)
    assert err < 1e-8
    assert np.all(res["u"][0] == 0.0)


def test_pcgmg_with_w_cycle_converges_to_direct_solution():
    nelx, nely = 32, 32
    x = dirichlet_design(nelx, nely, 4, seed=3)
    f = load_top_edge(nelx, nely)
    ud = solver.solve_direct(nelx, nely, x, EP, 3.0, f)
    rv = solver.solve_pcgmg(nelx, nely, x, EP, 3.0, f, n_coarsen=4, tol=1e-12)
    rw = solver.solve_pcgmg(nelx, nely, x, EP, 3.0, f, n_coarsen=4, tol=1e-12, gamma=2)
    assert rw["converged"]
    assert np.linalg.norm(rw["u"] - ud) / np.linalg.norm(ud) < 1e-8
    assert rw["iters"] != rv["iters"] or not np.array_equal(rw["history"], rv["history"])


def test_pcgmg_flexible_and_replacement_and_warm_start():
    nelx, nely = 32, 16
    x = dirichlet_design(nelx, nely, 4, seed=1)
    f = load_top_edge(nelx, nely)
    ud = solver.solve_direct(nelx, nely, x, EP, 3.0, f)
    a = solver.solve_pcgmg(nelx, nely, x, EP, 3.0, f, n_coarsen=3, tol=1e-10)
    b = solver.solve_pcgmg(nelx, nely, x, EP, 3.0, f, n_coarsen=3, tol=1e-10, flexible=True,
                           rr_every=5)
    assert abs(a["iters"] - b["iters"]) <= 1
    for r in (a, b):
        assert np.linalg.norm(r["u"] - ud) / np.linalg.norm(ud) < 1e-7
    # Warm start from the solution stops at once.
    c = solver.solve_pcgmg(nelx, nely, x, EP, 3.0, f, n_coarsen=3, tol=1e-8, u0=ud)
    assert c["iters"] == 0


def test_multigrid_iterations_nearly_mesh_independent():
    # Sec. 5.1 remark: pCGMG iteration counts do not grow with the mesh for
    # a homogeneous modulus.
    its = []
    for n in (16, 32, 64):
        x = np.zeros((4, n, n)); x[0] = 1.0
        r = solver.solve_pcgmg(n, n, x, EP, 3.0, load_top_edge(n, n), n_coarsen=int(np.log2(n)) - 2,
                               tol=1e-8)
        its.append(r["iters"])
    assert max(its) - min(its) <= 3, its


def test_unsupported_mesh_rejected():
    with pytest.raises(ValueError):
        multigrid.build_hierarchy(6, 4, np.ones((4, 6)), fem.element_stiffness(0.3), BOTTOM, 2)


def test_rediscretised_coarse_modulus_is_the_child_mean():
    # Sec. 2.1 rediscretisation with non-constant moduli.  (1) A field of
    # constant strain gives every fine element the same energy density, so its
    # Galerkin energy (P^T K P, built by the sparse product, not by assembly)
    # is the density times the sum of the fine moduli; the rediscretised
    # coarse element must carry the same energy, which holds for the
    # arithmetic mean of its four children and fails for a geometric or
    # harmonic mean or a child counted twice.  (2) A corner node of the coarse
    # mesh touches one coarse element, so its diagonal is that element's
    # modulus times the closed-form KE_00 = (3 - nu) / (6 (1 - nu^2)); this
    # catches a mean assigned to the wrong coarse element.
    nu = 0.3
    nelx, nely = 4, 4
    E = np.array([[1.0, 9.0, 0.5, 2.0],
                  [4.0, 0.25, 3.0, 7.0],
                  [0.1, 5.0, 6.0, 1.5],
                  [8.0, 2.5, 0.75, 11.0]])
    KE = fem.element_stiffness(nu)
    free_edges = 0
    red = multigrid.build_hierarchy(nelx, nely, E, KE, free_edges, 1, "rediscretize",
                                    factor_coarsest=False)
    gal = multigrid.build_hierarchy(nelx, nely, E, KE, free_edges, 1, "galerkin",
                                    factor_coarsest=False)
    J, I = np.meshgrid(np.arange(3) * 2.0, np.arange(3) * 2.0, indexing="ij")
    for ux, uy in ((I, 0 * I), (0 * I, J), (J, I), (0.3 * I - J, 2 * J + 0.5 * I)):
        v = np.stack([ux, uy], axis=-1).ravel()
        e_red = v @ (red[0].K @ v)
        e_gal = v @ (gal[0].K @ v)
        assert e_red == pytest.approx(e_gal, rel=1e-12)
        assert e_red > 0
    kdiag = (3 - nu) / (6 * (1 - nu * nu))
    diag = red[0].K.diagonal().reshape(3, 3, 2)
    means = {(0, 0): E[0:2, 0:2].mean(), (0, 2): E[0:2, 2:4].mean(),
             (2, 0): E[2:4, 0:2].mean(), (2, 2): E[2:4, 2:4].mean()}
    for (j, i), m in means.items():
        np.testing.assert_allclose(diag[j, i], [m * kdiag, m * kdiag], rtol=1e-13)
    # The bending energy of a single coarse element differs between the two
    # coarse operators (Galerkin resolves where the stiff children sit).
    v = np.zeros((3, 3, 2)); v[1, 1, 0] = 1.0
    assert abs(v.ravel() @ (red[0].K @ v.ravel()) - v.ravel() @ (gal[0].K @ v.ravel())) > 1e-3


def _spd(n, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return (Q * np.geomspace(1.0, cond, n)) @ Q.T


def test_flexible_beta_equals_fletcher_reeves_for_a_fixed_preconditioner():
    # With a fixed symmetric positive definite M, z_{i+1} . r_i = 0 in exact
    # arithmetic, so the flexible numerator z_{i+1} . (r_{i+1} - r_i) equals the
    # Fletcher-Reeves one and both runs take the same steps.
    n = 40
    A = _spd(n, 30)
    Minv = np.linalg.inv(_spd(n, 31, cond=20.0) + np.diag(np.diag(A)))
    b = np.random.default_rng(32).standard_normal(n)
    for k in range(1, 9):
        xf, *_ = pcg.pcg(lambda v: A @ v, b, lambda r: Minv @ r, tol=0.0, max_it=k, flexible=True)
        xr, *_ = pcg.pcg(lambda v: A @ v, b, lambda r: Minv @ r, tol=0.0, max_it=k, flexible=False)
        assert np.linalg.norm(xf - xr) <= 1e-10 * np.linalg.norm(xr), k


def test_flexible_beta_keeps_consecutive_directions_conjugate():
    # With a preconditioner that changes at every call (here a new random
    # positive diagonal each time), the flexible beta is the one that makes
    # p_{i+1} A-orthogonal to p_i: z.(r_new - r_old) = -alpha z.A p_i and
    # alpha = rho / p_i.A p_i give p_{i+1}.A p_i = 0.  A sign or index error
    # in the numerator breaks the identity; the Fletcher-Reeves form, which
    # assumes a fixed preconditioner, breaks it too (the teeth of this test).
    n = 60
    A = _spd(n, 33, cond=100.0)
    b = np.random.default_rng(34).standard_normal(n)

    def varying():
        rng = np.random.default_rng(35)
        return lambda r: rng.uniform(0.2, 5.0, r.size) * r

    def worst_cosine(trace):
        w = 0.0
        for (p0, q0, _), (p1, _, _) in zip(trace, trace[1:]):
            w = max(w, abs(p1 @ q0) / (np.linalg.norm(p1) * np.linalg.norm(q0)))
        return w

    tr_flex, tr_fr = [], []
    x, it, conv, _ = pcg.pcg(lambda v: A @ v, b, varying(), tol=1e-10, max_it=1000,
                             flexible=True, trace=tr_flex)
    _, _, conv_fr, _ = pcg.pcg(lambda v: A @ v, b, varying(), tol=1e-10, max_it=2 * it,
                               flexible=False, trace=tr_fr)
    assert conv and not conv_fr
    np.testing.assert_allclose(A @ x, b, atol=1e-8 * np.linalg.norm(b))
    assert worst_cosine(tr_flex) < 1e-12
    assert worst_cosine(tr_fr) > 1e-3
    # The first step uses p_0 = z_0 (no beta).
    assert tr_flex[0][2] == 0.0
    # Residual replacement every 3 steps keeps the identity on the steps
    # where r_new - r_old is the recursive update.
    tr_rr = []
    pcg.pcg(lambda v: A @ v, b, varying(), tol=0.0, max_it=12, flexible=True, rr_every=3,
            trace=tr_rr)
    for i in range(len(tr_rr) - 1):
        if (i + 1) % 3:
            p0, q0, _ = tr_rr[i]
            p1 = tr_rr[i + 1][0]
            assert abs(p1 @ q0) < 1e-12 * np.linalg.norm(p1) * np.linalg.norm(q0)
