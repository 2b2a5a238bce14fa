"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Each test builds the same seeded input for both sides.  Tolerances:
  * float64 operators: the two sides differ only in summation order, so
    relative L2 differences stay near 1e-15 per application; the bar is 1e-12.
  * float64 V-cycles: as above, except that the coarsest solve is an explicit
    inverse on the GPU and a Cholesky substitution in the oracle, which agree
    to O(kappa(K_0) eps); the bar is max(1e-12, 20 kappa(K_0) eps).
  * float32 V-cycle (mixed path): compared with the oracle's float64 V-cycle
    built from the same bfloat16-rounded moduli.  float32 carries 2^-24 ~ 6e-8
    relative rounding per operation; residual cancellation in the smoother and
    seven levels of transfers amplify it by O(100), so the bar is 2e-5.
  * solves: relative compliance error <= 1e-9 and relative L2 displacement
    error <= 1e-8 against the direct solve at solver tolerance 1e-10;
    mixed solves reach a float64 true residual <= the requested 1e-8.
"""

import numpy as np
import pytest
import torch

from oracle import fem, multigrid, precision, solver
from synth import BOTTOM, LEFT, RIGHT, TOP, dirichlet_design, load_right_edge, load_top_edge

pytestmark = pytest.mark.gpu
EP = [1.0, 0.5, 0.25, 1e-9]
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def mto():
    import paper_2301_07457_gb300 as m
    return m


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def random_nodal(nx, ny, fixed, seed):
    v = np.random.default_rng(seed).standard_normal((ny + 1, nx + 1, 2))
    v[fem.fixed_node_mask(nx, ny, fixed)] = 0.0
    return v


MESHES = [
    (64, 64, 3, BOTTOM),        # the 64x64 square wall
    (64, 64, 2, BOTTOM),        # the same with three grids (down to 16 x 16)
    (200, 136, 3, BOTTOM),      # several strips and chunks, ragged in both directions
    (96, 40, 2, BOTTOM | LEFT),
    (48, 80, 4, BOTTOM | RIGHT | TOP),
]


@pytest.mark.parametrize("nelx,nely,nc,fixed", MESHES)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_level_operators(mto, nelx, nely, nc, fixed, prec):
    x = dirichlet_design(nelx, nely, 4, seed=nelx + nely)
    E = fem.simp_moduli(x, EP, 3.0)
    KE = fem.element_stiffness(0.3)
    mesh = mto.Mesh(nelx, nely, fixed_edges=fixed, n_coarsen=nc, precision=prec)
    mesh.set_design(to_dev(x), EP, 3.0)
    E_pre = precision.round_to_bf16(E) if prec == "mixed" else E
    lv = multigrid.build_hierarchy(nelx, nely, E_pre, KE, fixed, nc, "galerkin")
    lv64 = multigrid.build_hierarchy(nelx, nely, E, KE, fixed, nc, "galerkin")
    np.testing.assert_allclose(mesh.moduli().cpu().numpy(), E, rtol=1e-15)
    for l in range(nc + 1):
        nx, ny = nelx >> (nc - l), nely >> (nc - l)
        v = random_nodal(nx, ny, fixed, seed=l)
        y = mesh.apply_operator(l, to_dev(v), vcycle_operator=True).cpu().numpy()
        ref = np.zeros(v.size)
        ref[lv[l].free] = lv[l].K @ v.ravel()[lv[l].free]
        tol = 1e-12 if prec == "fp64" else 2e-6
        assert rel(y, ref) < tol, (l, rel(y, ref))
        assert np.all(y[fem.fixed_node_mask(nx, ny, fixed)] == 0.0)
    # The outer operator of the mixed path is float64 with float64 moduli.
    v = random_nodal(nelx, nely, fixed, seed=99)
    y = mesh.apply_operator(nc, to_dev(v), vcycle_operator=False).cpu().numpy()
    ref = np.zeros(v.size)
    ref[lv64[-1].free] = lv64[-1].K @ v.ravel()[lv64[-1].free]
    assert rel(y, ref) < 1e-13
    mesh.close()


@pytest.mark.parametrize("nelx,nely,nc,fixed", MESHES)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_vcycle(mto, nelx, nely, nc, fixed, prec):
    x = dirichlet_design(nelx, nely, 4, seed=3 * nelx + nely)
    E = fem.simp_moduli(x, EP, 3.0)
    mesh = mto.Mesh(nelx, nely, fixed_edges=fixed, n_coarsen=nc, precision=prec)
    mesh.set_design(to_dev(x), EP, 3.0)
    E_pre = precision.round_to_bf16(E) if prec == "mixed" else E
    lv = multigrid.build_hierarchy(nelx, nely, E_pre, fem.element_stiffness(0.3), fixed, nc)
    M = multigrid.vcycle_preconditioner(lv, 0.6, 2, 2)
    r = random_nodal(nelx, nely, fixed, seed=7)
    z = mesh.apply_preconditioner(to_dev(r)).cpu().numpy()
    ref = np.zeros(r.size)
    ref[lv[-1].free] = M(r.ravel()[lv[-1].free])
    # The coarsest solve is an explicit K_0^-1 on the GPU and a Cholesky
    # substitution in the oracle; the two agree to O(kappa(K_0) eps).
    kappa0 = np.linalg.cond(lv[0].K.toarray())
    bar64 = max(1e-12, 20 * kappa0 * np.finfo(float).eps)
    assert rel(z, ref) < (bar64 if prec == "fp64" else 2e-5), (rel(z, ref), kappa0)
    mesh.close()


def test_solve_64_square_wall(mto):
    nelx = nely = 64
    x = dirichlet_design(nelx, nely, 4, seed=0)
    f = load_top_edge(nelx, nely)
    ud = solver.solve_direct(nelx, nely, x, EP, 3.0, f)
    ref = solver.solve_pcgmg(nelx, nely, x, EP, 3.0, f, n_coarsen=3, tol=1e-10)
    C_ref, g_ref = solver.compliance_and_gradient(nelx, nely, x, EP, 3.0, f, ud)
    mesh = mto.Mesh(nelx, nely, n_coarsen=3, tol=1e-10, precision="fp64")
    mesh.set_design(to_dev(x), EP, 3.0)
    u, st = mesh.solve(to_dev(f))
    C, g = mesh.compliance_grad(to_dev(f), u)
    un = u.cpu().numpy()
    assert rel(un, ud) <= 1e-8
    assert abs(C.item() - C_ref) / C_ref <= 1e-9
    assert abs(st["iters"] - ref["iters"]) <= 1, (st["iters"], ref["iters"])
    assert st["converged"] == 1 and st["rel_res_true"] <= 2e-10
    np.testing.assert_allclose(g.cpu().numpy(), g_ref, rtol=1e-7, atol=1e-9 * np.abs(g_ref).max())
    mesh.close()


@pytest.mark.parametrize("kind", ["galerkin", "rediscretize"])
def test_solve_ragged_and_iteration_count(mto, kind):
    nelx, nely = 200, 136
    x = dirichlet_design(nelx, nely, 4, seed=4)
    f = load_top_edge(nelx, nely) + 0.3 * load_right_edge(nelx, nely)
    ud = solver.solve_direct(nelx, nely, x, EP, 3.0, f)
    ref = solver.solve_pcgmg(nelx, nely, x, EP, 3.0, f, n_coarsen=3, tol=1e-10, coarse_kind=kind)
    mesh = mto.Mesh(nelx, nely, n_coarsen=3, tol=1e-10, coarse_kind=kind)
    mesh.set_design(to_dev(x), EP, 3.0)
    u, st = mesh.solve(to_dev(f))
    assert rel(u.cpu().numpy(), ud) <= 1e-8
    assert abs(st["iters"] - ref["iters"]) <= 1, (st["iters"], ref["iters"])
    mesh.close()


def test_mixed_solve_reaches_fp64_residual(mto):
    nelx, nely = 256, 256
    x = dirichlet_design(nelx, nely, 4, seed=0)
    f = load_top_edge(nelx, nely)
    E = fem.simp_moduli(x, EP, 3.0)
    mesh = mto.Mesh(nelx, nely, n_coarsen=4, tol=1e-8, precision="mixed")
    mesh.set_design(to_dev(x), EP, 3.0)
    u, st = mesh.solve(to_dev(f))
    un = u.cpu().numpy()
    assert solver.true_relative_residual(nelx, nely, E, f, un) <= 1e-8
    assert st["rel_res_true"] <= 1e-8
    ud = solver.solve_direct(nelx, nely, x, EP, 3.0, f)
    assert rel(un, ud) < 1e-5
    mesh.close()


def test_multiple_rhs_and_warm_start(mto):
    nelx = nely = 64
    x = dirichlet_design(nelx, nely, 4, seed=5)
    F = np.stack([load_top_edge(nelx, nely), load_right_edge(nelx, nely)])
    mesh = mto.Mesh(nelx, nely, n_coarsen=3, tol=1e-10)
    mesh.set_design(to_dev(x), EP, 3.0)
    U, st = mesh.solve(to_dev(F))
    for k in range(2):
        ud = solver.solve_direct(nelx, nely, x, EP, 3.0, F[k])
        assert rel(U[k].cpu().numpy(), ud) <= 1e-8
    # Warm start from the converged solution: zero iterations.
    U2, st2 = mesh.solve(to_dev(F), u0=U)
    assert st2["iters"] == 0
    C, g = mesh.compliance_grad(to_dev(F), U)
    for k in range(2):
        assert abs(C[k].item() - float(np.dot(F[k].ravel(), U[k].cpu().numpy().ravel()))) < 1e-12 * abs(C[k].item())
    mesh.close()


@pytest.mark.parametrize("tol", [1e-8, 1e-10])
def test_mixed_pcg_matches_oracle_reading(mto, tol):
    # The mixed path's PCG against the oracle's reading of it: the outer CG in
    # float64 with flexible beta and residual replacement every 25 steps,
    # preconditioned by a V-cycle built from the bfloat16-rounded moduli (the
    # oracle's V-cycle runs in float64, the GPU's in float32, so the iteration
    # counts may differ by a step or two).  u is compared element by element
    # with the oracle's iterate and with the direct solve.
    nelx = nely = 256
    x = dirichlet_design(nelx, nely, 4, seed=0)
    f = load_top_edge(nelx, nely)
    E = fem.simp_moduli(x, EP, 3.0)
    ref = solver.solve_pcgmg(nelx, nely, x, EP, 3.0, f, n_coarsen=4, tol=tol,
                             vcycle_E=precision.round_to_bf16(E), flexible=True, rr_every=25)
    ud = solver.solve_direct(nelx, nely, x, EP, 3.0, f)
    mesh = mto.Mesh(nelx, nely, n_coarsen=4, tol=tol, precision="mixed", rr_every=25, flexible=True,
                    max_it=200)
    mesh.set_design(to_dev(x), EP, 3.0)
    u, st = mesh.solve(to_dev(f))
    un = u.cpu().numpy()
    assert st["converged"] == 1, st
    assert abs(st["iters"] - ref["iters"]) <= 2, (st["iters"], ref["iters"])
    assert rel(un, ref["u"]) <= 1e-6
    assert rel(un, ud) <= 100 * tol
    assert solver.true_relative_residual(nelx, nely, E, f, un) <= tol
    mesh.close()
