"""Edge cases of the C ABI on the GPU: degenerate meshes, constraints,
statuses.  Every case is checked against the oracle or against the status the
header promises."""

import numpy as np
import pytest
import torch

from oracle import fem, multigrid, solver
from synth import BOTTOM, LEFT, RIGHT, TOP, dirichlet_design, load_right_edge, load_top_edge

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
EP = [1.0, 0.5, 0.25, 1e-9]


@pytest.fixture(scope="module")
def mto():
    import paper_2301_07457_gb300 as m
    return m


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.mark.parametrize("nelx,nely,nc", [(2, 2, 1), (4, 2, 1), (8, 2, 1), (2, 8, 1), (6, 10, 1)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_tiny_meshes(mto, nelx, nely, nc, prec):
    x = dirichlet_design(nelx, nely, 4, seed=nelx * 10 + nely)
    f = load_top_edge(nelx, nely) + load_right_edge(nelx, nely)
    m = mto.Mesh(nelx, nely, n_coarsen=nc, precision=prec, tol=1e-10 if prec == "fp64" else 1e-8)
    m.set_design(to_dev(x), EP, 3.0)
    u, st = m.solve(to_dev(f))
    ud = solver.solve_direct(nelx, nely, x, EP, 3.0, f)
    assert rel(u.cpu().numpy(), ud) < (1e-8 if prec == "fp64" else 1e-5)
    m.close()


@pytest.mark.parametrize("fixed", [BOTTOM, LEFT, RIGHT, TOP, BOTTOM | TOP, LEFT | RIGHT,
                                   BOTTOM | LEFT | RIGHT | TOP])
def test_every_clamped_edge_pattern(mto, fixed):
    nelx, nely = 40, 24
    x = dirichlet_design(nelx, nely, 4, seed=fixed)
    f = np.random.default_rng(fixed).standard_normal((nely + 1, nelx + 1, 2))
    m = mto.Mesh(nelx, nely, fixed_edges=fixed, n_coarsen=2, tol=1e-10)
    m.set_design(to_dev(x), EP, 3.0)
    u, st = m.solve(to_dev(f))
    ud = solver.solve_direct(nelx, nely, x, EP, 3.0, f, fixed_edges=fixed)
    assert rel(u.cpu().numpy(), ud) < 1e-8
    un = u.cpu().numpy()
    assert np.all(un[fem.fixed_node_mask(nelx, nely, fixed)] == 0.0)
    m.close()


def test_material_law_variants(mto):
    nelx, nely = 32, 32
    for n_phase, Ep, penal, nu in [(1, [1.0], 3.0, 0.3), (4, EP, 2.5, 0.3), (4, EP, 3.0, 0.25),
                                   (2, [2.0, 0.1], 1.0, 0.45)]:
        x = dirichlet_design(nelx, nely, n_phase, seed=n_phase)
        f = load_top_edge(nelx, nely)
        m = mto.Mesh(nelx, nely, nu=nu, n_coarsen=2, tol=1e-10)
        m.set_design(to_dev(x), Ep, penal)
        u, _ = m.solve(to_dev(f))
        C, g = m.compliance_grad(to_dev(f), u)
        ud = solver.solve_direct(nelx, nely, x, Ep, penal, f, nu=nu)
        C_ref, g_ref = solver.compliance_and_gradient(nelx, nely, x, Ep, penal, f, ud, nu=nu)
        assert rel(u.cpu().numpy(), ud) < 1e-8
        assert abs(C.item() - C_ref) / C_ref < 1e-9
        assert np.abs(g.cpu().numpy() - g_ref).max() <= 1e-7 * np.abs(g_ref).max()
        m.close()


def test_statuses(mto):
    from paper_2301_07457_gb300 import MtoError, _lib
    nelx = nely = 32
    x = to_dev(dirichlet_design(nelx, nely, 4, seed=1))
    f = to_dev(load_top_edge(nelx, nely))
    m = mto.Mesh(nelx, nely, n_coarsen=2, tol=1e-12, max_it=3)
    with pytest.raises(MtoError) as e:
        m.solve(f)
    assert e.value.code == _lib.ERR_STATE  # solve before set_design
    m.set_design(x, EP, 3.0)
    u, st = m.solve(f, raise_on_failure=False)
    assert st["status"] == "MTO_ERR_NOT_CONVERGED" and st["iters"] == 3
    assert torch.isfinite(u).all() and u.abs().max() > 0
    # Zero load: converged at once with u = 0.
    u0, st0 = m.solve(torch.zeros_like(f))
    assert st0["iters"] == 0 and st0["converged"] == 1 and u0.abs().max().item() == 0.0
    # A NaN in the design cannot be factorised: breakdown, not a fault.
    xb = x.clone()
    xb[0, 5, 5] = float("nan")
    with pytest.raises(MtoError) as e2:
        m.set_design(xb, EP, 3.0)
    assert e2.value.code == _lib.ERR_BREAKDOWN
    # The context stays usable.
    m.set_design(x, EP, 3.0)
    u2, st2 = m.solve(f, raise_on_failure=False)
    assert st2["iters"] == 3
    m.close()


def test_mesh_limits(mto):
    from paper_2301_07457_gb300 import MtoError, _lib
    with pytest.raises(MtoError) as e:
        mto.Mesh(256, 256, n_coarsen=1)  # coarsest 128 x 128: 33,024 free DOFs > 16,896
    assert e.value.code == _lib.ERR_UNSUPPORTED_MESH
    with pytest.raises(MtoError) as e:
        mto.Mesh(320, 4, n_coarsen=1)  # coarsest 160 x 2: 644 free DOFs, half-bandwidth 325 > 320
    assert e.value.code == _lib.ERR_UNSUPPORTED_MESH
    with pytest.raises(MtoError) as e:
        mto.Mesh(100, 64, n_coarsen=3)
    assert e.value.code == _lib.ERR_UNSUPPORTED_MESH
    with pytest.raises(MtoError) as e:  # 2^31 elements: above the 2^30 cap, rejected before allocating
        mto.Mesh(65536, 32768, n_coarsen=11)
    assert e.value.code == _lib.ERR_UNSUPPORTED_MESH
    m = mto.Mesh(64, 64, n_coarsen=1)  # coarsest 32 x 32: 2112 free DOFs, band Cholesky in global memory
    x = dirichlet_design(64, 64, 4, seed=9)
    f = load_top_edge(64, 64)
    m.set_design(to_dev(x), EP, 3.0)
    u, st = m.solve(to_dev(f))
    assert rel(u.cpu().numpy(), solver.solve_direct(64, 64, x, EP, 3.0, f)) < 1e-7
    assert m.info()["coarsest_free_dofs"] == 2112
    m.close()


def test_mixed_rediscretised_and_partial_warm_start(mto):
    nelx, nely = 128, 128
    x = dirichlet_design(nelx, nely, 4, seed=12)
    f = load_top_edge(nelx, nely)
    E = fem.simp_moduli(x, EP, 3.0)
    m = mto.Mesh(nelx, nely, n_coarsen=3, precision="mixed", coarse_kind="rediscretize", tol=1e-8)
    m.set_design(to_dev(x), EP, 3.0)
    u, st = m.solve(to_dev(f))
    assert solver.true_relative_residual(nelx, nely, E, f, u.cpu().numpy()) <= 1e-8
    u_half, st_half = m.solve(to_dev(f), u0=0.5 * u)
    assert st_half["iters"] <= st["iters"]
    assert solver.true_relative_residual(nelx, nely, E, f, u_half.cpu().numpy()) <= 1e-8
    m.close()


@pytest.mark.parametrize("nelx,nely,n0", [(64, 128, 4224), (128, 128, 8320), (128, 256, 16640)])
def test_large_coarsest_system(mto, nelx, nely, n0):
    # One coarsening (the paper's two-level method) on its larger meshes: a
    # dense coarsest system of up to 16,640 free DOFs (explicit inverse by
    # columns for half-bandwidths of 128 and more, the GEMV's right-hand side
    # in opt-in shared memory).  The two-grid cycle is composed here from the
    # oracle's operators with a sparse direct coarse solve.
    import scipy.sparse.linalg as sla
    x = dirichlet_design(nelx, nely, 4, seed=nelx + nely)
    E = fem.simp_moduli(x, EP, 3.0)
    m = mto.Mesh(nelx, nely, n_coarsen=1, tol=1e-10)
    m.set_design(to_dev(x), EP, 3.0)
    assert m.info()["coarsest_free_dofs"] == n0
    lv = multigrid.build_hierarchy(nelx, nely, E, fem.element_stiffness(0.3), BOTTOM, 1,
                                   factor_coarsest=False)
    K1, K0, P, free = lv[1].K, lv[0].K.tocsc(), lv[1].P, lv[1].free
    assert K0.shape[0] == n0
    r = np.random.default_rng(n0).standard_normal((nely + 1, nelx + 1, 2))
    r[fem.fixed_node_mask(nelx, nely, BOTTOM)] = 0.0
    rf = r.ravel()[free]
    U = multigrid.damped_jacobi(K1, lv[1].diag, np.zeros_like(rf), rf, 0.6, 2)
    U = U + P @ sla.spsolve(K0, P.T @ (rf - K1 @ U))
    U = multigrid.damped_jacobi(K1, lv[1].diag, U, rf, 0.6, 2)
    ref = np.zeros(r.size)
    ref[free] = U
    z = m.apply_preconditioner(to_dev(r)).cpu().numpy()
    lmax = sla.eigsh(K0, 1, which="LA", return_eigenvectors=False)[0]
    lmin = sla.eigsh(K0, 1, sigma=0.0, which="LM", return_eigenvectors=False)[0]
    bar = max(1e-12, 20 * (lmax / lmin) * np.finfo(float).eps)
    assert rel(z, ref) < bar, (rel(z, ref), lmax / lmin)
    f = load_top_edge(nelx, nely)
    u, st = m.solve(to_dev(f))
    assert rel(u.cpu().numpy(), solver.solve_direct(nelx, nely, x, EP, 3.0, f)) < 1e-7
    m.close()
    mm = mto.Mesh(nelx, nely, n_coarsen=1, tol=1e-8, precision="mixed")
    mm.set_design(to_dev(x), EP, 3.0)
    u, st = mm.solve(to_dev(f))
    assert solver.true_relative_residual(nelx, nely, E, f, u.cpu().numpy()) <= 1e-8
    mm.close()


def test_two_live_contexts_with_large_coarsest_systems(mto):
    # The opt-in shared memory of the coarsest factorisation and GEMV kernels
    # is a per-process attribute of each kernel.  Creating a context with a
    # smaller coarsest system (8,320 DOFs, 66.5 KB) after one with a larger
    # system (16,640 DOFs, 133 KB) must not lower the limit the larger one
    # launches with: its set_design and solve still work.
    nelx, nely = 128, 256
    x = dirichlet_design(nelx, nely, 4, seed=77)
    f = load_top_edge(nelx, nely)
    big = mto.Mesh(nelx, nely, n_coarsen=1, tol=1e-10)
    small = mto.Mesh(128, 128, n_coarsen=1, tol=1e-10)
    assert big.info()["coarsest_free_dofs"] == 16640
    assert small.info()["coarsest_free_dofs"] == 8320
    big.set_design(to_dev(x), EP, 3.0)
    u, st = big.solve(to_dev(f))
    assert st["converged"] == 1
    assert rel(u.cpu().numpy(), solver.solve_direct(nelx, nely, x, EP, 3.0, f)) < 1e-7
    xs = dirichlet_design(128, 128, 4, seed=78)
    small.set_design(to_dev(xs), EP, 3.0)
    us, sts = small.solve(to_dev(load_top_edge(128, 128)))
    assert sts["converged"] == 1
    small.close()
    big.close()
