"""V-cycle and solves with other smoothing counts and damping (Alg. 1 with
theta_1 pre- and theta_2 post-smoothing sweeps of damped Jacobi), and the
W-cycle (gamma = 2, 3 below the finest grid), through the C ABI, against the
oracle.

The default (two and two, omega = 0.6) runs fused passes on the float32
levels and a fused first sweep on the finest level; other counts take the
separate-kernel paths (the first sweep from zero as a kernel of its own, the
prolongation sweep carrying the dot products, extra plain sweeps), and the
repeated coarse calls of a W-cycle start their smoothing from the last
iterate.  Bars as in
test_gpu_parity.py: float64 V-cycle max(1e-12, 20 kappa(K_0) eps), float32
V-cycle 2e-5 against the oracle's float64 V-cycle on the same bf16-rounded
moduli; solves reach the requested float64 true residual.
"""

import numpy as np
import pytest
import torch

from oracle import fem, multigrid, precision, solver
from synth import BOTTOM, dirichlet_design, load_top_edge

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


@pytest.mark.parametrize("nu1,nu2,omega", [(1, 1, 0.6), (1, 2, 0.6), (2, 1, 0.6), (3, 3, 0.6),
                                           (2, 2, 0.8), (3, 1, 0.5)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_vcycle_smoothing_counts(mto, prec, nu1, nu2, omega):
    nelx, nely, nc = 200, 136, 3
    x = dirichlet_design(nelx, nely, 4, seed=21)
    E = fem.simp_moduli(x, EP, 3.0)
    mesh = mto.Mesh(nelx, nely, n_coarsen=nc, precision=prec, nu1=nu1, nu2=nu2, omega=omega)
    mesh.set_design(to_dev(x), EP, 3.0)
    E_pre = precision.round_to_bf16(E) if prec == "mixed" else E
    lv = multigrid.build_hierarchy(nelx, nely, E_pre, fem.element_stiffness(0.3), BOTTOM, nc)
    M = multigrid.vcycle_preconditioner(lv, omega, nu1, nu2)
    r = np.random.default_rng(5).standard_normal((nely + 1, nelx + 1, 2))
    r[fem.fixed_node_mask(nelx, nely, BOTTOM)] = 0.0
    z = mesh.apply_preconditioner(to_dev(r)).cpu().numpy()
    ref = np.zeros(r.size)
    ref[lv[-1].free] = M(r.ravel()[lv[-1].free])
    kappa0 = np.linalg.cond(lv[0].K.toarray())
    bar64 = max(1e-12, 20 * kappa0 * np.finfo(float).eps)
    assert rel(z, ref) < (bar64 if prec == "fp64" else 2e-5), (rel(z, ref), kappa0)
    mesh.close()


@pytest.mark.parametrize("nu1,nu2", [(1, 1), (3, 3), (2, 1)])
def test_mixed_solve_smoothing_counts(mto, nu1, nu2):
    nelx = nely = 128
    x = dirichlet_design(nelx, nely, 4, seed=8)
    f = load_top_edge(nelx, nely)
    E = fem.simp_moduli(x, EP, 3.0)
    mesh = mto.Mesh(nelx, nely, n_coarsen=3, tol=1e-8, precision="mixed", nu1=nu1, nu2=nu2)
    mesh.set_design(to_dev(x), EP, 3.0)
    u, st = mesh.solve(to_dev(f))
    assert st["status"] == "MTO_OK", st
    assert solver.true_relative_residual(nelx, nely, E, f, u.cpu().numpy()) <= 1e-8
    mesh.close()


@pytest.mark.parametrize("gamma", [2, 3])
@pytest.mark.parametrize("nu1,nu2", [(2, 2), (1, 2), (3, 1)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_w_cycle(mto, prec, nu1, nu2, gamma):
    # Five grids (192 x 128 down to 12 x 8): the coarse grids are called
    # 1, gamma and gamma^2 times per cycle.
    nelx, nely, nc = 192, 128, 4
    x = dirichlet_design(nelx, nely, 4, seed=22)
    E = fem.simp_moduli(x, EP, 3.0)
    mesh = mto.Mesh(nelx, nely, n_coarsen=nc, precision=prec, nu1=nu1, nu2=nu2, gamma=gamma)
    mesh.set_design(to_dev(x), EP, 3.0)
    E_pre = precision.round_to_bf16(E) if prec == "mixed" else E
    lv = multigrid.build_hierarchy(nelx, nely, E_pre, fem.element_stiffness(0.3), BOTTOM, nc)
    r = np.random.default_rng(6).standard_normal((nely + 1, nelx + 1, 2))
    r[fem.fixed_node_mask(nelx, nely, BOTTOM)] = 0.0
    z = mesh.apply_preconditioner(to_dev(r)).cpu().numpy()
    ref = np.zeros(r.size)
    ref[lv[-1].free] = multigrid.vcycle_preconditioner(lv, 0.6, nu1, nu2, gamma)(r.ravel()[lv[-1].free])
    vref = np.zeros(r.size)
    vref[lv[-1].free] = multigrid.vcycle_preconditioner(lv, 0.6, nu1, nu2)(r.ravel()[lv[-1].free])
    assert rel(ref, vref) > 1e-3  # the W-cycle is not the V-cycle here
    # Each coarsest solve (explicit inverse against Cholesky) contributes up
    # to ~kappa(K_0) eps, and the cycle carries each contribution to the
    # output without amplifying it: the V-cycle bar times the gamma^(nc-2)
    # coarsest solves of one W-cycle.
    kappa0 = np.linalg.cond(lv[0].K.toarray())
    bar64 = max(1e-12, 20 * kappa0 * np.finfo(float).eps * gamma ** (nc - 2))
    assert rel(z, ref) < (bar64 if prec == "fp64" else 2e-5), (rel(z, ref), kappa0)
    mesh.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_w_cycle_solve(mto, prec):
    nelx = nely = 128
    x = dirichlet_design(nelx, nely, 4, seed=9)
    f = load_top_edge(nelx, nely)
    E = fem.simp_moduli(x, EP, 3.0)
    mesh = mto.Mesh(nelx, nely, n_coarsen=4, tol=1e-8, precision=prec, gamma=2)
    mesh.set_design(to_dev(x), EP, 3.0)
    u, st = mesh.solve(to_dev(f))
    assert st["status"] == "MTO_OK", st
    assert solver.true_relative_residual(nelx, nely, E, f, u.cpu().numpy()) <= 1e-8
    if prec == "fp64":
        ref = solver.solve_pcgmg(nelx, nely, x, EP, 3.0, f, n_coarsen=4, tol=1e-8, gamma=2)
        assert abs(st["iters"] - ref["iters"]) <= 1, (st["iters"], ref["iters"])
    mesh.close()
