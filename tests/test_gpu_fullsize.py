"""Parity at the full size of the mixed-vs-float64 workload: the 2048 x 2048
square wall (8,396,802 DOFs, three solids + void, seeded Dirichlet fractions),
seven coarsenings to 16 x 16, in the launch configuration the bench times
(tuned launch shapes).

Paper passages: Alg. 2 preconditioned by Alg. 1 (the solve), Eq. 6 (the
compliance), Sec. 4 (the sensitivities).  The oracle's pCGMG runs once at this
size (float64, Fletcher-Reeves PCG, float64 V-cycle, Cholesky coarsest solve:
about two minutes and 13 GB of host memory) at tolerance 1e-10.  Bars:
  * float64 GPU path at 1e-10: relative L2 displacement error <= 1e-8 and
    relative compliance error <= 1e-9 against the oracle's solution, its PCG
    iteration count within one of the oracle's;
  * mixed path (float32 V-cycle, bf16 moduli, float64 outer CG) at 1e-10: the
    same displacement bar against the oracle and against the float64 GPU path;
  * both: the float64 true residual ||f - K u|| / ||f||, recomputed by the
    oracle element by element from the returned u, at most 1.1 times the
    tolerance (the stopping rule tests the recursive residual, which drifts
    from the true one by a few percent) and within 5% of the residual the
    GPU reports;
    the energy identity |f.u - u^T K u| <= ||u|| ||f - K u|| (Cauchy-Schwarz)
    with u^T K u from the oracle's element energies;
  * the W-cycle (mixed, gamma = 2) and the rediscretised coarse operators
    (float64): the same residual, energy and sensitivity checks, and u within
    1e-8 of the oracle's solution;
  * sensitivities: 4,096 seeded (phase, element) picks recomputed one by one
    by the oracle from the returned u, relative error <= 1e-12 (same u, same
    formula: only the order of roundings differs).
"""

import numpy as np
import pytest
import torch

from oracle import fem, sensitivity, solver
from synth import dirichlet_design, load_top_edge, uniform01

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
EP = [1.0, 0.5, 0.25, 1e-9]
N, NC, TOL = 2048, 7, 1e-10


@pytest.fixture(scope="module")
def mto():
    import paper_2301_07457_gb300 as m
    return m


@pytest.fixture(scope="module")
def problem():
    x = dirichlet_design(N, N, 4, seed=0)
    f = load_top_edge(N, N)
    E = fem.simp_moduli(x, EP, 3.0)
    return x, f, E


@pytest.fixture(scope="module")
def oracle_solution(problem):
    x, f, _ = problem
    r = solver.solve_pcgmg(N, N, x, EP, 3.0, f, n_coarsen=NC, tol=TOL)
    out = {"u": r["u"], "iters": r["iters"], "converged": r["converged"]}
    del r  # the hierarchy holds several GB
    return out


@pytest.fixture(scope="module")
def gpu_solutions(mto, problem):
    x, f, _ = problem
    xt = torch.from_numpy(x).to(DEV)
    ft = torch.from_numpy(f).to(DEV)
    out = {}
    variants = {"fp64": dict(precision="fp64"), "mixed": dict(precision="mixed"),
                "mixed_w": dict(precision="mixed", gamma=2),
                "fp64_redisc": dict(precision="fp64", coarse_kind="rediscretize")}
    for name, kw in variants.items():
        mesh = mto.Mesh(N, N, n_coarsen=NC, tol=TOL, max_it=1000, rr_every=25,
                        flexible=kw["precision"] == "mixed", **kw)
        mesh.set_design(xt, EP, 3.0)
        mesh.autotune()
        u, st = mesh.solve(ft)
        C, g = mesh.compliance_grad(ft, u)
        out[name] = {"u": u.cpu().numpy(), "st": st, "C": C.item(), "g": g.cpu().numpy()}
        mesh.close()
        del u, g
    torch.cuda.empty_cache()
    return out


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed_w", "fp64_redisc"])
def test_fullsize_residual_energy_and_sensitivities(problem, gpu_solutions, prec):
    x, f, E = problem
    sol = gpu_solutions[prec]
    u = sol["u"]
    assert sol["st"]["converged"] == 1, sol["st"]
    KE = fem.element_stiffness(0.3)
    r = np.asarray(f).ravel() - fem.apply_K(N, N, E, KE, u)
    free = fem.free_dofs(N, N, fem.BOTTOM)
    res = np.linalg.norm(r[free]) / np.linalg.norm(np.ravel(f)[free])
    print(f"{prec} 2048^2: iters {sol['st']['iters']}, oracle true residual {res:.3e}, "
          f"GPU-reported {sol['st']['rel_res_true']:.3e}")
    # The stopping rule tests the recursive residual (Alg. 2, tested before
    # the preconditioner); the float64 recursion drifts from the true
    # residual by a few percent at this tolerance (measured: 3% at 2048^2),
    # the mixed path's replacement every 25 steps keeps them closer.
    assert res <= 1.1 * TOL
    assert abs(res - sol["st"]["rel_res_true"]) <= 0.05 * res
    # Compliance and the energy identity.
    fu = sensitivity.compliance(f, u)
    assert abs(sol["C"] - fu) <= 1e-12 * abs(fu)
    w = sensitivity.element_energy_relative(N, N, KE, u)
    uKu = float(np.sum(E * w))
    assert abs(fu - uKu) <= np.linalg.norm(u) * np.linalg.norm(r[free]) * (1 + 1e-6)
    # Sensitivities at seeded picks, one element at a time.
    picks = uniform01(5, np.arange(2 * 4096, dtype=np.uint64)).reshape(4096, 2)
    phase = np.minimum((picks[:, 0] * 4).astype(np.int64), 3)
    elem = np.minimum((picks[:, 1] * N * N).astype(np.int64), N * N - 1)
    xe = x.reshape(4, -1)[phase, elem]
    ref = -3.0 * xe ** 2 * np.asarray(EP)[phase] * w.ravel()[elem]
    got = sol["g"].reshape(4, -1)[phase, elem]
    scale = np.abs(ref).max()
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-15 * scale)


def test_fullsize_fp64_matches_oracle(gpu_solutions, oracle_solution):
    sol = gpu_solutions["fp64"]
    ref = oracle_solution
    assert ref["converged"]
    err = rel(sol["u"], ref["u"])
    C_ref = float(np.dot(load_top_edge(N, N).ravel(), ref["u"].ravel()))
    print(f"fp64 2048^2 vs oracle: iters {sol['st']['iters']} vs {ref['iters']}, u rel {err:.3e}, "
          f"C rel {abs(sol['C'] - C_ref) / abs(C_ref):.3e}")
    assert err <= 1e-8
    assert abs(sol["C"] - C_ref) <= 1e-9 * abs(C_ref)
    assert abs(sol["st"]["iters"] - ref["iters"]) <= 1


def test_fullsize_mixed_matches_oracle_and_fp64(gpu_solutions, oracle_solution):
    mixed, fp64 = gpu_solutions["mixed"], gpu_solutions["fp64"]
    e_or = rel(mixed["u"], oracle_solution["u"])
    e_64 = rel(mixed["u"], fp64["u"])
    print(f"mixed 2048^2: iters {mixed['st']['iters']}, u rel vs oracle {e_or:.3e}, vs fp64 {e_64:.3e}")
    assert e_or <= 1e-8
    assert e_64 <= 1e-8


@pytest.mark.parametrize("variant", ["mixed_w", "fp64_redisc"])
def test_fullsize_other_cycles_match_oracle(gpu_solutions, oracle_solution, variant):
    # The W-cycle (gamma = 2 below the finest grid, Alg. 1) and the
    # rediscretised coarse operators (Sec. 2.1) change the preconditioner,
    # not the solution: u within the same 1e-8 of the oracle's V-cycle solve.
    sol = gpu_solutions[variant]
    err = rel(sol["u"], oracle_solution["u"])
    print(f"{variant} 2048^2: iters {sol['st']['iters']}, u rel vs oracle {err:.3e}")
    assert err <= 1e-8
