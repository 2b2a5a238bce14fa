"""Control paths of the mixed-precision PCG step (Alg. 2 with the float32
V-cycle of Alg. 1 as preconditioner), through the C ABI.

The update r -= alpha q of each step is applied by the next V-cycle's first
smoothing sweep, out of place into a second r buffer, and residual
replacement (every rr_every steps) supersedes it.  These tests drive the
paths around it: frequent replacement, the iteration limit, warm starts, the
host-polled loop against the device-side loop, and repeated solves on the
same context.  Pass criterion of every converged solve: the float64 true
relative residual, recomputed by the oracle from the returned u, is at most
the requested tolerance.
"""

import numpy as np
import pytest
import torch

from oracle import fem, solver
from synth import dirichlet_design, load_right_edge, load_top_edge

pytestmark = pytest.mark.gpu
EP = [1.0, 0.5, 0.25, 1e-9]
DEV = torch.device("cuda", 0)
N, NC = 128, 3


@pytest.fixture(scope="module")
def mto():
    import paper_2301_07457_gb300 as m
    return m


@pytest.fixture(scope="module")
def problem():
    x = dirichlet_design(N, N, 4, seed=11)
    f = load_top_edge(N, N)
    return x, f, fem.simp_moduli(x, EP, 3.0)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def solve(mto, x, f, **kw):
    m = mto.Mesh(N, N, n_coarsen=NC, tol=kw.pop("tol", 1e-8), precision="mixed", **kw)
    m.set_design(to_dev(x), EP, 3.0)
    u, st = m.solve(to_dev(f), raise_on_failure=False)
    return m, u.cpu().numpy(), st


@pytest.mark.parametrize("rr_every", [0, 1, 3, 25])
def test_replacement_interval(mto, problem, rr_every):
    x, f, E = problem
    m, u, st = solve(mto, x, f, rr_every=rr_every)
    assert st["status"] == "MTO_OK", st
    assert solver.true_relative_residual(N, N, E, f, u) <= 1e-8
    assert st["rel_res_true"] <= 1e-8
    m.close()


def test_replacement_keeps_iteration_count(mto, problem):
    x, f, _ = problem
    counts = []
    for rr in (0, 3, 25):
        m, _, st = solve(mto, x, f, rr_every=rr)
        counts.append(st["iters"])
        m.close()
    assert max(counts) - min(counts) <= 2, counts


def test_iteration_limit(mto, problem):
    x, f, E = problem
    m, u, st = solve(mto, x, f, max_it=5)
    assert st["status"] == "MTO_ERR_NOT_CONVERGED", st
    assert st["iters"] == 5
    # The returned u is the iterate of step 5: its true residual is the one
    # the solver reports.
    r = solver.true_relative_residual(N, N, E, f, u)
    assert abs(r - st["rel_res_true"]) <= 1e-6 * r
    m.close()


def test_polled_loop_matches_device_loop(mto, problem):
    x, f, _ = problem
    m, u_dev, st_dev = solve(mto, x, f)
    m.set_kernel_timing(True)  # host-polled loop with event nodes
    u_pol, st_pol = m.solve(to_dev(f))
    m.set_kernel_timing(False)
    assert st_pol["iters"] == st_dev["iters"]
    assert np.array_equal(u_pol.cpu().numpy(), u_dev)
    m.close()


def test_repeated_solves_and_warm_start(mto, problem):
    x, f, E = problem
    m, u1, st1 = solve(mto, x, f)
    u2, st2 = m.solve(to_dev(f))
    assert st2["iters"] == st1["iters"]
    assert np.array_equal(u2.cpu().numpy(), u1)
    # Another right-hand side on the same context, then a warm start from
    # the converged solution (no step needed).
    g = load_right_edge(N, N)
    u3, st3 = m.solve(to_dev(g))
    assert solver.true_relative_residual(N, N, E, g, u3.cpu().numpy()) <= 1e-8
    u4, st4 = m.solve(to_dev(g), u0=u3)
    assert st4["iters"] == 0
    m.close()
