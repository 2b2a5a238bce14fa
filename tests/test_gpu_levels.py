"""pCGMG with every number of grids on the paper's small meshes (Sec. 5.2,
Tables 2-3: 32 x 32 and 32 x 64 with l = 2 ... 6 grids, Table 2's moduli),
through the C ABI, against the oracle.

l counts the grids (l = 2 is the two-level method), so n_coarsen = l - 1 and
the coarsest grids run down to 1 x 1 and 1 x 2 elements, with coarse levels
of 2 x 2 and 2 x 4 elements in between: the smallest grids the sweeps,
transfers and the dense coarsest solve see.  Bars: float64 solves at 1e-10
match the direct solve to 1e-8 and take the oracle's PCG iteration count
(+-1, summation order); at Table 2's cgtol 1e-6 the count is the oracle's
too; mixed solves reach a float64 true residual of 1e-8.
"""

import numpy as np
import pytest
import torch

from oracle import fem, solver
from synth import dirichlet_design, load_top_edge

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
E2 = [9.0, 3.0, 1.0, 1e-9]  # Table 2


@pytest.fixture(scope="module")
def mto():
    import paper_2301_07457_gb300 as m
    return m


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("l", [2, 3, 4, 5, 6])
@pytest.mark.parametrize("nelx,nely", [(32, 32), (32, 64)])
def test_levels_fp64(mto, nelx, nely, l):
    x = dirichlet_design(nelx, nely, 4, seed=l)
    f = load_top_edge(nelx, nely)
    ud = solver.solve_direct(nelx, nely, x, E2, 3.0, f)
    for tol in (1e-6, 1e-10):
        ref = solver.solve_pcgmg(nelx, nely, x, E2, 3.0, f, n_coarsen=l - 1, tol=tol)
        m = mto.Mesh(nelx, nely, n_coarsen=l - 1, tol=tol, max_it=1000)
        m.set_design(to_dev(x), E2, 3.0)
        u, st = m.solve(to_dev(f))
        assert m.info()["n_levels"] == l
        assert abs(st["iters"] - ref["iters"]) <= 1, (st["iters"], ref["iters"])
        if tol == 1e-10:
            err = np.linalg.norm(u.cpu().numpy() - ud) / np.linalg.norm(ud)
            assert err < 1e-8, err
        m.close()


@pytest.mark.parametrize("l", [2, 3, 4, 5, 6])
@pytest.mark.parametrize("nelx,nely", [(32, 32), (32, 64)])
def test_levels_mixed(mto, nelx, nely, l):
    x = dirichlet_design(nelx, nely, 4, seed=10 + l)
    f = load_top_edge(nelx, nely)
    E = fem.simp_moduli(x, E2, 3.0)
    m = mto.Mesh(nelx, nely, n_coarsen=l - 1, tol=1e-8, max_it=1000, precision="mixed")
    m.set_design(to_dev(x), E2, 3.0)
    u, st = m.solve(to_dev(f))
    assert st["status"] == "MTO_OK", st
    assert solver.true_relative_residual(nelx, nely, E, f, u.cpu().numpy()) <= 1e-8
    m.close()
