"""Load cases solved at the same time (opts.concurrent_rhs) through the C ABI.

mto_solve with several right-hand sides runs right-hand side k on workspace
k mod S, each with its own vectors, scalars, stream and solve graph, all
reading the same design data.  The arithmetic of every solve is the same as
when the load cases run one after another, so the results must agree bit for
bit, in both precisions, with more load cases than workspaces, after a new
design, and after the launch shapes change.
"""

import numpy as np
import pytest
import torch

from oracle import fem, solver
from synth import dirichlet_design, load_right_edge, load_top_edge

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
EP = [1.0, 0.5, 0.25, 1e-9]


@pytest.fixture(scope="module")
def mto():
    import paper_2301_07457_gb300 as m
    return m


def loads(n, k):
    base = [load_top_edge(n, n), load_right_edge(n, n)]
    out = [base[i % 2] * (1.0 + 0.25 * i) for i in range(k)]
    return torch.from_numpy(np.stack(out)).to(DEV)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("slots,n_rhs", [(2, 2), (2, 5), (3, 4), (4, 4)])
def test_concurrent_equals_sequential(mto, prec, slots, n_rhs):
    n = 128
    x = torch.from_numpy(dirichlet_design(n, n, 4, seed=21)).to(DEV)
    F = loads(n, n_rhs)
    kw = dict(n_coarsen=3, precision=prec, tol=1e-10 if prec == "fp64" else 1e-8)
    seq = mto.Mesh(n, n, concurrent_rhs=1, **kw)
    con = mto.Mesh(n, n, concurrent_rhs=slots, **kw)
    for m in (seq, con):
        m.set_design(x, EP, 3.0)
    U1, s1 = seq.solve(F)
    U2, s2 = con.solve(F)
    assert torch.equal(U1, U2)
    assert s1["iters"] == s2["iters"] and s1["rel_res_true"] == s2["rel_res_true"]
    # The context counts every kernel its workspaces launched.
    assert con.launch_count() == seq.launch_count()
    # A new design is seen by every workspace.
    x2 = torch.from_numpy(dirichlet_design(n, n, 4, seed=22)).to(DEV)
    for m in (seq, con):
        m.set_design(x2, EP, 3.0)
    U1, _ = seq.solve(F)
    U2, _ = con.solve(F)
    assert torch.equal(U1, U2)
    E = fem.simp_moduli(x2.cpu().numpy(), EP, 3.0)
    for k in range(n_rhs):
        r = solver.true_relative_residual(n, n, E, F[k].cpu().numpy(), U2[k].cpu().numpy())
        assert r <= (1.1e-10 if prec == "fp64" else 1e-8)
    seq.close()
    con.close()


def test_concurrent_after_tuning_and_with_timing(mto):
    n = 256
    x = torch.from_numpy(dirichlet_design(n, n, 4, seed=23)).to(DEV)
    F = loads(n, 2)
    seq = mto.Mesh(n, n, n_coarsen=4, precision="mixed", concurrent_rhs=1)
    con = mto.Mesh(n, n, n_coarsen=4, precision="mixed", concurrent_rhs=2)
    for m in (seq, con):
        m.set_design(x, EP, 3.0)
    con.solve(F)  # builds the workspace's graph with the default launch shapes
    for m in (seq, con):
        m.autotune()  # may change the shapes: the workspace's graph is rebuilt
    U1, _ = seq.solve(F)
    U2, _ = con.solve(F)
    assert torch.equal(U1, U2)
    # Kernel timing drives the loop from the host: one load case at a time.
    con.set_kernel_timing(True)
    U3, _ = con.solve(F)
    con.set_kernel_timing(False)
    assert torch.equal(U3, U1)
    seq.close()
    con.close()
