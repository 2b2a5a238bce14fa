"""Out-of-memory paths, driven by the library's device-memory limit
(mto_set_device_memory_limit) instead of by filling the GPU: an allocation
that would pass the limit fails as cudaMalloc would, and the call returns
MTO_ERR_OOM (contexts, Poisson solvers) or runs its load cases one after
another (a concurrent-load-case workspace that does not fit).  Nothing may
leak: the ledger returns to where it was."""

import numpy as np
import pytest
import torch

from synth import dirichlet_design, load_right_edge, load_top_edge

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
EP = [1.0, 0.5, 0.25, 1e-9]


@pytest.fixture(scope="module")
def mto():
    import paper_2301_07457_gb300 as m
    yield m
    m.set_device_memory_limit(0)


def test_limit_gives_oom_without_leaks(mto):
    from paper_2301_07457_gb300 import _lib
    base = mto.device_memory_in_use()
    mto.set_device_memory_limit(base + (1 << 20))
    try:
        with pytest.raises(mto.MtoError) as e:
            mto.Mesh(256, 256, n_coarsen=4)
        assert e.value.code == _lib.ERR_OOM
        assert mto.device_memory_in_use() == base
        with pytest.raises(mto.MtoError) as e:
            mto.Poisson(256, 256, n_coarsen=7)
        assert e.value.code == _lib.ERR_OOM
        assert mto.device_memory_in_use() == base
    finally:
        mto.set_device_memory_limit(0)
    m = mto.Mesh(256, 256, n_coarsen=4)
    assert mto.device_memory_in_use() > base
    m.close()
    assert mto.device_memory_in_use() == base


def test_workspace_that_does_not_fit_runs_load_cases_in_turn(mto):
    n = 256
    x = torch.from_numpy(dirichlet_design(n, n, 4, seed=31)).to(DEV)
    F = torch.from_numpy(np.stack([load_top_edge(n, n), load_right_edge(n, n)])).to(DEV)
    ref = mto.Mesh(n, n, n_coarsen=4, precision="mixed", concurrent_rhs=1)
    ref.set_design(x, EP, 3.0)
    U_ref, s_ref = ref.solve(F)
    m = mto.Mesh(n, n, n_coarsen=4, precision="mixed", concurrent_rhs=2)
    m.set_design(x, EP, 3.0)
    held = mto.device_memory_in_use()
    mto.set_device_memory_limit(held + (1 << 20))  # no room for a second workspace
    try:
        U1, s1 = m.solve(F)
    finally:
        mto.set_device_memory_limit(0)
    assert mto.device_memory_in_use() == held
    assert torch.equal(U1, U_ref) and s1["iters"] == s_ref["iters"]
    U2, _ = m.solve(F)  # now the workspace is created
    assert mto.device_memory_in_use() > held
    assert torch.equal(U2, U_ref)
    m.close()
    ref.close()
