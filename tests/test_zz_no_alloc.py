"""The allocation-free compliance entry point against the context-based one.

mto_compliance_grad_noalloc serves callers that cannot allocate device memory
(for example when their memory pool owns the whole device).  It must give what
mto_compliance_grad gives, call after call, although every call reuses the
same fixed scratch array inside the library.  This file is collected last so
that a run stopping at the first failure has run every other test first.
"""

import ctypes

import numpy as np
import pytest
import torch

from synth import dirichlet_design, load_right_edge, load_top_edge

pytestmark = pytest.mark.gpu
EP = [1.0, 0.5, 0.25, 1e-9]
DEV = torch.device("cuda", 0)


def noalloc(lib, nelx, nely, x, f, u, want_grad=True):
    C = torch.full((1,), float("nan"), dtype=torch.float64, device=DEV)
    g = torch.full(x.shape, float("nan"), dtype=torch.float64, device=DEV) if want_grad else None
    Ep = (ctypes.c_double * 4)(*EP)
    code = lib.mto_compliance_grad_noalloc(
        nelx, nely, 0.3, 4, ctypes.c_void_p(x.data_ptr()), Ep, 3.0, ctypes.c_void_p(f.data_ptr()),
        ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(C.data_ptr()),
        ctypes.c_void_p(g.data_ptr()) if g is not None else None, 0,
        ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream))
    assert code == 0, code
    return C, g


@pytest.mark.parametrize("nelx,nely,nc,load", [(64, 64, 3, "top"), (200, 136, 3, "right"),
                                               (1024, 512, 5, "top")])
def test_noalloc_matches_context_entry_point(nelx, nely, nc, load):
    import paper_2301_07457_gb300 as mto
    from paper_2301_07457_gb300 import _lib
    lib = _lib.load()
    x = torch.from_numpy(dirichlet_design(nelx, nely, 4, seed=nelx)).to(DEV)
    fnp = load_top_edge(nelx, nely) if load == "top" else load_right_edge(nelx, nely)
    f = torch.from_numpy(fnp).to(DEV)
    mesh = mto.Mesh(nelx, nely, n_coarsen=nc, tol=1e-10)
    mesh.set_design(x, EP, 3.0)
    u, _ = mesh.solve(f)
    C_ref, g_ref = mesh.compliance_grad(f, u)
    # Two calls in a row: the second starts from whatever the first left in
    # the shared scratch array.
    for _ in range(2):
        C, g = noalloc(lib, nelx, nely, x, f, u)
        torch.cuda.synchronize()
        assert abs(C.item() - C_ref.item()) <= 1e-12 * abs(C_ref.item())
        np.testing.assert_allclose(g.cpu().numpy(), g_ref.cpu().numpy(), rtol=1e-12, atol=0.0)
    C2, g2 = noalloc(lib, nelx, nely, x, f, u, want_grad=False)
    assert g2 is None and abs(C2.item() - C_ref.item()) <= 1e-12 * abs(C_ref.item())
    mesh.close()


def test_noalloc_rejects_oversized_mesh():
    from paper_2301_07457_gb300 import _lib
    lib = _lib.load()
    t = torch.zeros(4, dtype=torch.float64, device=DEV)
    p = ctypes.c_void_p(t.data_ptr())
    Ep = (ctypes.c_double * 4)(*EP)
    # 8192 x 8192 elements = 67,125,249 nodes > 33,554,432: rejected before any device access.
    code = lib.mto_compliance_grad_noalloc(8192, 8192, 0.3, 4, p, Ep, 3.0, p, p, p, None, 0, None)
    assert code == _lib.ERR_UNSUPPORTED_MESH
    code = lib.mto_compliance_grad_noalloc(8, 8, 0.3, 4, p, Ep, 3.0, None, p, p, None, 0, None)
    assert code == _lib.ERR_ARG
    # The node count is formed in 64 bits: INT_MAX columns do not wrap around
    # to a small count that would pass the size check.
    code = lib.mto_compliance_grad_noalloc(2**31 - 1, 1, 0.3, 4, p, Ep, 3.0, p, p, p, None, 0, None)
    assert code == _lib.ERR_UNSUPPORTED_MESH
