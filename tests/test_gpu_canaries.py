"""Guard zones around every caller buffer of the C ABI (no compute-sanitizer
on this pool, so out-of-bounds accesses are caught by canaries instead).

Each input array is placed inside a larger allocation whose margins hold
NaN, so that an out-of-bounds read would poison the result; each output
array sits between margins holding a sentinel, so that an out-of-bounds
write would show.  The results must equal those of unguarded buffers bit
for bit, and every margin must be intact, on ragged meshes (strips and warp
tasks that do not divide the mesh) in both precisions.
"""

import ctypes

import numpy as np
import pytest
import torch

from synth import BOTTOM, LEFT, dirichlet_design, load_right_edge, load_top_edge

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
EP = [1.0, 0.5, 0.25, 1e-9]
G = 4098  # margin, in float64 elements: keeps nodal vectors 16-byte aligned, not 256-byte
SENTINEL = -1.2345678e300


@pytest.fixture(scope="module")
def mto():
    import paper_2301_07457_gb300 as m
    return m


def guarded(values, fill):
    """A device buffer [margin | values | margin]; returns (buffer, view of values)."""
    v = torch.as_tensor(values, dtype=torch.float64).reshape(-1)
    buf = torch.full((v.numel() + 2 * G,), fill, dtype=torch.float64, device=DEV)
    view = buf[G:G + v.numel()]
    view.copy_(v.to(DEV))
    return buf, view


def margins_intact(buf, n, fill):
    m = torch.cat([buf[:G], buf[G + n:]])
    return bool(torch.isnan(m).all()) if np.isnan(fill) else bool((m == fill).all())


def ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("nelx,nely,nc,fixed", [(200, 136, 3, BOTTOM), (96, 40, 2, BOTTOM | LEFT)])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_elasticity_entry_points(mto, nelx, nely, nc, fixed, prec):
    from paper_2301_07457_gb300 import _lib
    lib = _lib.load()
    x = dirichlet_design(nelx, nely, 4, seed=nelx + nely)
    F = np.stack([load_top_edge(nelx, nely), load_right_edge(nelx, nely)])
    nd = F[0].size
    kw = dict(fixed_edges=fixed, n_coarsen=nc, precision=prec, tol=1e-10 if prec == "fp64" else 1e-8)
    # Reference: ordinary tensors.
    ref = mto.Mesh(nelx, nely, **kw)
    ref.set_design(torch.from_numpy(x).to(DEV), EP, 3.0)
    U_ref, _ = ref.solve(torch.from_numpy(F).to(DEV))
    C_ref, g_ref = ref.compliance_grad(torch.from_numpy(F).to(DEV), U_ref)
    v = np.random.default_rng(1).standard_normal(nd)
    y_ref = ref.apply_operator(nc, torch.from_numpy(v.reshape(F[0].shape)).to(DEV))
    z_ref = ref.apply_preconditioner(torch.from_numpy(v.reshape(F[0].shape)).to(DEV))
    # Guarded: inputs in NaN margins, outputs in sentinel margins.
    m = mto.Mesh(nelx, nely, **kw)
    xb, xv = guarded(x, float("nan"))
    Ep = (ctypes.c_double * 4)(*EP)
    assert lib.mto_set_design(m._h, 4, ptr(xv), Ep, 3.0) == 0
    fb, fv = guarded(F, float("nan"))
    ub, uv = guarded(np.zeros(F.size), SENTINEL)
    st = _lib.SolveStats()
    assert lib.mto_solve(m._h, 2, ptr(fv), ptr(uv), ctypes.byref(st)) == 0
    cb, cv = guarded(np.zeros(2), SENTINEL)
    gb, gv = guarded(np.zeros(x.size), SENTINEL)
    assert lib.mto_compliance_grad(m._h, 2, ptr(fv), ptr(uv), ptr(cv), ptr(gv)) == 0
    vb, vv = guarded(v, float("nan"))
    yb, yv = guarded(np.zeros(nd), SENTINEL)
    assert lib.mto_apply_operator(m._h, nc, 0, ptr(vv), ptr(yv)) == 0
    zb, zv = guarded(np.zeros(nd), SENTINEL)
    assert lib.mto_apply_preconditioner(m._h, ptr(vv), ptr(zv)) == 0
    torch.cuda.synchronize()
    for buf, view, fill in ((xb, xv, float("nan")), (fb, fv, float("nan")), (vb, vv, float("nan")),
                            (ub, uv, SENTINEL), (cb, cv, SENTINEL), (gb, gv, SENTINEL),
                            (yb, yv, SENTINEL), (zb, zv, SENTINEL)):
        assert margins_intact(buf, view.numel(), fill)
    assert torch.equal(uv, U_ref.reshape(-1))
    assert torch.equal(cv, C_ref) and torch.equal(gv, g_ref.reshape(-1))
    assert torch.equal(yv, y_ref.reshape(-1)) and torch.equal(zv, z_ref.reshape(-1))
    # A nodal vector that is not 16-byte aligned is rejected before any device work.
    assert lib.mto_solve(m._h, 1, ctypes.c_void_p(fv.data_ptr() + 8), ptr(uv), None) == _lib.ERR_ARG
    assert lib.mto_compliance_grad(m._h, 1, ptr(fv), ctypes.c_void_p(uv.data_ptr() + 8), ptr(cv),
                                   None) == _lib.ERR_ARG
    assert lib.mto_apply_preconditioner(m._h, ctypes.c_void_p(vv.data_ptr() + 8), ptr(zv)) == _lib.ERR_ARG
    m.close()
    ref.close()


def test_host_buffers_and_noalloc(mto):
    from paper_2301_07457_gb300 import _lib
    lib = _lib.load()
    nelx, nely = 120, 72
    x = dirichlet_design(nelx, nely, 4, seed=5)
    f = load_top_edge(nelx, nely)
    m = mto.Mesh(nelx, nely, n_coarsen=3, precision="mixed")
    u_ref, C_ref, g_ref, _ = m.run_host(x, EP, 3.0, f)

    def host_guarded(values, fill):
        buf = np.full(np.asarray(values).size + 2 * G, fill)
        buf[G:G + np.asarray(values).size] = np.asarray(values).ravel()
        return buf

    xb, fb = host_guarded(x, np.nan), host_guarded(f, np.nan)
    ub, cb, gb = host_guarded(np.zeros(f.size), SENTINEL), host_guarded([0.0], SENTINEL), \
        host_guarded(np.zeros(x.size), SENTINEL)
    Ep = (ctypes.c_double * 4)(*EP)
    at = lambda a: ctypes.c_void_p(a.ctypes.data + 8 * G)
    st = _lib.SolveStats()
    assert lib.mto_run_host(m._h, 4, at(xb), Ep, 3.0, 1, at(fb), at(ub), at(cb), at(gb), ctypes.byref(st)) == 0
    for buf, n, fill in ((ub, f.size, SENTINEL), (cb, 1, SENTINEL), (gb, x.size, SENTINEL)):
        assert (buf[:G] == fill).all() and (buf[G + n:] == fill).all()
    assert np.isnan(xb[:G]).all() and np.isnan(fb[G + f.size:]).all()
    assert np.array_equal(ub[G:G + f.size], u_ref.ravel())
    assert cb[G] == C_ref[0] and np.array_equal(gb[G:G + x.size], g_ref.ravel())
    # The allocation-free compliance entry point.
    ud = torch.from_numpy(u_ref).to(DEV)
    xd = torch.from_numpy(x).to(DEV)
    fd = torch.from_numpy(f).to(DEV)
    cdb, cdv = guarded([0.0], SENTINEL)
    gdb, gdv = guarded(np.zeros(x.size), SENTINEL)
    assert lib.mto_compliance_grad_noalloc(nelx, nely, 0.3, 4, ptr(xd), Ep, 3.0, ptr(fd), ptr(ud), ptr(cdv),
                                           ptr(gdv), 0, ctypes.c_void_p(torch.cuda.current_stream(DEV).cuda_stream)) == 0
    torch.cuda.synchronize()
    assert margins_intact(cdb, 1, SENTINEL) and margins_intact(gdb, x.size, SENTINEL)
    np.testing.assert_allclose(gdv.cpu().numpy(), g_ref.ravel(), rtol=1e-12, atol=0)
    m.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_poisson_entry_points(mto, prec):
    from paper_2301_07457_gb300 import _lib
    lib = _lib.load()
    nx, ny = 200, 136
    p = mto.Poisson(nx, ny, n_coarsen=3, tol=1e-10, precision=prec)
    F = np.random.default_rng(2).standard_normal((2, ny + 1, nx + 1))
    U_ref, _ = p.solve(torch.from_numpy(F).to(DEV))
    v = np.random.default_rng(3).standard_normal((ny + 1, nx + 1))
    y_ref = p.apply_operator(torch.from_numpy(v).to(DEV))
    z_ref = p.apply_preconditioner(torch.from_numpy(v).to(DEV))
    fb, fv = guarded(F, float("nan"))
    ub, uv = guarded(np.zeros(F.size), SENTINEL)
    st = _lib.SolveStats()
    assert lib.mto_poisson_solve(p._h, 2, ptr(fv), ptr(uv), ctypes.byref(st)) == 0
    vb, vv = guarded(v, float("nan"))
    yb, yv = guarded(np.zeros(v.size), SENTINEL)
    zb, zv = guarded(np.zeros(v.size), SENTINEL)
    assert lib.mto_poisson_apply_operator(p._h, ptr(vv), ptr(yv)) == 0
    assert lib.mto_poisson_apply_preconditioner(p._h, ptr(vv), ptr(zv)) == 0
    torch.cuda.synchronize()
    for buf, view, fill in ((fb, fv, float("nan")), (vb, vv, float("nan")), (ub, uv, SENTINEL),
                            (yb, yv, SENTINEL), (zb, zv, SENTINEL)):
        assert margins_intact(buf, view.numel(), fill)
    assert torch.equal(uv, U_ref.reshape(-1))
    assert torch.equal(yv, y_ref.reshape(-1)) and torch.equal(zv, z_ref.reshape(-1))
    p.close()
