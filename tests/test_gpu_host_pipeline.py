"""Pipelined host calls (mto_run_host_async / mto_run_host_wait) through the C ABI.

Each pipelined call runs the same kernels on the same data as the blocking
mto_run_host, so u, the compliances, the sensitivities and the iteration
counts must agree bit for bit, in both precisions, while two calls are in
flight, across calls that change the design, the number of load cases and
whether sensitivities are wanted, and with device work of other entry points
issued in between.  Also: the state errors, and guard zones around pinned
host buffers.
"""

import ctypes

import numpy as np
import pytest
import torch

from synth import BOTTOM, LEFT, dirichlet_design, load_right_edge, load_top_edge

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
EP = [1.0, 0.5, 0.25, 1e-9]


@pytest.fixture(scope="module")
def mto():
    import paper_2301_07457_gb300 as m
    return m


def calls(nelx, nely):
    """(x, f, want_grad) of six calls: new designs, one or two load cases."""
    top, right = load_top_edge(nelx, nely), load_right_edge(nelx, nely)
    out = []
    for k in range(6):
        x = dirichlet_design(nelx, nely, 4, seed=100 + k)
        f = np.stack([top * (1 + k), right]) if k % 3 == 1 else top * (1 + 0.5 * k)
        out.append((x, f, k != 4))
    return out


def same(a, b):
    ua, Ca, ga, sa = a
    ub, Cb, gb, sb = b
    assert np.array_equal(ua, ub) and np.array_equal(Ca, Cb)
    assert (ga is None and gb is None) or np.array_equal(ga, gb)
    assert sa["iters"] == sb["iters"] and sa["rel_res_true"] == sb["rel_res_true"]


@pytest.mark.parametrize("prec,fixed", [("fp64", BOTTOM), ("mixed", BOTTOM | LEFT)])
def test_pipelined_equals_blocking(mto, prec, fixed):
    nelx, nely = 200, 136
    kw = dict(fixed_edges=fixed, n_coarsen=3, precision=prec, tol=1e-10 if prec == "fp64" else 1e-8)
    cs = calls(nelx, nely)
    ref_mesh = mto.Mesh(nelx, nely, **kw)
    ref = [ref_mesh.run_host(x, EP, 3.0, f, want_grad=g) for x, f, g in cs]
    ref_mesh.close()
    m = mto.Mesh(nelx, nely, **kw)
    got = []
    x, f, g = cs[0]
    m.run_host_async(x, EP, 3.0, f, want_grad=g)
    for k in range(1, len(cs)):
        # Pinned torch inputs are used in place, numpy ones copied first.
        x, f, g = cs[k]
        if k % 2:
            x, f = torch.from_numpy(x).pin_memory(), torch.from_numpy(f).pin_memory()
        m.run_host_async(x, EP, 3.0, f, want_grad=g)
        got.append(m.run_host_wait())
    got.append(m.run_host_wait())
    for a, b in zip(got, ref):
        same(a, b)
    assert m.design_version == len(cs)
    m.close()


def test_other_entry_points_in_between(mto):
    nelx, nely = 128, 96
    kw = dict(n_coarsen=3, precision="mixed")
    x0, x1 = dirichlet_design(nelx, nely, 4, seed=7), dirichlet_design(nelx, nely, 4, seed=8)
    f = load_top_edge(nelx, nely)
    ref_mesh = mto.Mesh(nelx, nely, **kw)
    r0 = ref_mesh.run_host(x0, EP, 3.0, f)
    ref_mesh.set_design(torch.from_numpy(x1).to(DEV), EP, 3.0)
    U_ref, _ = ref_mesh.solve(torch.from_numpy(f).to(DEV))
    C_ref, g_ref = ref_mesh.compliance_grad(torch.from_numpy(f).to(DEV), U_ref)
    ref_mesh.close()
    m = mto.Mesh(nelx, nely, **kw)
    m.run_host_async(x0, EP, 3.0, f)
    # A device-side design and solve while the host call is outstanding.
    m.set_design(torch.from_numpy(x1).to(DEV), EP, 3.0)
    U, _ = m.solve(torch.from_numpy(f).to(DEV))
    C, g = m.compliance_grad(torch.from_numpy(f).to(DEV), U)
    same(m.run_host_wait(), r0)
    assert torch.equal(U, U_ref) and torch.equal(C, C_ref) and torch.equal(g, g_ref)
    # Closing with a call outstanding waits for it.
    m.run_host_async(x0, EP, 3.0, f)
    m.close()


def test_state_errors(mto):
    from paper_2301_07457_gb300 import _lib
    lib = _lib.load()
    nelx, nely = 64, 48
    m = mto.Mesh(nelx, nely, n_coarsen=2, precision="fp64", tol=1e-10)
    x, f = dirichlet_design(nelx, nely, 4, seed=3), load_top_edge(nelx, nely)
    st = _lib.SolveStats()
    assert lib.mto_run_host_wait(m._h, ctypes.byref(st)) == _lib.ERR_STATE
    r = m.run_host(x, EP, 3.0, f)
    m.run_host_async(x, EP, 3.0, f)
    m.run_host_async(x, EP, 3.0, f)
    with pytest.raises(RuntimeError):  # a third outstanding call
        m.run_host_async(x, EP, 3.0, f)
    with pytest.raises(RuntimeError):  # the blocking call while calls are outstanding
        m.run_host(x, EP, 3.0, f)
    same(m.run_host_wait(), r)
    same(m.run_host_wait(), r)
    with pytest.raises(RuntimeError):
        m.run_host_wait()
    m.set_kernel_timing(True)
    with pytest.raises(RuntimeError):
        m.run_host_async(x, EP, 3.0, f)
    m.set_kernel_timing(False)
    same(m.run_host(x, EP, 3.0, f), r)
    # Bad arguments are rejected before anything is enqueued.
    Ep = (ctypes.c_double * 4)(*EP)
    xp = torch.from_numpy(x).pin_memory()
    fp = torch.from_numpy(f).pin_memory()
    out = torch.empty(f.size + 1, dtype=torch.float64).pin_memory()
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    assert lib.mto_run_host_async(m._h, 4, p(xp), Ep, 3.0, 0, p(fp), p(out), p(out), None) == _lib.ERR_ARG
    assert lib.mto_run_host_async(m._h, 4, None, Ep, 3.0, 1, p(fp), p(out), p(out), None) == _lib.ERR_ARG
    assert lib.mto_run_host_wait(m._h, None) == _lib.ERR_STATE
    m.close()


G = 4098  # margin in float64 elements
SENTINEL = -1.2345678e300


def test_guard_zones_pinned(mto):
    from paper_2301_07457_gb300 import _lib
    lib = _lib.load()
    nelx, nely = 120, 72
    x = dirichlet_design(nelx, nely, 4, seed=5)
    F = np.stack([load_top_edge(nelx, nely), load_right_edge(nelx, nely)])
    m = mto.Mesh(nelx, nely, n_coarsen=3, precision="mixed")
    u_ref, C_ref, g_ref, _ = m.run_host(x, EP, 3.0, F)

    def guarded(values, fill):
        v = np.asarray(values, dtype=np.float64).ravel()
        buf = torch.full((v.size + 2 * G,), fill, dtype=torch.float64).pin_memory()
        buf[G:G + v.size] = torch.from_numpy(v)
        return buf, v.size

    at = lambda b: ctypes.c_void_p(b.data_ptr() + 8 * G)
    bufs = {}
    for k in range(2):  # two calls in flight, each with its own guarded arrays
        bufs[k] = dict(x=guarded(x, np.nan), f=guarded(F, np.nan), u=guarded(np.zeros(F.size), SENTINEL),
                       C=guarded(np.zeros(2), SENTINEL), g=guarded(np.zeros(x.size), SENTINEL))
        b = bufs[k]
        Ep = (ctypes.c_double * 4)(*EP)
        assert lib.mto_run_host_async(m._h, 4, at(b["x"][0]), Ep, 3.0, 2, at(b["f"][0]), at(b["u"][0]),
                                      at(b["C"][0]), at(b["g"][0])) == 0
    for k in range(2):
        assert lib.mto_run_host_wait(m._h, None) == 0
        b = bufs[k]
        for name, fill in (("x", np.nan), ("f", np.nan), ("u", SENTINEL), ("C", SENTINEL), ("g", SENTINEL)):
            buf, n = b[name]
            edge = torch.cat([buf[:G], buf[G + n:]])
            assert bool(torch.isnan(edge).all()) if np.isnan(fill) else bool((edge == fill).all()), name
        assert np.array_equal(b["u"][0][G:G + F.size].numpy(), u_ref.ravel())
        assert np.array_equal(b["C"][0][G:G + 2].numpy(), C_ref)
        assert np.array_equal(b["g"][0][G:G + x.size].numpy(), g_ref.ravel())
    m.close()


def test_breakdown_in_flight(mto):
    # A design whose coarsest system cannot be factorised (a NaN fraction)
    # between two good calls: its wait reports the breakdown, the calls
    # around it are unaffected, and the context keeps working.
    from paper_2301_07457_gb300 import MtoError, _lib
    nelx, nely = 96, 64
    m = mto.Mesh(nelx, nely, n_coarsen=3, precision="mixed")
    x, f = dirichlet_design(nelx, nely, 4, seed=11), load_top_edge(nelx, nely)
    r = m.run_host(x, EP, 3.0, f)
    bad = x.copy()
    bad[0, 7, 9] = np.nan
    m.run_host_async(x, EP, 3.0, f)
    m.run_host_async(bad, EP, 3.0, f)
    same(m.run_host_wait(), r)
    with pytest.raises(MtoError) as e:
        m.run_host_wait()
    assert e.value.code == _lib.ERR_BREAKDOWN
    m.run_host_async(x, EP, 3.0, f)
    same(m.run_host_wait(), r)
    same(m.run_host(x, EP, 3.0, f), r)
    m.close()
