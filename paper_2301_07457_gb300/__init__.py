"""GB300 pCGMG solver for multi-material compliance topology optimisation.

Python layer over libmto (C ABI in include/mto.h).  PyTorch provides device
memory and the current CUDA stream; every arithmetic step of the solve runs in
libmto's sm_103a kernels.  Paper: Luu & Banh, arXiv 2301.07457 -- Alg. 2
(PCG) preconditioned by Alg. 1 (V-cycle), Eq. 5 (multi-material SIMP),
Eqs. 6-9 (Q4 plane-stress compliance problem).
"""

import ctypes

import torch

from . import _lib
from ._lib import (  # noqa: F401
    COARSE_GALERKIN,
    COARSE_REDISCRETIZE,
    EDGE_BOTTOM,
    EDGE_LEFT,
    EDGE_RIGHT,
    EDGE_TOP,
    PRECISION_FP64,
    PRECISION_MIXED,
    MtoError,
    SolverOpts,
    SolveStats,
)

__all__ = ["Mesh", "Batch", "Poisson", "Compliance", "compliance", "measure_fp64_rate",
           "set_device_memory_limit", "device_memory_in_use", "MtoError", "SolverOpts", "SolveStats"]


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _dev_f64(t, device, name):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.device != device or t.dtype != torch.float64:
        raise ValueError(f"{name} must be a float64 tensor on {device}")
    return t.contiguous()


def set_device_memory_limit(nbytes):
    """Limit on the device memory this library holds (0: none); see include/mto.h."""
    _lib.load().mto_set_device_memory_limit(int(nbytes))


def device_memory_in_use():
    """Bytes of device memory this library holds now."""
    return int(_lib.load().mto_device_memory_in_use())


def measure_fp64_rate(device=None):
    """Measured float64 FMA issue rate of the device (operations per second)."""
    lib = _lib.load()
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
    v = ctypes.c_double()
    with torch.cuda.device(dev):
        _lib.check(lib.mto_measure_fp64_rate(dev.index, _stream(dev), ctypes.byref(v)),
                   "mto_measure_fp64_rate")
    return v.value


class Mesh:
    """A square-wall mesh (nelx x nely unit Q4 elements) with its level hierarchy.

    precision: "fp64" or "mixed" (float32 V-cycle with bfloat16 moduli inside a
    float64 CG).  Other keywords are the fields of mto_solver_opts.
    """

    def __init__(self, nelx, nely, nu=0.3, fixed_edges=EDGE_BOTTOM, n_coarsen=3,
                 precision="fp64", tol=1e-8, max_it=500, omega=0.6, nu1=2, nu2=2,
                 coarse_kind="galerkin", rr_every=25, flexible=None, check_every=4,
                 gamma=1, concurrent_rhs=2, device=None):
        lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        o = _lib.default_opts()
        o.tol, o.max_it, o.omega, o.nu1, o.nu2 = tol, max_it, omega, nu1, nu2
        o.n_coarsen = n_coarsen
        o.coarse_kind = {"galerkin": COARSE_GALERKIN, "rediscretize": COARSE_REDISCRETIZE}[coarse_kind]
        o.precision = {"fp64": PRECISION_FP64, "mixed": PRECISION_MIXED}[precision]
        o.rr_every = rr_every
        o.flexible = int(precision == "mixed") if flexible is None else int(flexible)
        o.check_every = check_every
        o.gamma = gamma
        o.concurrent_rhs = concurrent_rhs
        self.opts = o
        self.nelx, self.nely, self.nu, self.fixed_edges = nelx, nely, nu, fixed_edges
        self.precision = precision
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            code = lib.mto_create_mesh(ctypes.byref(self._h), nelx, nely, nu, fixed_edges,
                                       ctypes.byref(o), self.device.index, _stream(self.device))
        _lib.check(code, "mto_create_mesh")
        self._lib = lib
        self.n_phase = None
        self.E_phase = None
        self.penal = None
        # Counts set_design calls: a saved value tells whether the operators
        # on the device are still those of a given design.
        self.design_version = 0
        self.last_solve_stats = None
        self._pending = []  # host arrays of outstanding run_host_async calls

    # -- lifecycle -----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.mto_destroy(self._h)  # waits for outstanding host calls
            self._h = ctypes.c_void_p()
            self._pending = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def node_shape(self):
        return (self.nely + 1, self.nelx + 1, 2)

    def info(self):
        nl, n0 = ctypes.c_int(), ctypes.c_int()
        _lib.check(self._lib.mto_get_info(self._h, ctypes.byref(nl), ctypes.byref(n0)), "mto_get_info")
        return {"n_levels": nl.value, "coarsest_free_dofs": n0.value}

    # -- solver --------------------------------------------------------------
    def set_design(self, x, E_phase, penal=3.0):
        """x: float64 [n_phase][nely][nelx] on the mesh's device (Eq. 5)."""
        x = _dev_f64(x, self.device, "x")
        if x.dim() != 3 or x.shape[1:] != (self.nely, self.nelx):
            raise ValueError("x must be [n_phase][nely][nelx]")
        E = (ctypes.c_double * len(E_phase))(*[float(e) for e in E_phase])
        with torch.cuda.device(self.device):
            code = self._lib.mto_set_design(self._h, x.shape[0], _ptr(x), E, float(penal))
        _lib.check(code, "mto_set_design")
        self.n_phase, self.E_phase, self.penal = x.shape[0], list(E_phase), float(penal)
        self._x = x
        self.design_version += 1

    def solve(self, f, u0=None, raise_on_failure=True):
        """Solve K u = f (f: [n_rhs?][nely+1][nelx+1][2] float64).  Returns (u, stats)."""
        f = _dev_f64(f, self.device, "f")
        batched = f.dim() == 4
        if f.shape[-3:] != self.node_shape:
            raise ValueError(f"f must end in {self.node_shape}")
        u = torch.zeros_like(f) if u0 is None else _dev_f64(u0, self.device, "u0").clone()
        n_rhs = f.shape[0] if batched else 1
        st = SolveStats()
        with torch.cuda.device(self.device):
            code = self._lib.mto_solve(self._h, n_rhs, _ptr(f), _ptr(u), ctypes.byref(st))
        if code not in (_lib.OK, _lib.ERR_NOT_CONVERGED, _lib.ERR_BREAKDOWN) or (
                raise_on_failure and code != _lib.OK):
            _lib.check(code, "mto_solve")
        d = st.as_dict()
        d["status"] = _lib.STATUS[code]
        self.last_solve_stats = d
        return u, d

    def compliance_grad(self, f, u, want_grad=True):
        """C_k = f_k . u_k and dC/dx summed over load cases (Eq. 6, Sec. 4)."""
        f = _dev_f64(f, self.device, "f")
        u = _dev_f64(u, self.device, "u")
        n_rhs = f.shape[0] if f.dim() == 4 else 1
        C = torch.empty(n_rhs, dtype=torch.float64, device=self.device)
        g = None
        if want_grad:
            g = torch.empty((self.n_phase, self.nely, self.nelx), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            code = self._lib.mto_compliance_grad(self._h, n_rhs, _ptr(f), _ptr(u), _ptr(C),
                                                 _ptr(g) if g is not None else None)
        _lib.check(code, "mto_compliance_grad")
        return C, g

    def run_host(self, x, E_phase, penal, f, want_grad=True):
        """set_design + solve + compliance with host (numpy, float64) buffers."""
        import numpy as np
        x = np.ascontiguousarray(x, dtype=np.float64)
        f = np.ascontiguousarray(f, dtype=np.float64)
        n_rhs = f.shape[0] if f.ndim == 4 else 1
        u = np.zeros_like(f)
        C = np.zeros(n_rhs)
        g = np.zeros(x.shape) if want_grad else None
        E = (ctypes.c_double * len(E_phase))(*[float(e) for e in E_phase])
        st = SolveStats()
        with torch.cuda.device(self.device):
            code = self._lib.mto_run_host(
                self._h, x.shape[0], x.ctypes.data_as(ctypes.c_void_p), E, float(penal), n_rhs,
                f.ctypes.data_as(ctypes.c_void_p), u.ctypes.data_as(ctypes.c_void_p),
                C.ctypes.data_as(ctypes.c_void_p),
                g.ctypes.data_as(ctypes.c_void_p) if g is not None else None, ctypes.byref(st))
        _lib.check(code, "mto_run_host")
        self._host_design(x.shape[0], E_phase, penal)
        return u, C, g, st.as_dict()

    def _host_design(self, n_phase, E_phase, penal):
        # A host call leaves its design on the device, as set_design does.
        self.n_phase, self.E_phase, self.penal = n_phase, list(E_phase), float(penal)
        self.design_version += 1

    def run_host_async(self, x, E_phase, penal, f, want_grad=True):
        """Enqueue run_host without waiting (at most two calls outstanding).

        x and f: float64 host arrays; pinned CPU tensors are used in place
        (the caller leaves them unchanged until the matching run_host_wait),
        anything else is first copied into pinned memory.  The outputs are
        pinned and handed back by run_host_wait, oldest call first.
        """
        def pinned(a):
            if isinstance(a, torch.Tensor) and a.device.type == "cpu" and a.dtype == torch.float64 \
                    and a.is_contiguous() and a.is_pinned():
                return a
            t = torch.as_tensor(a, dtype=torch.float64).contiguous()
            return t.pin_memory()
        xt, ft = pinned(x), pinned(f)
        n_rhs = ft.shape[0] if ft.dim() == 4 else 1
        u = torch.empty(ft.shape, dtype=torch.float64, pin_memory=True)
        C = torch.empty(n_rhs, dtype=torch.float64, pin_memory=True)
        g = torch.empty(xt.shape, dtype=torch.float64, pin_memory=True) if want_grad else None
        E = (ctypes.c_double * len(E_phase))(*[float(e) for e in E_phase])
        with torch.cuda.device(self.device):
            code = self._lib.mto_run_host_async(
                self._h, xt.shape[0], ctypes.c_void_p(xt.data_ptr()), E, float(penal), n_rhs,
                ctypes.c_void_p(ft.data_ptr()), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(C.data_ptr()),
                ctypes.c_void_p(g.data_ptr()) if g is not None else None)
        _lib.check(code, "mto_run_host_async")
        self._pending.append((xt, ft, u, C, g))
        self._host_design(xt.shape[0], E_phase, penal)

    def run_host_wait(self):
        """Result of the oldest outstanding run_host_async: (u, C, g, stats),
        numpy views of pinned buffers (g None without gradients)."""
        st = SolveStats()
        with torch.cuda.device(self.device):
            code = self._lib.mto_run_host_wait(self._h, ctypes.byref(st))
        if code == _lib.ERR_STATE and not self._pending:
            _lib.check(code, "mto_run_host_wait")
        _, _, u, C, g = self._pending.pop(0)
        _lib.check(code, "mto_run_host_wait")
        return u.numpy(), C.numpy(), g.numpy() if g is not None else None, st.as_dict()

    # -- diagnostics ---------------------------------------------------------
    def level_shape(self, level):
        s = self.opts.n_coarsen - level
        return ((self.nely >> s) + 1, (self.nelx >> s) + 1, 2)

    def apply_operator(self, level, v, vcycle_operator=False):
        v = _dev_f64(v, self.device, "v")
        y = torch.empty_like(v)
        with torch.cuda.device(self.device):
            code = self._lib.mto_apply_operator(self._h, level, int(vcycle_operator), _ptr(v), _ptr(y))
        _lib.check(code, "mto_apply_operator")
        return y

    def apply_preconditioner(self, r):
        r = _dev_f64(r, self.device, "r")
        z = torch.empty_like(r)
        with torch.cuda.device(self.device):
            code = self._lib.mto_apply_preconditioner(self._h, _ptr(r), _ptr(z))
        _lib.check(code, "mto_apply_preconditioner")
        return z

    def autotune(self):
        """Time launch shapes on the device and keep the fastest per level."""
        with torch.cuda.device(self.device):
            _lib.check(self._lib.mto_autotune(self._h), "mto_autotune")
        return [self.launch_shape(l) for l in range(self.opts.n_coarsen + 1)]

    def launch_shape(self, level):
        t = ctypes.c_int()
        _lib.check(self._lib.mto_get_launch_shape(self._h, level, ctypes.byref(t)), "mto_get_launch_shape")
        return t.value

    def set_launch_shape(self, level, target_warps):
        """Warps per launch of a level's sweeps (0: one full wave; level -1: the
        float64 outer sweeps)."""
        _lib.check(self._lib.mto_set_launch_shape(self._h, level, int(target_warps)), "mto_set_launch_shape")

    def set_kernel_timing(self, enable):
        _lib.check(self._lib.mto_set_kernel_timing(self._h, int(enable)), "mto_set_kernel_timing")

    def kernel_times(self):
        avg = (ctypes.c_double * 2)()
        cnt = (ctypes.c_longlong * 2)()
        _lib.check(self._lib.mto_get_kernel_times(self._h, avg, cnt), "mto_get_kernel_times")
        return list(avg), list(cnt)

    def launch_count(self):
        c = ctypes.c_longlong()
        _lib.check(self._lib.mto_get_launch_count(self._h, ctypes.byref(c)), "mto_get_launch_count")
        return c.value

    def moduli(self):
        E = torch.empty((self.nely, self.nelx), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.mto_get_moduli(self._h, _ptr(E)), "mto_get_moduli")
        return E


class Batch:
    """Independent problems (one Mesh each, any sizes) solved by one graph launch.

    problems: list of dicts with keys mesh, x, E_phase, penal (default 3),
    f ([n_rhs][ny+1][nx+1][2] or [ny+1][nx+1][2]), optional u0.  The outputs
    (u, compliance, dcdx per problem) are device tensors owned by the batch
    and refreshed by every run().
    """

    def __init__(self, problems, want_grad=True):
        lib = _lib.load()
        self._lib = lib
        self.problems = []
        n = len(problems)
        items = (_lib.BatchItem * n)()
        ctxs = (ctypes.c_void_p * n)()
        self._keep = []
        dev = problems[0]["mesh"].device
        for i, pr in enumerate(problems):
            mesh = pr["mesh"]
            x = _dev_f64(pr["x"], mesh.device, "x")
            f = _dev_f64(pr["f"], mesh.device, "f")
            if f.dim() == 3:
                f = f.unsqueeze(0)
            u = torch.zeros_like(f) if pr.get("u0") is None else _dev_f64(pr["u0"], mesh.device, "u0").clone()
            C = torch.zeros(f.shape[0], dtype=torch.float64, device=mesh.device)
            g = torch.zeros(x.shape, dtype=torch.float64, device=mesh.device) if want_grad else None
            E = (ctypes.c_double * len(pr["E_phase"]))(*[float(e) for e in pr["E_phase"]])
            it = items[i]
            it.n_phase, it.x_dev, it.E_phase, it.penal = x.shape[0], x.data_ptr(), E, float(pr.get("penal", 3.0))
            it.n_rhs, it.f_dev, it.u_dev = f.shape[0], f.data_ptr(), u.data_ptr()
            it.compliance_dev = C.data_ptr()
            it.dcdx_dev = g.data_ptr() if g is not None else None
            ctxs[i] = mesh._h.value
            self._keep += [x, f, E]
            self.problems.append({"mesh": mesh, "u": u, "compliance": C, "dcdx": g, "x": x, "f": f})
        self._h = ctypes.c_void_p()
        with torch.cuda.device(dev):
            code = lib.mto_batch_create(ctypes.byref(self._h), n, ctxs, items, _stream(dev))
        _lib.check(code, "mto_batch_create")
        self.device = dev

    def run(self, raise_on_failure=True):
        n = len(self.problems)
        st = (SolveStats * n)()
        with torch.cuda.device(self.device):
            code = self._lib.mto_batch_run(self._h, st)
        if code not in (_lib.OK, _lib.ERR_NOT_CONVERGED, _lib.ERR_BREAKDOWN) or (
                raise_on_failure and code != _lib.OK):
            _lib.check(code, "mto_batch_run")
        return [s.as_dict() for s in st]

    def ms_last(self):
        v = ctypes.c_double()
        _lib.check(self._lib.mto_batch_time(self._h, ctypes.byref(v)), "mto_batch_time")
        return v.value

    def tune(self):
        """Launch shapes for the batch as a whole (mto_batch_tune, timed on cold
        solves); returns the chosen cap in warps per SM (0: each mesh's own
        shapes).  The problems' u tensors keep their contents."""
        w = ctypes.c_int()
        with torch.cuda.device(self.device):
            _lib.check(self._lib.mto_batch_tune(self._h, ctypes.byref(w)), "mto_batch_tune")
        return w.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.mto_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Poisson:
    """The scalar Poisson problem of Sec. 5.1 (-Laplace u = f, u = 0 on the
    boundary, nelx x nely unit Q4 elements) solved by pCGMG in one cluster
    kernel launch per solve; precision "fp64" or "mixed" (float32 V-cycle).  Nodal vectors are float64 [ny+1][nx+1] (or
    [n_rhs][ny+1][nx+1]) on the device."""

    def __init__(self, nelx, nely, n_coarsen=3, tol=1e-8, max_it=500, omega=0.6, nu1=2, nu2=2,
                 cluster_ctas=0, precision="fp64", device=None):
        lib = _lib.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        o = _lib.PoissonOpts()
        lib.mto_poisson_default_opts(ctypes.byref(o))
        o.tol, o.max_it, o.omega, o.nu1, o.nu2 = tol, max_it, omega, nu1, nu2
        o.n_coarsen, o.cluster_ctas = n_coarsen, cluster_ctas
        o.precision = {"fp64": PRECISION_FP64, "mixed": PRECISION_MIXED}[precision]
        self.opts, self.nelx, self.nely, self._lib = o, nelx, nely, lib
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            code = lib.mto_poisson_create(ctypes.byref(self._h), nelx, nely, ctypes.byref(o),
                                          self.device.index, _stream(self.device))
        _lib.check(code, "mto_poisson_create")

    @property
    def node_shape(self):
        return (self.nely + 1, self.nelx + 1)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.mto_poisson_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        nl, n0, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        la = ctypes.c_longlong()
        _lib.check(self._lib.mto_poisson_get_info(self._h, ctypes.byref(nl), ctypes.byref(n0), ctypes.byref(c),
                                                  ctypes.byref(la)), "mto_poisson_get_info")
        return {"n_levels": nl.value, "coarsest_free_dofs": n0.value, "cluster_ctas": c.value,
                "launches": la.value}

    def solve(self, f, u0=None, raise_on_failure=True):
        """Solve K u = f (f: [n_rhs?][nely+1][nelx+1] float64).  Returns (u, stats)."""
        f = _dev_f64(f, self.device, "f")
        if f.shape[-2:] != self.node_shape:
            raise ValueError(f"f must end in {self.node_shape}")
        u = torch.zeros_like(f) if u0 is None else _dev_f64(u0, self.device, "u0").clone()
        n_rhs = f.shape[0] if f.dim() == 3 else 1
        st = SolveStats()
        with torch.cuda.device(self.device):
            code = self._lib.mto_poisson_solve(self._h, n_rhs, _ptr(f), _ptr(u), ctypes.byref(st))
        if code not in (_lib.OK, _lib.ERR_NOT_CONVERGED, _lib.ERR_BREAKDOWN) or (
                raise_on_failure and code != _lib.OK):
            _lib.check(code, "mto_poisson_solve")
        d = st.as_dict()
        d["status"] = _lib.STATUS[code]
        return u, d

    def apply_operator(self, v):
        v = _dev_f64(v, self.device, "v")
        y = torch.empty_like(v)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.mto_poisson_apply_operator(self._h, _ptr(v), _ptr(y)),
                       "mto_poisson_apply_operator")
        return y

    def apply_preconditioner(self, r):
        r = _dev_f64(r, self.device, "r")
        z = torch.empty_like(r)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.mto_poisson_apply_preconditioner(self._h, _ptr(r), _ptr(z)),
                       "mto_poisson_apply_preconditioner")
        return z


class Compliance(torch.autograd.Function):
    """C(x) = sum_k f_k . u_k(x) with K(x) u_k = f_k; backward is the adjoint sensitivity.

    The compliance problem is self-adjoint (Eq. 6), so the backward needs no
    second solve: dC/dx_{e,i} = -p x^{p-1} E_i u_e^T KE u_e with the forward u.
    The backward rebuilds the operators only if the mesh was given another
    design since the forward (mesh.design_version).  When keep_u is False the
    forward keeps only a float32 copy of u (half the memory of the float64
    solution); the backward re-solves for u warm-started from it, which takes
    fewer PCG iterations than a cold solve.
    """

    @staticmethod
    def forward(ctx, x, mesh, f, E_phase, penal, keep_u=True):
        mesh.set_design(x.detach(), E_phase, penal)
        u, _ = mesh.solve(f)
        C, _ = mesh.compliance_grad(f, u, want_grad=False)
        ctx.mesh, ctx.E_phase, ctx.penal, ctx.keep_u = mesh, E_phase, penal, keep_u
        ctx.design_version = mesh.design_version
        ctx.save_for_backward(x.detach(), f, u if keep_u else u.float())
        return C.sum()

    @staticmethod
    def backward(ctx, gC):
        x, f, u = ctx.saved_tensors
        mesh = ctx.mesh
        if mesh.design_version != ctx.design_version:
            mesh.set_design(x, ctx.E_phase, ctx.penal)
            ctx.design_version = mesh.design_version
        if not ctx.keep_u:
            u, _ = mesh.solve(f, u0=u.double())
        _, g = mesh.compliance_grad(f, u, want_grad=True)
        return g * gC, None, None, None, None, None


def compliance(x, mesh, f, E_phase, penal=3.0, keep_u=True):
    """Differentiable compliance (see Compliance)."""
    return Compliance.apply(x, mesh, f, E_phase, penal, keep_u)
