"""Alternating active-phase compliance minimisation driving the pCGMG solver.

Sec. 4 describes the loop the solver serves: an optimality-criteria update,
one pair of active phases (a, b) at a time in Gauss-Seidel fashion, each
binary sub-problem re-solving K(alpha) U = F, computing the sensitivities,
filtering them and updating the two active fractions.  The paper takes the
sub-problem algorithm from Tavakoli & Mohseni (2014) without printing it; the
steps below are this library's reading of it:

  * pairs (a, b), a < b over all phases (void included): 6 sub-problems per
    outer iteration for 4 phases, each with one warm-started solve;
  * in a sub-problem only x_a and x_b move and their sum s = x_a + x_b is kept
    per element, so moving mass from b to a changes the compliance at rate
    d_e = dC/dx_a - dC/dx_b;
  * d is smoothed by the distance-weighted sensitivity filter of radius rf
    (element units): d_e <- sum_f H_ef x_f d_f / (max(x_e, 1e-3) sum_f H_ef),
    H_ef = max(0, rf - |c_e - c_f|), with x = x_a;
  * optimality-criteria step with move limit m and damping eta:
    x_a <- clip(x_a (max(0, -d) / lam)^eta, max(eps, x_a - m), min(s - eps, x_a + m)),
    with lam found on the device (a bracketing search in log(lam)) so that
    the phase-a volume equals V_a; then x_b = s - x_a;
  * stopping rule (Table 2 gives a tolerance as the optimiser's only stopping
    criterion): stop after the outer iteration in which no phase fraction of
    any element changed by more than tol.

The solve and the sensitivities run in libmto; the filter (float32) and the
OC step are elementwise/convolution tensor operations on the device.  Checkpoints hold the
design, the displacement (the next warm start), the iteration counter and the
history.
"""

import math

import torch
import torch.nn.functional as F

from . import Mesh  # noqa: F401  (type of the `mesh` argument)


def filter_kernel(rf, device, dtype=torch.float64):
    """Weights H(d) = max(0, rf - d) on the integer offsets |d| < rf, as a conv kernel."""
    r = int(math.ceil(rf)) - 1
    ax = torch.arange(-r, r + 1, device=device, dtype=dtype)
    d = torch.sqrt(ax[:, None] ** 2 + ax[None, :] ** 2)
    return torch.clamp(rf - d, min=0.0)[None, None]


def filter_sensitivity(d, x, H):
    """Distance-weighted sensitivity filter (see module docstring); d, x: [nely][nelx].

    The filter is a smoothing heuristic of the optimiser, so it runs in float32
    (the result is returned in d's dtype).
    """
    pad = H.shape[-1] // 2
    H32 = H.to(torch.float32)
    num = F.conv2d((x * d).to(torch.float32)[None, None], H32, padding=pad)[0, 0]
    den = F.conv2d(torch.ones_like(x, dtype=torch.float32)[None, None], H32, padding=pad)[0, 0]
    return (num / (torch.clamp(x.to(torch.float32), min=1e-3) * den)).to(d.dtype)


def oc_update(xa, s, d, target, move=0.2, eta=0.5, eps=1e-3, rounds=10, candidates=16):
    """Optimality-criteria step for phase a of a pair with fixed per-element sum s.

    Returns new x_a with mean(x_a) == target (to the search's accuracy) and
    eps <= x_a <= s - eps where s > 2 eps (elements with s <= 2 eps keep s/2).

    The multiplier is searched on log(lam) in [-60, 60], all on the device: the
    volume is non-increasing in lam, so each round evaluates it at `candidates`
    + 1 points of the current bracket at once and keeps the sub-interval where
    it crosses the target (10 rounds of 16: a bracket of 1.1e-10 in log(lam)).
    """
    lo_b = torch.clamp(xa - move, min=eps)
    hi_b = torch.clamp(torch.minimum(xa + move, s - eps), min=eps)
    lo_b = torch.minimum(lo_b, hi_b)
    base = xa * torch.clamp(-d, min=0.0) ** eta  # x(lam) = base * lam^-eta before the bounds
    frac = torch.linspace(0.0, 1.0, candidates + 1, dtype=xa.dtype, device=xa.device)
    lo = torch.tensor(-60.0, dtype=xa.dtype, device=xa.device)
    hi = torch.tensor(60.0, dtype=xa.dtype, device=xa.device)
    flat_b, flat_lo, flat_hi = base.reshape(1, -1), lo_b.reshape(1, -1), hi_b.reshape(1, -1)
    for _ in range(rounds):
        grid = lo + (hi - lo) * frac
        xs = torch.minimum(torch.maximum(flat_b * torch.exp(-eta * grid)[:, None], flat_lo), flat_hi)
        too_big = (xs.mean(dim=1) > target).sum()
        j = torch.clamp(too_big - 1, 0, candidates - 1)
        lo, hi = grid[j], grid[j + 1]
    lam = 0.5 * (lo + hi)
    return torch.minimum(torch.maximum(base * torch.exp(-eta * lam), lo_b), hi_b)


class ActivePhaseOptimizer:
    """Multi-material compliance minimisation with the pCGMG solver of `mesh`.

    volumes: target volume fraction of every phase (void included), summing
    to 1.  The design starts uniform at those fractions.
    """

    def __init__(self, mesh, E_phase, volumes, f, penal=3.0, rf=8.0, move=0.2, eta=0.5, eps=1e-3):
        self.mesh, self.E_phase, self.penal = mesh, list(E_phase), float(penal)
        self.volumes = [float(v) for v in volumes]
        if abs(sum(self.volumes) - 1.0) > 1e-9 or len(self.volumes) != len(self.E_phase):
            raise ValueError("one volume fraction per phase, summing to 1")
        dev = mesh.device
        self.f = f.to(dev)
        n_phase = len(self.E_phase)
        self.x = torch.stack([torch.full((mesh.nely, mesh.nelx), v, dtype=torch.float64, device=dev)
                              for v in self.volumes])
        self.u = torch.zeros_like(self.f)
        self.H = filter_kernel(rf, dev)
        self.move, self.eta, self.eps = move, eta, eps
        self.pairs = [(a, b) for a in range(n_phase) for b in range(a + 1, n_phase)]
        self.iteration = 0
        self.history = []  # (outer iteration, pair, compliance, PCG iterations)
        self.change = float("inf")  # largest fraction change of the last outer iteration

    def subproblem(self, a, b):
        mesh = self.mesh
        mesh.set_design(self.x, self.E_phase, self.penal)
        self.u, st = mesh.solve(self.f, u0=self.u)
        C, g = mesh.compliance_grad(self.f, self.u)
        d = filter_sensitivity(g[a] - g[b], self.x[a], self.H)
        s = self.x[a] + self.x[b]
        xa = oc_update(self.x[a], s, d, self.volumes[a], self.move, self.eta, self.eps)
        self.x[a] = xa
        self.x[b] = s - xa
        return C.sum().item(), st["iters"]

    def step(self):
        """One outer iteration: every pair once; returns the last compliance."""
        C = None
        x_before = self.x.clone()
        for a, b in self.pairs:
            C, it = self.subproblem(a, b)
            self.history.append((self.iteration, (a, b), C, it))
        self.change = (self.x - x_before).abs().max().item()
        self.iteration += 1
        return C

    def run(self, n_outer):
        for _ in range(n_outer):
            self.step()
        return self.history

    def run_until(self, tol, max_outer, max_seconds=None):
        """Outer iterations until one changes no fraction by more than tol, at
        most max_outer of them and (if given) until max_seconds of wall time
        have passed; returns why it stopped: "tol", "outer cap" or "time"."""
        import time
        t0 = time.perf_counter()
        for _ in range(max_outer):
            self.step()
            if self.change <= tol:
                return "tol"
            if max_seconds is not None and time.perf_counter() - t0 > max_seconds:
                return "time"
        return "outer cap"

    def state_dict(self):
        return {"x": self.x.cpu(), "u": self.u.cpu(), "iteration": self.iteration,
                "history": list(self.history), "volumes": self.volumes, "E_phase": self.E_phase,
                "penal": self.penal, "change": self.change}

    def load_state_dict(self, sd):
        dev = self.mesh.device
        self.x = sd["x"].to(dev)
        self.u = sd["u"].to(dev)
        self.iteration = sd["iteration"]
        self.history = list(sd["history"])
        self.change = sd.get("change", float("inf"))

    def save(self, path):
        torch.save(self.state_dict(), path)

    def load(self, path):
        self.load_state_dict(torch.load(path, weights_only=False))
