"""Harness pieces of the active-phase optimiser that need no GPU (torch on CPU)."""

import math

import pytest

torch = pytest.importorskip("torch")

from paper_2301_07457_gb300.optimize import filter_kernel, filter_sensitivity, oc_update  # noqa: E402


def test_filter_kernel_weights():
    H = filter_kernel(2.0, "cpu")[0, 0]
    assert H.shape == (3, 3)
    assert H[1, 1].item() == pytest.approx(2.0)
    assert H[0, 1].item() == pytest.approx(1.0)
    assert H[0, 0].item() == pytest.approx(2.0 - math.sqrt(2.0))


def test_filter_keeps_constant_fields_and_symmetry():
    H = filter_kernel(3.0, "cpu")
    x = torch.full((12, 20), 0.4, dtype=torch.float64)
    d = torch.full((12, 20), -2.5, dtype=torch.float64)
    out = filter_sensitivity(d, x, H)
    assert torch.allclose(out, d, rtol=1e-6)
    g = torch.rand(12, 20, dtype=torch.float64)
    sym = g + g.flip(1)
    fs = filter_sensitivity(sym, x, H)
    assert torch.allclose(fs, fs.flip(1), rtol=1e-5)


def test_oc_update_meets_volume_bounds_and_move_limit():
    torch.manual_seed(0)
    xa = torch.rand(30, 40, dtype=torch.float64) * 0.5 + 0.1
    s = xa + torch.rand(30, 40, dtype=torch.float64) * 0.3
    d = -torch.rand(30, 40, dtype=torch.float64)
    target = xa.mean().item() * 0.97
    new = oc_update(xa, s, d, target, move=0.2, eta=0.5, eps=1e-3)
    assert abs(new.mean().item() - target) < 1e-9
    assert (new >= 1e-3 - 1e-15).all() and (new <= s - 1e-3 + 1e-15).all()
    assert ((new - xa).abs() <= 0.2 + 1e-15).all()
    # Larger benefit (more negative d) gets at least as much material.
    d2 = d.clone()
    d2[0, 0] = -10.0
    new2 = oc_update(xa, s, d2, target)
    assert new2[0, 0] >= new[0, 0] - 1e-12


class OracleMesh:
    """Stands in for Mesh on the CPU: the oracle's direct solve and gradient."""

    def __init__(self, nelx, nely):
        self.nelx, self.nely, self.device = nelx, nely, torch.device("cpu")

    def set_design(self, x, E_phase, penal):
        self.x, self.E_phase, self.penal = x.numpy().copy(), list(E_phase), penal

    def solve(self, f, u0=None):
        from oracle import solver
        u = solver.solve_direct(self.nelx, self.nely, self.x, self.E_phase, self.penal, f.numpy())
        return torch.from_numpy(u), {"iters": 0}

    def compliance_grad(self, f, u):
        from oracle import solver
        C, g = solver.compliance_and_gradient(self.nelx, self.nely, self.x, self.E_phase,
                                              self.penal, f.numpy(), u.numpy())
        return torch.tensor([C]), torch.from_numpy(g)


def test_stopping_rule_of_the_outer_loop():
    # Table 2 moduli and volume fractions on a 12 x 8 wall: the loop stops
    # after the first outer iteration that moves no fraction by more than tol.
    from paper_2301_07457_gb300.optimize import ActivePhaseOptimizer
    from synth import load_top_edge
    E, V = [9.0, 3.0, 1.0, 1e-9], [0.16, 0.08, 0.08, 0.68]
    f = torch.from_numpy(load_top_edge(12, 8))
    opt = ActivePhaseOptimizer(OracleMesh(12, 8), E, V, f, rf=1.5)
    assert opt.run_until(tol=2e-2, max_outer=60) == "tol"
    changes = []
    ref = ActivePhaseOptimizer(OracleMesh(12, 8), E, V, f, rf=1.5)
    for _ in range(opt.iteration):
        ref.step()
        changes.append(ref.change)
    assert changes[-1] <= 2e-2 and all(c > 2e-2 for c in changes[:-1])
    assert torch.equal(ref.x, opt.x)
    # A tolerance it cannot meet: exactly max_outer outer iterations.
    opt2 = ActivePhaseOptimizer(OracleMesh(12, 8), E, V, f, rf=1.5)
    assert opt2.run_until(tol=-1.0, max_outer=3) == "outer cap"
    assert opt2.iteration == 3 and len(opt2.history) == 18
    # A wall-time budget ends the loop after the outer iteration that exceeds it.
    opt3 = ActivePhaseOptimizer(OracleMesh(12, 8), E, V, f, rf=1.5)
    assert opt3.run_until(tol=-1.0, max_outer=50, max_seconds=0.0) == "time"
    assert opt3.iteration == 1
