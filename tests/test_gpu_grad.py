"""Differentiable compliance (autograd Function over libmto) on the GPU.

Paper: Eq. 6 (compliance), Sec. 4 (sensitivities follow the solve).  The
backward is the self-adjoint sensitivity dC/dx_{e,i} = -p x^{p-1} E_i u_e^T KE u_e.

Checks: (1) against the oracle's gradient at 16 x 16 (1e-10 relative at solver
tolerance 1e-12); (2) against central finite differences (h = 1e-6) on 32
seeded elements of a 512 x 512 mesh with five phases.  The finite differences
use the variational energy Pi(u) = 2 f.u - u^T K u, whose error is quadratic
in the solve error (plain f.u has an error of order tol * C / h, larger than a
single element's gradient at this size); re-solves are warm-started at
tolerance 1e-12.  At this size C ~ 4e6 while 2 h times one element's gradient
is ~1e-5, so the two energies of a difference quotient must agree to ~1e-16
of C.  The oracle therefore evaluates them on nodal differences (strain-sized
numbers instead of displacements, see element_energy_relative) and sums the
terms of both energies in one exact sum (math.fsum), so that neither total is
rounded.  The remaining noise is measured, not guessed: Pi is evaluated after
two solves of the unperturbed problem from different warm starts (both at
tolerance 1e-12, so their exact energies agree to the square of the solve
error) and their spread s sets the noise scale s / (2h) of a difference
quotient.  The bar is |fd - g| <= 1e-4 |g| + 4 s / (2h) for every pick.
"""

import numpy as np
import pytest
import torch

from oracle import fem, sensitivity, solver
from synth import dirichlet_design, load_top_edge, uniform01

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
EP5 = [1.0, 0.7, 0.5, 0.3, 0.15]


@pytest.fixture(scope="module")
def mto():
    import paper_2301_07457_gb300 as m
    return m


def test_autograd_matches_oracle_gradient_16(mto):
    n = 16
    xn = dirichlet_design(n, n, 5, seed=2)
    fn = load_top_edge(n, n)
    mesh = mto.Mesh(n, n, n_coarsen=2, tol=1e-12, max_it=200)
    x = torch.from_numpy(xn).to(DEV).requires_grad_(True)
    C = mto.compliance(x, mesh, torch.from_numpy(fn).to(DEV), EP5, 3.0)
    C.backward()
    ud = solver.solve_direct(n, n, xn, EP5, 3.0, fn)
    C_ref, g_ref = solver.compliance_and_gradient(n, n, xn, EP5, 3.0, fn, ud)
    assert abs(C.item() - C_ref) / C_ref < 1e-10
    g = x.grad.cpu().numpy()
    assert np.abs(g - g_ref).max() <= 1e-10 * np.abs(g_ref).max()
    # keep_u=False recomputes u in the backward: same gradient.
    x2 = torch.from_numpy(xn).to(DEV).requires_grad_(True)
    mto.compliance(x2, mesh, torch.from_numpy(fn).to(DEV), EP5, 3.0, keep_u=False).backward()
    assert torch.allclose(x2.grad, x.grad, rtol=1e-9, atol=1e-14)
    mesh.close()


def test_gradient_against_central_differences_512(mto):
    n = 512
    xn = dirichlet_design(n, n, 5, seed=2)
    fn = load_top_edge(n, n)
    f = torch.from_numpy(fn).to(DEV)
    mesh = mto.Mesh(n, n, n_coarsen=5, tol=1e-12, max_it=500)
    x = torch.from_numpy(xn).to(DEV).requires_grad_(True)
    C = mto.compliance(x, mesh, f, EP5, 3.0)
    C.backward()
    grad = x.grad.cpu().numpy()
    KE = fem.element_stiffness(0.3)
    # 32 seeded (phase, element) picks.
    u_pick = uniform01(2, np.arange(64, dtype=np.uint64))
    picks = [(int(u_pick[2 * k] * 5) % 5, int(u_pick[2 * k + 1] * n * n) % (n * n)) for k in range(32)]
    mesh.set_design(x.detach(), EP5, 3.0)
    u0, _ = mesh.solve(f)
    h = 1e-6

    def energy_terms(xp, u_start):
        mesh.set_design(xp, EP5, 3.0)
        u, st = mesh.solve(f, u0=u_start)
        assert st["rel_res_true"] <= 1e-11, st
        E = fem.simp_moduli(xp.cpu().numpy(), EP5, 3.0)
        return sensitivity.variational_energy_terms(n, n, E, KE, fn, u.cpu().numpy())

    # Measured noise of an energy difference (two solves of the same problem).
    spread = abs(sensitivity.energy_difference(energy_terms(x.detach(), u0),
                                               energy_terms(x.detach(), 0.999 * u0)))
    floor = 4 * spread / (2 * h)
    worst, detail = 0.0, []
    for i, e in picks:
        xp = x.detach().clone()
        xm = x.detach().clone()
        xp.view(5, -1)[i, e] += h
        xm.view(5, -1)[i, e] -= h
        step = (xp.view(5, -1)[i, e] - xm.view(5, -1)[i, e]).item()  # 2h as rounded
        fd = sensitivity.energy_difference(energy_terms(xp, u0), energy_terms(xm, u0)) / step
        g = grad.reshape(5, -1)[i, e]
        err = abs(fd - g) / (1e-4 * abs(g) + floor)
        detail.append((i, e, g, fd))
        worst = max(worst, err)
    rel = sorted(abs(fd - g) / abs(g) for _, _, g, fd in detail)
    print(f"FD 512^2: spread {spread:.3e}, floor {floor:.3e}, worst bar use {worst:.3f}, "
          f"median rel {rel[len(rel) // 2]:.2e}, max rel {rel[-1]:.2e}")
    assert worst < 1.0, (worst, floor, spread, rel[len(rel) // 2], detail[:4])
    mesh.close()


def test_backward_reuses_the_forward_design_and_warm_starts(mto):
    n = 64
    xn = dirichlet_design(n, n, 5, seed=9)
    fn = load_top_edge(n, n)
    f = torch.from_numpy(fn).to(DEV)
    mesh = mto.Mesh(n, n, n_coarsen=3, tol=1e-10, max_it=200)
    # keep_u=True: the mesh still holds the forward's design, so the backward
    # launches only the compliance dot and the sensitivity kernel (no set-up).
    x = torch.from_numpy(xn).to(DEV).requires_grad_(True)
    C = mto.compliance(x, mesh, f, EP5, 3.0)
    l0 = mesh.launch_count()
    C.backward()
    assert mesh.launch_count() - l0 == 2
    ud = solver.solve_direct(n, n, xn, EP5, 3.0, fn)
    _, g_ref = solver.compliance_and_gradient(n, n, xn, EP5, 3.0, fn, ud)
    np.testing.assert_allclose(x.grad.cpu().numpy(), g_ref, rtol=1e-7, atol=1e-9 * np.abs(g_ref).max())
    # keep_u=False: the backward re-solves from the float32 copy of u and
    # needs fewer iterations than the forward's cold solve.
    x2 = torch.from_numpy(xn).to(DEV).requires_grad_(True)
    C2 = mto.compliance(x2, mesh, f, EP5, 3.0, keep_u=False)
    cold = mesh.last_solve_stats["iters"]
    C2.backward()
    warm = mesh.last_solve_stats["iters"]
    assert warm < cold, (warm, cold)
    assert torch.allclose(x2.grad, x.grad, rtol=1e-8, atol=1e-12 * x.grad.abs().max().item())
    # Another design set between forward and backward: the backward rebuilds
    # the operators of its own design.
    x3 = torch.from_numpy(xn).to(DEV).requires_grad_(True)
    C3 = mto.compliance(x3, mesh, f, EP5, 3.0)
    mesh.set_design(torch.from_numpy(dirichlet_design(n, n, 5, seed=10)).to(DEV), EP5, 3.0)
    C3.backward()
    assert torch.allclose(x3.grad, x.grad, rtol=1e-12, atol=0.0)
    mesh.close()
