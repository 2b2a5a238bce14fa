"""Pins of compliance and sensitivities (Eq. 6, Sec. 4) and of the bf16 rounding."""

import numpy as np
import pytest

from oracle import fem, precision, sensitivity, solver
from synth import dirichlet_design, load_right_edge, load_top_edge

EP = [1.0, 0.5, 0.25, 1e-9]


def test_energy_identity():
    nelx, nely = 12, 8
    x = dirichlet_design(nelx, nely, 4, seed=11)
    f = load_top_edge(nelx, nely)
    u = solver.solve_direct(nelx, nely, x, EP, 3.0, f)
    E = fem.simp_moduli(x, EP, 3.0)
    w = sensitivity.element_energy(nelx, nely, fem.element_stiffness(0.3), u)
    assert sensitivity.compliance(f, u) == pytest.approx(sensitivity.energy_sum(E, w), rel=1e-10)
    assert sensitivity.compliance(f, u) > 0


def test_gradient_matches_central_differences():
    nelx, nely = 6, 4
    x = dirichlet_design(nelx, nely, 4, seed=12)
    f = load_top_edge(nelx, nely) + 0.5 * load_right_edge(nelx, nely)
    u = solver.solve_direct(nelx, nely, x, EP, 3.0, f)
    C, g = solver.compliance_and_gradient(nelx, nely, x, EP, 3.0, f, u)
    h = 1e-6
    rng = np.random.default_rng(0)
    for _ in range(8):
        i, jy, ix = rng.integers(0, 3), rng.integers(0, nely), rng.integers(0, nelx)
        xp, xm = x.copy(), x.copy()
        xp[i, jy, ix] += h
        xm[i, jy, ix] -= h
        Cp = sensitivity.compliance(f, solver.solve_direct(nelx, nely, xp, EP, 3.0, f))
        Cm = sensitivity.compliance(f, solver.solve_direct(nelx, nely, xm, EP, 3.0, f))
        fd = (Cp - Cm) / (2 * h)
        assert g[i, jy, ix] == pytest.approx(fd, rel=1e-6, abs=1e-9 * abs(C))
    assert np.all(g[:3] <= 0)  # adding stiff material never raises compliance


def test_gradient_formula_special_case():
    # One element, one phase fully present: dC/dx = -p E w.
    x = np.zeros((2, 1, 1)); x[0] = 1.0
    w = np.array([[2.0]])
    g = sensitivity.compliance_gradient(x, [3.0, 1.0], 3.0, w)
    assert g[0, 0, 0] == pytest.approx(-3 * 3.0 * 2.0)
    assert g[1, 0, 0] == 0.0


def test_bf16_rounding():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    # float32-exact inputs: torch's float32 -> bfloat16 cast is round-to-nearest-even.
    v = rng.standard_normal(10000).astype(np.float32).astype(np.float64) * 10.0 ** rng.integers(-12, 3, 10000)
    v = v.astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(precision.round_to_bf16(v), ref)
    # Ties go to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7.
    assert precision.round_to_bf16(1 + 2.0**-8) == 1.0
    assert precision.round_to_bf16(1 + 3 * 2.0**-8) == 1 + 2.0**-6
    # Just above a tie rounds up (direct rounding from float64, no float32 step).
    assert precision.round_to_bf16(1 + 2.0**-8 + 2.0**-40) == 1 + 2.0**-7
    assert precision.round_to_bf16(0.0) == 0.0


def test_relative_element_energy_is_the_element_energy():
    # Eq. 7: a rigid translation carries no strain, so measuring the nodal
    # values from the element's first node changes nothing in exact
    # arithmetic; on a field shifted by a large translation the relative form
    # keeps its accuracy while the plain form loses digits.
    nelx, nely = 10, 6
    KE = fem.element_stiffness(0.3)
    u = np.random.default_rng(3).standard_normal((nely + 1, nelx + 1, 2))
    w_plain = sensitivity.element_energy(nelx, nely, KE, u)
    w_rel = sensitivity.element_energy_relative(nelx, nely, KE, u)
    np.testing.assert_allclose(w_rel, w_plain, rtol=1e-12, atol=1e-13)
    shifted = u + np.array([3e7, -5e7])
    w_shift = sensitivity.element_energy_relative(nelx, nely, KE, shifted)
    np.testing.assert_allclose(w_shift, w_plain, rtol=1e-6, atol=1e-7)
    assert np.all(w_rel >= -1e-12)  # KE is positive semi-definite


def test_variational_energy_is_stationary_at_the_solution():
    # Pi(u) = 2 f.u - u^T K u equals the compliance at K u = f (Eq. 6) and
    # falls by exactly delta^T K delta away from it (checked against the
    # assembled K, a separate code path from the element loop).
    nelx, nely = 12, 8
    x = dirichlet_design(nelx, nely, 4, seed=21)
    f = load_top_edge(nelx, nely) + 0.4 * load_right_edge(nelx, nely)
    E = fem.simp_moduli(x, EP, 3.0)
    KE = fem.element_stiffness(0.3)
    u = solver.solve_direct(nelx, nely, x, EP, 3.0, f)
    pi_star = float(np.sum(sensitivity.variational_energy_terms(nelx, nely, E, KE, f, u)))
    assert pi_star == pytest.approx(sensitivity.compliance(f, u), rel=1e-12)
    K = fem.assemble(nelx, nely, E, KE)
    free = fem.free_dofs(nelx, nely, fem.BOTTOM)
    rng = np.random.default_rng(22)
    for scale in (1e-3, 1e-1):
        delta = np.zeros(u.size)
        delta[free] = scale * rng.standard_normal(free.size) * np.abs(u).max()
        ud = u + delta.reshape(u.shape)
        pi = float(np.sum(sensitivity.variational_energy_terms(nelx, nely, E, KE, f, ud)))
        drop = float(delta @ (K @ delta))
        assert pi_star - pi == pytest.approx(drop, rel=1e-8)


def test_energy_difference_sums_exactly():
    a = np.array([1e16, 1.0, -1e16, 3.0])
    b = np.array([2.0, 1e-20])
    assert sensitivity.energy_difference(a, b) == 2.0 - 1e-20
    assert sensitivity.energy_difference(a, a) == 0.0
