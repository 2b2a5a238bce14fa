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
