"""Alternating active-phase loop (Sec. 4) over the GPU solver: constraints,
descent, and checkpoint/resume."""

import numpy as np
import pytest
import torch

from synth import load_top_edge

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda", 0)
EP = [1.0, 0.5, 0.25, 1e-9]
VOL = [0.2, 0.15, 0.1, 0.55]


def make(mto):
    from paper_2301_07457_gb300.optimize import ActivePhaseOptimizer
    mesh = mto.Mesh(64, 64, n_coarsen=3, tol=1e-8, precision="fp64")
    f = torch.from_numpy(load_top_edge(64, 64)).to(DEV)
    return ActivePhaseOptimizer(mesh, EP, VOL, f, rf=2.5)


def test_loop_keeps_constraints_and_descends(tmp_path):
    import paper_2301_07457_gb300 as mto
    opt = make(mto)
    opt.step()
    C_first = opt.history[0][2]
    opt.step()
    x = opt.x
    assert torch.allclose(x.sum(0), torch.ones_like(x[0]), atol=1e-12)
    for i, v in enumerate(VOL):
        assert abs(x[i].mean().item() - v) < 1e-8
    assert x.min().item() >= 1e-3 - 1e-12
    assert opt.history[-1][2] < C_first
    assert len(opt.history) == 12 and all(h[3] >= 0 for h in opt.history)
    # Warm starts: later sub-problems need fewer PCG iterations than the first.
    assert min(h[3] for h in opt.history[1:]) < opt.history[0][3]
    # Checkpoint after two outer iterations, continue, and compare with a
    # fresh optimiser resumed from the checkpoint.
    path = tmp_path / "ckpt.pt"
    opt.save(path)
    opt.step()
    other = make(mto)
    other.load(path)
    other.step()
    assert torch.equal(other.x, opt.x)
    assert other.history[-1][2] == opt.history[-1][2]
    opt.mesh.close()
    other.mesh.close()
