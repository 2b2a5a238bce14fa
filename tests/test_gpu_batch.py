"""Device-side PCG loop, batched graphs and the launch-shape tuner (GPU).

The batch graph runs the same kernels as single solves (deterministic
reductions, same launch shapes), so its results must equal theirs exactly;
the device-side loop and the host-polled loop likewise.
"""

import numpy as np
import pytest
import torch

from oracle import solver
from synth import dirichlet_design, load_right_edge, load_top_edge

pytestmark = pytest.mark.gpu
EP = [1.0, 0.5, 0.25, 1e-9]
DEV = torch.device("cuda", 0)


@pytest.fixture(scope="module")
def mto():
    import paper_2301_07457_gb300 as m
    return m


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_device_loop_equals_polled_loop(mto, prec):
    nelx, nely = 128, 96
    x = to_dev(dirichlet_design(nelx, nely, 4, seed=21))
    f = to_dev(np.stack([load_top_edge(nelx, nely), load_right_edge(nelx, nely)]))
    tol = 1e-10 if prec == "fp64" else 1e-8
    a = mto.Mesh(nelx, nely, n_coarsen=3, precision=prec, tol=tol)
    a.set_design(x, EP, 3.0)
    ua, sa = a.solve(f)
    b = mto.Mesh(nelx, nely, n_coarsen=3, precision=prec, tol=tol)
    b.set_kernel_timing(True)  # forces the host-polled loop
    b.set_design(x, EP, 3.0)
    ub, sb = b.solve(f)
    assert sa["iters"] == sb["iters"]
    assert torch.equal(ua, ub)
    times, counts = b.kernel_times()
    assert counts[0] > 0 and times[0] > 0
    assert a.launch_count() > 0
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_equals_individual_solves(mto, prec):
    sizes = [(64, 64, 2), (128, 64, 3), (96, 160, 3), (256, 256, 4)]
    tol = 1e-10 if prec == "fp64" else 1e-8
    problems, refs = [], []
    for k, (nx, ny, nc) in enumerate(sizes):
        x = to_dev(dirichlet_design(nx, ny, 4, seed=100 + k))
        F = to_dev(np.stack([load_top_edge(nx, ny), load_right_edge(nx, ny)]))
        single = mto.Mesh(nx, ny, n_coarsen=nc, precision=prec, tol=tol)
        single.set_design(x, EP, 3.0)
        u, st = single.solve(F)
        C, g = single.compliance_grad(F, u)
        refs.append((u, C, g, st))
        single.close()
        problems.append({"mesh": mto.Mesh(nx, ny, n_coarsen=nc, precision=prec, tol=tol),
                         "x": x, "E_phase": EP, "penal": 3.0, "f": F})
    batch = mto.Batch(problems)
    for run in range(2):  # a second cold launch of the same graph gives the same answer
        for pr in batch.problems:
            pr["u"].zero_()  # u is the warm start of the next run
        stats = batch.run()
        for pr, (u, C, g, st), bst in zip(batch.problems, refs, stats):
            assert torch.equal(pr["u"], u)
            assert torch.equal(pr["compliance"], C)
            assert torch.equal(pr["dcdx"], g)
            assert bst["iters"] == st["iters"] and bst["converged"] == 1
    assert batch.ms_last() > 0
    # Warm start from the converged solutions: no iterations.
    assert all(s["iters"] == 0 for s in batch.run())
    batch.close()
    for pr in problems:
        pr["mesh"].close()


def test_batch_solution_matches_oracle(mto):
    nx, ny = 96, 64
    xn = dirichlet_design(nx, ny, 4, seed=7)
    fn = load_top_edge(nx, ny)
    mesh = mto.Mesh(nx, ny, n_coarsen=3, precision="fp64", tol=1e-10)
    batch = mto.Batch([{"mesh": mesh, "x": to_dev(xn), "E_phase": EP, "f": to_dev(fn)}])
    batch.run()
    ud = solver.solve_direct(nx, ny, xn, EP, 3.0, fn)
    u = batch.problems[0]["u"][0].cpu().numpy()
    assert np.linalg.norm(u - ud) / np.linalg.norm(ud) < 1e-8
    C_ref, g_ref = solver.compliance_and_gradient(nx, ny, xn, EP, 3.0, fn, ud)
    assert abs(batch.problems[0]["compliance"][0].item() - C_ref) / C_ref < 1e-9
    batch.close()
    mesh.close()


def test_batch_rejects_repeated_context(mto):
    from paper_2301_07457_gb300 import MtoError
    mesh = mto.Mesh(32, 32, n_coarsen=2)
    x = to_dev(dirichlet_design(32, 32, 4, seed=1))
    f = to_dev(load_top_edge(32, 32))
    with pytest.raises(MtoError):
        mto.Batch([{"mesh": mesh, "x": x, "E_phase": EP, "f": f}] * 2)
    mesh.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_autotune_keeps_results(mto, prec):
    nx = ny = 256
    x = to_dev(dirichlet_design(nx, ny, 4, seed=5))
    f = to_dev(load_top_edge(nx, ny))
    m = mto.Mesh(nx, ny, n_coarsen=4, precision=prec, tol=1e-8)
    m.set_design(x, EP, 3.0)
    u0, s0 = m.solve(f)
    shapes = m.autotune()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # 0 = one full wave of the kernel (default), else warps per launch.
    assert all(s == 0 or (s % sms == 0 and 4 <= s // sms <= 128) for s in shapes)
    u1, s1 = m.solve(f)
    # Launch shapes change summation order only: same convergence, same answer.
    assert abs(s1["iters"] - s0["iters"]) <= 1
    assert (u1 - u0).norm().item() <= 1e-6 * u0.norm().item()
    m.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_tune(mto, prec):
    # mto_batch_tune times shared launch-shape caps over the whole batch and
    # recaptures its graph with the fastest: the answers change only in the
    # order of partial sums, the caller's u comes back unchanged, and each
    # mesh keeps its own shapes for its own solves.
    sizes = [(64, 64, 2), (128, 64, 3), (256, 256, 4), (256, 128, 4)]
    tol = 1e-10 if prec == "fp64" else 1e-8
    problems, own = [], []
    for k, (nx, ny, nc) in enumerate(sizes):
        x = to_dev(dirichlet_design(nx, ny, 4, seed=200 + k))
        F = to_dev(np.stack([load_top_edge(nx, ny), load_right_edge(nx, ny)]))
        m = mto.Mesh(nx, ny, n_coarsen=nc, precision=prec, tol=tol)
        m.set_design(x, EP, 3.0)
        own.append((m.solve(F)[0], [m.launch_shape(l) for l in range(-1, nc + 1)]))
        problems.append({"mesh": m, "x": x, "E_phase": EP, "penal": 3.0, "f": F})
    batch = mto.Batch(problems)
    for pr in batch.problems:
        pr["u"].zero_()
    st0 = batch.run()
    U0 = [pr["u"].clone() for pr in batch.problems]
    for pr, u in zip(batch.problems, U0):
        pr["u"].copy_(0.5 * u)  # a warm start that the tuner must leave in place
    w = batch.tune()
    assert w in (0, 16, 8, 6, 4, 3, 2)
    for pr, u in zip(batch.problems, U0):
        assert torch.equal(pr["u"], 0.5 * u)
    for pr in batch.problems:
        pr["u"].zero_()
    st1 = batch.run()
    for pr, u0, a, b in zip(batch.problems, U0, st0, st1):
        assert b["converged"] == 1 and abs(a["iters"] - b["iters"]) <= 1
        assert (pr["u"] - u0).norm().item() <= 1e-6 * u0.norm().item()
    # Each mesh's own solve: its own shapes, the same answer as before.
    for pr, (u_own, shapes) in zip(problems, own):
        m = pr["mesh"]
        assert [m.launch_shape(l) for l in range(-1, m.opts.n_coarsen + 1)] == shapes
        m.set_design(pr["x"], EP, 3.0)
        assert torch.equal(m.solve(pr["f"])[0], u_own)
    batch.close()
    for pr in problems:
        pr["mesh"].close()
