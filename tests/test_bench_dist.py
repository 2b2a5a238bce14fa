"""Multi-rank host logic of bench.py on CPU ranks (gloo, world size 2).

Every rank solves its own problems (no collective on the data path); only
the timing is reduced: the job's time is the slowest rank's, and the value
counts every rank's solves.
"""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 100.0 + 50.0 * rank  # rank 1 is slower
    ms = bench.max_over_ranks(ms_local, world, "cpu")
    out[rank] = (ms, bench.job_value(world, 5, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    port = free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0] == out[1]
    ms, value = out[0]
    assert ms == 150.0
    assert value == pytest.approx(2 * 5 / 0.150)


def replica_worker(rank, world, port, out):
    # Each rank solves its own replica of the seeded workload (the CPU oracle
    # stands in for the device solve); nothing crosses ranks on the data path.
    # The all_gather below is the test's, to compare the ranks' answers.
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import solver
    from synth import dirichlet_design, load_top_edge
    n = 32
    x, f = dirichlet_design(n, n, 4, 0), load_top_edge(n, n)
    r = solver.solve_pcgmg(n, n, x, [1.0, 0.5, 0.25, 1e-9], 3.0, f, n_coarsen=2, tol=1e-10)
    mine = torch.tensor([float(f.ravel() @ r["u"].ravel()), float(r["iters"])], dtype=torch.float64)
    got = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(got, mine)
    out[rank] = [tuple(g.tolist()) for g in got]
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_solve_identical_replicas():
    port = free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(replica_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0] == out[1]
    (c0, it0), (c1, it1) = out[0]
    assert c0 == c1 and it0 == it1
    # The same answer as one process alone.
    sys.path.insert(0, ROOT)
    from oracle import solver
    from synth import dirichlet_design, load_top_edge
    n = 32
    x, f = dirichlet_design(n, n, 4, 0), load_top_edge(n, n)
    r = solver.solve_pcgmg(n, n, x, [1.0, 0.5, 0.25, 1e-9], 3.0, f, n_coarsen=2, tol=1e-10)
    assert c0 == float(f.ravel() @ r["u"].ravel()) and it0 == r["iters"]


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_value(1, 4, 2000.0) == 2.0


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")

    class Args:
        size, n_coarsen, warmup, steps, gpus, gamma = 2048, 7, 3, 5, 2, 1

    called = []
    monkeypatch.setattr(bench, "oracle_run", lambda *a, **k: called.append(1))
    assert bench.run_reference(Args()) == 0
    assert not called


def test_cpu_sample_completes_the_solve_at_the_measured_iteration_time():
    sys.path.insert(0, ROOT)
    import bench
    d = {"setup_s": 20.0, "start_s": 0.5, "iter_s": [2.0, 2.2]}
    assert bench.cpu_sample_value(d, 32) == 1.0 / (20.0 + 0.5 + 32 * 2.1)
