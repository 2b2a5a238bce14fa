#!/usr/bin/env python
"""Benchmark of the pCGMG solve on GB300: one JSON line on stdout.

Step = one pass of the whole hot path on the 2048 x 2048 Q4 square wall:
mto_set_design (moduli, coarse operators, coarsest inverse) + mto_solve
(mixed-precision pCGMG to a 1e-8 relative residual) + mto_compliance_grad
(compliance and sensitivities).  value = solves/s over all ranks.

--impl reference times the CPU oracle instead (a bounded sample of the same
workload on the host cores).  Under torchrun every rank runs its own
independent solves (weak scaling, no collective on the data path).
"""

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pCGMG solves/s and GDOF-iter/s at 2048² Q4, mixed vs FP64, to 1e-8 residual; HBM % peak"
UNIT = "solves/s"
EP = [1.0, 0.5, 0.25, 1e-9]
PENAL = 3.0
SEED = 0
# Algorithmic work per finest-level node of the two timed kernels:
#  * outer sweep p = z + beta p, q = K p, p.q in float64: 36 FP64 pipe
#    operations (11 edge-difference add/sub, 7 core mul/fma on pre-scaled
#    moduli, 14 edge-force add/sub, 2 fma for p, 2 fma for the dot); bytes:
#    z (float32 in the mixed path: 8, float64: 16), p 16, x 16 (the lagged
#    step x += alpha p), the element's modulus 8 in; p 16, x 16, q 16 out;
#  * float32 fused pre-smoothing (two damped-Jacobi sweeps from zero, the
#    first formed on the fly) carrying the CG update r -= alpha q of the last
#    step: reads the last r and q (float64, 16 B each) and the element's bf16
#    modulus (2 B), writes the new r (16 B), its float32 copy (8 B) and z
#    (8 B): 66 B;
#  * float64 fused pre-smoothing (float64 path): b 16, modulus 8, w/D 8 in,
#    z 16 out: 48 B; 38 FP64 operations (K v 32, w D^-1 b 2, z + d (b - K v) 4).
KP_OPS_PER_NODE = 36
KP_BYTES_PER_NODE = {"mixed": 96, "fp64": 104}
SMOOTH32_BYTES_PER_NODE = 66
SMOOTH64_OPS_PER_NODE = 38
SMOOTH64_BYTES_PER_NODE = 48
# DRAM bytes per launch at 2048^2 from an ncu --set full capture of one
# launch of each kernel in this bench's step (dram__bytes_read.sum +
# dram__bytes_write.sum); to be set to None whenever the kernel changes.
KP_TRAFFIC = 354_211_328
SMOOTH32_TRAFFIC = 249_079_296
# Nominal float64 pipe rate, for context next to the measured one: 2
# operations per clock per SM (1.25 TFLOP/s at 2 flops per FMA), 152 SMs,
# 2070 MHz.
FP64_OPS_NOMINAL = 2 * 152 * 2.070e9
# PCG iterations of the bounded CPU sample at the full size.
CPU_SAMPLE_ITERS = 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=2048)
    ap.add_argument("--n-coarsen", type=int, default=7)
    ap.add_argument("--gamma", type=int, default=1, help="cycle index of Alg. 1 (1: V, 2: W)")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-poisson", action="store_true")
    ap.add_argument("--no-two-load-cases", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="default launch shapes (for profiling)")
    ap.add_argument("--sweep-outer", type=int, default=50)
    ap.add_argument("--study", choices=["levels", "configs"], default=None,
                    help="instead of the bench line: pCGMG level study on the paper's meshes (levels), "
                         "or one row per single-solve workload: oracle and GPU (configs)")
    ap.add_argument("--study-precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--study-outer", type=int, default=500,
                    help="level study: most outer optimiser iterations per mesh and level")
    ap.add_argument("--study-seconds", type=float, default=150.0,
                    help="level study: wall-time budget of the optimiser loop per mesh and level")
    ap.add_argument("--study-meshes", default=None,
                    help="level study: comma-separated subset of the meshes, e.g. 128x128,128x256")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# Clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples (every 50 ms) kept only inside the timed window."""

    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"clocks_bench_{os.getpid()}_{index}.csv")
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=self.fh, stderr=subprocess.DEVNULL)
            time.sleep(0.5)  # let the sampler start before the timed region
        except Exception:
            self.proc = None
        self.t0 = time.time()
        return self

    def __exit__(self, *a):
        self.t1 = time.time()
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        import datetime
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                p = [t.strip() for t in line.split(",")]
                if len(p) < 8:
                    continue
                try:
                    ts = datetime.datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    continue
                rows.append((ts, p[1:]))
        inside = [r for ts, r in rows if self.t0 - 0.05 <= ts <= self.t1 + 0.05] or [r for _, r in rows]
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return None
        sm = sorted(v for v in (num(r[0]) for r in inside) if v is not None)
        smax = max((v for v in (num(r[1]) for r in inside) if v is not None), default=None)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in inside for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": reasons,
                "samples": len(inside)}


# ---------------------------------------------------------------------------
# CPU oracle timing (test infrastructure; only this leg of the bench uses it)
# ---------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import json, os, sys
sys.path.insert(0, {root!r})
from oracle import solver
from synth import dirichlet_design, load_top_edge
n, nc, max_it, gamma = {n}, {nc}, {max_it}, {gamma}
x = dirichlet_design(n, n, 4, {seed}); f = load_top_edge(n, n)
t = {{}}
r = solver.solve_pcgmg(n, n, x, {ep!r}, {penal}, f, n_coarsen=nc, tol={tol!r}, max_it=max_it,
                       gamma=gamma, timings=t)
t.update(iters=r["iters"], converged=bool(r["converged"]), host_cores=os.cpu_count())
print(json.dumps(t))
"""


def oracle_run(n, nc, max_it, gamma=1, tol=1e-8):
    """One oracle pCGMG solve (1 thread) in a subprocess, stopped after max_it
    PCG iterations; returns its set-up, start and per-iteration wall times."""
    code = ORACLE_SNIPPET.format(root=ROOT, n=n, nc=nc, max_it=max_it, seed=SEED, ep=EP, penal=PENAL,
                                 gamma=gamma, tol=tol)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    return json.loads(out.stdout.strip().splitlines()[-1])


def ndof(n):
    return 2 * (n + 1) * (n + 1)


def max_over_ranks(v, world, device):
    """Largest v over the ranks (the slowest rank's time); v itself on one rank."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, ms_max):
    """Whole-job throughput: every rank solved `steps` problems in at most ms_max."""
    return world * steps / (ms_max / 1000.0)


def cpu_sample_value(d, iters_full):
    """solves/s of the oracle at the measured size: its set-up and start as
    measured, plus iters_full iterations at the measured mean iteration time
    (every PCG iteration does the same work)."""
    t_it = sum(d["iter_s"]) / len(d["iter_s"])
    return 1.0 / (d["setup_s"] + d["start_s"] + iters_full * t_it)


def run_reference(args):
    """The oracle's pCGMG on the same workload (2048^2, 7 coarsenings, tol
    1e-8), one thread, on the host cores: ONE full solve whose PCG iterations
    are the steps (warmup untimed, then `steps` timed, then on to
    convergence).  value = 1 / wall time of the whole solve (set-up included)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    n, nc = args.size, args.n_coarsen
    d = oracle_run(n, nc, 1000, gamma=args.gamma)
    its = d["iter_s"]
    timed = its[args.warmup:args.warmup + args.steps] or its[-1:]
    total = d["setup_s"] + d["start_s"] + sum(its)
    v = 1.0 / total
    sample = (f"one full oracle pCGMG solve (numpy/scipy, FP64, 1 thread of {d['host_cores']} host cores) "
              f"at {n}x{n}, {nc} coarsenings, tol 1e-8: set-up {d['setup_s']:.1f} s + {d['iters']} "
              f"iterations {sum(its):.1f} s; steps = PCG iterations {args.warmup}..{args.warmup + len(timed) - 1}")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": len(timed), "warmup": args.warmup, "ms_per_step": 1000.0 * sum(timed) / len(timed),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"pCGMG {n}x{n} Q4 square wall (3 solids + void, p=3, seeded Dirichlet "
                               f"fractions), {nc} coarsenings to 16x16, tol 1e-8; oracle, one solve",
                   "iters": d["iters"], "converged": d["converged"], "gamma": args.gamma,
                   "step": "one PCG iteration of the oracle solve",
                   "ms_setup": 1000.0 * d["setup_s"], "s_total": total},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_batched(mto, dev, local):
    """Batched workload: 32 square-wall problems, sizes drawn from {128,256,512,1024}^2
    with seed 3, two load cases each (top -y, right +x), mixed path, one graph
    launch per batch; next to it one float64 4096^2 solve."""
    import numpy as np
    import torch
    from synth import batch_sizes, dirichlet_design, load_right_edge, load_top_edge

    sizes = batch_sizes(32, seed=3)
    problems = []
    for k, s in enumerate(sizes):
        nc = s.bit_length() - 1 - 4  # coarsest 16 x 16
        m = mto.Mesh(s, s, n_coarsen=nc, precision="mixed", tol=1e-8, rr_every=25, flexible=True,
                     device=local)
        xk = torch.from_numpy(dirichlet_design(s, s, 4, seed=3000 + k)).to(dev)
        F = torch.from_numpy(np.stack([load_top_edge(s, s), load_right_edge(s, s)])).to(dev)
        m.set_design(xk, EP, PENAL)
        m.autotune()
        problems.append({"mesh": m, "x": xk, "E_phase": EP, "penal": PENAL, "f": F})
    t0 = time.perf_counter()
    batch = mto.Batch(problems)
    build_ms = 1000 * (time.perf_counter() - t0)
    t0 = time.perf_counter()
    tuned_w = batch.tune()
    tune_ms = 1000 * (time.perf_counter() - t0)
    def cold_run():
        for pr in batch.problems:
            pr["u"].zero_()  # every run solves from u = 0
        return batch.run()

    cold_run()  # warm-up
    times, iters = [], 0
    for _ in range(2):
        st = cold_run()
        times.append(batch.ms_last())
        iters = sum(s["iters"] for s in st)
    ms = min(times)
    dof_iters = sum(ndof(pr["mesh"].nelx) * s["iters"] for pr, s in zip(problems, st))
    out = {"problems": len(problems), "load_cases": 2 * len(problems),
           "sizes": {str(s): sizes.count(s) for s in sorted(set(sizes))},
           "ms_per_batch": ms, "load_cases_per_s": 2 * len(problems) / (ms / 1000.0),
           "gdof_iter_s": dof_iters / (ms / 1000.0) / 1e9, "iters_total": iters,
           "all_converged": all(s["converged"] == 1 for s in st), "graph_build_ms": build_ms,
           "batch_tune": {"warps_per_sm": tuned_w, "ms": tune_ms},
           "max_rel_res_true": max(s["rel_res_true"] for s in st)}
    batch.close()
    for pr in problems:
        pr["mesh"].close()
    # One float64 4096^2 solve (8 coarsenings to 16 x 16).
    n4 = 4096
    m4 = mto.Mesh(n4, n4, n_coarsen=8, precision="fp64", tol=1e-8, max_it=1000, device=local)
    x4 = torch.from_numpy(dirichlet_design(n4, n4, 4, seed=3)).to(dev)
    f4 = torch.from_numpy(load_top_edge(n4, n4)).to(dev)
    m4.set_design(x4, EP, PENAL)
    m4.autotune()
    m4.solve(f4)
    m4.set_design(x4, EP, PENAL)
    u4, st4 = m4.solve(f4)
    out["fp64_4096"] = {"dofs": ndof(n4), "iters": st4["iters"], "ms_solve": st4["ms_solve"],
                        "ms_setup": st4["ms_setup"], "rel_res_true": st4["rel_res_true"],
                        "gdof_iter_s": ndof(n4) * st4["iters"] / (st4["ms_solve"] / 1000.0) / 1e9}
    m4.close()
    del x4, f4, u4
    torch.cuda.empty_cache()
    return out


# Table 1 (Sec. 5.1): the paper's pCGMG wall times for the Poisson problem,
# hardware and language not stated (context only; the 32 x 32 entry is
# printed without a unit).
TABLE1_PCGMG_S = {16: 0.23, 32: 2.62, 64: 0.56, 128: 0.65, 256: 0.41}


def run_poisson(mto, dev, local, reps=20):
    """Scalar Poisson pCGMG of Sec. 5.1 on Table 1's meshes (16^2 ... 256^2,
    coarsened to 2 x 2), f = 1 at every node, tol 1e-8: one cluster kernel
    per solve; device time per solve (median of reps), in float64 and with the
    float32 V-cycle ("mixed"), and the throughput of 64 right-hand sides at
    256^2 solved by concurrent clusters in one launch."""
    import torch
    out = {}
    for prec in ("fp64", "mixed"):
        for n in sorted(TABLE1_PCGMG_S):
            nc = n.bit_length() - 2
            p = mto.Poisson(n, n, n_coarsen=nc, tol=1e-8, precision=prec, device=local)
            f = torch.ones((n + 1, n + 1), dtype=torch.float64, device=dev)
            p.solve(f)
            ms = []
            for _ in range(reps):
                _, st = p.solve(f)
                ms.append(st["ms_solve"])
            ms.sort()
            t = ms[len(ms) // 2]
            key = str(n) if prec == "fp64" else f"{n}_mixed"
            out[key] = {"n_coarsen": nc, "cluster_ctas": p.info()["cluster_ctas"], "iters": st["iters"],
                        "ms_solve": t, "rel_res_true": st["rel_res_true"],
                        "gdof_iter_s": (n + 1) ** 2 * st["iters"] / (t / 1000.0) / 1e9,
                        "paper_pcgmg_s": TABLE1_PCGMG_S[n]}
            p.close()
        n = 256
        p = mto.Poisson(n, n, n_coarsen=n.bit_length() - 2, tol=1e-8, precision=prec, device=local)
        F = torch.ones((64, n + 1, n + 1), dtype=torch.float64, device=dev)
        p.solve(F)
        ms = []
        for _ in range(5):
            _, st = p.solve(F)
            ms.append(st["ms_solve"])
        t = min(ms)
        key = "batch_256_64rhs" if prec == "fp64" else "batch_256_64rhs_mixed"
        out[key] = {"ms": t, "solves_s": 64 / (t / 1000.0), "iters_total": st["iters"]}
        p.close()
    return out


def run_sweep(mto, dev, local, n_outer):
    """Mesh sweep: the alternating active-phase loop (float64 solves, each
    warm-started from the previous u) at 256^2, 512^2, 1024^2 with 4, 5, 6
    coarsenings and volume fractions [0.2, 0.15, 0.1] + void 0.55."""
    import torch
    from paper_2301_07457_gb300.optimize import ActivePhaseOptimizer
    from synth import load_top_edge

    out = {}
    for n, nc in ((256, 4), (512, 5), (1024, 6)):
        mesh = mto.Mesh(n, n, n_coarsen=nc, precision="fp64", tol=1e-8, max_it=1000, device=local)
        f = torch.from_numpy(load_top_edge(n, n)).to(dev)
        opt = ActivePhaseOptimizer(mesh, EP, [0.2, 0.15, 0.1, 0.55], f, penal=PENAL, rf=8.0)
        opt.step()  # first outer iteration: cold start, tuning of the launch shapes
        mesh.autotune()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        opt.run(n_outer - 1)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        timed = opt.history[len(opt.pairs):]
        its = [h[3] for h in timed]
        out[str(n)] = {"outer_iterations": n_outer, "solves": len(opt.history),
                       "s_timed": dt, "timed_solves": len(timed),
                       "loop_solves_s": len(timed) / dt,
                       "mean_pcg_iters_warm": sum(its) / len(its),
                       "first_solve_iters": opt.history[0][3],
                       "compliance_first": opt.history[0][2], "compliance_last": opt.history[-1][2]}
        mesh.close()
    return out


def run_ours(args):
    import ctypes

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    from paper_2301_07457_gb300.build import build
    build()
    import paper_2301_07457_gb300 as mto
    from paper_2301_07457_gb300 import _lib
    from synth import dirichlet_design, load_top_edge

    n, nc = args.size, args.n_coarsen
    x_np = dirichlet_design(n, n, 4, SEED)
    f_np = load_top_edge(n, n)
    x = torch.from_numpy(x_np).to(dev)
    f = torch.from_numpy(f_np).to(dev)
    nodes = (n + 1) * (n + 1)
    hbm_peak, peak_kind = peaks()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks_here(v):
        return max_over_ranks(v, world, dev)

    def launches(mesh):
        c = ctypes.c_longlong()
        _lib.check(mesh._lib.mto_get_launch_count(mesh._h, ctypes.byref(c)), "launch count")
        return c.value

    def step(mesh):
        mesh.set_design(x, EP, PENAL)
        u, st = mesh.solve(f)
        C, g = mesh.compliance_grad(f, u)
        return st, C

    def timed(mesh, steps, warmup):
        for _ in range(warmup):
            step(mesh)
        torch.cuda.synchronize()
        barrier()
        l0 = launches(mesh)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stats = []
        with ClockSampler(local) as clk:
            e0.record()
            for _ in range(steps):
                st, C = step(mesh)
                stats.append(st)
            e1.record()
            torch.cuda.synchronize()
        barrier()
        ms = max_over_ranks_here(e0.elapsed_time(e1))
        return ms, stats, launches(mesh) - l0, clk.summary()

    def kernel_times(mesh, steps):
        # Events around the two hot kernels of every iteration (the solver
        # then drives its loop from the host); a second timed region.
        mesh.set_kernel_timing(True)
        step(mesh)  # builds the graph with event nodes
        mesh.set_kernel_timing(True)  # resets the sums
        for _ in range(steps):
            step(mesh)
        t, cnt = mesh.kernel_times()
        mesh.set_kernel_timing(False)
        return {"ms": t, "samples": cnt}

    common = dict(n_coarsen=nc, tol=1e-8, max_it=1000, gamma=args.gamma, device=local)
    mixed = mto.Mesh(n, n, precision="mixed", rr_every=25, flexible=True, **common)
    mixed.set_design(x, EP, PENAL)
    shapes_mixed = [mixed.launch_shape(l) for l in range(nc + 1)] if args.no_tune else mixed.autotune()
    ms, stats, nlaunch, clocks = timed(mixed, args.steps, args.warmup)
    kt = kernel_times(mixed, 2)
    iters = [s["iters"] for s in stats]
    solve_ms = [s["ms_solve"] for s in stats]
    value = job_value(world, args.steps, ms)
    gdof = ndof(n) * sum(iters) / (ms / 1000.0) / 1e9
    gdof_solve = ndof(n) * sum(iters) / (sum(solve_ms) / 1000.0) / 1e9

    # Roofline of the two timed kernels (live CUDA events inside the solver
    # graph).  The float64 sweep's peak is the float64 FMA issue rate measured
    # on this device right here (mto_measure_fp64_rate), with its clocks.
    with ClockSampler(local) as clk_probe:
        fp64_peak = mto.measure_fp64_rate(local)
    fp64_probe = {"ops_per_s": fp64_peak, "nominal_ops_per_s": FP64_OPS_NOMINAL,
                  "clocks": clk_probe.summary(),
                  "how": "mto_measure_fp64_rate: 8 independent DFMA chains per thread, 8 x 256-thread "
                         "blocks per SM, CUDA events, best of 5 after 3 warm-up launches"}
    kp_ms, sm_ms = kt["ms"]
    kp_ops = KP_OPS_PER_NODE * nodes / (kp_ms / 1000.0)
    kp_gbs = KP_BYTES_PER_NODE["mixed"] * nodes / (kp_ms / 1000.0) / 1e9
    sm_bytes = SMOOTH32_BYTES_PER_NODE * nodes / (sm_ms / 1000.0)
    roofline = {"bound": "alu", "kernel": "outer sweep p=z+beta p, q=Kp, p.q (float64)",
                "achieved": kp_ops / 1e12, "peak": fp64_peak / 1e12, "unit": "T FP64-op/s",
                "frac": kp_ops / fp64_peak, "traffic": KP_TRAFFIC, "ms_per_launch": kp_ms,
                "samples": kt["samples"][0],
                "peak_kind": "measured: float64 FMA issue rate of this GPU (fp64_peak)",
                "hbm": {"achieved_gbs": kp_gbs, "peak_gbs": hbm_peak, "frac": kp_gbs / hbm_peak,
                        "bytes_per_node": KP_BYTES_PER_NODE["mixed"], "peak_kind": peak_kind}}
    roofline_vcycle = {"bound": "hbm",
                       "kernel": "finest fused pre-smoothing with the CG update (float32, bf16 E; float64 r)",
                       "achieved": sm_bytes / 1e9, "peak": hbm_peak, "unit": "GB/s",
                       "frac": sm_bytes / 1e9 / hbm_peak, "traffic": SMOOTH32_TRAFFIC,
                       "ms_per_launch": sm_ms, "samples": kt["samples"][1], "peak_kind": peak_kind}

    # Two load cases (top-edge and right-edge loads) on the same design:
    # solved at the same time (two workspaces) and one after the other,
    # against one load case (device time of mto_solve, median of 3).
    two_lc = None
    if not args.no_two_load_cases:
        from synth import load_right_edge
        F2 = torch.from_numpy(np.stack([f_np, load_right_edge(n, n)])).to(dev)
        seq = mto.Mesh(n, n, precision="mixed", rr_every=25, flexible=True, concurrent_rhs=1, **common)
        seq.set_design(x, EP, PENAL)
        if not args.no_tune:
            seq.autotune()

        def med_solve(m, rhs):
            m.solve(rhs)
            t = sorted(m.solve(rhs)[1]["ms_solve"] for _ in range(3))
            return t[1]
        ms1 = med_solve(mixed, f)
        ms2c = med_solve(mixed, F2)
        ms2s = med_solve(seq, F2)
        Uc, _ = mixed.solve(F2)
        Us, _ = seq.solve(F2)
        two_lc = {"ms_one_load_case": ms1, "ms_two_concurrent": ms2c, "ms_two_sequential": ms2s,
                  "ratio_concurrent_to_one": ms2c / ms1, "ratio_sequential_to_one": ms2s / ms1,
                  "bit_identical": bool(torch.equal(Uc, Us))}
        seq.close()
        del F2, Uc, Us

    # End to end through the C ABI with pinned host buffers (right after the
    # device-timed steps, on the same context, before the other workloads).
    # The headline number pipelines the steps (mto_run_host_async: step k+1's
    # inputs go up and step k-1's results come down while step k computes,
    # two sets of host buffers in turn); the blocking mto_run_host loop is
    # reported beside it.
    e2e = None
    if not args.no_e2e:
        def host_set():
            b = {k: torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
                 for k, a in (("x", x_np), ("f", f_np), ("u", f_np), ("g", x_np))}
            b["x"].copy_(torch.from_numpy(x_np))
            b["f"].copy_(torch.from_numpy(f_np))
            b["c"] = torch.empty(1, dtype=torch.float64, pin_memory=True)
            return b

        sets = [host_set(), host_set()]
        Ep = (ctypes.c_double * 4)(*EP)
        st = _lib.SolveStats()
        vp = lambda t: ctypes.c_void_p(t.data_ptr())

        def host_step():
            b = sets[0]
            code = mixed._lib.mto_run_host(mixed._h, 4, vp(b["x"]), Ep, PENAL, 1, vp(b["f"]), vp(b["u"]),
                                           vp(b["c"]), vp(b["g"]), ctypes.byref(st))
            _lib.check(code, "mto_run_host")

        def host_enqueue(k):
            b = sets[k % 2]
            code = mixed._lib.mto_run_host_async(mixed._h, 4, vp(b["x"]), Ep, PENAL, 1, vp(b["f"]), vp(b["u"]),
                                                 vp(b["c"]), vp(b["g"]))
            _lib.check(code, "mto_run_host_async")

        def host_wait():
            _lib.check(mixed._lib.mto_run_host_wait(mixed._h, ctypes.byref(st)), "mto_run_host_wait")

        def pipelined(k_steps):
            for k in range(k_steps):
                host_enqueue(k)
                if k >= 1:
                    host_wait()
            host_wait()

        host_step()
        pipelined(2)
        # Wall-clock over at least 20 steps, three times each: one host-side
        # stall weighs on a short loop, and the median of three repeats
        # keeps the number to what the path sustains.
        e2e_steps = max(args.steps, 20)
        blocking_vals, pipelined_vals = [], []
        with ClockSampler(local) as clk_e2e:
            for _ in range(3):
                barrier()
                t0 = time.perf_counter()
                for _ in range(e2e_steps):
                    host_step()
                blocking_vals.append(world * e2e_steps / max_over_ranks_here(time.perf_counter() - t0))
                barrier()
                t0 = time.perf_counter()
                pipelined(e2e_steps)
                pipelined_vals.append(world * e2e_steps / max_over_ranks_here(time.perf_counter() - t0))
        b = sets[0]
        e2e = {"value": sorted(pipelined_vals)[1], "unit": UNIT,
               "h2d_bytes_per_step": b["x"].numel() * 8 + b["f"].numel() * 8,
               "d2h_bytes_per_step": b["u"].numel() * 8 + b["g"].numel() * 8 + 8,
               "api": "mto_run_host_async + mto_run_host_wait, two steps in flight",
               "steps": e2e_steps, "repeats": pipelined_vals,
               "blocking_value": sorted(blocking_vals)[1], "blocking_repeats": blocking_vals,
               "clocks": clk_e2e.summary()}

    # FP64 path on the same input.
    fp64 = None
    if args.fp64_steps > 0:
        m64 = mto.Mesh(n, n, precision="fp64", **common)
        m64.set_design(x, EP, PENAL)
        if not args.no_tune:
            m64.autotune()
        ms64, st64, _, clk64 = timed(m64, args.fp64_steps, 1)
        kt64 = kernel_times(m64, 1)
        it64 = [s["iters"] for s in st64]
        v64 = job_value(world, args.fp64_steps, ms64)
        kp64_s, sm64_s = kt64["ms"][0] / 1000.0, kt64["ms"][1] / 1000.0
        fp64 = {"solves_s": v64, "ms_per_step": ms64 / args.fp64_steps, "iters": it64,
                "gdof_iter_s": ndof(n) * sum(it64) / (ms64 / 1000.0) / 1e9,
                "rel_res_true": max(s["rel_res_true"] for s in st64),
                "kernel_ms": kt64["ms"],
                # Both bounds of the float64 sweeps: the float64 pipe (binding)
                # and HBM (the >= 60% target, out of reach while the pipe binds).
                "kp_fp64_frac_alu": KP_OPS_PER_NODE * nodes / kp64_s / fp64_peak,
                "kp_fp64_frac_hbm": KP_BYTES_PER_NODE["fp64"] * nodes / kp64_s / 1e9 / hbm_peak,
                "smoother_fp64_frac_alu": SMOOTH64_OPS_PER_NODE * nodes / sm64_s / fp64_peak,
                "smoother_fp64_frac_hbm": SMOOTH64_BYTES_PER_NODE * nodes / sm64_s / 1e9 / hbm_peak,
                "clocks": clk64}
        m64.close()

    batched = None
    if not args.no_batch:
        batched = run_batched(mto, dev, local)
    poisson_t1 = None
    if not args.no_poisson:
        poisson_t1 = run_poisson(mto, dev, local)
    sweep = None
    if not args.no_sweep:
        sweep = run_sweep(mto, dev, local, args.sweep_outer)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # A bounded sample of the same workload: the oracle's set-up and its
        # first CPU_SAMPLE_ITERS PCG iterations at the full size, measured;
        # the solve is completed at the measured iteration time with the
        # iteration count of the float64 GPU path on the same input (the
        # oracle's count is within one of it, as the parity tests check).
        d = oracle_run(n, nc, CPU_SAMPLE_ITERS, gamma=args.gamma)
        iters_full = fp64["iters"][0] if fp64 else iters[0]
        cpu = {"value": cpu_sample_value(d, iters_full), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": (f"oracle pCGMG (numpy/scipy FP64, 1 thread of {d['host_cores']} host cores) at "
                          f"{n}^2, measured: set-up {d['setup_s']:.1f} s + start {d['start_s']:.2f} s + "
                          f"{len(d['iter_s'])} PCG iterations at {sum(d['iter_s']) / len(d['iter_s']):.2f} s; "
                          f"completed to {iters_full} iterations (the float64 GPU path's count)")}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": f"mixed pCGMG {n}x{n} Q4 square wall (3 solids + void, p=3, seeded "
                               f"Dirichlet fractions), {nc} coarsenings to 16x16, tol 1e-8; step = "
                               "set_design + solve + compliance/sensitivities",
                   "nelx": n, "nely": n, "dofs": ndof(n), "n_coarsen": nc, "precision": "mixed",
                   "gamma": args.gamma,
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (design 134 MB + load 67 MB read every step)"},
        "gdof_iter_s": gdof, "gdof_iter_s_solve_only": gdof_solve, "iters": iters,
        "rel_res_true_max": max(s["rel_res_true"] for s in stats),
        "ms_setup": stats[-1]["ms_setup"], "ms_solve": solve_ms,
        "fp64": fp64, "speedup_mixed_vs_fp64": (value / fp64["solves_s"]) if fp64 else None,
        "roofline": roofline, "roofline_vcycle": roofline_vcycle, "fp64_peak": fp64_probe,
        "launch_shapes": shapes_mixed, "batched": batched, "mesh_sweep": sweep,
        "poisson_table1": poisson_t1, "two_load_cases": two_lc,
        "clocks": clocks, "gpu_launches": nlaunch, "e2e": e2e, "cpu_baseline": cpu,
    }
    mixed.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# Level study (Sec. 5.2, Tables 2-5): pCGMG with l = 2 ... 6 grids on the
# paper's meshes, Table 2's parameters
# ---------------------------------------------------------------------------
PAPER_MESHES = ((32, 32), (32, 64), (64, 64), (64, 128), (128, 128), (128, 256))
TABLE2 = {"E": [9.0, 3.0, 1.0, 1e-9], "V": [0.16, 0.08, 0.08, 0.68], "penal": 3.0, "rf": 8.0,
          "tol": 1e-3, "cgtol": 1e-6, "cgmax": 1000}


def run_level_study(args):
    """One JSON line per (mesh, l): a cold set_design + solve on the seeded
    design with Table 2's moduli (device time, median of args.steps), then the
    outer optimiser loop of Sec. 4 from the uniform design until no fraction
    moves by more than Table 2's tol (at most args.study_outer outer
    iterations, wall time).  Meshes are nelx x nely as printed; l counts the
    grids (l = 2 is the two-level method), so n_coarsen = l - 1."""
    import torch

    from paper_2301_07457_gb300.build import build
    build()
    import paper_2301_07457_gb300 as mto
    from paper_2301_07457_gb300 import MtoError
    from paper_2301_07457_gb300.optimize import ActivePhaseOptimizer
    from synth import dirichlet_design, load_top_edge

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    T = TABLE2
    meshes = PAPER_MESHES
    if args.study_meshes:
        keep = set(args.study_meshes.split(","))
        meshes = [m for m in PAPER_MESHES if f"{m[0]}x{m[1]}" in keep]
    for nelx, nely in meshes:
        f = torch.from_numpy(load_top_edge(nelx, nely)).to(dev)
        x = torch.from_numpy(dirichlet_design(nelx, nely, 4, SEED)).to(dev)
        for l in range(2, 7):
            row = {"study": "levels", "mesh": f"{nelx}x{nely}", "l": l, "n_coarsen": l - 1,
                   "coarsest": f"{nelx >> (l - 1)}x{nely >> (l - 1)}", "precision": args.study_precision}
            try:
                mesh = mto.Mesh(nelx, nely, n_coarsen=l - 1, precision=args.study_precision,
                                tol=T["cgtol"], max_it=T["cgmax"], device=0)
            except MtoError as e:
                row["unsupported"] = str(e)
                print(json.dumps(row), flush=True)
                continue
            row["coarsest_free_dofs"] = mesh.info()["coarsest_free_dofs"]
            ms = []
            for rep in range(args.warmup + args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                mesh.set_design(x, T["E"], T["penal"])
                u, st = mesh.solve(f, raise_on_failure=False)
                e1.record()
                torch.cuda.synchronize()
                if rep >= args.warmup:
                    ms.append(e0.elapsed_time(e1))
            row["solve"] = {"iters": st["iters"], "status": st["status"], "ms": sorted(ms)[len(ms) // 2],
                            "ms_setup": st["ms_setup"], "ms_solve": st["ms_solve"]}
            opt = ActivePhaseOptimizer(mesh, T["E"], T["V"], f, penal=T["penal"], rf=T["rf"])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            why = opt.run_until(T["tol"], args.study_outer, args.study_seconds)
            torch.cuda.synchronize()
            its = [h[3] for h in opt.history]
            row["optimiser"] = {"outer": opt.iteration, "stopped_by": why, "last_change": opt.change,
                                "solves": len(its),
                                "pcg_iters_mean": sum(its) / len(its), "pcg_iters_max": max(its),
                                "seconds": time.perf_counter() - t0, "compliance": opt.history[-1][2]}
            mesh.close()
            print(json.dumps(row), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Per-workload table: the single-solve workloads (64^2 to 1e-10 with three
# grids; 256^2, 512^2, 1024^2 with 4-6 coarsenings; 2048^2 with 7), each
# timed on the GPU in both precisions and as one full oracle solve on one
# host core, in the same run.
# ---------------------------------------------------------------------------
CONFIG_ROWS = ((64, 2, 1e-10), (256, 4, 1e-8), (512, 5, 1e-8), (1024, 6, 1e-8), (2048, 7, 1e-8))


def run_config_study(args):
    """One JSON line per workload: per precision the median device time of
    set_design + cold solve + compliance and sensitivities over args.steps
    steps (after args.warmup), PCG iterations, float64 true residual,
    GDOF-iterations/s, and the K p and first-smoothing kernels' times with
    their HBM (and float64-pipe) fractions; then one full oracle solve."""
    import torch

    from paper_2301_07457_gb300.build import build
    build()
    import paper_2301_07457_gb300 as mto
    from synth import dirichlet_design, load_top_edge

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    hbm_peak, peak_kind = peaks()
    fp64_peak = mto.measure_fp64_rate(0)
    for n, nc, tol in CONFIG_ROWS:
        x = torch.from_numpy(dirichlet_design(n, n, 4, SEED)).to(dev)
        f = torch.from_numpy(load_top_edge(n, n)).to(dev)
        nodes = (n + 1) * (n + 1)
        row = {"study": "configs", "mesh": f"{n}x{n}", "dofs": ndof(n), "n_coarsen": nc, "tol": tol,
               "hbm_peak_gbs": hbm_peak, "hbm_peak_kind": peak_kind, "fp64_peak_ops": fp64_peak}
        for prec in ("fp64", "mixed"):
            mesh = mto.Mesh(n, n, n_coarsen=nc, precision=prec, tol=tol, max_it=1000, device=0)
            mesh.set_design(x, EP, PENAL)
            mesh.autotune()

            def step():
                mesh.set_design(x, EP, PENAL)
                u, st = mesh.solve(f)
                mesh.compliance_grad(f, u)
                return st

            ms = []
            for rep in range(args.warmup + args.steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                st = step()
                e1.record()
                torch.cuda.synchronize()
                if rep >= args.warmup:
                    ms.append(e0.elapsed_time(e1))
            med = sorted(ms)[len(ms) // 2]
            mesh.set_kernel_timing(True)
            step()
            mesh.set_kernel_timing(True)
            step()
            (kp_ms, sm_ms), _ = mesh.kernel_times()
            mesh.set_kernel_timing(False)
            kp_bytes = KP_BYTES_PER_NODE[prec] * nodes
            sm_bytes = (SMOOTH64_BYTES_PER_NODE if prec == "fp64" else SMOOTH32_BYTES_PER_NODE) * nodes
            row[prec] = {"ms_step": med, "ms_solve": st["ms_solve"], "iters": st["iters"],
                         "rel_res_true": st["rel_res_true"],
                         "gdof_iter_s": ndof(n) * st["iters"] / (med / 1000.0) / 1e9,
                         "kp_ms": kp_ms, "kp_frac_hbm": kp_bytes / (kp_ms / 1000.0) / 1e9 / hbm_peak,
                         "kp_frac_fp64": KP_OPS_PER_NODE * nodes / (kp_ms / 1000.0) / fp64_peak,
                         "smooth_ms": sm_ms,
                         "smooth_frac_hbm": sm_bytes / (sm_ms / 1000.0) / 1e9 / hbm_peak}
            if prec == "fp64":
                row[prec]["smooth_frac_fp64"] = SMOOTH64_OPS_PER_NODE * nodes / (sm_ms / 1000.0) / fp64_peak
            mesh.close()
        d = oracle_run(n, nc, 1000, tol=tol)
        row["oracle"] = {"threads": 1, "host_cores": d["host_cores"], "iters": d["iters"],
                         "converged": d["converged"], "s_setup": d["setup_s"],
                         "s_total": d["setup_s"] + d["start_s"] + sum(d["iter_s"])}
        print(json.dumps(row), flush=True)
    return 0


def main():
    args = parse()
    if args.study == "levels":
        return run_level_study(args)
    if args.study == "configs":
        return run_config_study(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
