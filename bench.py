#!/usr/bin/env python
"""Benchmark: seconds per density-matrix build D = 1/2 (I - sign(K - mu I)).

The default workload is the large-scale one: 20,736 water-like molecules
with 6 functions each (n = 124,416), a 9 Angstrom cutoff (504-672-dim
submatrices), the gap shrunk to +-0.15 and mu = 0 (synthetic, seeded; the
paper's CP2K water matrices are not available).  One step is one whole
build: gather, FP16x3 tensor-core Newton-Schulz, FP64-anchored correction
(BF16x3 and exact sliced tensor-core products),
scatter -- every submatrix of the system.  Beside it the plain FP64 and FP32
GPU paths are each timed over one whole build, and the CPU oracle on a
bounded sample of block columns.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (launched by torch.distributed.run)
every rank builds its own seeded instance of the workload (weak scaling);
the timed region is bracketed by barriers and the maximum over ranks is used.
``--impl reference`` times the CPU FP64 oracle (the reference arm) on a
bounded sample of block columns of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (generator config index, description)
    "water1024_b23_rc8": (1, "1024 water-like molecules x 23 functions (n=23552), cutoff 8 A, mu=0"),
    "water32_b6_rc6": (0, "32 water-like molecules x 6 functions (n=192), cutoff 6 A, mu=0"),
    "slab4096_b6": (2, "4096-molecule slab (liquid + vapour) x 6 functions, cutoff U[7,10] A, mu=0"),
    "water2048_b23_rc8": (3, "2048 water-like molecules x 23 functions (n=47104), cutoff 8 A, mu=0"),
    "water20736_b6_rc9": (4, "20736 water-like molecules x 6 functions (n=124416), cutoff 9 A, gap 0.15"),
}
METRIC = "s per D build & TFLOP/s: BF16+refine vs FP64 path, same GB300, max|dD|<=1e-7"
FP64_NOMINAL_GFLOPS = 1250.0   # GB300 FP64 rate (recipe's nominal table)
# FP32 FMA pipes: 152 SMs x 128 lanes x 2 flops x 2.07 GHz (maximum SM clock)
FP32_NOMINAL_GFLOPS = 152 * 128 * 2 * 2.07
L2_BYTES = 129 << 20           # GB300 L2
CLASS_NAMES = ["tc_gemm_newton_schulz", "tc_gemm_correction", "simt_gemm_fp64", "gather",
               "tc_gemm_sliced_fp64", "tc_gemm_adjoint", "scatter", "reserved"]
NCLASS = len(CLASS_NAMES)
HBM_CLASSES = (3, 6)   # byte-counted kernels: gather, scatter


def host_cores():
    """(cores this process may run on, os.cpu_count(), the affinity list as a
    compact string)."""
    try:
        aff = sorted(os.sched_getaffinity(0))
    except Exception:  # pragma: no cover
        aff = list(range(os.cpu_count() or 1))
    runs, start = [], None
    for i, c in enumerate(aff):
        if start is None:
            start = c
        if i + 1 == len(aff) or aff[i + 1] != c + 1:
            runs.append(f"{start}-{c}" if c != start else f"{c}")
            start = None
    return len(aff), os.cpu_count(), ",".join(runs)


def oracle_sample(m, target_s, workers, cap=None):
    """Block columns for a CPU oracle sample of about target_s seconds: a probe
    of 2 x workers columns fixes the rate, the count follows from it."""
    probe = sample_columns(m.nblk, min(m.nblk, 2 * workers))
    _d, t = run_oracle_sample(m, probe, workers)
    count = int(len(probe) * target_s / max(t, 1e-3))
    count = max(len(probe), min(m.nblk, count if cap is None else min(cap, count)))
    return sample_columns(m.nblk, count), len(probe), t


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def sample_columns(nblk, count):
    step = max(1, nblk // count)
    return list(range(0, nblk, step))[:count]


def run_oracle_sample(m, cols, workers):
    import oracle
    t0 = time.perf_counter()
    d = oracle.density_matrix(m, m.mu, columns=cols, workers=workers)
    return d, time.perf_counter() - t0


def reference_arm(args, m, desc):
    """The oracle as it stands, on host cores, a bounded sample per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    workers, ncpu, aff = host_cores()
    if args.cpu_sample > 0:
        cols = sample_columns(m.nblk, args.cpu_sample)
    else:  # about 2 minutes of oracle work over all steps, at most 15 s per step
        cols, _np, _tp = oracle_sample(m, min(15.0, 120.0 / max(1, args.steps)), workers)
    for _ in range(args.warmup):
        run_oracle_sample(m, cols[: max(1, len(cols) // 8)], workers)
    times = []
    for _ in range(args.steps):
        _d, t = run_oracle_sample(m, cols, workers)
        times.append(t)
    per_build = statistics.median(times) * m.nblk / len(cols)
    line = {
        "impl": "reference", "metric": METRIC, "value": per_build, "unit": "s/build",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "sampled_block_columns": len(cols)},
        "cpu_baseline": {"value": per_build, "unit": "s/build", "cores": workers, "cpu_count": ncpu,
                         "affinity": aff, "kind": "oracle",
                         "sample": f"{len(cols)} of {m.nblk} block columns per step (numpy eigh per "
                                   f"submatrix in a {workers}-process pool, one per core this job may "
                                   f"use), scaled to a full build"},
        "e2e": {"value": per_build, "unit": "s/build", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def sweep(args):
    """Time per D build against system size at a fixed cutoff (the submatrix
    method's linear scaling, Section V): the 1024x23 recipe at other molecule
    counts, fixed tile widths, one JSON line per size."""
    import torch
    import __graft_entry__ as entry
    entry.build()
    import paper_2004_10811_gb300 as pkg
    from synth.water import make_water
    for n_mol in (int(x) for x in args.sweep.split(",")):
        m = make_water(n_mol, 23, 8.0, (4, -1.0, -0.3), (19, 0.3, 1.5), seed=3000 + n_mol)
        K = torch.from_numpy(m.vals).cuda()
        D = torch.empty_like(K)
        with pkg.Plan.from_bsr(m, prec="mixed", tile_n_ns=256, tile_n_corr=256, tile_n_hp=128) as plan:
            for _ in range(max(1, args.warmup)):
                plan.sign(K, m.mu, out=D)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                plan.sign(K, m.mu, out=D)
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) / 1e3 / args.steps
            st = plan.stats()
        print(json.dumps({"sweep": "water_b23_rc8", "n_mol": n_mol, "n": int(m.n), "s_per_build": t,
                          "ms_per_molecule": 1e3 * t / n_mol, "sum_n3": st["sum_n3"],
                          "sub_dim_min": int(st["n_min"]), "sub_dim_max": int(st["n_max"]),
                          "waves": int(st["waves"]), "iters_max": int(st["iters_max"]),
                          "fp64_fallback_submatrices": int(st["refine_fallback"])}), flush=True)


def shard_run(args, m, desc, pkg, dist, rank, world, local, dev):
    """Strong scaling (shard.py): every rank holds the blocks of its own block
    rows, a device halo exchange brings what its chunk's submatrices need, the
    chunk is evaluated by a column-range plan and Tr D is allreduced.  A step
    is that whole sequence; the time is the maximum over ranks."""
    import numpy as np
    import torch
    from paper_2004_10811_gb300.shard import ShardedPattern, gpu_solver, sharded_density

    class _Single:  # the world-size-1 stand-ins for the collectives
        P2POp = None

        @staticmethod
        def all_reduce(t):
            return t

        @staticmethod
        def all_gather_object(out, obj):
            out[0] = obj

        @staticmethod
        def barrier():
            pass

    comm = dist if dist is not None else _Single
    sp = ShardedPattern(m.block_sizes, m.row_ptr, m.col_idx, rank, world)
    owned = np.zeros_like(m.vals)
    for p in np.nonzero(sp.owner == rank)[0]:
        owned[sp.vp[p]:sp.vp[p + 1]] = m.vals[sp.vp[p]:sp.vp[p + 1]]
    K0 = torch.from_numpy(owned).to(dev)
    solve = gpu_solver(sp, device=dev, prec=args.prec)
    K = K0.clone()
    for _ in range(max(1, args.warmup)):
        K.copy_(K0)
        sharded_density(sp, K, m.mu, solve, comm, exchange=world > 1)
    comm.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            K.copy_(K0)
            _d, tr = sharded_density(sp, K, m.mu, solve, comm, exchange=world > 1)
        e1.record(stream)
        torch.cuda.synchronize()
    comm.barrier()
    t = e0.elapsed_time(e1) / 1e3
    tt = torch.tensor([t], device=dev)
    comm.all_reduce(tt, op=dist.ReduceOp.MAX) if dist is not None else None
    t = float(tt.item())
    clocks = clk.summary()
    if rank == 0:
        value = t / args.steps
        line = {"metric": METRIC, "value": value, "unit": "s/build", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * value, "higher_is_better": False,
                "scaling": "strong", "vs_baseline": None,
                "dtype": "f16x3+bf16x3+f64" if args.prec == "mixed" else args.prec, "data": "synthetic",
                "config": {"workload": args.workload, "description": desc, "prec": args.prec,
                           "parallelism": f"{world} ranks, Sigma n^3-balanced column chunks, device halo "
                                          "exchange and trace allreduce", "chunk_rank0": list(sp.chunk)},
                "trace": tr, "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                                        "reasons": clocks["reasons"]}}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="water20736_b6_rc9")
    ap.add_argument("--prec", choices=["mixed", "fp64", "fp32"], default="mixed")
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="block columns in the oracle sample (0: as many as about 15 s of oracle work)")
    ap.add_argument("--fp64-sample", type=int, default=0,
                    help="block columns timed on the FP64 path (0: the whole build)")
    ap.add_argument("--no-fp32", action="store_true", help="skip the whole-build FP32 path timing")
    ap.add_argument("--shard", action="store_true",
                    help="strong scaling: all ranks share one system, each evaluates a Sigma n^3-balanced "
                         "chunk of block columns after a device halo exchange (shard.py); default is weak "
                         "scaling, one seeded instance per rank")
    ap.add_argument("--group-size", type=int, default=2,
                    help="block columns per submatrix for the grouped key (periodic k-means on the molecule "
                         "centres, Section IV-C); 0 skips it")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--adjoint-sample", type=int, default=32,
                    help="block columns timed for the adjoint (submat_sign_backward); 0 skips it")
    ap.add_argument("--kT", type=float, default=0.05,
                    help="finite-temperature key: one whole build with the Fermi function at this kT "
                         "(Section IV-F) on the FP32 and FP64 paths; 0 skips it")
    ap.add_argument("--mu-search", action="store_true",
                    help="also time submat_mu_search for the workload's electron count")
    ap.add_argument("--columns", default=None,
                    help="a:b -- evaluate only block columns [a, b) (small cases for profiling)")
    ap.add_argument("--tile-n-ns", type=int, default=0, choices=[0, 128, 256])
    ap.add_argument("--tile-n-corr", type=int, default=0, choices=[0, 128, 256])
    ap.add_argument("--tile-n-hp", type=int, default=0, choices=[0, 128, 256])
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the plan's default tile widths (autotuning runs unless widths are given)")
    ap.add_argument("--iteration", type=int, default=0, choices=[0, 1],
                    help="sign iteration of the mixed path: 0 Newton-Schulz, 1 third order")
    ap.add_argument("--sweep", default=None,
                    help="comma-separated molecule counts: time the mixed path on the 1024x23 recipe "
                         "(block 23, cutoff 8 A) at each size, one JSON line per size (linear scaling)")
    args = ap.parse_args()

    if args.sweep:
        sweep(args)
        return
    cfg_index, desc = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from synth import make_config
    # weak scaling: each rank builds its own seeded instance of the workload;
    # --shard: one instance shared by all ranks
    m = make_config(cfg_index, seed=None if (rank == 0 or args.shard) else 1000 + cfg_index + 7919 * rank)

    if args.impl == "reference":
        reference_arm(args, m, desc)
        return

    import numpy as np
    import torch
    import __graft_entry__ as graft
    graft.build()
    import paper_2004_10811_gb300 as pkg

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    peaks, peak_src = load_peaks()
    dev = torch.device("cuda", local)
    if args.shard:
        shard_run(args, m, desc, pkg, dist, rank, world, local, dev)
        return
    K = torch.from_numpy(m.vals).to(dev)
    D = torch.empty_like(K)
    columns = tuple(int(x) for x in args.columns.split(":")) if args.columns else None
    plan = pkg.Plan.from_bsr(m, prec=args.prec, timing=True, columns=columns, tile_n_ns=args.tile_n_ns,
                             tile_n_corr=args.tile_n_corr, tile_n_hp=args.tile_n_hp,
                             iteration=args.iteration if args.prec == "mixed" else 0)
    tiles = {"ns": args.tile_n_ns, "correction": args.tile_n_corr, "sliced": args.tile_n_hp, "source": "options"}
    if args.prec == "mixed" and not args.no_autotune and not (args.tile_n_ns or args.tile_n_corr or args.tile_n_hp):
        t0 = time.perf_counter()
        tiles = dict(plan.autotune(K, m.mu, out=D), source="submat_autotune")
        torch.cuda.synchronize()
        tiles["autotune_s"] = round(time.perf_counter() - t0, 3)
    for _ in range(args.warmup):
        plan.sign(K, m.mu, out=D)
    torch.cuda.synchronize()
    plan_tiles = (plan.options.tile_n_ns, plan.options.tile_n_corr, plan.options.tile_n_hp)

    # ---- device-resident timed region ----
    acc = {"kernel_ms": [0.0] * NCLASS, "kernel_launches": [0] * NCLASS, "kernel_work": [0.0] * NCLASS,
           "kernel_exec": [0.0] * NCLASS,
           "launches": 0, "flops_ns": 0.0, "flops_refine": 0.0}
    barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    # a working set that L2 (129 MB) could hold is flushed between steps, outside
    # the timed event pairs, by writing a 256 MB buffer
    working_set = 2 * m.vals.nbytes + plan.stats()["workspace_bytes"]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev) if working_set < 4 * L2_BYTES else None
    l2_note = ("L2 flushed between steps (256 MB write outside the timed events)" if flush is not None else
               "inputs larger than L2")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            if flush is not None:
                flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            plan.sign(K, m.mu, out=D)
            ev[i][1].record(stream)
            st = plan.stats()
            for k in ("kernel_ms", "kernel_launches", "kernel_work", "kernel_exec"):
                acc[k] = [a + b for a, b in zip(acc[k], st[k])]
            for k in ("launches", "flops_ns", "flops_refine"):
                acc[k] += st[k]
        torch.cuda.synchronize()
    barrier()
    t_dev = sum(a.elapsed_time(b) for a, b in ev) / 1e3
    if dist is not None:
        tt = torch.tensor([t_dev], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_dev = float(tt.item())
    clocks = clk.summary()
    stats = plan.stats()
    sub = plan.sub_stats()

    # ---- end to end through the host-buffer entry point ----
    Kh = torch.from_numpy(m.vals).pin_memory()
    Dh = torch.empty_like(Kh).pin_memory()
    plan.sign_host(Kh.numpy(), m.mu, out=Dh.numpy())
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        plan.sign_host(Kh.numpy(), m.mu, out=Dh.numpy())
    t_e2e = time.perf_counter() - t0
    barrier()
    if dist is not None:
        tt = torch.tensor([t_e2e], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_e2e = float(tt.item())
    # ---- mu search (bisection on Tr D(mu) = N_el), opt-in: each step is one build ----
    mu_line = None
    if args.mu_search and world == 1 and not columns:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # started 1.0 above the workload's mu, inside the virtual band, so
        # that the bracket has to be bisected down into the gap
        mu0 = m.mu + 1.0
        mu_found, _Dm, status = plan.mu_search(K, m.n_el, mu0=mu0, tol=1e-9, max_steps=120, out=D)
        torch.cuda.synchronize()
        tm = time.perf_counter() - t0
        stm = plan.stats()
        steps, probes = int(stm["mu_steps"]), int(stm["mu_probes"])
        mu_line = {"mu0": mu0, "mu": mu_found, "status": status, "s_total": tm, "full_evaluations": steps,
                   "probes": probes, "builds_equivalent": tm / (t_dev / args.steps),
                   "n_el": float(m.n_el)}
    plan.close()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    builds = args.steps * world
    if columns:
        line_cols = {"columns": list(columns)}
    else:
        line_cols = {}
    value = t_dev / builds
    flops_std = (acc["flops_ns"] + acc["flops_refine"]) / args.steps  # per build
    line = {
        "metric": METRIC, "value": value, "unit": "s/build", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f16x3+bf16x3+f64" if args.prec == "mixed" else args.prec,
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "prec": args.prec,
                   "iteration": "third order" if args.iteration == 1 else "Newton-Schulz",
                   "n": int(m.n), "nsub": int(m.nblk), "nnzb": int(m.nnzb),
                   "sub_dim_min": int(stats["n_min"]), "sub_dim_max": int(stats["n_max"]), **line_cols,
                   "tiles": tiles,
                   "l2": "%s (K %.2f GB, workspace %.2f GB)" % (l2_note, m.vals.nbytes / 1e9,
                                                                 stats["workspace_bytes"] / 1e9)},
        "tflops": flops_std / value / 1e12 / world if value > 0 else None,
        "iters": {"min": int(sub["iters"].min()), "max": int(sub["iters"].max())},
        "refine": {"rounds": stats["refine_rounds"], "cg_iters": stats["refine_cg_iters"],
                   "fp64_fallback_submatrices": stats["refine_fallback"]},
        "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"], "reasons": clocks["reasons"]},
        "gpu_launches": int(acc["launches"]),
        "e2e": {"value": t_e2e / builds, "unit": "s/build", "h2d_bytes_per_step": int(m.vals.nbytes),
                "d2h_bytes_per_step": int(m.vals.nbytes)},
    }

    # ---- per-kernel-class roofline ----
    kernels = {}
    for c in range(NCLASS):
        n = acc["kernel_launches"][c]
        if n == 0:
            continue
        ms = acc["kernel_ms"][c]
        work = acc["kernel_work"][c]
        exec_tf = None
        if c in HBM_CLASSES:
            achieved = work / (ms / 1e3) / 1e9
            unit, peak, bound, psrc = "GB/s", peaks["hbm_gbs"], "hbm", peak_src
        elif c in (0, 1, 4):
            achieved = work / (ms / 1e3) / 1e12
            exec_tf = acc["kernel_exec"][c] / (ms / 1e3) / 1e12
            # FP16 and BF16 share one nominal dense rate, so the measured BF16
            # peak (ratio 1) serves the FP16 Newton-Schulz products too
            unit, peak, bound = "TFLOP/s", peaks["bf16_tflops_sustained"], "tensor"
            psrc = peak_src + (" (bf16 sustained = fp16 rate)" if c == 0 else " (bf16 sustained)")
        else:
            achieved = work / (ms / 1e3) / 1e12
            unit, peak, bound, psrc = "TFLOP/s", FP64_NOMINAL_GFLOPS / 1e3, "alu", "nominal FP64"
        kernels[CLASS_NAMES[c]] = {"launches": n, "ms_total": ms, "ms_per_launch": ms / n,
                                   "share": ms / (1e3 * t_dev), "achieved": achieved, "unit": unit,
                                   "peak": peak, "peak_source": psrc, "bound": bound,
                                   "frac": achieved / peak if peak else None}
        if exec_tf is not None:
            kernels[CLASS_NAMES[c]]["executed_mma_tflops"] = exec_tf
            kernels[CLASS_NAMES[c]]["executed_frac"] = exec_tf / peak
    # the three tensor-core classes are launches of one kernel, k_tc_gemm: its
    # roofline sums their algorithmic work and time (executed MMA work beside it)
    tc = [c for c in (0, 1, 4) if acc["kernel_launches"][c]]
    if tc:
        ms = sum(acc["kernel_ms"][c] for c in tc)
        work = sum(acc["kernel_work"][c] for c in tc)
        ex = sum(acc["kernel_exec"][c] for c in tc)
        n = sum(acc["kernel_launches"][c] for c in tc)
        peak = peaks["bf16_tflops_sustained"]
        kernels["k_tc_gemm"] = {"launches": n, "ms_total": ms, "ms_per_launch": ms / n,
                                "share": ms / (1e3 * t_dev), "achieved": work / (ms / 1e3) / 1e12,
                                "unit": "TFLOP/s", "peak": peak, "bound": "tensor",
                                "peak_source": peak_src + " (bf16 sustained; fp16 runs at the same rate)",
                                "frac": work / (ms / 1e3) / 1e12 / peak,
                                "executed_mma_tflops": ex / (ms / 1e3) / 1e12,
                                "executed_frac": ex / (ms / 1e3) / 1e12 / peak,
                                "classes": [CLASS_NAMES[c] for c in tc]}
    if kernels:
        cands = {k: v for k, v in kernels.items() if k not in ("tc_gemm_newton_schulz", "tc_gemm_correction",
                                                               "tc_gemm_sliced_fp64")}
        dom = max(cands, key=lambda k: cands[k]["ms_total"])
        kd = kernels[dom]
        traffic = None
        tpath = os.path.join(ROOT, "profiles", "traffic.json")
        if os.path.exists(tpath):
            try:
                tj = json.load(open(tpath))
                ent = tj.get(args.workload, {}).get(dom)
                if ent and ent.get("valid", True):
                    traffic = ent["bytes_per_launch"]
            except Exception:
                traffic = None
        line["roofline"] = {"kernel": dom, "bound": kd["bound"], "achieved": kd["achieved"], "peak": kd["peak"],
                            "unit": kd["unit"], "frac": kd["frac"], "traffic": traffic,
                            "peak_source": kd["peak_source"]}
        if "executed_frac" in kd:
            line["roofline"]["executed_mma_tflops"] = kd["executed_mma_tflops"]
            line["roofline"]["executed_frac"] = kd["executed_frac"]
        line["kernels"] = kernels

    # ---- parity on sampled block columns and the CPU oracle baseline ----
    want = cols = None
    if not args.no_cpu and world == 1 and not columns:
        workers, ncpu, aff = host_cores()
        if args.cpu_sample > 0:
            cols = sample_columns(m.nblk, args.cpu_sample)
        else:  # about 15 s of oracle work
            cols, _np, _tp = oracle_sample(m, 15.0, workers)
        want, t_cpu = run_oracle_sample(m, cols, workers)
        got = Dh.numpy()
        mask = ~np.isnan(want)
        line["max_abs_err_vs_oracle"] = float(np.max(np.abs(got[mask] - want[mask])))
        line["parity_sample"] = f"{len(cols)} of {m.nblk} block columns"
        line["cpu_baseline"] = {"value": t_cpu * m.nblk / len(cols), "unit": "s/build", "cores": workers,
                                "cpu_count": ncpu, "affinity": aff, "kind": "oracle",
                                "sample": f"{len(cols)} of {m.nblk} block columns (numpy eigh per submatrix, "
                                          f"{workers}-process pool, one per core this job may use), time "
                                          f"scaled to the full build"}

    # ---- the plain FP64 and FP32 GPU paths, each over one whole build ----
    def other_path(prec, ncols):
        cols_opt = (0, ncols) if ncols else None
        with pkg.Plan.from_bsr(m, prec=prec, columns=cols_opt, timing=True) as po:
            Dtmp = torch.zeros_like(K)
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            f0.record(stream)
            po.sign(K, m.mu, out=Dtmp)
            f1.record(stream)
            torch.cuda.synchronize()
            t = f0.elapsed_time(f1) / 1e3
            so = po.stats()
        out = {"iters_max": int(so["iters_max"]), "tflops": so["flops_ns"] / t / 1e12,
               "waves": int(so["waves"]), "scale_reduced": int(so["scale_reduced"])}
        if ncols:
            sub_n3 = float(np.sum(sub["dims"].astype(np.float64) ** 3))
            chunk_n3 = float(np.sum(sub["dims"][:ncols].astype(np.float64) ** 3))
            out.update(s_per_build_est=t * sub_n3 / chunk_n3, chunk_s=t,
                       measured=f"block columns [0, {ncols}) timed, scaled by sum n^3")
        else:
            out.update(s_per_build=t, measured="one whole build (every block column), CUDA events")
            if want is not None:
                got = Dtmp.cpu().numpy()
                mask = ~np.isnan(want)
                out["max_abs_err_vs_oracle"] = float(np.max(np.abs(got[mask] - want[mask])))
                out["parity_sample"] = f"{len(cols)} of {m.nblk} block columns"
        return out

    if not args.no_fp64 and args.prec == "mixed" and world == 1 and not columns:
        nc = min(args.fp64_sample, m.nblk)
        f64 = other_path("fp64", nc)
        t64 = f64.get("s_per_build", f64.get("s_per_build_est"))
        f64["speedup_mixed_vs_fp64"] = t64 / value
        line["fp64_path"] = f64
    if not args.no_fp32 and args.prec == "mixed" and world == 1 and not columns:
        # FP32 Newton-Schulz without refinement: its error is reported, not held
        # to the mixed path's 1e-7
        f32 = other_path("fp32", 0)
        f32["speedup_mixed_vs_fp32"] = f32["s_per_build"] / value
        line["fp32_path"] = f32
    # ---- submatrices shared by k-means groups of block columns (Section IV-C) ----
    if args.group_size > 1 and args.prec == "mixed" and world == 1 and not columns:
        from paper_2004_10811_gb300 import grouping
        t0 = time.perf_counter()
        groups = grouping.periodic_kmeans(m.coords, m.box, max(1, m.nblk // args.group_size), seed=1)
        t_km = time.perf_counter() - t0
        single_dims = sub["dims"]
        gdims, _gl = grouping.group_dims(m.block_sizes, m.row_ptr, m.col_idx, groups)
        with pkg.Plan.from_bsr(m, prec="mixed", groups=groups, timing=True, tile_n_ns=plan_tiles[0],
                               tile_n_corr=plan_tiles[1], tile_n_hp=plan_tiles[2]) as pg:
            Dg = torch.empty_like(K)
            pg.sign(K, m.mu, out=Dg)
            torch.cuda.synchronize()
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            reps = 2
            g0.record(stream)
            for _ in range(reps):
                pg.sign(K, m.mu, out=Dg)
            g1.record(stream)
            torch.cuda.synchronize()
            tg = g0.elapsed_time(g1) / 1e3 / reps
            sg = pg.stats()
        gline = {"group_size": args.group_size, "submatrices": int(groups.max()) + 1,
                 "sub_dim_min": int(gdims.min()), "sub_dim_max": int(gdims.max()),
                 "s_per_build": tg, "speedup_vs_single_columns": value / tg,
                 "estimated_speedup_sum_n3": grouping.estimated_speedup(single_dims, gdims),
                 "kmeans_s": round(t_km, 2), "iters_max": int(sg["iters_max"]),
                 "fp64_fallback_submatrices": int(sg["refine_fallback"])}
        if not args.no_cpu:
            import oracle
            sample = np.linspace(0, groups.max(), 16).astype(int)
            wantg = oracle.density_matrix_grouped(m, m.mu, groups, only=sample)
            mk = ~np.isnan(wantg)
            gline["max_abs_err_vs_grouped_oracle"] = float(np.max(np.abs(Dg.cpu().numpy()[mk] - wantg[mk])))
            gline["parity_sample"] = f"{len(sample)} of {int(groups.max()) + 1} groups"
        line["grouped"] = gline

    # ---- finite temperature: D = f(K - mu I) with the Fermi function (Section IV-F) ----
    if args.kT > 0 and args.prec == "mixed" and world == 1 and not columns:
        ft = {"kT": args.kT}
        for prec in ("fp32", "fp64"):
            # FP64 over a contiguous chunk of 1/16 of the block columns (a
            # whole build at FP64 rates takes minutes)
            nc = max(1, m.nblk // 16) if prec == "fp64" and m.nblk >= 32 else 0
            with pkg.Plan.from_bsr(m, prec=prec, kT=args.kT, columns=(0, nc) if nc else None) as pt:
                Dt = torch.zeros_like(K)
                pt.sign(K, m.mu, out=Dt)  # warm-up: workspace and polynomial
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pt.sign(K, m.mu, out=Dt)
                e1.record(stream)
                torch.cuda.synchronize()
                tt = e0.elapsed_time(e1) / 1e3
                st_t = pt.stats()
                mu_t = None
                if args.mu_search and prec == "fp32":
                    # Newton on the smooth N(mu), started 0.5 above mu (FP32 traces: tol 1e-6)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    try:
                        mu_f, _Dt, status_t = pt.mu_search(K, m.n_el, mu0=m.mu + 0.5, tol=1e-6, max_steps=40,
                                                           out=Dt)
                    except pkg.SubmatError as exc:  # reported, not fatal to the line
                        mu_f, status_t = None, str(exc)
                    torch.cuda.synchronize()
                    tm_t = time.perf_counter() - t0
                    mu_t = {"mu0": m.mu + 0.5, "mu": mu_f, "status": status_t, "s_total": tm_t,
                            "evaluations": int(pt.stats()["mu_steps"]), "builds_equivalent": tm_t / tt}
            leg = {"poly_degree": int(st_t["poly_degree"]), "poly_trunc": float(st_t["poly_trunc"]),
                   "dn_dmu": float(st_t["dn_dmu"])}
            if mu_t is not None:
                leg["mu_search"] = mu_t
            if nc:
                sub_n3 = float(np.sum(sub["dims"].astype(np.float64) ** 3))
                chunk_n3 = float(np.sum(sub["dims"][:nc].astype(np.float64) ** 3))
                leg.update(chunk_s=tt, s_per_build_est=tt * sub_n3 / chunk_n3,
                           measured=f"block columns [0, {nc}) timed, scaled by sum n^3")
            else:
                leg.update(s_per_build=tt, measured="one whole build (every block column), CUDA events")
            if not args.no_cpu:
                import oracle
                tcols = sample_columns(nc if nc else m.nblk, 12)
                wantt = oracle.density_matrix_T(m, m.mu, args.kT, columns=tcols, workers=host_cores()[0])
                mk = ~np.isnan(wantt)
                leg["max_abs_err_vs_oracle"] = float(np.max(np.abs(Dt.cpu().numpy()[mk] - wantt[mk])))
                leg["parity_sample"] = f"{len(tcols)} block columns"
            ft[prec] = leg
        line["finite_t"] = ft

    # ---- the adjoint (vector-Jacobian product) on a contiguous chunk of block columns ----
    if args.adjoint_sample > 0 and world == 1 and not columns:
        nc = min(args.adjoint_sample, m.nblk)
        rng = np.random.default_rng(20041)
        dbar_h = rng.standard_normal(m.vals.shape)
        Dbar = torch.from_numpy(dbar_h).to(dev)
        sub_n3 = float(np.sum(sub["dims"].astype(np.float64) ** 3))
        chunk_n3 = float(np.sum(sub["dims"][:nc].astype(np.float64) ** 3))
        want = None
        pc = min(4, nc)
        if not args.no_cpu and rank == 0:
            import oracle
            want, _ = oracle.sign_backward(m, dbar_h, m.mu, columns=range(pc))
        # mode 0: SIMT GEMM in the plan's precision; mode 1 (mixed plans): tensor cores
        for mode in ((0, 1) if args.prec == "mixed" else (0,)):
            with pkg.Plan.from_bsr(m, prec=args.prec, columns=(0, nc), timing=True, adjoint_mode=mode) as pa:
                Kbar = torch.empty_like(K)
                pa.sign_backward(K, m.mu, Dbar, out=Kbar)  # warm-up: the adjoint's workspace
                torch.cuda.synchronize()
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                pa.sign_backward(K, m.mu, Dbar, out=Kbar)
                a1.record(stream)
                torch.cuda.synchronize()
                ta = a0.elapsed_time(a1) / 1e3
                sa = pa.stats()
                suba = pa.sub_stats()
            if mode == 0:
                cls = 2
                adj_prec = "fp64" if args.prec == "fp64" else "fp32"
                peak = FP64_NOMINAL_GFLOPS / 1e3 if adj_prec == "fp64" else FP32_NOMINAL_GFLOPS / 1e3
                roof = {"kernel": "k_gemm_simt", "bound": "alu", "peak": peak,
                        "peak_source": "nominal FP64" if adj_prec == "fp64" else
                        "nominal FP32 (152 SMs x 128 lanes x 2 x 2.07 GHz)"}
            else:
                cls = 5
                adj_prec = "bf16x3"
                roof = {"kernel": "k_tc_gemm", "bound": "tensor", "peak": peaks["bf16_tflops_sustained"],
                        "peak_source": peak_src + " (bf16 sustained)"}
            k_s = sa["kernel_ms"][cls] / 1e3
            achieved = sa["kernel_work"][cls] / k_s / 1e12
            roof.update(achieved=achieved, unit="TFLOP/s", frac=achieved / roof["peak"])
            if mode == 1:
                roof["executed_frac"] = sa["kernel_exec"][cls] / k_s / 1e12 / roof["peak"]
            adj = {"prec": adj_prec, "gemm": "SIMT" if mode == 0 else "tcgen05",
                   "sample": f"block columns [0, {nc}) timed, scaled by sum n^3",
                   "chunk_s": ta, "s_per_build_est": ta * sub_n3 / chunk_n3,
                   "iters_max": int(suba["iters"][:nc].max()), "tflops": sa["flops_ns"] / ta / 1e12,
                   "roofline": roof}
            if want is not None:
                # parity on a few of the timed columns against the oracle's Daleckii-Krein gradient
                with pkg.Plan.from_bsr(m, prec=args.prec, columns=(0, pc), adjoint_mode=mode) as pp:
                    got = pp.sign_backward(K, m.mu, Dbar).cpu().numpy()
                adj["max_rel_err_vs_oracle"] = float(np.max(np.abs(got - want)) / np.max(np.abs(want)))
                adj["parity_sample"] = f"block columns [0, {pc})"
            line["adjoint" if mode == 0 else "adjoint_tc"] = adj

    if mu_line is not None:
        line["mu_search"] = mu_line
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
