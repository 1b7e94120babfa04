"""Benchmark: global-coarsening matrix-free multigrid on one GB300 per rank.

Workload: Poisson -Lap u = f on [0,1]^3, Q4, one cell refined globally 5
times and twice more in the octant x, y, z < 1/2 (296,535 cells, 8 levels,
18,740,987 free DoFs), f = seeded Gaussian random field (8 Fourier modes,
seed 2203).

One step = one pass of the whole hot path: CG in fp64 preconditioned by one
fp32 V-cycle per iteration (Chebyshev(3)/Jacobi smoothing, residual,
restriction, exact level-0 solve, prolongation on every level), from x = 0 to
a relative residual of 1e-8, with b already resident in HBM.

value = fine-level fp32 operator throughput n_free / t_vmult (GDoF/s),
t_vmult = mean duration of the 48 fine-level operator applications of one
solve, from CUDA events on the library's stream (event-record nodes in the
captured graphs) in a profiled solve after the timed region; ms_per_step is
the time of the timed solves, which run without those timers.  Solve times of the
mixed (fp32 V-cycle) and plain fp64 (fp64 V-cycle) variants are reported
beside it, and two further parts of the method:

* learned: the per-cell network smoother trained on the GPU from the plain
  solver's V-cycle states (8 training right-hand sides), then the A/B
  comparison of time to 1e-8 with Chebyshev only / Chebyshev plus the
  learned step / the learned step instead of postsmoothing; the variant kept
  is the fastest that converges;
* batch: 256 independent problems of uneven degree and size (degree 1..4,
  depth 2..5, 0..2 octant levels, Fourier right-hand sides, one SplitMix64
  stream with seed 12292), operator tile size and thread mapping from the
  autotuner, solved to 1e-8 by one CUDA-graph launch.

Under torchrun every rank solves its own copy (replicas, weak scaling);
value sums the ranks.

--impl reference times the oracle (plain CPU implementation, test
infrastructure) on a bounded sample of the workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = synth.WORKLOAD_Q4_OCTANT
METRIC = "fine-level vmult GDoF/s; solve time to 1e-8 rel. res., mixed/learned vs FP64"
# algorithmic bytes per DoF of one operator application: source and
# destination vector plus the per-cell metadata (roofline model of the
# workload, per free DoF)
BYTES_PER_DOF = {"fp32": 9.8, "fp64": 17.8}
# DRAM bytes (read + write) of one fine-level fp32 operator application on
# this workload, both of its launches (tile kernel vmult_lines<4,float,4>:
# 135.1 MB read + 58.7 MB written; halo pass: 90.4 MB + 3.3 MB), from the
# ncu capture summarised in profiles/vmult_lines_q4_octant_fp32.md; set to 0
# (reported as null) when the kernel changes until it is re-captured
VMULT_TRAFFIC_BYTES = 287.5e6
SAMPLE = synth.cube_octant(4, 2)  # 1/8 of the workload's cells, same recipe family


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def oracle_vmult_sample(seconds: float = 6.0):
    """Time the oracle's fp64 cell-by-cell operator on the sample mesh."""
    from oracle import mesh as omesh, space as ospace

    s = ospace.Space(omesh.build_mesh(SAMPLE), WORKLOAD.degree)
    x = synth.point_values(s.free_coordinates(), 1)
    s.apply(x)
    reps, t0 = 0, time.perf_counter()
    while True:
        s.apply(x)
        reps += 1
        el = time.perf_counter() - t0
        if el > seconds:
            break
    cores = os.cpu_count() or 1
    return {"value": s.n_free * reps / el / 1e9, "unit": "GDoF/s", "cores": cores, "kind": "oracle",
            "sample": f"fp64 cell-by-cell operator of the oracle on {SAMPLE.name} (Q4, {s.nc} cells, "
                      f"{s.n_free} free DoFs, 1/8 of the workload), {reps} applications"}


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the
    timed region (read only)."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.proc = None
        self.device = device

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.5)  # nvidia-smi is up and sampling before the timed region starts
        except Exception:
            self.proc = None

    def stop(self, t0: float, t1: float):
        """Samples stamped within [t0, t1] (host epoch seconds, the timed
        region) widened by one sampling interval; without any, the nearest."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=10)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return self.parse(out, t0, t1)

    @staticmethod
    def parse(out: str, t0: float, t1: float, interval: float = 0.05):
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                day, frac = parts[0].rsplit(".", 1) if "." in parts[0] else (parts[0], "0")
                ts = time.mktime(time.strptime(day, "%Y/%m/%d %H:%M:%S")) + float("0." + frac)
            except ValueError:
                ts = None  # an unknown stamp format: the sample counts as inside
            try:
                rows.append((ts, float(parts[1]), float(parts[2]),
                             [nm for nm, v in zip(names, parts[5:9]) if v.lower() == "active"]))
            except ValueError:
                continue
        inside = [r for r in rows if r[0] is None or t0 - interval <= r[0] <= t1 + interval]
        if not inside and rows:
            mid = 0.5 * (t0 + t1)
            inside = [min(rows, key=lambda r: abs(r[0] - mid))]
        sm = [r[1] for r in inside]
        reasons = sorted({nm for r in inside for nm in r[3]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": inside[-1][2] if inside else None,
                "reasons": reasons, "samples": len(inside), "samples_total": len(rows)}


def run_reference(args, rank):
    if rank != 0:
        return
    t0 = time.perf_counter()
    from oracle import mesh as omesh, space as ospace

    s = ospace.Space(omesh.build_mesh(SAMPLE), WORKLOAD.degree)
    x = synth.point_values(s.free_coordinates(), 1)
    for _ in range(args.warmup):
        s.apply(x)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        s.apply(x)
        times.append(time.perf_counter() - t)
    ms = 1e3 * float(np.mean(times))
    value = s.n_free / (ms * 1e-3) / 1e9
    cores = os.cpu_count() or 1
    line = {"metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"oracle sample: {SAMPLE.name}, Q4, {s.nc} cells, {s.n_free} free DoFs "
                                   f"(1/8 of {WORKLOAD.name})"},
            "cpu_baseline": {"value": value, "unit": "GDoF/s", "cores": cores, "kind": "oracle",
                             "sample": f"one fp64 operator application per step on {SAMPLE.name}"},
            "e2e": {"value": value, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "setup_s": time.perf_counter() - t0}
    print(json.dumps(finite(line), allow_nan=False), flush=True)


def run_learned(g, mg, mg64):
    """Train the learned smoother on the GPU and compare time to 1e-8."""
    import torch
    from paper_2203_12292_gb300 import learned as lrn

    tr = lrn.train(mg64, epochs=100)
    cmp = lrn.compare(mg, tr.net, rhs_seed=WORKLOAD.rhs_seed, rtol=1e-8, repeats=2, maxit=60)
    mg.set_smoother(mg.finest, g.SMOOTHER_CHEBYSHEV)
    return {"train_rows": tr.n_train, "val_rows": tr.n_val, "val_loss": tr.val_mse,
            "val_loss_zero_correction": tr.val_mse_zero, "val_loss_initial_network": tr.val_mse_init,
            "data_s": tr.seconds_data, "train_s": tr.seconds_train,
            "variants": [v.__dict__ for v in cmp["variants"]], "kept": cmp["kept"],
            "network": "250-128-128-125 GELU, bf16 operands, fp32 accumulation"}


def run_batch(g, seed: int = 12292, n: int = 256):
    """256 uneven problems solved to 1e-8 by one graph launch."""
    import torch

    rec = synth.batch_recipes(seed, n)
    t0 = time.perf_counter()
    meshes = {}
    for k, d, e, _ in rec:
        if (d, e) not in meshes:
            meshes[(d, e)] = g.Mesh.from_recipe(synth.cube_octant(d, e))
    # probe large enough that every candidate tile size is kept on its finest
    # level (61,440 cells; smaller levels halve their tiles)
    probe = g.Mesh.from_recipe(synth.cube_octant(5, 1))
    tuning = {}
    for k in sorted({r[0] for r in rec}):
        best, _ = g.autotune(probe, k, True, 10)
        tuning[k] = best
    t1 = time.perf_counter()
    cfgs = [g.make_config(k, mg_fp32=True, tile_cells=tuning[k].tile_cells, cell_kernel=tuning[k].cell_kernel)
            for k, _, _, _ in rec]
    B = g.Batch([meshes[(d, e)] for _, d, e, _ in rec], cfgs)
    t2 = time.perf_counter()
    bs = []
    for i, (_, _, _, s) in enumerate(rec):
        f = synth.fourier_rhs(s)
        bs.append(B.problems[i].rhs((f.kappa, f.phi, f.amp)))
    xs = [torch.zeros_like(b) for b in bs]
    dofs = int(sum(b.numel() for b in bs))
    st = B.cg_solve(bs, xs, 1e-8, 100)  # builds and launches the graph
    torch.cuda.synchronize()
    launches0 = g.launch_count()
    times = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(B.stream)
        st = B.cg_solve(bs, xs, 1e-8, 100)
        e1.record(B.stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    its = [s_.iterations for s_ in st]
    out = {"problems": n, "dofs": dofs, "solve_ms": ms, "solve_ms_all": times,
           "gdofs_solved_per_s": dofs / (ms * 1e-3) / 1e9, "iterations_min": min(its), "iterations_max": max(its),
           "all_converged": all(s_.status == 0 for s_ in st), "graph_launches_per_solve": 1,
           "kernels_per_solve": (g.launch_count() - launches0) // 3,
           "tuning": {k: {"tile_cells": t.tile_cells, "cell_kernel": t.cell_kernel, "gdofs": t.gdofs}
                      for k, t in tuning.items()},
           "tune_s": t1 - t0, "setup_s": t2 - t1}
    del B
    return out


def finite(v):
    """The JSON line with non-finite numbers (a diverged variant) as null."""
    if isinstance(v, float):
        return v if np.isfinite(v) else None
    if isinstance(v, dict):
        return {k: finite(x) for k, x in v.items()}
    if isinstance(v, (list, tuple)):
        return [finite(x) for x in v]
    return v


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gcmg", choices=["gcmg", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-graphs", action="store_true",
                    help="stream launches instead of CUDA graphs (for per-kernel profiler launch lists)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps")

    import torch

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_2203_12292_gb300 import build as gbuild

    if rank == 0:
        gbuild.build()
    barrier()
    import paper_2203_12292_gb300 as g

    # cpu baseline first (no GPU work in flight), rank 0 only
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_vmult_sample()

    t0 = time.perf_counter()
    mesh = g.Mesh.from_recipe(WORKLOAD.recipe)
    mg = g.Multigrid(mesh, WORKLOAD.degree, mg_fp32=True)
    if args.no_graphs:
        mg.set_graphs(False)
    setup_s = time.perf_counter() - t0
    L = mg.finest
    n = mg.n_free(L)
    f = synth.fourier_rhs(WORKLOAD.rhs_seed)
    b = mg.rhs((f.kappa, f.phi, f.amp))
    x = torch.zeros_like(b)
    stream = mg.stream

    def step():
        return mg.cg_solve(b, x, 1e-8, 100)

    for _ in range(args.warmup):
        st = step()
    torch.cuda.synchronize()
    launches0 = g.launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_region0 = time.time()
    e0.record(stream)
    iters = []
    for _ in range(args.steps):
        st = step()
        iters.append(st.iterations)
    e1.record(stream)
    torch.cuda.synchronize()
    t_region1 = time.time()
    barrier()
    clk = clocks.stop(t_region0, t_region1)
    launches = g.launch_count() - launches0
    ms_total = e0.elapsed_time(e1)
    if dist is not None:
        t = torch.tensor([ms_total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    # one more solve with the per-level, per-stage timers (event nodes in the
    # graphs): the duration of every fine-level operator application and the
    # time split; the timed solves above run without timers
    mg.set_profiling(True)
    step()
    torch.cuda.synchronize()
    cnt, vms = mg.profile(L, "vmult")
    cnt64, vms64 = mg.profile(L, "cg_vmult")
    stage_ms = {s: mg.profile(L, s)[1] for s in g.STAGES}
    coarse_ms = sum(mg.profile(l, s)[1] for l in range(L) for s in g.STAGES)
    per_level = []
    for l in range(mg.num_levels):
        row = {"level": l, "n_free": mg.n_free(l), "cells": mg.level_info(l).n_cells}
        for s_ in ("vmult", "presmooth", "residual", "restrict", "coarse", "prolongate", "postsmooth"):
            c_, m_ = mg.profile(l, s_)
            row[s_ + "_ms"] = m_
            if s_ == "vmult":
                row["vmult_calls"] = c_
        per_level.append(row)
    mg.set_profiling(False)
    t_vmult = vms / cnt  # ms
    value = n / (t_vmult * 1e-3) / 1e9
    value64 = n / (vms64 / cnt64 * 1e-3) / 1e9
    if dist is not None:
        t = torch.tensor([value], device="cuda", dtype=torch.float64)
        dist.all_reduce(t)
        value = float(t.item())

    # plain fp64 variant (fp64 V-cycle) of the same solve
    mg64 = g.Multigrid(mesh, WORKLOAD.degree, mg_fp32=False)
    if args.no_graphs:
        mg64.set_graphs(False)
    x64 = torch.zeros_like(b)
    mg64.cg_solve(b, x64, 1e-8, 100)
    torch.cuda.synchronize()
    e0.record(stream)
    st64 = mg64.cg_solve(b, x64, 1e-8, 100)
    e1.record(stream)
    torch.cuda.synchronize()
    fp64_ms = e0.elapsed_time(e1)
    sol_diff = float(torch.linalg.norm(x - x64) / torch.linalg.norm(x64))

    learned = None
    if not args.no_learned:
        learned = run_learned(g, mg, mg64)
    del mg64

    # end to end through the C ABI with pinned host buffers
    hsrc = torch.empty(n, dtype=torch.float32, pin_memory=True)
    hdst = torch.empty(n, dtype=torch.float32, pin_memory=True)
    hsrc.copy_(torch.from_numpy(synth.uniform_vector(n, 3).astype(np.float32)))
    hs, hd = hsrc.numpy(), hdst.numpy()
    for _ in range(2):
        mg.vmult_host(L, hs, hd)
    reps = max(args.steps, 5)
    t = time.perf_counter()
    for _ in range(reps):
        mg.vmult_host(L, hs, hd)
    e2e_s = (time.perf_counter() - t) / reps

    batch = None
    if not args.no_batch:
        batch = run_batch(g)

    hbm, peak_kind = peaks()
    achieved = BYTES_PER_DOF["fp32"] * n / (t_vmult * 1e-3) / 1e9
    traffic = VMULT_TRAFFIC_BYTES if VMULT_TRAFFIC_BYTES > 0 else None
    if rank == 0:
        res = {
            "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 V-cycle / f64 CG", "data": "synthetic",
            "config": {"workload": WORKLOAD.name, "degree": WORKLOAD.degree, "cells": mg.level_info(L).n_cells,
                       "n_free": n, "levels": mg.num_levels, "rhs": "8 Fourier modes, seed 2203",
                       "rtol": 1e-8, "l2": "inputs larger than L2 (finest level vectors and metadata > 129 MB)",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "kernel": "vmult_lines<4,float,4> line-parallel tile kernel + halo pass "
                                   "(fine-level fp32 operator, 32-cell tiles)",
                         "peak_kind": peak_kind, "bytes_per_dof": BYTES_PER_DOF["fp32"],
                         "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the tile kernel "
                                           "and the halo pass, one application on this workload"},
            "cpu_baseline": cpu,
            "e2e": {"value": n / e2e_s / 1e9, "unit": "GDoF/s", "h2d_bytes_per_step": 4 * n,
                    "d2h_bytes_per_step": 4 * n, "call": "gcmg_vmult_host, pinned host buffers, fp32"},
            "gpu_launches": launches,
            "clocks": clk,
            "solve": {"mixed_ms": ms_step, "mixed_iterations": iters[-1], "mixed_rel_residual": st.rel_residual,
                      "fp64_ms": fp64_ms, "fp64_iterations": st64.iterations,
                      "fp64_rel_residual": st64.rel_residual, "speedup_mixed_vs_fp64": fp64_ms / ms_step,
                      "solution_rel_diff_mixed_vs_fp64": sol_diff},
            "vmult": {"fp32_ms": t_vmult, "fp32_gdofs": value / world, "fp64_ms": vms64 / cnt64,
                      "fp64_gdofs": value64},
            "stage_ms_per_step_finest": stage_ms, "coarser_levels_ms_per_step": coarse_ms,
            "per_level_ms_per_step": per_level,
            "setup_s": setup_s,
            "learned": learned,
            "batch": batch,
        }
        print(json.dumps(finite(res), allow_nan=False), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
