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
t_vmult = mean duration of 50 complete operator applications (tile kernel
and halo pass) through gcmg_vmult, CUDA events on the library's stream, after
warm-up; ms_per_step is the time of the timed solves.  Solve times of the
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

Beside it: the fp32 and fp64 operators' fractions of the measured HBM
bandwidth and of the measured CUDA-core peak (an FMA microbenchmark of the
library), the V-cycle throughput, the same solve on the other two workloads
of this path (Q2 octant, f = 1, fp64 multigrid; Q4 sphere with p-coarsening
4 -> 2 -> 1, f = 1), and the oracle's single-threaded timings (operator,
V-cycle, PCG) on samples of the workload as the CPU baseline.

--impl reference times the oracle (plain CPU implementation, test
infrastructure) on a bounded sample of the workload on one host core.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

# the oracle's timings (the reference arm and the CPU baseline) run its numpy
# code on one thread: fix the thread count before numpy loads its BLAS
if "--oracle-timings" in sys.argv or ("--impl" in sys.argv and "reference" in sys.argv):
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

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
# this workload, both of its launches, from one ncu capture of
# dram__bytes_read.sum + dram__bytes_write.sum with caches flushed before each
# kernel (ncu's default), mean of two applications: tile kernel vmult_lanes<4>
# 136.9 MB read + 56.5 MB written, halo pass 89.8 MB + 0.7 MB; set to 0
# (reported as null) when the kernels change until they are captured again
VMULT_TRAFFIC_BYTES = 283.8e6
# V-cycle bytes per finest-level DoF (fp32): six operator applications and
# five vector updates per level, the transfers, summed over the levels with
# the 1/(1 - 1/8) factor of the coarser levels
VCYCLE_BYTES_PER_DOF = 250.0
SAMPLE = synth.cube_octant(4, 2)  # 1/8 of the workload's cells, same recipe family
SAMPLE_MG = synth.cube_octant(3, 2)  # 1/64 of the cells: the oracle's V-cycle and PCG


def flops_per_cell(k: int) -> int:
    """Algorithmic flops of one cell of the fast-diagonalisation operator:
    six 1D even-odd transforms on (k+1)^2 lines each (fold: 2 floor(n/2)
    adds; symmetric modes: ceil(n/2) rows of 2 ceil(n/2) - 1 flops;
    antisymmetric: floor(n/2) rows of 2 floor(n/2) - 1), and one scaling per
    node (a multiply-add counts two; Q4: 3,875)."""
    n = k + 1
    nh, ne = n // 2, (n + 1) // 2
    f1d = 2 * nh + ne * (2 * ne - 1) + nh * (2 * nh - 1)
    return 6 * n * n * f1d + n ** 3


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def oracle_timings():
    """The oracle as it stands, on one thread (set before numpy loads): its
    fp64 cell-by-cell operator on SAMPLE, and one V-cycle and the PCG solve to
    1e-8 on SAMPLE_MG (fp64 multigrid, f = the workload's Fourier field).
    Runs in a child process of bench.py (--oracle-timings)."""
    from oracle import mesh as omesh, mg as omg, space as ospace

    t0 = time.perf_counter()
    s = ospace.Space(omesh.build_mesh(SAMPLE), WORKLOAD.degree)
    x = synth.point_values(s.free_coordinates(), 1)
    s.apply(x)
    reps, t = 0, time.perf_counter()
    while True:
        s.apply(x)
        reps += 1
        el = time.perf_counter() - t
        if el > 5.0:
            break
    out = {"vmult": {"gdofs": s.n_free * reps / el / 1e9, "ms": 1e3 * el / reps, "n_free": s.n_free,
                     "cells": s.nc, "reps": reps, "mesh": SAMPLE.name}}
    levels = omg.build_levels(omesh.build_mesh(SAMPLE_MG), WORKLOAD.degree, assembled=False)
    sp = levels[-1].space
    f = synth.fourier_rhs(WORKLOAD.rhs_seed)
    b = sp.rhs(ospace.fourier_function(f))
    omg.multigrid_vcycle(levels, b)
    t = time.perf_counter()
    for _ in range(3):
        omg.multigrid_vcycle(levels, b)
    vc = (time.perf_counter() - t) / 3
    t = time.perf_counter()
    r = omg.solve(levels, b, 1e-8)
    cg = time.perf_counter() - t
    out["vcycle"] = {"ms": 1e3 * vc, "gdofs": sp.n_free / vc / 1e9, "n_free": sp.n_free, "mesh": SAMPLE_MG.name}
    out["pcg"] = {"ms": 1e3 * cg, "iterations": r.iterations, "gdofs_solved": sp.n_free / cg / 1e9,
                  "n_free": sp.n_free, "mesh": SAMPLE_MG.name, "rtol": 1e-8}
    out["threads"] = 1
    out["seconds"] = time.perf_counter() - t0
    return out


def cpu_baseline_line():
    """cpu_baseline of the JSON line: the oracle's timings from a child
    process pinned to one thread."""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-timings"], capture_output=True,
                       text=True, timeout=900)
    if r.returncode != 0:
        return {"value": None, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
                "sample": "oracle timings failed: " + r.stderr.strip().splitlines()[-1][:200]}
    o = json.loads(r.stdout.strip().splitlines()[-1])
    v = o["vmult"]
    return {"value": v["gdofs"], "unit": "GDoF/s", "cores": 1, "kind": "oracle",
            "sample": f"fp64 cell-by-cell operator of the oracle on {v['mesh']} (Q4, {v['cells']} cells, "
                      f"{v['n_free']} free DoFs, 1/8 of the workload), {v['reps']} applications, one thread "
                      f"(OMP/OpenBLAS/MKL threads = 1)",
            "vcycle": o["vcycle"], "pcg": o["pcg"], "seconds": o["seconds"]}


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
    cores = 1  # OMP/OpenBLAS/MKL threads fixed to 1 before numpy was loaded
    line = {"metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"oracle sample: {SAMPLE.name}, Q4, {s.nc} cells, {s.n_free} free DoFs "
                                   f"(1/8 of {WORKLOAD.name})"},
            "cpu_baseline": {"value": value, "unit": "GDoF/s", "cores": cores, "kind": "oracle",
                             "sample": f"one fp64 operator application per step on {SAMPLE.name}, one thread"},
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
    tuning, tried = {}, {}
    for k in sorted({r[0] for r in rec}):
        best, allc = g.autotune(probe, k, True, 10)
        tuning[k] = best
        tried[k] = [{"tile_cells": t.tile_cells, "cell_kernel": t.cell_kernel, "cell_threads": t.cell_threads,
                     "gdofs": t.gdofs} for t in allc]
    t1 = time.perf_counter()
    cfgs = [g.make_config(k, mg_fp32=True, tile_cells=tuning[k].tile_cells, cell_kernel=tuning[k].cell_kernel,
                          cell_threads=tuning[k].cell_threads)
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
           "tuning": {k: {"tile_cells": t.tile_cells, "cell_kernel": t.cell_kernel, "cell_threads": t.cell_threads,
                          "gdofs": t.gdofs} for k, t in tuning.items()},
           "tuning_candidates": tried,
           "tune_s": t1 - t0, "setup_s": t2 - t1}
    # the same batch in one persistent kernel (device work list, lockstep over the problems)
    xp = [torch.zeros_like(b) for b in bs]
    try:
        t3 = time.perf_counter()
        stp = B.cg_solve(bs, xp, 1e-8, 100, persistent=True)  # records the work list, launches it
        torch.cuda.synchronize()
        build_s = time.perf_counter() - t3
        ptimes = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(B.stream)
            stp = B.cg_solve(bs, xp, 1e-8, 100, persistent=True)
            e1.record(B.stream)
            torch.cuda.synchronize()
            ptimes.append(e0.elapsed_time(e1))
        info = B.persistent_info()
        pms = float(np.median(ptimes))
        diff = max(float((a - c).norm() / max(float(c.norm()), 1e-300)) for a, c in zip(xp, xs) if c.numel())
        out["persistent"] = {
            "solve_ms": pms, "solve_ms_all": ptimes, "gdofs_solved_per_s": dofs / (pms * 1e-3) / 1e9,
            "kernels_per_solve": 1, "in_graph": bool(info.in_graph), "ctas": info.grid,
            "smem_bytes": info.smem_bytes, "work_list_ops": info.ops, "lockstep_steps": info.steps,
            "record_and_first_solve_s": build_s,
            "iterations_min": min(s_.iterations for s_ in stp), "iterations_max": max(s_.iterations for s_ in stp),
            "all_converged": all(s_.status == 0 for s_ in stp),
            "max_rel_diff_vs_graph_batch": diff}
    except Exception as exc:  # reported, not fatal: the graph batch above is the reference
        out["persistent"] = {"error": str(exc)}
    del B
    return out


def time_solves(mg, b, reps: int = 5):
    """median time (ms) of reps CG solves to 1e-8 after warm-up, and the last stats"""
    import torch

    x = torch.zeros_like(b)
    for _ in range(3):
        st = mg.cg_solve(b, x, 1e-8, 100)
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(mg.stream)
        st = mg.cg_solve(b, x, 1e-8, 100)
        e1.record(mg.stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return float(np.median(times)), st, x


def time_vcycle(mg, b, reps: int = 20):
    """mean time (ms) of one V-cycle (Algorithms 1-2, captured graph) of the handle"""
    import torch

    x = torch.zeros_like(b)
    for _ in range(3):
        mg.vcycle(b, x)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(mg.stream)
    for _ in range(reps):
        mg.vcycle(b, x)
    e1.record(mg.stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def per_level_profile(g, mg, b):
    """one profiled solve: per level the stage times (ms) and the finest operator's mean time"""
    import torch

    x = torch.zeros_like(b)
    mg.set_profiling(True)
    mg.cg_solve(b, x, 1e-8, 100)
    torch.cuda.synchronize()
    rows = []
    for l in range(mg.num_levels):
        row = {"level": l, "n_free": mg.n_free(l), "cells": mg.level_info(l).n_cells,
               "degree": mg.level_info(l).degree}
        for s_ in ("vmult", "presmooth", "residual", "restrict", "coarse", "prolongate", "postsmooth"):
            row[s_ + "_ms"] = mg.profile(l, s_)[1]
        rows.append(row)
    cnt, vms = mg.profile(mg.finest, "vmult")
    mg.set_profiling(False)
    return rows, (vms / cnt if cnt else None)


def run_other_config(g, w, hbm):
    """the same path on another workload of the configuration list: solve to
    1e-8 with the fp32 V-cycle and with the fp64 V-cycle, finest operator
    throughput, per-level times"""
    mesh = g.Mesh.from_recipe(w.recipe)
    out = {"workload": w.name, "degree": w.degree, "p_coarsening": bool(w.p_coarsening), "rhs": "f = 1"}
    for fp32 in (True, False):
        mg = g.Multigrid(mesh, w.degree, p_coarsening=w.p_coarsening, mg_fp32=fp32)
        b = mg.rhs()
        ms, st, _ = time_solves(mg, b)
        key = "mixed" if fp32 else "fp64"
        out[key + "_ms"] = ms
        out[key + "_iterations"] = st.iterations
        out[key + "_rel_residual"] = st.rel_residual
        rows, t_vm = per_level_profile(g, mg, b)
        n = mg.n_free(mg.finest)
        out["n_free"] = n
        out["cells"] = mg.level_info(mg.finest).n_cells
        out["levels"] = mg.num_levels
        out[key + "_vmult_ms"] = t_vm
        out[key + "_vmult_gdofs"] = n / (t_vm * 1e-3) / 1e9 if t_vm else None
        if fp32 and t_vm:
            out["fp32_vmult_hbm_frac"] = BYTES_PER_DOF["fp32"] * n / (t_vm * 1e-3) / 1e9 / hbm
        out[key + "_per_level"] = rows
        del mg
    out["speedup_mixed_vs_fp64"] = out["fp64_ms"] / out["mixed_ms"]
    out["fp64_arithmetic"] = "fp64 CG and vectors; operators in double-float (two fp32, about 48-bit significand)"
    return out


def ranks_max(dist, v: float, device: str) -> float:
    """The largest of the ranks' values (the timed region's milliseconds: the
    slowest replica sets the time)."""
    import torch

    t = torch.tensor([v], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def ranks_sum(dist, v: float, device: str) -> float:
    """The sum of the ranks' values (whole-job throughput of the replicas)."""
    import torch

    t = torch.tensor([v], device=device, dtype=torch.float64)
    dist.all_reduce(t)
    return float(t.item())


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
    ap.add_argument("--no-configs", action="store_true", help="skip the Q2 octant and Q4 sphere workloads")
    ap.add_argument("--oracle-timings", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_timings:
        print(json.dumps(oracle_timings()), flush=True)
        return
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
        cpu = cpu_baseline_line()
    # measured CUDA-core peaks (fp32, native fp64): denominators of the ALU fractions
    fma = {"fp32_tflops": g.fma_peak(False, 1 << 20), "fp64_tflops": g.fma_peak(True, 1 << 15),
           "how": "gcmg_fma_peak: 8 independent multiply-add chains per thread, 2048 threads per SM, CUDA events"}

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
    torch.cuda.nvtx.range_push("timed")  # lets a profiler select exactly the timed solves
    e0.record(stream)
    iters = []
    for _ in range(args.steps):
        st = step()
        iters.append(st.iterations)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    t_region1 = time.time()
    barrier()
    clk = clocks.stop(t_region0, t_region1)
    launches = g.launch_count() - launches0
    ms_total = e0.elapsed_time(e1)
    if dist is not None:
        ms_total = ranks_max(dist, ms_total, "cuda")
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
    t_vc = time_vcycle(mg, b)
    # the fine-level fp32 operator as one complete application (tile kernel and halo pass): 50
    # standalone applications, CUDA events, after warm-up
    xv = torch.tensor(synth.uniform_vector(n, 5).astype(np.float32), device="cuda")
    yv = torch.empty_like(xv)
    for _ in range(5):
        mg.vmult(L, xv, yv)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(50):
        mg.vmult(L, xv, yv)
    e1.record(stream)
    torch.cuda.synchronize()
    t_vmult = e0.elapsed_time(e1) / 50  # ms
    t_vmult_solve = vms / cnt  # the same from the in-solve event timers (graph event-record nodes)
    value = n / (t_vmult * 1e-3) / 1e9
    value64 = n / (vms64 / cnt64 * 1e-3) / 1e9
    if dist is not None:
        value = ranks_sum(dist, value, "cuda")

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

    # end to end through the C ABI with pinned host buffers: every step copies its input vector in
    # and its result out (gcmg_vmult_host_many: the copies of neighbouring steps overlap the operators)
    hsrc = [torch.empty(n, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    hdst = [torch.empty(n, dtype=torch.float32, pin_memory=True) for _ in range(2)]
    for i, h in enumerate(hsrc):
        h.copy_(torch.from_numpy(synth.uniform_vector(n, 3 + i).astype(np.float32)))
    reps = max(args.steps, 5)
    srcs = [hsrc[i % 2].numpy() for i in range(reps)]
    dsts = [hdst[i % 2].numpy() for i in range(reps)]
    mg.vmult_host_many(L, srcs[:4], dsts[:4])
    t = time.perf_counter()
    mg.vmult_host_many(L, srcs, dsts)
    e2e_s = (time.perf_counter() - t) / reps
    t = time.perf_counter()
    for _ in range(reps):
        mg.vmult_host(L, srcs[0], dsts[0])
    e2e_single_s = (time.perf_counter() - t) / reps

    batch = None
    if not args.no_batch:
        batch = run_batch(g)

    hbm, peak_kind = peaks()
    configs = None
    if not args.no_configs:
        configs = {"q2_octant": run_other_config(g, synth.WORKLOAD_Q2_OCTANT, hbm),
                   "q4_sphere_p": run_other_config(g, synth.WORKLOAD_Q4_SPHERE, hbm)}
    achieved = BYTES_PER_DOF["fp32"] * n / (t_vmult * 1e-3) / 1e9
    cells = mg.level_info(L).n_cells
    fpc = flops_per_cell(WORKLOAD.degree)
    tflops32 = fpc * cells / (t_vmult * 1e-3) / 1e12
    tflops64 = fpc * cells / (vms64 / cnt64 * 1e-3) / 1e12
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
                         "kernel": "vmult_lanes<4> one-lane-per-cell tile kernel + halo_add_kernel<float> "
                                   "(fine-level fp32 operator, 32-cell tiles)",
                         "peak_kind": peak_kind, "bytes_per_dof": BYTES_PER_DOF["fp32"],
                         "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the tile kernel "
                                           "and the halo pass, one application on this workload, caches "
                                           "flushed before each kernel",
                         "alu_frac": tflops32 / fma["fp32_tflops"], "alu_achieved_tflops": tflops32,
                         "alu_peak_tflops": fma["fp32_tflops"], "alu_peak_kind": "measured (gcmg_fma_peak, fp32)",
                         "flop_per_cell": fpc},
            "alu_peaks": fma,
            "vcycle": {"ms": t_vc, "gdofs": n / (t_vc * 1e-3) / 1e9, "bytes_per_dof": VCYCLE_BYTES_PER_DOF,
                       "roofline_gdofs": hbm / VCYCLE_BYTES_PER_DOF,
                       "frac": n / (t_vc * 1e-3) / 1e9 / (hbm / VCYCLE_BYTES_PER_DOF),
                       "what": "one fp32 V-cycle of the finest level (Algorithms 1-2, captured graph), "
                               "including the fp64 <-> fp32 copies"},
            "cpu_baseline": cpu,
            "e2e": {"value": n / e2e_s / 1e9, "unit": "GDoF/s", "h2d_bytes_per_step": 4 * n,
                    "d2h_bytes_per_step": 4 * n,
                    "call": "gcmg_vmult_host_many over the steps' vectors, pinned host buffers, fp32 (copies of "
                            "neighbouring steps overlap the operators)",
                    "one_vector_per_call_gdofs": n / e2e_single_s / 1e9},
            "gpu_launches": launches,
            "clocks": clk,
            "solve": {"mixed_ms": ms_step, "mixed_iterations": iters[-1], "mixed_rel_residual": st.rel_residual,
                      "fp64_ms": fp64_ms, "fp64_iterations": st64.iterations,
                      "fp64_rel_residual": st64.rel_residual, "speedup_mixed_vs_fp64": fp64_ms / ms_step,
                      "solution_rel_diff_mixed_vs_fp64": sol_diff,
                      "fp64_arithmetic": "fp64 CG, fp64 vectors on every level; the operators in double-float "
                                         "(two fp32 per value, about 48-bit significand)"},
            "vmult": {"fp32_ms": t_vmult, "fp32_gdofs": value / world, "fp32_tflops": tflops32,
                      "fp32_in_solve_ms": t_vmult_solve,
                      "fp64_ms": vms64 / cnt64, "fp64_gdofs": value64,
                      "fp64_arithmetic": "double-float (two fp32 per value, about 48-bit significand), fp64 "
                                         "vectors in and out, on the FP32 pipe",
                      "fp64_equiv_tflops": tflops64,
                      "fp64_frac_of_native_fp64_peak": tflops64 / fma["fp64_tflops"],
                      "fp64_frac_of_fp32_peak": tflops64 / fma["fp32_tflops"],
                      "fp64_hbm_frac": BYTES_PER_DOF["fp64"] * value64 / hbm},
            "configs": configs,
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
