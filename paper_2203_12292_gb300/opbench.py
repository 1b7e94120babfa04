"""Kernel microbenchmark: time one operation of one level.

    python -m paper_2203_12292_gb300.opbench [--workload q4octant] [--level -1]
        [--op vmult|restrict|prolong|mlp|diag|coarse|mlp_grad|batch_graph|batch_persistent]
        [--dtype f32|f64] [--reps 20] [--problems 16]
        [--tile-cells 0] [--cell-kernel 0|1|2|3] [--cell-threads 0] [--warp EPS]

vmult: the level's operator; restrict/prolong: the transfer between the
level and the next coarser one; mlp: the learned-smoother correction (Q4,
random initial network); diag: the level's Jacobi diagonal (Eqs. 3-4, the
per-mask table and the tile loop); coarse: the level-0 solve; mlp_grad: loss
and gradient of the Q4 network on 256 training rows (the tcgen05 products of
one training step); batch_graph / batch_persistent: CG to 1e-8 for the first
--problems problems of the benchmark's batch recipe, as one graph of kernels
or as one persistent kernel (the workload and level options do not apply to
these three).  The timed calls run inside an NVTX range named
"opbench", so a profiler can select exactly them.  Prints one JSON line
(ms per call, GDoF/s of the level's free DoFs).
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOADS = {"q4octant": synth.WORKLOAD_Q4_OCTANT, "q2octant": synth.WORKLOAD_Q2_OCTANT,
             "q4sphere": synth.WORKLOAD_Q4_SPHERE,
             "q4uniform": synth.Workload("Q4 uniform cube, 6 refinements (262,144 cells)", synth.uniform_cube(6), 4, 0)}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="q4octant", choices=sorted(WORKLOADS))
    ap.add_argument("--level", type=int, default=-1)
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--op", default="vmult", choices=["vmult", "restrict", "prolong", "mlp", "diag", "coarse",
                                                      "mlp_grad", "batch_graph", "batch_persistent"])
    ap.add_argument("--problems", type=int, default=16)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--tile-cells", type=int, default=0)
    ap.add_argument("--cell-kernel", type=int, default=0, choices=[0, 1, 2, 3])
    ap.add_argument("--cell-threads", type=int, default=0, choices=[0, 128, 256, 384, 512])
    ap.add_argument("--warp", type=float, default=None, help="cells mapped by the warp of this eps")
    a = ap.parse_args(argv)
    import torch

    import synth as sy

    from . import MLP, Mesh, Multigrid, build as b

    b.build()
    if a.op in ("mlp_grad", "batch_graph", "batch_persistent"):
        return _other_op(a)
    w = WORKLOADS[a.workload]
    mesh = Mesh.from_recipe(w.recipe)
    mg = Multigrid(mesh, w.degree, p_coarsening=w.p_coarsening, mg_fp32=True, tile_cells=a.tile_cells,
                   cell_kernel=a.cell_kernel, cell_threads=a.cell_threads)
    if a.warp is not None:
        from . import GEOM_WARP
        mg.set_geometry(GEOM_WARP, a.warp)
    lev = a.level if a.level >= 0 else mg.num_levels + a.level
    n = mg.n_free(lev)
    dt = torch.float32 if a.dtype == "f32" else torch.float64
    x = torch.rand(n, dtype=dt, device="cuda")
    y = torch.empty_like(x)
    xc = torch.rand(mg.n_free(max(lev - 1, 0)), dtype=dt, device="cuda")
    b0 = torch.rand(mg.n_free(0), dtype=dt, device="cuda")
    x0 = torch.empty_like(b0)
    if a.op == "mlp":
        net = MLP(*sy.mlp_shape(w.degree))
        net.set_params(torch.tensor(sy.mlp_init(*sy.mlp_shape(w.degree), 1), dtype=torch.float32, device="cuda"))

    def call():
        if a.op == "vmult":
            mg.vmult(lev, x, y)
        elif a.op == "restrict":
            mg.restrict_add(lev, x, xc)
        elif a.op == "prolong":
            mg.prolongate_add(lev, xc, y)
        elif a.op == "diag":
            mg.diagonal(lev)
        elif a.op == "coarse":
            mg.coarse_solve(b0, x0)
        else:
            mg.mlp_correct(lev, net, x, y)

    for _ in range(3):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("opbench")
    e0.record()
    for _ in range(a.reps):
        call()
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / a.reps
    info = mg.level_info(lev)
    print(json.dumps({"workload": w.name, "op": a.op, "level": lev, "dtype": a.dtype, "n_free": n,
                      "cells": info.n_cells,
                      "tiles": info.n_tiles, "halo_dofs": info.n_halo, "tile_cells": info.tile_cells,
                      "cell_kernel": a.cell_kernel, "cell_threads": a.cell_threads, "warp": a.warp,
                      "ms": ms, "gdofs": n / ms / 1e6}))


def _timed(call, reps):
    import torch
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("opbench")
    e0.record()
    for _ in range(reps):
        call()
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _other_op(a):
    import torch

    import synth as sy

    from . import MLP, Batch, Mesh, make_config
    if a.op == "mlp_grad":
        shape = sy.mlp_shape(4)
        net = MLP(*shape)
        net.set_params(torch.tensor(sy.mlp_init(*shape, 1), dtype=torch.float32, device="cuda"))
        rows = 256
        X = torch.tensor(sy.uniform_vector(rows * shape[0], 2).reshape(rows, shape[0]), dtype=torch.float32,
                         device="cuda")
        T = torch.tensor(sy.uniform_vector(rows * shape[2], 3).reshape(rows, shape[2]), dtype=torch.float32,
                         device="cuda")
        ms = _timed(lambda: net.gradient(X, T), a.reps)
        flops = 3 * 2 * rows * (shape[0] * shape[1] + shape[1] * shape[1] + shape[1] * shape[2])
        print(json.dumps({"op": a.op, "rows": rows, "network": list(shape), "ms": ms,
                          "gemm_tflops": flops / (ms * 1e-3) / 1e12}))
        return
    rec = sy.batch_recipes(12292, a.problems)
    meshes = [Mesh.from_recipe(sy.cube_octant(d, e)) for _, d, e, _ in rec]
    B = Batch(meshes, [make_config(k, mg_fp32=True) for k, _, _, _ in rec])
    bs = []
    for i, (_, _, _, seed) in enumerate(rec):
        f = sy.fourier_rhs(seed)
        bs.append(B.problems[i].rhs((f.kappa, f.phi, f.amp)))
    xs = [torch.zeros_like(v) for v in bs]
    persistent = a.op == "batch_persistent"
    ms = _timed(lambda: B.cg_solve(bs, xs, 1e-8, 100, persistent=persistent), a.reps)
    dofs = int(sum(v.numel() for v in bs))
    print(json.dumps({"op": a.op, "problems": a.problems, "dofs": dofs, "ms": ms,
                      "gdofs_solved": dofs / (ms * 1e-3) / 1e9}))


if __name__ == "__main__":
    main()
