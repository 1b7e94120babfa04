"""Time to solution of the paper's own test cases on one GPU.

    python -m paper_2203_12292_gb300.tables [--case octant|gaussian|ls|shell|shell_ls|all] [--reps 3]

octant: -Delta u = 1, homogeneous Dirichlet data, the octant mesh of Sec. 4
("Examples") on [-1,1]^3, L = 3..8 for p = 1 and L = 3..7 for p = 4 (the
set-up of Tables A.3-A.4: CG to a 1e-4 reduction of the residual, one
global-coarsening V-cycle with Chebyshev(3) in fp32, fp64 CG).
gaussian: the same meshes with the Gaussian manufactured solution of
Table A.1 (inhomogeneous Dirichlet data).
ls: the octant case with geometric local smoothing instead of global
coarsening (Sec. 2.1; the LS columns of Table 4).
shell, shell_ls: the shell mesh of Sec. 4 (three radius bands), global
coarsening and local smoothing (Table 5), L = 5..9 for p = 1, 5..8 for p = 4.

Prints one JSON line per case: iterations, DoFs, and the time of one solve
(CUDA events on the solve's stream, the best of ``reps`` solves after one
warm-up solve; set-up excluded, as in the paper's tables).
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

GAUSSIAN = [0.1, -0.5, -0.5, -0.5]  # alpha, x0 (Table A.1)


def run_case(g, case: str, L: int, k: int, reps: int) -> dict:
    import torch
    mesh = g.Mesh.from_recipe(synth.shell(L) if case.startswith("shell") else synth.octant(L))
    mg = g.Multigrid(mesh, k, mg_fp32=True, local_smoothing=case.endswith("ls"))
    b = mg.rhs_dirichlet(g.FUNC_GAUSSIAN, GAUSSIAN) if case == "gaussian" else mg.rhs()
    x = torch.zeros_like(b)
    st = mg.cg_solve(b, x, 1e-4, maxit=50)  # warm-up: graphs captured here
    best = float("inf")
    for _ in range(reps):
        x.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = mg.cg_solve(b, x, 1e-4, maxit=50)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return {"case": case, "L": L, "p": k, "n_free": mg.n_free(mg.finest), "cells": mg.n_cells(mg.finest),
            "iterations": st.iterations, "rel_residual": st.rel_residual, "ms": best}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="all", choices=["octant", "gaussian", "ls", "shell", "shell_ls", "all"])
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    from . import build as b
    b.build()
    import paper_2203_12292_gb300 as g
    cases = ["octant", "gaussian", "ls", "shell", "shell_ls"] if a.case == "all" else [a.case]
    for case in cases:
        ranges = ((1, range(5, 10)), (4, range(5, 9))) if case.startswith("shell") else ((1, range(3, 9)), (4, range(3, 8)))
        for k, levels in ranges:
            for L in levels:
                print(json.dumps(run_case(g, case, L, k, a.reps)), flush=True)


if __name__ == "__main__":
    main()
