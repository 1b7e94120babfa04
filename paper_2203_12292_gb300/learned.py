"""Learned fine-level smoother: training data from the plain solver, training
on the GPU, and the A/B comparison against Chebyshev that decides whether
the network is kept.  Host-side orchestration of library calls only; every
arithmetic step runs in libgcmg's kernels.

Recipe (an extension outside the paper, whose smoother is Chebyshev around
point Jacobi, Sec. 3.3):

* data: for every training right-hand side (Fourier fields with seeds
  1..8), the V-cycles of the first three iterations of plain fp64
  multigrid-preconditioned CG, taken at the point where the postsmoother
  acts (after the coarse-grid correction of the finest level): features of
  that iterate's residual, target from its error against the exact
  finest-level solution of the V-cycle's system (relative residual 1e-13);
  a seeded set of finest-level cells of each of these states gives the
  rows, 10,000 in all (or every cell when the mesh has fewer);
* training: Adam (lr 1e-3) on batches of 256 rows of a seeded 90 % split,
  the other 10 % kept for validation; the loss weights every row by
  (s_e / (h_e a_k))^2, so that it measures the error of the correction
  itself rather than of the normalised network output;
* comparison: time to a relative residual of 1e-8 of the mixed-precision
  solve with Chebyshev(3) only, with Chebyshev followed by the learned step
  ("augment") and with the learned step instead of postsmoothing
  ("replace"), on the evaluation right-hand side; the fastest variant is
  kept (Chebyshev when neither learned variant is faster).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

import synth

from . import MLP, Multigrid, SMOOTHER_CHEBYSHEV, SMOOTHER_MLP_AUGMENT, SMOOTHER_MLP_REPLACE


def fourier_modes(seed: int):
    f = synth.fourier_rhs(seed)
    return np.asarray(f.kappa, dtype=np.float64), np.asarray(f.phi, dtype=np.float64), f.amp


@dataclass
class TrainResult:
    net: MLP
    n_train: int
    n_val: int
    losses: np.ndarray
    val_mse: float           # trained network on the validation rows
    val_mse_zero: float      # zero correction on the validation rows
    val_mse_init: float      # initial network on the validation rows
    seconds_data: float
    seconds_train: float


def generate_samples(mg64: Multigrid, rhs_seeds=range(1, 9), cycles: int = 3, n_samples: int = 10000,
                     seed: int = 2022, ref_rtol: float = 1e-13):
    """Training rows (X, T) from the first `cycles` V-cycles of plain fp64
    MG-CG on every training right-hand side.  The V-cycle of CG iteration k
    solves A z = r_k (r_k the CG residual); the rows are taken where the
    postsmoother acts: z = the coarse-grid corrected iterate, residual
    r_k - A z, error z* - z with z* = A^{-1} r_k to `ref_rtol`."""
    import torch
    L = mg64.finest
    nc = mg64.n_cells(L)
    per = max(1, n_samples // (len(rhs_seeds) * cycles))
    Xs, Ts, Ws = [], [], []
    for si, s in enumerate(rhs_seeds):
        b = mg64.rhs(fourier_modes(s))
        for k in range(cycles):
            x = torch.zeros_like(b)
            mg64.cg_solve(b, x, 1e-30, maxit=k, raise_on_fail=False)  # x_k (x_0 = 0)
            rk = torch.empty_like(b)
            mg64.residual(L, b, x, rk)
            z = torch.empty_like(b)
            mg64.vcycle_cgc(rk, z)
            zstar = torch.zeros_like(b)
            mg64.cg_solve(rk, zstar, ref_rtol, maxit=200, raise_on_fail=False)
            keys = synth.splitmix64_array(seed * 7919 + si * 31 + k, nc)
            cells = np.sort(np.argsort(keys, kind="stable")[:min(per, nc)]).astype(np.int32)
            X, T, W = mg64.mlp_samples(L, rk, z, zstar, torch.tensor(cells, device="cuda"))
            Xs.append(X)
            Ts.append(T)
            Ws.append(W)
    return torch.cat(Xs), torch.cat(Ts), torch.cat(Ws)


def _mse(net: Optional[MLP], X, T, W) -> float:
    """Weighted loss of the network (None: the zero correction) on rows."""
    d = T.double() if net is None else net.forward(X).double() - T.double()
    return float(0.5 * (W.double() * (d ** 2).sum(dim=1)).sum() / W.double().sum())


def train(mg64: Multigrid, epochs: int = 100, batch: int = 256, lr: float = 1e-3, init_seed: int = 1,
          split_seed: int = 7, **sample_kw) -> TrainResult:
    import torch
    k = mg64.info[mg64.finest].degree
    t0 = time.perf_counter()
    X, T, W = generate_samples(mg64, **sample_kw)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    n = X.shape[0]
    perm = np.argsort(synth.splitmix64_array(split_seed, n), kind="stable")
    n_val = max(1, n // 10)
    vi = torch.tensor(perm[:n_val], device="cuda", dtype=torch.int64)
    ti = torch.tensor(perm[n_val:], device="cuda", dtype=torch.int64)
    Xtr, Ttr, Wtr = X[ti].contiguous(), T[ti].contiguous(), W[ti].contiguous()
    Xv, Tv, Wv = X[vi].contiguous(), T[vi].contiguous(), W[vi].contiguous()
    net = MLP(*synth.mlp_shape(k))
    net.set_params(torch.tensor(synth.mlp_init(*synth.mlp_shape(k), init_seed), dtype=torch.float32, device="cuda"))
    val_init = _mse(net, Xv, Tv, Wv)
    order = torch.tensor(synth.sample_order(Xtr.shape[0], epochs, split_seed + 1), device="cuda")
    losses = net.train(Xtr, Ttr, order, min(batch, Xtr.shape[0]), lr, W=Wtr)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return TrainResult(net, Xtr.shape[0], n_val, losses.cpu().numpy(), _mse(net, Xv, Tv, Wv),
                       _mse(None, Xv, Tv, Wv), val_init, t1 - t0, t2 - t1)


@dataclass
class Variant:
    name: str
    iterations: int
    rel_residual: float
    ms: float


def compare(mg: Multigrid, net: MLP, rhs_seed: int = 2203, rtol: float = 1e-8, repeats: int = 3,
            maxit: int = 200) -> Dict:
    """Solve times of Chebyshev / augment / replace on one right-hand side;
    the finest level's smoother is left at the fastest variant."""
    import torch
    b = mg.rhs(fourier_modes(rhs_seed)) if rhs_seed else mg.rhs()
    L = mg.finest
    out: List[Variant] = []
    for name, kind in (("chebyshev", SMOOTHER_CHEBYSHEV), ("augment", SMOOTHER_MLP_AUGMENT),
                       ("replace", SMOOTHER_MLP_REPLACE)):
        mg.set_smoother(L, kind, net)
        best, st = None, None
        for _ in range(repeats + 1):  # the first solve captures the graphs
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st = mg.cg_solve(b, x, rtol, maxit=maxit, raise_on_fail=False)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        out.append(Variant(name, st.iterations, st.rel_residual if st.status == 0 else float("inf"), best))
    ok = [v for v in out if v.rel_residual <= rtol]
    keep = min(ok, key=lambda v: v.ms) if ok else out[0]
    kinds = {"chebyshev": SMOOTHER_CHEBYSHEV, "augment": SMOOTHER_MLP_AUGMENT, "replace": SMOOTHER_MLP_REPLACE}
    mg.set_smoother(L, kinds[keep.name], net)
    return {"variants": out, "kept": keep.name}
