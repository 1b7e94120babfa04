"""Textbook geometric multigrid and conjugate gradients.

Test infrastructure (see ``oracle/__init__``).

Follows:
* Algorithm 1: copy to the multigrid levels, V-cycle, copy back; with global
  coarsening the copy is to/from the finest level only (Sec. 2.2), and it is
  where single precision may be switched on (Sec. 2).
* Algorithm 2: coarse solve on level 0, otherwise presmoothing from zero,
  residual, restriction added to the coarse right-hand side, recursion,
  prolongation added to x, postsmoothing.
* Sec. 3.3: Chebyshev iteration around point Jacobi; Sec. 5 set-up: degree 3
  on all levels.
* Sec. 3.4: the coarse-grid solver may be a direct solver; here a dense
  Cholesky factorisation of the level-0 matrix.
* Sec. 2 / Sec. 5: CG preconditioned by one V-cycle, stopped on the
  relative reduction of the unpreconditioned l2 residual.

Readings where the paper is silent (Chebyshev parameters): the largest
eigenvalue of D^{-1}A is estimated from the Lanczos tridiagonal matrix of 12
Jacobi-preconditioned CG steps on A y = s (starting from y = 0), s the
all-ones vector plus a seeded perturbation 1 + u(x), u the position-keyed
uniform values of synth.point_values (a smooth start vector alone misses the
top of the spectrum on uniform meshes and the smoother then amplifies
it); the
smoother works on [1.2 lam / 20, 1.2 lam]; the recurrence is the
three-term Chebyshev acceleration of Saad (Iterative Methods for Sparse
Linear Systems, 2nd ed., Algorithm 12.1), so that degree 3 costs 2 operator
applications from a zero start and 3 otherwise (matching the 2/1/3
evaluations of pre-smoothing/residual/post-smoothing reported in Sec. 5.2).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

import synth

from . import coefficient as ocoef
from . import mesh as omesh
from .space import Space
from .transfer import prolongation_matrix

EIG_CG_STEPS = 12
EIG_SAFETY = 1.2
SMOOTHING_RANGE = 20.0
CHEB_DEGREE = 3


def lanczos_lambda_max(apply: Callable, dinv: np.ndarray, n_steps: int = EIG_CG_STEPS,
                       start: Optional[np.ndarray] = None) -> float:
    """Largest eigenvalue of the Lanczos tridiagonal matrix built from the
    coefficients alpha_k, beta_k of Jacobi-preconditioned CG on A y = start
    (all ones when not given)."""
    n = len(dinv)
    if n == 0:
        return 1.0
    b = np.ones(n) if start is None else np.asarray(start, dtype=np.float64)
    x = np.zeros(n)
    r = b.copy()
    z = dinv * r
    p = z.copy()
    rz = r @ z
    rz0 = rz
    alphas, betas = [], []
    for _ in range(n_steps):
        q = apply(p)
        pq = p @ q
        if pq <= 0.0:
            break
        alpha = rz / pq
        alphas.append(alpha)
        x += alpha * p
        r -= alpha * q
        z = dinv * r
        rz_new = r @ z
        beta = rz_new / rz
        if rz_new <= 1e-30 * rz0:  # Krylov space exhausted
            break
        betas.append(beta)
        p = z + beta * p
        rz = rz_new
    m = len(alphas)
    T = np.zeros((m, m))
    for i in range(m):
        T[i, i] = 1.0 / alphas[i] + (betas[i - 1] / alphas[i - 1] if i > 0 else 0.0)
        if i + 1 < m:
            T[i, i + 1] = T[i + 1, i] = np.sqrt(betas[i]) / alphas[i]
    return float(np.max(np.linalg.eigvalsh(T)))


def chebyshev(apply: Callable, dinv: np.ndarray, b: np.ndarray, x: Optional[np.ndarray],
              lam_max: float, degree: int = CHEB_DEGREE, smoothing_range: float = SMOOTHING_RANGE):
    """Chebyshev iteration of the given degree for A x = b with the point
    Jacobi preconditioner D^{-1} on the interval [lam_max / range, lam_max].
    x = None means a zero initial guess (the first residual is b)."""
    dt = b.dtype
    lmin = lam_max / smoothing_range
    theta = (lam_max + lmin) / 2
    delta = (lam_max - lmin) / 2
    if x is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = x.copy()
        r = b - apply(x)
    rho = delta / theta
    d = (dinv * r) * dt.type(1.0 / theta)
    x = x + d
    for _ in range(1, degree):
        r = b - apply(x)
        rho_new = 1.0 / (2.0 * theta / delta - rho)
        d = dt.type(rho_new * rho) * d + dt.type(2.0 * rho_new / delta) * (dinv * r)
        rho = rho_new
        x = x + d
    return x


@dataclass
class Level:
    space: Space
    A: object  # sparse matrix or None (cell-by-cell apply)
    diag: np.ndarray
    lam_max: float = 1.0
    P: Optional[sp.csr_matrix] = None  # from level-1 to this level
    chol: object = None
    dtype: type = np.float64
    A32: object = None
    learned: Optional[Callable] = None  # residual -> correction (learned smoother)
    learned_mode: str = "augment"       # "augment": after postsmoothing; "replace": instead of it

    def apply64(self, x):
        """The fp64 operator."""
        if self.A is not None:
            return self.A @ x
        return self.space.apply(x)

    def apply(self, x):
        """The operator in the level's precision."""
        if self.dtype == np.float32:
            return self.A32 @ x if self.A32 is not None else self.space.apply(x)
        return self.apply64(x)


def build_levels(fine_mesh: omesh.Mesh, k: int, p_coarsening: bool = False,
                 assembled: bool = True, lam_max: Optional[List[float]] = None,
                 coefficient: Optional[Callable] = None, warp_eps: Optional[float] = None) -> List[Level]:
    """Global-coarsening levels (coarsest first). With p_coarsening the
    finest mesh is first coarsened in degree k -> floor(k/2) -> ... -> 1
    (Sec. 2.3), then geometrically with degree 1.  ``coefficient``: nu(x) of
    -div(nu grad u), set on all levels as in oracle.coefficient.  ``warp_eps``:
    the cells mapped by oracle.mapped.warp on every level."""
    meshes = omesh.gc_hierarchy(fine_mesh)
    specs = []
    if p_coarsening:
        degs = [k]
        while degs[-1] > 1:
            degs.append(degs[-1] // 2)
        specs = [(m, 1) for m in meshes[:-1]] + [(meshes[-1], d) for d in degs[::-1]]
    else:
        specs = [(m, k) for m in meshes]
    if warp_eps is None:
        spaces = [Space(m, kk) for m, kk in specs]
    else:
        from .mapped import MappedSpace
        spaces = [MappedSpace(m, kk, warp_eps) for m, kk in specs]
    if coefficient is not None:
        ocoef.set_level_coefficients(spaces, coefficient)
        if warp_eps is not None:
            for s in spaces:
                s.set_coefficient(s.nu)
    levels: List[Level] = []
    for idx, s in enumerate(spaces):
        A = s.assemble() if assembled else None
        lev = Level(s, A, s.diagonal())
        if idx > 0:
            lev.P = prolongation_matrix(s, levels[-1].space)
        levels.append(lev)
    for idx, lev in enumerate(levels):
        if idx == 0:
            if lev.space.n_free:
                A0 = lev.A.toarray() if lev.A is not None else _dense(lev)
                lev.chol = sla.cho_factor(A0, lower=True)
            continue
        if lam_max is not None:
            lev.lam_max = lam_max[idx]
        else:
            start = 1.0 + synth.point_values(lev.space.free_coordinates(), synth.LANCZOS_START_SEED)
            lev.lam_max = EIG_SAFETY * lanczos_lambda_max(lev.apply64, 1.0 / lev.diag, start=start)
    return levels


def _dense(lev: Level) -> np.ndarray:
    n = lev.space.n_free
    return np.stack([lev.space.apply(np.eye(n)[:, i]) for i in range(n)], axis=1)


def vcycle(levels: List[Level], l: int, b: np.ndarray) -> np.ndarray:
    """The multigrid V-cycle on level l for A_l x = b, written as a
    residual-correction method (the cycle of Sec. 2.1 / Algorithm 2): a
    smoothed start from zero, the coarse-grid correction P e_c with e_c the
    V-cycle's solution of R = P^T applied to the defect, and a second smoothing
    from the corrected iterate; on level 0 the exact solve."""
    lev = levels[l]
    dt = b.dtype
    if l == 0:
        if lev.space.n_free == 0:
            return np.zeros_like(b)
        return sla.cho_solve(lev.chol, b.astype(np.float64)).astype(dt)
    dinv = (1.0 / lev.diag).astype(dt)

    def smooth(x0):
        return chebyshev(lev.apply, dinv, b, x0, lev.lam_max)

    P = lev.P.astype(dt) if dt == np.float32 else lev.P
    x = smooth(None)
    defect = b - lev.apply(x)
    x = x + P @ vcycle(levels, l - 1, P.T @ defect)
    if lev.learned is not None and lev.learned_mode == "replace":
        return learned_step(lev, b, x)  # the learned step takes the second smoothing's place
    x = smooth(x)
    return learned_step(lev, b, x) if lev.learned is not None else x


def learned_step(lev: Level, b: np.ndarray, x: np.ndarray) -> np.ndarray:
    """x + omega c with c the learned correction of the residual and omega
    the Galerkin step length (r.c) / (c.A c): the A-norm of the error cannot
    grow whatever the network returns (omega = 0 when c.A c <= 0).  Inner
    products in fp64."""
    dt = x.dtype
    r = b - lev.apply(x)
    c = lev.learned(r).astype(dt)
    w = lev.apply(c)
    num = float(np.dot(r.astype(np.float64), c.astype(np.float64)))
    den = float(np.dot(c.astype(np.float64), w.astype(np.float64)))
    om = num / den if den > 0 else 0.0
    return x + dt.type(om) * c


def set_precision(levels: List[Level], dtype) -> None:
    """FP32 V-cycle mode: level matrices and vectors rounded to float."""
    for lev in levels:
        lev.dtype = dtype
        if dtype == np.float32 and lev.A is not None:
            lev.A32 = lev.A.astype(np.float32)


def multigrid_vcycle(levels: List[Level], b: np.ndarray, dtype=np.float64) -> np.ndarray:
    """Algorithm 1: copy to the finest level (with the precision switch),
    V-cycle, copy back."""
    bl = b.astype(dtype)
    x = vcycle(levels, len(levels) - 1, bl)
    return x.astype(np.float64)


@dataclass
class SolveResult:
    x: np.ndarray
    iterations: int
    residuals: List[float] = field(default_factory=list)


def pcg(apply: Callable, b: np.ndarray, precond: Callable, rtol: float, maxit: int = 200,
        flexible: bool = False) -> SolveResult:
    """Preconditioned CG from x = 0, stopped when ||b - A x||_2 <= rtol ||b||_2.
    flexible: beta = r_{k+1}.(z_{k+1} - z_k) / r_k.z_k (Notay, SIAM J. Sci.
    Comput. 22 (2000), flexible CG with one stored direction), the variant
    for a preconditioner that is not a fixed linear map."""
    x = np.zeros_like(b)
    r = b.copy()
    nb = np.linalg.norm(b)
    res = [nb]
    if nb == 0.0:
        return SolveResult(x, 0, res)
    z = precond(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = apply(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        nr = np.linalg.norm(r)
        res.append(nr)
        if nr <= rtol * nb:
            return SolveResult(x, it, res)
        cross = r @ z if flexible else 0.0
        z = precond(r)
        rz_new = r @ z
        p = z + ((rz_new - cross) / rz) * p
        rz = rz_new
    return SolveResult(x, maxit, res)


def solve(levels: List[Level], b: np.ndarray, rtol: float, mg_dtype=np.float64, maxit: int = 200,
          flexible: bool = False) -> SolveResult:
    """CG in fp64 preconditioned by one V-cycle in ``mg_dtype``."""
    set_precision(levels, mg_dtype)
    return pcg(levels[-1].apply64, b, lambda r: multigrid_vcycle(levels, r, mg_dtype), rtol, maxit, flexible)
