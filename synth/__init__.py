"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the multigrid method itself: only
mesh *recipes* (plain parameter records that say how a test mesh is refined),
a counter-based random number generator (SplitMix64, Steele, Lea & Flood,
OOPSLA 2014) and the random draws built from it (vectors, Fourier modes of
the right-hand side, the batch of uneven problems).

Workload recipes (all on hexahedral octree meshes):

* ``octant(L)``       -- the paper's ``octant`` mesh on [-1,1]^3 (Sec. 4,
  "Examples"): L steps, each refining every leaf whose centre lies in the
  closed first octant [-1,0]^3, each step followed by the 2:1 closure.
* ``shell(L)``        -- the paper's ``shell`` mesh on [-1,1]^3 (Sec. 4):
  L-3 uniform steps, then three local steps on |c| <= 0.55,
  0.30 <= |c| <= 0.43 and 0.335 <= |c| <= 0.39 (c = cell centre).
* ``cube_octant(g, e)`` -- [0,1]^3, g uniform steps, then e steps refining the
  leaves whose centre lies in the closed octant [0,1/2]^3.
* ``sphere(cycles)``  -- [0,1]^3, ``cycles`` steps each refining every leaf
  whose box intersects the sphere |x-(1/2,1/2,1/2)| = 0.3.

The five benchmark workloads:

* ``WORKLOAD_Q2_OCTANT``  Q2, cube_octant(3, 1), f = 1
* ``WORKLOAD_Q4_OCTANT``  Q4, cube_octant(5, 2), f = Fourier field, seed 2203
* ``WORKLOAD_Q4_SPHERE``  Q4, sphere(7), f = 1, p-coarsening 4 -> 2 -> 1
* ``batch_recipes()``     256 problems (k, depth, extra) from seed 12292
* learned smoother        the Q4 octant mesh, RHS seeds 1..8 for training
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64_next(state: int) -> Tuple[int, int]:
    """One step of SplitMix64: returns (new_state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & MASK64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return state, z ^ (z >> 31)


class SplitMix64:
    """Sequential SplitMix64 stream (host-side, for small draws)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state, out = splitmix64_next(self.state)
        return out

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive)."""
        return lo + int(self.uniform() * (hi - lo + 1))


def splitmix64_array(seed: int, n: int) -> np.ndarray:
    """Counter-based SplitMix64: output i is the (i+1)-th output of the stream
    seeded with ``seed`` (vectorised, uint64)."""
    with np.errstate(over="ignore"):
        idx = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed & MASK64) + idx * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_vector(n: int, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """n doubles uniform in [lo, hi) from the counter-based stream."""
    u = (splitmix64_array(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return lo + (hi - lo) * u


# --------------------------------------------------------------------------
# mesh recipes
# --------------------------------------------------------------------------

PRED_ALL = 0            # refine every leaf
PRED_OCTANT_CENTRE = 1  # centre in the closed box [box_lo, box_hi]^3
PRED_SPHERE = 2         # leaf box intersects the sphere |x - c| = r
PRED_SHELL = 3          # r0 <= |centre| <= r1
PRED_OCTANT_STRICT = 4  # all vertex coordinates strictly below box_hi


@dataclass
class RefineStep:
    """One refinement step: refine every leaf matching the predicate, then
    apply the 2:1 closure. ``a``..``d`` are the predicate parameters:
    octant: a = box_lo, b = box_hi; sphere: (a, a, a) = centre, b = radius;
    shell: a = r0, b = r1."""
    pred: int
    a: float = 0.0
    b: float = 0.0
    c: float = 0.0
    d: float = 0.0


@dataclass
class MeshRecipe:
    lo: float
    hi: float
    steps: List[RefineStep] = field(default_factory=list)
    name: str = ""


def octant(L: int) -> MeshRecipe:
    return MeshRecipe(-1.0, 1.0, [RefineStep(PRED_OCTANT_CENTRE, -1.0, 0.0)] * L, f"octant L={L}")


def shell(L: int) -> MeshRecipe:
    steps = [RefineStep(PRED_ALL)] * (L - 3)
    steps += [RefineStep(PRED_SHELL, 0.0, 0.55), RefineStep(PRED_SHELL, 0.3, 0.43),
              RefineStep(PRED_SHELL, 0.335, 0.39)]
    return MeshRecipe(-1.0, 1.0, steps, f"shell L={L}")


def cube_octant(n_global: int, n_extra: int, strict: bool = False) -> MeshRecipe:
    pred = PRED_OCTANT_STRICT if strict else PRED_OCTANT_CENTRE
    steps = [RefineStep(PRED_ALL)] * n_global + [RefineStep(pred, 0.0, 0.5)] * n_extra
    return MeshRecipe(0.0, 1.0, steps, f"cube global={n_global} octant+{n_extra}")


def sphere(cycles: int, centre: float = 0.5, radius: float = 0.3) -> MeshRecipe:
    return MeshRecipe(0.0, 1.0, [RefineStep(PRED_SPHERE, centre, radius)] * cycles,
                      f"sphere cycles={cycles}")


def uniform_cube(n_global: int, lo: float = 0.0, hi: float = 1.0) -> MeshRecipe:
    return MeshRecipe(lo, hi, [RefineStep(PRED_ALL)] * n_global, f"uniform {n_global}")


# --------------------------------------------------------------------------
# right-hand sides
# --------------------------------------------------------------------------

@dataclass
class FourierRHS:
    """f(x) = amp * sum_m cos(2 pi kappa_m . x + phi_m).

    With 8 modes of distinct wave vectors and amp = 1/2 the field has unit
    variance: 8 * amp^2 / 2 = 1."""
    kappa: np.ndarray  # (m, 3) int
    phi: np.ndarray    # (m,) float
    amp: float


def fourier_rhs(seed: int, n_modes: int = 8, kmax: int = 4) -> FourierRHS:
    """Random Fourier field: wave vectors in {-kmax..kmax}^3 \\ {0}, distinct
    up to sign; phases uniform in [0, 2 pi)."""
    rng = SplitMix64(seed)
    kap: List[Tuple[int, int, int]] = []
    while len(kap) < n_modes:
        v = tuple(rng.randint(-kmax, kmax) for _ in range(3))
        if v == (0, 0, 0):
            continue
        if v in kap or tuple(-t for t in v) in kap:
            continue
        kap.append(v)
    phi = np.array([2.0 * math.pi * rng.uniform() for _ in range(n_modes)])
    return FourierRHS(np.array(kap, dtype=np.int64), phi, 1.0 / math.sqrt(n_modes / 2.0))


# --------------------------------------------------------------------------
# benchmark workloads
# --------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    recipe: MeshRecipe
    degree: int
    rhs_seed: int  # 0 = constant f = 1
    p_coarsening: bool = False


WORKLOAD_Q2_OCTANT = Workload("Q2 cube octant global3+1 (960 cells)", cube_octant(3, 1), 2, 0)
WORKLOAD_Q4_OCTANT = Workload("Q4 cube octant global5+2 (296,535 cells)", cube_octant(5, 2), 4, 2203)
WORKLOAD_Q4_SPHERE = Workload("Q4 sphere-adapted cube, 7 cycles (82,776 cells)", sphere(7), 4, 0, True)


def batch_recipes(seed: int = 12292, n: int = 256):
    """The batch of uneven problems: (degree in 1..4, global depth in 2..5,
    extra octant levels in 0..2, rhs seed) drawn from one SplitMix64 stream."""
    rng = SplitMix64(seed)
    out = []
    for p in range(n):
        k = rng.randint(1, 4)
        depth = rng.randint(2, 5)
        extra = rng.randint(0, 2)
        rhs_seed = rng.next_u64() & 0x7FFFFFFF
        out.append((k, depth, extra, rhs_seed))
    return out


# --------------------------------------------------------------------------
# position-keyed random values: the same input vector for any DoF numbering
# --------------------------------------------------------------------------

# seed of the perturbation of the Lanczos start vector of the eigenvalue
# estimate (both the oracle and the library use 1 + point_values(x, seed))
LANCZOS_START_SEED = 2203


def point_values(xyz: np.ndarray, seed: int, resolution_bits: int = 20) -> np.ndarray:
    """Uniform values in [-1, 1) attached to points: each coordinate is
    rounded to a multiple of 2^-resolution_bits, the three integers are mixed
    with SplitMix64's finaliser together with the seed.  Two programs that
    number the same support points differently get the same vector."""
    q = np.rint(np.asarray(xyz, dtype=np.float64) * float(1 << resolution_bits)).astype(np.int64)
    mask = np.uint64(MASK64)
    with np.errstate(over="ignore"):
        h = np.full(len(q), np.uint64(seed & MASK64), dtype=np.uint64)
        for d in range(3):
            h = h ^ q[:, d].astype(np.uint64)
            h = h + np.uint64(0x9E3779B97F4A7C15)
            h = (h ^ (h >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            h = (h ^ (h >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            h = (h ^ (h >> np.uint64(31))) & mask
    return -1.0 + 2.0 * (h >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


# --------------------------------------------------------------------------
# coefficient fields nu(x) of -div(nu grad u)
# --------------------------------------------------------------------------

@dataclass
class Inclusions:
    """nu(x) = 1 + (contrast - 1) * max_i exp(-|x - c_i|^2 / width^2): smooth
    high-viscosity inclusions at seeded centres c_i in [lo, hi]^3 in a unit
    background (a stand-in for the sinker viscosity of a Stokes benchmark)."""
    centres: np.ndarray  # (n, 3)
    width: float
    contrast: float

    def __call__(self, xyz: np.ndarray) -> np.ndarray:
        x = np.asarray(xyz, dtype=np.float64)
        d2 = ((x[:, None, :] - self.centres[None, :, :]) ** 2).sum(axis=2)
        return 1.0 + (self.contrast - 1.0) * np.exp(-d2 / (self.width * self.width)).max(axis=1)


def inclusions(seed: int, lo: float, hi: float, n: int = 7, width: float = 0.1,
               contrast: float = 1e3) -> Inclusions:
    u = (splitmix64_array(seed, 3 * n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))
    return Inclusions(lo + (hi - lo) * u.reshape(n, 3), width * (hi - lo), contrast)


def random_cells(seed: int, contrast: float = 1e2):
    """nu(x) = contrast^(v(x)) with v the position-keyed values in [-1, 1):
    unrelated values at every point (rough coefficient, parity tests)."""
    def nu(xyz):
        return contrast ** point_values(xyz, seed)
    return nu


def step(x_c: float, nu_lo: float, nu_hi: float):
    """nu = nu_lo for x < x_c, nu_hi otherwise (a jump across a plane)."""
    def nu(xyz):
        return np.where(np.asarray(xyz)[:, 0] < x_c, nu_lo, nu_hi)
    return nu


# --------------------------------------------------------------------------
# learned smoother: network size, initial parameters, sample orders
# --------------------------------------------------------------------------

MLP_HIDDEN = 128


def mlp_shape(k: int):
    """(n_in, n_hidden, n_out) of the per-cell network for degree k: the
    residual and the diagonal at the (k+1)^3 support points in, the
    correction at them out."""
    n3 = (k + 1) ** 3
    return 2 * n3, MLP_HIDDEN, n3


def mlp_init(n_in: int, n_h: int, n_out: int, seed: int) -> np.ndarray:
    """Initial packed parameters (W1, b1, W2, b2, W3, b3; matrices row-major,
    one row per output unit), each entry uniform in +-1/sqrt(fan_in), rounded
    to float32."""
    parts = []
    for i, (rows, fan_in) in enumerate([(n_h, n_in), (n_h, n_h), (n_out, n_h)]):
        bound = 1.0 / np.sqrt(fan_in)
        parts.append(uniform_vector(rows * fan_in, seed * 8 + 2 * i + 1, -bound, bound))
        parts.append(uniform_vector(rows, seed * 8 + 2 * i + 2, -bound, bound))
    return np.concatenate(parts).astype(np.float32).astype(np.float64)


def sample_order(n_samples: int, epochs: int, seed: int) -> np.ndarray:
    """Concatenated random permutations of range(n_samples), one per epoch:
    the order that sorts SplitMix64 keys (stable for equal keys)."""
    out = np.empty(n_samples * epochs, dtype=np.int32)
    for e in range(epochs):
        keys = splitmix64_array(seed * 1000003 + e, n_samples)
        out[e * n_samples:(e + 1) * n_samples] = np.argsort(keys, kind="stable")
    return out
