"""Variable coefficient -div(nu grad u) on the GPU (gcmg_set_coefficient)
against the oracle (oracle/coefficient.py), through the C ABI.

Inputs: the coefficient is a function of position (synth), evaluated by each
side at its own Gauss points; no value crosses from the CUDA path to the
oracle.  Tolerances as in test_gpu_parity (fp64 1e-12, fp32 2e-6, lambda
1e-8); cell averages 1e-14 (a different summation order of 8 to 125 terms).
"""
import numpy as np
import pytest

import synth
from oracle import coefficient as oc
from oracle import dirichlet as od
from oracle import mesh as omesh
from oracle import mg as omg
from parity import match, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


class CoefCase:
    def __init__(self, gcmg, rec, k, nu, fp32=False, tile_cells=0, cell_kernel=0):
        self.mg = gcmg.Multigrid(gcmg.Mesh.from_recipe(rec), k, mg_fp32=fp32, tile_cells=tile_cells,
                                 cell_kernel=cell_kernel)
        xq = self.mg.quadrature_points().cpu().numpy()
        nq = torch.tensor(nu(xq.reshape(-1, 3)).reshape(xq.shape[:2]), dtype=torch.float64, device="cuda")
        self.mg.set_coefficient(nq)
        self.levels = omg.build_levels(omesh.build_mesh(rec), k, assembled=False, coefficient=nu)
        self.n = self.mg.num_levels
        assert self.n == len(self.levels)
        self.perm = [match(self.mg.dof_coords(l), self.levels[l].space.free_coordinates()) for l in range(self.n)]

    def cell_perm(self, l):
        """oracle cell index of every library cell of level l"""
        s = self.levels[l].space
        g = self.mg.level_cells(l).astype(np.int64)
        return s.find_cells(g[:, 0], g[:, 1], g[:, 2], g[:, 3])


RANDOM = synth.random_cells(11)
CASES = [(synth.octant(3), 2, RANDOM), (synth.octant(3), 4, synth.inclusions(5, -1.0, 1.0, contrast=1e3)),
         (synth.shell(5), 1, RANDOM), (synth.cube_octant(2, 1), 3, synth.step(0.5, 10.0, 0.1))]
IDS = ["octant-Q2-random", "octant-Q4-inclusions", "shell-Q1-random", "cube-Q3-step"]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=IDS)
def case(gcmg, request):
    rec, k, nu = CASES[request.param]
    return CoefCase(gcmg, rec, k, nu)


def test_quadrature_points(gcmg):
    rec = synth.octant(3)
    c = CoefCase(gcmg, rec, 3, RANDOM)
    xq = c.mg.quadrature_points().cpu().numpy()
    ref = oc.quadrature_points(c.levels[-1].space)[c.cell_perm(c.n - 1)]
    assert np.abs(xq - ref).max() <= 1e-15


def test_level_coefficients(case):
    for l in range(case.n):
        cp = case.cell_perm(l)
        assert np.all(cp >= 0)
        g = case.mg.get_coefficient(l).cpu().numpy()
        ref = case.levels[l].space.nu[cp]
        assert np.abs(g - ref).max() <= 1e-14 * np.abs(ref).max(), l


def test_vmult_and_diagonal(case):
    for l in range(case.n):
        s = case.levels[l].space
        xo = synth.point_values(s.free_coordinates(), 40 + l)
        xg = torch.tensor(synth.point_values(case.mg.dof_coords(l), 40 + l), dtype=torch.float64, device="cuda")
        y = torch.empty_like(xg)
        case.mg.vmult(l, xg, y)
        assert rel_err(y.cpu().numpy(), s.apply(xo)[case.perm[l]]) < 1e-12, l
        d = case.mg.diagonal(l).cpu().numpy()
        assert rel_err(d, s.diagonal()[case.perm[l]]) < 1e-12, l


def test_lambda_estimates(case):
    for l in range(1, case.n):
        ref = case.levels[l].lam_max
        assert abs(case.mg.get_lambda(l) - ref) < 1e-8 * ref, l


@pytest.mark.parametrize("cell_kernel", [0, 1, 2])
def test_fp32_operator_kernels(gcmg, cell_kernel):
    c = CoefCase(gcmg, synth.octant(3), 4, RANDOM, fp32=True, cell_kernel=cell_kernel)
    l = c.n - 1
    s = c.levels[l].space
    xo = synth.point_values(s.free_coordinates(), 7)
    xg = torch.tensor(synth.point_values(c.mg.dof_coords(l), 7), dtype=torch.float32, device="cuda")
    y = torch.empty_like(xg)
    c.mg.vmult(l, xg, y)
    assert rel_err(y.double().cpu().numpy(), s.apply(xo)[c.perm[l]]) < 2e-6


def test_rhs_dirichlet_with_coefficient(gcmg, case):
    k = case.levels[-1].space.k
    terms = [(1.0, k, 0, 0), (0.5, 1, k, 1), (-0.25, 0, 1, k), (0.3, 0, 0, 0)]
    u, f = od.polynomial(terms)
    b = case.mg.rhs_dirichlet(gcmg.FUNC_POLYNOMIAL, terms).cpu().numpy()
    bo = od.rhs(case.levels[-1].space, f, u)[case.perm[-1]]
    assert np.abs(b - bo).max() <= 1e-12 * np.abs(bo).max()


def test_cg_matches_oracle(case):
    s = case.levels[-1].space
    b = torch.tensor(s.rhs()[case.perm[-1]], dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    st = case.mg.cg_solve(b, x, 1e-8, maxit=100)
    ref = omg.solve(case.levels, s.rhs(), 1e-8, np.float64)
    assert st.status == 0 and abs(st.iterations - ref.iterations) <= 1, (st.iterations, ref.iterations)
    xo = np.empty(len(case.perm[-1]))
    xo[case.perm[-1]] = x.cpu().numpy()
    assert np.linalg.norm(s.rhs() - s.apply(xo)) <= 1.01e-8 * np.linalg.norm(s.rhs())


@pytest.mark.parametrize("k", [1, 2, 4])
def test_exact_solution_across_a_jump(gcmg, k):
    """nu jumps across x = 0 (a plane of cell faces); u harmonic and
    independent of x has zero flux across the plane, so for u in Q_k the
    discrete solution is u's interpolant whatever the jump."""
    terms = [(1.0, 0, 1, 0), (2.0, 0, 0, 1), (1.0, 0, 1, 1)]
    if k >= 2:
        terms += [(1.0, 0, 2, 0), (-1.0, 0, 0, 2)]
    mg = gcmg.Multigrid(gcmg.Mesh.from_recipe(synth.octant(3)), k)
    xq = mg.quadrature_points().cpu().numpy()
    nu = synth.step(0.0, 100.0, 1.0)(xq.reshape(-1, 3)).reshape(xq.shape[:2])
    mg.set_coefficient(torch.tensor(nu, dtype=torch.float64, device="cuda"))
    b = mg.rhs_dirichlet(gcmg.FUNC_POLYNOMIAL, terms)
    x = torch.zeros_like(b)
    assert mg.cg_solve(b, x, 1e-13, maxit=80).status == 0
    u, _ = od.polynomial(terms)
    ref = u(mg.dof_coords(mg.finest))
    assert np.abs(x.cpu().numpy() - ref).max() <= 1e-9 * np.abs(ref).max()


def test_inclusions_solve_q4(gcmg):
    """octant L = 5, Q4 (0.3 M DoFs), contrast 1e3, fp32 V-cycle"""
    rec = synth.octant(5)
    mg = gcmg.Multigrid(gcmg.Mesh.from_recipe(rec), 4)
    xq = mg.quadrature_points()
    nu = synth.inclusions(5, -1.0, 1.0, contrast=1e3)(xq.reshape(-1, 3).cpu().numpy())
    mg.set_coefficient(torch.tensor(nu, dtype=torch.float64, device="cuda"))
    b = mg.rhs()
    x = torch.zeros_like(b)
    st = mg.cg_solve(b, x, 1e-8, maxit=100)
    assert st.status == 0 and st.iterations <= 30, st.iterations


def test_coefficient_arguments(gcmg):
    mg = gcmg.Multigrid(gcmg.Mesh.from_recipe(synth.octant(2)), 2)
    nc = mg.n_cells(mg.finest)
    lam = [mg.get_lambda(l) for l in range(1, mg.num_levels)]
    for bad in (-1.0, 0.0, float("nan"), float("inf")):
        nu = torch.ones(nc, dtype=torch.float64, device="cuda")
        nu[nc // 2] = bad
        with pytest.raises(gcmg.GcmgError):
            mg.set_coefficient(nu)
    with pytest.raises(gcmg.GcmgError):  # neither 1 nor (k+1)^3 values per cell
        mg.set_coefficient(torch.ones(nc * 2, dtype=torch.float64, device="cuda"))
    # the handle is unchanged
    assert [mg.get_lambda(l) for l in range(1, mg.num_levels)] == lam
    assert torch.all(mg.get_coefficient(mg.finest) == 1.0)
    # one value per cell
    mg.set_coefficient(torch.full((nc,), 3.0, dtype=torch.float64, device="cuda"))
    assert torch.all(mg.get_coefficient(0) == 3.0)
    for l, v in zip(range(1, mg.num_levels), lam):
        assert abs(mg.get_lambda(l) - v) <= 1e-10 * v  # D^-1 A does not change
