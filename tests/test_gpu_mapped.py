"""Non-Cartesian cells on the GPU (gcmg_set_geometry) against the mapped
oracle (oracle/mapped.py), through the C ABI.

Inputs are position-keyed (synth.point_values) in parameter space, evaluated
by each side at its own support points.  Tolerances as in test_gpu_parity:
fp64 operator, diagonal and right-hand sides 1e-12 (quadrature-point sum
factorisation against per-cell assembled element matrices in fp64), fp32
operator 2e-6, lambda 1e-8; CG: iterations = oracle's +- 1 and the oracle's
residual of the GPU solution <= rtol; patch test 1e-10.
"""
import numpy as np
import pytest

import synth
from oracle import dirichlet as od
from oracle import mapped as om
from oracle import mesh as omesh
from oracle import mg as omg
from parity import match, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPS = 0.3


class GeomCase:
    def __init__(self, gcmg, rec, k, eps=EPS, fp32=False, tile_cells=0):
        self.mg = gcmg.Multigrid(gcmg.Mesh.from_recipe(rec), k, mg_fp32=fp32, tile_cells=tile_cells)
        self.mg.set_geometry(gcmg.GEOM_WARP, eps)
        self.levels = omg.build_levels(omesh.build_mesh(rec), k, assembled=False, warp_eps=eps)
        self.n = self.mg.num_levels
        assert self.n == len(self.levels)
        self.perm = [match(self.mg.dof_coords(l), self.levels[l].space.free_coordinates()) for l in range(self.n)]

    def gvec(self, l, seed, dtype=torch.float64):
        return torch.tensor(synth.point_values(self.mg.dof_coords(l), seed), dtype=dtype, device="cuda")

    def ovec(self, l, seed):
        return synth.point_values(self.levels[l].space.free_coordinates(), seed)

    def cmp(self, l, gpu, oracle):
        return rel_err(gpu.double().cpu().numpy(), oracle[self.perm[l]])


CASES = [(synth.octant(3), 1), (synth.octant(3), 2), (synth.octant(3), 4), (synth.cube_octant(2, 1), 3),
         (synth.shell(5), 2)]
IDS = ["oct3-Q1", "oct3-Q2", "oct3-Q4", "cube2+1-Q3", "shell5-Q2"]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=IDS)
def case(gcmg, request):
    rec, k = CASES[request.param]
    return GeomCase(gcmg, rec, k)


def test_operator_diagonal_lambda(case):
    for l in range(case.n):
        if case.mg.n_free(l) == 0:
            continue
        s = case.levels[l].space
        x = case.gvec(l, 20 + l)
        y = torch.empty_like(x)
        case.mg.vmult(l, x, y)
        ref = s.apply(case.ovec(l, 20 + l))
        assert case.cmp(l, y, ref) < 1e-12, l
        x32 = case.gvec(l, 20 + l, torch.float32)
        y32 = torch.empty_like(x32)
        case.mg.vmult(l, x32, y32)
        assert case.cmp(l, y32, ref) < 2e-6, l
        assert case.cmp(l, case.mg.diagonal(l), s.diagonal()) < 1e-12, l
    for l in range(1, case.n):
        assert abs(case.mg.get_lambda(l) - case.levels[l].lam_max) < 1e-8 * case.levels[l].lam_max, l


def test_right_hand_sides(gcmg, case):
    s = case.levels[-1].space
    l = case.n - 1
    assert case.cmp(l, case.mg.rhs(), s.rhs()) < 1e-12
    terms = [(1.0, 1, 0, 0), (0.5, 1, 1, 0), (-0.25, 0, 1, 2), (0.3, 0, 0, 0)]
    u, f = od.polynomial(terms)
    b = case.mg.rhs_dirichlet(gcmg.FUNC_POLYNOMIAL, terms)
    assert case.cmp(l, b, om.rhs_dirichlet(s, f, u)) < 1e-12


def test_cg_matches_oracle(gcmg):
    c = GeomCase(gcmg, synth.octant(4), 2, fp32=True)
    s = c.levels[-1].space
    bo = s.rhs()
    l = c.n - 1
    b = torch.tensor(bo[c.perm[l]], dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    st = c.mg.cg_solve(b, x, 1e-8)
    ref = omg.solve(c.levels, bo, 1e-8, np.float32)
    assert st.status == 0 and abs(st.iterations - ref.iterations) <= 1, (st.iterations, ref.iterations)
    xo = np.empty(len(c.perm[l]))
    xo[c.perm[l]] = x.cpu().numpy()
    assert np.linalg.norm(bo - s.apply(xo)) <= 1.01e-8 * np.linalg.norm(bo)


@pytest.mark.parametrize("k", [1, 2, 4])
def test_patch_test(gcmg, k):
    """A function linear in the physical coordinates, its own Dirichlet
    data, f = 0: the discrete solution is exact (hanging nodes included)."""
    mg = gcmg.Multigrid(gcmg.Mesh.from_recipe(synth.octant(3)), k)
    mg.set_geometry(gcmg.GEOM_WARP, EPS)
    terms = [(0.7, 1, 0, 0), (-0.4, 0, 1, 0), (1.3, 0, 0, 1), (0.25, 0, 0, 0)]
    b = mg.rhs_dirichlet(gcmg.FUNC_POLYNOMIAL, terms)
    x = torch.zeros_like(b)
    assert mg.cg_solve(b, x, 1e-13, maxit=80).status == 0
    y = om.warp(mg.dof_coords(mg.finest), EPS)
    ref = y @ np.array([0.7, -0.4, 1.3]) + 0.25
    assert np.abs(x.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()


def test_eps_zero_and_back_to_cartesian(gcmg):
    mesh = gcmg.Mesh.from_recipe(synth.cube_octant(2, 1))
    mg = gcmg.Multigrid(mesh, 3)
    l = mg.finest
    x = torch.tensor(synth.point_values(mg.dof_coords(l), 5), dtype=torch.float64, device="cuda")
    y0, y1, y2 = (torch.empty_like(x) for _ in range(3))
    mg.vmult(l, x, y0)
    lam0 = [mg.get_lambda(q) for q in range(1, mg.num_levels)]
    mg.set_geometry(gcmg.GEOM_WARP, 0.0)  # the quadrature-point operator of Cartesian cells
    mg.vmult(l, x, y1)
    assert rel_err(y1.cpu().numpy(), y0.cpu().numpy()) < 1e-12
    mg.set_geometry(gcmg.GEOM_CARTESIAN)
    mg.vmult(l, x, y2)
    assert torch.equal(y2, y0)
    assert [mg.get_lambda(q) for q in range(1, mg.num_levels)] == lam0


def test_geometry_arguments(gcmg):
    mg = gcmg.Multigrid(gcmg.Mesh.from_recipe(synth.octant(2)), 2)
    with pytest.raises(gcmg.GcmgError):
        mg.set_geometry(7, 0.1)
    with pytest.raises(gcmg.GcmgError):  # folds [-1, 1]^3
        mg.set_geometry(gcmg.GEOM_WARP, 2.0)


def test_mapped_with_coefficient(gcmg):
    """geometry and a cell-wise coefficient together (either order) against
    the oracle's mapped levels with the same coefficient"""
    rec, k = synth.octant(3), 2
    nu_f = synth.random_cells(11)
    levels = omg.build_levels(omesh.build_mesh(rec), k, assembled=False, coefficient=nu_f, warp_eps=EPS)
    for order in ("geometry first", "coefficient first"):
        mg = gcmg.Multigrid(gcmg.Mesh.from_recipe(rec), k)
        xq = mg.quadrature_points().cpu().numpy()
        nu = torch.tensor(nu_f(xq.reshape(-1, 3)).reshape(xq.shape[:2]), dtype=torch.float64, device="cuda")
        if order == "geometry first":
            mg.set_geometry(gcmg.GEOM_WARP, EPS)
            mg.set_coefficient(nu)
        else:
            mg.set_coefficient(nu)
            mg.set_geometry(gcmg.GEOM_WARP, EPS)
        for l in range(mg.num_levels):
            if mg.n_free(l) == 0:
                continue
            s = levels[l].space
            perm = match(mg.dof_coords(l), s.free_coordinates())
            x = torch.tensor(synth.point_values(mg.dof_coords(l), 3 + l), dtype=torch.float64, device="cuda")
            y = torch.empty_like(x)
            mg.vmult(l, x, y)
            ref = s.apply(synth.point_values(s.free_coordinates(), 3 + l))
            assert rel_err(y.cpu().numpy(), ref[perm]) < 1e-12, (order, l)
            assert rel_err(mg.diagonal(l).cpu().numpy(), s.diagonal()[perm]) < 1e-12, (order, l)


def test_mapped_with_local_smoothing(gcmg):
    """the patch test through local smoothing on mapped cells"""
    mg = gcmg.Multigrid(gcmg.Mesh.from_recipe(synth.octant(3)), 2, local_smoothing=True)
    mg.set_geometry(gcmg.GEOM_WARP, EPS)
    terms = [(0.7, 1, 0, 0), (-0.4, 0, 1, 0), (1.3, 0, 0, 1), (0.25, 0, 0, 0)]
    b = mg.rhs_dirichlet(gcmg.FUNC_POLYNOMIAL, terms)
    x = torch.zeros_like(b)
    assert mg.cg_solve(b, x, 1e-13, maxit=80).status == 0
    y = om.warp(mg.dof_coords(mg.finest), EPS)
    ref = y @ np.array([0.7, -0.4, 1.3]) + 0.25
    assert np.abs(x.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()
