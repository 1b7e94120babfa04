"""Local smoothing on the GPU (gcmg_config.local_smoothing) against the
local-smoothing oracle (oracle/ls.py), through the C ABI.

Inputs are position-keyed (synth.point_values), evaluated by each side at its
own support points.  Tolerances as in test_gpu_parity: fp64 operator,
diagonal, transfer 1e-12; V-cycle 1e-10 (all levels chained, the oracle's
lambda set on the GPU); lambda 1e-8; CG: iterations = oracle's +- 1 and the
oracle's residual of the GPU solution <= rtol.
"""
import numpy as np
import pytest

import synth
from golden_data import table
from oracle import ls
from oracle import mesh as omesh
from oracle.space import Space
from parity import match, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


class LSCase:
    def __init__(self, gcmg, rec, k, fp32=False):
        self.mg = gcmg.Multigrid(gcmg.Mesh.from_recipe(rec), k, mg_fp32=fp32, local_smoothing=True)
        fine = omesh.build_mesh(rec)
        self.levels = ls.build_ls_levels(fine, k)
        self.act = Space(fine, k)
        self.cm = ls.copy_map(self.act, self.levels)
        self.n = len(self.levels)
        assert self.mg.num_levels == self.n + 1  # the refinement levels, then the active mesh
        self.perm = [match(self.mg.dof_coords(l), self.levels[l].space.free_coordinates()) for l in range(self.n)]
        self.aperm = match(self.mg.dof_coords(self.mg.finest), self.act.free_coordinates())

    def gvec(self, l, seed):
        return torch.tensor(synth.point_values(self.mg.dof_coords(l), seed), dtype=torch.float64, device="cuda")

    def ovec(self, l, seed):
        s = self.act if l == self.n else self.levels[l].space
        return synth.point_values(s.free_coordinates(), seed)

    def cmp(self, l, gpu, oracle):
        p = self.aperm if l == self.n else self.perm[l]
        return rel_err(gpu.double().cpu().numpy(), oracle[p])


CASES = [(synth.octant(3), 1), (synth.octant(4), 2), (synth.octant(3), 4), (synth.cube_octant(2, 2), 3)]
IDS = ["oct3-Q1", "oct4-Q2", "oct3-Q4", "cube2+2-Q3"]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=IDS)
def case(gcmg, request):
    rec, k = CASES[request.param]
    return LSCase(gcmg, rec, k)


def test_levels_and_edges(case):
    assert any(np.any(lev.edge) for lev in case.levels)
    for l in range(case.n):
        e = case.mg.edge_dofs(l)
        mask = np.zeros(case.mg.n_free(l), dtype=bool)
        mask[e] = True
        # GPU DoF i is oracle DoF perm[i]
        assert np.array_equal(mask, case.levels[l].edge[case.perm[l]]), l


def test_level_operators(case):
    for l in range(case.n):
        if case.mg.n_free(l) == 0:
            continue
        x = case.gvec(l, 10 + l)
        y = torch.empty_like(x)
        case.mg.vmult(l, x, y)
        assert case.cmp(l, y, case.levels[l].A @ case.ovec(l, 10 + l)) < 1e-12, l
        assert case.cmp(l, case.mg.diagonal(l), case.levels[l].diag) < 1e-12, l
    for l in range(1, case.n):
        assert abs(case.mg.get_lambda(l) - case.levels[l].lam_max) < 1e-8 * case.levels[l].lam_max, l


def test_transfer_between_refinement_levels(case):
    for l in range(1, case.n):
        nc, nf = case.mg.n_free(l - 1), case.mg.n_free(l)
        if nc == 0 or nf == 0:
            continue
        P = case.levels[l].P
        xc = case.gvec(l - 1, 30 + l)
        yf = torch.zeros(nf, dtype=torch.float64, device="cuda")
        case.mg.prolongate_add(l, xc, yf)
        xf = case.gvec(l, 40 + l)
        yc = torch.zeros(nc, dtype=torch.float64, device="cuda")
        case.mg.restrict_add(l, xf, yc)
        assert case.cmp(l, yf, P @ case.ovec(l - 1, 30 + l)) < 1e-12, l
        assert case.cmp(l - 1, yc, P.T @ case.ovec(l, 40 + l)) < 1e-12, l


def test_vcycle_fp64(gcmg):
    c = LSCase(gcmg, synth.octant(4), 2)
    for l in range(1, c.n):
        c.mg.set_lambda(l, c.levels[l].lam_max)
    b = c.gvec(c.n, 9)
    x = torch.zeros_like(b)
    c.mg.vcycle(b, x)
    ls.set_precision(c.levels, np.float64)
    ref = ls.multigrid_vcycle(c.levels, c.cm, c.ovec(c.n, 9))
    assert c.cmp(c.n, x, ref) < 1e-10


@pytest.mark.parametrize("fp32", [False, True], ids=["mg64", "mg32"])
def test_cg_matches_oracle(gcmg, fp32):
    c = LSCase(gcmg, synth.octant(4), 2, fp32=fp32)
    bo = c.act.rhs()
    b = torch.tensor(bo[c.aperm], dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    st = c.mg.cg_solve(b, x, 1e-8)
    ref = ls.solve(c.act, c.levels, c.cm, bo, 1e-8, np.float32 if fp32 else np.float64)
    assert st.status == 0 and abs(st.iterations - ref.iterations) <= 1, (st.iterations, ref.iterations)
    xo = np.empty(len(c.aperm))
    xo[c.aperm] = x.cpu().numpy()
    assert np.linalg.norm(bo - c.act.apply(xo)) <= 1.01e-8 * np.linalg.norm(bo)


def test_uniform_mesh_equals_global_coarsening(gcmg):
    """No local refinement: the refinement levels are the global-coarsening
    levels and the copy is the identity, so the V-cycles agree bit for bit."""
    mesh = gcmg.Mesh.from_recipe(synth.uniform_cube(4))
    a = gcmg.Multigrid(mesh, 3, local_smoothing=True)
    g = gcmg.Multigrid(mesh, 3)
    assert a.num_levels == g.num_levels + 1
    assert np.array_equal(a.dof_coords(a.finest), g.dof_coords(g.finest))
    b = torch.tensor(synth.point_values(g.dof_coords(g.finest), 2), dtype=torch.float64, device="cuda")
    xa, xg = torch.zeros_like(b), torch.zeros_like(b)
    a.vcycle(b, xa)
    g.vcycle(b, xg)
    assert torch.equal(xa, xg)


@pytest.mark.parametrize("k,L", [(1, l) for l in range(3, 8)] + [(4, l) for l in range(3, 7)])
def test_iterations_table_4(gcmg, k, L):
    row = [r for r in table("octant_t4") if int(r[0]) == L][0]
    ref = row[1] if k == 1 else row[3]
    mg = gcmg.Multigrid(gcmg.Mesh.from_recipe(synth.octant(L)), k, local_smoothing=True)
    b = mg.rhs()
    x = torch.zeros_like(b)
    st = mg.cg_solve(b, x, 1e-4, maxit=50)
    assert st.status == 0 and st.rel_residual <= 1e-4
    assert ref - 1 <= st.iterations <= ref, (k, L, st.iterations, ref)


def test_unsupported_combinations(gcmg):
    mesh = gcmg.Mesh.from_recipe(synth.octant(2))
    with pytest.raises(gcmg.GcmgError):
        gcmg.Multigrid(mesh, 4, p_coarsening=True, local_smoothing=True)
    mg = gcmg.Multigrid(mesh, 2, local_smoothing=True)
    with pytest.raises(gcmg.GcmgError):
        mg.set_coefficient(torch.ones(mg.n_cells(mg.finest), dtype=torch.float64, device="cuda"))
    with pytest.raises(gcmg.GcmgError):  # no transfer into the active mesh
        mg.prolongate_add(mg.finest, torch.zeros(mg.n_free(mg.finest - 1), dtype=torch.float64, device="cuda"),
                          torch.zeros(mg.n_free(mg.finest), dtype=torch.float64, device="cuda"))
