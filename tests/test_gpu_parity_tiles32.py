"""Parity, row by row against the oracle, of the kernels in the launch
configuration the benchmark times, on a mesh with hanging nodes that the
oracle takes whole: Q4 on the unit cube refined globally four times and twice
more in the octant x, y, z < 1/2 (37,871 cells, 2,363,419 free DoFs; the
benchmark is the same recipe with five global refinements).  The finest level
has more than 2 x 152 x 32 cells, so it runs the default 32-cell tiles: the
one-lane-per-cell fp32 operator and the double-float fp64 operator with the
tile size of the benchmark level, on tiles with and without hanging cells
(3,896 cells with a hanging support point, 248,560 rows touched by one).

Every row of A x is compared (Eq. 2 with the constraints of Sec. 3.2): the
relative 2-norm, and the largest element-wise error relative to max |A x|,
over all rows and over the rows of DoFs that lie in a cell with a hanging
node (where the constraint interpolation C_e acts), so that a wrong value at
a few hundred hanging rows cannot hide in the norm of 2.4 M rows.
Tolerances from the arithmetic:
* fp32 operators: 2-norm 2e-6 (unit roundoff 6e-8 times a chain of about 30
  dependent roundings); element-wise 1e-5 of max |A x| (a row sums up to
  8 x 125 products whose magnitudes exceed the row's value by up to a factor
  of 5);
* fp64 (double-float, about 48 significand bits): 1e-12 both ways.
The transfers of the finest level (Sec. 3.5, Eqs. 5-7) are compared with the
oracle's prolongation matrix P (fine point values of the coarse function) and
R = P^T, the restriction in both chunk sizes of its kernel (4 coarse cells per
chunk, which the benchmark's finest transfer runs, and 8): fp64 1e-12, fp32
2e-6 / 1e-5 as above.
"""
import numpy as np
import pytest

import synth
from oracle import mesh as omesh, space as ospace, transfer as otr
from parity import match, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

REC = synth.cube_octant(4, 2)
K = 4


@pytest.fixture(scope="module")
def oracle_spaces():
    meshes = omesh.gc_hierarchy(omesh.build_mesh(REC))
    fine = ospace.Space(meshes[-1], K)
    coarse = ospace.Space(meshes[-2], K)
    return fine, coarse, otr.prolongation_matrix(fine, coarse)


def _hanging_rows(space):
    """free DoFs of the oracle space that lie in a cell with a hanging node"""
    nodes = space.cell_nodes[space.cell_has_hanging].ravel()
    fi = space.free_index[nodes]
    return np.unique(fi[fi >= 0])


class Gpu:
    def __init__(self, gcmg, fine, coarse, **kw):
        self.mg = gcmg.Multigrid(gcmg.Mesh.from_recipe(REC), K, mg_fp32=True, **kw)
        self.l = self.mg.finest
        assert self.mg.n_free(self.l) == fine.n_free == 2363419
        self.perm_f = match(self.mg.dof_coords(self.l), fine.free_coordinates())
        self.perm_c = match(self.mg.dof_coords(self.l - 1), coarse.free_coordinates())

    def vec(self, level, seed, dtype):
        xyz = self.mg.dof_coords(level)
        return torch.tensor(synth.point_values(xyz, seed), dtype=dtype, device="cuda")


def _check(gpu_vals, perm, ref, rows, tol2, tolmax, what):
    g = gpu_vals.double().cpu().numpy()
    o = ref[perm]
    scale = np.abs(o).max()
    err = np.abs(g - o)
    hang = np.zeros(len(ref), dtype=bool)
    hang[rows] = True
    e2, emax, ehang = rel_err(g, o), err.max() / scale, err[hang[perm]].max() / scale
    print(f"{what}: 2-norm {e2:.2e}, max {emax:.2e}, max over hanging rows {ehang:.2e}")
    assert e2 < tol2, (what, e2)
    assert emax < tolmax, (what, emax)
    assert ehang < tolmax, (what, ehang)
    return e2, emax, ehang


_GPUS = {}


def _gpu(gcmg, oracle_spaces, **kw):
    """one handle per configuration for the whole module"""
    key = tuple(sorted(kw.items()))
    if key not in _GPUS:
        fine, coarse, _ = oracle_spaces
        _GPUS[key] = Gpu(gcmg, fine, coarse, **kw)
    return _GPUS[key]


@pytest.fixture(scope="module")
def default_gpu(gcmg, oracle_spaces):
    g = _gpu(gcmg, oracle_spaces)
    info = g.mg.level_info(g.l)
    assert info.tile_cells == 32 and info.n_tiles == (37871 + 31) // 32
    yield g
    _GPUS.clear()


def test_mesh_has_hanging_tiles(oracle_spaces):
    fine, _, _ = oracle_spaces
    assert int(fine.cell_has_hanging.sum()) > 1000 and fine.n_hanging > 10000


@pytest.mark.parametrize("kernel", ["lanes", "lines"])
def test_fp32_operator_rows(gcmg, oracle_spaces, default_gpu, kernel):
    fine, coarse, _ = oracle_spaces
    g = default_gpu if kernel == "lanes" else _gpu(gcmg, oracle_spaces, cell_kernel=1)
    x = g.vec(g.l, 11, torch.float32)
    y = torch.empty_like(x)
    g.mg.vmult(g.l, x, y)
    torch.cuda.synchronize()
    xo = synth.point_values(fine.free_coordinates(), 11).astype(np.float32).astype(np.float64)
    _check(y, g.perm_f, fine.apply(xo), _hanging_rows(fine), 2e-6, 1e-5, f"fp32 {kernel}")


def test_fp64_operator_rows(oracle_spaces, default_gpu):
    fine, _, _ = oracle_spaces
    g = default_gpu
    x = g.vec(g.l, 12, torch.float64)
    y = torch.empty_like(x)
    g.mg.vmult(g.l, x, y)
    torch.cuda.synchronize()
    ref = fine.apply(synth.point_values(fine.free_coordinates(), 12))
    _check(y, g.perm_f, ref, _hanging_rows(fine), 1e-12, 1e-12, "fp64")


@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
def test_prolongation_rows(oracle_spaces, default_gpu, dtype):
    fine, coarse, P = oracle_spaces
    g = default_gpu
    dt = torch.float64 if dtype == "fp64" else torch.float32
    xc = g.vec(g.l - 1, 13, dt)
    yf = torch.zeros(g.mg.n_free(g.l), dtype=dt, device="cuda")
    g.mg.prolongate_add(g.l, xc, yf)
    torch.cuda.synchronize()
    xo = synth.point_values(coarse.free_coordinates(), 13)
    if dtype == "fp32":
        xo = xo.astype(np.float32).astype(np.float64)
    tol2, tolm = (1e-12, 1e-12) if dtype == "fp64" else (2e-6, 1e-5)
    _check(yf, g.perm_f, P @ xo, _hanging_rows(fine), tol2, tolm, f"prolongation {dtype}")


@pytest.mark.parametrize("chunk", [4, 8])
@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
def test_restriction_rows(gcmg, oracle_spaces, default_gpu, chunk, dtype):
    fine, coarse, P = oracle_spaces
    g = _gpu(gcmg, oracle_spaces, transfer_chunk=chunk)
    dt = torch.float64 if dtype == "fp64" else torch.float32
    xf = g.vec(g.l, 14, dt)
    yc = torch.zeros(g.mg.n_free(g.l - 1), dtype=dt, device="cuda")
    g.mg.restrict_add(g.l, xf, yc)
    torch.cuda.synchronize()
    xo = synth.point_values(fine.free_coordinates(), 14)
    if dtype == "fp32":
        xo = xo.astype(np.float32).astype(np.float64)
    tol2, tolm = (1e-12, 1e-12) if dtype == "fp64" else (2e-6, 1e-5)
    _check(yc, g.perm_c, P.T @ xo, _hanging_rows(coarse), tol2, tolm, f"restriction {dtype} chunk {chunk}")
