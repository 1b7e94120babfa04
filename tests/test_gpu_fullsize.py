"""The benchmark workload at full size, in the launch configuration the
benchmark times: Q4 on the unit cube with five global refinements and two
more of the octant (296,535 cells, 18,740,987 free DoFs), 32-cell tiles, fp32
V-cycle inside fp64 CG.  The oracle cannot take this mesh whole in seconds,
so the checks are outputs it computes one by one and properties that hold at
any size:

* sampled operator rows: at support points whose neighbourhood is one level
  (all cells of that level within two cells are leaves, so no hanging node
  touches the row), (A x)_i is the sum over the cells around the point of
  h times the oracle's reference element matrix (Eq. 2 on a cube of edge h)
  times x at the cells' nodes; fp64 to 1e-12, fp32 to 2e-6;
* the fp32 operator against the fp64 operator on all 18.7 M rows, 2e-6;
* patch test (exactness for Q_k, hanging nodes included): for a polynomial u
  of degree <= 4 in each variable with -Delta u = f, the operator applied to
  u at the free DoFs equals the right-hand side with the lifted Dirichlet
  data, two independent kernels (the line operator and the cell kernel);
  fp64 to 1e-12, fp32 to 2e-6 (the oracle's own rounding on the same mesh
  family with 0.3 M DoFs: 3e-15 and 4e-7);
* symmetry <A x, y> = <x, A y>;
* transfer (Sec. 3.5): the prolongation reproduces a coarse Q_4 function that
  vanishes on the boundary exactly, and the restriction is its transpose;
* the benchmark's mixed-precision CG solve reaches 1e-8, the residual
  recomputed with the fp64 operator.
"""
import numpy as np
import pytest

import synth
from oracle import mesh as omesh
from parity import rel_err
from sampled import deep_cells, sampled_rows

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

W = synth.WORKLOAD_Q4_OCTANT
K = W.degree
N_FREE = 18740987
RES = 1 << 20  # the coordinate resolution of synth.point_values


@pytest.fixture(scope="module")
def big(gcmg):
    mg = gcmg.Multigrid(gcmg.Mesh.from_recipe(W.recipe), K, mg_fp32=True)
    xyz = mg.dof_coords(mg.finest)
    assert len(xyz) == N_FREE
    return mg, xyz


def _keys(xyz):
    q = np.rint(np.asarray(xyz, dtype=np.float64) * RES).astype(np.int64)
    return (q[:, 0] << 42) | (q[:, 1] << 21) | q[:, 2]


def test_sampled_rows_against_the_oracle(big):
    mg, xyz = big
    m = omesh.build_mesh(W.recipe)
    rng = np.random.default_rng(2203)
    cells = deep_cells(m, rng, 24)
    assert {c[0] for c in cells} >= {5, 7}  # the coarse region and the twice-refined octant
    seed = 41
    pos, ref = sampled_rows(m, K, cells, rng, seed)
    keys = _keys(xyz)
    order = np.argsort(keys)
    kp = _keys(pos)
    at = np.searchsorted(keys[order], kp)
    assert np.all(keys[order][at] == kp), "sampled support points are DoFs"
    rows = order[at]
    assert np.abs(xyz[rows] - pos).max() < 1e-12
    x = torch.tensor(synth.point_values(xyz, seed), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    mg.vmult(mg.finest, x, y)
    assert rel_err(y.cpu().numpy()[rows], ref) < 1e-12
    x32 = x.float()
    y32 = torch.empty_like(x32)
    mg.vmult(mg.finest, x32, y32)
    assert rel_err(y32.double().cpu().numpy()[rows], ref) < 2e-6
    # and on every row, against the fp64 operator
    assert rel_err(y32.double().cpu().numpy(), y.cpu().numpy()) < 2e-6


def test_patch_test_with_hanging_nodes(gcmg, big):
    mg, xyz = big
    terms = [(1.0, 2, 1, 0), (-0.5, 0, 0, 3), (0.3, 1, 1, 1), (0.25, 4, 0, 0), (0.7, 0, 2, 2), (0.1, 0, 0, 0)]
    u = sum(c * xyz[:, 0] ** a * xyz[:, 1] ** b * xyz[:, 2] ** d for c, a, b, d in terms)
    b = mg.rhs_dirichlet(gcmg.FUNC_POLYNOMIAL, terms)
    x = torch.tensor(u, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    mg.vmult(mg.finest, x, y)
    assert rel_err(y.cpu().numpy(), b.cpu().numpy()) < 1e-12
    x32 = x.float()
    y32 = torch.empty_like(x32)
    mg.vmult(mg.finest, x32, y32)
    assert rel_err(y32.double().cpu().numpy(), b.cpu().numpy()) < 2e-6


def test_symmetry(big):
    mg, xyz = big
    x = torch.tensor(synth.point_values(xyz, 5), dtype=torch.float64, device="cuda")
    z = torch.tensor(synth.point_values(xyz, 6), dtype=torch.float64, device="cuda")
    ax, az = torch.empty_like(x), torch.empty_like(z)
    mg.vmult(mg.finest, x, ax)
    mg.vmult(mg.finest, z, az)
    a, b = float(torch.dot(ax, z)), float(torch.dot(x, az))
    assert abs(a - b) <= 1e-12 * float(torch.linalg.norm(ax) * torch.linalg.norm(z))


def _bubble(p):
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    return x * (1 - x) * y * (1 - y) * z * (1 - z) * (0.5 + x * y)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 1e-6)], ids=["f64", "f32"])
def test_prolongation_reproduces_coarse_functions(big, dtype, tol):
    mg, xyz = big
    l = mg.finest
    xc = torch.tensor(_bubble(mg.dof_coords(l - 1)), dtype=dtype, device="cuda")
    yf = torch.zeros(mg.n_free(l), dtype=dtype, device="cuda")
    mg.prolongate_add(l, xc, yf)
    assert rel_err(yf.double().cpu().numpy(), _bubble(xyz)) < tol


def test_restriction_is_the_transpose(big):
    mg, xyz = big
    l = mg.finest
    xf = torch.tensor(synth.point_values(xyz, 7), dtype=torch.float64, device="cuda")
    yc = torch.tensor(synth.point_values(mg.dof_coords(l - 1), 8), dtype=torch.float64, device="cuda")
    rx = torch.zeros_like(yc)
    mg.restrict_add(l, xf, rx)
    py = torch.zeros_like(xf)
    mg.prolongate_add(l, yc, py)
    a, b = float(torch.dot(rx, yc)), float(torch.dot(xf, py))
    assert abs(a - b) <= 1e-12 * float(torch.linalg.norm(xf) * torch.linalg.norm(py))


def test_benchmark_solve(big):
    mg, _ = big
    f = synth.fourier_rhs(W.rhs_seed)
    b = mg.rhs((f.kappa, f.phi, f.amp))
    x = torch.zeros_like(b)
    st = mg.cg_solve(b, x, 1e-8, 100)
    assert st.status == 0 and st.rel_residual <= 1e-8 and st.iterations <= 10, st
    ax = torch.empty_like(x)
    mg.vmult(mg.finest, x, ax)
    assert float(torch.linalg.norm(b - ax)) <= 1.01e-8 * float(torch.linalg.norm(b))
