"""Parity of the CUDA path (through the C ABI) with the oracle, element by
element on the same seeded inputs.

Inputs are position-keyed random values (synth.point_values): each side
evaluates them at its own support points, so no input crosses from the CUDA
path to the oracle; outputs are compared after matching support points.

Tolerances (relative 2-norm):
* fp64 operator, diagonal, right-hand side, transfer, smoother, coarse
  solve: 1e-12 (sum-factorised vs assembled fp64: rounding differences of a
  few hundred operations, far below 1e-12);
* fp64 V-cycle: 1e-10 (all levels chained);
* fp32 operator: 2e-6 (unit roundoff 6e-8 times a chain of about 30
  dependent roundings through the gather, six sweeps, the scaling and the
  accumulation);
* CG: same iteration count as the oracle and ||b - A x|| / ||b|| <= rtol,
  evaluated with the oracle's own operator and right-hand side.
"""
import numpy as np
import pytest

import synth
from oracle import mesh as omesh, mg as omg, space as ospace
from parity import match, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


class Case:
    def __init__(self, gcmg, rec, k, p=False, fp32=False, tile_cells=0, cell_kernel=0):
        self.rec, self.k = rec, k
        self.mesh = gcmg.Mesh.from_recipe(rec)
        self.mg = gcmg.Multigrid(self.mesh, k, p_coarsening=p, mg_fp32=fp32, tile_cells=tile_cells,
                                 cell_kernel=cell_kernel)
        self.levels = omg.build_levels(omesh.build_mesh(rec), k, p_coarsening=p, assembled=(k <= 2))
        assert self.mg.num_levels == len(self.levels)
        self.xyz = [self.mg.dof_coords(l) for l in range(self.mg.num_levels)]
        self.perm = [match(self.xyz[l], self.levels[l].space.free_coordinates()) for l in range(self.mg.num_levels)]

    def gvec(self, l, seed, dtype=torch.float64):
        return torch.tensor(synth.point_values(self.xyz[l], seed), dtype=dtype, device="cuda")

    def ovec(self, l, seed):
        return synth.point_values(self.levels[l].space.free_coordinates(), seed)

    def cmp(self, l, gpu, oracle):
        """relative error of a GPU vector against an oracle vector"""
        g = gpu.double().cpu().numpy() if hasattr(gpu, "cpu") else gpu
        return rel_err(g, oracle[self.perm[l]])


CASES = [
    (synth.octant(3), 1), (synth.octant(3), 2), (synth.octant(3), 3), (synth.octant(3), 4),
    (synth.cube_octant(3, 1), 2), (synth.cube_octant(2, 1), 4), (synth.sphere(4), 3), (synth.octant(4), 2),
    (synth.shell(5), 1),
]
IDS = [f"{r.name}-Q{k}" for r, k in CASES]


@pytest.fixture(scope="module", params=list(range(len(CASES))), ids=IDS)
def case(request, gcmg):
    rec, k = CASES[request.param]
    return Case(gcmg, rec, k)


def test_level_sizes(case):
    for l, lev in enumerate(case.levels):
        assert case.mg.n_free(l) == lev.space.n_free
        assert case.mg.level_info(l).n_cells == lev.space.nc


def test_vmult_fp64(case):
    for l in range(case.mg.num_levels):
        n = case.mg.n_free(l)
        if n == 0:
            continue
        x = case.gvec(l, 100 + l)
        y = torch.empty_like(x)
        case.mg.vmult(l, x, y)
        torch.cuda.synchronize()
        ref = case.levels[l].apply64(case.ovec(l, 100 + l))
        assert case.cmp(l, y, ref) < 1e-12, l


def test_vmult_fp32(case):
    l = case.mg.finest
    if case.mg.n_free(l) == 0:
        return
    x = case.gvec(l, 7, torch.float32)
    y = torch.empty_like(x)
    case.mg.vmult(l, x, y)
    torch.cuda.synchronize()
    ref = case.levels[l].apply64(case.ovec(l, 7).astype(np.float32).astype(np.float64))
    assert case.cmp(l, y, ref) < 2e-6


def test_diagonal(case):
    for l in range(case.mg.num_levels):
        if case.mg.n_free(l) == 0:
            continue
        assert case.cmp(l, case.mg.diagonal(l), case.levels[l].diag) < 1e-12, l


def test_rhs_constant_and_fourier(case):
    l = case.mg.finest
    if case.mg.n_free(l) == 0:
        return
    sp = case.levels[l].space
    assert case.cmp(l, case.mg.rhs(), sp.rhs()) < 1e-12
    f = synth.fourier_rhs(2203)
    assert case.cmp(l, case.mg.rhs((f.kappa, f.phi, f.amp)), sp.rhs(ospace.fourier_function(f))) < 1e-12


def test_transfer(case):
    for l in range(1, case.mg.num_levels):
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
        torch.cuda.synchronize()
        assert case.cmp(l, yf, P @ case.ovec(l - 1, 30 + l)) < 1e-12, l
        assert case.cmp(l - 1, yc, P.T @ case.ovec(l, 40 + l)) < 1e-12, l


def test_lambda_estimate(case):
    for l in range(1, case.mg.num_levels):
        if case.mg.n_free(l) == 0:
            continue
        assert abs(case.mg.get_lambda(l) - case.levels[l].lam_max) < 1e-8 * case.levels[l].lam_max, l


def test_smoother_fp64(case):
    for l in range(1, case.mg.num_levels):
        if case.mg.n_free(l) == 0:
            continue
        lev = case.levels[l]
        case.mg.set_lambda(l, lev.lam_max)
        b = case.gvec(l, 50 + l)
        x = torch.zeros_like(b)
        case.mg.smooth(l, x, b, True)
        x2 = case.gvec(l, 60 + l)
        case.mg.smooth(l, x2, b, False)
        torch.cuda.synchronize()
        bo = case.ovec(l, 50 + l)
        ref = omg.chebyshev(lev.apply64, 1.0 / lev.diag, bo, None, lev.lam_max)
        ref2 = omg.chebyshev(lev.apply64, 1.0 / lev.diag, bo, case.ovec(l, 60 + l), lev.lam_max)
        assert case.cmp(l, x, ref) < 1e-12, l
        assert case.cmp(l, x2, ref2) < 1e-12, l


def test_coarse_solve(case):
    n = case.mg.n_free(0)
    if n == 0:
        return
    b = case.gvec(0, 3)
    x = torch.zeros_like(b)
    case.mg.coarse_solve(b, x)
    torch.cuda.synchronize()
    lev = case.levels[0]
    import scipy.linalg as sla
    assert case.cmp(0, x, sla.cho_solve(lev.chol, case.ovec(0, 3))) < 1e-12


def test_vcycle_fp64(gcmg):
    c = Case(gcmg, synth.cube_octant(2, 1), 4)
    for l in range(1, c.mg.num_levels):
        c.mg.set_lambda(l, c.levels[l].lam_max)
    l = c.mg.finest
    b = c.gvec(l, 9)
    x = torch.zeros_like(b)
    c.mg.vcycle(b, x)
    torch.cuda.synchronize()
    omg.set_precision(c.levels, np.float64)
    ref = omg.multigrid_vcycle(c.levels, c.ovec(l, 9))
    assert c.cmp(l, x, ref) < 1e-10


@pytest.mark.parametrize("rec,k", [(synth.octant(3), 1), (synth.octant(4), 1), (synth.octant(3), 4),
                                   (synth.cube_octant(3, 1), 2)], ids=["oct3-Q1", "oct4-Q1", "oct3-Q4", "cfg-Q2"])
@pytest.mark.parametrize("fp32", [False, True], ids=["mg64", "mg32"])
def test_cg_solve(gcmg, rec, k, fp32):
    c = Case(gcmg, rec, k, fp32=fp32)
    l = c.mg.finest
    b = c.mg.rhs()
    x = torch.zeros_like(b)
    st = c.mg.cg_solve(b, x, 1e-8, 100)
    torch.cuda.synchronize()
    lev = c.levels[-1]
    bo = lev.space.rhs()
    xo = np.empty(lev.space.n_free)
    xo[c.perm[l]] = x.cpu().numpy()
    res = np.linalg.norm(bo - lev.apply64(xo)) / np.linalg.norm(bo)
    assert res <= 1e-8 * 1.01
    ref = omg.solve(c.levels, bo, 1e-8, np.float64)
    assert abs(st.iterations - ref.iterations) <= (1 if fp32 else 0)


def test_p_coarsening_hierarchy(gcmg):
    c = Case(gcmg, synth.sphere(3), 4, p=True)
    degs = [c.mg.level_info(l).degree for l in range(c.mg.num_levels)]
    assert degs[-3:] == [1, 2, 4] and all(d == 1 for d in degs[:-2])
    for l in range(1, c.mg.num_levels):
        nc, nf = c.mg.n_free(l - 1), c.mg.n_free(l)
        if nc == 0 or nf == 0:
            continue
        xc = c.gvec(l - 1, 70 + l)
        yf = torch.zeros(nf, dtype=torch.float64, device="cuda")
        c.mg.prolongate_add(l, xc, yf)
        xf = c.gvec(l, 80 + l)
        yc = torch.zeros(nc, dtype=torch.float64, device="cuda")
        c.mg.restrict_add(l, xf, yc)
        torch.cuda.synchronize()
        P = c.levels[l].P
        assert c.cmp(l, yf, P @ c.ovec(l - 1, 70 + l)) < 1e-12, l
        assert c.cmp(l - 1, yc, P.T @ c.ovec(l, 80 + l)) < 1e-12, l
    b = c.mg.rhs()
    x = torch.zeros_like(b)
    st = c.mg.cg_solve(b, x, 1e-8, 100)
    ref = omg.solve(c.levels, c.levels[-1].space.rhs(), 1e-8, np.float64)
    assert abs(st.iterations - ref.iterations) <= 1


def test_results_are_bit_reproducible(gcmg):
    c = Case(gcmg, synth.octant(4), 2)
    l = c.mg.finest
    x = c.gvec(l, 1)
    y1, y2 = torch.empty_like(x), torch.empty_like(x)
    c.mg.vmult(l, x, y1)
    c.mg.vmult(l, x, y2)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)


def test_tile_size_does_not_change_the_operator(gcmg):
    a = Case(gcmg, synth.octant(3), 3, tile_cells=4)
    b = Case(gcmg, synth.octant(3), 3, tile_cells=200)
    l = a.mg.finest
    xa, xb = a.gvec(l, 2), b.gvec(l, 2)
    ya, yb = torch.empty_like(xa), torch.empty_like(xb)
    a.mg.vmult(l, xa, ya)
    b.mg.vmult(l, xb, yb)
    torch.cuda.synchronize()
    ref = a.levels[l].apply64(a.ovec(l, 2))
    assert a.cmp(l, ya, ref) < 1e-12 and b.cmp(l, yb, ref) < 1e-12


def test_single_cell_q1_has_no_dofs(gcmg):
    m = gcmg.Mesh(0.0, 1.0, [])
    mg = gcmg.Multigrid(m, 1)
    assert mg.num_levels == 1 and mg.n_free(0) == 0
    b = torch.zeros(0, dtype=torch.float64, device="cuda")
    st = mg.cg_solve(b, torch.zeros_like(b), 1e-8, 10)
    assert st.iterations == 0


@pytest.mark.parametrize("fp32", [False, True], ids=["mg64", "mg32"])
def test_zero_right_hand_side(gcmg, fp32):
    """b = 0: no iteration, x = 0 whatever it held"""
    mg = gcmg.Multigrid(gcmg.Mesh.from_recipe(synth.octant(3)), 2, mg_fp32=fp32)
    b = torch.zeros(mg.n_free(mg.finest), dtype=torch.float64, device="cuda")
    x = torch.full_like(b, 3.0)
    st = mg.cg_solve(b, x, 1e-8, 10)
    assert st.status == 0 and st.iterations == 0
    assert torch.count_nonzero(x) == 0


@pytest.mark.parametrize("n", [1, 255, 1000, 304 * 256 + 17, 3_000_001])
def test_dot_fp64(gcmg, n):
    mg = gcmg.Multigrid(gcmg.Mesh(0.0, 1.0, [(0,)]), 2)
    x = torch.tensor(synth.uniform_vector(n, 1), dtype=torch.float64, device="cuda")
    y = torch.tensor(synth.uniform_vector(n, 2), dtype=torch.float64, device="cuda")
    r1 = mg.dot(x, y).item()
    r2 = mg.dot(x, y).item()
    ref = float(np.dot(synth.uniform_vector(n, 1), synth.uniform_vector(n, 2)))
    assert r1 == r2  # deterministic
    assert abs(r1 - ref) <= 1e-13 * max(1.0, np.sqrt(n))


def test_graphs_match_stream_launches(gcmg):
    mesh = gcmg.Mesh.from_recipe(synth.octant(4))
    a = gcmg.Multigrid(mesh, 3, mg_fp32=True)
    b = gcmg.Multigrid(mesh, 3, mg_fp32=True)
    b.set_graphs(False)
    rhs = a.rhs()
    xa, xb = torch.zeros_like(rhs), torch.zeros_like(rhs)
    sa = a.cg_solve(rhs, xa, 1e-8)
    sb = b.cg_solve(rhs, xb, 1e-8)
    assert sa.iterations == sb.iterations
    assert torch.equal(xa, xb)
    # a second solve replays the captured graphs
    xa2 = torch.zeros_like(rhs)
    a.cg_solve(rhs, xa2, 1e-8)
    assert torch.equal(xa, xa2)
    ya, yb = torch.zeros_like(rhs), torch.zeros_like(rhs)
    a.vcycle(rhs, ya)
    b.vcycle(rhs, yb)
    torch.cuda.synchronize()
    assert torch.equal(ya, yb)


def test_profiling_inside_graphs(gcmg):
    mesh = gcmg.Mesh.from_recipe(synth.octant(4))
    mg = gcmg.Multigrid(mesh, 2, mg_fp32=True)
    rhs = mg.rhs()
    x = torch.zeros_like(rhs)
    mg.set_profiling(True)
    st = mg.cg_solve(rhs, x, 1e-8)
    L = mg.finest
    cnt, ms = mg.profile(L, "vmult")
    cnt64, ms64 = mg.profile(L, "cg_vmult")
    assert cnt64 == st.iterations and ms64 > 0
    # presmoothing 2, residual 1, postsmoothing 3 operator applications per V-cycle
    assert cnt == 6 * (st.iterations) and ms > 0
    mg.set_profiling(False)


@pytest.mark.parametrize("rec,k", [(synth.octant(3), 4), (synth.cube_octant(3, 1), 2), (synth.sphere(4), 3)],
                         ids=["octant3-Q4", "cube3+1-Q2", "sphere4-Q3"])
@pytest.mark.parametrize("tc", [32, 64])
def test_vmult_fp32_slab_kernel(gcmg, rec, k, tc):
    """The slab-thread mapping (k+1 threads per cell) computes the same operator."""
    c = Case(gcmg, rec, k, tile_cells=tc, cell_kernel=2)
    for l in range(c.mg.num_levels):
        if c.mg.n_free(l) == 0:
            continue
        x = c.gvec(l, 700 + l, torch.float32)
        y = torch.empty_like(x)
        c.mg.vmult(l, x, y)
        torch.cuda.synchronize()
        ref = c.levels[l].apply64(c.ovec(l, 700 + l).astype(np.float32).astype(np.float64))
        assert c.cmp(l, y, ref) < 2e-6, l


@pytest.mark.parametrize("rec,k", [(synth.octant(3), 4), (synth.cube_octant(2, 1), 4), (synth.sphere(4), 3),
                                   (synth.octant(4), 2)], ids=["octant3-Q4", "cube2+1-Q4", "sphere4-Q3", "octant4-Q2"])
def test_vmult_lane_kernel_on_every_tile_size(gcmg, rec, k):
    """cell_kernel 3 runs the one-lane-per-cell kernels (fp32 and double-float)
    on every level, also on the coarse levels' 8- and 16-cell tiles (the
    default takes the line kernels there): Eq. 2 on every level against the
    oracle, fp64 to 1e-12 and fp32 to 2e-6."""
    c = Case(gcmg, rec, k, cell_kernel=3)
    for l in range(c.mg.num_levels):
        if c.mg.n_free(l) == 0:
            continue
        x = c.gvec(l, 800 + l)
        y = torch.empty_like(x)
        c.mg.vmult(l, x, y)
        x32 = c.gvec(l, 900 + l, torch.float32)
        y32 = torch.empty_like(x32)
        c.mg.vmult(l, x32, y32)
        torch.cuda.synchronize()
        lev = c.levels[l]
        assert c.cmp(l, y, lev.apply64(c.ovec(l, 800 + l))) < 1e-12, l
        assert c.cmp(l, y32, lev.apply64(c.ovec(l, 900 + l).astype(np.float32).astype(np.float64))) < 2e-6, l


@pytest.mark.parametrize("tc", [20, 24, 12])
def test_tile_sizes_compute_the_same_operator(gcmg, tc):
    """Tiles of 20 cells put the fp64 kernel's dynamic shared memory just
    under 48 KB, where the static shared memory pushes the total over the
    default limit (a launch error before the opt-in threshold was lowered)."""
    mesh = gcmg.Mesh.from_recipe(synth.cube_octant(4, 1))
    a = gcmg.Multigrid(mesh, 4, tile_cells=tc)
    b = gcmg.Multigrid(mesh, 4)
    assert a.info[a.finest].tile_cells == tc
    perm = match(a.dof_coords(a.finest), b.dof_coords(b.finest))
    for dt, tol in ((torch.float64, 1e-13), (torch.float32, 2e-6)):
        xa = torch.tensor(synth.point_values(a.dof_coords(a.finest), 9), dtype=dt, device="cuda")
        xb = torch.tensor(synth.point_values(b.dof_coords(b.finest), 9), dtype=dt, device="cuda")
        ya, yb = torch.empty_like(xa), torch.empty_like(xb)
        a.vmult(a.finest, xa, ya)
        b.vmult(b.finest, xb, yb)
        assert rel_err(ya.double().cpu().numpy(), yb.double().cpu().numpy()[perm]) < tol


@pytest.mark.parametrize("fp64", [False, True], ids=["f32", "f64"])
def test_vmult_host_pipeline_equals_device_vmult(gcmg, fp64):
    """gcmg_vmult_host overlaps the input copy (in DoF order, on a second
    stream) with groups of tiles; the result is the device operator's, bit
    for bit"""
    mg = gcmg.Multigrid(gcmg.Mesh.from_recipe(synth.cube_octant(3, 1)), 4)
    l = mg.finest
    assert mg.level_info(l).n_tiles >= 8
    dt = torch.float64 if fp64 else torch.float32
    x = torch.tensor(synth.point_values(mg.dof_coords(l), 12), dtype=dt, device="cuda")
    y = torch.empty_like(x)
    mg.vmult(l, x, y)
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    mg.vmult_host(l, xh.numpy(), yh.numpy())
    assert torch.equal(yh, y.cpu())


@pytest.mark.parametrize("fp64", [False, True], ids=["f32", "f64"])
def test_vmult_host_many_equals_device_vmult(gcmg, fp64):
    """gcmg_vmult_host_many overlaps the copies of neighbouring vectors with
    the operators (two device buffer pairs, three streams); every result is
    the device operator's, bit for bit, also for an odd count and when an
    input buffer is reused"""
    mg = gcmg.Multigrid(gcmg.Mesh.from_recipe(synth.cube_octant(3, 1)), 4)
    l = mg.finest
    dt = torch.float64 if fp64 else torch.float32
    xyz = mg.dof_coords(l)
    xs = [torch.tensor(synth.point_values(xyz, 20 + i), dtype=dt, device="cuda") for i in range(5)]
    ys = []
    for x in xs:
        y = torch.empty_like(x)
        mg.vmult(l, x, y)
        ys.append(y.cpu())
    xh = [x.cpu().pin_memory() for x in xs]
    srcs = [xh[0], xh[1], xh[2], xh[3], xh[4], xh[1]]
    yh = [torch.empty_like(xh[0]).pin_memory() for _ in srcs]
    mg.vmult_host_many(l, [a.numpy() for a in srcs], [b.numpy() for b in yh])
    for i, j in enumerate([0, 1, 2, 3, 4, 1]):
        assert torch.equal(yh[i], ys[j]), i
    mg.vmult_host_many(l, [], [])  # nothing to do
