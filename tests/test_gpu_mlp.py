"""Parity of the learned per-cell smoother (CUDA path through the C ABI)
with the oracle (oracle/mlp.py), on the same seeded inputs.

Tolerances:
* cell gather and training rows: fp64 gather, fp32 rows -> 1e-6 relative
  (fp32 rounding of the rows);
* network forward / gradient / correction against the oracle's bf16 mode
  (the same operands rounded to bf16): 5e-3 relative; the remaining
  differences are fp32 vs fp64 accumulation, which moves a few operands
  across a bf16 rounding boundary (one bf16 ulp is 2^-8 relative);
* against the exact fp64 network: 3e-2 relative (bf16 operands, 8
  significand bits, through three layers);
* a constant network (zero weights, output bias v) has no bf16 operand that
  matters, so owners and scaling are checked to 1e-6.

The inference kernel works on batches of 128 cells; the 120-cell mesh is one
ragged batch, the 960-cell mesh (cube refined three times, octant once more)
seven full batches and a ragged one.  Every tensor-core wait is bounded, and
the count of waits that gave up must stay zero.
"""
import numpy as np
import pytest

import synth
from oracle import mesh as omesh, mg as omg, mlp as omlp
from oracle.space import Space
from parity import match, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

Q4_MESH = synth.cube_octant(2, 1)  # 120 cells, hanging faces and edges


class Q4Case:
    def __init__(self, gcmg, rec=Q4_MESH, fp32=False):
        self.gm = gcmg.Multigrid(gcmg.Mesh.from_recipe(rec), 4, mg_fp32=fp32)
        self.space = Space(omesh.build_mesh(rec), 4)
        L = self.gm.finest
        self.L = L
        self.xyz = self.gm.dof_coords(L)
        self.perm = match(self.xyz, self.space.free_coordinates())  # gpu i <-> oracle perm[i]
        lijk = self.gm.level_cells(L)
        index = {tuple(int(v) for v in c): i for i, c in enumerate(self.space.cells)}
        self.cell_map = np.array([index[tuple(int(v) for v in c)] for c in lijk])  # gpu cell -> oracle cell
        self.shape = omlp.Shape(*synth.mlp_shape(4))

    def gvec(self, seed, dtype=torch.float64):
        return torch.tensor(synth.point_values(self.xyz, seed), dtype=dtype, device="cuda")

    def ovec(self, seed):
        return synth.point_values(self.space.free_coordinates(), seed)

    def to_oracle(self, g):
        """GPU free vector -> oracle numbering."""
        out = np.empty(len(self.perm))
        out[self.perm] = g.double().cpu().numpy()
        return out


@pytest.fixture(scope="module")
def q4(gcmg):
    return Q4Case(gcmg)


def _net(gcmg, theta):
    net = gcmg.MLP(*synth.mlp_shape(4))
    net.set_params(torch.tensor(theta, dtype=torch.float32, device="cuda"))
    return net


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_cell_gather(gcmg, k):
    rec = synth.cube_octant(2, 1)
    gm = gcmg.Multigrid(gcmg.Mesh.from_recipe(rec), k)
    s = Space(omesh.build_mesh(rec), k)
    L = gm.finest
    xyz = gm.dof_coords(L)
    x = torch.tensor(synth.point_values(xyz, 7), dtype=torch.float64, device="cuda")
    lijk = gm.level_cells(L)
    index = {tuple(int(v) for v in c): i for i, c in enumerate(s.cells)}
    cmap = np.array([index[tuple(int(v) for v in c)] for c in lijk])
    ref = omlp.cell_values(s, synth.point_values(s.free_coordinates(), 7))[cmap]
    got = gm.cell_gather(L, x).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(ref).max()
    # a subset of cells in a given order
    cells = torch.tensor([5, 0, len(lijk) - 1, 17], dtype=torch.int32, device="cuda")
    got = gm.cell_gather(L, x, cells).cpu().numpy()
    assert np.array_equal(got, gm.cell_gather(L, x).cpu().numpy()[[5, 0, len(lijk) - 1, 17]])


def test_samples(q4):
    b, x, xs = q4.gvec(1), q4.gvec(2), q4.gvec(3)
    cells = torch.arange(q4.gm.n_cells(q4.L), dtype=torch.int32, device="cuda")
    X, T, W = q4.gm.mlp_samples(q4.L, b, x, xs, cells)
    s = q4.space
    r = q4.ovec(1) - s.apply(q4.ovec(2))
    Xo, _ = omlp.cell_features(s, r, s.diagonal())
    To = omlp.cell_targets(s, r, q4.ovec(3) - q4.ovec(2))
    Wo = omlp.cell_weights(s, r)
    assert rel_err(X.cpu().numpy(), Xo[q4.cell_map]) < 1e-6
    assert rel_err(T.cpu().numpy(), To[q4.cell_map]) < 1e-6
    assert rel_err(W.cpu().numpy(), Wo[q4.cell_map]) < 1e-6
    X2, T2, W2 = q4.gm.mlp_samples(q4.L, b, x, None, cells)
    assert T2 is None and torch.equal(X, X2) and torch.equal(W, W2)
    with pytest.raises(ValueError):
        q4.gm.mlp_samples(q4.L, b, x, xs, torch.tensor([0, q4.gm.n_cells(q4.L)], dtype=torch.int32, device="cuda"))


def test_forward(gcmg):
    shape = omlp.Shape(250, 128, 125)
    theta = synth.mlp_init(250, 128, 125, 11)
    X = synth.uniform_vector(300 * 250, 12).reshape(300, 250).astype(np.float32).astype(np.float64)
    net = _net(gcmg, theta)
    Y = net.forward(torch.tensor(X, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    Yb, _ = omlp.forward(shape, theta, X, bf16=True)
    Ye, _ = omlp.forward(shape, theta, X)
    assert np.abs(Y - Yb).max() <= 5e-3 * np.abs(Yb).max()
    assert rel_err(Y, Ye) < 3e-2


@pytest.mark.parametrize("sizes", [(250, 128, 125, 64, False), (250, 128, 125, 64, True), (54, 128, 27, 200, True),
                                   (7, 33, 5, 3, False)])
def test_gradient(gcmg, sizes):
    n_in, n_h, n_out, B, weighted = sizes
    shape = omlp.Shape(n_in, n_h, n_out)
    theta = synth.mlp_init(n_in, n_h, n_out, 13)
    X = synth.uniform_vector(B * n_in, 14).reshape(B, n_in).astype(np.float32).astype(np.float64)
    T = synth.uniform_vector(B * n_out, 15).reshape(B, n_out).astype(np.float32).astype(np.float64)
    W = synth.uniform_vector(B, 16, 0.0, 5.0).astype(np.float32).astype(np.float64) if weighted else None
    net = gcmg.MLP(n_in, n_h, n_out)
    net.set_params(torch.tensor(theta, dtype=torch.float32, device="cuda"))
    L, g = net.gradient(torch.tensor(X, dtype=torch.float32, device="cuda"),
                        torch.tensor(T, dtype=torch.float32, device="cuda"),
                        None if W is None else torch.tensor(W, dtype=torch.float32, device="cuda"))
    Lb, gb = omlp.loss_and_grad(shape, theta, X, T, bf16=True, W=W)
    Le, ge = omlp.loss_and_grad(shape, theta, X, T, W=W)
    g = g.double().cpu().numpy()
    assert abs(L.item() - Lb) <= 5e-3 * Lb
    assert rel_err(g, gb) < 5e-3
    assert rel_err(g, ge) < 3e-2
    # every block of the packed gradient, separately
    pos = 0
    for name, sh in shape.sizes():
        m = int(np.prod(sh))
        assert rel_err(g[pos:pos + m], gb[pos:pos + m]) < 1e-2, name
        pos += m


def test_training_steps(gcmg):
    shape = omlp.Shape(250, 128, 125)
    theta = synth.mlp_init(250, 128, 125, 21)
    n = 256
    X = synth.uniform_vector(n * 250, 22).reshape(n, 250).astype(np.float32).astype(np.float64)
    W = synth.uniform_vector(250 * 125, 23).reshape(250, 125) / 16
    T = (np.tanh(X @ W)).astype(np.float32).astype(np.float64)
    order = synth.sample_order(n, 3, 24)
    W = synth.uniform_vector(n, 25, 0.5, 2.0).astype(np.float32).astype(np.float64)
    net = _net(gcmg, theta)
    losses = net.train(torch.tensor(X, dtype=torch.float32, device="cuda"),
                       torch.tensor(T, dtype=torch.float32, device="cuda"),
                       torch.tensor(order, device="cuda"), 32, 1e-3,
                       W=torch.tensor(W, dtype=torch.float32, device="cuda")).double().cpu().numpy()
    theta_o, losses_o = omlp.train(shape, theta, X, T, order, 32, 1e-3, bf16=True, W=W)
    assert len(losses) == len(losses_o) == 24
    assert np.abs(losses - losses_o).max() <= 2e-2 * losses_o.max()
    assert losses[-4:].mean() < losses[:4].mean()
    th = net.get_params().double().cpu().numpy()
    assert rel_err(th - theta, theta_o - theta) < 5e-2  # the updates agree


def test_correct_constant_network(gcmg, q4):
    p = omlp.unpack(q4.shape, np.zeros(q4.shape.n_params()))
    v = synth.uniform_vector(125, 31)
    p["b3"] = v.astype(np.float32).astype(np.float64)
    theta = omlp.pack(q4.shape, p)
    net = _net(gcmg, theta)
    r = q4.gvec(32)
    x = torch.zeros_like(r)
    q4.gm.mlp_correct(q4.L, net, r, x)
    ref = omlp.correction(q4.space, q4.shape, theta, q4.ovec(32), q4.space.diagonal())
    assert rel_err(q4.to_oracle(x), ref) < 1e-6
    # it adds to x
    q4.gm.mlp_correct(q4.L, net, r, x)
    assert rel_err(q4.to_oracle(x), 2 * ref) < 1e-6


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_correct(gcmg, q4, dtype):
    theta = synth.mlp_init(250, 128, 125, 41)
    net = _net(gcmg, theta)
    dt = torch.float64 if dtype == "f64" else torch.float32
    rv = q4.ovec(42)
    if dtype == "f32":
        rv = rv.astype(np.float32).astype(np.float64)
    r = q4.gvec(42, dt)
    x = torch.zeros_like(r)
    q4.gm.mlp_correct(q4.L, net, r, x)
    got = q4.to_oracle(x)
    diag = q4.space.diagonal()
    ref_b = omlp.correction(q4.space, q4.shape, theta, rv, diag, bf16=True)
    ref_e = omlp.correction(q4.space, q4.shape, theta, rv, diag)
    assert np.abs(got - ref_b).max() <= 5e-3 * np.abs(ref_b).max()
    assert rel_err(got, ref_e) < 3e-2
    # positively 1-homogeneous in r
    x2 = torch.zeros_like(r)
    q4.gm.mlp_correct(q4.L, net, 4 * r, x2)
    assert rel_err(x2.double().cpu().numpy(), 4 * x.double().cpu().numpy()) < 1e-6
    assert gcmg.wait_timeouts() == 0


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_correct_several_batches(gcmg, dtype):
    case = Q4Case(gcmg, synth.cube_octant(3, 1))
    assert case.gm.n_cells(case.L) == 960
    theta = synth.mlp_init(250, 128, 125, 43)
    net = _net(gcmg, theta)
    dt = torch.float64 if dtype == "f64" else torch.float32
    rv = case.ovec(44)
    if dtype == "f32":
        rv = rv.astype(np.float32).astype(np.float64)
    x = torch.zeros(case.gm.n_free(case.L), dtype=dt, device="cuda")
    case.gm.mlp_correct(case.L, net, case.gvec(44, dt), x)
    got = case.to_oracle(x)
    ref_b = omlp.correction(case.space, case.shape, theta, rv, case.space.diagonal(), bf16=True)
    assert np.abs(got - ref_b).max() <= 5e-3 * np.abs(ref_b).max()
    assert gcmg.wait_timeouts() == 0


def test_correct_fp64_equals_fp32_on_the_rounded_residual(gcmg):
    """the network runs in fp32/bf16 either way: with x = 0 the fp64 result is
    the fp32 result widened, bit for bit, when r is rounded to fp32 first
    (this pins the fp64 <-> fp32 conversions of the kernel)"""
    case = Q4Case(gcmg, synth.cube_octant(3, 1))
    net = _net(gcmg, synth.mlp_init(250, 128, 125, 48))
    r64 = case.gvec(49) * torch.logspace(-30, 15, case.gm.n_free(case.L), dtype=torch.float64, device="cuda")
    r64[::97] = 0.0
    x64 = torch.zeros_like(r64)
    case.gm.mlp_correct(case.L, net, r64, x64)
    r32 = r64.float()
    x32 = torch.zeros_like(r32)
    case.gm.mlp_correct(case.L, net, r32, x32)
    assert torch.equal(x64, x32.double())
    assert gcmg.wait_timeouts() == 0


def test_correct_follows_parameter_changes(gcmg, q4):
    """the weight image and the first layer's diagonal part are rebuilt when
    the parameters change (set_params, Adam steps), and only then"""
    ta, tb = synth.mlp_init(250, 128, 125, 45), synth.mlp_init(250, 128, 125, 46)
    r = q4.gvec(47)
    net = _net(gcmg, ta)
    xa = torch.zeros_like(r)
    q4.gm.mlp_correct(q4.L, net, r, xa)
    xa2 = torch.zeros_like(r)
    q4.gm.mlp_correct(q4.L, net, r, xa2)
    assert torch.equal(xa, xa2)
    net.set_params(torch.tensor(tb, dtype=torch.float32, device="cuda"))
    xb = torch.zeros_like(r)
    q4.gm.mlp_correct(q4.L, net, r, xb)
    xb_ref = torch.zeros_like(r)
    q4.gm.mlp_correct(q4.L, _net(gcmg, tb), r, xb_ref)
    assert torch.equal(xb, xb_ref) and not torch.equal(xa, xb)
    # one Adam step changes the parameters, hence the correction
    X = torch.rand(64, 250, dtype=torch.float32, device="cuda")
    T = torch.rand(64, 125, dtype=torch.float32, device="cuda")
    net.train(X, T, torch.arange(64, dtype=torch.int32, device="cuda"), 64, 1e-3)
    xc = torch.zeros_like(r)
    q4.gm.mlp_correct(q4.L, net, r, xc)
    assert not torch.equal(xb, xc)
    assert gcmg.wait_timeouts() == 0


def test_smoother_arguments(gcmg, q4):
    net = gcmg.MLP(*synth.mlp_shape(4))
    with pytest.raises(gcmg.GcmgError):
        q4.gm.set_smoother(0, gcmg.SMOOTHER_MLP_AUGMENT, net)
    with pytest.raises(gcmg.GcmgError):
        q4.gm.set_smoother(q4.L, gcmg.SMOOTHER_MLP_AUGMENT, gcmg.MLP(54, 128, 27))
    with pytest.raises(gcmg.GcmgError):
        q4.gm.set_smoother(q4.L, 7, net)
    g2 = gcmg.Multigrid(gcmg.Mesh.from_recipe(Q4_MESH), 2)
    with pytest.raises(gcmg.GcmgError):
        g2.set_smoother(g2.finest, gcmg.SMOOTHER_MLP_AUGMENT, net)


@pytest.mark.parametrize("kind", ["augment", "replace"])
def test_learned_vcycle(gcmg, kind):
    rec = Q4_MESH
    gm = gcmg.Multigrid(gcmg.Mesh.from_recipe(rec), 4, mg_fp32=False)
    levels = omg.build_levels(omesh.build_mesh(rec), 4, assembled=False)
    top = levels[-1]
    s = top.space
    theta = synth.mlp_init(250, 128, 125, 51)
    shape = omlp.Shape(250, 128, 125)
    own = omlp.owners(s)
    top.learned = lambda r: omlp.correction(s, shape, theta, r, top.diag, bf16=True, own=own)
    top.learned_mode = kind
    net = _net(gcmg, theta)
    kind_id = gcmg.SMOOTHER_MLP_AUGMENT if kind == "augment" else gcmg.SMOOTHER_MLP_REPLACE
    gm.set_smoother(gm.finest, kind_id, net)
    xyz = gm.dof_coords(gm.finest)
    perm = match(xyz, s.free_coordinates())
    b = torch.tensor(synth.point_values(xyz, 52), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    gm.vcycle(b, x)
    xo = omg.multigrid_vcycle(levels, synth.point_values(s.free_coordinates(), 52))
    assert rel_err(x.cpu().numpy(), xo[perm]) < 5e-3


def test_flexible_cg_with_learned_smoother(gcmg):
    rec = Q4_MESH
    gm = gcmg.Multigrid(gcmg.Mesh.from_recipe(rec), 4, mg_fp32=True)
    levels = omg.build_levels(omesh.build_mesh(rec), 4, assembled=False)
    top = levels[-1]
    s = top.space
    theta = synth.mlp_init(250, 128, 125, 61)
    shape = omlp.Shape(250, 128, 125)
    own = omlp.owners(s)
    top.learned = lambda r: omlp.correction(s, shape, theta, r, top.diag, bf16=True, own=own)
    gm.set_smoother(gm.finest, gcmg.SMOOTHER_MLP_AUGMENT, _net(gcmg, theta))
    b = gm.rhs()
    x = torch.zeros_like(b)
    st = gm.cg_solve(b, x, 1e-8)
    bo = s.rhs()
    res = omg.solve(levels, bo, 1e-8, mg_dtype=np.float32, flexible=True)
    assert abs(st.iterations - res.iterations) <= 1
    xyz = gm.dof_coords(gm.finest)
    perm = match(xyz, s.free_coordinates())
    xo = np.empty(len(perm))
    xo[perm] = x.cpu().numpy()
    assert np.linalg.norm(bo - s.apply(xo)) <= 1.01e-8 * np.linalg.norm(bo)
