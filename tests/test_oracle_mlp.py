"""Pins of oracle/mlp.py (learned per-cell smoother) and of the flexible CG
and learned-step hooks of oracle/mg.py: closed forms, finite differences,
textbook element matrices, brute-force orderings and invariants."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as sla

import synth
from oracle import fe, mesh as omesh, mg, mlp
from oracle.space import Space


# ---------------------------------------------------------------------------
# GELU and bf16 rounding
# ---------------------------------------------------------------------------
def test_gelu_closed_forms():
    z = np.linspace(-6, 6, 97)
    # Phi(z) + Phi(-z) = 1  =>  g(z) - g(-z) = z
    assert np.abs(mlp.gelu(z) - mlp.gelu(-z) - z).max() < 1e-15 * 8
    assert mlp.gelu(0.0) == 0.0
    # g(1) = Phi(1), the standard normal distribution at 1
    assert abs(mlp.gelu(1.0) - 0.8413447460685429) < 1e-15
    # g(z) -> z for large z, -> 0 for very negative z
    assert abs(mlp.gelu(10.0) - 10.0) < 1e-15 and abs(mlp.gelu(-10.0)) < 1e-20
    assert abs(mlp.gelu_grad(0.0) - 0.5) < 1e-16
    h = 1e-5
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.abs(fd - mlp.gelu_grad(z)).max() < 1e-9


def test_round_bf16():
    exact = np.array([1.0, 0.5, -3.0, 2.0 ** -20, 0.0, 1.0 + 2.0 ** -7, 384.0])
    assert np.array_equal(mlp.round_bf16(exact), exact)
    # 8 significand bits: 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> even (1)
    assert mlp.round_bf16(1.0 + 2.0 ** -8) == 1.0
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6 -> even (1 + 2^-6)
    assert mlp.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert mlp.round_bf16(1.0 + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7
    assert mlp.round_bf16(-(1.0 + 3 * 2.0 ** -8)) == -(1.0 + 2.0 ** -6)
    x = synth.uniform_vector(10000, 3, -100, 100)
    r = mlp.round_bf16(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x) * 1.0000001)
    assert np.array_equal(mlp.round_bf16(r), r)
    # rounded values have at most 8 significand bits
    m, _ = np.frexp(r[r != 0])
    assert np.all(np.abs(m * 2 ** 8 - np.rint(m * 2 ** 8)) == 0)


# ---------------------------------------------------------------------------
# network, loss, gradient, Adam
# ---------------------------------------------------------------------------
def _small(seed=1, n_in=6, n_h=5, n_out=4, B=7):
    shape = mlp.Shape(n_in, n_h, n_out)
    theta = synth.mlp_init(n_in, n_h, n_out, seed)
    X = synth.uniform_vector(B * n_in, seed + 10).reshape(B, n_in)
    T = synth.uniform_vector(B * n_out, seed + 20).reshape(B, n_out)
    return shape, theta, X, T


def test_forward_is_the_composition():
    shape, theta, X, T = _small()
    p = mlp.unpack(shape, theta)
    Y, _ = mlp.forward(shape, theta, X)
    for b in range(X.shape[0]):
        h1 = [mlp.gelu(sum(p["W1"][j, i] * X[b, i] for i in range(6)) + p["b1"][j]) for j in range(5)]
        h2 = [mlp.gelu(sum(p["W2"][j, i] * h1[i] for i in range(5)) + p["b2"][j]) for j in range(5)]
        y = [sum(p["W3"][o, i] * h2[i] for i in range(5)) + p["b3"][o] for o in range(4)]
        assert np.allclose(Y[b], y, rtol=0, atol=1e-14)
    assert np.array_equal(mlp.pack(shape, p), theta)


@pytest.mark.parametrize("sizes", [(6, 5, 4, 7), (250, 128, 125, 3)])
def test_gradient_matches_finite_differences(sizes):
    n_in, n_h, n_out, B = sizes
    shape, theta, X, T = _small(2, n_in, n_h, n_out, B)
    L, g = mlp.loss_and_grad(shape, theta, X, T)
    Y, _ = mlp.forward(shape, theta, X)
    assert abs(L - 0.5 * np.sum((Y - T) ** 2) / B) < 1e-14
    idx = np.arange(len(theta)) if len(theta) < 200 else \
        (synth.splitmix64_array(5, 60) % np.uint64(len(theta))).astype(np.int64)
    # the biases of the last layer and some of the first are always checked
    idx = np.concatenate([idx, [len(theta) - 1, n_h * n_in, n_h * n_in - 1]])
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(shape, tp, X, T)[0] - mlp.loss_and_grad(shape, tm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, np.abs(g).max()), (i, fd, g[i])


def test_weighted_loss():
    shape, theta, X, T = _small(4, 6, 5, 4, 9)
    W = synth.uniform_vector(9, 50, 0.1, 3.0)
    L1, g1 = mlp.loss_and_grad(shape, theta, X, T)
    L2, g2 = mlp.loss_and_grad(shape, theta, X, T, W=np.ones(9))
    assert L1 == L2 and np.array_equal(g1, g2)
    # invariant under scaling all weights
    La, ga = mlp.loss_and_grad(shape, theta, X, T, W=W)
    Lb, gb = mlp.loss_and_grad(shape, theta, X, T, W=7.5 * W)
    assert abs(La - Lb) < 1e-14 * La and np.abs(ga - gb).max() < 1e-14 * np.abs(ga).max()
    # integer weights = repeated rows
    Wi = np.array([1, 2, 1, 3, 1, 1, 2, 1, 1], dtype=float)
    rep = np.repeat(np.arange(9), Wi.astype(int))
    Lr, gr = mlp.loss_and_grad(shape, theta, X[rep], T[rep])
    Lw, gw = mlp.loss_and_grad(shape, theta, X, T, W=Wi)
    assert abs(Lr - Lw) < 1e-14 and np.abs(gr - gw).max() < 1e-14
    # finite differences with weights
    h = 1e-6
    for i in range(0, len(theta), 7):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(shape, tp, X, T, W=W)[0] - mlp.loss_and_grad(shape, tm, X, T, W=W)[0]) / (2 * h)
        assert abs(fd - ga[i]) <= 1e-7 * max(1.0, np.abs(ga).max())


def test_bf16_mode_close_to_exact():
    shape, theta, X, T = _small(3, 250, 128, 125, 16)
    Y, _ = mlp.forward(shape, theta, X)
    Yb, _ = mlp.forward(shape, theta, X, bf16=True)
    assert np.linalg.norm(Yb - Y) <= 2e-2 * np.linalg.norm(Y)
    _, g = mlp.loss_and_grad(shape, theta, X, T)
    _, gb = mlp.loss_and_grad(shape, theta, X, T, bf16=True)
    assert np.linalg.norm(gb - g) <= 3e-2 * np.linalg.norm(g)
    # inputs that are already bf16 numbers with bf16 weights: the forward
    # pass of the first layer is exact up to fp64 accumulation
    tb = mlp.round_bf16(theta)
    Xb = mlp.round_bf16(X)
    _, c1 = mlp.forward(shape, tb, Xb, bf16=True)
    _, c2 = mlp.forward(shape, tb, Xb, bf16=False)
    assert np.abs(c1["Z1"] - c2["Z1"]).max() < 1e-12


def test_adam_closed_form():
    # constant gradient g: mhat = g, vhat = g^2, every step moves by lr g / (|g| + eps)
    theta = np.array([0.3, -1.0, 2.0, 0.0])
    g = np.array([1e-3, -4.0, 0.5, 0.0])
    m = np.zeros(4)
    v = np.zeros(4)
    th = theta.copy()
    for t in range(1, 6):
        th, m, v = mlp.adam_step(th, g, m, v, t, 0.01)
        expect = theta - t * 0.01 * g / (np.abs(g) + mlp.ADAM_EPS)
        assert np.abs(th - expect).max() < 1e-14


def test_training_reduces_the_loss():
    # a learnable target: T is a fixed smooth function of X
    shape = mlp.Shape(8, 16, 3)
    theta = synth.mlp_init(8, 16, 3, 4)
    X = synth.uniform_vector(512 * 8, 40).reshape(512, 8)
    T = np.stack([np.sin(X[:, 0] + X[:, 1]), X[:, 2] * X[:, 3], np.cos(X[:, 4])], axis=1)
    order = synth.sample_order(512, 20, 9)
    _, losses = mlp.train(shape, theta, X, T, order, 64, 1e-2)
    assert losses[-10:].mean() < 0.25 * losses[:5].mean()


def test_sample_order_is_a_permutation_per_epoch():
    o = synth.sample_order(100, 3, 1)
    for e in range(3):
        assert np.array_equal(np.sort(o[e * 100:(e + 1) * 100]), np.arange(100))
    assert not np.array_equal(o[:100], o[100:200])


# ---------------------------------------------------------------------------
# cells: reference diagonal, cell values, Morton order, owners, correction
# ---------------------------------------------------------------------------
def test_mean_reference_diagonal_textbook():
    # Q1: the trilinear brick of unit size has stiffness diagonal 1/3
    assert abs(mlp.mean_reference_diagonal(1) - 1.0 / 3.0) < 1e-14
    # Q2 on {0, 1/2, 1}: 1D K = [[7,-8,1],[-8,16,-8],[1,-8,7]]/3 (trace 10),
    # M = [[4,2,-1],[2,16,2],[-1,2,4]]/30 (trace 4/5); mean of the diagonal of
    # K x M x M + M x K x M + M x M x K = 3 tr(K) tr(M)^2 / 27
    assert abs(mlp.mean_reference_diagonal(2) - 3 * 10 * 0.64 / 27) < 1e-13


def _hanging_space(k):
    m = omesh.build_mesh(synth.cube_octant(2, 1))
    return Space(m, k)


@pytest.mark.parametrize("k", [2, 4])
def test_cell_values_of_a_polynomial(k):
    s = _hanging_space(k)
    assert s.n_hanging > 0
    # a polynomial of degree <= k per variable vanishing on the boundary
    extra = (lambda p: 1 + p[:, 0] - p[:, 1] * p[:, 2]) if k >= 3 else (lambda p: 1.0)
    u = lambda p: p[:, 0] * (1 - p[:, 0]) * p[:, 1] * (1 - p[:, 1]) * p[:, 2] * (1 - p[:, 2]) * extra(p)
    ue = mlp.cell_values(s, s.interpolate(u))
    xi = fe.gll_nodes(k)
    n = k + 1
    j = np.arange(n ** 3)
    for ci in range(0, s.nc, 7):
        pts = s.origin[ci] + s.h[ci] * np.stack([xi[j % n], xi[(j // n) % n], xi[j // (n * n)]], axis=1)
        assert np.abs(ue[ci] - u(pts)).max() < 1e-13


def _dfs_order(mesh):
    out = []

    def visit(c):
        if c in mesh.leaves:
            out.append(c)
            return
        l, i, j, k = c
        for ch in range(8):
            visit((l + 1, 2 * i + (ch & 1), 2 * j + ((ch >> 1) & 1), 2 * k + ((ch >> 2) & 1)))

    visit((0, 0, 0, 0))
    return out


def test_morton_key_is_depth_first_order():
    m = omesh.build_mesh(synth.cube_octant(2, 2))
    lmax = m.max_level
    by_key = sorted(m.leaves, key=lambda c: mlp.morton_key(c, lmax))
    assert by_key == _dfs_order(m)


def test_owners_uniform_mesh_brute_force():
    s = Space(omesh.build_mesh(synth.uniform_cube(2)), 2)
    oc, on = mlp.owners(s)
    lmax = int(s.level.max())
    keys = np.array([mlp.morton_key(c, lmax) for c in s.cells])
    for i in range(s.n_free):
        p = s.free_points[i]
        cand = np.nonzero(np.any(s.cell_nodes == p, axis=1))[0]
        best = cand[np.argmin(keys[cand])]
        assert oc[i] == best and s.cell_nodes[best, on[i]] == p


@pytest.mark.parametrize("k", [1, 2, 4])
def test_owners_hanging_mesh(k):
    s = _hanging_space(k)
    oc, on = mlp.owners(s)
    # the owner node is the free point itself, never a constrained point
    assert np.array_equal(s.cell_nodes[oc, on], s.free_points)
    assert not np.any(s.hanging[s.cell_nodes[oc, on]])
    # a node on a face shared with a coarser leaf is never regular: all
    # constrained points of a cell are irregular in it
    for ci in range(s.nc):
        reg = mlp.regular_nodes(s, ci)
        assert not np.any(reg & s.hanging[s.cell_nodes[ci]])
    # every cell of the finest level that touches no coarser leaf is regular
    # everywhere
    plain = [ci for ci in range(s.nc) if not s.cell_has_hanging[ci] and s.level[ci] == s.level.min()]
    for ci in plain:
        assert mlp.regular_nodes(s, ci).all()


def test_correction_constant_network_and_homogeneity():
    k = 2
    s = _hanging_space(k)
    shape = mlp.Shape(*synth.mlp_shape(k))
    own = mlp.owners(s)
    diag = s.diagonal()
    r = synth.uniform_vector(s.n_free, 8)
    # zero weights, output bias v: c_e = v s_e / (h_e a_k)
    p = mlp.unpack(shape, np.zeros(shape.n_params()))
    v = synth.uniform_vector(shape.n_out, 9)
    p["b3"] = v
    theta0 = mlp.pack(shape, p)
    c = mlp.correction(s, shape, theta0, r, diag, own=own)
    se = np.linalg.norm((s.C @ r)[s.cell_nodes], axis=1)
    a = mlp.mean_reference_diagonal(k)
    expect = v[own[1]] * se[own[0]] / (s.h[own[0]] * a)
    assert np.abs(c - expect).max() < 1e-13 * np.abs(expect).max()
    # positively 1-homogeneous in the residual, zero for a zero residual
    theta = synth.mlp_init(*synth.mlp_shape(k), 5)
    c1 = mlp.correction(s, shape, theta, r, diag, own=own)
    c2 = mlp.correction(s, shape, theta, 3.5 * r, diag, own=own)
    assert np.abs(c2 - 3.5 * c1).max() < 1e-12 * np.abs(c2).max()
    assert np.all(mlp.correction(s, shape, theta, 0 * r, diag, own=own) == 0)


def test_features_and_targets():
    k = 2
    s = _hanging_space(k)
    r = synth.uniform_vector(s.n_free, 1)
    e = synth.uniform_vector(s.n_free, 2)
    diag = s.diagonal()
    X, se = mlp.cell_features(s, r, diag)
    n3 = (k + 1) ** 3
    assert X.shape == (s.nc, 2 * n3)
    nz = se > 0
    assert np.allclose(np.linalg.norm(X[nz, :n3], axis=1), 1.0, atol=1e-14)
    T = mlp.cell_targets(s, r, e)
    a = mlp.mean_reference_diagonal(k)
    # the target maps back to the error through the correction scaling
    ee = (s.C @ e)[s.cell_nodes]
    assert np.allclose(T[nz] * (se[nz] / (s.h[nz] * a))[:, None], ee[nz], rtol=0, atol=1e-13)
    # weighted target error = error of the correction itself
    W = mlp.cell_weights(s, r)
    Y = synth.uniform_vector(T.size, 3).reshape(T.shape)
    C = Y * (se / (s.h * a))[:, None]
    assert np.allclose(W[nz] * np.sum((Y[nz] - T[nz]) ** 2, axis=1), np.sum((C[nz] - ee[nz]) ** 2, axis=1),
                       rtol=1e-12, atol=0)


# ---------------------------------------------------------------------------
# flexible CG and the learned-step hook
# ---------------------------------------------------------------------------
def test_flexible_cg_equals_cg_for_a_linear_preconditioner():
    n = 60
    A = sp.diags([np.full(n - 1, -1.0), np.full(n, 2.2), np.full(n - 1, -1.0)], [-1, 0, 1]).tocsr()
    b = synth.uniform_vector(n, 3)
    D = 1.0 / A.diagonal()
    r1 = mg.pcg(lambda v: A @ v, b, lambda v: D * v, 1e-10)
    r2 = mg.pcg(lambda v: A @ v, b, lambda v: D * v, 1e-10, flexible=True)
    assert r1.iterations == r2.iterations
    assert np.abs(r1.x - r2.x).max() < 1e-9 * np.abs(r1.x).max()


def test_learned_hook_zero_map_is_the_plain_vcycle():
    m = omesh.build_mesh(synth.octant(2))
    levels = mg.build_levels(m, 2)
    b = levels[-1].space.rhs()
    x0 = mg.multigrid_vcycle(levels, b)
    levels[-1].learned = lambda r: np.zeros_like(r)
    levels[-1].learned_mode = "augment"
    assert np.array_equal(mg.multigrid_vcycle(levels, b), x0)
    # "replace" skips the postsmoothing: the result is the V-cycle before it
    levels[-1].learned_mode = "replace"
    xr = mg.multigrid_vcycle(levels, b)
    top = levels[-1]
    post = mg.chebyshev(top.apply, 1.0 / top.diag, b, xr, top.lam_max)
    assert np.abs(post - x0).max() < 1e-14 * np.abs(x0).max()


def test_learned_step_is_the_energy_minimising_step_length():
    """Galerkin step length: along the learned direction c the A-norm of the
    error is smallest at omega = (r.c)/(c.A c) (pinned against a scan of
    omega), and never larger than before the step, for an arbitrary map."""
    m = omesh.build_mesh(synth.octant(2))
    levels = mg.build_levels(m, 2)
    top = levels[-1]
    A = top.space.assemble()
    b = top.space.rhs()
    xs = sla.spsolve(A.tocsc(), b)
    rng = np.random.default_rng(4)
    M = rng.standard_normal((len(b), len(b)))
    top.learned = lambda r: M @ r  # any map, e.g. an untrained network
    x = synth.uniform_vector(len(b), 8)
    xn = mg.learned_step(top, b, x)
    energy = lambda y: float((xs - y) @ (A @ (xs - y)))
    assert energy(xn) <= energy(x) * (1 + 1e-14)
    c = M @ (b - A @ x)
    for om in np.linspace(-2, 2, 41):
        assert energy(xn) <= energy(x + om * c) * (1 + 1e-12) + 1e-14
