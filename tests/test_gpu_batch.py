"""Batched solve (one graph launch for many independent problems; or the
whole batch in one persistent kernel) and the operator autotuner, through
the C ABI.

The batched CG runs the same kernels in the same order as the single-problem
solve, so every problem's iterate must equal its own single solve bit for
bit; a few problems are also checked against the oracle (relative residual
of the returned x with the oracle's operator and right-hand side <= 1e-8).
The persistent kernel runs the line-parallel operators on every level and
sums the CG reductions with 256 threads, so its iterates agree with the
graph's to rounding: the same convergence (iterations within one, relative
residual <= 1e-8, also by the oracle), and bit-identical repeats.
"""
import numpy as np
import pytest

import synth
from oracle import mesh as omesh
from oracle.space import Space
from parity import match

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# (degree, global depth, extra octant levels): uneven sizes and degrees
PROBLEMS = [(1, 2, 0), (2, 3, 1), (3, 2, 2), (4, 2, 1), (1, 4, 2), (2, 2, 0), (4, 3, 0), (3, 3, 1)]


def _rhs(mg, seed):
    f = synth.fourier_rhs(seed)
    return mg.rhs((f.kappa, f.phi, f.amp))


@pytest.fixture(scope="module")
def batch(gcmg):
    meshes = [gcmg.Mesh.from_recipe(synth.cube_octant(d, e)) for _, d, e in PROBLEMS]
    cfgs = [gcmg.make_config(k, mg_fp32=True) for k, _, _ in PROBLEMS]
    return gcmg.Batch(meshes, cfgs, n_threads=4)


def test_batch_matches_single_solves(gcmg, batch):
    bs = [_rhs(m, 100 + i) for i, m in enumerate(batch.problems)]
    xs = [torch.zeros_like(b) for b in bs]
    stats = batch.cg_solve(bs, xs, 1e-8)
    for i, (k, d, e) in enumerate(PROBLEMS):
        single = gcmg.Multigrid(gcmg.Mesh.from_recipe(synth.cube_octant(d, e)), k, mg_fp32=True)
        b = _rhs(single, 100 + i)
        assert torch.equal(b, bs[i])
        x = torch.zeros_like(b)
        st = single.cg_solve(b, x, 1e-8)
        assert stats[i].status == 0
        assert stats[i].iterations == st.iterations, (i, stats[i].iterations, st.iterations)
        assert torch.equal(x, xs[i]), i
        assert stats[i].rel_residual <= 1e-8
    # a second launch replays the same graph
    xs2 = [torch.zeros_like(b) for b in bs]
    stats2 = batch.cg_solve(bs, xs2, 1e-8)
    assert [s.iterations for s in stats2] == [s.iterations for s in stats]
    assert all(torch.equal(a, c) for a, c in zip(xs, xs2))


@pytest.mark.parametrize("i", [0, 3, 5])
def test_batch_residual_by_oracle(batch, i):
    k, d, e = PROBLEMS[i]
    mg = batch.problems[i]
    b = _rhs(mg, 200 + i)
    bs = [torch.zeros_like(_rhs(m, 1)) for m in batch.problems]
    bs[i] = b
    xs = [torch.zeros_like(v) for v in bs]
    stats = batch.cg_solve(bs, xs, 1e-8)
    # zero right-hand sides: no iteration, x = 0
    for j, s in enumerate(stats):
        if j != i:
            assert s.iterations == 0 and s.status == 0 and not torch.any(xs[j])
    s = Space(omesh.build_mesh(synth.cube_octant(d, e)), k)
    perm = match(mg.dof_coords(mg.finest), s.free_coordinates())
    f = synth.fourier_rhs(200 + i)
    from oracle.space import fourier_function
    bo = s.rhs(fourier_function(f))
    xo = np.empty(len(perm))
    xo[perm] = xs[i].cpu().numpy()
    assert np.linalg.norm(bo - s.apply(xo)) <= 1.01e-8 * np.linalg.norm(bo)


def test_batch_maxit(batch):
    bs = [_rhs(m, 300 + i) for i, m in enumerate(batch.problems)]
    xs = [torch.zeros_like(b) for b in bs]
    stats = batch.cg_solve(bs, xs, 1e-14, maxit=2)
    for s in stats:
        assert s.iterations == 2 and s.status == 4  # GCMG_ERR_NOT_CONVERGED


def test_persistent_batch(gcmg, batch):
    bs = [_rhs(m, 100 + i) for i, m in enumerate(batch.problems)]
    xg = [torch.zeros_like(b) for b in bs]
    sg = batch.cg_solve(bs, xg, 1e-8)
    xp = [torch.zeros_like(b) for b in bs]
    sp = batch.cg_solve(bs, xp, 1e-8, persistent=True)
    for i in range(len(bs)):
        assert sp[i].status == 0 and sp[i].rel_residual <= 1e-8, i
        assert abs(sp[i].iterations - sg[i].iterations) <= 1, (i, sp[i].iterations, sg[i].iterations)
        assert float((xp[i] - xg[i]).norm() / xg[i].norm()) < 1e-5, i
    info = batch.persistent_info()
    assert info.grid >= 1 and info.in_graph == 1 and info.ops > 0
    assert info.steps >= max(s.iterations for s in sp)
    # a second launch of the captured persistent kernel repeats the solve bit for bit
    xp2 = [torch.zeros_like(b) for b in bs]
    sp2 = batch.cg_solve(bs, xp2, 1e-8, persistent=True)
    assert [s.iterations for s in sp2] == [s.iterations for s in sp]
    assert all(torch.equal(a, c) for a, c in zip(xp, xp2))


@pytest.mark.parametrize("i", [0, 3])
def test_persistent_residual_by_oracle(batch, i):
    k, d, e = PROBLEMS[i]
    mg = batch.problems[i]
    bs = [torch.zeros_like(_rhs(m, 1)) for m in batch.problems]
    bs[i] = _rhs(mg, 200 + i)
    xs = [torch.zeros_like(v) for v in bs]
    stats = batch.cg_solve(bs, xs, 1e-8, persistent=True)
    for j, s in enumerate(stats):
        if j != i:
            assert s.iterations == 0 and s.status == 0 and not torch.any(xs[j])
    s = Space(omesh.build_mesh(synth.cube_octant(d, e)), k)
    perm = match(mg.dof_coords(mg.finest), s.free_coordinates())
    from oracle.space import fourier_function
    bo = s.rhs(fourier_function(synth.fourier_rhs(200 + i)))
    xo = np.empty(len(perm))
    xo[perm] = xs[i].cpu().numpy()
    assert np.linalg.norm(bo - s.apply(xo)) <= 1.01e-8 * np.linalg.norm(bo)


def test_persistent_maxit(batch):
    bs = [_rhs(m, 300 + i) for i, m in enumerate(batch.problems)]
    xs = [torch.zeros_like(b) for b in bs]
    stats = batch.cg_solve(bs, xs, 1e-14, maxit=2, persistent=True)
    for s in stats:
        assert s.iterations == 2 and s.status == 4  # GCMG_ERR_NOT_CONVERGED


def test_persistent_barrier_wait_gives_up(gcmg, batch):
    """one CTA leaves before the first grid barrier: the others' bounded waits
    run out, the kernel records it and returns, the call fails with an error,
    and the next normal persistent solve still converges (no GPU fault, no hang)"""
    bs = [_rhs(m, 400 + i) for i, m in enumerate(batch.problems)]
    xs = [torch.zeros_like(b) for b in bs]
    batch.persistent_wait_test(absent_cta=0, spin_limit=1 << 14)
    with pytest.raises(gcmg.GcmgError, match="grid-barrier wait gave up"):
        batch.cg_solve(bs, xs, 1e-8, persistent=True)
    batch.persistent_wait_test()
    xs = [torch.zeros_like(b) for b in bs]
    stats = batch.cg_solve(bs, xs, 1e-8, persistent=True)
    assert all(s.status == 0 and s.rel_residual <= 1e-8 for s in stats)


def test_autotune(gcmg):
    probe = gcmg.Mesh.from_recipe(synth.cube_octant(3, 1))
    best, cands = gcmg.autotune(probe, 2, mg_fp32=True, reps=5)
    assert len(cands) == 13  # lane, line and slab mappings over tile sizes 8..128
    assert all(c.gdofs > 0 for c in cands)
    assert best.gdofs == max(c.gdofs for c in cands)
    assert (best.tile_cells, best.cell_kernel) in [(c.tile_cells, c.cell_kernel) for c in cands]
    # the tuned configuration computes the same operator
    a = gcmg.Multigrid(probe, 2, tile_cells=best.tile_cells, cell_kernel=best.cell_kernel,
                       cell_threads=best.cell_threads)
    b = gcmg.Multigrid(probe, 2)
    x = torch.tensor(synth.point_values(a.dof_coords(a.finest), 5), dtype=torch.float32, device="cuda")
    xb = torch.tensor(synth.point_values(b.dof_coords(b.finest), 5), dtype=torch.float32, device="cuda")
    ya, yb = torch.empty_like(x), torch.empty_like(xb)
    a.vmult(a.finest, x, ya)
    b.vmult(b.finest, xb, yb)
    perm = match(a.dof_coords(a.finest), b.dof_coords(b.finest))
    assert torch.allclose(ya, yb[torch.tensor(perm, device="cuda")], rtol=0, atol=2e-5 * float(yb.abs().max()))
