"""gcmg_dot_noalloc: the inner product for callers that cannot allocate
device memory (code running under stream capture, plugins in applications
that own all GPU memory, real-time loops).  It must agree with gcmg_dot,
whose partial sums live in a buffer the handle allocated, and it must not
allocate.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MAX_N = 65536 * 8192


def _dot_noalloc(lib, x, y, n, out, stream=None):
    return lib.gcmg_dot_noalloc(ctypes.c_void_p(x.data_ptr() if n else None),
                                ctypes.c_void_p(y.data_ptr() if n else None), n,
                                ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


@pytest.mark.parametrize("n", [1, 8191, 8192, 8193, 1_000_003, 4 * 8192 * 100 + 5])
def test_matches_allocating_entry_point_twice(gcmg, n):
    lib = gcmg.lib()
    handle_owner = gcmg.Multigrid(gcmg.Mesh(0.0, 1.0, [(0,)]), 2)
    xs, ys = synth.uniform_vector(n, 21), synth.uniform_vector(n, 22)
    x = torch.tensor(xs, dtype=torch.float64, device="cuda")
    y = torch.tensor(ys, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    scale = float(np.sum(np.abs(xs * ys)))
    for _ in range(2):  # two calls in a row: the shared array keeps old partials
        ref = handle_owner.dot(x, y).item()
        out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        assert _dot_noalloc(lib, x, y, n, out, stream) == 0, lib.gcmg_last_error()
        got = out.item()
        assert abs(got - ref) <= 1e-13 * scale
        assert abs(got - float(np.dot(xs, ys))) <= 1e-13 * scale


def test_second_call_allocates_nothing(gcmg):
    lib = gcmg.lib()
    n = 3_000_000
    x = torch.tensor(synth.uniform_vector(n, 5), dtype=torch.float64, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    assert _dot_noalloc(lib, x, x, n, out, stream) == 0  # first call: per-device set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    torch0 = torch.cuda.memory_allocated()
    for _ in range(3):
        assert _dot_noalloc(lib, x, x, n, out, stream) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == torch0
    assert abs(out.item() - float(torch.dot(x, x).item())) <= 1e-13 * out.item()


def test_rejects_sizes_beyond_the_array(gcmg):
    lib = gcmg.lib()
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # the size check happens on the host before any device work
    rc = lib.gcmg_dot_noalloc(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(x.data_ptr()), MAX_N + 1,
                              ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 1
    assert b"exceeds the maximum" in lib.gcmg_last_error()


def test_empty_input_gives_zero(gcmg):
    lib = gcmg.lib()
    out = torch.full((1,), 7.0, dtype=torch.float64, device="cuda")
    assert lib.gcmg_dot_noalloc(None, None, 0, ctypes.c_void_p(out.data_ptr()), None) == 0
    torch.cuda.synchronize()
    assert out.item() == 0.0
