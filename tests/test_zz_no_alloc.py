"""mesh_codec_adjacency_static: the adjacency build for callers that cannot
allocate device memory where they need it (real-time hosts that allocate
everything up front, plug-ins whose device memory belongs to another
framework's allocator).  Its result must equal the adjacency that
mesh_codec_create builds, on consecutive calls that share the library's
static scratch array, at sizes up to its stated limits, and a call must not
change the device's free memory.

This file is named so that pytest collects it last."""

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

MAX_V = 1 << 17
MAX_T = 1 << 18


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_10105_gb300 import build, codec
    build.build()
    return codec.load_library()


def _static_adjacency(lib, tris, n, capacity=None):
    t = torch.from_numpy(np.ascontiguousarray(tris, dtype=np.int32)).cuda()
    T = t.shape[0]
    cap = 6 * T if capacity is None else capacity
    row_ptr = torch.full((n + 1,), -7, dtype=torch.int32, device="cuda")
    col_idx = torch.full((max(cap, 1),), -7, dtype=torch.int32, device="cuda")
    deg = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    nnz = ctypes.c_int32(-1)
    stream = torch.cuda.current_stream()
    st = lib.mesh_codec_adjacency_static(
        ctypes.c_void_p(t.data_ptr()), T, n, ctypes.c_void_p(row_ptr.data_ptr()),
        ctypes.c_void_p(col_idx.data_ptr()), cap, ctypes.c_void_p(deg.data_ptr()),
        ctypes.byref(nnz), ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return st, nnz.value, row_ptr.cpu().numpy(), col_idx.cpu().numpy()[: max(nnz.value, 0)], \
        deg.cpu().numpy()


def _create_adjacency(tris, n):
    from paper_2111_10105_gb300 import MeshCodec, codec as cb
    with MeshCodec(tris, n, n_frames=2, rank=1, n_anchors=1) as mc:
        return (mc.buffer(cb.BUF_ROW_PTR).cpu().numpy(), mc.buffer(cb.BUF_COL_IDX).cpu().numpy(),
                mc.buffer(cb.BUF_DEGREE).cpu().numpy())


def test_two_calls_in_a_row_match_create(lib):
    from synth import torus_grid, icosphere
    meshes = [torus_grid(120, 70), icosphere(4), torus_grid(120, 70)]
    for v, t in meshes:      # consecutive calls reuse the same scratch array
        n = v.shape[0]
        st, nnz, rp, ci, dg = _static_adjacency(lib, t, n)
        assert st == 0
        rp0, ci0, dg0 = _create_adjacency(t, n)
        assert nnz == rp0[-1]
        np.testing.assert_array_equal(rp, rp0)
        np.testing.assert_array_equal(ci, ci0)
        np.testing.assert_array_equal(dg, dg0)


def test_limits_and_errors(lib):
    from synth import icosphere
    v, t = icosphere(2)
    n = v.shape[0]
    # sizes beyond the stated maximum are rejected before any work
    big = np.zeros((1, 3), dtype=np.int32)
    st, *_ = _static_adjacency(lib, big, MAX_V + 1)
    assert st == 1
    st, *_ = _static_adjacency(lib, np.zeros((MAX_T + 1, 3), dtype=np.int32), 3)
    assert st == 1
    # too small an output buffer: nnz is still reported
    st, nnz, *_ = _static_adjacency(lib, t, n, capacity=10)
    assert st == 8 and nnz == 2 * (3 * t.shape[0] // 2)
    # a bad triangle, then a good call: the error word is cleared between calls
    bad = t.copy()
    bad[5, 1] = n + 3
    st, *_ = _static_adjacency(lib, bad, n)
    assert st == 2
    st, nnz, rp, ci, dg = _static_adjacency(lib, t, n)
    assert st == 0 and nnz == rp[-1]


def test_at_the_limits_and_no_device_memory_taken(lib):
    # a 512 x 256 torus has exactly MAX_V vertices and MAX_T triangles, where
    # the scratch carve is fullest
    from synth import torus_grid
    v, t = torus_grid(512, 256)
    n = v.shape[0]
    assert n == MAX_V and t.shape[0] == MAX_T
    st, nnz, rp, ci, dg = _static_adjacency(lib, t, n)     # first call: address lookup
    assert st == 0 and nnz == 6 * n
    rp0, ci0, dg0 = _create_adjacency(t, n)
    np.testing.assert_array_equal(rp, rp0)
    np.testing.assert_array_equal(ci, ci0)
    np.testing.assert_array_equal(dg, dg0)
    # inputs and outputs are allocated first; the call itself must leave the
    # device's free memory and torch's allocator untouched
    tt = torch.from_numpy(np.ascontiguousarray(t, dtype=np.int32)).cuda()
    row_ptr = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    col_idx = torch.empty(6 * MAX_T, dtype=torch.int32, device="cuda")
    deg = torch.empty(n, dtype=torch.int32, device="cuda")
    nnz_c = ctypes.c_int32(-1)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(2):
        st = lib.mesh_codec_adjacency_static(
            ctypes.c_void_p(tt.data_ptr()), MAX_T, n, ctypes.c_void_p(row_ptr.data_ptr()),
            ctypes.c_void_p(col_idx.data_ptr()), 6 * MAX_T, ctypes.c_void_p(deg.data_ptr()),
            ctypes.byref(nnz_c), ctypes.c_void_p(stream.cuda_stream))
        assert st == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    np.testing.assert_array_equal(row_ptr.cpu().numpy(), rp0)
    np.testing.assert_array_equal(col_idx.cpu().numpy()[:nnz_c.value], ci0)
