"""Host-side checks of the C ABI: the library builds for sm_103a, loads
without a GPU, exports every entry point the header declares, and its
structs have the layout the binding assumes."""

import ctypes
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mesh_codec.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2111_10105_gb300 import build, codec
    build.build()
    return codec.load_library()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"MESH_CODEC_API[^;(]*?\b(mesh_codec_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (mesh_codec_\w+)", out))
    assert set(names) == exported


def test_struct_layout_matches_c(lib):
    from paper_2111_10105_gb300.codec import Params, Stats
    src = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "mesh_codec.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(mesh_codec_params_t),
             offsetof(mesh_codec_params_t, oi_tol), offsetof(mesh_codec_params_t, seed),
             offsetof(mesh_codec_params_t, solve_mode), sizeof(mesh_codec_stats_t),
             offsetof(mesh_codec_stats_t, oi_change), offsetof(mesh_codec_stats_t, workspace_bytes));
      return 0;
    }
    """
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), c, "-o", exe], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert vals == [ctypes.sizeof(Params), Params.oi_tol.offset, Params.seed.offset,
                    Params.solve_mode.offset, ctypes.sizeof(Stats), Stats.oi_change.offset,
                    Stats.workspace_bytes.offset]


def test_defaults_and_status_strings_without_gpu(lib):
    from paper_2111_10105_gb300.codec import default_params
    p = default_params()
    assert (p.coeff_bits, p.dict_bits, p.anchor_bits) == (12, 16, 16)
    assert p.cg_rtol == 1e-14 and p.oi_sweeps == 30
    for s in range(11):
        assert lib.mesh_codec_status_string(s)
    assert lib.mesh_codec_status_string(999) == b"unknown status"


def test_invalid_params_rejected_before_any_device_work(lib):
    from paper_2111_10105_gb300.codec import default_params
    p = default_params()
    p.n_vertices, p.n_triangles, p.n_frames, p.rank = 10, 5, 8, 9   # rank > F
    h = ctypes.c_void_p()
    tris = (ctypes.c_int32 * 15)()
    st = lib.mesh_codec_create(ctypes.byref(p), ctypes.cast(tris, ctypes.c_void_p), 0, None, 0,
                               None, ctypes.byref(h))
    assert st == 1 and not h.value
    p.rank = 4
    p.coeff_bits = 40
    assert lib.mesh_codec_create(ctypes.byref(p), ctypes.cast(tris, ctypes.c_void_p), 0, None, 0,
                                 None, ctypes.byref(h)) == 1
    p.coeff_bits = 12
    for field, bad in (("block_delta", 2), ("block_delta_bits", 32), ("block_delta_bits", -1)):
        setattr(p, field, bad)
        assert lib.mesh_codec_create(ctypes.byref(p), ctypes.cast(tris, ctypes.c_void_p), 0, None,
                                     0, None, ctypes.byref(h)) == 1
        setattr(p, field, 0)
    # block CG only as the refined solve's inner solver, and only 0 / 1
    for refine, block in ((0, 1), (2, 2), (2, -1)):
        p.refine, p.block_cg = refine, block
        assert lib.mesh_codec_create(ctypes.byref(p), ctypes.cast(tris, ctypes.c_void_p), 0, None,
                                     0, None, ctypes.byref(h)) == 1
    p.refine, p.block_cg = 0, 0
    assert lib.mesh_codec_create(None, None, 0, None, 0, None, ctypes.byref(h)) == 1
    lib.mesh_codec_destroy(None)


def test_stream_size_formula_matches_oracle(lib):
    # the size arithmetic of the bitstream must agree between the two sides;
    # the library reports it only from a handle, so compare through the
    # oracle's formula on the documented layout
    from oracle import codec as oc
    assert oc.stream_size(2562, 64, 16, 20, 12, 16, 16) == 64 + 80 + 3 * (
        8 * 66 + ((64 * 16 + 31) // 32) * 16 * 4 + ((16 * 2562 + 31) // 32) * 12 * 4 +
        ((20 * 64 + 31) // 32) * 16 * 4)


@pytest.mark.parametrize("n_blocks,delta", [(1, 0), (4, 0), (4, 1)])
def test_rates_match_the_oracle(lib, n_blocks, delta):
    # host-only entry point: Eq. 13's terms for what the stream holds, and the
    # stream's own rate from its size, against the oracle's formulas
    from oracle import blocks as ob, codec as oc, metrics
    from paper_2111_10105_gb300.codec import Params, default_params
    lib.mesh_codec_rates.restype = ctypes.c_int
    lib.mesh_codec_rates.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ctypes.c_void_p]
    p = default_params()
    p.n_vertices, p.n_triangles, p.n_frames, p.rank, p.n_anchors = 10002, 20000, 175, 20, 100
    p.block_delta, p.block_delta_bits = delta, 10 if delta else 0
    out = (ctypes.c_double * 5)()
    assert lib.mesh_codec_rates(ctypes.byref(p), n_blocks, out) == 0
    r = metrics.rates(10002, 175, 20, 100, 12, 16, 16, n_b=1, dict_cols=20)
    assert out[0] == pytest.approx(r["q"], rel=1e-15)
    assert out[1] == pytest.approx(r["q_a"], rel=1e-15)
    # Table I's anchor rate: 16 bits, 1% anchors, n = 10002 (Handstand)
    assert round(out[1], 4) == 0.1600
    dict_bits = [16] + [10 if delta else 16] * (n_blocks - 1)
    assert out[2] == pytest.approx(sum(dict_bits) * 20 / (10002 * n_blocks), rel=1e-15)
    assert out[3] == pytest.approx(out[0] + out[1] + out[2], rel=1e-15)
    op = oc.Params(n_frames=175, rank=20, n_anchors=100)
    if n_blocks == 1:
        nbytes = oc.stream_size(10002, 175, 20, 100, 12, 16, 16)
    else:
        nbytes = ob.container_size(10002, op, n_blocks, bool(delta), 10)[0]
    assert out[4] == pytest.approx(nbytes * 8 / (10002 * 175 * n_blocks), rel=1e-15)
    p.rank = 0
    assert lib.mesh_codec_rates(ctypes.byref(p), 1, out) == 1
