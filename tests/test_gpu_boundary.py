"""Boundary behaviour of the C ABI on the GPU: meshes with several connected
components (Eq. 12 needs an anchor in each), the bounded waits of the
tensor-core kernels, and the vertex-major position layout."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

NO_ANCHOR = 11
TIMEOUT = 12


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_10105_gb300 import build, codec
    build.build()
    return codec.load_library()


def _two_spheres(F=12):
    from synth import disjoint_union, icosphere
    a, b = icosphere(2), icosphere(2)
    v, t = disjoint_union([a, b], offsets=[(0, 0, 0), (3, 0, 0)])
    n1 = a[0].shape[0]
    rng = np.random.default_rng(5)
    # smooth, full-rank motion: every vertex moves along its own trajectory
    f = np.arange(F)[:, None, None] / F
    w = rng.uniform(0.5, 2.0, size=(1, v.shape[0], 3))
    ph = rng.uniform(0, 2 * np.pi, size=(1, v.shape[0], 3))
    pos = v[None] + 0.05 * np.sin(2 * np.pi * w * f + ph) + 0.2 * f
    return t, np.ascontiguousarray(pos), n1


def test_anchor_free_component_rejected_at_create(lib):
    from paper_2111_10105_gb300 import MeshCodec
    from paper_2111_10105_gb300.codec import MeshCodecError
    t, pos, n1 = _two_spheres()
    n = pos.shape[1]
    kw = dict(n_frames=pos.shape[0], rank=4, n_anchors=3)
    with pytest.raises(MeshCodecError) as e:
        MeshCodec(t, n, anchors=np.array([1, 7, 40], dtype=np.int32), **kw)
    assert e.value.status == NO_ANCHOR
    # one anchor in each sphere: accepted
    MeshCodec(t, n, anchors=np.array([1, 7, n1 + 3], dtype=np.int32), **kw).close()
    # an encode-only handle (no anchors) is accepted; its decode is refused
    with MeshCodec(t, n, n_frames=pos.shape[0], rank=4, n_anchors=0) as mc:
        bits = mc.encode(torch.from_numpy(pos).cuda())
        with pytest.raises(MeshCodecError) as e:
            mc.decode(bits)
        assert e.value.status == 1


def test_stream_anchors_checked_per_component_at_decode(lib):
    from oracle import codec as ocodec, metrics
    from oracle.graph import AnchorCoverageError
    from paper_2111_10105_gb300 import MeshCodec
    from paper_2111_10105_gb300.codec import MeshCodecError
    t, pos, n1 = _two_spheres()
    n, F = pos.shape[1], pos.shape[0]
    anchors = np.array([1, 7, n1 + 3], dtype=np.int32)
    kw = dict(n_frames=F, rank=4, n_anchors=3, oi_sweeps=20)
    with MeshCodec(t, n, anchors=anchors, **kw) as mc:
        bits = mc.encode(torch.from_numpy(pos).cuda())
        rec = mc.decode(bits).cpu().numpy()
        # the same mesh and anchors in the oracle: both components anchored
        p = ocodec.Params(n_frames=F, rank=4, n_anchors=3, oi_sweeps=20)
        blob = ocodec.encode(t, pos, p, anchors=anchors)
        rec_o = ocodec.decode(blob, t)
        e_gpu, e_ora = metrics.nmse(pos, rec), metrics.nmse(pos, rec_o)
        assert abs(e_gpu - e_ora) <= 1e-9 * e_ora
        # the stream's anchor list rewritten to lie in the first sphere only
        # (still ascending and in range): the decoder refuses it before solving
        bad = bits.clone()
        moved = torch.tensor([1, 7, 40], dtype=torch.int32).view(torch.uint8).cuda()
        bad[64:64 + 12] = moved
        with pytest.raises(MeshCodecError) as e:
            mc.decode(bad)
        assert e.value.status == NO_ANCHOR
        blob_bad = bytearray(blob)
        blob_bad[64:76] = np.array([1, 7, 40], dtype="<i4").tobytes()
        with pytest.raises(AnchorCoverageError):
            ocodec.decode(bytes(blob_bad), t)
        # the handle still decodes a good stream afterwards
        rec2 = mc.decode(bits).cpu().numpy()
        np.testing.assert_array_equal(rec2, rec)


def test_component_labels_on_many_pieces(lib):
    # 40 small pieces in shuffled vertex order: every anchor set that misses
    # one piece is refused, one anchor per piece is accepted
    from oracle import graph
    from paper_2111_10105_gb300 import MeshCodec
    from paper_2111_10105_gb300.codec import MeshCodecError
    from synth import disjoint_union, icosphere, torus_grid
    pieces = [icosphere(1) if i % 2 else torus_grid(4 + i % 5, 3) for i in range(40)]
    v, t = disjoint_union(pieces)
    n = v.shape[0]
    perm = np.random.default_rng(11).permutation(n).astype(np.int32)
    t = perm[t]
    rp, ci, _ = graph.build_adjacency(t, n)
    lab = graph.components(rp, ci)
    roots = np.unique(lab)
    assert roots.size == 40
    one_each = np.sort(np.array([np.nonzero(lab == r)[0][-1] for r in roots], dtype=np.int32))
    kw = dict(n_frames=4, rank=2, n_anchors=40)
    MeshCodec(t, n, anchors=one_each, **kw).close()
    for drop in (0, 17, 39):
        keep = np.delete(one_each, drop)
        other = np.setdiff1d(np.nonzero(lab == lab[keep[0]])[0], keep)[0]
        anc = np.sort(np.append(keep, other)).astype(np.int32)
        with pytest.raises(MeshCodecError) as e:
            MeshCodec(t, n, anchors=anc, **kw)
        assert e.value.status == NO_ANCHOR


def test_tensor_core_wait_limit_runs_out_then_recovers(lib):
    # a wait limit of 2 us on a long product: a wait runs out, the kernel
    # drains its copies and products, frees its tensor memory and the call
    # reports MC_E_TIMEOUT; with the default limit the next call succeeds
    from paper_2111_10105_gb300.codec import MeshCodecError, selftest_gemm, set_wait_limit
    g = torch.Generator(device="cuda").manual_seed(3)
    M, N, K = 128, 64, 1 << 17
    A = torch.rand((M, K), device="cuda", generator=g) - 0.5
    B = torch.rand((N, K), device="cuda", generator=g) - 0.5
    try:
        set_wait_limit(2000)
        with pytest.raises(MeshCodecError) as e:
            selftest_gemm(0, A, B, splits=1)
        assert e.value.status == TIMEOUT
    finally:
        set_wait_limit(0)
    torch.cuda.synchronize()
    Ks = 4096
    C = selftest_gemm(0, A[:, :Ks].contiguous(), B[:, :Ks].contiguous(), splits=2)
    ref = A[:, :Ks].double() @ B[:, :Ks].double().T
    scale = (A[:, :Ks].double().abs() @ B[:, :Ks].double().abs().T).max()
    assert float((C - ref).abs().max() / scale) < 2e-3


@pytest.mark.parametrize("precision", [0, 1])
def test_vertex_major_layout_equals_frames_layout(lib, precision):
    from paper_2111_10105_gb300 import MeshCodec
    from synth import SequenceSpec, make_sequence
    spec = SequenceSpec(name="lay", mesh="icosphere:3", n_frames=40, rank=8, n_anchors=12,
                        seed=21)
    t, pos = make_sequence(spec)
    n, F = pos.shape[1], pos.shape[0]
    kw = dict(n_frames=F, rank=8, n_anchors=12, seed=21, oi_sweeps=20, precision=precision,
              oi_refine_sweeps=1 if precision else 0, cg_rtol=1e-6 if precision else 1e-14)
    pos_d = torch.from_numpy(pos).cuda()
    vm = pos_d.permute(1, 2, 0).contiguous()          # [n][3][F]
    with MeshCodec(t, n, **kw) as a, MeshCodec(t, n, layout=1, **kw) as b:
        bits_a = a.encode(pos_d)
        bits_b = b.encode(vm)
        assert torch.equal(bits_a, bits_b)
        rec_a = a.decode(bits_a)
        rec_b = b.decode(bits_b)
        assert tuple(rec_b.shape) == (n, 3, F)
        assert torch.equal(rec_b, rec_a.permute(1, 2, 0))
        # host-buffer entry points take the same layout
        rec_h = b.decode_host(b.encode_host(vm.cpu().numpy()))
        np.testing.assert_array_equal(rec_h, rec_b.cpu().numpy())
