"""Farthest-point anchor selection on the GPU (mesh_codec_farthest_anchors)
against the oracle, index for index, and the codec with such anchors
against the oracle's codec with the same anchors."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import anchors as oa, codec as oc, metrics  # noqa: E402
from synth import SequenceSpec, make_sequence  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_10105_gb300 import build
    build.build()


def _fps(xyz, n_c, start=0):
    from paper_2111_10105_gb300.codec import farthest_anchors
    return farthest_anchors(torch.from_numpy(np.ascontiguousarray(xyz)).cuda(), n_c,
                            start).cpu().numpy()


@pytest.mark.parametrize("n_c,start", [(1, 7), (2, 0), (50, 0), (200, 12345)])
def test_torus_pose_matches_the_oracle(n_c, start):
    spec = SequenceSpec(name="t", mesh="torus:200:100", n_frames=2, rank=1, n_anchors=1, seed=9,
                        bend=0.1)
    _, pos = make_sequence(spec)
    xyz = pos[1]
    np.testing.assert_array_equal(_fps(xyz, n_c, start), oa.farthest_point(xyz, n_c, start))


def test_flat_grid_with_equal_distances_matches_the_oracle():
    i, j = np.meshgrid(np.arange(40.0), np.arange(40.0), indexing="ij")
    xyz = np.stack([i.ravel(), j.ravel(), np.zeros(1600)], axis=1)   # integer lattice: exact ties
    for n_c in (3, 4, 37, 400):
        np.testing.assert_array_equal(_fps(xyz, n_c, 0), oa.farthest_point(xyz, n_c, 0))


def test_every_vertex_and_ragged_sizes():
    rng = np.random.default_rng(3)
    for n in (1, 5, 257, 1025):
        xyz = rng.standard_normal((n, 3))
        np.testing.assert_array_equal(_fps(xyz, n, n // 2), np.arange(n, dtype=np.int32))
        k = max(1, n // 3)
        np.testing.assert_array_equal(_fps(xyz, k, n - 1), oa.farthest_point(xyz, k, n - 1))


def test_bad_arguments_are_rejected():
    from paper_2111_10105_gb300 import MeshCodecError
    xyz = np.zeros((4, 3))
    for n_c, start in ((0, 0), (5, 0), (2, 4), (2, -1)):
        with pytest.raises(MeshCodecError):
            _fps(xyz, n_c, start)


def test_codec_with_farthest_anchors_matches_the_oracle():
    from paper_2111_10105_gb300 import MeshCodec
    spec = SequenceSpec(name="a", mesh="icosphere:3", n_frames=24, rank=6, n_anchors=12, seed=8)
    tris, pos = make_sequence(spec)
    n = pos.shape[1]
    anchors = oa.farthest_point(pos[0], 12)
    np.testing.assert_array_equal(_fps(pos[0], 12), anchors)
    with MeshCodec(tris, n, anchors=torch.from_numpy(anchors).cuda(), n_frames=24, rank=6,
                   n_anchors=12, seed=8) as mc:
        rec = mc.decode(mc.encode(torch.from_numpy(pos).cuda())).cpu().numpy()
    o = oc.encode(tris, pos, oc.Params(n_frames=24, rank=6, n_anchors=12, seed=8),
                  anchors=anchors)
    e_o = metrics.nmse(pos, oc.decode(o, tris))
    assert abs(metrics.nmse(pos, rec) - e_o) <= 1e-9 * e_o
