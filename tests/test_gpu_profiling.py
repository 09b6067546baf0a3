"""Kernel timing (mesh_codec_set_profiling) times one CG iteration per
32-iteration run and replays the others from a CUDA graph: the decode's
result must not change, and every CG kernel must be timed."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from synth import SequenceSpec, make_sequence  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_10105_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", [0, 1])
def test_timed_decode_equals_untimed_decode(precision):
    from paper_2111_10105_gb300 import MeshCodec
    spec = SequenceSpec(name="p", mesh="icosphere:3", n_frames=24, rank=6, n_anchors=8, seed=21)
    tris, pos = make_sequence(spec)
    kw = dict(n_frames=24, rank=6, n_anchors=8, seed=21, solve_mode=1, precision=precision,
              cg_rtol=1e-6 if precision else 1e-14, oi_refine_sweeps=1 if precision else 0)
    with MeshCodec(tris, pos.shape[1], **kw) as mc:
        bits = mc.encode(torch.from_numpy(pos).cuda())
        mc.decode(bits)                         # keeps the anchor response
        plain = mc.decode(bits).cpu().numpy()
        iters = mc.stats()["cg_iters_max"]
        if precision == 0:
            assert iters > 64                   # several 32-iteration runs
        mc.set_profiling(16)
        timed = mc.decode(bits).cpu().numpy()
        prof = mc.profile()
        mc.set_profiling(0)
        assert mc.stats()["cg_iters_max"] == iters
    np.testing.assert_array_equal(timed, plain)
    names = {"k_cg_L", "k_cg_LT", "k_cg_alpha", "k_cg_update", "k_cg_beta", "k_cg_dir"}
    assert names <= set(prof)
    for k in names:
        launches, ms = prof[k]
        assert launches >= iters // 32 and ms > 0.0
    # the graph-replayed iterations, timed as whole runs without per-kernel events
    runs, ms = prof["cg_iteration"]
    assert runs >= 31 * (iters // 32) and ms > 0.0


def test_refined_solve_timing():
    from paper_2111_10105_gb300 import MeshCodec
    spec = SequenceSpec(name="p", mesh="icosphere:3", n_frames=24, rank=6, n_anchors=8, seed=21)
    tris, pos = make_sequence(spec)
    with MeshCodec(tris, pos.shape[1], n_frames=24, rank=6, n_anchors=8, seed=21, solve_mode=1,
                   precision=1, refine=2, cg_rtol=1e-13, oi_refine_sweeps=1) as mc:
        bits = mc.encode(torch.from_numpy(pos).cuda())
        mc.decode(bits)                         # keeps the anchor response
        plain = mc.decode(bits).cpu().numpy()
        run = mc.stats()["cg_iterations_run"]
        mc.set_profiling(1)
        timed = mc.decode(bits).cpu().numpy()
        prof = mc.profile()
        mc.set_profiling(0)
        assert mc.stats()["cg_iterations_run"] == run
    np.testing.assert_array_equal(timed, plain)
    runs, ms = prof["cg_iteration"]
    launches, _ = prof["k_cg_update"]
    # every refined run: its last iteration per kernel, the others as one run
    assert runs + launches == run and ms > 0.0
