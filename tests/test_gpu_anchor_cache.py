"""The factored decoder keeps the anchor response G = M^-1 P^T (it depends
only on the connectivity and the anchor set): later decodes with the same
anchors solve only the 3k data columns and give the same reconstruction."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import codec as oc, metrics  # noqa: E402
from synth import SequenceSpec, make_sequence  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_10105_gb300 import build
    build.build()


def _seq(seed=31):
    spec = SequenceSpec(name="a", mesh="icosphere:3", n_frames=40, rank=6, n_anchors=12,
                        seed=seed)
    return make_sequence(spec)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_second_decode_solves_only_the_data_columns(precision):
    from paper_2111_10105_gb300 import MeshCodec
    tris, pos = _seq()
    n = pos.shape[1]
    kw = dict(n_frames=40, rank=6, n_anchors=12, seed=4, solve_mode=1, precision=precision)
    if precision:
        kw.update(oi_refine_sweeps=1, cg_rtol=1e-6)
    with MeshCodec(tris, n, **kw) as mc:
        bits = mc.encode(torch.from_numpy(pos).cuda())
        first = mc.decode(bits).cpu().numpy()
        cols_first = mc.stats()["cg_columns"]
        second = mc.decode(bits).cpu().numpy()
        cols_second = mc.stats()["cg_columns"]
    pad = (lambda w: (w + 3) // 4 * 4) if precision else (lambda w: w)
    assert cols_first == pad(3 * 6 + 12)
    assert cols_second == pad(3 * 6)
    e1, e2 = metrics.nmse(pos, first), metrics.nmse(pos, second)
    assert abs(e1 - e2) <= {0: 1e-9, 1: 1e-3, 2: 1e-2}[precision] * e1
    if precision == 0:
        o = oc.encode(tris, pos, oc.Params(n_frames=40, rank=6, n_anchors=12, seed=4))
        e_o = metrics.nmse(pos, oc.decode(o, tris))
        assert abs(e2 - e_o) <= 1e-9 * e_o


def test_other_anchors_solve_every_column_again():
    from paper_2111_10105_gb300 import MeshCodec
    tris, pos = _seq()
    n = pos.shape[1]
    kw = dict(n_frames=40, rank=6, n_anchors=12, solve_mode=1)
    pos_d = torch.from_numpy(pos).cuda()
    with MeshCodec(tris, n, seed=4, **kw) as a, MeshCodec(tris, n, seed=5, **kw) as b:
        bits_a = a.encode(pos_d).clone()
        bits_b = b.encode(pos_d).clone()
        a.decode(bits_a)                                  # keeps G for a's anchors
        rec = a.decode(bits_b).cpu().numpy()              # b's anchors: full solve
        assert a.stats()["cg_columns"] == 3 * 6 + 12
        ref = b.decode(bits_b).cpu().numpy()
    assert np.abs(rec - ref).max() <= 1e-12 * np.abs(ref).max()


def test_unconverged_decode_keeps_nothing():
    from paper_2111_10105_gb300 import MeshCodec
    tris, pos = _seq()
    n = pos.shape[1]
    with MeshCodec(tris, n, n_frames=40, rank=6, n_anchors=12, seed=4, solve_mode=1,
                   cg_max_iters=3) as mc:
        bits = mc.encode(torch.from_numpy(pos).cuda())
        mc.decode(bits, allow_not_converged=True)
        mc.decode(bits, allow_not_converged=True)
        assert mc.stats()["cg_columns"] == 3 * 6 + 12


def _short(seed=31):
    # 3k + n_c = 18 + 12 > 3F = 24: the automatic mode starts with the frames solve
    spec = SequenceSpec(name="s", mesh="icosphere:3", n_frames=8, rank=6, n_anchors=12,
                        seed=seed)
    return make_sequence(spec)


def test_automatic_mode_switches_when_the_anchors_repeat():
    from paper_2111_10105_gb300 import MeshCodec
    tris, pos = _short()
    n = pos.shape[1]
    kw = dict(n_frames=8, rank=6, n_anchors=12, seed=4)
    o = oc.encode(tris, pos, oc.Params(**kw))
    e_o = metrics.nmse(pos, oc.decode(o, tris))
    cols, errs = [], []
    with MeshCodec(tris, n, solve_mode=2, **kw) as mc:
        bits = mc.encode(torch.from_numpy(pos).cuda())
        for _ in range(3):
            rec = mc.decode(bits).cpu().numpy()
            cols.append(mc.stats()["cg_columns"])
            errs.append(metrics.nmse(pos, rec))
    assert cols == [3 * 8, 3 * 6 + 12, 3 * 6]     # frames, factored (keeps G), kept G
    for e in errs:
        assert abs(e - e_o) <= 1e-9 * e_o


def test_automatic_mode_follows_the_latest_anchors():
    from paper_2111_10105_gb300 import MeshCodec
    tris, pos = _short()
    n = pos.shape[1]
    kw = dict(n_frames=8, rank=6, n_anchors=12, solve_mode=2)
    pos_d = torch.from_numpy(pos).cuda()
    with MeshCodec(tris, n, seed=4, **kw) as a, MeshCodec(tris, n, seed=5, **kw) as b:
        bits_a = a.encode(pos_d).clone()
        bits_b = b.encode(pos_d).clone()
        ref = b.decode(bits_b).cpu().numpy()
        cols = []
        for bits in (bits_a, bits_a, bits_b, bits_b, bits_b):
            rec = a.decode(bits).cpu().numpy()
            cols.append(a.stats()["cg_columns"])
    # a's anchors: frames, then factored; b's: new anchors -> frames, then factored, kept G
    assert cols == [24, 30, 24, 30, 18]
    assert np.abs(rec - ref).max() <= 1e-12 * np.abs(ref).max()


def test_automatic_mode_with_a_first_iterate_stays_on_frames():
    from paper_2111_10105_gb300 import MeshCodec
    tris, pos = _short()
    n = pos.shape[1]
    with MeshCodec(tris, n, n_frames=8, rank=6, n_anchors=12, seed=4, solve_mode=2) as mc:
        pos_d = torch.from_numpy(pos).cuda()
        bits = mc.encode(pos_d)
        x0 = pos_d.clone()
        for _ in range(2):
            mc.decode(bits, x0=x0)
            assert mc.stats()["cg_columns"] == 3 * 8
