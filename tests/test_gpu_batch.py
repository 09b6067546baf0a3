"""Batched encode/decode of independent sequences of uneven sizes, through
the C ABI: every sequence's bitstream and reconstruction equal those of the
same handle used alone, and the reconstructions match the FP64 oracle's
NMSE."""

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


SPECS = [
    SequenceSpec(name="a", mesh="icosphere:3", n_frames=40, rank=8, n_anchors=9, seed=11),
    SequenceSpec(name="b", mesh="torus:30:12", n_frames=23, rank=5, n_anchors=4, seed=12, bend=0.1),
    SequenceSpec(name="c", mesh="grid:20:31", n_frames=64, rank=12, n_anchors=7, seed=13,
                 n_bumps=2, rigid=False),
    SequenceSpec(name="d", mesh="icosphere:2", n_frames=9, rank=9, n_anchors=3, seed=14),
]


def _codecs(seqs, precision=0, autotune=0):
    from paper_2111_10105_gb300 import MeshCodec
    out = []
    for spec, (tris, pos) in zip(SPECS, seqs):
        out.append(MeshCodec(tris, pos.shape[1], n_frames=spec.n_frames, rank=spec.rank,
                             n_anchors=spec.n_anchors, seed=spec.seed, oi_sweeps=25,
                             solve_mode=2, precision=precision, autotune=autotune,
                             oi_refine_sweeps=1 if precision else 0,
                             cg_rtol=1e-6 if precision else 1e-13))
    return out


def test_batch_equals_single_and_oracle():
    from paper_2111_10105_gb300.codec import encode_batch, decode_batch
    seqs = [make_sequence(s) for s in SPECS]
    pos_d = [torch.from_numpy(p).cuda() for _, p in seqs]
    cs = _codecs(seqs)
    bits = encode_batch(cs, pos_d)
    recs = decode_batch(cs, bits)
    # fresh handles for the single calls: a handle's later decodes may take
    # another (equal up to rounding) solve path once its anchors repeat
    singles = _codecs(seqs)
    for c, b, r, (tris, pos), spec in zip(singles, bits, recs, seqs, SPECS):
        b1 = c.encode(torch.from_numpy(pos).cuda())
        assert torch.equal(b1, b)
        r1 = c.decode(b1)
        assert torch.equal(r1, r)
        p = oc.Params(n_frames=spec.n_frames, rank=spec.rank, n_anchors=spec.n_anchors,
                      seed=spec.seed, oi_sweeps=25)
        e_o = metrics.nmse(pos, oc.decode(oc.encode(tris, pos, p), tris))
        assert abs(metrics.nmse(pos, r.cpu().numpy()) - e_o) <= 1e-8 * e_o
    for c in cs + singles:
        c.close()


# the mixed batch: the same sequences with k < F throughout (truncation sets
# their NMSE, so the stated TF32 bound against the oracle applies)
MIXED = SPECS[:3] + [SequenceSpec(name="d6", mesh="icosphere:2", n_frames=9, rank=6,
                                  n_anchors=3, seed=14)]


def test_batch_mixed_autotuned_against_oracle():
    from paper_2111_10105_gb300 import MeshCodec
    from paper_2111_10105_gb300.codec import encode_batch, decode_batch
    seqs = [make_sequence(s) for s in MIXED]
    cs = [MeshCodec(tris, pos.shape[1], n_frames=spec.n_frames, rank=spec.rank,
                    n_anchors=spec.n_anchors, seed=spec.seed, oi_sweeps=25, solve_mode=2,
                    precision=1, autotune=1, oi_refine_sweeps=1, cg_rtol=1e-6)
          for spec, (tris, pos) in zip(MIXED, seqs)]
    pos_d = [torch.from_numpy(p).cuda() for _, p in seqs]
    bits = encode_batch(cs, pos_d)
    # two decodes: the automatic solve mode keeps the anchor response on the
    # second; the first with each sequence on its own stream, the second grouped
    for rnd in range(2):
        recs = decode_batch(cs, bits, grouped=rnd == 1)
        for spec, (tris, pos), r in zip(MIXED, seqs, recs):
            p = oc.Params(n_frames=spec.n_frames, rank=spec.rank, n_anchors=spec.n_anchors,
                          seed=spec.seed, oi_sweeps=25)
            e_o = metrics.nmse(pos, oc.decode(oc.encode(tris, pos, p), tris))
            e = metrics.nmse(pos, r.cpu().numpy())
            assert abs(e - e_o) <= 0.01 * e_o, (spec.name, e, e_o)
    for c in cs:
        c.close()


def test_grouped_batch_equals_single_decodes():
    # the FP32 solves of a batch advance as grouped batches (work-table
    # kernels over all sequences); every sequence's reconstruction must equal,
    # to the bit, the one its own handle gives alone, on the first decode
    # (frames or factored solves) and on the second (kept anchor response)
    from paper_2111_10105_gb300 import MeshCodec
    from paper_2111_10105_gb300.codec import encode_batch, decode_batch
    seqs = [make_sequence(s) for s in MIXED]

    def handles():
        return [MeshCodec(tris, pos.shape[1], n_frames=spec.n_frames, rank=spec.rank,
                          n_anchors=spec.n_anchors, seed=spec.seed, oi_sweeps=25, solve_mode=2,
                          precision=1, autotune=0, oi_refine_sweeps=1, cg_rtol=1e-6)
                for spec, (tris, pos) in zip(MIXED, seqs)]

    cs, singles = handles(), handles()
    pos_d = [torch.from_numpy(p).cuda() for _, p in seqs]
    bits = encode_batch(cs, pos_d)
    for rnd in range(3):
        recs = decode_batch(cs, bits, grouped=True)
        for c, b, r in zip(singles, bits, recs):
            r1 = c.decode(b)
            assert torch.equal(r1, r), rnd
            assert c.stats()["cg_iters_max"] > 0
    for c in cs + singles:
        c.close()
