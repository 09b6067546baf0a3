"""Mixed-precision modes (TF32 / BF16 tensor-core products, FP32 CG with
compensated dot products) against the FP64 oracle (oracle.codec) on the
same seeded input, through the C ABI.  Stated bounds, per result:

* plain mixed modes (the tensor cores in the orthogonal-iteration sweeps,
  the projection of Eq. 9 and the final products; FP32 CG to 1e-6):
  reconstruction NMSE within 1% (TF32) / 10% (BF16) of the oracle's NMSE,
  where that NMSE is set by the data (noise, truncation at k < rank): the
  noisy grids and the truncated icosphere below;
* mixed modes with the refined solve (FP64 residuals, FP32 corrections,
  FP64 projection and final products): within 1% of the oracle's NMSE also
  where the codec is near-lossless (k close to F, NMSE ~1e-8), the case
  where the plain modes' float32 and TF32 rounding would dominate;
* the dictionary is orthonormal to 1e-12 (its QR is FP64) and spans the
  oracle's dictionary subspace to a principal-angle sine below 0.05 (TF32)
  and 0.25 (BF16);
* header, sizes and anchor indices of the bitstream equal the oracle's.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import codec as oc, metrics  # noqa: E402
from synth import SequenceSpec, make_sequence  # noqa: E402

pytestmark = pytest.mark.gpu

BOUNDS = {1: (0.01, 0.05), 2: (0.10, 0.25)}   # precision: (NMSE rel, max principal sine)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_10105_gb300 import build
    build.build()


def _oracle(spec, tris, pos, sweeps=30):
    p = oc.Params(n_frames=spec.n_frames, rank=spec.rank, n_anchors=spec.n_anchors,
                  seed=spec.seed, oi_sweeps=sweeps)
    blob, info = oc.encode(tris, pos, p, return_info=True)
    return blob, metrics.nmse(pos, oc.decode(blob, tris)), info["U"]


def _codec(spec, n, tris, precision, mode=2, refine=0):
    from paper_2111_10105_gb300 import MeshCodec
    single = precision and not refine
    return MeshCodec(tris, n, n_frames=spec.n_frames, rank=spec.rank, n_anchors=spec.n_anchors,
                     seed=spec.seed, oi_sweeps=30, precision=precision,
                     oi_refine_sweeps=1 if precision else 0, solve_mode=mode, refine=refine,
                     cg_rtol=1e-6 if single else 1e-13)


SPECS = [
    SequenceSpec(name="grid64", mesh="grid:64:64", n_frames=64, rank=16, n_anchors=41, seed=77,
                 n_bumps=4, rigid=False, noise=0.02),
    SequenceSpec(name="ico", mesh="icosphere:3", n_frames=37, rank=5, n_anchors=11, seed=78),
    # 16,384 vertices, k = 64: split-K tensor-core sweeps, the projection and
    # final products over several tiles, 356 then (kept anchor response) 192
    # CG columns, i.e. two FP32 CG tile widths
    SequenceSpec(name="grid128", mesh="grid:128:128", n_frames=128, rank=64, n_anchors=164,
                 seed=79, n_bumps=4, rigid=False, noise=0.02),
]


@pytest.mark.parametrize("spec", SPECS, ids=lambda s: s.name)
@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_precision_against_oracle(spec, precision):
    from paper_2111_10105_gb300 import codec as cb
    tris, pos = make_sequence(spec)
    blob, e_o, U_o = _oracle(spec, tris, pos)
    nmse_rel, sine = BOUNDS[precision]
    with _codec(spec, pos.shape[1], tris, precision, mode=1) as mc:
        bits = mc.encode(torch.from_numpy(pos).cuda())
        U = mc.buffer(cb.BUF_BASIS).cpu().numpy().reshape(3, spec.n_frames, spec.rank)
        # first decode solves 3k + n_c columns, the second keeps the anchor response
        for rnd in range(2):
            rec = mc.decode(bits).cpu().numpy()
            cols = mc.stats()["cg_columns"]
            # FP32 solves pad their column count to a multiple of four
            want = 3 * spec.rank + (spec.n_anchors if rnd == 0 else 0)
            assert cols == (want + 3) // 4 * 4
            e = metrics.nmse(pos, rec)
            assert abs(e - e_o) <= nmse_rel * e_o, (rnd, e, e_o)
    b = bits.cpu().numpy()
    n_c = spec.n_anchors
    assert bytes(b[:64 + 4 * n_c]) == blob[:64 + 4 * n_c]
    for c in range(3):
        np.testing.assert_allclose(U[c].T @ U[c], np.eye(spec.rank), atol=1e-12)
        s = np.linalg.svd(U_o[c].T @ U[c], compute_uv=False)
        assert np.sqrt(max(0.0, 1 - s.min() ** 2)) < sine


SMOOTH = [
    SequenceSpec(name="torus60_k40", mesh="torus:60:30", n_frames=48, rank=40, n_anchors=18,
                 seed=80, bend=0.1),
    SequenceSpec(name="grid48_k40", mesh="grid:48:40", n_frames=40, rank=40, n_anchors=19,
                 seed=81, n_bumps=3, rigid=False),
]


@pytest.mark.parametrize("spec", SMOOTH, ids=lambda s: s.name)
@pytest.mark.parametrize("precision", [1, 2])
def test_refined_mixed_modes_on_near_lossless_sequences(spec, precision):
    tris, pos = make_sequence(spec)
    _, e_o, _ = _oracle(spec, tris, pos)
    with _codec(spec, pos.shape[1], tris, precision, mode=2, refine=2) as mc:
        rec = mc.decode(mc.encode(torch.from_numpy(pos).cuda())).cpu().numpy()
    e = metrics.nmse(pos, rec)
    assert abs(e - e_o) <= BOUNDS[precision][0] * e_o, (e, e_o)


def test_mixed_frames_and_factored_agree_with_oracle():
    spec = SPECS[0]
    tris, pos = make_sequence(spec)
    _, e_o, _ = _oracle(spec, tris, pos)
    for mode in (0, 1):
        with _codec(spec, pos.shape[1], tris, 1, mode=mode) as mc:
            rec = mc.decode(mc.encode(torch.from_numpy(pos).cuda())).cpu().numpy()
        assert abs(metrics.nmse(pos, rec) - e_o) <= 0.01 * e_o


def _stored_nmse(name):
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "nmse_reference.txt")
    for line in open(path):
        parts = line.split()
        if parts and not line.startswith("#") and parts[0] == name:
            return int(parts[1]), float(parts[2])
    raise KeyError(name)


def test_grid316_tf32_against_stored_oracle_nmse():
    # the 99,856-vertex mixed-precision workload at full size, in the form the
    # benchmark times (TF32, factored solve, kept anchor response on the
    # second decode), against the oracle's NMSE stored by
    # tests/golden/make_nmse_reference.py
    from synth import config_spec
    spec = config_spec("grid316_F512_k64")
    sweeps, e_o = _stored_nmse("grid316_F512_k64")
    tris, pos = make_sequence(spec)
    from paper_2111_10105_gb300 import MeshCodec
    with MeshCodec(tris, pos.shape[1], n_frames=spec.n_frames, rank=spec.rank,
                   n_anchors=spec.n_anchors, seed=spec.seed, oi_sweeps=sweeps, precision=1,
                   oi_refine_sweeps=1, solve_mode=1, cg_rtol=1e-6) as mc:
        pos_d = torch.from_numpy(pos).cuda()
        bits = mc.encode(pos_d)
        for _ in range(2):
            rec = mc.decode(bits).cpu().numpy()
            assert abs(metrics.nmse(pos, rec) - e_o) <= 0.01 * e_o


def test_grid512_refined_tf32_against_stored_oracle_nmse():
    # the 262,144-vertex workload at full size in the form the benchmark times
    # (TF32 sweeps, FP64-residual refined solve to 1e-9 with FP32 corrections
    # of up to 5 decades, factored solve, seeded random anchors): the cold
    # decode (3k + n_c columns) and the decode with the kept anchor response
    # (3k columns) against the oracle's stored NMSE
    from synth import config_spec
    spec = config_spec("grid512_F300_k64")
    sweeps, e_o = _stored_nmse("grid512_F300_k64")
    tris, pos = make_sequence(spec)
    from paper_2111_10105_gb300 import MeshCodec
    with MeshCodec(tris, pos.shape[1], n_frames=spec.n_frames, rank=spec.rank,
                   n_anchors=spec.n_anchors, seed=spec.seed, coeff_bits=spec.coeff_bits,
                   dict_bits=spec.dict_bits, anchor_bits=spec.anchor_bits, oi_sweeps=sweeps,
                   precision=1, oi_refine_sweeps=1, solve_mode=1, refine=5,
                   cg_rtol=1e-9) as mc:
        bits = mc.encode(torch.from_numpy(pos).cuda())
        for want_cols in (3 * spec.rank + spec.n_anchors, 3 * spec.rank):
            rec = mc.decode(bits).cpu().numpy()
            st = mc.stats()
            assert st["cg_columns"] == (want_cols + 3) // 4 * 4
            assert st["cg_not_converged"] == 0
            assert abs(metrics.nmse(pos, rec) - e_o) <= 0.01 * e_o
