"""Mixed-precision modes (TF32 / BF16 tensor-core products, FP32 CG with
compensated dot products) against the FP64 mode of the same codec, through
the C ABI.  Stated bounds, per result:

* reconstruction NMSE: TF32 within 1% and BF16 within 10% of the FP64
  mode's NMSE on the small noisy grid workload and on the icosphere
  workload (measured: 5e-5 relative on the 99,856-vertex grid, 2e-5 on the
  icosphere);
* the dictionary is orthonormal to 1e-12 (its QR is FP64) and spans the
  FP64 dictionary's subspace to a principal-angle sine below 0.05 (TF32)
  and 0.25 (BF16);
* header, sizes and anchor indices of the bitstream are identical.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import metrics  # noqa: E402
from synth import SequenceSpec, make_sequence  # noqa: E402

pytestmark = pytest.mark.gpu

BOUNDS = {1: (0.01, 0.05), 2: (0.10, 0.25)}   # precision: (NMSE rel, max principal sine)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_10105_gb300 import build
    build.build()


def _run(spec, tris, pos, precision, mode=2):
    from paper_2111_10105_gb300 import MeshCodec, codec as cb
    n, F = pos.shape[1], pos.shape[0]
    kw = dict(n_frames=F, rank=spec.rank, n_anchors=spec.n_anchors, seed=spec.seed,
              oi_sweeps=30, precision=precision, oi_refine_sweeps=1 if precision else 0,
              solve_mode=mode, cg_rtol=1e-6 if precision else 1e-13)
    with MeshCodec(tris, n, **kw) as mc:
        bits = mc.encode(torch.from_numpy(pos).cuda())
        rec = mc.decode(bits).cpu().numpy()
        U = mc.buffer(cb.BUF_BASIS).cpu().numpy().reshape(3, F, spec.rank)
        return bits.cpu().numpy(), rec, U


SPECS = [
    SequenceSpec(name="grid", mesh="grid:64:64", n_frames=64, rank=16, n_anchors=41, seed=77,
                 n_bumps=4, rigid=False, noise=0.02),
    SequenceSpec(name="ico", mesh="icosphere:3", n_frames=37, rank=5, n_anchors=11, seed=78),
]


@pytest.mark.parametrize("spec", SPECS, ids=lambda s: s.name)
@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_precision_bounds(spec, precision):
    tris, pos = make_sequence(spec)
    b64, r64, U64 = _run(spec, tris, pos, 0)
    bmx, rmx, Umx = _run(spec, tris, pos, precision)
    e64, emx = metrics.nmse(pos, r64), metrics.nmse(pos, rmx)
    nmse_rel, sine = BOUNDS[precision]
    assert abs(emx - e64) <= nmse_rel * e64, (emx, e64)
    n_c = spec.n_anchors
    assert bytes(bmx[:64 + 4 * n_c]) == bytes(b64[:64 + 4 * n_c])
    for c in range(3):
        np.testing.assert_allclose(Umx[c].T @ Umx[c], np.eye(spec.rank), atol=1e-12)
        s = np.linalg.svd(U64[c].T @ Umx[c], compute_uv=False)
        assert np.sqrt(max(0.0, 1 - s.min() ** 2)) < sine


def test_mixed_frames_and_factored_agree():
    spec = SPECS[0]
    tris, pos = make_sequence(spec)
    _, ra, _ = _run(spec, tris, pos, 1, mode=0)
    _, rb, _ = _run(spec, tris, pos, 1, mode=1)
    ea, eb = metrics.nmse(pos, ra), metrics.nmse(pos, rb)
    assert abs(ea - eb) <= 1e-3 * ea
