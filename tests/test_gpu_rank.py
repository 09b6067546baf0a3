"""Numerically rank-deficient trajectories: the orthonormalisation completes
the basis instead of failing, the well-determined part of the subspace
matches the oracle's Householder QR, and the reconstruction matches the
oracle's NMSE."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import codec as oc, metrics  # noqa: E402
from synth import icosphere  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_10105_gb300 import build
    build.build()


def _low_rank_sequence(F=24, level=3, seed=3):
    """Each coordinate's trajectory matrix has rank 3: rest pose, a linear
    translation and one separable field (spatial pattern x sin(t))."""
    verts, tris = icosphere(level)
    r = np.random.default_rng(seed)
    t = np.arange(F, dtype=np.float64)
    shift = r.uniform(-0.3, 0.3, size=3)
    d = r.normal(size=3)
    d /= np.linalg.norm(d)
    g = np.sin(3.0 * verts @ r.normal(size=3))
    pos = (verts[None] + (t / F)[:, None, None] * shift[None, None, :]
           + 0.05 * np.sin(2 * np.pi * t / F)[:, None, None] * g[None, :, None] * d[None, None, :])
    return tris, np.ascontiguousarray(pos)


@pytest.mark.parametrize("k", [6, 12])
def test_rank_deficient_encode_completes_basis(k):
    from paper_2111_10105_gb300 import MeshCodec, codec as cb
    tris, pos = _low_rank_sequence()
    F, n = pos.shape[0], pos.shape[1]
    p = oc.Params(n_frames=F, rank=k, n_anchors=9, seed=11, oi_sweeps=30)
    o = oc.encode(tris, pos, p)
    rec_o = oc.decode(o, tris)
    with MeshCodec(tris, n, n_frames=F, rank=k, n_anchors=9, seed=11, oi_sweeps=30) as mc:
        bits = mc.encode(torch.from_numpy(pos).cuda())
        U = mc.buffer(cb.BUF_BASIS).cpu().numpy().reshape(3, F, k)
        rec = mc.decode(bits).cpu().numpy()
    info = oc.parse(o)
    for c in range(3):
        # orthonormal, although only 3 directions carry data
        assert np.abs(U[c].T @ U[c] - np.eye(k)).max() < 1e-12
        # the three data directions agree with the oracle's (both sign-ruled;
        # the oracle's dictionary is the 16-bit dequantized one)
        assert np.abs(U[c][:, :3] - info["U"][c][:, :3]).max() < 1e-3
    e_o = metrics.nmse(pos, rec_o)
    e_g = metrics.nmse(pos, rec)
    assert abs(e_g - e_o) <= 1e-6 * e_o + 1e-15, (e_g, e_o)


def test_rank_deficient_start_basis():
    from paper_2111_10105_gb300 import MeshCodec, codec as cb
    tris, pos = _low_rank_sequence(F=20)
    F, n, k = 20, pos.shape[1], 5
    r = np.random.default_rng(1)
    q0 = r.normal(size=(3, F, k))
    q0[:, :, 3] = q0[:, :, 0] + q0[:, :, 1]        # dependent column
    q0[:, :, 4] = 0.0                              # zero column
    with MeshCodec(tris, n, n_frames=F, rank=k, n_anchors=4, seed=2) as mc:
        mc.set_start_basis(torch.from_numpy(q0).cuda())
        Q = mc.buffer(cb.BUF_START).cpu().numpy().reshape(3, F, k)
    for c in range(3):
        assert np.abs(Q[c].T @ Q[c] - np.eye(k)).max() < 1e-12
        # the independent leading columns span what they spanned
        Qr, _ = np.linalg.qr(q0[c][:, :3])
        P = Q[c][:, :3] @ Q[c][:, :3].T
        assert np.abs(P @ Qr - Qr).max() < 1e-10
