"""Blocks variant (Section III-A, Algorithm 1) on the GPU against the oracle:
block 1's basis from the eigendecomposition of R[1], later blocks from
Algorithm 1's sweeps started at the previous basis, closed-loop dictionary
differences, and the container."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import blocks as ob, codec as oc, metrics  # noqa: E402
from synth import SequenceSpec, make_sequence  # noqa: E402

pytestmark = pytest.mark.gpu

NMSE_RTOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_10105_gb300 import build
    build.build()


def _seq(nb, kf, level=3, seed=21):
    spec = SequenceSpec(name="b", mesh=f"icosphere:{level}", n_frames=nb * kf, rank=6,
                        n_anchors=10, seed=seed)
    return make_sequence(spec)


def _params(kf, k=6, sweeps=8):
    return oc.Params(n_frames=kf, rank=k, n_anchors=10, seed=5, oi_sweeps=sweeps)


def _codec(tris, n, p, **kw):
    from paper_2111_10105_gb300 import MeshCodec
    return MeshCodec(tris, n, n_frames=p.n_frames, rank=p.rank, n_anchors=p.n_anchors,
                     seed=p.seed, oi_sweeps=p.oi_sweeps, **kw)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _bytes(blob):
    return torch.from_numpy(np.frombuffer(blob, dtype=np.uint8).copy()).cuda()


def test_first_block_basis_is_the_eigenbasis_of_R1():
    from paper_2111_10105_gb300 import codec as cb
    tris, pos = _seq(1, 24)
    p = _params(24)
    n = pos.shape[1]
    with _codec(tris, n, p) as mc:
        mc.encode_blocks(_cuda(pos), 1)
        U = mc.buffer(cb.BUF_BASIS).cpu().numpy().reshape(3, 24, p.rank)
        theta = mc.buffer(cb.BUF_RITZ).cpu().numpy().reshape(3, p.rank)
    for c in range(3):
        Uo, to = ob.direct_basis(pos[:, :, c], p.rank)
        assert np.abs(U[c] - Uo).max() < 1e-10
        assert np.allclose(theta[c], to, rtol=1e-12, atol=0)


@pytest.mark.parametrize("delta,mode", [(False, 0), (True, 0), (False, 1), (True, 1)])
def test_blocks_parity(delta, mode):
    from paper_2111_10105_gb300 import codec as cb
    nb, kf = 3, 16
    tris, pos = _seq(nb, kf)
    p = _params(kf)
    o = ob.encode_blocks(tris, pos, p, nb, delta=delta, delta_bits=10)
    rec_o = ob.decode_blocks(o, tris)
    n = pos.shape[1]
    with _codec(tris, n, p, solve_mode=mode, block_delta=int(delta),
                block_delta_bits=10 if delta else 0) as mc:
        g = mc.encode_blocks(_cuda(pos), nb)
        assert g.numel() == len(o) == mc.blocks_size(nb)
        assert g[:64].cpu().numpy().tobytes() == o[:64]
        U_last = mc.buffer(cb.BUF_BASIS).cpu().numpy().reshape(3, kf, p.rank)
        rec_g = mc.decode_blocks(g, nb).cpu().numpy()
        rec_go = mc.decode_blocks(_bytes(o), nb).cpu().numpy()
        assert mc.stats()["cg_not_converged"] == 0
    # the last block's basis: Algorithm 1's chain on the oracle
    U_prev = None
    for b in range(nb):
        U_prev = ob.block_bases(pos[b * kf:(b + 1) * kf], p, U_prev)
    for c in range(3):
        assert np.abs(U_last[c] - U_prev[c]).max() < 1e-8
    e_o = metrics.nmse(pos, rec_o)
    assert abs(metrics.nmse(pos, rec_g) - e_o) <= NMSE_RTOL * e_o
    # the GPU decoder on the oracle's container reproduces the oracle's decode
    assert np.abs(rec_go - rec_o).max() <= 1e-9 * np.abs(rec_o).max()


def test_long_first_block_uses_the_seeded_iterations():
    nb, kf = 2, 72                     # F > 64: no direct eigendecomposition on the GPU
    tris, pos = _seq(nb, kf, level=2)
    p = _params(kf, k=5, sweeps=30)
    o = ob.encode_blocks(tris, pos, p, nb)
    rec_o = ob.decode_blocks(o, tris)
    with _codec(tris, pos.shape[1], p) as mc:
        rec_g = mc.decode_blocks(mc.encode_blocks(_cuda(pos), nb), nb).cpu().numpy()
    e_o = metrics.nmse(pos, rec_o)
    assert abs(metrics.nmse(pos, rec_g) - e_o) <= NMSE_RTOL * e_o


def test_container_mismatch_is_rejected():
    from paper_2111_10105_gb300 import MeshCodecError
    nb, kf = 2, 12
    tris, pos = _seq(nb, kf, level=2)
    p = _params(kf, k=4)
    n = pos.shape[1]
    with _codec(tris, n, p) as mc:
        g = mc.encode_blocks(_cuda(pos), nb)
        bad = g.clone()
        bad[0] = 0
        with pytest.raises(MeshCodecError):
            mc.decode_blocks(bad, nb)
        with pytest.raises(MeshCodecError):
            mc.decode_blocks(g[:-8], nb)
    with _codec(tris, n, p, block_delta=1, block_delta_bits=8) as md:
        with pytest.raises(MeshCodecError):      # flags do not match the handle
            md.decode_blocks(g, nb)
