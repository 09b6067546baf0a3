"""Pins of the blocks variant (oracle/blocks.py, Section III-A, Algorithm 1)."""

import numpy as np
import pytest

from oracle import blocks, codec, metrics, subspace
from synth import SequenceSpec, make_sequence


def _seq(n_blocks=3, kf=12, level=2, seed=7, **kw):
    spec = SequenceSpec(name="b", mesh=f"icosphere:{level}", n_frames=n_blocks * kf, rank=5,
                        n_anchors=6, seed=seed, **kw)
    return make_sequence(spec)


def _params(kf=12, k=5, **kw):
    d = dict(n_frames=kf, rank=k, n_anchors=6, seed=3, oi_sweeps=8)
    d.update(kw)
    return codec.Params(**d)


def test_direct_basis_is_the_brute_force_eigenbasis():
    _, pos = _seq(n_blocks=1)
    for c in range(3):
        U, theta = blocks.direct_basis(pos[:, :, c], 5)
        Ub = subspace.sign_rule(subspace.brute_force_basis(pos[:, :, c], 5)[0])
        assert np.abs(U - Ub).max() < 1e-9
        assert np.all(np.diff(theta) <= 0)


def test_one_block_container_is_the_direct_one_block_stream():
    tris, pos = _seq(n_blocks=1)
    p = _params()
    blob = blocks.encode_blocks(tris, pos, p, 1)
    U = [blocks.direct_basis(pos[:, :, c], p.rank)[0] for c in range(3)]
    assert blob[blocks.HEADER_BYTES:] == codec.encode(tris, pos, p, basis=U)
    d = blocks.parse_container(blob)
    assert d["n_blocks"] == 1 and not d["delta"]


def test_warm_started_blocks_converge_to_their_own_eigenbasis():
    _, pos = _seq(n_blocks=2)
    kf = 12
    for c in range(3):
        U1, _ = blocks.direct_basis(pos[:kf, :, c], 5)
        U2, _ = blocks.warm_basis(pos[kf:, :, c], U1, 300)
        Ub = subspace.sign_rule(subspace.brute_force_basis(pos[kf:, :, c], 5)[0])
        assert np.abs(U2 - Ub).max() < 1e-8


@pytest.mark.parametrize("delta", [False, True])
def test_full_rank_raw_blocks_reconstruct_exactly(delta):
    tris, pos = _seq(n_blocks=3, kf=8)
    p = _params(kf=8, k=8, coeff_bits=0, dict_bits=0, anchor_bits=0, oi_sweeps=4)
    blob = blocks.encode_blocks(tris, pos, p, 3, delta=delta, delta_bits=0)
    rec = blocks.decode_blocks(blob, tris)
    assert np.abs(rec - pos).max() < 1e-9


def test_closed_loop_dictionary_within_half_a_step():
    tris, pos = _seq(n_blocks=3)
    p = _params()
    bits = 10
    blob = blocks.encode_blocks(tris, pos, p, 3, delta=True, delta_bits=bits)
    d = blocks.parse_container(blob)
    assert d["delta"] and d["delta_bits"] == bits
    kf = p.n_frames
    U_prev, U_hat = None, None
    for b in range(3):
        U = blocks.block_bases(pos[b * kf:(b + 1) * kf], p, U_prev)
        ref = U_hat if b > 0 else None
        got = codec.parse(d["streams"][b], ref)["U"]
        for c in range(3):
            D = U[c] - (ref[c] if ref is not None else 0.0)
            step = (D.max(axis=0) - D.min(axis=0)) / (2 ** (bits if b else p.dict_bits) - 1)
            err = np.abs(got[c] - U[c])
            assert np.all(err <= 0.5 * step[None, :] * (1 + 1e-9) + 1e-15)
        U_prev, U_hat = U, got


def test_differences_shrink_the_dictionary_error():
    # coherent blocks (every block repeats the first one's motion plus a small
    # drift): U[i] - U^[i-1] spans less than U[i], so at equal bits the
    # closed-loop dictionary is closer to the exact one
    tris, first = _seq(n_blocks=1, kf=16, level=3, seed=11)
    r = np.random.default_rng(2)
    pos = np.concatenate([first + 1e-3 * b * r.normal(size=first.shape) for b in range(4)])
    p = _params(kf=16, k=4, dict_bits=8)
    err = {}
    for delta in (False, True):
        blob = blocks.encode_blocks(tris, pos, p, 4, delta=delta, delta_bits=8)
        d = blocks.parse_container(blob)
        U_prev, U_hat, e = None, None, 0.0
        for b in range(4):
            U = blocks.block_bases(pos[b * 16:(b + 1) * 16], p, U_prev)
            ref = U_hat if (delta and b > 0) else None
            got = codec.parse(d["streams"][b], ref)["U"]
            if b > 0:
                e += sum(np.abs(got[c] - U[c]).max() for c in range(3))
            U_prev, U_hat = U, got
        err[delta] = e
    assert err[True] < err[False]


def test_blocks_decode_matches_per_block_decodes_and_quality():
    tris, pos = _seq(n_blocks=3)
    p = _params()
    blob = blocks.encode_blocks(tris, pos, p, 3)
    rec = blocks.decode_blocks(blob, tris)
    d = blocks.parse_container(blob)
    for b in range(3):
        np.testing.assert_array_equal(rec[b * 12:(b + 1) * 12], codec.decode(d["streams"][b], tris))
    assert metrics.nmse(pos, rec) < 1e-2


def test_container_errors():
    tris, pos = _seq(n_blocks=2)
    blob = blocks.encode_blocks(tris, pos, _params(), 2)
    with pytest.raises(codec.BitstreamError):
        blocks.parse_container(blob[:-8])
    with pytest.raises(codec.BitstreamError):
        blocks.parse_container(b"XXXX" + blob[4:])
