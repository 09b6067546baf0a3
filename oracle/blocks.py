"""Blocks variant of the codec (Section III-A, Algorithm 1).

Test infrastructure (see ``oracle/__init__``).

A sequence of n_b * k_f frames is cut into n_b blocks of k_f consecutive
frames (the paper's k_f = k / n_b, k its frame count), each coded as a
stream of its own with the same connectivity, anchors and parameters:

* block 1: U[1] from the eigendecomposition of R[1] = A A^T (Algorithm 1's
  SVD of R[1]; k_f x k_f), the k eigenvectors of the largest eigenvalues,
  ordered and signed as in ``subspace`` (reading: for k_f above 64 the
  codec's GPU eigensolver does not apply and block 1 runs the one-block
  orthogonal iterations from the seeded start instead);
* block i >= 2: Algorithm 1's update, U[i]^(1) = U[i-1] and p.oi_sweeps
  sweeps Q <- QR(R[i] Q), then Rayleigh-Ritz ordering and signs;
* with difference coding (Section IV, Fig. 6), blocks i >= 2 carry
  U[i] - U^[i-1] in their dictionary section, U^[i-1] being the decoder's
  dequantized previous dictionary (closed loop, so quantization errors do not
  accumulate), in `delta_bits` bits.

Container (little-endian): 64-byte header magic "DMCB", u32 version = 1,
u32 n_blocks, u32 flags (bit 0: dictionary differences), u32 delta_bits,
u64 first block bytes, u64 other block bytes, u64 total bytes, zero
padding; then the block streams in order (each a v1 stream of
``codec``, 8-byte aligned by construction).

Pinned by (tests/test_oracle_blocks.py): with one block the container holds
exactly the one-block stream of the direct basis; block 1's basis is the
brute-force eigenbasis; later blocks converge to their own brute-force
eigenbasis from the previous block's; the closed-loop dictionary stays
within half a quantizer step of the exact one; decoding reproduces each
block's one-block decode.
"""

import struct

import numpy as np

from . import codec, subspace

MAGIC = b"DMCB"
VERSION = 1
HEADER_BYTES = 64
DIRECT_MAX_FRAMES = 64


def direct_basis(A_c, k):
    """Top-k eigenvectors of A_c A_c^T (F x F), descending, signed."""
    R = A_c @ A_c.T
    R = 0.5 * (R + R.T)
    theta, V = np.linalg.eigh(R)
    order = np.argsort(-theta, kind="stable")[:k]
    return subspace.sign_rule(V[:, order]), theta[order]


def warm_basis(A_c, U_prev, sweeps):
    """Algorithm 1's update from the previous block's basis, then
    Rayleigh-Ritz ordering and signs."""
    Q, _, _ = subspace.orthogonal_iterations(A_c, U_prev, sweeps)
    U, theta = subspace.rayleigh_ritz(A_c, Q)
    return subspace.sign_rule(U), theta


def block_bases(positions_block, p, U_prev):
    F = positions_block.shape[0]
    out = []
    for c in range(3):
        A_c = positions_block[:, :, c]
        if U_prev is not None:
            U, _ = warm_basis(A_c, U_prev[c], p.oi_sweeps)
        elif F <= DIRECT_MAX_FRAMES:
            U, _ = direct_basis(A_c, p.rank)
        else:
            U, _, _, _ = subspace.top_k_basis(A_c, p.rank, p.seed, c, p.oi_sweeps)
        out.append(U)
    return out


def container_size(n, p, n_blocks, delta=False, delta_bits=16):
    first = codec.stream_size(n, p.n_frames, p.rank, p.n_anchors, p.coeff_bits, p.dict_bits,
                              p.anchor_bits)
    other = codec.stream_size(n, p.n_frames, p.rank, p.n_anchors, p.coeff_bits,
                              delta_bits if delta else p.dict_bits, p.anchor_bits)
    return HEADER_BYTES + first + (n_blocks - 1) * other, first, other


def encode_blocks(tris, positions, p, n_blocks, delta=False, delta_bits=16):
    positions = np.asarray(positions, dtype=np.float64)
    kf = p.n_frames
    assert positions.shape[0] == n_blocks * kf
    n = positions.shape[1]
    total, first, other = container_size(n, p, n_blocks, delta, delta_bits)
    header = bytearray(HEADER_BYTES)
    struct.pack_into("<4sIIIIQQQ", header, 0, MAGIC, VERSION, n_blocks, 1 if delta else 0,
                     delta_bits if delta else 0, first, other, total)
    parts = [bytes(header)]
    U_prev = None      # encoder's exact previous basis (Algorithm 1)
    U_hat = None       # decoder's dequantized previous dictionary
    for b in range(n_blocks):
        blk = positions[b * kf:(b + 1) * kf]
        U = block_bases(blk, p, U_prev)
        ref = U_hat if (delta and b > 0) else None
        blob = codec.encode(tris, blk, p, basis=U, dict_ref=ref,
                            dict_bits=delta_bits if ref is not None else None)
        parts.append(blob)
        U_hat = codec.parse(blob, ref)["U"]
        U_prev = U
    out = b"".join(parts)
    assert len(out) == total
    return out


def parse_container(blob):
    if len(blob) < HEADER_BYTES:
        raise codec.BitstreamError("truncated container")
    magic, version, n_blocks, flags, delta_bits, first, other, total = struct.unpack_from(
        "<4sIIIIQQQ", blob, 0)
    if magic != MAGIC or version != VERSION or n_blocks < 1 or total != len(blob):
        raise codec.BitstreamError("bad container header")
    if HEADER_BYTES + first + (n_blocks - 1) * other != total:
        raise codec.BitstreamError("bad container sizes")
    streams = [blob[HEADER_BYTES:HEADER_BYTES + first]]
    off = HEADER_BYTES + first
    for _ in range(n_blocks - 1):
        streams.append(blob[off:off + other])
        off += other
    return {"n_blocks": n_blocks, "delta": bool(flags & 1), "delta_bits": delta_bits,
            "streams": streams}


def decode_blocks(blob, tris):
    d = parse_container(blob)
    outs = []
    U_hat = None
    for b, s in enumerate(d["streams"]):
        ref = U_hat if (d["delta"] and b > 0) else None
        outs.append(codec.decode(s, tris, dict_ref=ref))
        U_hat = codec.parse(s, ref)["U"]
    return np.concatenate(outs, axis=0)
