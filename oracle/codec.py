"""Encoder and decoder of the codec, with the bitstream layout.

Test infrastructure (see ``oracle/__init__``).

Notation: F frames (the paper's k), n vertices, rank k (the paper's k_l),
n_c anchors (the paper's n_c, index set N).  Positions are float64
[F, n, 3]; A_c = positions[:, :, c] is the F x n matrix of Section III.

Encoder (Section III, Fig. 1), per coordinate c:
  1. U_c: top-k eigen-trajectories of R_c = A_c A_c^T (Eq. 7, Eq. 5) by
     orthogonal iterations (Algorithm 1) and Rayleigh-Ritz (``subspace``).
  2. delta_c = L A_c^T, n x F (Eq. 8), with L from the fixed connectivity.
  3. C_c = U_c^T delta_c^T, k x n: the first k rows of the projection of
     Eq. 9 (projecting on all F eigenvectors and zeroing rows >= k, Eq. 10,
     is the same thing).
  4. Q(.) of Eq. 10 on C_c (per row), on U_c (per column, the dictionary
     that the decoder needs, Section IV) and on the anchor positions
     (per coordinate, Eq. 12's Q(A^T) restricted to N).
Anchors: n_c vertices drawn uniformly without replacement (the paper picks
them at random, Section V): the n_c smallest splitmix64 keys
(seed ^ ANCHOR_SALT, element i for vertex i), ties by index, sorted.

Decoder (Eq. 11-12): delta~_c = (U_c' C_c')^T from the dequantized
dictionary and coefficients; the positions solve the stacked least-squares
problem of Eq. 12,  min_X ||L X - delta~_c||^2 + ||P X - a^_c||^2  with P the
rows of the identity at N and unit weights, through its normal equations
(L^T L + P^T P) X = L^T delta~_c + P^T a^_c for all F frames at once (the
paper's parallel reconstruction "PCA+qp", Section IV (v)).  The oracle
solves them with sparse LU (SuperLU through scipy) of the assembled matrix,
then refines the result with residuals of the unassembled operator
L^T (L X) + P^T P X computed in extended precision, so that it returns the
binary64 rounding of the exact solution.  Eq. 12 as printed stacks an F x n block on
an n_c x F block; reading it as the least-squares problem above is the
only dimensionally consistent form.

Bitstream v1 (little-endian):
  header, 64 bytes: magic "DMC1", u32 version=1, u32 n, u32 F, u32 k,
    u32 n_anchors, u8 coeff_bits, u8 dict_bits, u8 anchor_bits,
    u8 laplacian_kind, u32 header_bytes=64, u64 total_bytes, zero padding.
  anchor indices: int32[n_anchors], ascending, padded to 8 bytes.
  per coordinate c = 0, 1, 2:
    f64 dict_lo[k], dict_hi[k], coef_lo[k], coef_hi[k], anc_lo, anc_hi
    dictionary: F*k symbols, index j*F + f (column-major U_c)
    coefficients: k*n symbols, index r*n + i (row-major C_c)
    anchors: n_anchors*F symbols, index a*F + f
  Each symbol section is packed b-bit words (``quant.pack_bits``), or raw
  f64 values when its bit count is 0, and is padded to 8 bytes.

Pinned by: k = F with raw coefficients and anchors reproduces A to
rounding; consistent systems return their exact solution; the
normal-equation residual; dense least squares on small meshes
(tests/test_oracle_codec.py).
"""

from dataclasses import dataclass
import struct

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import graph, quant, rng, subspace

MAGIC = b"DMC1"
VERSION = 1
HEADER_BYTES = 64


@dataclass
class Params:
    n_frames: int
    rank: int
    n_anchors: int
    coeff_bits: int = 12
    dict_bits: int = 16
    anchor_bits: int = 16
    laplacian_kind: int = 0
    oi_sweeps: int = 30
    oi_tol: float = 0.0
    seed: int = 0


def select_anchors(n, n_anchors, seed):
    if n_anchors < 0 or n_anchors > n:
        raise ValueError("n_anchors out of range")
    keys = rng.stream((seed ^ rng.ANCHOR_SALT) & rng.MASK64, n)
    order = np.lexsort((np.arange(n), keys))
    return np.sort(order[:n_anchors]).astype(np.int32)


def _pad8(nbytes):
    return (nbytes + 7) // 8 * 8


def _section_bytes(count, bits):
    if bits == 0:
        return count * 8
    return _pad8(quant.packed_words(count, bits) * 4)


def stream_size(n, F, k, n_anchors, coeff_bits, dict_bits, anchor_bits):
    size = HEADER_BYTES + _pad8(4 * n_anchors)
    per_c = 8 * (4 * k + 2)
    per_c += _section_bytes(F * k, dict_bits)
    per_c += _section_bytes(k * n, coeff_bits)
    per_c += _section_bytes(n_anchors * F, anchor_bits)
    return size + 3 * per_c


def _encode_section(values, lo, hi, bits):
    if bits == 0:
        return np.ascontiguousarray(values, dtype="<f8").tobytes()
    s = quant.quantize(values, lo, hi, bits)
    w = quant.pack_bits(s.ravel(), bits).astype("<u4").tobytes()
    return w + b"\0" * (_pad8(len(w)) - len(w))


def encode(tris, positions, p, return_info=False, basis=None, dict_ref=None, dict_bits=None,
           anchors=None):
    """Encodes one block.  `basis` (three F x k matrices) replaces the
    orthogonal iterations from the seeded start (the blocks variant, Section
    III-A, supplies its own U[i]); with `dict_ref` (three F x k matrices) the
    dictionary section carries U - dict_ref (the difference coding of
    consecutive dictionaries, Section IV, Fig. 6) in `dict_bits` bits.
    `anchors` (p.n_anchors strictly increasing vertex indices) replaces the
    seeded anchor choice."""
    positions = np.asarray(positions, dtype=np.float64)
    F, n, three = positions.shape
    assert three == 3 and F == p.n_frames
    k = p.rank
    if not (1 <= k <= F):
        raise ValueError("rank must satisfy 1 <= k <= F")
    db = p.dict_bits if dict_bits is None else dict_bits
    row_ptr, col_idx, deg = graph.build_adjacency(tris, n)
    if anchors is None:
        anchors = select_anchors(n, p.n_anchors, p.seed)
    else:
        anchors = np.asarray(anchors, dtype=np.int32)
        if anchors.shape != (p.n_anchors,) or (anchors.size and (
                anchors[0] < 0 or anchors[-1] >= n or np.any(np.diff(anchors) <= 0))):
            raise ValueError("anchors must be n_anchors strictly increasing indices in [0, n)")

    header = bytearray(HEADER_BYTES)
    total = stream_size(n, F, k, p.n_anchors, p.coeff_bits, db, p.anchor_bits)
    struct.pack_into("<4sIIIIIBBBBIQ", header, 0, MAGIC, VERSION, n, F, k,
                     p.n_anchors, p.coeff_bits, db, p.anchor_bits,
                     p.laplacian_kind, HEADER_BYTES, total)
    out = [bytes(header)]
    a = anchors.astype("<i4").tobytes()
    out.append(a + b"\0" * (_pad8(len(a)) - len(a)))

    info = {"U": [], "theta": [], "C": [], "delta": [], "sweeps": [], "change": [],
            "anchors": anchors, "csr": (row_ptr, col_idx, deg)}
    for c in range(3):
        A_c = positions[:, :, c]                                    # F x n
        if basis is None:
            U, theta, done, change = subspace.top_k_basis(A_c, k, p.seed, c, p.oi_sweeps,
                                                          p.oi_tol)
        else:
            U, theta, done, change = basis[c], None, 0, 0.0
        delta = graph.apply_laplacian(row_ptr, col_idx, deg, A_c.T, p.laplacian_kind)  # n x F
        C = U.T @ delta.T                                            # k x n
        anc_vals = A_c[:, anchors].T                                 # n_c x F
        Ud = U if dict_ref is None else U - dict_ref[c]             # coded dictionary
        d_lo, d_hi = quant.quant_params(Ud, axis=0)
        c_lo, c_hi = quant.quant_params(C, axis=1)
        if anchors.shape[0]:
            a_lo, a_hi = quant.quant_params(anc_vals)
        else:
            a_lo, a_hi = np.float64(0.0), np.float64(0.0)
        out.append(np.concatenate([d_lo, d_hi, c_lo, c_hi, [a_lo, a_hi]]).astype("<f8").tobytes())
        out.append(_encode_section(Ud.T, d_lo[:, None], d_hi[:, None], db))
        out.append(_encode_section(C, c_lo[:, None], c_hi[:, None], p.coeff_bits))
        out.append(_encode_section(anc_vals, a_lo, a_hi, p.anchor_bits))
        for key, v in (("U", U), ("theta", theta), ("C", C), ("delta", delta),
                       ("sweeps", done), ("change", change)):
            info[key].append(v)
    blob = b"".join(out)
    assert len(blob) == total
    return (blob, info) if return_info else blob


class BitstreamError(ValueError):
    pass


def parse(blob, dict_ref=None):
    """Bitstream -> dict of dequantized pieces (per coordinate lists); with
    `dict_ref` the dictionary section holds differences and dict_ref is added
    back."""
    if len(blob) < HEADER_BYTES:
        raise BitstreamError("truncated header")
    (magic, version, n, F, k, n_c, cb, db, ab, kind, hb, total) = struct.unpack_from(
        "<4sIIIIIBBBBIQ", blob, 0)
    if magic != MAGIC or version != VERSION or hb != HEADER_BYTES:
        raise BitstreamError("bad magic/version")
    if k < 1 or k > F or n_c > n or n < 1:
        raise BitstreamError("inconsistent sizes")
    if total != stream_size(n, F, k, n_c, cb, db, ab) or total != len(blob):
        raise BitstreamError("size mismatch")
    off = HEADER_BYTES
    anchors = np.frombuffer(blob, "<i4", n_c, off).astype(np.int32)
    off += _pad8(4 * n_c)
    if n_c and (anchors.min() < 0 or anchors.max() >= n or np.any(np.diff(anchors) <= 0)):
        raise BitstreamError("bad anchor indices")

    def section(count, bits, lo, hi):
        nonlocal off
        if bits == 0:
            v = np.frombuffer(blob, "<f8", count, off).copy()
            off += count * 8
            return v
        nw = quant.packed_words(count, bits)
        w = np.frombuffer(blob, "<u4", nw, off)
        off += _pad8(nw * 4)
        s = quant.unpack_bits(w, bits, count)
        return quant.dequantize(s, lo, hi, bits)

    res = {"n": n, "F": F, "k": k, "anchors": anchors, "kind": kind,
           "bits": (cb, db, ab), "U": [], "C": [], "a": []}
    for c in range(3):
        par = np.frombuffer(blob, "<f8", 4 * k + 2, off).copy()
        off += 8 * (4 * k + 2)
        d_lo, d_hi = par[0:k], par[k:2 * k]
        c_lo, c_hi = par[2 * k:3 * k], par[3 * k:4 * k]
        a_lo, a_hi = par[4 * k], par[4 * k + 1]
        Ut = section(F * k, db, np.repeat(d_lo, F), np.repeat(d_hi, F)).reshape(k, F)
        C = section(k * n, cb, np.repeat(c_lo, n), np.repeat(c_hi, n)).reshape(k, n)
        A = section(n_c * F, ab, a_lo, a_hi).reshape(n_c, F)
        res["U"].append(Ut.T if dict_ref is None else Ut.T + dict_ref[c])
        res["C"].append(C)
        res["a"].append(A)
    assert off == total
    return res


def normal_matrix(row_ptr, col_idx, deg, anchors, kind=0):
    n = row_ptr.shape[0] - 1
    L = graph.laplacian_matrix(row_ptr, col_idx, deg, kind)
    P = sp.csr_matrix((np.ones(anchors.shape[0]), (np.arange(anchors.shape[0]), anchors)),
                      shape=(anchors.shape[0], n))
    return (L.T @ L + P.T @ P).tocsc(), L, P


def normal_operator_ext(row_ptr, col_idx, deg, anchors, kind=0):
    """X -> (L^T L + P^T P) X applied as two Laplacian sweeps in extended
    precision (numpy longdouble), with the exact division by d_i of Eq. 3.

    Forming L^T L in binary64 perturbs the operator's smallest eigenvalues
    enough to move the least-squares solution by ~1e-10 relative; the
    unassembled operator in extended precision does not."""
    n = row_ptr.shape[0] - 1
    ext = np.longdouble
    rows = np.repeat(np.arange(n), np.diff(row_ptr.astype(np.int64)))
    C = sp.csr_matrix((np.ones(rows.shape[0], dtype=ext), (rows, col_idx.astype(np.int64))),
                      shape=(n, n))
    d = deg.astype(ext)[:, None]
    is_anchor = np.zeros(n, dtype=bool)
    is_anchor[anchors] = True

    def apply(X):
        X = np.asarray(X).astype(ext)
        if kind == 0:
            Y = X - (C @ X) / d
            Z = Y - C @ (Y / d)
        else:
            Y = d * X - C @ X
            Z = d * Y - C @ Y
        Z[is_anchor] += X[is_anchor]
        return Z

    return apply


def _refined_solve(lu, op_ext, b, max_steps=8):
    """Sparse LU as the approximate solver, then iterative refinement with
    residuals b - (L^T L + P^T P) X computed in extended precision, until the
    correction is below one unit in the last place of X."""
    X = lu.solve(b)
    b_ext = b.astype(np.longdouble)
    for _ in range(max_steps):
        r = (b_ext - op_ext(X)).astype(np.float64)
        dx = lu.solve(r)
        X = X + dx
        if np.abs(dx).max() <= 2.0 ** -52 * np.abs(X).max():
            break
    return X


def _factor(M):
    return spla.splu(M, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                     options={"SymmetricMode": True})


def check_anchor_coverage(row_ptr, col_idx, anchors):
    """Eq. 12 has a unique solution only when every connected component of
    the mesh holds an anchor; raises graph.AnchorCoverageError otherwise."""
    bad = graph.uncovered_components(row_ptr, col_idx, anchors)
    if bad.size:
        raise graph.AnchorCoverageError(
            f"{bad.size} connected component(s) without an anchor (first vertex {bad[0]})")


def solve_anchored_ls(row_ptr, col_idx, deg, anchors, delta_t, a_hat, kind=0):
    """X minimising ||L X - delta_t||^2 + ||P X - a_hat||^2 (Eq. 12), through
    the normal equations (L^T L + P^T P) X = L^T delta_t + P^T a_hat."""
    check_anchor_coverage(row_ptr, col_idx, anchors)
    M, L, P = normal_matrix(row_ptr, col_idx, deg, anchors, kind)
    b = graph.apply_laplacian_transpose(row_ptr, col_idx, deg, delta_t, kind)
    b[anchors] += a_hat
    op = normal_operator_ext(row_ptr, col_idx, deg, anchors, kind)
    X = _refined_solve(_factor(M), op, b)
    return X, b, M


def decode(blob, tris, dict_ref=None):
    d = parse(blob, dict_ref)
    n, F = d["n"], d["F"]
    row_ptr, col_idx, deg = graph.build_adjacency(tris, n)
    check_anchor_coverage(row_ptr, col_idx, d["anchors"])
    out = np.empty((F, n, 3), dtype=np.float64)
    M, L, P = normal_matrix(row_ptr, col_idx, deg, d["anchors"], d["kind"])
    lu = _factor(M)
    op = normal_operator_ext(row_ptr, col_idx, deg, d["anchors"], d["kind"])
    for c in range(3):
        delta_t = (d["U"][c] @ d["C"][c]).T                          # n x F (Eq. 11)
        b = graph.apply_laplacian_transpose(row_ptr, col_idx, deg, delta_t, d["kind"])
        b[d["anchors"]] += d["a"][c]
        out[:, :, c] = _refined_solve(lu, op, b).T
    return out
