"""Pins for the oracle's encoder/decoder (Eq. 7-12), bitstream and Eq. 13."""

import os

import numpy as np
import pytest

from oracle import codec, graph, metrics
from synth import icosphere, SequenceSpec, sinusoid_rigid_motion, make_sequence, config_spec

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tiny(level=1, F=16, seed=3):
    v, t = icosphere(level)
    spec = SequenceSpec(name="t", mesh=f"icosphere:{level}", n_frames=F, rank=4,
                        n_anchors=3, seed=seed)
    return t, sinusoid_rigid_motion(v, spec)


def test_full_rank_raw_codec_reconstructs_exactly():
    # k = F, raw coefficients / dictionary / anchors: Eq. 12 is consistent and
    # its least-squares solution is the input itself.
    tris, pos = _tiny(level=1, F=12)
    p = codec.Params(n_frames=12, rank=12, n_anchors=4, coeff_bits=0, dict_bits=0,
                     anchor_bits=0, oi_sweeps=200, seed=9)
    blob = codec.encode(tris, pos, p)
    rec = codec.decode(blob, tris)
    assert np.abs(rec - pos).max() < 1e-10


def test_anchored_ls_matches_dense_least_squares():
    tris, pos = _tiny(level=1)
    n = pos.shape[1]
    rp, ci, dg = graph.build_adjacency(tris, n)
    anchors = np.array([0, 7, 30], dtype=np.int32)
    r = np.random.default_rng(4)
    delta_t = r.normal(size=(n, 5))
    a_hat = r.normal(size=(3, 5))
    X, b, M = codec.solve_anchored_ls(rp, ci, dg, anchors, delta_t, a_hat)
    # dense stacked system of Eq. 12, solved by Householder least squares
    Ld = graph.laplacian_matrix(rp, ci, dg).toarray()
    Pd = np.eye(n)[anchors]
    Xd, *_ = np.linalg.lstsq(np.vstack([Ld, Pd]), np.vstack([delta_t, a_hat]), rcond=None)
    np.testing.assert_allclose(X, Xd, atol=1e-10)
    res = b - M @ X
    assert np.linalg.norm(res) <= 1e-13 * np.linalg.norm(b)


def test_factored_form_equals_the_frames_solve():
    # The decoder's factored form (Eq. 12 reassociated): with M = L^T L + P^T P,
    # M Y = L^T C'^T and M G = P^T, the frames solution is X = Y U'^T + G A^.
    tris, pos = _tiny(level=2, F=20)
    n = pos.shape[1]
    rp, ci, dg = graph.build_adjacency(tris, n)
    anchors = codec.select_anchors(n, 5, 2)
    r = np.random.default_rng(8)
    k, F = 4, 20
    U = np.linalg.qr(r.normal(size=(F, k)))[0]          # dictionary, F x k
    C = r.normal(size=(k, n))                            # coefficients
    A = r.normal(size=(anchors.size, F))                 # anchor trajectories
    X, _, M = codec.solve_anchored_ls(rp, ci, dg, anchors, (U @ C).T, A)
    Mf = M.toarray()
    Y = np.linalg.solve(Mf, graph.apply_laplacian_transpose(rp, ci, dg, C.T))
    Pt = np.zeros((n, anchors.size))
    Pt[anchors, np.arange(anchors.size)] = 1.0
    G = np.linalg.solve(Mf, Pt)
    np.testing.assert_allclose(Y @ U.T + G @ A, X, atol=1e-9 * np.abs(X).max())
    # M 1 = P^T 1 (L 1 = 0), so every row of the anchor response sums to one
    np.testing.assert_allclose(G.sum(axis=1), 1.0, atol=1e-9)


def test_consistent_system_returns_exact_solution():
    v, tris = icosphere(2)
    n = v.shape[0]
    rp, ci, dg = graph.build_adjacency(tris, n)
    anchors = codec.select_anchors(n, 6, 1)
    Xt = np.random.default_rng(5).normal(size=(n, 4))
    delta_t = graph.apply_laplacian(rp, ci, dg, Xt)
    X, _, _ = codec.solve_anchored_ls(rp, ci, dg, anchors, delta_t, Xt[anchors])
    assert np.abs(X - Xt).max() < 1e-10


def test_anchor_selection_uniform_seeded_sorted():
    a = codec.select_anchors(1000, 50, 17)
    assert a.shape == (50,) and np.all(np.diff(a) > 0) and a.min() >= 0 and a.max() < 1000
    np.testing.assert_array_equal(a, codec.select_anchors(1000, 50, 17))
    assert not np.array_equal(a, codec.select_anchors(1000, 50, 18))
    assert codec.select_anchors(10, 10, 3).tolist() == list(range(10))
    # roughly uniform over the index range
    hits = np.zeros(10)
    for s in range(200):
        np.add.at(hits, codec.select_anchors(1000, 10, s) // 100, 1)
    assert hits.min() > 120 and hits.max() < 280


def test_bitstream_roundtrip_and_size():
    tris, pos = _tiny(level=2, F=20)
    p = codec.Params(n_frames=20, rank=6, n_anchors=5, seed=2, oi_sweeps=20)
    blob, info = codec.encode(tris, pos, p, return_info=True)
    n = pos.shape[1]
    assert len(blob) == codec.stream_size(n, 20, 6, 5, 12, 16, 16)
    d = codec.parse(blob)
    assert d["n"] == n and d["F"] == 20 and d["k"] == 6
    np.testing.assert_array_equal(d["anchors"], info["anchors"])
    for c in range(3):
        # dequantized pieces within half a step of the encoder's values
        U = info["U"][c]
        step = (U.max(0) - U.min(0)) / 65535
        assert np.all(np.abs(d["U"][c] - U) <= step * 0.5 + 1e-15)
        C = info["C"][c]
        step = (C.max(1) - C.min(1)) / 4095
        assert np.all(np.abs(d["C"][c] - C) <= step[:, None] * 0.5 + 1e-15)


@pytest.mark.parametrize("mutate", ["magic", "truncate", "anchor_order", "size"])
def test_corrupt_bitstreams_rejected(mutate):
    tris, pos = _tiny(level=1, F=8)
    p = codec.Params(n_frames=8, rank=3, n_anchors=3, seed=2, oi_sweeps=5)
    blob = bytearray(codec.encode(tris, pos, p))
    if mutate == "magic":
        blob[0] = ord("X")
    elif mutate == "truncate":
        blob = blob[:-8]
    elif mutate == "anchor_order":
        blob[64:68], blob[68:72] = blob[68:72], blob[64:68]
    else:
        blob[32] ^= 0xFF
    with pytest.raises(codec.BitstreamError):
        codec.parse(bytes(blob))


def test_nmse_definition():
    a = np.zeros((2, 3, 3))
    a[:, 1, 0] = 1.0
    a[:, 2, 1] = 2.0
    # centred energy per frame: centroid (1/3, 2/3, 0)
    cen = a - a.mean(axis=1, keepdims=True)
    S = np.sum(cen ** 2)
    b = a.copy()
    b[0, 0, 2] += 0.1
    assert metrics.nmse(a, b) == pytest.approx(0.01 / S, rel=1e-14)
    assert metrics.nmse(a, a) == 0.0


def test_eq13_reproduces_table1():
    rows = {}
    with open(os.path.join(GOLDEN, "table1_rates.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            rows[parts[0]] = [float(x) for x in parts[1:]]
    for model in ("Handstand", "Samba"):
        n, F, q_d, q_a, q, q_s = rows[model]
        r = metrics.rates(int(n), int(F), 1, round(0.01 * n), 0, 16, 16)
        assert round(r["q_d"], 4) == q_d
    n, F, q_d, q_a, q, q_s = rows["Handstand"]
    r = metrics.rates(int(n), int(F), 1, round(0.01 * n), 0, 16, 16)
    assert round(r["q_a"], 4) == q_a
    assert round(q + q_a + q_d, 4) == q_s
    for col in ("PCA", "PCA+q", "v2v", "blocks"):
        q, q_a, q_d, q_s = rows[col]
        assert round(q + q_a + q_d, 4) == q_s


@pytest.mark.slow
def test_small_config_error_is_small():
    spec = config_spec("icosphere4_F64_k16")
    tris, pos = make_sequence(spec)
    p = codec.Params(n_frames=spec.n_frames, rank=spec.rank, n_anchors=spec.n_anchors,
                     seed=spec.seed)
    rec = codec.decode(codec.encode(tris, pos, p), tris)
    assert metrics.nmse(pos, rec) < 1e-3
