"""Parity of the CUDA codec (through the C ABI) with the FP64 oracle.

Bars (FP64 mode):
* connectivity, degrees, anchors, delta coordinates: bit-exact;
* quantized symbols: equal except at rounding ties: at most 1e-6 of the
  symbols differ, each by exactly 1, and only where the oracle's
  t = (x - lo) * scale lies within TIE_WINDOW of a .5 boundary;
* reconstruction NMSE within 1e-9 relative of the oracle's.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import codec as oc, graph as og, metrics, quant as oq, subspace as osub  # noqa: E402
from synth import SequenceSpec, make_sequence, config_spec, icosphere, torus_grid, open_grid  # noqa: E402

pytestmark = pytest.mark.gpu

TIE_WINDOW = 1e-6   # |t - (m + 0.5)| below which a one-off symbol counts as a tie
NMSE_RTOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_10105_gb300 import build
    build.build()


def _codec(tris, n, **kw):
    from paper_2111_10105_gb300 import MeshCodec
    return MeshCodec(tris, n, **kw)


def _oracle_params(spec, **kw):
    d = dict(n_frames=spec.n_frames, rank=spec.rank, n_anchors=spec.n_anchors, seed=spec.seed,
             coeff_bits=spec.coeff_bits, dict_bits=spec.dict_bits, anchor_bits=spec.anchor_bits)
    d.update(kw)
    return oc.Params(**d)


def _gpu_kw(p):
    return dict(n_frames=p.n_frames, rank=p.rank, n_anchors=p.n_anchors, seed=p.seed,
                coeff_bits=p.coeff_bits, dict_bits=p.dict_bits, anchor_bits=p.anchor_bits,
                laplacian_kind=p.laplacian_kind, oi_sweeps=p.oi_sweeps)


# ------------------------------------------------------------------ graph
@pytest.mark.parametrize("mesh", ["icosphere:4", "torus:40:25", "grid:37:23", "icosphere:0"])
def test_csr_and_degrees_bit_exact(mesh):
    from paper_2111_10105_gb300 import codec as cb
    from synth.motion import base_mesh
    v, t = base_mesh(mesh)
    n = v.shape[0]
    rp, ci, dg = og.build_adjacency(t, n)
    with _codec(t, n, n_frames=4, rank=2, n_anchors=3) as mc:
        np.testing.assert_array_equal(mc.buffer(cb.BUF_ROW_PTR).cpu().numpy(), rp)
        np.testing.assert_array_equal(mc.buffer(cb.BUF_COL_IDX).cpu().numpy(), ci)
        np.testing.assert_array_equal(mc.buffer(cb.BUF_DEGREE).cpu().numpy(), dg)


def test_csr_from_shuffled_and_duplicated_triangles():
    from paper_2111_10105_gb300 import codec as cb
    v, t = torus_grid(30, 11)
    r = np.random.default_rng(0)
    t2 = np.concatenate([t, t[:50][:, ::-1]])[r.permutation(t.shape[0] + 50)]
    rp, ci, dg = og.build_adjacency(t2, v.shape[0])
    with _codec(t2, v.shape[0], n_frames=3, rank=1, n_anchors=1) as mc:
        np.testing.assert_array_equal(mc.buffer(cb.BUF_COL_IDX).cpu().numpy(), ci)


@pytest.mark.parametrize("tris,n,status", [
    ([[0, 1, 5]], 4, "MC_E_BAD_MESH"),
    ([[0, 1, -2], [0, 1, 2]], 3, "MC_E_BAD_MESH"),
    ([[0, 2, 2], [0, 1, 2]], 3, "MC_E_BAD_MESH"),
    ([[0, 1, 2]], 4, "MC_E_ISOLATED_VERTEX"),
])
def test_invalid_meshes_rejected(tris, n, status):
    from paper_2111_10105_gb300 import MeshCodecError
    with pytest.raises(MeshCodecError) as e:
        _codec(np.array(tris, dtype=np.int32), n, n_frames=2, rank=1, n_anchors=1)
    assert e.value.name == status


@pytest.mark.parametrize("n,n_c,seed", [(2562, 20, 1000), (20000, 50, 1001), (1000, 1000, 3),
                                        (99856, 999, 1002), (7, 1, 0), (513, 257, 99)])
def test_anchor_selection_bit_exact(n, n_c, seed):
    from paper_2111_10105_gb300 import codec as cb
    i = np.arange(n - 2)
    t = np.stack([i, i + 1, i + 2], 1).astype(np.int32)      # a triangle strip
    with _codec(t, n, n_frames=2, rank=1, n_anchors=n_c, seed=seed) as mc:
        got = mc.buffer(cb.BUF_ANCHORS).cpu().numpy()
    np.testing.assert_array_equal(got, oc.select_anchors(n, n_c, seed))


def test_caller_anchors_validated():
    from paper_2111_10105_gb300 import MeshCodecError, codec as cb
    v, t = icosphere(2)
    n = v.shape[0]
    with _codec(t, n, n_frames=4, rank=2, n_anchors=3, anchors=[1, 5, 100]) as mc:
        assert mc.buffer(cb.BUF_ANCHORS).cpu().tolist() == [1, 5, 100]
    for bad in ([5, 1, 100], [1, 1, 2], [1, 2, n]):
        with pytest.raises(MeshCodecError) as e:
            _codec(t, n, n_frames=4, rank=2, n_anchors=3, anchors=bad)
        assert e.value.name == "MC_E_BAD_ANCHORS"


# ------------------------------------------------------------------ encoder
def _seq(level=3, F=37, k=5, n_c=11, seed=5, **kw):
    spec = SequenceSpec(name="t", mesh=f"icosphere:{level}", n_frames=F, rank=k, n_anchors=n_c,
                        seed=seed, **kw)
    tris, pos = make_sequence(spec)
    return spec, tris, pos


@pytest.mark.parametrize("kind", [0, 1])
def test_delta_coordinates_bit_exact(kind):
    from paper_2111_10105_gb300 import codec as cb
    spec, tris, pos = _seq(level=3, F=37)
    n, F = pos.shape[1], pos.shape[0]
    rp, ci, dg = og.build_adjacency(tris, n)
    X = pos.transpose(1, 2, 0).reshape(n, 3 * F)
    want = og.apply_laplacian(rp, ci, dg, X, kind)
    with _codec(tris, n, n_frames=F, rank=3, n_anchors=5, laplacian_kind=kind, oi_sweeps=1) as mc:
        mc.encode(torch.from_numpy(pos).cuda())
        got = mc.buffer(cb.BUF_DELTA).cpu().numpy().reshape(n, 3 * F)
    assert np.array_equal(got, want)


def test_start_basis_matches_oracle():
    from paper_2111_10105_gb300 import codec as cb
    spec, tris, pos = _seq(level=2, F=40, k=7)
    with _codec(tris, pos.shape[1], n_frames=40, rank=7, n_anchors=4, seed=123) as mc:
        Q0 = mc.buffer(cb.BUF_START).cpu().numpy().reshape(3, 40, 7)
    for c in range(3):
        np.testing.assert_allclose(Q0[c], osub.start_basis(40, 7, 123, c), atol=1e-13)


def _tie_distance(x, lo, hi, bits):
    levels = float((1 << bits) - 1)
    rng = hi - lo
    scale = np.where(rng > 0, levels / np.where(rng > 0, rng, 1.0), 0.0)
    t = (x - lo) * scale
    return np.abs(t - (np.floor(t) + 0.5))


def _raw_sections(blob):
    """Per coordinate: the f64 range block and the raw symbols of the three
    sections, read straight from the stream (layout of oracle.codec)."""
    hdr = np.frombuffer(blob, "<u4", 6, 0)
    n, F, k, n_c = int(hdr[2]), int(hdr[3]), int(hdr[4]), int(hdr[5])
    cb_, db_, ab_ = blob[24], blob[25], blob[26]
    off = 64 + ((4 * n_c + 7) // 8) * 8
    out = []
    for c in range(3):
        par = np.frombuffer(blob, "<f8", 4 * k + 2, off).copy()
        off += 8 * (4 * k + 2)
        secs = []
        for count, bits in ((F * k, db_), (k * n, cb_), (n_c * F, ab_)):
            if bits == 0:
                secs.append(np.frombuffer(blob, "<f8", count, off).copy())
                off += 8 * count
            else:
                nw = oq.packed_words(count, bits)
                secs.append(oq.unpack_bits(np.frombuffer(blob, "<u4", nw, off), bits, count))
                off += oc._pad8(4 * nw)
        out.append((par, secs))
    assert off == len(blob)
    return out


def _check_bitstreams(g, o, info, p, n):
    """GPU stream g against the oracle stream o: identical header and anchor
    indices, anchor symbols bit-exact, coefficient and dictionary symbols
    equal except one-off ties.  Returns (mismatches, symbols compared)."""
    assert len(g) == len(o)
    assert g[:64] == o[:64]
    n_c = p.n_anchors
    assert g[64:64 + 4 * n_c] == o[64:64 + 4 * n_c]
    k = p.rank
    sg, so = _raw_sections(g), _raw_sections(o)
    mism = total = 0
    for c in range(3):
        (pg, (dg_, cg_, ag_)), (po, (do_, co_, ao_)) = sg[c], so[c]
        np.testing.assert_allclose(pg, po, rtol=1e-9, atol=1e-12 * np.abs(po).max())
        np.testing.assert_array_equal(pg[4 * k:], po[4 * k:])      # anchor range: exact
        np.testing.assert_array_equal(ag_, ao_)                    # anchor symbols: exact
        checks = [(cg_, co_, info["C"][c], po[2 * k:3 * k], po[3 * k:4 * k], p.coeff_bits)]
        checks.append((dg_, do_, info["U"][c].T, po[0:k], po[k:2 * k], p.dict_bits))
        for got, want, x, lo, hi, bits in checks:
            if bits == 0:
                continue
            got = got.reshape(x.shape)
            want = want.reshape(x.shape)
            bad = got != want
            total += want.size
            mism += int(bad.sum())
            if bad.any():
                assert np.all(np.abs(got[bad] - want[bad]) == 1)
                dist = _tie_distance(x, lo[:, None], hi[:, None], bits)[bad]
                assert np.all(dist < TIE_WINDOW), dist.max()
    return mism, total


@pytest.mark.parametrize("level,F,k,n_c,sweeps", [(3, 37, 5, 11, 25), (4, 64, 16, 20, 30),
                                                  (2, 9, 9, 3, 40)])
def test_encoder_parity(level, F, k, n_c, sweeps):
    from paper_2111_10105_gb300 import codec as cb
    spec, tris, pos = _seq(level=level, F=F, k=k, n_c=n_c, seed=1000 + level)
    p = _oracle_params(spec, oi_sweeps=sweeps)
    o, info = oc.encode(tris, pos, p, return_info=True)
    n = pos.shape[1]
    with _codec(tris, n, **_gpu_kw(p)) as mc:
        g = bytes(mc.encode(torch.from_numpy(pos).cuda()).cpu().numpy().tobytes())
        U = mc.buffer(cb.BUF_BASIS).cpu().numpy().reshape(3, F, k)
        th = mc.buffer(cb.BUF_RITZ).cpu().numpy().reshape(3, k)
        C = mc.buffer(cb.BUF_COEFF).cpu().numpy().reshape(3, k, n)
    assert len(g) == len(o)
    for c in range(3):
        np.testing.assert_allclose(th[c], info["theta"][c], rtol=1e-10,
                                   atol=1e-13 * info["theta"][c][0])
        np.testing.assert_allclose(U[c], info["U"][c], atol=1e-9)
        scale = np.abs(info["C"][c]).max(axis=1, keepdims=True)
        np.testing.assert_allclose(C[c], info["C"][c], atol=1e-9 * scale.max())
    mism, total = _check_bitstreams(g, o, info, p, n)
    assert mism <= max(1, int(1e-6 * total))


def test_full_rank_raw_roundtrip():
    spec, tris, pos = _seq(level=2, F=12, k=12, n_c=6)
    n = pos.shape[1]
    with _codec(tris, n, n_frames=12, rank=12, n_anchors=6, seed=9, coeff_bits=0, dict_bits=0,
                anchor_bits=0, oi_sweeps=200) as mc:
        bits = mc.encode(torch.from_numpy(pos).cuda())
        rec = mc.decode(bits).cpu().numpy()
    assert np.abs(rec - pos).max() < 1e-9


# ------------------------------------------------------------------ decoder
@pytest.mark.parametrize("level,F,k,n_c,mode", [(3, 37, 5, 11, 0), (4, 64, 16, 20, 0),
                                                (3, 37, 5, 11, 1), (4, 64, 16, 20, 1),
                                                (4, 64, 16, 20, 2)])
def test_decoder_nmse_parity(level, F, k, n_c, mode):
    spec, tris, pos = _seq(level=level, F=F, k=k, n_c=n_c, seed=2000 + level)
    p = _oracle_params(spec, oi_sweeps=30)
    o = oc.encode(tris, pos, p)
    rec_o = oc.decode(o, tris)
    n = pos.shape[1]
    with _codec(tris, n, solve_mode=mode, **_gpu_kw(p)) as mc:
        # decode the oracle's own stream: isolates the decoder
        ot = torch.from_numpy(np.frombuffer(o, dtype=np.uint8).copy()).cuda()
        rec_g = mc.decode(ot).cpu().numpy()
        st = mc.stats()
        # and the GPU's stream
        gb = mc.encode(torch.from_numpy(pos).cuda())
        rec_gg = mc.decode(gb).cpu().numpy()
    e_o = metrics.nmse(pos, rec_o)
    assert st["cg_not_converged"] == 0
    assert abs(metrics.nmse(pos, rec_g) - e_o) <= NMSE_RTOL * e_o
    assert abs(metrics.nmse(pos, rec_gg) - e_o) <= NMSE_RTOL * e_o
    assert np.abs(rec_g - rec_o).max() <= 1e-9 * np.abs(pos).max()


def test_host_entry_points_match_device():
    spec, tris, pos = _seq(level=2, F=16, k=4, n_c=5)
    n = pos.shape[1]
    with _codec(tris, n, n_frames=16, rank=4, n_anchors=5, seed=1) as mc:
        gd = mc.encode(torch.from_numpy(pos).cuda()).cpu().numpy()
        gh = mc.encode_host(np.ascontiguousarray(pos))
        assert np.array_equal(gd, gh)
        rd = mc.decode(torch.from_numpy(gd).cuda()).cpu().numpy()
        rh = mc.decode_host(gh)
        assert np.array_equal(rd, rh)


def test_corrupt_and_short_buffers():
    from paper_2111_10105_gb300 import MeshCodecError
    spec, tris, pos = _seq(level=2, F=8, k=3, n_c=4)
    n = pos.shape[1]
    with _codec(tris, n, n_frames=8, rank=3, n_anchors=4, seed=2) as mc:
        bits = mc.encode(torch.from_numpy(pos).cuda())
        with pytest.raises(MeshCodecError) as e:
            mc.encode(torch.from_numpy(pos).cuda(), out=torch.empty(10, dtype=torch.uint8,
                                                                    device="cuda"))
        assert e.value.name == "MC_E_BUFFER_TOO_SMALL"
        bad = bits.clone()
        bad[0] = 0
        with pytest.raises(MeshCodecError) as e:
            mc.decode(bad)
        assert e.value.name == "MC_E_BITSTREAM_CORRUPT"
        bad = bits.clone()
        # swap two anchor indices: not increasing any more
        a = bad[64:68].clone()
        bad[64:68] = bad[68:72]
        bad[68:72] = a
        with pytest.raises(MeshCodecError) as e:
            mc.decode(bad)
        assert e.value.name == "MC_E_BITSTREAM_CORRUPT"
        with pytest.raises(MeshCodecError) as e:
            mc.decode(bits[:-8])
        assert e.value.name == "MC_E_BITSTREAM_CORRUPT"


def test_cg_cap_reports_not_converged():
    spec, tris, pos = _seq(level=3, F=8, k=3, n_c=4)
    n = pos.shape[1]
    with _codec(tris, n, n_frames=8, rank=3, n_anchors=4, seed=2, cg_max_iters=5) as mc:
        bits = mc.encode(torch.from_numpy(pos).cuda())
        from paper_2111_10105_gb300 import MeshCodecError
        with pytest.raises(MeshCodecError) as e:
            mc.decode(bits)
        assert e.value.name == "MC_E_NOT_CONVERGED"
        st = mc.stats()
        assert st["cg_iters_max"] == 5 and st["cg_not_converged"] > 0


# ------------------------------------------------------------------ full size
@pytest.mark.slow
@pytest.mark.parametrize("mode", [0, 1])
def test_mid_config_parity_full_size(mode):
    """The 20 000-vertex torus sequence (F = 256, k = 32, 50 anchors) in the
    configuration the benchmark times."""
    spec = config_spec("torus200x100_F256_k32")
    tris, pos = make_sequence(spec)
    p = _oracle_params(spec, oi_sweeps=30)
    o, info = oc.encode(tris, pos, p, return_info=True)
    n = pos.shape[1]
    with _codec(tris, n, solve_mode=mode, **_gpu_kw(p)) as mc:
        pt = torch.from_numpy(pos).cuda()
        g = mc.encode(pt)
        gb = bytes(g.cpu().numpy().tobytes())
        rec_g = mc.decode(g).cpu().numpy()
        st = mc.stats()
    mism, total = _check_bitstreams(gb, o, info, p, n)
    assert mism <= max(1, int(1e-6 * total))
    rec_o = oc.decode(o, tris)
    e_o = metrics.nmse(pos, rec_o)
    assert st["cg_not_converged"] == 0
    assert abs(metrics.nmse(pos, rec_g) - e_o) <= NMSE_RTOL * e_o
