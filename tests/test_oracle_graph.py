"""Pins for the oracle's graph and Laplacian (Section II, Eq. 1-4)."""

import numpy as np
import pytest

from oracle import graph
from oracle.graph import MeshError
from synth import icosphere, torus_grid, open_grid


def _euler_edges(n_vertices, n_tris, boundary_edges=0):
    # closed surface: 3T = 2E; with b boundary edges: 3T = 2E - b
    return (3 * n_tris + boundary_edges) // 2


@pytest.mark.parametrize("mesh,expected_nnzL", [
    ("icosphere4", 17922),
    ("torus200x100", 140000),
    ("grid316", 696466),
    ("grid512", 1830914),
])
def test_nnz_matches_euler(mesh, expected_nnzL):
    if mesh == "icosphere4":
        v, t = icosphere(4)
        E = _euler_edges(v.shape[0], t.shape[0])
    elif mesh == "torus200x100":
        v, t = torus_grid(200, 100)
        E = _euler_edges(v.shape[0], t.shape[0])
    else:
        a = int(mesh[4:])
        v, t = open_grid(a, a)
        E = _euler_edges(v.shape[0], t.shape[0], boundary_edges=4 * (a - 1))
    n = v.shape[0]
    rp, ci, dg = graph.build_adjacency(t, n)
    assert rp[-1] == 2 * E
    assert n + rp[-1] == expected_nnzL


def test_pattern_symmetric_sorted_and_degrees():
    v, t = icosphere(4)
    n = v.shape[0]
    rp, ci, dg = graph.build_adjacency(t, n)
    rows = np.repeat(np.arange(n), np.diff(rp))
    pairs = set(zip(rows.tolist(), ci.tolist()))
    assert all((j, i) in pairs for (i, j) in pairs)
    assert all(i != j for (i, j) in pairs)
    for i in range(n):
        seg = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(seg) > 0)
    assert np.sum(dg == 5) == 12 and np.sum(dg == 6) == n - 12

    v, t = torus_grid(20, 10)
    rp, ci, dg = graph.build_adjacency(t, v.shape[0])
    assert np.all(dg == 6)

    v, t = open_grid(5, 7)
    rp, ci, dg = graph.build_adjacency(t, v.shape[0])
    # corners of the split-quad grid have degree 2 or 3, other border
    # vertices 3 or 4, interior vertices 6
    interior = [i * 7 + j for i in range(1, 4) for j in range(1, 6)]
    assert np.all(dg[interior] == 6)
    assert sorted(dg[[0, 6, 28, 34]].tolist()) == [2, 2, 3, 3]


def _dense_laplacian_by_loops(tris, n, kind):
    """Eq. 1-2 written out with Python loops over triangles."""
    C = np.zeros((n, n))
    for a, b, c in tris:
        for i, j in ((a, b), (b, c), (c, a)):
            C[i, j] = 1.0
            C[j, i] = 1.0
    d = C.sum(1)
    if kind == 1:
        return np.diag(d) - C
    return np.eye(n) - C / d[:, None]


@pytest.mark.parametrize("kind", [0, 1])
def test_laplacian_matches_dense_definition(kind):
    v, t = icosphere(1)
    n = v.shape[0]
    rp, ci, dg = graph.build_adjacency(t, n)
    Ld = _dense_laplacian_by_loops(t.tolist(), n, kind)
    X = np.random.default_rng(3).normal(size=(n, 7))
    np.testing.assert_allclose(graph.apply_laplacian(rp, ci, dg, X, kind), Ld @ X,
                               rtol=0, atol=1e-13)
    np.testing.assert_allclose(graph.apply_laplacian_transpose(rp, ci, dg, X, kind),
                               Ld.T @ X, rtol=0, atol=1e-13)
    np.testing.assert_allclose(graph.laplacian_matrix(rp, ci, dg, kind).toarray(), Ld,
                               rtol=0, atol=1e-15)


def test_rows_sum_to_zero_exactly():
    for v, t in (icosphere(3), torus_grid(30, 12), open_grid(9, 4)):
        n = v.shape[0]
        rp, ci, dg = graph.build_adjacency(t, n)
        ones = np.ones((n, 3))
        assert np.all(graph.apply_laplacian(rp, ci, dg, ones, 0) == 0.0)
        assert np.all(graph.apply_laplacian(rp, ci, dg, ones, 1) == 0.0)
        assert np.all(graph.apply_laplacian(rp, ci, dg, 3.25 * ones, 0) == 0.0)


def test_random_walk_delta_is_vertex_minus_neighbour_mean():
    # Eq. 3 on a planar grid: interior vertices of a uniform grid have a
    # symmetric 1-ring, so delta = 0 for the flat base positions.
    v, t = open_grid(6, 6)
    rp, ci, dg = graph.build_adjacency(t, v.shape[0])
    delta = graph.apply_laplacian(rp, ci, dg, v, 0)
    interior = [i * 6 + j for i in range(1, 5) for j in range(1, 5)]
    np.testing.assert_allclose(delta[interior], 0.0, atol=1e-15)


@pytest.mark.parametrize("tris,n,msg", [
    ([[0, 1, 5]], 3, "out of range"),
    ([[0, 1, -1]], 3, "out of range"),
    ([[0, 1, 1]], 3, "degenerate"),
    ([[0, 1, 2]], 4, "isolated"),
])
def test_rejects_invalid_meshes(tris, n, msg):
    with pytest.raises(MeshError, match=msg):
        graph.build_adjacency(np.array(tris, dtype=np.int32), n)


# ---------------------------------------------------------------- components
def test_components_of_a_disjoint_union_are_its_pieces():
    from synth import disjoint_union
    pieces = [icosphere(1), torus_grid(6, 4), icosphere(0), open_grid(3, 5)]
    v, t = disjoint_union(pieces)
    rp, ci, _ = graph.build_adjacency(t, v.shape[0])
    lab = graph.components(rp, ci)
    expect, base = [], 0
    for pv, _ in pieces:
        expect += [base] * pv.shape[0]
        base += pv.shape[0]
    np.testing.assert_array_equal(lab, np.array(expect))


def test_components_match_the_null_space_of_L_and_csgraph():
    # a shuffled disjoint union: each label is the smallest index of its
    # piece, the partition equals scipy's connected components, and each
    # component's indicator vector spans the null space of L (L 1 = 0 per
    # component, Eq. 3): dim null(L) = number of components
    from scipy.sparse.csgraph import connected_components
    from synth import disjoint_union
    v, t = disjoint_union([icosphere(1), torus_grid(5, 3), open_grid(4, 4)])
    n = v.shape[0]
    perm = np.random.default_rng(3).permutation(n)
    t = perm[t].astype(np.int32)
    rp, ci, dg = graph.build_adjacency(t, n)
    lab = graph.components(rp, ci)
    A = graph.laplacian_matrix(rp, ci, dg) != 0
    ncomp, ref = connected_components(A, directed=False)
    assert len(np.unique(lab)) == ncomp == 3
    for c in range(ncomp):
        members = np.nonzero(ref == c)[0]
        assert np.all(lab[members] == members.min())
    L = graph.laplacian_matrix(rp, ci, dg).toarray()
    sv = np.linalg.svd(L, compute_uv=False)
    assert np.sum(sv < 1e-10 * sv.max()) == ncomp
    for root in np.unique(lab):
        ind = (lab == root).astype(np.float64)[:, None]
        assert np.all(graph.apply_laplacian(rp, ci, dg, ind) == 0.0)


def test_uncovered_components_and_the_decoder_check():
    from oracle import codec
    from oracle.graph import AnchorCoverageError
    from synth import disjoint_union
    a, b = icosphere(1), icosphere(1)
    v, t = disjoint_union([a, b], offsets=[(0, 0, 0), (3, 0, 0)])
    rp, ci, _ = graph.build_adjacency(t, v.shape[0])
    n1 = a[0].shape[0]
    np.testing.assert_array_equal(graph.uncovered_components(rp, ci, [0, 5]), [n1])
    np.testing.assert_array_equal(graph.uncovered_components(rp, ci, []), [0, n1])
    assert graph.uncovered_components(rp, ci, [3, n1 + 1]).size == 0
    F = 6
    pos = np.repeat(v[None], F, 0) + 0.01 * np.arange(F)[:, None, None]
    p = codec.Params(n_frames=F, rank=2, n_anchors=2)
    blob = codec.encode(t, pos, p, anchors=np.array([3, n1 + 1], dtype=np.int32))
    codec.decode(blob, t)
    bad = codec.encode(t, pos, p, anchors=np.array([3, 7], dtype=np.int32))
    with pytest.raises(AnchorCoverageError):
        codec.decode(bad, t)
