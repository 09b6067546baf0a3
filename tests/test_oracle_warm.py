"""Pins of the warm-start inputs (oracle/warm.py): nearest anchors of
hand-made point sets and one feature row written out by hand."""

import numpy as np

from oracle import warm


def _line(m):
    p = np.zeros((m, 3))
    p[:, 0] = np.arange(m)
    return p


def test_nearest_anchors_ties_by_index():
    rest = _line(5)
    anchors = np.array([4, 0, 2])
    idx, dist = warm.nearest_anchors(rest, anchors)
    # vertex 1: anchor 1 (vertex 0) and anchor 2 (vertex 2) both at 1, then anchor 0 at 3
    np.testing.assert_array_equal(idx[1], [1, 2, 0])
    np.testing.assert_array_equal(dist[1], [1, 1, 3])
    # vertex 3: anchor 0 (vertex 4) and anchor 2 (vertex 2) at 1, anchor 1 at 3
    np.testing.assert_array_equal(idx[3], [0, 2, 1])
    # anchors are their own nearest at distance 0
    np.testing.assert_array_equal(idx[4][:1], [0])
    assert dist[4][0] == 0.0


def test_nearest_anchors_fewer_than_three():
    rest = _line(4)
    idx, dist = warm.nearest_anchors(rest, np.array([2]))
    np.testing.assert_array_equal(idx, np.zeros((4, 3), dtype=np.int32))
    np.testing.assert_array_equal(dist[0], [2, 2, 2])
    idx, dist = warm.nearest_anchors(rest, np.array([3, 0]))
    np.testing.assert_array_equal(idx[1], [1, 0, 0])
    np.testing.assert_array_equal(dist[1], [1, 2, 2])


def test_nearest_anchors_3d_distance():
    rest = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0], [1.0, 2.0, 2.0], [0.0, 0.0, 1.0]])
    idx, dist = warm.nearest_anchors(rest, np.array([1, 2, 3]))
    np.testing.assert_array_equal(idx[0], [2, 1, 0])       # distances 1, 3, 5
    np.testing.assert_array_equal(dist[0], [1, 3, 5])


def test_feature_row_by_hand():
    n, F = 2, 2
    anchors = np.array([1])
    nearest = np.zeros((n, 3), dtype=np.int32)
    dist = np.array([[0.5, 0.5, 0.5], [0.0, 0.0, 0.0]], dtype=np.float32)
    x_last = np.array([[0.0, 1.0, 2.0], [10.0, 20.0, 30.0]])
    a_cur = np.zeros((3, 1, F))
    a_cur[:, 0, 1] = [11.0, 22.0, 33.0]           # anchor (vertex 1) at frame 1
    delta_cur = np.arange(n * 3 * F, dtype=np.float64).reshape(n, 3 * F)
    delta_prev = np.zeros((n, 3 * F))
    delta_prev[0, [1, 3, 5]] = 1.0                 # last frame (column c*F + F-1) of vertex 0
    x_cur = np.zeros((F, n, 3))
    x_cur[1, 0] = [0.5, 1.5, 2.5]
    feat, tgt = warm.features(x_last, a_cur, anchors, nearest, dist, delta_cur, delta_prev,
                              dscale=2.0, x_cur=x_cur)
    # sample e = f*n + v = 2 (frame 1, vertex 0): anchor displacement (1, 2, 3) three
    # times with distance 0.5; delta columns c*F + 1 = 1, 3, 5 minus 1, times 2
    want = [1, 2, 3, 0.5] * 3 + [0.0, 4.0, 8.0, 1.0]
    np.testing.assert_array_equal(feat[2], np.array(want, dtype=np.float32))
    np.testing.assert_array_equal(tgt[2], [0.5, 0.5, 0.5])
    # frame 0: position feature (0 + 1) / 2
    assert feat[0, 15] == np.float32(0.5)


def test_compose():
    x_last = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0]])
    pred = np.arange(12, dtype=np.float32).reshape(4, 3)
    x0 = warm.compose(x_last, 2, pred)
    np.testing.assert_array_equal(x0[1, 0], [1 + 6, 2 + 7, 3 + 8])
    np.testing.assert_array_equal(warm.compose(x_last, 2)[1], x_last)


def test_basis_features_and_compose():
    F, k = 2, 3
    U_prev = np.arange(3 * F * k, dtype=np.float64).reshape(3, F, k)
    U_cur = U_prev + 0.5
    feat, tgt = warm.basis_features(U_prev, U_cur)
    # row r = c*F + f: c = 1, f = 1 is row 3 = U_prev[1, 1] = (9, 10, 11), then (1 + 1) / 2
    np.testing.assert_array_equal(feat[3], [9, 10, 11, 1.0])
    np.testing.assert_array_equal(feat[2], [6, 7, 8, 0.5])
    np.testing.assert_array_equal(tgt, np.full((6, 3), 0.5, dtype=np.float32))
    q0 = warm.basis_compose(U_prev, tgt)
    np.testing.assert_array_equal(q0, U_cur)


def test_sample_rows_uses_splitmix64_outputs():
    X = np.arange(20, dtype=np.float32).reshape(10, 2)
    # splitmix64 with seed 0: first outputs from the published table, modulo 10
    out = warm.sample_rows(X, 0, 3)
    want_rows = [0xE220A8397B1DCDAF % 10, 0x6E789E6AA1B965F4 % 10, 0x06C45D188009454F % 10]
    np.testing.assert_array_equal(out, X[want_rows])
