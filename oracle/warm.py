"""Reference of the decoder warm start's inputs.

Test infrastructure (see ``oracle/__init__``).  The paper decodes every
segment from scratch; the warm start only supplies the first iterate of the
CG solve of Eq. 12, which does not change the solution.

``nearest_anchors``: the WARM_ANCHORS anchors nearest to each vertex of the
rest pose (squared Euclidean distance as the sum of the three rounded
squares in coordinate order, nearest first, equal distances by the lower
anchor index; with fewer anchors the last one found repeats).

``features``: for sample e = f*n + v of segment s (vertex v, frame f),
WARM_FEATURES float32 values:
  [4j .. 4j+2]  a_cur(a_j, f) - x_last(anchors[a_j])   (j = 0, 1, 2)
  [4j + 3]      the rest-pose distance to a_j
  [12 .. 14]    (delta_cur(v, f) - delta_prev(v, F-1)) * dscale
  [15]          (f + 1) / F (in float32)
where x_last is the last decoded frame of segment s-1, a_cur the
dequantized anchor positions of segment s and delta_cur, delta_prev the
back-projected delta coordinates of segments s and s-1 (Eq. 10-11).  Each
difference is taken in float64 and rounded once to float32.  Targets:
x_cur(v, f) - x_last(v).

``compose``: x0(f, v) = x_last(v) + prediction(f*n + v).

``basis_features`` / ``basis_compose``: the start-basis head.  Row
r = c*F + f of the previous dictionary U_prev [3, F, k] gives the features
[U_prev(c, f, :), (f + 1) / F] and the target U_cur - U_prev; the start is
U_prev + prediction.

``sample_rows``: minibatch rows r_i = splitmix64(seed) output i mod N.

Parity pinned by brute force in tests/test_oracle_warm.py (distances of a
hand-made point set, ties, the fewer-anchors rule, one feature row written
out by hand).
"""

import numpy as np

from . import rng

WARM_ANCHORS = 3
WARM_FEATURES = 16


def nearest_anchors(rest, anchors):
    rest = np.asarray(rest, dtype=np.float64)
    anchors = np.asarray(anchors, dtype=np.int64)
    n = rest.shape[0]
    idx = np.zeros((n, WARM_ANCHORS), dtype=np.int32)
    dist = np.zeros((n, WARM_ANCHORS), dtype=np.float32)
    for v in range(n):
        t = rest[v][None, :] - rest[anchors]
        d2 = (t[:, 0] * t[:, 0] + t[:, 1] * t[:, 1]) + t[:, 2] * t[:, 2]
        order = np.lexsort((np.arange(len(anchors)), d2))   # by distance, then index
        take = list(order[:WARM_ANCHORS])
        while len(take) < WARM_ANCHORS:
            take.append(take[-1])
        idx[v] = take
        dist[v] = np.sqrt(d2[take]).astype(np.float32)
    return idx, dist


def features(x_last, a_cur, anchors, nearest, dist, delta_cur, delta_prev, dscale=1.0,
             x_cur=None):
    """x_last [n, 3]; a_cur [3, n_c, F]; delta_cur, delta_prev [n, 3F]
    (column c*F + f); x_cur [F, n, 3] or None."""
    x_last = np.asarray(x_last, dtype=np.float64)
    n = x_last.shape[0]
    F = a_cur.shape[2]
    anchors = np.asarray(anchors, dtype=np.int64)
    ds = np.float64(np.float32(dscale))
    feat = np.zeros((F * n, WARM_FEATURES), dtype=np.float32)
    tgt = None if x_cur is None else np.zeros((F * n, 3), dtype=np.float32)
    for f in range(F):
        rows = slice(f * n, (f + 1) * n)
        for j in range(WARM_ANCHORS):
            a = nearest[:, j].astype(np.int64)
            for c in range(3):
                feat[rows, 4 * j + c] = (a_cur[c, a, f] - x_last[anchors[a], c]).astype(np.float32)
            feat[rows, 4 * j + 3] = dist[:, j]
        for c in range(3):
            feat[rows, 12 + c] = ((delta_cur[:, c * F + f] - delta_prev[:, c * F + F - 1]) * ds
                                  ).astype(np.float32)
            if x_cur is not None:
                tgt[rows, c] = (x_cur[f, :, c] - x_last[:, c]).astype(np.float32)
        feat[rows, 15] = np.float32(f + 1) / np.float32(F)
    return feat, tgt


def compose(x_last, F, pred=None):
    x0 = np.repeat(np.asarray(x_last, dtype=np.float64)[None], F, axis=0)
    if pred is not None:
        x0 = x0 + np.asarray(pred, dtype=np.float32).astype(np.float64).reshape(F, -1, 3)
    return x0


def basis_features(U_prev, U_cur=None):
    """U_prev, U_cur [3, F, k] -> (features [3F, k+1], target [3F, k] or None)."""
    U_prev = np.asarray(U_prev, dtype=np.float64)
    _, F, k = U_prev.shape
    feat = np.zeros((3 * F, k + 1), dtype=np.float32)
    feat[:, :k] = U_prev.reshape(3 * F, k).astype(np.float32)
    feat[:, k] = np.tile(np.arange(1, F + 1, dtype=np.float32) / np.float32(F), 3)
    tgt = None
    if U_cur is not None:
        tgt = (np.asarray(U_cur, dtype=np.float64) - U_prev).reshape(3 * F, k).astype(np.float32)
    return feat, tgt


def basis_compose(U_prev, pred=None):
    U_prev = np.asarray(U_prev, dtype=np.float64)
    if pred is None:
        return U_prev.copy()
    return U_prev + np.asarray(pred, dtype=np.float32).astype(np.float64).reshape(U_prev.shape)


def sample_rows(X, seed, count):
    X = np.asarray(X)
    r = rng.stream(seed, count) % np.uint64(X.shape[0])
    return X[r.astype(np.int64)]
