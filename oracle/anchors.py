"""Anchor selection by farthest points - TEST INFRASTRUCTURE (oracle).

Section III-B of the paper quantizes n_c "uniformly distributed" anchor
vertices (about 1% of n); Section V reports that a random choice changes the
results little and leaves the best choice open.  The codec's default draws
the anchors at random (``codec.select_anchors``); this module gives the
evenly spread alternative used in the anchor-selection study: the greedy
farthest-point rule for the k-center problem (T. F. Gonzalez, "Clustering to
minimize the maximum intercluster distance", Theoretical Computer Science 38,
1985).

Definition followed: start from vertex ``start``; then, n_c - 1 times, add the
vertex whose squared Euclidean distance to its nearest chosen vertex is
largest, the lowest index among equal distances.  A squared distance is
(dx*dx + dy*dy) + dz*dz with every operation rounded separately in binary64.
The chosen set is returned in ascending order.

Pinned by: the dyadic closed form on equally spaced collinear points, the
factor-2 guarantee of the greedy rule against the brute-force optimal
k-center radius on small point sets, and the invariants of the output
(tests/test_oracle_anchors.py).
"""

import numpy as np


def farthest_point(xyz, n_c, start=0):
    """Greedy farthest-point selection: int32 [n_c] vertex indices, ascending."""
    xyz = np.asarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    if not (1 <= n_c <= n and 0 <= start < n):
        raise ValueError("need 1 <= n_c <= n and 0 <= start < n")
    nearest = np.full(n, np.inf)       # squared distance to the nearest chosen vertex
    nearest[start] = -1.0              # chosen vertices are never chosen again
    chosen = [start]
    for _ in range(1, n_c):
        d = xyz - xyz[chosen[-1]]
        dist = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]
        nearest = np.minimum(nearest, dist)
        nxt = int(np.argmax(nearest))  # first maximum: the lowest index on ties
        chosen.append(nxt)
        nearest[nxt] = -1.0
    return np.sort(np.asarray(chosen, dtype=np.int32))


def covering_radius(xyz, anchors):
    """Largest Euclidean distance from a vertex to its nearest anchor."""
    xyz = np.asarray(xyz, dtype=np.float64)
    d = np.linalg.norm(xyz[:, None, :] - xyz[None, np.asarray(anchors), :], axis=2)
    return float(d.min(axis=1).max())
