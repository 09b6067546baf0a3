"""Mesh graph and Laplacian (Section II, Eq. 1-4).

Test infrastructure (see ``oracle/__init__``).

* The 1-ring Psi_i of vertex i is the set of vertices that share a triangle
  edge with i; C_ij = 1 iff j in Psi_i (Eq. 2); d_i = sum_j C_ij (Eq. 1).
* The adjacency is stored as CSR without the diagonal: ``row_ptr`` int32
  [n+1], ``col_idx`` int32 [nnz] with each row sorted ascending, ``deg``
  int32 [n].  The Laplacian pattern is this plus the diagonal, so
  nnz(L) = n + nnz(C).
* Two Laplacians (the paper states both and they differ by the factor d_i):
  - kind 0, "random walk" (Eq. 3): delta_i = v_i - (1/|Psi_i|) sum_j v_j,
    i.e. L = I - D^-1 C.  Evaluated as: sum the neighbours in ascending j,
    one correctly rounded division by d_i, one subtraction, so that L 1 = 0
    holds exactly.
  - kind 1, "combinatorial" (Eq. 1, Eq. 4): L = D - C, delta_i =
    d_i v_i - sum_j v_j (neighbour sum in ascending j, then d_i*v_i minus it).

* Connected components (``components``): the normal matrix L^T L + P^T P
  of Eq. 12 is singular unless every connected component of the mesh graph
  holds an anchor (L annihilates the constants of each component, Eq. 3:
  L 1 = 0 row by row), so the decoder needs one anchor per component.
  Each vertex is labelled with the smallest vertex index of its component,
  found by breadth-first search from the lowest unlabelled vertex.

Pinned by: Euler-formula edge counts on closed and open meshes, symmetric
pattern, degree histograms (icosphere: 12 vertices of degree 5, all others 6;
torus: all 6), exact zero row sums, component labels against the null space
of L and against disjoint unions of meshes (tests/test_oracle_graph.py).
"""

from collections import deque

import numpy as np
import scipy.sparse as sp


class MeshError(ValueError):
    """Raised for triangles that do not describe a valid mesh graph."""


class AnchorCoverageError(ValueError):
    """Raised when a connected component holds no anchor (Eq. 12 singular)."""


def build_adjacency(tris, n):
    """CSR adjacency from triangles.

    Rejects: n < 1, indices outside [0, n), a triangle that repeats a vertex,
    and isolated vertices (d_i = 0 leaves Eq. 3 undefined).
    """
    tris = np.asarray(tris)
    if n < 1:
        raise MeshError("n must be positive")
    if tris.ndim != 2 or tris.shape[1] != 3 or tris.shape[0] == 0:
        raise MeshError("triangles must be a non-empty [T, 3] array")
    t = tris.astype(np.int64)
    if t.min() < 0 or t.max() >= n:
        raise MeshError("vertex index out of range")
    if np.any(t[:, 0] == t[:, 1]) or np.any(t[:, 1] == t[:, 2]) or np.any(t[:, 0] == t[:, 2]):
        raise MeshError("degenerate triangle (repeated vertex)")
    # every triangle edge in both directions
    src = np.concatenate([t[:, 0], t[:, 1], t[:, 1], t[:, 2], t[:, 2], t[:, 0]])
    dst = np.concatenate([t[:, 1], t[:, 0], t[:, 2], t[:, 1], t[:, 0], t[:, 2]])
    key = np.unique(src * n + dst)            # sorted by (row, col), duplicates removed
    rows = key // n
    cols = key % n
    deg = np.bincount(rows, minlength=n)
    if np.any(deg == 0):
        raise MeshError("isolated vertex")
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    return (row_ptr.astype(np.int32), cols.astype(np.int32), deg.astype(np.int32))


def _neighbour_sum(row_ptr, col_idx, X):
    """S_i = sum over j in Psi_i of X_j, added one neighbour at a time in
    ascending j (a fixed, documented order)."""
    n = row_ptr.shape[0] - 1
    deg = np.diff(row_ptr.astype(np.int64))
    S = np.zeros_like(X)
    for m in range(int(deg.max())):
        rows = np.nonzero(deg > m)[0]
        S[rows] += X[col_idx[row_ptr[rows] + m]]
    return S


def apply_laplacian(row_ptr, col_idx, deg, X, kind=0):
    """delta = L X for X of shape [n, m] (Eq. 3 / Eq. 4, column by column)."""
    X = np.asarray(X, dtype=np.float64)
    S = _neighbour_sum(row_ptr, col_idx, X)
    d = deg.astype(np.float64)[:, None]
    if kind == 0:
        return X - S / d
    if kind == 1:
        return d * X - S
    raise ValueError("laplacian kind must be 0 or 1")


def laplacian_matrix(row_ptr, col_idx, deg, kind=0):
    """L as a scipy CSR matrix (for the decoder's normal equations)."""
    n = row_ptr.shape[0] - 1
    rows = np.repeat(np.arange(n), np.diff(row_ptr.astype(np.int64)))
    d = deg.astype(np.float64)
    if kind == 0:
        off = -1.0 / d[rows]
        diag = np.ones(n)
    else:
        off = -np.ones(rows.shape[0])
        diag = d
    C = sp.csr_matrix((off, col_idx.astype(np.int64), row_ptr.astype(np.int64)), shape=(n, n))
    return (C + sp.diags(diag)).tocsr()


def apply_laplacian_transpose(row_ptr, col_idx, deg, Y, kind=0):
    """L^T Y.  For kind 0: (L^T y)_j = y_j - sum_{i in Psi_j} y_i / d_i
    (the adjacency is symmetric); kind 1 is symmetric, L^T = L."""
    Y = np.asarray(Y, dtype=np.float64)
    if kind == 1:
        return apply_laplacian(row_ptr, col_idx, deg, Y, kind=1)
    Wd = Y / deg.astype(np.float64)[:, None]
    return Y - _neighbour_sum(row_ptr, col_idx, Wd)


def components(row_ptr, col_idx):
    """Component label per vertex: the smallest vertex index of its
    connected component (breadth-first search, one component at a time in
    ascending order of its lowest vertex)."""
    n = row_ptr.shape[0] - 1
    label = np.full(n, -1, dtype=np.int64)
    for root in range(n):
        if label[root] >= 0:
            continue
        label[root] = root
        queue = deque([root])
        while queue:
            i = queue.popleft()
            for j in col_idx[row_ptr[i]:row_ptr[i + 1]]:
                if label[j] < 0:
                    label[j] = root
                    queue.append(j)
    return label.astype(np.int32)


def uncovered_components(row_ptr, col_idx, anchors):
    """Labels (ascending) of the components that hold no anchor."""
    label = components(row_ptr, col_idx)
    roots = np.unique(label)
    covered = np.unique(label[np.asarray(anchors, dtype=np.int64)]) if len(anchors) else []
    return np.setdiff1d(roots, covered).astype(np.int32)
