"""Base meshes: icosphere, closed torus grid and open planar grid.

Each function returns ``(verts float64[n,3], tris int32[T,3])`` with
consistently oriented triangles and no repeated vertex inside a triangle.
Vertex and triangle counts follow closed forms that the tests check:

* icosphere level L:  n = 10*4**L + 2,   T = 20*4**L
* torus grid a x b:   n = a*b,           T = 2*a*b      (a, b >= 3)
* open grid a x b:    n = a*b,           T = 2*(a-1)*(b-1)
"""

import numpy as np


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array(
        [[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
         [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
         [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]],
        dtype=np.float64,
    )
    f = np.array(
        [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
         [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
         [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]],
        dtype=np.int64,
    )
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


def icosphere(level):
    """Unit icosphere by repeated 1-to-4 midpoint subdivision.

    Every new midpoint is shared by the two triangles of its edge and pushed
    back onto the unit sphere.
    """
    if level < 0:
        raise ValueError("level must be >= 0")
    v, f = _icosahedron()
    verts = [row for row in v]
    for _ in range(level):
        midpoint = {}
        new_f = []

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            idx = midpoint.get(key)
            if idx is None:
                m = verts[a] + verts[b]
                m = m / np.linalg.norm(m)
                idx = len(verts)
                verts.append(m)
                midpoint[key] = idx
            return idx

        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new_f += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        f = np.array(new_f, dtype=np.int64)
    return np.array(verts, dtype=np.float64), f.astype(np.int32)


def torus_grid(n_major, n_minor, R=1.0, r=0.3):
    """Closed torus sampled on an n_major x n_minor periodic grid.

    Vertex (i, j) has index i*n_minor + j; each grid quad is split along the
    (i, j)-(i+1, j+1) diagonal.  Every vertex has degree 6.
    """
    if n_major < 3 or n_minor < 3:
        raise ValueError("torus grid needs at least 3 x 3 vertices")
    th = 2.0 * np.pi * np.arange(n_major) / n_major
    ph = 2.0 * np.pi * np.arange(n_minor) / n_minor
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    x = (R + r * np.cos(PH)) * np.cos(TH)
    y = (R + r * np.cos(PH)) * np.sin(TH)
    z = r * np.sin(PH)
    verts = np.stack([x, y, z], axis=-1).reshape(-1, 3)
    i, j = np.meshgrid(np.arange(n_major), np.arange(n_minor), indexing="ij")
    i, j = i.ravel(), j.ravel()
    ip, jp = (i + 1) % n_major, (j + 1) % n_minor
    v00 = i * n_minor + j
    v10 = ip * n_minor + j
    v11 = ip * n_minor + jp
    v01 = i * n_minor + jp
    tris = np.concatenate(
        [np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)], 0)
    return verts, tris.astype(np.int32)


def open_grid(nx, ny):
    """Planar grid on [0,1]^2 (z = 0), vertex (i, j) at index i*ny + j."""
    if nx < 2 or ny < 2:
        raise ValueError("grid needs at least 2 x 2 vertices")
    xs = np.linspace(0.0, 1.0, nx)
    ys = np.linspace(0.0, 1.0, ny)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    verts = np.stack([X, Y, np.zeros_like(X)], axis=-1).reshape(-1, 3)
    i, j = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), indexing="ij")
    i, j = i.ravel(), j.ravel()
    v00 = i * ny + j
    v10 = (i + 1) * ny + j
    v11 = (i + 1) * ny + j + 1
    v01 = i * ny + j + 1
    tris = np.concatenate(
        [np.stack([v00, v10, v11], 1), np.stack([v00, v11, v01], 1)], 0)
    return verts, tris.astype(np.int32)


def disjoint_union(meshes, offsets=None):
    """Several meshes as one vertex set with several connected components:
    the vertices of mesh m follow those of meshes 0..m-1 (translated by
    offsets[m], a 3-vector, when given) and its triangle indices are shifted
    by the vertex count before it."""
    verts, tris, base = [], [], 0
    for m, (v, t) in enumerate(meshes):
        shift = np.zeros(3) if offsets is None else np.asarray(offsets[m], dtype=np.float64)
        verts.append(np.asarray(v, dtype=np.float64) + shift)
        tris.append(np.asarray(t, dtype=np.int64) + base)
        base += v.shape[0]
    return np.concatenate(verts, 0), np.concatenate(tris, 0).astype(np.int32)


def sub_mesh(tris, keep):
    """The part of a mesh on the vertices flagged in `keep` (bool [n]): the
    triangles whose three vertices are all kept, renumbered in the kept
    vertices' order.  Returns (tris int32 [T', 3], kept vertex indices)."""
    keep = np.asarray(keep, dtype=bool)
    idx = np.nonzero(keep)[0]
    new = np.full(keep.shape[0], -1, dtype=np.int64)
    new[idx] = np.arange(idx.shape[0])
    t = np.asarray(tris, dtype=np.int64)
    t = t[np.all(keep[t], axis=1)]
    return new[t].astype(np.int32), idx
