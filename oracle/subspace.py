"""Eigen-trajectory subspace: orthogonal iterations and Rayleigh-Ritz.

Test infrastructure (see ``oracle/__init__``).

Notation: the paper's k (number of frames) is F here and its k_l (number of
retained rows, Eq. 10) is k.  For one coordinate, A_c is the F x n matrix of
that coordinate over all frames (Section III).

* ``start_basis``      - Q0: an F x k matrix of splitmix64 uniforms in [-1,1)
                         (seed ^ (BASIS_SALT + c), element f*k+j), made
                         orthonormal by ``qr_pos``.  Algorithm 1 starts from
                         a previous block's basis or an SVD; a single block
                         (n_b = 1) has neither, so the codec starts from a
                         seeded random basis.
* ``qr_pos``           - thin Householder QR (LAPACK through numpy) with the
                         signs fixed so that diag(R) > 0, which makes Q unique
                         for a full-rank argument.
* ``orthogonal_iterations`` - Algorithm 1's inner loop for one block:
                         Q <- QR(R Q) with R = A_c A_c^T (Eq. 7) applied as
                         A_c (A_c^T Q), never formed.  Stops after ``sweeps``
                         sweeps, or earlier once ||Q_new - Q (Q^T Q_new)||_F
                         <= tol when tol > 0.
* ``rayleigh_ritz``    - orders the basis as eigenvectors of R restricted to
                         span(Q): H = W^T W with W = A_c^T Q, eigenpairs of H
                         by LAPACK, eigenvalues descending (ties keep the
                         lower index), U = Q V, then ``sign_rule``.  Eq. 10
                         keeps "the first k_l rows", i.e. the eigenvectors of
                         the k largest eigenvalues (Eq. 5 lists them in
                         decreasing order).
* ``sign_rule``        - the paper leaves the sign of each eigenvector open;
                         the codec flips column u so that sum_i (i+1) u_i > 0,
                         and when |sum| < 1e-12 * ||u||_1 * F uses the sign of
                         the entry of largest magnitude (lowest index on ties).

Pinned by: U^T U = I; on tiny meshes the span and Ritz values match a
brute-force eigendecomposition of A A^T (Eq. 5); trajectory data of exact
rank r <= k is reproduced exactly (tests/test_oracle_subspace.py).
"""

import numpy as np

from . import rng


def qr_pos(Z):
    Q, R = np.linalg.qr(Z, mode="reduced")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :]


def start_basis(F, k, seed, c):
    z = rng.uniform_pm1((seed ^ (rng.BASIS_SALT + c)) & rng.MASK64, F * k)
    return qr_pos(z.reshape(F, k))


def orthogonal_iterations(A_c, Q0, sweeps, tol=0.0):
    """Returns (Q, sweeps_done, last_change)."""
    Q = Q0
    change = np.inf
    done = 0
    for _ in range(sweeps):
        W = A_c.T @ Q          # n x k
        Z = A_c @ W            # F x k  = R Q
        Q_new = qr_pos(Z)
        done += 1
        if tol > 0:
            change = np.linalg.norm(Q_new - Q @ (Q.T @ Q_new))
            Q = Q_new
            if change <= tol:
                break
        else:
            Q = Q_new
    return Q, done, change


def sign_rule(U):
    U = U.copy()
    F = U.shape[0]
    w = np.arange(1, F + 1, dtype=np.float64)
    for j in range(U.shape[1]):
        u = U[:, j]
        s = float(np.dot(w, u))
        if abs(s) < 1e-12 * float(np.abs(u).sum()) * F:
            s = u[int(np.argmax(np.abs(u)))]
        if s < 0:
            U[:, j] = -u
    return U


def rayleigh_ritz(A_c, Q):
    """Returns (U F x k with orthonormal columns, theta k descending)."""
    W = A_c.T @ Q
    H = W.T @ W
    H = 0.5 * (H + H.T)
    theta, V = np.linalg.eigh(H)
    order = np.argsort(-theta, kind="stable")
    theta = theta[order]
    V = V[:, order]
    U = sign_rule(Q @ V)
    return U, theta


def top_k_basis(A_c, k, seed, c, sweeps, tol=0.0):
    """Start basis, orthogonal iterations, Rayleigh-Ritz: the encoder's U_c."""
    F = A_c.shape[0]
    Q0 = start_basis(F, k, seed, c)
    Q, done, change = orthogonal_iterations(A_c, Q0, sweeps, tol)
    U, theta = rayleigh_ritz(A_c, Q)
    return U, theta, done, change


def brute_force_basis(A_c, k):
    """Top-k eigenvectors of R = A_c A_c^T by a dense eigensolver (Eq. 5,
    Eq. 7): the pin for the iterative path on small inputs."""
    R = A_c @ A_c.T
    lam, V = np.linalg.eigh(0.5 * (R + R.T))
    order = np.argsort(-lam, kind="stable")
    return sign_rule(V[:, order[:k]]), lam[order]
