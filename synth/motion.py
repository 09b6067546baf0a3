"""Seeded motion models that turn a base mesh into an F-frame sequence.

Recipe (all draws from ``numpy.random.default_rng(seed)``, in this order):

1. Sinusoidal displacement fields, j = 1..n_fields (8 by default), each
   ``amp * d_j * sin(2*pi*<w_j, p> + phi_j + beta_j*<kappa_j, p>*sin(2*pi*f_j*t/F + psi_j))``
   with d_j a random unit vector, w_j a random unit direction scaled by
   |w_j| ~ U[1, 4] (spatial frequency), f_j ~ U[0.5, 3] cycles per sequence
   (temporal frequency), phases ~ U[0, 2*pi), kappa_j a random unit vector
   and beta_j ~ U[4, 8].  The position-dependent phase modulation makes each
   field non-separable in space and time, so the trajectory matrix has full
   rank with a geometrically decaying spectrum, as captured animations do; a
   separable field (spatial pattern times temporal sine) would give every
   coordinate a trajectory rank of only 3 + n_fields + 1.
2. Optional travelling bend wave (torus): a z-displacement
   ``bend * sin(2*theta_i - 2*pi*t/F)`` with theta_i the major angle of the
   base vertex.
3. Optional moving Gaussian bumps (planar grids): n_bumps bumps of height
   U[0.1, 0.3] and width U[0.05, 0.15] whose centres move on straight lines
   between two U[0,1]^2 points over the sequence, displacing z.
4. Optional rigid motion: a rotation about a random unit axis whose angle
   ramps linearly from 0 to U[0, pi/4] over the frames, then a translation
   ramping from 0 to U[0, 0.5]^3.
5. Optional i.i.d. N(0, noise^2) noise on every coordinate of every frame.

Frame f uses t = f (f = 0..F-1).  Positions are float64 [F, n, 3].
"""

from dataclasses import dataclass, field
import math

import numpy as np

from .meshes import icosphere, torus_grid, open_grid


@dataclass
class SequenceSpec:
    """A named synthetic workload: a base mesh plus a motion model plus the
    codec settings it is evaluated with (rank k, bits, anchors)."""

    name: str
    mesh: str                 # "icosphere:L" | "torus:a:b" | "grid:a:b"
    n_frames: int
    rank: int
    n_anchors: int
    seed: int
    coeff_bits: int = 12
    dict_bits: int = 16
    anchor_bits: int = 16
    n_fields: int = 8
    amp: float = 0.05
    bend: float = 0.0
    n_bumps: int = 0
    rigid: bool = True
    noise: float = 0.0
    # temporal frequency multiplier (cycles per sequence are drawn in
    # [0.5, 3] * tfreq); a sequence cut into S segments with tfreq = S gives
    # every segment the temporal content of a standalone sequence
    tfreq: float = 1.0
    extra: dict = field(default_factory=dict)


def base_mesh(mesh):
    kind, *args = mesh.split(":")
    if kind == "icosphere":
        return icosphere(int(args[0]))
    if kind == "torus":
        return torus_grid(int(args[0]), int(args[1]))
    if kind == "grid":
        return open_grid(int(args[0]), int(args[1]))
    raise ValueError(f"unknown mesh kind {mesh!r}")


def _unit(rng, m):
    v = rng.normal(size=(m, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _rotation(axis, angle):
    """Rotation matrix about a unit axis (Rodrigues' formula)."""
    x, y, z = axis
    K = np.array([[0.0, -z, y], [z, 0.0, -x], [-y, x, 0.0]])
    return np.eye(3) + math.sin(angle) * K + (1.0 - math.cos(angle)) * (K @ K)


def sinusoid_rigid_motion(verts, spec, rng=None, frame_range=None):
    """Apply the motion model of ``spec`` to base vertices ``verts``.

    Returns float64 [F, n, 3], or only frames f0 .. f1-1 of the same
    sequence for ``frame_range = (f0, f1)`` (identical values; the random
    parameters are drawn the same way; not with noise, whose draw depends
    on the number of frames).
    """
    if rng is None:
        rng = np.random.default_rng(spec.seed)
    F = spec.n_frames
    n = verts.shape[0]
    f0, f1 = (0, F) if frame_range is None else frame_range
    if frame_range is not None and spec.noise:
        raise ValueError("frame_range with noise")
    t = np.arange(f0, f1, dtype=np.float64)
    Fr = f1 - f0
    pos = np.broadcast_to(verts, (Fr, n, 3)).copy()

    if spec.n_fields:
        d = _unit(rng, spec.n_fields)
        wdir = _unit(rng, spec.n_fields)
        wmag = rng.uniform(1.0, 4.0, size=spec.n_fields)
        w = wdir * wmag[:, None]
        fr = rng.uniform(0.5, 3.0, size=spec.n_fields) * spec.tfreq
        phi = rng.uniform(0.0, 2 * np.pi, size=spec.n_fields)
        psi = rng.uniform(0.0, 2 * np.pi, size=spec.n_fields)
        kappa = _unit(rng, spec.n_fields)
        beta = rng.uniform(4.0, 8.0, size=spec.n_fields)
        for j in range(spec.n_fields):
            x = 2 * np.pi * (verts @ w[j]) + phi[j]                         # [n]
            h = beta[j] * (verts @ kappa[j])                                # [n]
            y = np.sin(2 * np.pi * fr[j] * t / F + psi[j])                  # [F]
            g = np.sin(x[None, :] + h[None, :] * y[:, None])                # [F,n]
            pos += spec.amp * g[:, :, None] * d[j][None, None, :]

    if spec.bend:
        theta = np.arctan2(verts[:, 1], verts[:, 0])
        wave = spec.bend * np.sin(2.0 * theta[None, :] - 2 * np.pi * spec.tfreq * t[:, None] / F)
        pos[:, :, 2] += wave

    if spec.n_bumps:
        h = rng.uniform(0.1, 0.3, size=spec.n_bumps)
        s = rng.uniform(0.05, 0.15, size=spec.n_bumps)
        c0 = rng.uniform(0.0, 1.0, size=(spec.n_bumps, 2))
        c1 = rng.uniform(0.0, 1.0, size=(spec.n_bumps, 2))
        lam = t / max(F - 1, 1)
        for b in range(spec.n_bumps):
            c = c0[b][None, :] + lam[:, None] * (c1[b] - c0[b])[None, :]   # [F,2]
            for f in range(Fr):
                r2 = ((verts[:, :2] - c[f]) ** 2).sum(1)
                pos[f, :, 2] += h[b] * np.exp(-r2 / (2 * s[b] ** 2))

    if spec.rigid:
        axis = _unit(rng, 1)[0]
        ang_max = rng.uniform(0.0, np.pi / 4)
        tr_max = rng.uniform(0.0, 0.5, size=3)
        lam = t / max(F - 1, 1)
        for f in range(Fr):
            Rf = _rotation(axis, ang_max * lam[f])
            pos[f] = pos[f] @ Rf.T + lam[f] * tr_max[None, :]

    if spec.noise:
        pos += rng.normal(0.0, spec.noise, size=pos.shape)
    return pos


def make_sequence(spec):
    """Build (tris int32[T,3], positions float64[F,n,3]) for a spec."""
    verts, tris = base_mesh(spec.mesh)
    pos = sinusoid_rigid_motion(verts, spec)
    return tris, np.ascontiguousarray(pos)


# Workloads.  Sizes, ranks and anchor counts follow the evaluation setups of
# the codec; seeds are fixed per workload.
CONFIGS = {
    "icosphere4_F64_k16": SequenceSpec(
        name="icosphere4_F64_k16", mesh="icosphere:4", n_frames=64, rank=16,
        n_anchors=20, seed=1000),
    "torus200x100_F256_k32": SequenceSpec(
        name="torus200x100_F256_k32", mesh="torus:200:100", n_frames=256,
        rank=32, n_anchors=50, seed=1001, bend=0.1),
    "grid316_F512_k64": SequenceSpec(
        name="grid316_F512_k64", mesh="grid:316:316", n_frames=512, rank=64,
        n_anchors=999, seed=1002, n_bumps=4, rigid=False, noise=0.02),
    "grid512_F300_k64": SequenceSpec(
        name="grid512_F300_k64", mesh="grid:512:512", n_frames=300, rank=64,
        n_anchors=2621, seed=1004, n_bumps=4, rigid=False),
    # the profiling case: the 512 x 512 workload's kind of mesh, motion and
    # rank (its 192 data columns) at a quarter of its vertices (positions
    # 403 MB, above the 129 MB L2)
    "grid256_F256_k64": SequenceSpec(
        name="grid256_F256_k64", mesh="grid:256:256", n_frames=256, rank=64,
        n_anchors=655, seed=1005, n_bumps=4, rigid=False),
}


def config_spec(name, **overrides):
    spec = CONFIGS[name]
    if overrides:
        d = dict(spec.__dict__)
        d.update(overrides)
        spec = SequenceSpec(**d)
    return spec


def batched_specs(n_seq=64, seed=1003):
    """Ragged batch: n log-uniform in [1k, 50k], mesh type round-robin
    (icosphere / torus / grid, sized to the nearest n), F ~ U[32, 300],
    k ~ U[8, min(48, F)]."""
    rng = np.random.default_rng(seed)
    specs = []
    for s in range(n_seq):
        n_target = math.exp(rng.uniform(math.log(1000), math.log(50000)))
        F = int(rng.integers(32, 301))
        k = int(rng.integers(8, min(48, F) + 1))
        kind = s % 3
        if kind == 0:
            L = int(round(math.log((n_target - 2) / 10.0, 4)))
            L = max(3, min(L, 6))
            mesh = f"icosphere:{L}"
            n = 10 * 4 ** L + 2
        elif kind == 1:
            b = max(3, int(round(math.sqrt(n_target / 2))))
            mesh = f"torus:{2 * b}:{b}"
            n = 2 * b * b
        else:
            a = max(3, int(round(math.sqrt(n_target))))
            mesh = f"grid:{a}:{a}"
            n = a * a
        specs.append(SequenceSpec(
            name=f"batch{s}", mesh=mesh, n_frames=F, rank=k,
            n_anchors=max(4, n // 100), seed=seed * 1000 + s,
            bend=0.1 if kind == 1 else 0.0,
            n_bumps=4 if kind == 2 else 0))
    return specs
