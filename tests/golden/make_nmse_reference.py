"""Writes tests/golden/nmse_reference.txt: the FP64 oracle's reconstruction
NMSE for the benchmark workloads at their default codec settings, with the
seeded random anchors (name) and with farthest-point anchors over the first
frame from vertex 0 (name:farthest).

Calls only ``oracle/`` (and the seeded generators of ``synth``).  Run from
the repository root:  python tests/golden/make_nmse_reference.py
(--only NAME[,NAME] recomputes those entries and keeps the others).
"""

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import anchors, codec, metrics  # noqa: E402
from synth import make_sequence, config_spec  # noqa: E402

WORKLOADS = {
    # name: sweeps
    "icosphere4_F64_k16": 30,
    "torus200x100_F256_k32": 30,
    "grid316_F512_k64": 30,
    "icosphere4_F64_k16:farthest": 30,
    "torus200x100_F256_k32:farthest": 30,
    "grid316_F512_k64:farthest": 30,
    "grid512_F300_k64": 30,
    "grid512_F300_k64:farthest": 30,
}
OUT = os.path.join(HERE, "nmse_reference.txt")


def oracle_nmse(name, sweeps):
    workload, _, rule = name.partition(":")
    spec = config_spec(workload)
    tris, pos = make_sequence(spec)
    p = codec.Params(n_frames=spec.n_frames, rank=spec.rank, n_anchors=spec.n_anchors,
                     seed=spec.seed, coeff_bits=spec.coeff_bits, dict_bits=spec.dict_bits,
                     anchor_bits=spec.anchor_bits, oi_sweeps=sweeps)
    anc = anchors.farthest_point(pos[0], spec.n_anchors, 0) if rule == "farthest" else None
    rec = codec.decode(codec.encode(tris, pos, p, anchors=anc), tris)
    return metrics.nmse(pos, rec)


def main(argv):
    only = None
    if len(argv) == 2 and argv[0] == "--only":
        only = set(argv[1].split(","))
    kept = {}
    if only is not None and os.path.exists(OUT):
        for line in open(OUT):
            parts = line.split()
            if parts and not line.startswith("#"):
                kept[parts[0]] = line.rstrip("\n")
    lines = ["# FP64 oracle NMSE per workload (oracle.codec defaults: 12/16/16 bits,",
             "# random-walk Laplacian, fixed orthogonal-iteration sweeps); name:farthest",
             "# with farthest-point anchors over frame 0 from vertex 0 (oracle.anchors).",
             "# Written by tests/golden/make_nmse_reference.py from oracle/ only.",
             "# workload  sweeps  nmse"]
    for name, sweeps in WORKLOADS.items():
        if only is not None and name not in only:
            if name in kept:
                lines.append(kept[name])
            continue
        lines.append(f"{name}  {sweeps}  {oracle_nmse(name, sweeps):.17e}")
        print(lines[-1], flush=True)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main(sys.argv[1:])
