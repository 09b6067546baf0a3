"""Writes tests/golden/nmse_reference.txt: the FP64 oracle's reconstruction
NMSE for the benchmark workloads at their default codec settings.

Calls only ``oracle/`` (and the seeded generators of ``synth``).  Run from
the repository root:  python tests/golden/make_nmse_reference.py
"""

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import codec, metrics  # noqa: E402
from synth import make_sequence, config_spec  # noqa: E402

WORKLOADS = {
    # name: (sweeps, frames or None for all)
    "icosphere4_F64_k16": (30, None),
    "torus200x100_F256_k32": (30, None),
    "grid316_F512_k64": (30, None),
}


def main():
    lines = ["# FP64 oracle NMSE per workload (oracle.codec defaults: 12/16/16 bits,",
             "# random-walk Laplacian, fixed orthogonal-iteration sweeps).",
             "# Written by tests/golden/make_nmse_reference.py from oracle/ only.",
             "# workload  sweeps  nmse"]
    for name, (sweeps, frames) in WORKLOADS.items():
        spec = config_spec(name)
        tris, pos = make_sequence(spec)
        p = codec.Params(n_frames=spec.n_frames, rank=spec.rank, n_anchors=spec.n_anchors,
                         seed=spec.seed, coeff_bits=spec.coeff_bits, dict_bits=spec.dict_bits,
                         anchor_bits=spec.anchor_bits, oi_sweeps=sweeps)
        rec = codec.decode(codec.encode(tris, pos, p), tris)
        lines.append(f"{name}  {sweeps}  {metrics.nmse(pos, rec):.17e}")
        print(lines[-1], flush=True)
    with open(os.path.join(HERE, "nmse_reference.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
