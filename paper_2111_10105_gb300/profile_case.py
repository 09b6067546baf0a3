"""A small profiling case: one encode and one decode of a named workload.

For a kernel profiler, which replays each captured launch many times: the
decoder's CG runs a fixed number of iterations (`--cg-iters`, the iteration
cap; the decode then reports that it did not converge, which is expected
here) and the encoder a given number of orthogonal-iteration sweeps, so that
every kernel of the path launches a few times on full-size data without the
long solve.  It prints nothing but the column and iteration counts: it is
not a benchmark (bench.py is).

    python -m paper_2111_10105_gb300.profile_case --workload grid316_F512_k64 \\
        --precision tf32 --sweeps 4 --cg-iters 40

With --warm-decode the decoder first runs one complete solve (the handle
then keeps the anchor response G), and the next decode, which solves only
the 3k data columns as every later decode of a stream does, runs inside the
NVTX range "profiled_decode" (ncu --nvtx --nvtx-include "profiled_decode/");
--cg-iters is then ignored.
"""

import argparse
import os
import sys


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="grid316_F512_k64")
    ap.add_argument("--precision", choices=["fp64", "tf32", "bf16"], default="tf32")
    ap.add_argument("--solve-mode", choices=["frames", "factored"], default="factored")
    ap.add_argument("--sweeps", type=int, default=4)
    ap.add_argument("--cg-iters", type=int, default=40)
    ap.add_argument("--warm-decode", action="store_true")
    args = ap.parse_args(argv)

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch

    from paper_2111_10105_gb300 import MeshCodec
    from synth import config_spec, make_sequence

    spec = config_spec(args.workload)
    tris, pos = make_sequence(spec)
    prec = {"fp64": 0, "tf32": 1, "bf16": 2}[args.precision]
    mc = MeshCodec(tris, pos.shape[1], n_frames=spec.n_frames, rank=spec.rank,
                   n_anchors=spec.n_anchors, seed=spec.seed, precision=prec,
                   oi_refine_sweeps=1 if prec else 0, cg_rtol=1e-6 if prec else 1e-14,
                   solve_mode={"frames": 0, "factored": 1}[args.solve_mode],
                   oi_sweeps=args.sweeps,
                   cg_max_iters=50000 if args.warm_decode else args.cg_iters)
    bits = mc.encode(torch.from_numpy(pos).cuda())
    if args.warm_decode:
        mc.decode(bits)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("profiled_decode")
        mc.decode(bits)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    else:
        mc.decode(bits, allow_not_converged=True)
    torch.cuda.synchronize()
    st = mc.stats()
    print("columns", st["cg_columns"], "iterations", st["cg_iters_max"])
    mc.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
