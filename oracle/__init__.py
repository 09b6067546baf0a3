"""FP64 CPU oracle for the spatio-temporal dynamic-mesh codec.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The product path (``paper_2111_10105_gb300``) never imports it and shares no
code with it; the two agree only through the paper's definitions and the
seeded inputs of ``synth``.

It is a plain, slow restatement of "Fast Spatio-temporal Compression of
Dynamic 3D Meshes" (Arvanitis, Lalos, Moustakas), following the paper's
steps in order:

* ``graph``    - 1-ring neighbourhoods, adjacency, degrees and the Laplacian
                 (Section II, Eq. 1-4).
* ``rng``      - splitmix64, the counter-based generator both sides use for
                 the anchor choice and the starting basis (published
                 definition by Steele, Lea and Flood, OOPSLA 2014).
* ``subspace`` - orthogonal iterations (Algorithm 1, Eq. 5, Eq. 7) with a
                 Householder QR, then the Rayleigh-Ritz ordering of the
                 retained eigen-trajectories.
* ``quant``    - the uniform scalar quantizer standing in for Q(.) of Eq. 10
                 and the bit-plane packing of the symbols.
* ``codec``    - encoder (Eq. 7-10) and decoder (anchored least squares,
                 Eq. 12), with the bitstream layout.
* ``metrics``  - NMSE and the bit-rate accounting of Eq. 13.
* ``blocks``   - the blocks variant (Section III-A, Algorithm 1 across
                 blocks) with the difference coding of consecutive
                 dictionaries (Section IV, Fig. 6).
* ``anchors``  - evenly spread anchors by greedy farthest points, the
                 alternative to the random choice in the anchor-selection
                 study (Section III-B, Section V).
* ``mlp``, ``warm`` - the learned warm start (not in the paper): the
                 perceptron in FP64 and its input features.

Parity status per function is stated in each module header; functions whose
output no pin fixes say "parity unpinned" there.
"""

from . import rng, graph, subspace, quant, codec, metrics  # noqa: F401
