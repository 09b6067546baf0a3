"""Learned warm starts for a long sequence coded in segments.

A sequence is cut into segments of F frames, each coded by the same
``MeshCodec`` (same connectivity and anchors).  Two starts can be learned
from what earlier segments left behind; neither changes a result, only the
work to reach it:

* decoder: the first CG iterate of Eq. 12's solve.  ``"cold"`` is X0 = 0 (the
  codec's default), ``"previous"`` repeats the last decoded frame of the
  previous segment, ``"learned"`` adds a perceptron's prediction of the
  motion since that frame, computed from the current segment's dequantized
  anchors and back-projected delta coordinates (what its stream carries) and
  trained online on the decoder's own earlier reconstructions;
* encoder: the start basis of the orthogonal iterations (Algorithm 1).
  ``"seeded"`` is the codec's random start, ``"previous"`` the previous
  segment's dictionary (Algorithm 1's own choice for blocks after the first),
  ``"learned"`` that dictionary plus a second perceptron's predicted change,
  trained on the encoder's earlier dictionaries.

Every step runs in ``libmesh_codec.so`` kernels; this module only sequences
the calls.
"""

from . import codec as _c


class _Trainer:
    def __init__(self, n_in, n_out, hidden, seed, lr, steps, batch):
        self.net = _c.Mlp(n_in, hidden, n_out, seed)
        self.seed = seed
        self.lr, self.steps, self.batch = lr, steps, batch
        self.fitted = False
        self.calls = 0
        self.last_loss = None

    def fit(self, feat, tgt):
        """`steps` Adam steps on seeded minibatches of (feat, tgt)."""
        if not self.fitted:
            self.net.fit_normalizer(feat)
        N = feat.shape[0]
        count = min(self.batch, N)
        loss = None
        for i in range(self.steps):
            s = (self.seed << 20) + (self.calls << 12) + i
            xb = _c.sample_rows(feat, s, count)
            tb = _c.sample_rows(tgt, s, count)
            loss = self.net.train_step(xb, tb, lr=self.lr, want_loss=(i == self.steps - 1))
        self.calls += 1
        self.fitted = True
        self.last_loss = loss
        return loss


class WarmStart:
    """Online warm starts for one codec handle (frames solve mode), or for
    a decoder handle plus an encoder handle of the same connectivity,
    anchors and sizes (e.g. an FP64 encoder and a mixed-precision decoder).

    rest: CUDA float64 [n, 3], the rest pose used for the anchor distances.
    """

    def __init__(self, codec, rest, hidden=256, seed=1, lr=1e-3, steps=200, batch=65536,
                 basis_steps=200, encoder=None):
        self.codec = codec
        self.enc = encoder if encoder is not None else codec
        self.n, self.F, self.k = codec.n, codec.F, codec.k
        self.anchors = codec.buffer(_c.BUF_ANCHORS)
        self.nearest, self.dist = _c.nearest_anchors(rest.contiguous(), self.anchors)
        self.pos = _Trainer(_c.WARM_FEATURES, 3, hidden, seed, lr, steps, batch)
        self.basis = _Trainer(self.k + 1, self.k, hidden, seed + 1, lr, basis_steps,
                              3 * self.F)
        self.x_prev = None        # decoded positions of the previous segment [F, n, 3]
        self.delta_prev = None    # its back-projected delta coordinates [n, 3F]
        self.U_prev = None        # the encoder's previous dictionary [3, F, k]

    # ------------------------------------------------------------ decoder
    def initial_positions(self, bitstream, start="learned"):
        """(x0 or None, delta~, anchors^) for one segment's stream."""
        delta, anc = self.codec.decode_stage(bitstream)
        if start == "cold" or self.x_prev is None:
            return None, delta, anc
        x_last = self.x_prev[-1]
        pred = None
        if start == "learned" and self.pos.fitted:
            feat, _ = _c.warm_features(x_last, anc, self.anchors, self.nearest, self.dist, delta,
                                       self.delta_prev)
            pred = self.pos.net.infer(feat)
        elif start not in ("previous", "learned"):
            raise ValueError(start)
        return _c.warm_compose(x_last, self.F, pred), delta, anc

    def observe_decoded(self, x, delta, anc, fit=True):
        """Learn from a decoded segment (the pair previous -> this one; not with
        fit=False, e.g. once the network is trained), then make it the
        previous segment."""
        if fit and self.x_prev is not None:
            feat, tgt = _c.warm_features(self.x_prev[-1], anc, self.anchors, self.nearest,
                                         self.dist, delta, self.delta_prev, x_cur=x)
            self.pos.fit(feat, tgt)
        self.x_prev, self.delta_prev = x, delta

    def decode(self, bitstream, start="learned", learn=True):
        x0, delta, anc = self.initial_positions(bitstream, start)
        x = self.codec.decode(bitstream, x0=x0)
        if learn:
            self.observe_decoded(x, delta, anc)
        return x

    # ------------------------------------------------------------ encoder
    def start_basis(self, start="learned"):
        """The q0 to pass to set_start_basis (None: the seeded start)."""
        if start == "seeded" or self.U_prev is None:
            return None
        pred = None
        if start == "learned" and self.basis.fitted:
            feat, _ = _c.basis_features(self.U_prev)
            pred = self.basis.net.infer(feat)
        elif start not in ("previous", "learned"):
            raise ValueError(start)
        return _c.basis_compose(self.U_prev, pred)

    def observe_basis(self, U, fit=True):
        """Learn from an encoded segment's dictionary (not with fit=False),
        then keep it."""
        if fit and self.U_prev is not None:
            feat, tgt = _c.basis_features(self.U_prev, U)
            self.basis.fit(feat, tgt)
        self.U_prev = U.clone()

    def encode(self, positions, start="learned", learn=True, out=None):
        self.enc.set_start_basis(self.start_basis(start))
        bs = self.enc.encode(positions, out=out)
        if learn:
            self.observe_basis(self.enc.buffer(_c.BUF_BASIS).view(3, self.F, self.k))
        return bs
