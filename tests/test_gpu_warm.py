"""Learned warm start on the GPU: the perceptron's kernels against the FP64
oracle (initialisation, standardisation, forward, gradients, Adam), the
feature kernels against the oracle, and the gain of the learned starts in
CG iterations and orthogonal-iteration sweeps over the plain starts."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp as omlp, warm as owarm  # noqa: E402
from synth import SequenceSpec  # noqa: E402
from synth.motion import base_mesh, sinusoid_rigid_motion  # noqa: E402

pytestmark = pytest.mark.gpu

N_IN, H, N_OUT = 16, 256, 3


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2111_10105_gb300 import build
    build.build()


def _c():
    from paper_2111_10105_gb300 import codec
    return codec


def _data(N, seed):
    r = np.random.default_rng(seed)
    scales = 10.0 ** r.uniform(-3, 1, size=N_IN)
    X = (r.normal(size=(N, N_IN)) * scales + r.normal(size=N_IN)).astype(np.float32)
    T = (0.1 * r.normal(size=(N, N_OUT))).astype(np.float32)
    return X, T


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _blocks(g):
    lay = omlp.layout(N_IN, H, N_OUT)
    return {k: g[lay[k][0]:lay[k][1]] for k in ("W1", "b1", "W2", "b2", "W3", "b3")}


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_mlp_init_matches_oracle():
    net = _c().Mlp(N_IN, H, N_OUT, seed=7)
    want = omlp.init_params(N_IN, H, N_OUT, 7)
    got = net.params(0).cpu().numpy()
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(net.params(1).cpu().numpy(), omlp.bf16_round(want))


def _net_with_norm(X, seed=3, check=False):
    net = _c().Mlp(N_IN, H, N_OUT, seed=seed)
    net.set_check_mode(check)
    net.fit_normalizer(_cuda(X))
    mu, inv = (t.cpu().numpy() for t in net.normalizer())
    return net, (mu, inv)


@pytest.mark.parametrize("N,hidden", [(1, 256), (3001, 256), (4194304 + 77, 256), (999, 36)])
def test_mlp_tensor_core_inference(N, hidden):
    """infer (hidden-to-hidden product as a TF32 GEMM) against forward (FP32
    products) and the FP64 oracle: TF32 rounds the activations to a 10-bit
    mantissa, so the outputs agree to ~1e-3 of their scale."""
    X, _ = _data(N, seed=N % 1000)
    net = _c().Mlp(N_IN, hidden, N_OUT, seed=5)
    net.fit_normalizer(_cuda(X))
    Xd = _cuda(X)
    Yf = net.forward(Xd)
    Yi = net.infer(Xd)
    scale = max(float(Yf.abs().max()), 1e-3)
    assert float((Yi - Yf).abs().max()) <= 2e-3 * scale
    if N <= 3001:
        w = net.params(0).cpu().numpy()
        norm = tuple(t.cpu().numpy() for t in net.normalizer())
        Yo = omlp.forward(w, X, N_IN, hidden, N_OUT, weight_round="bf16", norm=norm)
        assert np.max(np.abs(Yi.cpu().numpy() - Yo)) <= 2e-3 * max(np.max(np.abs(Yo)), 1e-3)


@pytest.mark.parametrize("N", [1, 3001])
def test_mlp_normalizer_and_forward(N):
    X, _ = _data(N, seed=N)
    net, norm = _net_with_norm(X)
    mu_o, inv_o = omlp.fit_normalizer(X)
    np.testing.assert_allclose(norm[0], mu_o, rtol=1e-6, atol=1e-6 * np.abs(X).max())
    np.testing.assert_allclose(norm[1], inv_o, rtol=1e-5)
    w = net.params(0).cpu().numpy()
    Y = net.forward(_cuda(X)).cpu().numpy()
    Yo = omlp.forward(w, X, N_IN, H, N_OUT, weight_round="bf16", norm=norm)
    assert np.max(np.abs(Y - Yo)) <= 1e-5 * max(np.max(np.abs(Yo)), 1e-3)


def test_mlp_gradients_bf16_vs_oracle():
    # ragged sizes, and N above 4096 so the weight gradients use split-K partials
    X, T = _data(10007, seed=21)
    net, norm = _net_with_norm(X)
    w = net.params(0).cpu().numpy()
    loss = net.train_step(_cuda(X), _cuda(T), update=False)
    g = net.params(2).cpu().numpy()
    Lo, go = omlp.loss_and_grad(w, X, T, N_IN, H, N_OUT, weight_round="bf16", norm=norm)
    assert abs(loss - Lo) <= 1e-5 * Lo
    Lu, gu = omlp.loss_and_grad(w, X, T, N_IN, H, N_OUT, norm=norm)
    gb, gob, gub = _blocks(g), _blocks(go), _blocks(gu)
    for k in gb:
        # same (bfloat16-rounded) weights: float32 accumulation only
        assert _rel(gb[k], gob[k]) <= 1e-4, (k, _rel(gb[k], gob[k]))
        # against unrounded FP64 weights: the bfloat16 rounding of the weights
        assert _rel(gb[k], gub[k]) <= 1e-2, (k, _rel(gb[k], gub[k]))


def _away_from_kinks(X, T, seed=3, margin=1e-4):
    """Drops samples whose hidden pre-activations (oracle, initial weights)
    lie within `margin` (relative to their rms) of zero: there float32
    rounding can flip a ReLU and move one sample's whole contribution,
    which is not an accumulation error."""
    w = omlp.init_params(N_IN, H, N_OUT, seed)
    lay = omlp.layout(N_IN, H, N_OUT)
    for _ in range(3):
        norm = omlp.fit_normalizer(X)
        _, (Xs, H1, _, W1, W2, _) = omlp.forward(w, X, N_IN, H, N_OUT, keep=True, norm=norm)
        z1 = Xs @ W1.T + w[lay["b1"][0]:lay["b1"][1]]
        z2 = H1 @ W2.T + w[lay["b2"][0]:lay["b2"][1]]
        ok = ((np.abs(z1) > margin * np.sqrt(np.mean(z1 ** 2))).all(axis=1)
              & (np.abs(z2) > margin * np.sqrt(np.mean(z2 ** 2))).all(axis=1))
        if ok.all():
            break
        X, T = X[ok], T[ok]
    return np.ascontiguousarray(X), np.ascontiguousarray(T)


def test_mlp_gradients_fp32_check_mode():
    X, T = _away_from_kinks(*_data(5003, seed=22))
    assert X.shape[0] > 4096            # still long enough for the split-K path
    net, norm = _net_with_norm(X, check=True)
    w = net.params(0).cpu().numpy()
    net.train_step(_cuda(X), _cuda(T), update=False)
    g = _blocks(net.params(2).cpu().numpy())
    _, go = omlp.loss_and_grad(w, X, T, N_IN, H, N_OUT, norm=norm)
    go = _blocks(go)
    for k in g:
        assert _rel(g[k], go[k]) <= 1e-6, (k, _rel(g[k], go[k]))


def test_mlp_adam_steps():
    X, T = _data(2048, seed=23)
    net, norm = _net_with_norm(X, check=True)
    w = net.params(0).cpu().numpy().astype(np.float64)
    opt = omlp.Adam(w.size, lr=1e-3)
    for _ in range(3):
        _, go = omlp.loss_and_grad(w.astype(np.float32), X, T, N_IN, H, N_OUT, norm=norm)
        w_next = opt.step(w, go)
        net.train_step(_cuda(X), _cuda(T), lr=1e-3, update=True, want_loss=False)
        w = w_next
    got = net.params(0).cpu().numpy().astype(np.float64)
    # Adam moves a weight by about lr per step whatever the gradient's size,
    # so a gradient entry near zero may step the other way on one side:
    # those few entries differ by up to 2 lr per step, all others agree to
    # float32 rounding
    step_err = np.abs(got - w)
    assert np.max(step_err) <= 6 * 1e-3 * 1.01
    assert np.mean(step_err > 1e-5) < 0.01


def test_training_reduces_loss():
    r = np.random.default_rng(5)
    X = r.normal(size=(20000, N_IN)).astype(np.float32)
    T = np.stack([np.sin(X[:, 0]) * X[:, 1], np.maximum(X[:, 2], 0), X[:, 3] * X[:, 4]],
                 axis=1).astype(np.float32)
    net = _c().Mlp(N_IN, H, N_OUT, seed=9)
    net.fit_normalizer(_cuda(X))
    Xc, Tc = _cuda(X), _cuda(T)
    first = net.train_step(Xc, Tc, lr=1e-3, update=False)
    for i in range(300):
        xb = _c().sample_rows(Xc, 1000 + i, 4096)
        tb = _c().sample_rows(Tc, 1000 + i, 4096)
        net.train_step(xb, tb, lr=1e-3, want_loss=False)
    last = net.train_step(Xc, Tc, lr=1e-3, update=False)
    assert last < 0.1 * first, (first, last)


# ------------------------------------------------------------------ feature kernels
def test_feature_kernels_match_oracle():
    c = _c()
    verts, _ = base_mesh("grid:23:17")
    n = verts.shape[0]
    F, n_c = 5, 7
    r = np.random.default_rng(3)
    anchors = np.sort(r.choice(n, n_c, replace=False)).astype(np.int32)
    # a regular grid: many vertices are equally far from two anchors (ties)
    rest = verts.copy()
    idx, dist = c.nearest_anchors(_cuda(rest), _cuda(anchors))
    io, do = owarm.nearest_anchors(rest, anchors)
    np.testing.assert_array_equal(idx.cpu().numpy(), io)
    np.testing.assert_array_equal(dist.cpu().numpy(), do)
    x_last = r.normal(size=(n, 3))
    a_cur = r.normal(size=(3, n_c, F))
    d_cur = r.normal(size=(n, 3 * F)) * 1e-3
    d_prev = r.normal(size=(n, 3 * F)) * 1e-3
    x_cur = r.normal(size=(F, n, 3))
    feat, tgt = c.warm_features(_cuda(x_last), _cuda(a_cur), _cuda(anchors), idx, dist,
                                _cuda(d_cur), _cuda(d_prev), dscale=3.0, x_cur=_cuda(x_cur))
    fo, to = owarm.features(x_last, a_cur, anchors, io, do, d_cur, d_prev, 3.0, x_cur)
    np.testing.assert_array_equal(feat.cpu().numpy(), fo)
    np.testing.assert_array_equal(tgt.cpu().numpy(), to)
    pred = r.normal(size=(n * F, 3)).astype(np.float32)
    x0 = c.warm_compose(_cuda(x_last), F, _cuda(pred))
    np.testing.assert_array_equal(x0.cpu().numpy(), owarm.compose(x_last, F, pred))
    np.testing.assert_array_equal(c.warm_compose(_cuda(x_last), F).cpu().numpy(),
                                  owarm.compose(x_last, F))
    rows = c.sample_rows(feat, 12345, 777)
    np.testing.assert_array_equal(rows.cpu().numpy(), owarm.sample_rows(fo, 12345, 777))
    k = 4
    Up, Uc = r.normal(size=(3, F, k)), r.normal(size=(3, F, k))
    bf, bt = c.basis_features(_cuda(Up), _cuda(Uc))
    bfo, bto = owarm.basis_features(Up, Uc)
    np.testing.assert_array_equal(bf.cpu().numpy(), bfo)
    np.testing.assert_array_equal(bt.cpu().numpy(), bto)
    q0 = c.basis_compose(_cuda(Up), bt)
    np.testing.assert_array_equal(q0.cpu().numpy(), owarm.basis_compose(Up, bto))


# ------------------------------------------------------------------ gain
SEG_F, SEGMENTS = 32, 5


def _segments():
    # one coherent 160-frame sequence (bumps + phase-modulated fields) cut in
    # five segments of 32 frames; rank 8 (the ninth singular value of a
    # segment is 1e-4 of the first at this length)
    spec = SequenceSpec(name="grid96_warm", mesh="grid:96:96", n_frames=SEG_F * SEGMENTS, rank=8,
                        n_anchors=92, seed=2024, n_bumps=4, rigid=False)
    verts, tris = base_mesh(spec.mesh)
    pos = sinusoid_rigid_motion(verts, spec)
    return spec, verts, tris, [np.ascontiguousarray(pos[s * SEG_F:(s + 1) * SEG_F])
                               for s in range(SEGMENTS)]


def test_learned_warm_start_gain():
    c = _c()
    from paper_2111_10105_gb300.warm import WarmStart
    spec, verts, tris, segs = _segments()
    n = verts.shape[0]
    cod = c.MeshCodec(tris, n, n_frames=SEG_F, rank=spec.rank, n_anchors=spec.n_anchors,
                      seed=spec.seed, oi_sweeps=400, oi_tol=1e-6)
    ws = WarmStart(cod, _cuda(verts), steps=300, basis_steps=300)
    # encoder: learn from the first segments, then compare starts on the last
    streams = [ws.encode(_cuda(s), start="learned") for s in segs[:-1]]
    sweeps = {}
    for start in ("seeded", "previous", "learned"):
        ws.encode(_cuda(segs[-1]), start=start, learn=False)
        sweeps[start] = sum(cod.stats()["oi_sweeps"])
    cod.set_start_basis(None)
    last = cod.encode(_cuda(segs[-1])).clone()
    # decoder: learn online from its own reconstructions, then compare
    for bs in streams:
        ws.decode(bs, start="previous")
    iters, xs = {}, {}
    for start in ("cold", "previous", "learned"):
        x0, _, _ = ws.initial_positions(last, start)
        xs[start] = cod.decode(last, x0=x0).cpu().numpy()
        iters[start] = cod.stats()["cg_iters_mean"]
    print("oi sweeps to 1e-6:", sweeps, "cg iterations (mean over columns):", iters,
          "position loss:", ws.pos.last_loss, "basis loss:", ws.basis.last_loss)
    # every start reaches the same solution of Eq. 12
    scale = np.max(np.abs(xs["cold"]))
    for start in ("previous", "learned"):
        assert np.max(np.abs(xs[start] - xs["cold"])) <= 1e-9 * scale
    # the previous segment's basis is Algorithm 1's start: fewer sweeps than
    # the seeded one on coherent motion (the oracle takes 22 and 18 on this
    # segment); the learned correction must not lose to the random start
    assert sweeps["previous"] < sweeps["seeded"]
    assert sweeps["learned"] <= sweeps["seeded"]
    # decoder: previous frame beats cold, the learned start beats the previous frame
    assert iters["previous"] < iters["cold"]
    assert iters["learned"] < iters["previous"]
