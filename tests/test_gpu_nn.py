"""Learned initial-pose proposal: the hand-written forward, backward and Adam
kernels against the FP64 oracle network (oracle/nn.py) evaluated with the same
BF16-rounded weights, training on the GPU, and the proposal stage of the
batched tracker against an FP64 composition of the oracle network's output.

Tolerances: outputs within 1e-4 (relative to max(1, |y|)); per-layer gradient
norms within 1e-3 relative (FP32 sums over up to 1286 products and 256 batch
rows against FP64); one Adam update within 1e-3 of the learning rate."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def glt():
    import paper_2607_16897_gb300 as g
    return g


@pytest.fixture(scope="module")
def onn():
    from oracle import nn
    return nn


def make_params(onn, seed):
    rng = np.random.default_rng(seed)
    p = onn.init_params(seed)
    for name, shape in onn.SHAPES:
        if name.endswith(".b"):
            p[name] = rng.normal(0.0, 0.05, size=shape)
    return onn.flatten(p).astype(np.float32)


def make_inputs(B, seed):
    rng = np.random.default_rng(seed)
    # residual images: integer gray differences / 64, as the proposal stage forms them
    x = (rng.integers(-48, 49, size=(B, 1200)) / 64.0).astype(np.float32)
    m = rng.normal(size=(B, 6)).astype(np.float32)
    t = rng.normal(size=(B, 8)).astype(np.float32)
    return x, m, t


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("B", [1, 7, 256])
def test_forward_matches_oracle(glt, onn, B):
    import torch
    w = make_params(onn, 3)
    x, m, _ = make_inputs(B, 10 + B)
    net = glt.NN(256, w)
    y = torch.zeros(B, 8, device="cuda")
    net.forward(dev(x), dev(m), y, B)
    torch.cuda.synchronize()
    yo, _ = onn.forward(onn.unflatten(onn.to_bf16(w)), x.reshape(B, 1, 30, 40), m)
    err = np.abs(y.cpu().numpy() - yo).max()
    assert err <= 1e-4 * max(1.0, np.abs(yo).max()), err
    net.close()


def test_gradient_matches_oracle(glt, onn):
    B = 64
    w = make_params(onn, 5)
    x, m, t = make_inputs(B, 21)
    net = glt.NN(B, w)
    g, loss = net.gradient(dev(x), dev(m), dev(t), B)
    p = onn.unflatten(onn.to_bf16(w))
    y, cache = onn.forward(p, x.reshape(B, 1, 30, 40), m)
    go, _, _ = onn.backward(p, cache, y, t)
    assert abs(loss - onn.loss(y, t)) <= 1e-5 * onn.loss(y, t)
    gg = onn.unflatten(g.astype(np.float64))
    for name, _ in onn.SHAPES:
        ref = np.linalg.norm(go[name])
        assert ref > 0, name
        rel = np.linalg.norm(gg[name] - go[name]) / ref
        assert rel <= 1e-3, (name, rel)
    # a plausible slip (one layer's gradient transposed or dropped) is far outside
    assert np.linalg.norm(gg["fc2.b"] - go["fc2.b"]) < 0.1 * np.linalg.norm(go["fc2.b"])
    net.close()


def test_gradient_is_deterministic(glt, onn):
    B = 256
    w = make_params(onn, 6)
    x, m, t = make_inputs(B, 22)
    net = glt.NN(B, w)
    g1, l1 = net.gradient(dev(x), dev(m), dev(t), B)
    g2, l2 = net.gradient(dev(x), dev(m), dev(t), B)
    assert np.array_equal(g1, g2) and l1 == l2
    net.close()


def test_adam_steps_match_oracle(glt, onn):
    """Two Adam steps on the GPU against the oracle's Adam fed the GPU
    gradients (which the gradient test pins separately)."""
    import torch
    B, lr = 32, 1e-3
    w0 = make_params(onn, 7)
    x, m, t = make_inputs(B, 23)
    xd, md, td = dev(x), dev(m), dev(t)
    net = glt.NN(B, w0)
    g0, _ = net.gradient(xd, md, td, B)
    loss = torch.zeros(1, device="cuda")
    net.train_step(xd, md, td, B, lr, loss)
    g1, _ = net.gradient(xd, md, td, B)
    net.train_step(xd, md, td, B, lr, loss)
    w2 = net.get_params()
    p = onn.unflatten(w0.astype(np.float64))
    state = {}
    p = onn.adam_step(p, onn.unflatten(g0.astype(np.float64)), state, lr=lr)
    p = onn.adam_step(p, onn.unflatten(g1.astype(np.float64)), state, lr=lr)
    ref = onn.flatten(p)
    moved = np.abs(ref - w0) > 0.5 * lr
    assert moved.mean() > 0.3          # Adam moves most weights by about lr per step
    err = np.abs(w2.astype(np.float64) - ref).max()
    assert err <= 1e-3 * lr, err
    net.close()


def test_training_reduces_loss(glt, onn):
    """Regression onto a fixed random teacher network: 300 Adam steps on the
    GPU cut the loss by more than half."""
    import torch
    B = 256
    x, m, _ = make_inputs(B, 24)
    teacher = make_params(onn, 8)
    yt, _ = onn.forward(onn.unflatten(onn.to_bf16(teacher)), x.reshape(B, 1, 30, 40), m)
    yt = yt.astype(np.float32)
    net = glt.NN(B, make_params(onn, 9))
    xd, md, td = dev(x), dev(m), dev(yt)
    losses = torch.zeros(300, device="cuda")
    for k in range(300):
        net.train_step(xd, md, td, B, 1e-3, losses[k:k + 1])
    ls = losses.cpu().numpy()
    assert np.all(np.isfinite(ls))
    assert ls[-10:].mean() < 0.5 * ls[:3].mean(), (ls[:3], ls[-10:])
    net.close()


def test_nn_argument_errors(glt, onn):
    import torch
    net = glt.NN(4)
    with pytest.raises(glt.GltError):
        net.set_params(np.zeros(10, np.float32))
    x = torch.zeros(8, 1200, device="cuda")
    m = torch.zeros(8, 6, device="cuda")
    y = torch.zeros(8, 8, device="cuda")
    with pytest.raises(glt.GltError):
        net.forward(x, m, y, 8)                # batch above max_batch
    with pytest.raises(glt.GltError):
        net.forward(x, m, y, 0)
    with pytest.raises(glt.GltError):
        glt.NN(0)
    net.close()


def test_proposal_stage_composes_network_output(glt, onn, orc, syn):
    """With every level's iteration budget at zero the batched tracker returns
    its initial state, so the output is the proposal itself:
    T_init exp(0.01 y[0:6]), a + 0.01 y[6], b + y[7] with y the network on the
    coarsest-level residual image (cur - ref) / 64 and the motion input
    log(M) / 0.02 the stage computes from each stream's inter-frame motion M
    (the oracle's SE(3) log on the other side; one M near a half turn takes
    the log's other branch, one is the identity)."""
    import torch
    specs = [(640, 480, 525.0, 5), (320, 240, 256.0, 4), (640, 480, 600.0, 5)]
    w = make_params(onn, 11)
    net = glt.NN(8, w)
    trks, curs, xs, inits = [], [], [], []
    rng = np.random.default_rng(4)
    for i, (W, H, f, L) in enumerate(specs):
        cam = syn.camera_for(W, H, f)
        seq = syn.sequence(700 + i, 6, cam, syn.ROOM_LARGE, 1.0, 45.0)
        ref, uvd = syn.reference_points(seq, 0, 300, 0.5, 8.0)
        cur, _ = seq.frame(4)
        trk = glt.Tracker(W, H, cam.K, levels=L, max_points=300, max_iters=[0] * 8)
        trk.build_pyramid(glt.GLT_REF, ref)
        trk.set_map_points(uvd)
        trks.append(trk)
        curs.append(torch.from_numpy(cur).cuda())
        xs.append((orc.pyramid(cur, L)[-1].astype(np.float64)
                   - orc.pyramid(ref, L)[-1].astype(np.float64)) / 64.0)
        T = syn.relative(seq.T_wc[0], seq.T_wc[3])
        inits.append(np.concatenate([T.ravel(), rng.normal(0, 0.05, 1), rng.normal(0, 3, 1)]))
    S = len(specs)
    twists = [rng.normal(0, 0.02, 6), np.array([0.01, -0.02, 0.03, 0.0, 0.0, 3.1415]), np.zeros(6)]
    Ms = [orc.se3_exp(t) for t in twists]
    batch = glt.Batch(trks)
    md = torch.tensor(np.stack([M.ravel() for M in Ms]), dtype=torch.float64).cuda()
    batch.set_proposal(net, md)
    motion = np.stack([onn.motion_input(M) for M in Ms])
    ptrs = torch.tensor([c.data_ptr() for c in curs], dtype=torch.int64).cuda()
    init = torch.tensor(np.stack(inits), dtype=torch.float64).cuda()
    out = torch.zeros(S * glt.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    st = torch.cuda.Stream()
    batch.capture(ptrs, init, out, st)
    batch.replay(stream=st)
    st.synchronize()
    res = glt.parse_results(out)
    y, _ = onn.forward(onn.unflatten(onn.to_bf16(w)), np.stack(xs)[:, None], motion)
    for s in range(S):
        d = y[s] * np.array([0.01] * 7 + [1.0])
        Te = orc.se3_mul(inits[s][:12].reshape(3, 4), orc.se3_exp(d[:6]))
        assert np.abs(res[s]["T"] - Te).max() <= 1e-6, s
        assert abs(res[s]["a"] - (inits[s][12] + d[6])) <= 1e-6
        assert abs(res[s]["b"] - (inits[s][13] + d[7])) <= 1e-4
    # detaching restores the plain initial state
    batch.set_proposal(None, None)
    batch.build_pyramid(ptrs)
    batch.track(init, out)
    torch.cuda.synchronize()
    for s, r in enumerate(glt.parse_results(out)):
        assert np.abs(r["T"] - inits[s][:12].reshape(3, 4)).max() <= 1e-12
    # a stream whose coarsest level is not 40 x 30 is refused
    t2 = glt.Tracker(640, 480, syn.camera_for(640, 480, 525.0).K, levels=4, max_points=10)
    b2 = glt.Batch([t2])
    with pytest.raises(glt.GltError):
        b2.set_proposal(net, md)
    b2.close()
    t2.close()
    batch.close()
    for t in trks:
        t.close()
    net.close()


def test_checkpoint_resumes_training_bit_for_bit(glt, onn, tmp_path):
    """Weights, Adam moments and step count go through glt_nn_save /
    glt_nn_load: training resumed from a checkpoint reproduces the
    uninterrupted run exactly (the kernels are deterministic)."""
    import torch
    B, lr = 64, 1e-3
    x, m, t = make_inputs(B, 31)
    xd, md, td = dev(x), dev(m), dev(t)
    a = glt.NN(B, make_params(onn, 12))
    for _ in range(3):
        a.train_step(xd, md, td, B, lr)
    ck = str(tmp_path / "net.ckpt")
    a.save(ck)
    assert (tmp_path / "net.ckpt").stat().st_size == 16 + 3 * 4 * glt.GLT_NN_PARAMS
    for _ in range(2):
        a.train_step(xd, md, td, B, lr)
    b = glt.NN(B)
    b.load(ck)
    for _ in range(2):
        b.train_step(xd, md, td, B, lr)
    assert np.array_equal(a.get_params(), b.get_params())
    # a fresh Adam state (weights only) gives a different trajectory
    c = glt.NN(B)
    c.set_params(np.zeros(glt.GLT_NN_PARAMS, np.float32))
    c.load(ck)
    w3 = c.get_params()
    c.set_params(w3)                 # resets the moments and the step count
    for _ in range(2):
        c.train_step(xd, md, td, B, lr)
    assert not np.array_equal(a.get_params(), c.get_params())
    for n in (a, b, c):
        n.close()


def test_load_npy_weights(glt, onn, tmp_path):
    import torch
    w = make_params(onn, 5)
    p = tmp_path / "w.npy"
    np.save(p, w)
    B = 7
    x, m, _ = make_inputs(B, 41)
    a, b = glt.NN(B, w), glt.NN(B)
    b.load(str(p))
    assert np.array_equal(b.get_params(), w)
    ya, yb = torch.zeros(B, 8, device="cuda"), torch.zeros(B, 8, device="cuda")
    a.forward(dev(x), dev(m), ya, B)
    b.forward(dev(x), dev(m), yb, B)
    torch.cuda.synchronize()
    assert torch.equal(ya, yb)
    # the committed proposal weights load the same way
    from paper_2607_16897_gb300 import proposal
    b.load(proposal.WEIGHTS_PATH)
    assert np.array_equal(b.get_params(), proposal.load_weights())
    # errors: missing file, wrong size, wrong dtype, not a weight file
    with pytest.raises(glt.GltError, match=r"\(-6\)"):
        b.load(str(tmp_path / "missing.npy"))
    np.save(tmp_path / "short.npy", w[:100])
    np.save(tmp_path / "f64.npy", w.astype(np.float64))
    (tmp_path / "junk.bin").write_bytes(b"0123456789abcdef")
    for bad in ("short.npy", "f64.npy", "junk.bin"):
        with pytest.raises(glt.GltError, match=r"\(-1\)"):
            b.load(str(tmp_path / bad))
    (tmp_path / "trunc.npy").write_bytes((tmp_path / "w.npy").read_bytes()[:4096])
    with pytest.raises(glt.GltError, match=r"\(-6\)"):
        b.load(str(tmp_path / "trunc.npy"))
    assert np.array_equal(b.get_params(), proposal.load_weights())   # failed loads change nothing
    a.close()
    b.close()


def test_training_loop_resumes_from_its_checkpoint(glt, onn, tmp_path):
    """proposal.train with a checkpoint: stopped after one epoch and called
    again, it ends where the uninterrupted two-epoch run ends."""
    from paper_2607_16897_gb300 import proposal
    S, per = 20, 40
    x, m, t = make_inputs(S * per, 51)
    data = dict(x=x, m=m, t=t * 0.1, seq=np.repeat(np.arange(S), per), S=S)
    kw = dict(batch=64, lr=1e-3, eval_every=5, seed=3, log=None)
    w_full, info_full = proposal.train(data, epochs=2, **kw)
    ck = str(tmp_path / "train.ckpt")
    proposal.train(data, epochs=1, checkpoint=ck, **kw)
    w_res, info_res = proposal.train(data, epochs=2, checkpoint=ck, **kw)
    assert np.array_equal(w_full, w_res)
    assert info_full["best_step"] == info_res["best_step"]
    assert [tuple(h) for h in info_full["history"]] == info_res["history"]


def test_proposal_form_at_full_size_matches_oracle(glt, onn, orc, syn):
    """Two streams of the learned-proposal workload (640x480, 2000 points,
    5 levels, fast motion), 6 frames each: the batch with the trained network
    in front of the LM against the FP64 oracle network and the oracle tracker,
    from the same constant-velocity starts and inter-frame motions."""
    import torch
    from paper_2607_16897_gb300.proposal import load_weights
    from synth.jobs import stream_motion
    from helpers import I34, pose_diff
    w = load_weights()
    pw = onn.unflatten(onn.to_bf16(w))
    net = glt.NN(2, w)
    S, N, L = 2, 2000, 5
    cam = syn.camera_for(640, 480, 525.0)
    seqs, trks, orcs, refs = [], [], [], []
    for s in range(S):
        v, a = stream_motion(5000 + s)
        seq = syn.sequence(5000 + s, 24, cam, syn.ROOM_LARGE, v, a)
        ref, uvd = syn.reference_points(seq, 0, N, 0.5, 8.0)
        t = glt.Tracker(640, 480, cam.K, levels=L, max_points=N)
        t.build_pyramid(glt.GLT_REF, ref)
        t.set_map_points(uvd)
        o = orc.OracleTracker(640, 480, cam.K, levels=L)
        o.build_pyramid(0, ref)
        o.set_map_points(uvd)
        seqs.append(seq)
        trks.append(t)
        orcs.append(o)
        refs.append(orc.pyramid(ref, L)[-1].astype(np.float64))
    batch = glt.Batch(trks)
    motion = torch.zeros((S, 12), dtype=torch.float64, device="cuda")
    batch.set_proposal(net, motion)
    init = torch.zeros((S, 14), dtype=torch.float64, device="cuda")
    out = torch.zeros(S * glt.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    T_prev = [I34] * S
    T_pp = [None] * S
    ab = [(0.0, 0.0)] * S
    for k in range(1, 7):
        curs = [torch.from_numpy(seq.frame(k)[0]).cuda() for seq in seqs]
        ptrs = torch.tensor([c.data_ptr() for c in curs], dtype=torch.int64, device="cuda")
        Ms = [syn.pose_mul(T_prev[s], syn.pose_inv(T_pp[s])) if T_pp[s] is not None else I34
              for s in range(S)]
        T0 = [syn.pose_mul(Ms[s], T_prev[s]) for s in range(S)]
        init.copy_(torch.tensor(np.stack([np.concatenate([T0[s].ravel(), ab[s]]) for s in range(S)])))
        motion.copy_(torch.tensor(np.stack([M.ravel() for M in Ms])))
        batch.build_pyramid(ptrs)
        batch.track(init, out)
        torch.cuda.synchronize()
        res = glt.parse_results(out)
        for s in range(S):
            cur = curs[s].cpu().numpy()
            x = (orc.pyramid(cur, L)[-1].astype(np.float64) - refs[s]) / 64.0
            y, _ = onn.forward(pw, x[None, None], onn.motion_input(Ms[s])[None])
            Tp, abp = onn.apply_output(T0[s], ab[s], y[0])
            orcs[s].build_pyramid(1, cur)
            r = orcs[s].track_frame(Tp, abp)
            ang, dt = pose_diff(res[s]["T"], r["T"])
            assert ang <= 1e-5 and dt <= 1e-5, (s, k, ang, dt)
            assert abs(res[s]["a"] - r["a"]) <= 1e-5 and abs(res[s]["b"] - r["b"]) <= 1e-3
            assert res[s]["status"] == r["status"] == 0
            T_pp[s], T_prev[s], ab[s] = T_prev[s], res[s]["T"], (res[s]["a"], res[s]["b"])
    batch.close()
    for t in trks:
        t.close()
    net.close()
