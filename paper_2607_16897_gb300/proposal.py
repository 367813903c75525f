"""Learned initial-pose proposal: host-side features, training-set generation
and the training loop.  The network, its training kernels and the proposal
stage of the batched tracker are CUDA (``glt_nn_*``, ``glt_batch_set_proposal``);
this module only prepares inputs and drives them.

The paper seeds every frame with a constant-velocity guess and has no learned
part; the proposal is this library's addition.  What it computes:

* input 1: the coarsest-level (40 x 30) residual image at the identity warp,
  (I_cur - I_ref) / 64, formed on the device by the proposal stage;
* input 2: the previous inter-frame motion: the SE(3) log of the last tracked
  camera motion (x_{k-1} = M x_{k-2}) divided by 0.02, computed on the device
  by the proposal stage from M itself (``motion_feature`` computes the same
  value on the host for the training set);
* output: y (8 values), increment delta = (0.01 y[0:7], y[7]) applied as
  T' = T_init exp(delta[0:6]), a' = a + delta[6], b' = b + delta[7].

Training pairs come from the plain tracker on seeded synthetic sequences:
the label of a frame is the pose and affine pair the plain batched tracker
converges to when started from the renderer's true relative pose (the basin
the constant-velocity start is meant to reach), and the input state is the
constant-velocity start the sequence driver would use, built from the
previous frames' labels.  Target t = (log(T_init^-1 T_conv) / 0.01,
(a_conv - a_init) / 0.01, b_conv - b_init).
"""
from __future__ import annotations

import os
import time

import numpy as np

MOTION_SCALE = 0.02
OUT_SCALE = np.array([0.01] * 7 + [1.0])
WEIGHTS_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "proposal_weights.npy")
TRAIN_SEED0 = 10_000       # training sequences use seeds >= 10000
TEST_SEED0 = 5_000         # held-out sequences 5000..5255
N_PARAMS = 189064          # GLT_NN_PARAMS


# ---------------------------------------------------------------------------
# SE(3) on the host (inputs and labels only)
# ---------------------------------------------------------------------------
def pose_mul(A, B):
    return np.hstack([A[:, :3] @ B[:, :3], (A[:, :3] @ B[:, 3] + A[:, 3])[:, None]])


def pose_inv(A):
    R = A[:, :3].T
    return np.hstack([R, (-R @ A[:, 3])[:, None]])


def se3_log(T) -> np.ndarray:
    """(v, w) with exp(v, w) = T; rotation angle below pi.  Closed form of the
    SO(3) log (axis from the skew part, angle by atan2) and V^-1 = I - W/2 +
    (1/th^2)(1 - A/(2B)) W^2, with A = sin th / th, B = (1 - cos th) / th^2,
    and its Taylor series 1/12 + th^2/720 + th^4/30240 for small th."""
    T = np.asarray(T, np.float64).reshape(3, 4)
    R, t = T[:, :3], T[:, 3]
    s = 0.5 * np.array([R[2, 1] - R[1, 2], R[0, 2] - R[2, 0], R[1, 0] - R[0, 1]])
    c = 0.5 * (np.trace(R) - 1.0)
    sn = np.linalg.norm(s)
    th = np.arctan2(sn, c)
    if sn < 1e-12:
        w = s.copy()
    else:
        w = s * (th / sn)
    W = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])
    th2 = th * th
    if th < 1e-3:
        k = 1.0 / 12.0 + th2 / 720.0 + th2 * th2 / 30240.0
    else:
        A = np.sin(th) / th
        B = (1.0 - np.cos(th)) / th2
        k = (1.0 - A / (2.0 * B)) / th2
    Vinv = np.eye(3) - 0.5 * W + k * (W @ W)
    return np.concatenate([Vinv @ t, w])


def motion_feature(Tw_prev, Tw_prevprev) -> np.ndarray:
    """Network motion input from two world->camera poses (None: zeros)."""
    if Tw_prev is None or Tw_prevprev is None:
        return np.zeros(6, np.float32)
    M = pose_mul(Tw_prev, pose_inv(Tw_prevprev))
    return (se3_log(M) / MOTION_SCALE).astype(np.float32)


def target(T_init, ab_init, T_conv, ab_conv) -> np.ndarray:
    xi = se3_log(pose_mul(pose_inv(np.asarray(T_init).reshape(3, 4)),
                          np.asarray(T_conv).reshape(3, 4)))
    d = np.concatenate([xi, [ab_conv[0] - ab_init[0], ab_conv[1] - ab_init[1]]])
    return (d / OUT_SCALE).astype(np.float32)


def orthonormalised(T):
    q0 = T[0, :3] / np.linalg.norm(T[0, :3])
    q1 = T[1, :3] - (T[1, :3] @ q0) * q0
    q1 = q1 / np.linalg.norm(q1)
    out = np.array(T, np.float64, copy=True)
    out[:, :3] = np.stack([q0, q1, np.cross(q0, q1)])
    return out


def load_weights(path: str = WEIGHTS_PATH) -> np.ndarray:
    w = np.load(path).astype(np.float32)
    if w.size != N_PARAMS:
        raise ValueError(f"{path}: {w.size} values, expected {N_PARAMS}")
    return w


# ---------------------------------------------------------------------------
# synthetic sequences: rendered in worker processes by the input generator
# ---------------------------------------------------------------------------
from synth.jobs import _render_job, _sequence, render_pool, stream_motion  # noqa: E402,F401


# ---------------------------------------------------------------------------
# training set
# ---------------------------------------------------------------------------
def generate(seeds, frames=224, W=640, H=480, f=525.0, N=2000, L=5, interval=8, pool=None,
             log=print):
    """Runs every sequence of `seeds` through the plain batched tracker (one
    stream per seed, one batch step per frame) and returns the training
    arrays x [P, 1200], m [P, 6], t [P, 8] plus statistics.  A frame k with
    k % interval == 0 is a reference (its map points from the renderer's depth),
    every other frame one training pair against the latest reference."""
    import torch
    from . import GLT_CUR, GLT_REF, Batch, Tracker, RESULT_BYTES, parse_results
    import synth

    seeds = list(seeds)
    S = len(seeds)
    own_pool = pool is None
    if own_pool:
        pool = render_pool()
    cam = synth.camera_for(W, H, f)
    seqs = [_sequence(s, frames, W, H, f) for s in seeds]
    trks = [Tracker(W, H, cam.K, levels=L, max_points=N) for _ in seeds]
    batch = Batch(trks)
    cur = [torch.empty((H, W), dtype=torch.uint8, device="cuda") for _ in seeds]
    ptrs = torch.tensor([c.data_ptr() for c in cur], dtype=torch.int64, device="cuda")
    init = torch.zeros((S, 14), dtype=torch.float64, device="cuda")
    out = torch.zeros(S * RESULT_BYTES, dtype=torch.uint8, device="cuda")
    xs, ms, ts, seq_of = [], [], [], []
    Tw = [dict() for _ in seeds]       # world->camera estimates per frame
    ab = [(0.0, 0.0)] * S
    ref_k = [0] * S
    ref_coarse = [None] * S
    dropped = 0
    t0 = time.time()
    for k in range(frames):
        is_ref = k % interval == 0
        jobs = [(s, frames, W, H, f, k, N if is_ref else 0) for s in seeds]
        rendered = pool.map(_render_job, jobs)
        if is_ref:
            for i, (img, uvd) in enumerate(rendered):
                trks[i].build_pyramid(GLT_REF, img)
                trks[i].set_map_points(uvd)
                ref_coarse[i] = trks[i].get_pyramid(GLT_REF, L - 1).astype(np.float32)
                ref_k[i] = k
                Tw[i][k] = pose_inv(seqs[i].T_wc[k])
                ab[i] = (0.0, 0.0)
            continue
        T_init, ab_init, mot = [], [], []
        gt = np.zeros((S, 14))
        for i in range(S):
            Tref = Tw[i][ref_k[i]]
            Tp = Tw[i][k - 1]
            Tpp = Tw[i].get(k - 2)
            M = pose_mul(Tp, pose_inv(Tpp)) if Tpp is not None else np.hstack([np.eye(3), np.zeros((3, 1))])
            T_init.append(pose_mul(pose_mul(M, Tp), pose_inv(Tref)))
            ab_init.append(ab[i])
            mot.append(motion_feature(Tp, Tpp))
            Tt = synth.relative(seqs[i].T_wc[ref_k[i]], seqs[i].T_wc[k])
            a_t, b_t = seqs[i].rel_affine(ref_k[i], k)
            gt[i] = np.concatenate([Tt.ravel(), [a_t, b_t]])
            cur[i].copy_(torch.from_numpy(rendered[i][0]))
        init.copy_(torch.from_numpy(gt))
        batch.build_pyramid(ptrs)
        batch.track(init, out)
        torch.cuda.synchronize()
        res = parse_results(out)
        for i in range(S):
            r = res[i]
            Tt = gt[i, :12].reshape(3, 4)
            dR = r["T"][:, :3].T @ Tt[:, :3]
            ang = np.arccos(np.clip(0.5 * (np.trace(dR) - 1.0), -1.0, 1.0))
            ok = r["status"] == 0 and ang < np.deg2rad(0.5) and np.linalg.norm(r["T"][:, 3] - Tt[:, 3]) < 0.02
            T_conv = r["T"] if ok else Tt
            ab_conv = (r["a"], r["b"]) if ok else (gt[i, 12], gt[i, 13])
            if ok:
                coarse = trks[i].get_pyramid(GLT_CUR, L - 1).astype(np.float32)
                xs.append(((coarse - ref_coarse[i]) / 64.0).ravel())
                ms.append(mot[i])
                ts.append(target(T_init[i], ab_init[i], T_conv, ab_conv))
                seq_of.append(i)
            else:
                dropped += 1
            Tw[i][k] = orthonormalised(pose_mul(T_conv, Tw[i][ref_k[i]]))
            ab[i] = ab_conv
            if k - 3 != ref_k[i]:
                Tw[i].pop(k - 3, None)
        if log and (k % 32 == 1 or k == frames - 1):
            log(f"frame {k}/{frames}: {len(ts)} pairs, {dropped} dropped, {time.time() - t0:.0f} s")
    batch.close()
    for t in trks:
        t.close()
    if own_pool:
        pool.close()
        pool.join()
    return dict(x=np.stack(xs).astype(np.float32), m=np.stack(ms).astype(np.float32),
                t=np.stack(ts).astype(np.float32), seq=np.array(seq_of, np.int32), S=S,
                dropped=dropped)


# ---------------------------------------------------------------------------
# training
# ---------------------------------------------------------------------------
def init_params(seed=0) -> np.ndarray:
    """He-uniform weights, zero biases, last layer scaled by 0.1 (the start
    proposes nearly the constant-velocity state)."""
    shapes = [(16, 1, 3, 3), (16,), (32, 16, 3, 3), (32,), (64, 32, 3, 3), (64,),
              (128, 1286), (128,), (8, 128), (8,)]
    rng = np.random.default_rng(seed)
    parts = []
    for i, sh in enumerate(shapes):
        if len(sh) == 1:
            parts.append(np.zeros(sh))
        else:
            lim = np.sqrt(6.0 / np.prod(sh[1:]))
            parts.append(rng.uniform(-lim, lim, size=sh) * (0.1 if i == 8 else 1.0))
    w = np.concatenate([p.ravel() for p in parts]).astype(np.float32)
    assert w.size == N_PARAMS
    return w


def train(data, epochs=20, batch=256, lr=3e-4, val_frac=0.1, eval_every=50, seed=0, log=print,
          checkpoint=None):
    """Adam on the GPU with the library's training kernels; returns (params,
    summary).  The pairs of the last `val_frac` of the sequences are held out;
    the parameters with the lowest held-out loss (evaluated every
    `eval_every` steps) are returned.

    `checkpoint` (a path): after every epoch the network's checkpoint
    (weights, Adam moments and step, glt_nn_save) goes to that path, the best
    weights to `<path>.best.npy` and the loop state (epoch, shuffling RNG,
    history) to `<path>.json`; a call that finds them resumes after the last
    finished epoch and ends with the same result as an uninterrupted run."""
    import json

    import torch
    from . import NN
    x, m, t, seq = data["x"], data["m"], data["t"], data["seq"]
    cut = int(round((1.0 - val_frac) * data["S"]))
    tr_idx = np.nonzero(seq < cut)[0]
    va_idx = np.nonzero(seq >= cut)[0]
    ntr, nval = len(tr_idx), len(va_idx)
    xd = torch.from_numpy(x[tr_idx]).cuda()
    md = torch.from_numpy(m[tr_idx]).cuda()
    td = torch.from_numpy(t[tr_idx]).cuda()
    xv = torch.from_numpy(x[va_idx]).cuda()
    mv = torch.from_numpy(m[va_idx]).cuda()
    tv = torch.from_numpy(t[va_idx]).cuda()
    net = NN(max(batch, nval), init_params(seed))
    rng = np.random.default_rng(seed)
    steps = ntr // batch
    loss_dev = torch.zeros(steps, device="cuda")
    yv = torch.zeros((nval, 8), device="cuda")
    base = float(0.5 * np.mean(np.sum(t[va_idx] ** 2, axis=1)))

    def val_loss():
        net.forward(xv, mv, yv, nval)
        torch.cuda.synchronize()
        return float(0.5 * torch.mean(torch.sum((yv - tv) ** 2, dim=1)))

    best, best_w, best_at = val_loss(), net.get_params(), 0
    hist = []
    start = 0
    if checkpoint and os.path.exists(checkpoint + ".json"):
        with open(checkpoint + ".json") as f:
            saved = json.load(f)
        net.load(checkpoint)
        best_w = np.load(checkpoint + ".best.npy")
        best, best_at, start = saved["best"], saved["best_at"], saved["epoch"] + 1
        hist = [tuple(h) for h in saved["history"]]
        rng.bit_generator.state = saved["rng"]
    for ep in range(start, epochs):
        perm = torch.from_numpy(rng.permutation(ntr)).cuda()
        for s in range(steps):
            idx = perm[s * batch:(s + 1) * batch]
            net.train_step(xd[idx].contiguous(), md[idx].contiguous(), td[idx].contiguous(), batch,
                           lr, loss_dev[s:s + 1])
            if (s + 1) % eval_every == 0 or s == steps - 1:
                vl = val_loss()
                if vl < best:
                    best, best_w, best_at = vl, net.get_params(), ep * steps + s + 1
        tl = float(loss_dev.mean())
        hist.append((tl, vl))
        if checkpoint:
            net.save(checkpoint)
            np.save(checkpoint + ".best.npy", best_w)
            with open(checkpoint + ".json", "w") as f:
                json.dump(dict(epoch=ep, best=best, best_at=best_at, history=hist,
                               rng=rng.bit_generator.state), f)
        if log:
            log(f"epoch {ep}: train {tl:.4f} val {vl:.4f} best {best:.4f} at step {best_at} "
                f"(zero proposal {base:.4f})")
    net.close()
    return best_w, dict(history=hist, zero_val=base, best_val=best, best_step=best_at,
                        train_pairs=ntr, val_pairs=nval, val_sequences=data["S"] - cut)


def evaluate(weights, seeds, frames=16, W=640, H=480, f=525.0, N=2000, L=5, interval=8,
             pool=None):
    """Paired comparison on the given sequences: every frame is tracked from
    the same constant-velocity start (the plain form's sequence driver) by the
    plain tracker, by the tracker behind the proposal stage, and by the
    proposal stage alone (no LM iterations), so the returned statistics isolate
    what the proposal changes: the distance of its start from the converged
    state against that of the constant-velocity start (|log(T0^-1 T)| of the
    pose part, in units of 0.01), the linearisation passes, and the agreement
    of the final poses."""
    import torch
    from . import GLT_REF, NN, Batch, Tracker, RESULT_BYTES, parse_results
    import synth

    seeds = list(seeds)
    S = len(seeds)
    own_pool = pool is None
    if own_pool:
        pool = render_pool()
    cam = synth.camera_for(W, H, f)
    seqs = [_sequence(s, frames, W, H, f) for s in seeds]
    forms = {"plain": {}, "proposal": {}, "init": {"max_iters": [0] * 8}}
    trk = {k: [Tracker(W, H, cam.K, levels=L, max_points=N, **kw) for _ in seeds]
           for k, kw in forms.items()}
    batches = {k: Batch(trk[k]) for k in forms}
    net = NN(S, weights)
    motion = torch.zeros((S, 12), dtype=torch.float64, device="cuda")   # M per stream
    batches["proposal"].set_proposal(net, motion)
    batches["init"].set_proposal(net, motion)
    cur = [torch.empty((H, W), dtype=torch.uint8, device="cuda") for _ in seeds]
    ptrs = torch.tensor([c.data_ptr() for c in cur], dtype=torch.int64, device="cuda")
    init = torch.zeros((S, 14), dtype=torch.float64, device="cuda")
    out = torch.zeros(S * RESULT_BYTES, dtype=torch.uint8, device="cuda")
    Tw = [dict() for _ in seeds]
    ab = [(0.0, 0.0)] * S
    ref_k = [0] * S
    rows = []
    for k in range(frames):
        is_ref = k % interval == 0
        rendered = pool.map(_render_job, [(s, frames, W, H, f, k, N if is_ref else 0) for s in seeds])
        if is_ref:
            for i, (img, uvd) in enumerate(rendered):
                for form in forms:
                    trk[form][i].build_pyramid(GLT_REF, img)
                    trk[form][i].set_map_points(uvd)
                ref_k[i] = k
                Tw[i][k] = pose_inv(seqs[i].T_wc[k])
                ab[i] = (0.0, 0.0)
            continue
        starts, mot = [], []
        for i in range(S):
            Tp, Tpp = Tw[i][k - 1], Tw[i].get(k - 2)
            M = pose_mul(Tp, pose_inv(Tpp)) if Tpp is not None else np.hstack([np.eye(3), np.zeros((3, 1))])
            starts.append(np.concatenate([pose_mul(pose_mul(M, Tp), pose_inv(Tw[i][ref_k[i]])).ravel(),
                                          list(ab[i])]))
            mot.append(M.ravel())
            cur[i].copy_(torch.from_numpy(rendered[i][0]))
        init.copy_(torch.from_numpy(np.stack(starts)))
        motion.copy_(torch.from_numpy(np.stack(mot)))
        res = {}
        for form in forms:
            batches[form].build_pyramid(ptrs)
            batches[form].track(init, out)
            torch.cuda.synchronize()
            res[form] = parse_results(out)
        for i in range(S):
            rp, rq, r0 = res["plain"][i], res["proposal"][i], res["init"][i]
            T_conv = rp["T"]
            e_cv = np.linalg.norm(se3_log(pose_mul(pose_inv(starts[i][:12].reshape(3, 4)), T_conv)))
            e_nn = np.linalg.norm(se3_log(pose_mul(pose_inv(r0["T"]), T_conv)))
            dR = rp["T"][:, :3].T @ rq["T"][:, :3]
            ang = float(np.arccos(np.clip(0.5 * (np.trace(dR) - 1.0), -1.0, 1.0)))
            rows.append((e_cv / 0.01, e_nn / 0.01, rp["passes"], rq["passes"], ang,
                         float(np.linalg.norm(rp["T"][:, 3] - rq["T"][:, 3]))))
            Tw[i][k] = orthonormalised(pose_mul(T_conv, Tw[i][ref_k[i]]))
            ab[i] = (rp["a"], rp["b"])
            if k - 3 != ref_k[i]:
                Tw[i].pop(k - 3, None)
    for form in forms:
        batches[form].close()
        for t in trk[form]:
            t.close()
    net.close()
    if own_pool:
        pool.close()
        pool.join()
    a = np.array(rows)
    return dict(frames=len(a), cv_start_err=float(a[:, 0].mean()), proposal_start_err=float(a[:, 1].mean()),
                proposal_closer=float((a[:, 1] < a[:, 0]).mean()),
                passes_plain=float(a[:, 2].mean()), passes_proposal=float(a[:, 3].mean()),
                agree_1e5=float(((a[:, 4] <= 1e-5) & (a[:, 5] <= 1e-5)).mean()),
                max_rot_diff=float(a[:, 4].max()), max_trans_diff=float(a[:, 5].max()))


def main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(description="generate the proposal training set and train it")
    ap.add_argument("--sequences", type=int, default=1024)
    ap.add_argument("--frames", type=int, default=56)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--out", default=WEIGHTS_PATH)
    ap.add_argument("--log", default=None, help="JSON summary file")
    ap.add_argument("--checkpoint", default=None,
                    help="checkpoint path: written every epoch, resumed from if present")
    a = ap.parse_args(argv)
    pool = render_pool()
    t0 = time.time()
    data = generate(range(TRAIN_SEED0, TRAIN_SEED0 + a.sequences), frames=a.frames, pool=pool)
    pool.close()
    pool.join()
    t1 = time.time()
    w, info = train(data, epochs=a.epochs, lr=a.lr, checkpoint=a.checkpoint)
    t2 = time.time()
    np.save(a.out, w)
    summary = dict(info, dropped=data["dropped"], generate_s=t1 - t0, train_s=t2 - t1,
                   target_rms=np.sqrt(np.mean(data["t"] ** 2, axis=0)).tolist())
    print(json.dumps(summary))
    if a.log:
        with open(a.log, "w") as fh:
            json.dump(summary, fh, indent=1)


if __name__ == "__main__":
    main()
