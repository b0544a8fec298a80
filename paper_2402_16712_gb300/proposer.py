"""Learned jhat proposer: training data from exact fits, training with the
library's own network kernels, and evaluation against the full scan.

Algorithm 1 scores every candidate jhat exactly (m of them, each scanning all
k).  The proposer ranks the candidates from four features with a small network
and only the K best-ranked ones are scored exactly; the exact objective still
decides among them, and the full scan is the reference for the regret
(objective lost by missing the best jhat).  The features are three column
statistics (l1 and l2 norms, median |x|) and the objective of Algorithm 1 on
the instance's heaviest rows (l1line_proposer_rows(n) of them), fitted by the
library itself: the objective is dominated by the few rows of large norm.

    python -m paper_2402_16712_gb300.proposer train --out DIR
    python -m paper_2402_16712_gb300.proposer eval [--theta FILE] [--count 200]

Training data: instances of datagen.proposer_spec (n ~ U[500,5000],
m ~ U[100,1000], lambda = 0.2), drawn on the GPU; labels are the exact
objectives z_jhat of every candidate from l1line.scan.  Target of an instance:
softmax of -(z - z_min) / (T (z_(16) - z_min)) with T = 0.25, z_(16) the 16th
smallest objective, so the probability mass sits on the best few candidates;
the network's scores are trained with the listwise cross entropy against it.
Every arithmetic step (features, forward, loss, backward, Adam) runs in the
CUDA library; this module only schedules the calls and keeps the books.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

from . import datagen, l1line

_HERE = os.path.dirname(os.path.abspath(__file__))
THETA_PATH = os.path.join(_HERE, "proposer_theta.f32")
TRAIN_SEEDS = (1, 20000)        # inclusive
VAL_SEEDS = (30001, 30400)      # validation during training (disjoint from both)
VAL_EVAL_SEED0 = 40001           # calibration of K at the evaluation shape
TEMPERATURE, TOP = 0.25, 16
K_DEFAULT = 32


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------
def init_theta(seed: int) -> np.ndarray:
    """He-normal weights, zero biases, in the flat order W1, b1, W2, b2, w3, b3."""
    rng = np.random.default_rng(seed)
    H, F = 128, l1line.MLP_FEATURES
    parts = [rng.normal(0.0, np.sqrt(2.0 / F), H * F), np.zeros(H),
             rng.normal(0.0, np.sqrt(2.0 / H), H * H), np.zeros(H),
             rng.normal(0.0, np.sqrt(1.0 / H), H), np.zeros(1)]
    th = np.concatenate(parts).astype(np.float32)
    assert th.size == l1line.MLP_PARAMS
    return th


def load_theta(path: str = THETA_PATH) -> np.ndarray:
    th = np.fromfile(path, dtype="<f4")
    if th.size != l1line.MLP_PARAMS or not np.isfinite(th).all():
        raise ValueError(f"{path}: not a network parameter file")
    return th


def network(device=None, path: str = THETA_PATH):
    """The trained network's packed image on the device."""
    import torch
    th = torch.from_numpy(load_theta(path)).to(device or "cuda")
    return l1line.mlp_pack(th)


def _targets(z: np.ndarray) -> np.ndarray:
    zs = np.sort(z)
    span = zs[min(TOP, z.size) - 1] - zs[0]
    if not span > 0:
        span = max(abs(zs[0]), 1.0)
    return (-(z - zs[0]) / (TEMPERATURE * span)).astype(np.float32)


# ---------------------------------------------------------------------------
# data
# ---------------------------------------------------------------------------
def build_dataset(seeds, device, log=None):
    """Standardised features [N, 4] and target logits [N] (device, float32),
    instance offsets, and per instance the best jhat and m.  The fits queue
    back to back on the device; the objectives come back to the host once per
    block of instances, where the device status is checked too."""
    import torch
    feats, zs, offs, ms = [], [], [0], []
    t0 = time.time()
    seeds = list(seeds)
    block = 100
    # one workspace per instance of a block, so that every call's device
    # status survives until the block is checked (100 x 48 MB at most)
    ring = []
    for q0 in range(0, len(seeds), block):
        used = []
        for r, seed in enumerate(seeds[q0:q0 + block]):
            spec = datagen.proposer_spec(seed)
            X, _, _ = datagen.planted_torch(spec, device)
            need = int(l1line.load().l1line_proposed_workspace_bytes(l1line.DTYPE_F32, spec.n,
                                                                     spec.m, 1))
            if r == len(ring):
                ring.append(l1line.Workspace(need, device))
            elif ring[r].nbytes < need:
                ring[r] = l1line.Workspace(need, device)
            ws = ring[r]
            # features first: the scan resets the status word and then keeps its own
            _, fz = l1line.features(X, datagen.PROPOSER_LAMBDA, workspace=ws, raw=False)
            _, _, z, _ = l1line.scan(X, [datagen.PROPOSER_LAMBDA], workspace=ws, z_only=True)
            feats.append(fz)
            zs.append(z[0])
            offs.append(offs[-1] + spec.m)
            ms.append(spec.m)
            used.append((seed, ws))
        for seed, ws in used:
            rc = l1line.status(ws)
            if rc != l1line.OK:
                raise l1line.L1LineError(rc, f"training instance {seed}")
        if log and (q0 + block) % 1000 == 0:
            log(f"  {q0 + block} instances labelled ({time.time() - t0:.0f} s)")
    zh = torch.cat(zs).cpu().numpy()
    if not np.isfinite(zh).all():
        raise RuntimeError("a training fit returned a non-finite objective")
    o = np.array(offs, dtype=np.int64)
    tg = np.concatenate([_targets(zh[o[b]:o[b + 1]]) for b in range(len(o) - 1)])
    best = np.array([int(np.argmin(zh[o[b]:o[b + 1]])) for b in range(len(o) - 1)])
    F = torch.cat(feats).contiguous()
    U = torch.from_numpy(tg).to(device)
    return {"feat": F, "tgt": U, "offs": o, "best": best, "m": np.array(ms)}


def _recall(data, mlp, K):
    """Fraction of instances whose exact best jhat is among the network's top K."""
    s = l1line.mlp_forward(data["feat"], mlp).cpu().numpy()
    hit = 0
    o = data["offs"]
    for b in range(len(o) - 1):
        sb = s[o[b]:o[b + 1]]
        kk = min(K, sb.size)
        top = np.argpartition(-sb, kk - 1)[:kk]
        hit += int(data["best"][b] in set(top.tolist()))
    return hit / (len(o) - 1)


# ---------------------------------------------------------------------------
# training
# ---------------------------------------------------------------------------
CHECKPOINT = "checkpoint.npz"


def save_checkpoint(path, config, epoch, step, theta, m1, m2, rng_state, history, best):
    """Training state after `epoch` epochs: parameters, Adam moments, step,
    the permutation generator's state, the history and the best epoch so far.
    Written to a temporary file and renamed, so a crash mid-write leaves the
    previous checkpoint intact."""
    tmp = f"{path}.tmp{os.getpid()}.npz"
    np.savez(tmp, theta=np.asarray(theta, dtype=np.float32), m1=np.asarray(m1, dtype=np.float32),
             m2=np.asarray(m2, dtype=np.float32),
             best_theta=np.asarray(best[2] if best else theta, dtype=np.float32),
             meta=np.array(json.dumps({
                 "config": config, "epoch": int(epoch), "step": int(step),
                 "rng_state": rng_state, "history": history,
                 "best": [best[0], best[1]] if best else None})))
    os.replace(tmp, path)


def load_checkpoint(path, config):
    """The state save_checkpoint wrote, checked against this run's config
    (a checkpoint of another run raises ValueError)."""
    with np.load(path) as d:
        meta = json.loads(str(d["meta"]))
        if meta["config"] != config:
            raise ValueError(f"checkpoint {path} was written by another run: "
                             f"{meta['config']} != {config}")
        best = None
        if meta["best"] is not None:
            best = (meta["best"][0], meta["best"][1], d["best_theta"].copy())
        return {"epoch": meta["epoch"], "step": meta["step"], "theta": d["theta"].copy(),
                "m1": d["m1"].copy(), "m2": d["m2"].copy(), "rng_state": meta["rng_state"],
                "history": meta["history"], "best": best}


def train(out_dir, n_train=None, epochs=24, batch_instances=16, lr=2e-3, seed=0, device=None,
          log=print, resume=False, n_val=None, stop_after=None):
    """Train the proposer network; after every epoch the state goes to
    out_dir/checkpoint.npz.  resume: continue from that checkpoint (same
    configuration), giving the parameters an uninterrupted run gives.
    stop_after: return after that many epochs of this call (for tests)."""
    import torch
    device = device or "cuda"
    os.makedirs(out_dir, exist_ok=True)
    s0, s1 = TRAIN_SEEDS
    if n_train is not None:
        s1 = s0 + n_train - 1
    v0, v1 = VAL_SEEDS
    if n_val is not None:
        v1 = v0 + n_val - 1
    config = {"train_seeds": [s0, s1], "val_seeds": [v0, v1], "epochs": epochs,
              "batch_instances": batch_instances, "lr": lr, "seed": seed}
    ckpt = os.path.join(out_dir, CHECKPOINT)
    state = load_checkpoint(ckpt, config) if resume and os.path.exists(ckpt) else None
    t_start = time.time()
    log(f"labelling {s1 - s0 + 1} training instances with exact fits")
    tr = build_dataset(range(s0, s1 + 1), device, log)
    t_label = time.time() - t_start
    va = build_dataset(range(v0, v1 + 1), device)
    n_inst = len(tr["offs"]) - 1
    N = int(tr["offs"][-1])
    log(f"{n_inst} instances, {N} candidate rows, labelled in {t_label:.0f} s")

    theta = torch.from_numpy(init_theta(seed)).to(device)
    m1, m2 = torch.zeros_like(theta), torch.zeros_like(theta)
    if state is not None:
        theta.copy_(torch.from_numpy(state["theta"]))
        m1.copy_(torch.from_numpy(state["m1"]))
        m2.copy_(torch.from_numpy(state["m2"]))
    mlp = l1line.mlp_pack(theta)
    score = torch.empty(N, dtype=torch.float32, device=device)
    dscore = torch.empty(N, dtype=torch.float32, device=device)
    loss = torch.empty(batch_instances, dtype=torch.float32, device=device)
    grad = torch.empty(l1line.MLP_PARAMS, dtype=torch.float32, device=device)
    max_rows = int(np.max(np.diff(tr["offs"]))) * batch_instances
    mws = l1line.MlpWorkspace(max_rows, device)
    rng = np.random.default_rng(seed + 1)
    sizes = np.diff(tr["offs"])
    steps_per_epoch = (n_inst + batch_instances - 1) // batch_instances
    total_steps = epochs * steps_per_epoch
    history, best = [], None
    step, ep0 = 0, 0
    if state is not None:
        rng.bit_generator.state = state["rng_state"]
        history, best, step, ep0 = state["history"], state["best"], state["step"], state["epoch"]
        log(f"resuming after epoch {ep0} (step {step})")
    t_train = time.time()
    for ep in range(ep0, epochs):
        if stop_after is not None and ep - ep0 >= stop_after:
            return None
        perm = rng.permutation(n_inst)
        rows = np.concatenate([np.arange(tr["offs"][b], tr["offs"][b + 1]) for b in perm])
        eoff = np.concatenate([[0], np.cumsum(sizes[perm])]).astype(np.int64)
        rows_d = torch.from_numpy(rows.astype(np.int32)).to(device)
        eoff_d = torch.from_numpy(eoff).to(device)
        ep_loss = torch.zeros((), dtype=torch.float64, device=device)
        for b0 in range(0, n_inst, batch_instances):
            b1 = min(n_inst, b0 + batch_instances)
            p0, p1 = int(eoff[b0]), int(eoff[b1])
            step += 1
            # linear warm-down of the learning rate to 5% over the run
            lr_t = lr * (1.0 - 0.95 * (step - 1) / max(1, total_steps - 1))
            l1line.mlp_forward(tr["feat"], mlp, rows=rows_d[p0:p1], out=score[p0:p1])
            l1line.rank_loss(score, tr["tgt"], eoff_d[b0:b1 + 1], rows=rows_d,
                             dscores=dscore, loss=loss[:b1 - b0])
            l1line.mlp_backward(tr["feat"], mlp, dscore[p0:p1], rows=rows_d[p0:p1], grad=grad,
                                workspace=mws)
            l1line.adam_step(theta, grad, m1, m2, step, lr_t, mlp=mlp)
            ep_loss += loss[:b1 - b0].sum(dtype=torch.float64)
        tr_loss = float(ep_loss) / n_inst
        rec = _recall(va, mlp, K_DEFAULT)
        history.append({"epoch": ep + 1, "train_loss": tr_loss, "val_recall_top32": rec})
        log(f"epoch {ep + 1}: train loss {tr_loss:.4f}, validation top-{K_DEFAULT} recall "
            f"{rec:.4f}")
        if best is None or rec >= best[0]:
            best = (rec, ep + 1, theta.detach().cpu().numpy().copy())
        save_checkpoint(ckpt, config, ep + 1, step, theta.cpu().numpy(), m1.cpu().numpy(),
                        m2.cpu().numpy(), rng.bit_generator.state, history, best)
    t_train = time.time() - t_train
    th = best[2]
    th.astype("<f4").tofile(os.path.join(out_dir, "proposer_theta.f32"))
    info = {"train_seeds": [s0, s1], "val_seeds": [v0, v1], "instances": n_inst,
            "rows": N, "epochs": epochs, "batch_instances": batch_instances, "lr": lr,
            "temperature": TEMPERATURE, "top": TOP, "label_seconds": t_label,
            "train_seconds": t_train, "kept_epoch": best[1], "val_recall_top32": best[0],
            "history": history}
    with open(os.path.join(out_dir, "proposer_train.json"), "w") as f:
        json.dump(info, f, indent=1)
    return info


# ---------------------------------------------------------------------------
# evaluation
# ---------------------------------------------------------------------------
def _ranks_of_best(z, score):
    """Smallest K whose top-K by `score` (ties to the smaller index) holds a
    jhat of minimal z, and the relative regret min(z over top-K) / min z - 1
    for every K (index K - 1)."""
    order = np.lexsort((np.arange(score.size), -score))
    pos = np.empty(score.size, dtype=np.int64)
    pos[order] = np.arange(score.size)
    zmin = z.min()
    regret = (np.minimum.accumulate(z[order]) - zmin) / (abs(zmin) if zmin != 0 else 1.0)
    return int(pos[z == zmin].min()) + 1, regret


def rank_study(count, seed0, n=5000, m=1000, theta_path=THETA_PATH, device=None, log=None):
    """Per instance (float32 n x m, proposer_spec seeds seed0 ...): the exact
    objectives of every jhat (one scan) and, for the learned scores, the l1,
    l2 and median features, the heavy-row objective alone (lowest first) and a
    random order, the smallest K that keeps a best jhat.  Zero regret at K <=>
    that rank <= K."""
    import torch
    device = device or "cuda"
    mlp = network(device, theta_path)
    ws = l1line.proposed_workspace("float32", n, m, 1, device)
    rng = np.random.default_rng(seed0)
    ranks = {"learned": [], "l1": [], "l2": [], "median": [], "heavy_rows": [], "random": []}
    regrets = {k: [] for k in ranks}
    for i in range(count):
        spec = datagen.proposer_spec(seed0 + i, n=n, m=m)
        X, _, _ = datagen.planted_torch(spec, device)
        raw, fz = l1line.features(X, datagen.PROPOSER_LAMBDA, workspace=ws)
        s = l1line.mlp_forward(fz, mlp)
        _, _, z, _ = l1line.scan(X, [datagen.PROPOSER_LAMBDA], workspace=ws, z_only=True)
        if l1line.status(ws) != l1line.OK:
            raise RuntimeError(f"instance {spec.seed} failed on the device")
        z = z[0].cpu().numpy()
        raw = raw.cpu().numpy().astype(np.float64)
        for key, sc in (("learned", s.cpu().numpy().astype(np.float64)), ("l1", raw[:, 0]),
                        ("l2", raw[:, 1]), ("median", raw[:, 2]), ("heavy_rows", -raw[:, 3]),
                        ("random", rng.random(m))):
            r, reg = _ranks_of_best(z, sc)
            ranks[key].append(r)
            regrets[key].append(reg)
        if log and (i + 1) % 50 == 0:
            log(f"  {i + 1} instances ranked")
    out = {k: np.array(v) for k, v in ranks.items()}
    out["regret"] = {k: np.array(v) for k, v in regrets.items()}  # [instance, K - 1]
    return out


def k_for(ranks, frac):
    """Smallest K with zero regret on at least `frac` of the instances."""
    r = np.sort(ranks)
    return int(r[int(np.ceil(frac * r.size)) - 1])


def evaluate(theta_path=THETA_PATH, count=200, Ks=(32, 64, 128, 256, 512), n=5000, m=1000,
             device=None, log=None, seed0=datagen.PROPOSER_HELDOUT_SEED0, target=0.99,
             calib_count=200):
    """Held-out float32 n x m instances.

    1. K_target: the smallest K with zero regret on `target` of a calibration
       set of the same shape (seeds VAL_EVAL_SEED0 ...), chosen before the
       held-out set is looked at.
    2. Held-out zero-regret curves (learned, each single feature, random) from
       one exact scan per instance, at the listed K and K_target.
    3. Times (CUDA events, L2 flushed before each call) of the full fit and of
       the learned path at each K; the learned path's objective is checked
       against the scan (the same kernels give the same bits)."""
    import torch
    device = device or "cuda"
    cal = rank_study(calib_count, VAL_EVAL_SEED0, n, m, theta_path, device, log)
    k_target = k_for(cal["learned"], target)
    Ks = tuple(sorted(set(Ks) | {k_target}))
    held = rank_study(count, seed0, n, m, theta_path, device, log)
    mlp = network(device, theta_path)
    lam = [datagen.PROPOSER_LAMBDA]
    ws = l1line.proposed_workspace("float32", n, m, 1, device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        flush.fill_(1)
        ev[0].record()
        r = fn()
        ev[1].record()
        torch.cuda.synchronize()
        return r, ev[0].elapsed_time(ev[1])

    t_full, t_prop = [], {K: [] for K in Ks}
    n_time = min(count, 40)
    for i in range(n_time):
        spec = datagen.proposer_spec(seed0 + i, n=n, m=m)
        X, _, _ = datagen.planted_torch(spec, device)
        if i == 0:
            l1line.fit(X, lam, workspace=ws)
            for K in Ks:
                l1line.fit_proposed(X, lam, mlp, K, workspace=ws)
        (_, of, _, _), tf = timed(lambda: l1line.fit(X, lam, workspace=ws))
        t_full.append(tf)
        for K in Ks:
            (_, op, _, _, _), tp = timed(lambda: l1line.fit_proposed(X, lam, mlp, K, workspace=ws))
            t_prop[K].append(tp)
            zero = bool(float(op[0]) == float(of[0]))
            if zero != bool(held["learned"][i] <= K):
                raise RuntimeError(f"instance {spec.seed}: learned path and rank study disagree")
        if l1line.status(ws) != l1line.OK:
            raise RuntimeError(f"held-out instance {spec.seed} failed on the device")
    out = {"instances": count, "timed_instances": n_time, "n": n, "m": m, "lambda": lam[0],
           "target": target, "calibration_instances": calib_count, "K_target": k_target,
           "full_ms_median": float(np.median(t_full)), "per_K": {},
           "K_for_target_on_heldout": {k: k_for(v, target) for k, v in held.items()
                                       if k != "regret"}}
    for K in Ks:
        d = {"learned_ms_median": float(np.median(t_prop[K])),
             "speedup_median": float(np.median(t_full) / np.median(t_prop[K])),
             "zero_regret_frac": {k: float(np.mean(v <= K)) for k, v in held.items()
                                  if k != "regret"},
             "mean_rel_regret": {k: float(v[:, K - 1].mean()) for k, v in held["regret"].items()},
             "max_rel_regret": {k: float(v[:, K - 1].max()) for k, v in held["regret"].items()}}
        out["per_K"][str(K)] = d
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_2402_16712_gb300.proposer")
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--out", required=True)
    t.add_argument("--instances", type=int, default=None)
    t.add_argument("--epochs", type=int, default=24)
    t.add_argument("--eval-count", type=int, default=200)
    t.add_argument("--resume", action="store_true",
                   help="continue from OUT/checkpoint.npz (written after every epoch)")
    e = sub.add_parser("eval")
    e.add_argument("--theta", default=THETA_PATH)
    e.add_argument("--count", type=int, default=200)
    e.add_argument("--K", type=int, nargs="+", default=[32, 64, 128, 256, 512])
    e.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    from . import build
    build.build()
    log = lambda s: print(s, flush=True)
    if a.cmd == "train":
        info = train(a.out, n_train=a.instances, epochs=a.epochs, log=log, resume=a.resume)
        log(json.dumps({k: v for k, v in info.items() if k != "history"}))
        if a.eval_count:
            res = evaluate(os.path.join(a.out, "proposer_theta.f32"), count=a.eval_count, log=log)
            with open(os.path.join(a.out, "proposer_eval.json"), "w") as f:
                json.dump(res, f, indent=1)
            log(json.dumps(res))
    else:
        res = evaluate(a.theta, count=a.count, Ks=tuple(a.K), log=log)
        if a.out:
            with open(a.out, "w") as f:
                json.dump(res, f, indent=1)
        log(json.dumps(res))
    return 0


if __name__ == "__main__":
    sys.exit(main())
