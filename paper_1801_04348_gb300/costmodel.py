"""Learned case selection: a small MLP ranks the feasible program parameters of a
GEMM so that only its top-k are timed (the paper leaves the choice of program
parameters to auto-tuning, Section 1; the case discussion of Section 3 decides
which of them are feasible).

Pipeline (all arithmetic in the library's CUDA kernels, called through `pgk`):
  1. collect: the autotuner (pgk_autotune) times every candidate on seeded
     shapes; each (shape, candidate, time) becomes a row of the timing log;
  2. train: features are z-scored on the training split, the target is
     ln(milliseconds) (z-scored); pgk_mlp_loss_grad + pgk_mlp_adam run the
     epochs on the GPU (minibatches are index slices of a host permutation);
  3. select: pgk_mlp_forward scores every candidate of a new shape, the k best
     predictions are timed, the fastest of them is used;
  4. evaluate: regret against exhaustive timing of all candidates.

Features (7 values, log2 of sizes): M, N, K, B0, B1, s and a form code
(0 = FP32 paper-form, 1 = FP32 register-blocked, 2 = BF16, 3 = split BF16,
4 = FP8).  In the learned candidate set a register-blocked variant has sr = s
and tile = 8, and a paper-form variant tile = B0, so (B0, B1, s, form) names
exactly one variant; for tensor-core forms B0 x B1 is the CTA tile and s the
number of pipeline stages.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from . import inputs, pgk

FORM_CODE = {"paper": 0, "rb": 1, pgk.BF16: 2, pgk.SPLIT_BF16: 3, pgk.FP8_E4M3: 4}


def candidates(dtype) -> list:
    """The learned candidate set of a form (see the module docstring)."""
    if dtype == pgk.F32:
        out = []
        for b0 in (8, 16, 32):
            for b1 in (8, 16, 32):
                for s in (1, 2, 4):
                    if b0 <= b1 * s:
                        out.append(pgk.params(b0, b1, s, 1, 0))
        for v in range(pgk.num_variants()):
            info = pgk.variant_info_get(v)
            if info.family == pgk.FAM_RB and info.sr == info.s and info.tile == 8:
                out.append(pgk.params(info.B0, info.B1, info.s, info.sr, info.tile))
        return out
    # the tile programs; the fused-conversion program (B1 = 64) is the case
    # discussion's choice for N <= 64 and is not ranked
    return [p for p in pgk.default_candidates(dtype) if p.B1 != 64]


def feature_row(M, N, K, p, dtype) -> list:
    if dtype == pgk.F32:
        code = FORM_CODE["rb"] if p.sr > 1 else FORM_CODE["paper"]
    else:
        code = FORM_CODE[dtype]
    return [math.log2(M), math.log2(N), math.log2(K), math.log2(p.B0), math.log2(p.B1),
            math.log2(p.s), float(code)]


def time_shape(M, N, K, dtype, cands, reps, dev, seed=0, log_path=None, stream=None):
    """Times every candidate on one shape (uniform[-1,1] operands); returns ms list."""
    import torch
    A, B = inputs.gemm_operands(M, N, K, seed=seed)
    Ad = torch.from_numpy(A).to(dev)
    Bd = torch.from_numpy(B).to(dev)
    C = torch.empty(M, N, device=dev)
    _, res = pgk.autotune(Ad, Bd, C, dtype, candidates=cands, reps=reps, log_path=log_path,
                          stream=stream)
    return [ms for _, ms in res]


def collect(shapes, dtype, dev, reps=2, log_path=None, seed=0):
    """Timing log rows (features, ms) for every candidate of every shape."""
    cands = candidates(dtype)
    X, y, meta = [], [], []
    for i, (M, N, K) in enumerate(shapes):
        ms = time_shape(int(M), int(N), int(K), dtype, cands, reps, dev, seed=seed + i,
                        log_path=log_path)
        for p, t in zip(cands, ms):
            if np.isfinite(t) and t > 0:
                X.append(feature_row(M, N, K, p, dtype))
                y.append(t)
                meta.append((int(M), int(N), int(K), dtype) + p.as_tuple())
    return np.asarray(X, np.float32), np.asarray(y, np.float64), meta


class CostModel:
    """The 7-64-64-1 network with its feature/target normalisation."""

    def __init__(self, theta=None, mu=None, sd=None, tmu=0.0, tsd=1.0):
        self.theta = None if theta is None else np.asarray(theta, np.float32)
        self.mu = mu
        self.sd = sd
        self.tmu = tmu
        self.tsd = tsd
        self.history = []

    def _norm(self, X):
        return ((np.asarray(X, np.float64) - self.mu) / self.sd).astype(np.float32)

    def fit(self, X, ms, dev, epochs=200, batch=256, lr=1e-3, seed=0, val_frac=0.1):
        """Trains on the GPU with pgk_mlp_loss_grad / pgk_mlp_adam.  Returns
        (train loss, validation loss) on the normalised ln-time target."""
        import torch
        X = np.asarray(X, np.float64)
        t = np.log(np.asarray(ms, np.float64))
        rng = np.random.default_rng(seed)
        perm = rng.permutation(len(X))
        nval = max(1, int(round(val_frac * len(X))))
        va, tr = perm[:nval], perm[nval:]
        self.mu = X[tr].mean(axis=0)
        self.sd = X[tr].std(axis=0)
        self.sd[self.sd == 0] = 1.0
        self.tmu = float(t[tr].mean())
        self.tsd = float(t[tr].std()) or 1.0
        Xn = self._norm(X)
        tn = ((t - self.tmu) / self.tsd).astype(np.float32)
        Xd = torch.from_numpy(Xn).to(dev)
        td = torch.from_numpy(tn).to(dev)
        th = torch.from_numpy(inputs.he_uniform_mlp(seed)).to(dev)
        m = torch.zeros_like(th)
        v = torch.zeros_like(th)
        g = torch.zeros_like(th)
        loss = torch.zeros(1, device=dev)
        tr_d = torch.from_numpy(tr.astype(np.int32)).to(dev)
        va_d = torch.from_numpy(va.astype(np.int32)).to(dev)
        step = 0
        for ep in range(epochs):
            order = torch.from_numpy(rng.permutation(len(tr)).astype(np.int64)).to(dev)
            idx_ep = tr_d[order]
            for b in range(0, len(tr), batch):
                step += 1
                pgk.mlp_loss_grad(Xd, td, th, g, loss, idx=idx_ep[b:b + batch])
                pgk.mlp_adam(th, g, m, v, step, lr=lr)
            if ep % 20 == 19 or ep == epochs - 1:
                pgk.mlp_loss_grad(Xd, td, th, g, loss, idx=tr_d)
                ltr = loss.item()
                pgk.mlp_loss_grad(Xd, td, th, g, loss, idx=va_d)
                self.history.append((ep + 1, ltr, loss.item()))
        self.theta = th.cpu().numpy()
        return self.history[-1][1], self.history[-1][2]

    def predict_ms(self, X, dev):
        import torch
        Xd = torch.from_numpy(self._norm(X)).to(dev)
        th = torch.from_numpy(self.theta).to(dev)
        y = torch.zeros(len(X), device=dev)
        pgk.mlp_forward(Xd, th, y)
        return np.exp(y.cpu().numpy().astype(np.float64) * self.tsd + self.tmu)

    def save(self, path):
        with open(path, "w") as f:
            json.dump({"theta": self.theta.tolist(), "mu": list(self.mu), "sd": list(self.sd),
                       "tmu": self.tmu, "tsd": self.tsd, "history": self.history}, f)

    @classmethod
    def load(cls, path):
        with open(path) as f:
            d = json.load(f)
        cm = cls(np.asarray(d["theta"], np.float32), np.asarray(d["mu"]), np.asarray(d["sd"]),
                 d["tmu"], d["tsd"])
        cm.history = d.get("history", [])
        return cm


def evaluate(model, shapes, dtype, dev, k=3, reps=1, seed=1000):
    """Exhaustive timing of every candidate per shape vs the model's top-k pick.

    Returns per-shape records and a summary: regret r = t(best of top-k) /
    t(exhaustive best) - 1 (geometric mean of 1 + r minus 1, mean, p90), the
    same for a random choice of k candidates and for the untuned default, and
    the tuning time saved (sum of all candidate times over the sum of the
    top-k times).  Every record keeps all candidate times and predictions, so
    `summarize_k` can evaluate other k on the same timings."""
    cands = candidates(dtype)
    rng = np.random.default_rng(seed)
    recs = []
    for i, (M, N, K) in enumerate(shapes):
        M, N, K = int(M), int(N), int(K)
        ms = np.asarray(time_shape(M, N, K, dtype, cands, reps, dev, seed=seed + i), np.float64)
        feas = np.isfinite(ms)
        feats = np.asarray([feature_row(M, N, K, p, dtype) for p in cands], np.float32)
        pred = model.predict_ms(feats, dev)
        pred[~feas] = np.inf
        top = np.argsort(pred)[:k]
        rnd = rng.choice(np.nonzero(feas)[0], size=min(k, int(feas.sum())), replace=False)
        best = float(np.min(ms[feas]))
        dflt = default_index(cands, M, N, K, dtype)
        recs.append({"M": M, "N": N, "K": K, "best_ms": best,
                     "model_ms": float(np.min(ms[top])), "random_ms": float(np.min(ms[rnd])),
                     "default_ms": float(ms[dflt]) if dflt is not None and feas[dflt] else float("nan"),
                     "exhaustive_cost_ms": float(np.sum(ms[feas])),
                     "topk_cost_ms": float(np.sum(ms[top][np.isfinite(ms[top])])),
                     "ms_all": [float(x) for x in ms], "pred_all": [float(x) for x in pred],
                     "default_index": dflt})
    return recs, summarize(recs, k)


def expected_random_min(ms, k):
    """Expected fastest time of k candidates drawn uniformly without replacement
    from the feasible times `ms`: sum over the sorted times t_(i) of t_(i) times
    the probability that t_(i) is the smallest drawn, C(n-1-i, k-1) / C(n, k)."""
    t = np.sort(np.asarray([x for x in ms if np.isfinite(x)], np.float64))
    n = len(t)
    k = min(k, n)
    w = np.asarray([math.comb(n - 1 - i, k - 1) for i in range(n)], np.float64) / math.comb(n, k)
    return float(np.dot(w, t))


def summarize_k(recs, k):
    """Regret at top-k of the recorded timings: the model's k best predictions,
    the expectation over random k-subsets (exact), and the untuned default."""
    def gm(r):
        r = np.asarray(r, np.float64)
        return {"geomean": float(np.exp(np.mean(np.log1p(r))) - 1.0), "mean": float(r.mean()),
                "p90": float(np.percentile(r, 90)), "max": float(r.max()), "n": int(r.size)}
    rm, rr, rd = [], [], []
    ex = tk = 0.0
    for x in recs:
        ms = np.asarray(x["ms_all"], np.float64)
        pred = np.asarray(x["pred_all"], np.float64)
        best = x["best_ms"]
        top = np.argsort(pred)[:k]
        rm.append(float(np.min(ms[top])) / best - 1.0)
        rr.append(expected_random_min(ms, k) / best - 1.0)
        d = x.get("default_index")
        if d is not None and np.isfinite(ms[d]):
            rd.append(ms[d] / best - 1.0)
        ex += float(np.sum(ms[np.isfinite(ms)]))
        tk += float(np.sum(ms[top][np.isfinite(ms[top])]))
    return {"k": k, "shapes": len(recs), "model": gm(rm), "random_k_expected": gm(rr),
            "untuned_default": gm(rd) if rd else None, "tuning_time_saved": ex / tk if tk else None}


def default_index(cands, M, N, K, dtype):
    """Index of the library's untuned default parameters in the candidate set."""
    if dtype == pgk.F32:
        big = M * N >= 2048 * 2048
        mid = M * N >= 256 * 256
        want = (16, 16, 8, 8, 8) if big else ((16, 16, 4, 4, 8) if mid else (8, 8, 8, 8, 8))
    elif dtype == pgk.BF16:
        want = (128, 256, 4, 0, 0)
    elif dtype == pgk.SPLIT_BF16:
        want = (128, 128, 3, 0, 0)
    else:
        want = (128, 128, 6, 0, 0)
    for i, p in enumerate(cands):
        if p.as_tuple() == want:
            return i
    return None


def summarize(recs, k):
    def stats(key):
        r = np.asarray([x[key] / x["best_ms"] - 1.0 for x in recs if np.isfinite(x[key])])
        if r.size == 0:
            return None
        return {"geomean": float(np.exp(np.mean(np.log1p(r))) - 1.0), "mean": float(r.mean()),
                "p90": float(np.percentile(r, 90)), "max": float(r.max()), "n": int(r.size)}
    ex = sum(x["exhaustive_cost_ms"] for x in recs)
    tk = sum(x["topk_cost_ms"] for x in recs)
    return {"k": k, "shapes": len(recs), "model": stats("model_ms"), "random_k": stats("random_ms"),
            "untuned_default": stats("default_ms"), "tuning_time_saved": ex / tk if tk else None}


def training_shapes(dtype=None):
    """Shapes whose tuning produces the timing log: the 256^3 correctness shape,
    the four large FP32 shapes and the 512 grouped-GEMM shapes.  The tensor-core
    forms add 300 shapes log-uniform in [64, 16384] (seed 777): the tuning
    workloads above reach 2048 at most apart from the four large shapes, and a
    tile program's rank among the few of a tensor-core form moves with the tile
    count, so their log needs the whole size range of the shapes it must rank."""
    big = [(4096, 4096, 4096), (8192, 8192, 8192), (8192, 1024, 4096), (16384, 64, 16384)]
    grouped = [tuple(int(v) for v in r) for r in inputs.log_uniform_dims(512, 0, 32, 2048, 16)]
    base = [(256, 256, 256)] + big + grouped
    if dtype is None or dtype in (pgk.F32, pgk.I32):
        return base
    seen = set(base)
    extra = []
    for r in inputs.log_uniform_dims(300, 777, 64, 16384, 16):
        t = tuple(int(v) for v in r)
        if t not in seen:
            seen.add(t)
            extra.append(t)
    return base + extra


def unseen_shapes(count=1000, seed=12345, exclude=()):
    """Held-out shapes: M, N, K log-uniform in [64, 16384] (multiples of 16),
    deduplicated against the training shapes."""
    ex = set(tuple(e) for e in exclude)
    out = []
    s = seed
    while len(out) < count:
        for r in inputs.log_uniform_dims(count, s, 64, 16384, 16):
            t = tuple(int(v) for v in r)
            if t not in ex and t not in out:
                out.append(t)
                if len(out) == count:
                    break
        s += 1
    return out


def main():
    import argparse

    import torch
    ap = argparse.ArgumentParser(description="learned case selection: collect, train, evaluate")
    ap.add_argument("--out", required=True, help="output directory")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "split"])
    ap.add_argument("--eval-shapes", type=int, default=1000)
    ap.add_argument("--k", type=int, default=3)
    ap.add_argument("--epochs", type=int, default=200)
    ap.add_argument("--model", default=None,
                    help="evaluate this trained model (JSON) instead of collecting and training")
    args = ap.parse_args()
    os.makedirs(args.out, exist_ok=True)
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    dt = pgk.DTYPES[args.dtype]
    t0 = time.time()
    shapes = training_shapes(dt)
    if args.model:
        cm = CostModel.load(args.model)
        X, ltr, lva = (), None, None
        t1 = t2 = time.time()
    else:
        X, y, _ = collect(shapes, dt, dev, reps=2,
                          log_path=os.path.join(args.out, f"timing_log_{args.dtype}.csv"))
        t1 = time.time()
        cm = CostModel()
        ltr, lva = cm.fit(X, y, dev, epochs=args.epochs)
        cm.save(os.path.join(args.out, f"costmodel_{args.dtype}.json"))
        t2 = time.time()
    ev = unseen_shapes(args.eval_shapes, exclude=shapes)
    recs, summ = evaluate(cm, ev, dt, dev, k=args.k)
    t3 = time.time()
    summ.update({"dtype": args.dtype, "train_rows": int(len(X)), "train_loss": ltr,
                 "val_loss": lva, "collect_s": t1 - t0, "train_s": t2 - t1, "eval_s": t3 - t2,
                 "candidates": len(candidates(dt)),
                 "by_k": [summarize_k(recs, kk) for kk in range(1, len(candidates(dt)))]})
    with open(os.path.join(args.out, f"regret_{args.dtype}.json"), "w") as f:
        json.dump({"summary": summ, "records": recs}, f)
    print(json.dumps(summ))


if __name__ == "__main__":
    main()
