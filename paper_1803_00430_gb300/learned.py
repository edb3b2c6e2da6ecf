"""Learned estimator workflow: data from the method itself, training and evaluation.

A network (rpr.MLP) maps the energy IR of a low-ray-count trace plus scene features
to per-band decay times and direct-to-reverberant ratios.  Its labels are the plain
estimator's parameters on high-ray-count traces of the same scenes (the method at a
high ray budget is the reference); it is judged by the decay-time error against
those labels, next to the plain estimator on the same low-ray IRs.

Every step on the data runs in the CUDA library: batched traces (rp_batch_*), the
plain estimator, feature extraction (rp_mlp_features), standardisation, and the
network's forward, backward and AdamW kernels.  This module only orchestrates.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import rpr, scenes

TRACE = dict(max_order=64, sh_order=0, num_bins=2000, min_order=1, ir_rate_hz=1000.0)
IN_DIM, OUT_DIM, BANDS = 528, 16, 8


@dataclass
class Dataset:
    X: object            # raw features, torch float32 [n, IN_DIM] on the device
    Y: np.ndarray        # targets [n, 16]: ln RT60 per band, DRR [dB] per band (high-ray trace)
    mask: np.ndarray     # [n, 16] 1 where the target exists
    plain_rt: np.ndarray  # RT60 of the plain estimator on the low-ray IR [n, 8] (NaN: no fit)
    ref_rt: np.ndarray   # RT60 labels [n, 8] (NaN: no usable label)
    rays: np.ndarray     # ray count of each row's input trace [n]
    high_rays: int
    label_frac: float = 1.0  # fraction of (scene, band) decay times kept as labels

    def rows(self, sel):
        """The sub-dataset of the rows selected by a boolean mask or index array."""
        import torch
        idx = np.nonzero(sel)[0] if np.asarray(sel).dtype == bool else np.asarray(sel)
        return Dataset(self.X[torch.as_tensor(idx, device=self.X.device)], self.Y[idx], self.mask[idx],
                       self.plain_rt[idx], self.ref_rt[idx], self.rays[idx], self.high_rays, self.label_frac)


S_SPREAD = 0.1


def learned_scenes(seed: int, n: int, bands: int = BANDS, max_tris: int = 4000, s_spread: float = S_SPREAD):
    """Procedural rooms and corridors with one source each; triangle counts
    log-uniform in [12, max_tris].  Scattering rises smoothly over the bands by at most
    s_spread: the per-band path weights s_b / s_mean and (1 - s_b) / (1 - s_mean)
    multiply from bounce to bounce, and their second moment grows per bounce by
    1 + (s_b - s_mean)^2 / (s_mean (1 - s_mean)); band-independent scattering makes
    late high-ray IRs (the labels) heavy-tailed."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        tris = int(np.exp(rng.uniform(np.log(12), np.log(max_tris))))
        out.append(scenes.room_or_corridor(seed * 7919 + i, tris, bands=bands, num_sources=1, s_spread=s_spread))
    return out


def _keys(seed: int, copies: int):
    """Philox keys: one per noisy low-ray trace, and a pair for the two halves of
    the high-ray labels."""
    base = scenes.PHILOX_KEY_BASE + 4096 * seed
    return [base + 2 * c for c in range(copies)], (base + 1, base + 3)


def make_dataset(ctx: rpr.Context, n: int, seed: int, low_rays=(2000,), high_rays: int = 100000,
                 copies: int = 1, bands: int = BANDS, slice_size: int = 1024, stability: float = 0.1):
    """n procedural scenes.  Inputs: for every ray count in `low_rays`, `copies`
    traces with independent Philox keys (the same label under different noise).
    Labels: the plain estimator on the mean of two traces of high_rays / 2 rays each
    (a high_rays trace); a decay time is kept only when it passes label_ok and the
    two halves agree within `stability` (relative).  Rows are ordered
    (ray count, copy, scene); Dataset.rays gives each row's ray count."""
    scs = learned_scenes(seed, n, bands)
    lows = [int(r) for r in np.atleast_1d(low_rays)]
    lo_keys, (hk_a, hk_b) = _keys(seed, len(lows) * copies)
    p = rpr.TraceParams(**TRACE)
    rows = len(lows) * copies
    X = [[] for _ in range(rows)]
    plain = [[] for _ in range(rows)]
    labs, stab = [], []
    for a in range(0, n, slice_size):
        part = scs[a:a + slice_size]
        rs = [rpr.Scene.from_scene(ctx, sc) for sc in part]
        feats = np.stack([rpr.scene_features(s) for s in rs])

        def items(rays):
            return [(rs[i], part[i].listener, part[i].sources, rays, a + i) for i in range(len(part))]

        for li, rays in enumerate(lows):
            lo = rpr.Batch(ctx, items(rays), p)
            for c in range(copies):
                r = li * copies + c
                lo.run(seed=lo_keys[r])
                X[r].append(rpr.mlp_features(ctx, lo.H, feats, p.ir_rate_hz, IN_DIM))
                plain[r].append(lo.params_dict()["rt60_raw"][:, :bands].astype(np.float64))
            lo.close()
        hi = rpr.Batch(ctx, items(max(1, high_rays // 2)), p)
        hi.run(seed=hk_a)
        Ha = hi.H.clone()
        rt_a = hi.params_dict()["rt60_raw"][:, :bands]
        hi.run(seed=hk_b)
        rt_b = hi.params_dict()["rt60_raw"][:, :bands]
        Ha.add_(hi.H).mul_(0.5)
        raw = rpr.estimate(ctx, Ha, hi.direct, p.ir_rate_hz)
        labs.append(rpr.params_to_dict(raw.cpu().numpy().tobytes(), hi.S, hi.B, hi.K))
        with np.errstate(invalid="ignore", divide="ignore"):
            stab.append(np.abs(rt_a - rt_b) / (0.5 * (rt_a + rt_b)))
        hi.close()
        del Ha
        for s in rs:
            s.close()
    import torch
    lab = {k: np.concatenate([d[k] for d in labs]) for k in ("rt60_raw", "drr_db", "range_kind", "fit_r2")}
    with np.errstate(invalid="ignore"):
        ok_rt = label_ok(lab, bands) & (np.concatenate(stab) <= stability)
    rt = lab["rt60_raw"][:, :bands]
    drr = lab["drr_db"][:, :bands]
    Y = np.zeros((n, OUT_DIM), np.float32)
    M = np.zeros((n, OUT_DIM), np.float32)
    ok_drr = np.isfinite(drr)
    Y[:, :bands] = np.where(ok_rt, np.log(np.where(ok_rt, rt, 1.0)), 0.0)
    Y[:, BANDS:BANDS + bands] = np.where(ok_drr, drr, 0.0)
    M[:, :bands] = ok_rt
    M[:, BANDS:BANDS + bands] = ok_drr
    return Dataset(torch.cat([torch.cat(x) for x in X]), np.tile(Y, (rows, 1)), np.tile(M, (rows, 1)),
                   np.concatenate([np.concatenate(pc) for pc in plain]),
                   np.tile(np.where(ok_rt, rt, np.nan), (rows, 1)), np.repeat(np.repeat(lows, copies), n),
                   high_rays, float(np.mean(ok_rt)))


def label_ok(params: dict, bands: int = BANDS) -> np.ndarray:
    """Decay times usable as labels: a T30 or T20 fit (the -35 or -25 dB floor was
    reached) that is close to a line (R^2 >= 0.95), within 0.02 .. 30 s.  Sparse IRs
    (a source hidden behind partitions) can give steep T10 fits that are not decay
    times of the room."""
    rt = params["rt60_raw"][:, :bands]
    kind = params["range_kind"][:, :bands]
    r2 = params["fit_r2"][:, :bands]
    with np.errstate(invalid="ignore"):
        return np.isfinite(rt) & (kind >= 1) & (kind <= 2) & (r2 >= 0.95) & (rt > 0.02) & (rt < 30.0)


def normalization(ds: Dataset):
    X = ds.X.double().cpu().numpy()
    in_mean = X.mean(axis=0)
    in_std = X.std(axis=0)
    in_std = np.where(in_std > 1e-6, in_std, 1.0)
    M = ds.mask.astype(bool)
    out_mean = np.array([ds.Y[M[:, j], j].mean() if M[:, j].any() else 0.0 for j in range(OUT_DIM)])
    out_std = np.array([ds.Y[M[:, j], j].std() if M[:, j].sum() > 1 else 1.0 for j in range(OUT_DIM)])
    out_std = np.where(out_std > 1e-6, out_std, 1.0)
    return in_mean, in_std, out_mean, out_std


def fit(ctx: rpr.Context, train: Dataset, steps: int = 3000, batch: int = 256, lr: float = 2e-3,
        weight_decay: float = 1e-4, seed: int = 1, log_every: int = 0):
    """Train a fresh network on `train`; returns (mlp, loss history)."""
    import torch
    n = train.X.shape[0]
    mlp = rpr.MLP(ctx, in_dim=IN_DIM, out_dim=OUT_DIM, max_batch=max(batch, 1), seed=seed)
    in_mean, in_std, out_mean, out_std = normalization(train)
    mlp.set_normalization(in_mean, in_std, out_mean, out_std)
    mlp.norm = (in_mean, in_std, out_mean, out_std)
    Xb = mlp.prepare(train.X)
    T = torch.tensor(((train.Y - out_mean) / out_std) * train.mask, dtype=torch.float32, device="cuda")
    Mk = torch.tensor(train.mask, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(seed)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    hist = []
    for s in range(steps):
        idx = torch.as_tensor(rng.choice(n, size=min(batch, n), replace=False), device="cuda")
        frac = s / max(1, steps)
        step_lr = lr * (0.5 * (1 + np.cos(np.pi * frac)))  # cosine decay
        mlp.train_step(Xb[idx].contiguous(), T[idx].contiguous(), Mk[idx].contiguous(), step_lr, weight_decay,
                       loss)
        if log_every and (s % log_every == 0 or s == steps - 1):
            hist.append((s, float(loss.item())))
    return mlp, hist


def predict(mlp: rpr.MLP, X):
    """De-standardised network outputs [n, 16] for raw features X (torch, device)."""
    import torch
    Xb = mlp.prepare(X)
    outs = []
    mb = mlp.cfg.max_batch
    for a in range(0, X.shape[0], mb):
        outs.append(mlp.forward(Xb[a:a + mb].contiguous()))
    return torch.cat(outs).cpu().numpy()


def evaluate(mlp: rpr.MLP, ds: Dataset, bands: int = BANDS) -> dict:
    """Decay-time relative errors |RT - RT_ref| / RT_ref against the high-ray labels,
    over every (row, band) with a label: the network and the plain estimator on the
    same low-ray IRs (a missing plain fit counts as an error of 1, and plain errors
    are capped at 1 in the mean)."""
    Y = predict(mlp, ds.X)
    ok = np.isfinite(ds.ref_rt)
    rt_net = np.exp(np.clip(Y[:, :bands], np.log(0.01), np.log(100.0)))
    with np.errstate(invalid="ignore"):
        e_net = np.abs(rt_net - ds.ref_rt) / ds.ref_rt
        e_plain = np.where(np.isfinite(ds.plain_rt), np.abs(ds.plain_rt - ds.ref_rt) / ds.ref_rt, 1.0)
    dm = ds.mask[:, BANDS:BANDS + bands].astype(bool)
    drr_err = np.abs(Y[:, BANDS:BANDS + bands] - ds.Y[:, BANDS:BANDS + bands])
    return {
        "rt_err_mean_net": float(e_net[ok].mean()),
        "rt_err_median_net": float(np.median(e_net[ok])),
        "rt_err_p95_net": float(np.percentile(e_net[ok], 95)),
        "rt_err_mean_plain": float(np.minimum(e_plain[ok], 1.0).mean()),
        "rt_err_median_plain": float(np.median(e_plain[ok])),
        "rt_err_p95_plain": float(np.percentile(e_plain[ok], 95)),
        "plain_fit_missing": float(np.mean(~np.isfinite(ds.plain_rt[ok]))),
        "drr_mae_db_net": float(drr_err[dm].mean()) if dm.any() else float("nan"),
        "n": int(ok.sum()),
    }


def _time_updates(fn, reps: int = 3) -> float:
    """Median wall time [s] of fn() with the device synchronised on both sides."""
    import time

    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        ts.append(time.perf_counter() - t0)
    return float(np.median(ts))


def updates_per_s(ctx: rpr.Context, scs, rays: int, mlp: rpr.MLP | None = None, seed: int = 1) -> float:
    """IR + reverberation-parameter updates per second of a batch of scenes (one
    listener each) at `rays` rays: the batched trace and the plain estimator, or with
    `mlp` the batched trace, the features and the network's forward pass."""
    p = rpr.TraceParams(**TRACE)
    rs = [rpr.Scene.from_scene(ctx, sc) for sc in scs]
    feats = np.stack([rpr.scene_features(s) for s in rs])
    b = rpr.Batch(ctx, [(rs[i], scs[i].listener, scs[i].sources, rays, i) for i in range(len(scs))], p,
                  estimate=mlp is None)
    if mlp is None:
        def step():
            b.run(seed=seed)
    else:
        def step():
            b.run(seed=seed, sync=False)
            X = rpr.mlp_features(ctx, b.H, feats, p.ir_rate_hz, IN_DIM)
            for a in range(0, X.shape[0], mlp.cfg.max_batch):
                mlp.forward(mlp.prepare(X[a:a + mlp.cfg.max_batch]))
    t = _time_updates(step)
    b.close()
    for s in rs:
        s.close()
    return len(scs) / t


def sweep(ctx: rpr.Context, mlp: rpr.MLP, test: Dataset, ray_counts, test_scenes, bar: float = 0.05) -> dict:
    """Per ray count: decay-time errors of both forms against the labels and their
    updates/s; then the smallest ray count at which each form's mean error is at
    most `bar`, with its updates/s."""
    out = {"per_rays": {}, "bar": bar}
    for n in ray_counts:
        ev = evaluate(mlp, test.rows(test.rays == n))
        ev["updates_per_s_plain"] = updates_per_s(ctx, test_scenes, n)
        ev["updates_per_s_net"] = updates_per_s(ctx, test_scenes, n, mlp)
        out["per_rays"][int(n)] = ev
    for form in ("plain", "net"):
        ok = [n for n in sorted(out["per_rays"]) if out["per_rays"][n][f"rt_err_mean_{form}"] <= bar]
        out[f"rays_at_bar_{form}"] = ok[0] if ok else None
        out[f"updates_per_s_at_bar_{form}"] = out["per_rays"][ok[0]][f"updates_per_s_{form}"] if ok else None
    return out


def mlp_flops_per_sample(in_dim: int = IN_DIM, hidden: int = 256, layers: int = 3, out_dim: int = OUT_DIM) -> float:
    """Multiply-adds x 2 of one sample's forward pass through the dense layers."""
    widths = [in_dim] + [hidden] * layers + [out_dim]
    return 2.0 * sum(a * b for a, b in zip(widths[:-1], widths[1:]))


def mlp_throughput(ctx: rpr.Context, batches=(512, 4096, 16384, 65536), reps: int = 20, seed: int = 3) -> dict:
    """Achieved TFLOP/s of the network's forward pass and of a training step (forward,
    backward and AdamW; counted as 3 x the forward flops) at each batch size, from
    CUDA events on the context's stream around `reps` back-to-back calls; plus the
    forward pass on the mma.sync GEMMs (forward_legacy) for comparison."""
    import torch
    out = {}
    rng = np.random.default_rng(seed)
    for n in batches:
        mlp = rpr.MLP(ctx, in_dim=IN_DIM, out_dim=OUT_DIM, max_batch=n, seed=seed)
        legacy = rpr.MLP(ctx, in_dim=IN_DIM, out_dim=OUT_DIM, max_batch=n, seed=seed, legacy_gemm=True)
        X = torch.tensor(rng.normal(size=(n, IN_DIM)), dtype=torch.float32, device="cuda")
        Xb = mlp.prepare(X)
        T = torch.tensor(rng.normal(size=(n, OUT_DIM)), dtype=torch.float32, device="cuda")
        M = torch.ones((n, OUT_DIM), dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        st = torch.cuda.current_stream()
        res = {}
        for name, fn in (("forward", lambda: mlp.forward(Xb, destandardize=False)),
                         ("forward_legacy", lambda: legacy.forward(Xb, destandardize=False)),
                         ("train_step", lambda: mlp.train_step(Xb, T, M, 1e-4, 0.0, loss))):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            for _ in range(reps):
                fn()
            b.record(st)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / reps
            flops = mlp_flops_per_sample() * n * (3.0 if name == "train_step" else 1.0)
            res[name] = {"ms": ms, "tflops": flops / (ms * 1e-3) / 1e12}
            if name.startswith("forward"):
                # the forward kernel(s) alone: events on the stream right around the launch
                ctx.profile(True)
                ctx.profile_reset()
                for _ in range(reps):
                    fn()
                kt = ctx.profile_read()
                ctx.profile(False)
                key = "mlp_forward_gemm" if name == "forward_legacy" else "mlp_forward_tc"
                if key in kt:
                    kms = kt[key][1] / kt[key][0]
                    res[name].update(kernel_ms=kms, kernel_tflops=mlp_flops_per_sample() * n / (kms * 1e-3) / 1e12)
        out[int(n)] = res
        mlp.close()
        legacy.close()
    return out


def main(argv=None):
    """Train the network on the method's own IRs and sweep ray counts; prints JSON."""
    import argparse
    import json
    import time

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--train", type=int, default=8192, help="training scenes")
    ap.add_argument("--test", type=int, default=512, help="held-out scenes")
    ap.add_argument("--train-rays", type=int, nargs="+", default=[2000, 4000, 8000])
    ap.add_argument("--copies", type=int, default=2, help="noisy traces per scene and ray count")
    ap.add_argument("--train-label-rays", type=int, default=100000)
    ap.add_argument("--test-label-rays", type=int, default=500000)
    ap.add_argument("--rays", type=int, nargs="+", default=[1000, 2000, 4000, 8000, 16000, 32000])
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--throughput-only", action="store_true", help="time the network's kernels on random data")
    ap.add_argument("--batches", type=int, nargs="+", default=[512, 4096, 16384, 65536])
    a = ap.parse_args(argv)
    t0 = time.time()
    import torch
    ctx = rpr.Context(a.device, torch.cuda.current_stream())
    if a.throughput_only:
        print(json.dumps({"mlp_flops_per_sample": mlp_flops_per_sample(),
                          "per_batch": mlp_throughput(ctx, a.batches)}))
        ctx.close()
        return
    train = make_dataset(ctx, a.train, seed=101, low_rays=a.train_rays, high_rays=a.train_label_rays,
                         copies=a.copies)
    t_data = time.time() - t0
    test_scenes = learned_scenes(202, a.test)
    test = make_dataset(ctx, a.test, seed=202, low_rays=a.rays, high_rays=a.test_label_rays)
    t1 = time.time()
    mlp, hist = fit(ctx, train, steps=a.steps, batch=512, lr=1e-3, weight_decay=1e-2, log_every=a.steps // 4)
    t_fit = time.time() - t1
    res = sweep(ctx, mlp, test, a.rays, test_scenes)
    res.update({"train_scenes": a.train, "train_rows": int(train.X.shape[0]), "test_scenes": a.test,
                "train_label_rays": a.train_label_rays, "test_label_rays": a.test_label_rays,
                "train_label_frac": train.label_frac, "test_label_frac": test.label_frac,
                "train_data_s": round(t_data, 1), "fit_s": round(t_fit, 1), "loss": hist})
    print(json.dumps(res, default=float))
    mlp.close()
    ctx.close()


if __name__ == "__main__":
    main()
