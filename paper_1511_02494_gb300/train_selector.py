"""Builds the learned selector: training set on the GPU, then training with
the library's own kernels.

The training set follows the paper's offline stage (Section 3.2.2, "Training
Data Selection" and "Labeling") with two changes: the matrices are seeded
synthetic ones from four generator families (the University of Florida
collection is not available), and each matrix is labelled with the variant
that was actually fastest when every variant was timed on it (the paper
labels with its profiling classifier).  For every matrix it records the
16-entry feature vector, the time of every variant, the profiling runs and
their rule's choice, and the cost of feature extraction and profiling.

Training: a 16-64-64-K ReLU network, full-batch Adam on the GPU
(spmv_mlp_loss_grad_soft + spmv_mlp_adam), 80/20 split by seed.  Targets are
cost-sensitive distributions over the variants built from the measured times
(soft_targets); their sharpness beta is picked on a validation quarter of
the training split.  The fallback margin (below which the profiling rule
decides instead of the network) is chosen on out-of-fold logits of the
training split: four networks, each trained without one quarter of it,
give every training matrix the margin of a network that has not seen it.
Outputs (in --out):
selector_dataset.npz, selector_mlp.bin, selector_report.json.

    python -m paper_1511_02494_gb300.train_selector --out DIR [--n 2000]

A stored training set that lacks variants added to the library since is
completed first (those variants are timed on its matrices).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_1511_02494_gb300 as sp  # noqa: E402
import synth  # noqa: E402

N_VAR = len(sp.VARIANTS)
FIELDS = ("seed", "family", "n_rows", "nnz", "vec", "times", "prof", "rule_variant",
          "features_ms", "profile_ms")


def matrix_spec(i: int):
    """Family and target row count of matrix i (log-uniform in [1e4, 1e7])."""
    g = np.random.default_rng(10_000 + i)
    family = synth.FAMILIES[i % 4]
    n_rows = int(round(10 ** g.uniform(4.0, 7.0)))
    return family, n_rows


def time_prepared(P, x, y, budget_ms: float = 25.0, window_ms: float = 0.5):
    """Milliseconds per SpMV of a prepared matrix, as in a solver's loop:
    after a warm-up, one launch is timed; unless it took budget_ms or more,
    the median of three runs of back-to-back launches, each about window_ms
    long (so that the few microseconds of launch and event overhead do not
    decide between variants of small matrices)."""
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sp.spmv(P, x, y)  # warm-up
    e0.record()
    sp.spmv(P, x, y)
    e1.record()
    e1.synchronize()
    first = e0.elapsed_time(e1)
    if first >= budget_ms:
        return float(first)
    reps = int(min(200, max(1, window_ms / max(first, 1e-3))))
    ts = []
    for _ in range(3):
        e0.record()
        for _ in range(reps):
            sp.spmv(P, x, y)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1) / reps)
    return float(np.median(ts))


def time_variant(dA, v: int, x, y, budget_ms: float = 25.0):
    P = sp.spmv_prepare(dA, sp.make_choice(v), trusted=True)
    t = time_prepared(P, x, y, budget_ms)
    P.free()
    return t


def build_dataset(n: int, out_path: str, resume: bool = True, log=print):
    rows = {k: [] for k in FIELDS}
    done = set()
    if resume and os.path.exists(out_path):
        d = np.load(out_path)
        for k in FIELDS:
            rows[k] = list(d[k])
        done = set(int(s) for s in d["seed"])
        log(f"resuming with {len(done)} matrices")
    t_start = time.time()
    for i in range(n):
        if i in done:
            continue
        family, n_rows = matrix_spec(i)
        A = synth.family_matrix(family, n_rows, seed=i, device="cuda")
        dA = sp.DeviceCSR(A.n_rows, A.n_cols, A.rowptr.contiguous(), A.colind.contiguous(),
                          A.val.contiguous())
        x = synth.uniform_vector(A.n_cols, i, device="cuda")
        y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        sp.spmv_features(dA)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        f = sp.spmv_features(dA)
        feat_ms = (time.perf_counter() - t0) * 1e3
        prof = sp.spmv_profile(dA, x, reps=3)
        rule = sp.spmv_select(profile=prof)
        times = [time_variant(dA, v, x, y) for v in range(N_VAR)]
        rows["seed"].append(i)
        rows["family"].append(synth.FAMILIES.index(family))
        rows["n_rows"].append(A.n_rows)
        rows["nnz"].append(A.nnz)
        rows["vec"].append(np.array(list(f.vec), np.float32))
        rows["times"].append(np.array(times, np.float64))
        rows["prof"].append(np.array([prof.s_noxmiss, prof.s_inflate, prof.s_balance], np.float64))
        rows["rule_variant"].append(rule.variant)
        rows["features_ms"].append(feat_ms)
        rows["profile_ms"].append(prof.total_ms)
        del dA, A, x, y
        if (i + 1) % 50 == 0 or i == n - 1:
            np.savez(out_path, **{k: np.array(v) for k, v in rows.items()})
            torch.cuda.empty_cache()
            log(f"{i + 1}/{n} matrices, {time.time() - t_start:.0f} s")
    np.savez(out_path, **{k: np.array(v) for k, v in rows.items()})
    return {k: np.array(v) for k, v in rows.items()}


def rule_of(prof_row) -> int:
    p = sp.Profile()
    p.s_noxmiss, p.s_inflate, p.s_balance = (float(v) for v in prof_row)
    return sp.spmv_select(profile=p).variant


def extend_dataset(out_path: str, log=print):
    """Times the variants a stored training set lacks (columns added to the
    library after it was built) on every one of its matrices, regenerated
    from their seeds; resumable through NaN entries, saved every 50."""
    d = {k: np.array(v) for k, v in np.load(out_path).items()}
    times = d["times"].astype(np.float64)
    if times.shape[1] < N_VAR:
        times = np.concatenate([times, np.full((times.shape[0], N_VAR - times.shape[1]), np.nan)], 1)
    todo = np.where(np.isnan(times).any(1))[0]
    log(f"timing missing variants on {len(todo)} matrices")
    t_start = time.time()
    for n, row in enumerate(todo):
        i = int(d["seed"][row])
        family, n_rows = matrix_spec(i)
        A = synth.family_matrix(family, n_rows, seed=i, device="cuda")
        dA = sp.DeviceCSR(A.n_rows, A.n_cols, A.rowptr.contiguous(), A.colind.contiguous(),
                          A.val.contiguous())
        x = synth.uniform_vector(A.n_cols, i, device="cuda")
        y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        for v in np.where(np.isnan(times[row]))[0]:
            times[row, v] = time_variant(dA, int(v), x, y)
        del dA, A, x, y
        if (n + 1) % 50 == 0 or n == len(todo) - 1:
            d["times"] = times
            np.savez(out_path, **d)
            torch.cuda.empty_cache()
            log(f"{n + 1}/{len(todo)} matrices, {time.time() - t_start:.0f} s")
    d["times"] = times
    return d


def init_params(h1, h2, k, seed=0):
    g = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((16, h1), (h1, h2), (h2, k)):
        bound = math.sqrt(6.0 / fan_in)
        parts.append(g.uniform(-bound, bound, (fan_out, fan_in)).astype(np.float32).reshape(-1))
        parts.append(np.zeros(fan_out, np.float32))
    return np.concatenate(parts)


def soft_targets(times: np.ndarray, beta: float) -> np.ndarray:
    """Cost-sensitive targets: q_v proportional to (t_best / t_v)^beta, so a
    variant 5 % slower than the best keeps weight 1.05^-beta and a variant
    twice as slow almost none.  beta = inf gives the one-hot best label."""
    r = times / times.min(1, keepdims=True)
    if not np.isfinite(beta):
        q = (r == 1.0).astype(np.float64)
    else:
        q = r ** -beta
    return (q / q.sum(1, keepdims=True)).astype(np.float32)


def train(z: np.ndarray, targets: np.ndarray, h1=64, h2=64, k=N_VAR, steps=3000, lr=3e-3,
          wd=1e-4, seed=0, log=print):
    """Full-batch Adam with the library's loss/gradient and Adam kernels;
    targets are integer labels [n] or target distributions [n][k].  Returns
    the parameters, the loss history and the steps' elapsed time on the
    stream (ms, CUDA events; host launch gaps included)."""
    p = torch.from_numpy(init_params(h1, h2, k, seed)).cuda()
    g = torch.zeros_like(p)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    dz = torch.from_numpy(np.ascontiguousarray(z, np.float32)).cuda()
    soft = targets.ndim == 2
    dl = torch.from_numpy(np.ascontiguousarray(targets, np.float32 if soft else np.int32)).cuda()
    hist = []
    gpu_ms = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for step in range(1, steps + 1):
        if soft:
            sp.spmv_mlp_loss_grad_soft(p, h1, h2, k, dz, dl, g, loss)
        else:
            sp.spmv_mlp_loss_grad(p, h1, h2, k, dz, dl, g, loss)
        sp.spmv_mlp_adam(p, g, m, v, step, lr=lr, weight_decay=wd)
        if step % 500 == 0 or step == 1:
            e1.record()
            hist.append((step, float(loss.item())))  # synchronizes
            gpu_ms += e0.elapsed_time(e1)
            log(f"step {step} loss {hist[-1][1]:.4f}")
            e0.record()
    e1.record()
    e1.synchronize()
    gpu_ms += e0.elapsed_time(e1)
    return p.cpu().numpy(), hist, gpu_ms


def logits_of(params, mean, istd, vec, h1, h2, k):
    out = torch.empty((vec.shape[0], k), dtype=torch.float32, device="cuda")
    sp.spmv_mlp_forward(torch.from_numpy(params).cuda(), torch.from_numpy(mean).cuda(),
                        torch.from_numpy(istd).cuda(), h1, h2, k,
                        torch.from_numpy(np.ascontiguousarray(vec, np.float32)).cuda(), out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def policy_times(times, pred, margin, rule, mu):
    pick = np.where(margin < mu, rule, pred)
    return times[np.arange(len(times)), pick], pick


def geomean(a):
    return float(np.exp(np.mean(np.log(a))))


def evaluate(d, params, mean, istd, mu, h1, h2, k, idx):
    times = d["times"][idx]
    best = times.min(1)
    lg = logits_of(params, mean, istd, d["vec"][idx], h1, h2, k)
    pred = lg.argmax(1)
    srt = np.sort(lg, 1)
    margin = srt[:, -1] - srt[:, -2]
    rule = d["rule_variant"][idx]
    t_mlp = times[np.arange(len(idx)), pred]
    t_pol, pick = policy_times(times, pred, margin, rule, mu)
    t_rule = times[np.arange(len(idx)), rule]
    fixed = int(np.argmin([geomean(times[:, v] / best) for v in range(times.shape[1])]))
    plain = times[:, 0]
    feat_spmv = d["features_ms"][idx] / plain
    prof_spmv = d["profile_ms"][idx] / plain
    return {
        "matrices": int(len(idx)),
        "label_counts": np.bincount(times.argmin(1), minlength=times.shape[1]).tolist(),
        "misselection_mlp": float(np.mean(pred != times.argmin(1))),
        "misselection_policy": float(np.mean(pick != times.argmin(1))),
        "misselection_rule": float(np.mean(rule != times.argmin(1))),
        "slowdown_vs_best_geomean": {"mlp": geomean(t_mlp / best), "mlp_with_fallback": geomean(t_pol / best),
                                     "profile_rule": geomean(t_rule / best),
                                     "best_fixed_variant": geomean(times[:, fixed] / best),
                                     "plain_csr": geomean(plain / best)},
        "best_fixed_variant": sp.VARIANTS[fixed],
        "speedup_vs_plain_geomean": {"best": geomean(plain / best), "mlp": geomean(plain / t_mlp),
                                     "mlp_with_fallback": geomean(plain / t_pol),
                                     "profile_rule": geomean(plain / t_rule)},
        "fallback_rate": float(np.mean(margin < mu)),
        "overhead_in_plain_spmvs": {"features_median": float(np.median(feat_spmv)),
                                    "profile_median": float(np.median(prof_spmv)),
                                    "features_mean": float(np.mean(feat_spmv)),
                                    "profile_mean": float(np.mean(prof_spmv))},
    }


def standardize(vec, idx):
    mean = vec[idx].mean(0).astype(np.float32)
    sd = vec[idx].std(0)
    return mean, np.where(sd > 1e-6, 1.0 / np.maximum(sd, 1e-6), 0.0).astype(np.float32)


def margin_curve(times, logits, rule, cands):
    """Geometric-mean slowdown against the best and fallback rate of the
    policy 'network, or the profiling rule when the top-two logit margin is
    below mu', for each mu in cands."""
    srt = np.sort(logits, 1)
    margin = srt[:, -1] - srt[:, -2]
    best = times.min(1)
    pred = logits.argmax(1)
    return [{"mu": float(mu), "fallback_rate": float(np.mean(margin < mu)),
             "slowdown": geomean(policy_times(times, pred, margin, rule, mu)[0] / best)} for mu in cands]


def calibrate_margin(d, tr, beta, h1, h2, k, steps):
    """The fallback margin mu from out-of-fold logits.  The training split is
    cut into four folds by seed (seed % 5 = 1, 2, 3, 4); a network trained
    (as the final one, same beta and steps) on three folds gives the logits
    of the fourth, so every training matrix gets the margin of a network that
    has not seen it -- the situation of a new matrix.  mu is the candidate
    (0, or a quantile of those margins) with the lowest out-of-fold slowdown
    against the best variant; 0 unless a positive mu is strictly better."""
    vec = d["vec"].astype(np.float32)
    seeds = d["seed"][tr]
    oof = np.empty((len(tr), k), np.float32)
    for f in (1, 2, 3, 4):
        out_pos = np.where(seeds % 5 == f)[0]
        fit = tr[seeds % 5 != f]
        mean, istd = standardize(vec, fit)
        p, _, _ = train(((vec - mean) * istd)[fit], soft_targets(d["times"][fit], beta), h1, h2, k,
                        steps=steps, log=lambda *_: None)
        oof[out_pos] = logits_of(p, mean, istd, vec[tr[out_pos]], h1, h2, k)
    srt = np.sort(oof, 1)
    margin = srt[:, -1] - srt[:, -2]
    cands = [0.0] + sorted(set(np.quantile(margin, np.linspace(0.01, 0.6, 40)).tolist()))
    curve = margin_curve(d["times"][tr], oof, d["rule_variant"][tr], cands)
    best = min(curve, key=lambda c: (c["slowdown"], c["mu"]))
    mu = best["mu"] if best["slowdown"] < curve[0]["slowdown"] else 0.0
    return float(mu), {"method": "out-of-fold logits, 4 folds of the training split by seed",
                       "oof_slowdown_without_fallback": curve[0]["slowdown"],
                       "oof_slowdown_at_mu": next(c["slowdown"] for c in curve if c["mu"] == mu),
                       "curve": curve}


# Launch configurations of SLICED among which the second-level network
# chooses (threads_per_row = slices per warp, block_nnz = sort window,
# items_per_warp = row-length cap; 0 = the prepare step's own rule)
SLICED_CONFIGS = (
    (0, 0, 0),        # the structural rules
    (1, 1, 1024),     # rows in order
    (4, 1, 1024),     # rows in order, four slices per warp
    (1, 4096, 32),    # sorted, cap 32
    (4, 4096, 32),    # sorted, cap 32, four slices per warp
    (1, 256, 1024),   # sorted in windows of 256
    (1, 4096, 64),    # sorted, cap 64
    (1, 4096, 1024),  # sorted, cap 1024
    (2, 1, 1024),     # rows in order, two slices per warp
)


def time_choice(dA, ch, x, y, budget_ms: float = 25.0):
    P = sp.spmv_prepare(dA, ch, trusted=True)
    t = time_prepared(P, x, y, budget_ms)
    P.free()
    return t


def sliced_dataset(d, out_path: str, retime: bool = False, log=print):
    """Times every SLICED launch configuration on the stored matrices
    (regenerated from their seeds), in the stored order; resumable through
    NaN entries (saved every 200 matrices); retime times every one again."""
    times = np.full((len(d["seed"]), len(SLICED_CONFIGS)), np.nan)
    if os.path.exists(out_path):
        s = np.load(out_path)
        if np.array_equal(s["seed"], d["seed"]) and s["times"].shape[1] == len(SLICED_CONFIGS):
            if not retime:
                times = s["times"].astype(np.float64)
    if retime or not os.path.exists(out_path):
        np.savez(out_path, seed=d["seed"], times=times, configs=np.array(SLICED_CONFIGS, np.int32))
    todo = np.where(np.isnan(times).any(1))[0]
    if len(todo) == 0:
        return times
    log(f"timing SLICED configurations on {len(todo)} matrices")
    t0 = time.time()
    for n, row in enumerate(todo):
        i = d["seed"][row]
        family, n_rows = matrix_spec(int(i))
        A = synth.family_matrix(family, n_rows, seed=int(i), device="cuda")
        dA = sp.DeviceCSR(A.n_rows, A.n_cols, A.rowptr.contiguous(), A.colind.contiguous(),
                          A.val.contiguous())
        x = synth.uniform_vector(A.n_cols, int(i), device="cuda")
        y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        for j, (r, sigma, cap) in enumerate(SLICED_CONFIGS):
            ch = sp.make_choice("sliced", threads_per_row=r, block_nnz=sigma, items_per_warp=cap)
            times[row, j] = time_choice(dA, ch, x, y)
        del dA, A, x, y
        if (n + 1) % 200 == 0 or n == len(todo) - 1:
            np.savez(out_path, seed=d["seed"], times=times, configs=np.array(SLICED_CONFIGS, np.int32))
            torch.cuda.empty_cache()
            log(f"{n + 1}/{len(todo)} matrices, {time.time() - t0:.0f} s")
    return times


def train_second_level(args, d, first):
    """The second level of selection: a 16-64-64-C network choosing SLICED's
    launch configuration from the same features, trained like the first
    level (cost-sensitive targets, beta on a validation quarter), saved with
    its launch table; the report compares it with the structural rules."""
    tcfg = sliced_dataset(d, os.path.join(args.out, "sliced_dataset.npz"), retime=args.retime_configs)
    seeds, vec = d["seed"], d["vec"].astype(np.float32)
    tr, te = np.where(seeds % 5 != 0)[0], np.where(seeds % 5 == 0)[0]
    fit, val = np.where((seeds % 5 != 0) & (seeds % 5 != 4))[0], np.where(seeds % 5 == 4)[0]
    h1, h2, k = 64, 64, len(SLICED_CONFIGS)

    def norm(idx):
        mean = vec[idx].mean(0).astype(np.float32)
        sd = vec[idx].std(0)
        return mean, np.where(sd > 1e-6, 1.0 / np.maximum(sd, 1e-6), 0.0).astype(np.float32)

    mean_f, istd_f = norm(fit)
    scores = {}
    for beta in args.betas:
        pf, _, _ = train(((vec - mean_f) * istd_f)[fit], soft_targets(tcfg[fit], beta), h1, h2, k,
                         steps=args.steps, log=lambda *_: None)
        lg = logits_of(pf, mean_f, istd_f, vec[val], h1, h2, k)
        scores[str(beta)] = geomean(tcfg[val, lg.argmax(1)] / tcfg[val].min(1))
    beta = float(min(args.betas, key=lambda b_: scores[str(b_)]))
    mean, istd = norm(tr)
    params, _, train_ms = train(((vec - mean) * istd)[tr], soft_targets(tcfg[tr], beta), h1, h2, k,
                                steps=args.steps, log=lambda *_: None)
    sl = sp.VARIANT_IDS["sliced"]
    model = sp.spmv_model_create(h1, h2, k, mean, istd, params, [sl] * k, 0.0)
    sp.spmv_model_set_launch(model, np.array(SLICED_CONFIGS, np.int32))
    sp.spmv_model_save(model, os.path.join(args.out, "selector_sliced_mlp.bin"))
    pick = logits_of(params, mean, istd, vec, h1, h2, k).argmax(1)
    # two levels against the best over every variant and every SLICED configuration
    first_pick = np.array([int(np.argmax(sp.spmv_model_logits(first, v, N_VAR))) for v in vec])
    var_t = d["times"]
    one = var_t[np.arange(len(vec)), first_pick]
    two = np.where(first_pick == sl, tcfg[np.arange(len(vec)), pick], one)
    overall = np.minimum(var_t.min(1), tcfg.min(1))
    rep = {"configs": [list(c) for c in SLICED_CONFIGS], "beta": beta, "beta_validation_slowdown": scores,
           "training_stream_ms": round(train_ms, 2)}
    for name, idx in (("train", tr), ("test", te)):
        best = tcfg[idx].min(1)
        rep[name] = {
            "matrices": int(len(idx)),
            "best_config_counts": np.bincount(tcfg[idx].argmin(1), minlength=k).tolist(),
            "sliced_slowdown_vs_best_config": {
                "network": geomean(tcfg[idx, pick[idx]] / best),
                "structural_rules": geomean(tcfg[idx, 0] / best),
                "each_config": [geomean(tcfg[idx, j] / best) for j in range(k)]},
            "slowdown_vs_best_overall": {
                "first_level_only": geomean(one[idx] / overall[idx]),
                "two_levels": geomean(two[idx] / overall[idx])},
            "first_level_picks_sliced": float(np.mean(first_pick[idx] == sl))}
    with open(os.path.join(args.out, "sliced_report.json"), "w") as f:
        json.dump(rep, f, indent=1)
    print(json.dumps(rep["test"], indent=1))


# SLICED forms beyond the second level's launch configurations that the
# class table may assign: (threads_per_row, block_nnz, items_per_warp,
# index_coding) -- Table 2's delta coding in the two base layouts
CLASS_EXTRA = (
    (1, 1, 1024, 1),   # rows in order, delta-coded columns
    (1, 4096, 32, 1),  # sorted, cap 32, delta-coded columns
)


def class_table(args, d):
    """The profiling rule's class -> choice table (Table 2 on GB300): for each
    class the rule names on the training split, the SLICED form -- one of the
    second level's launch configurations or CLASS_EXTRA -- with the lowest
    geometric-mean slowdown against the best form; written with its held-out
    evaluation to class_table.json (CLASS_EXTRA timings in class_dataset.npz)."""
    tcfg = sliced_dataset(d, os.path.join(args.out, "sliced_dataset.npz"))
    path = os.path.join(args.out, "class_dataset.npz")
    extra = None
    if os.path.exists(path):
        s = np.load(path)
        if np.array_equal(s["seed"], d["seed"]) and s["times"].shape[1] == len(CLASS_EXTRA):
            extra = s["times"]
    if extra is None:
        extra = np.empty((len(d["seed"]), len(CLASS_EXTRA)))
        t0 = time.time()
        for row, i in enumerate(d["seed"]):
            family, n_rows = matrix_spec(int(i))
            A = synth.family_matrix(family, n_rows, seed=int(i), device="cuda")
            dA = sp.DeviceCSR(A.n_rows, A.n_cols, A.rowptr.contiguous(), A.colind.contiguous(),
                              A.val.contiguous())
            x = synth.uniform_vector(A.n_cols, int(i), device="cuda")
            y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
            for j, (r, sigma, cap, code) in enumerate(CLASS_EXTRA):
                ch = sp.make_choice("sliced", threads_per_row=r, block_nnz=sigma, items_per_warp=cap,
                                    index_coding=code)
                extra[row, j] = time_choice(dA, ch, x, y)
            del dA, A, x, y
            if (row + 1) % 500 == 0:
                torch.cuda.empty_cache()
                print(f"{row + 1}/{len(d['seed'])} matrices, {time.time() - t0:.0f} s", flush=True)
        np.savez(path, seed=d["seed"], times=extra, forms=np.array(CLASS_EXTRA, np.int32))
    forms = [tuple(c) + (0,) for c in SLICED_CONFIGS] + list(CLASS_EXTRA)
    t_all = np.concatenate([tcfg, extra], 1)
    th = sp.spmv_default_thresholds()
    cls = np.array([_rule_class(p, th) for p in d["prof"]])
    seeds = d["seed"]
    tr, te = np.where(seeds % 5 != 0)[0], np.where(seeds % 5 == 0)[0]
    best = t_all.min(1)
    table, per_class = [], {}
    for c in range(4):
        m = tr[cls[tr] == c]
        slow = [geomean(t_all[m, j] / best[m]) if len(m) else math.inf for j in range(len(forms))]
        j = int(np.argmin(slow)) if len(m) else 0
        table.append([sp.VARIANT_IDS["sliced"], *forms[j]])
        per_class[sp.CLASSES[c]] = {"train_matrices": int(len(m)), "form": list(forms[j]),
                                    "train_slowdown_each_form": slow}
    pick = np.array([table[c][1:] for c in cls])
    idx = [forms.index(tuple(p)) for p in pick]
    t_rule = t_all[np.arange(len(seeds)), idx]
    overall = np.minimum(d["times"].min(1), t_all.min(1))
    rep = {"forms": [list(f) for f in forms], "table": table, "classes": per_class,
           "test": {"matrices": int(len(te)),
                    "rule_with_class_forms_vs_best_overall": geomean(t_rule[te] / overall[te]),
                    "rule_with_sliced_rules_vs_best_overall": geomean(tcfg[te, 0] / overall[te]),
                    "rule_with_class_forms_vs_best_variant": geomean(t_rule[te] / d["times"][te].min(1))}}
    with open(os.path.join(args.out, "class_table.json"), "w") as f:
        json.dump(rep, f, indent=1)
    print(json.dumps(rep["test"], indent=1))


def _rule_class(prof_row, th) -> int:
    p = sp.Profile()
    p.s_noxmiss, p.s_inflate, p.s_balance = (float(v) for v in prof_row)
    return sp.spmv_classify_profile(p, th)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--n", type=int, default=2000)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--no-resume", action="store_true")
    ap.add_argument("--betas", type=float, nargs="+", default=[2.0, 4.0, 8.0, 16.0, 32.0, math.inf])
    ap.add_argument("--retime", nargs="+", default=[], choices=list(sp.VARIANTS),
                    help="variants whose kernels changed: time them again on every stored matrix")
    ap.add_argument("--second-level", action="store_true",
                    help="also time SLICED's launch configurations and train the second-level network")
    ap.add_argument("--class-table", action="store_true",
                    help="only build the profiling rule's class -> SLICED form table from the stored data")
    ap.add_argument("--retime-configs", action="store_true",
                    help="with --second-level: time every SLICED launch configuration again")
    args = ap.parse_args()
    os.makedirs(args.out, exist_ok=True)
    from paper_1511_02494_gb300.build import build
    build()
    ds_path = os.path.join(args.out, "selector_dataset.npz")
    d = build_dataset(args.n, ds_path, resume=not args.no_resume)
    if args.class_table:
        return class_table(args, d)
    if args.retime:
        times = d["times"].astype(np.float64)
        if times.shape[1] < N_VAR:
            times = np.concatenate([times, np.full((times.shape[0], N_VAR - times.shape[1]), np.nan)], 1)
        for v in args.retime:
            times[:, sp.VARIANTS.index(v)] = np.nan
        d["times"] = times
        np.savez(ds_path, **d)
    if d["times"].shape[1] < N_VAR or np.isnan(d["times"]).any():
        d = extend_dataset(ds_path)
    # the profiling rule's choice under the library's current class map,
    # from the stored probe speedups
    d["rule_variant"] = np.array([rule_of(p) for p in d["prof"]], np.int64)
    seeds = d["seed"]
    test = np.where(seeds % 5 == 0)[0]
    tr = np.where(seeds % 5 != 0)[0]
    vec = d["vec"].astype(np.float32)
    mean = vec[tr].mean(0).astype(np.float32)
    sd = vec[tr].std(0)
    istd = np.where(sd > 1e-6, 1.0 / np.maximum(sd, 1e-6), 0.0).astype(np.float32)
    z = ((vec - mean) * istd).astype(np.float32)
    h1, h2, k = 64, 64, N_VAR
    # beta of the cost-sensitive targets, chosen on a validation part of the
    # training split (seed % 5 == 4), then the network is trained on all of it
    fit = np.where((seeds % 5 != 0) & (seeds % 5 != 4))[0]
    val = np.where(seeds % 5 == 4)[0]
    mean_f = vec[fit].mean(0).astype(np.float32)
    sd_f = vec[fit].std(0)
    istd_f = np.where(sd_f > 1e-6, 1.0 / np.maximum(sd_f, 1e-6), 0.0).astype(np.float32)
    z_f = ((vec - mean_f) * istd_f).astype(np.float32)
    beta_scores = {}
    for beta in args.betas:
        pf, _, _ = train(z_f[fit], soft_targets(d["times"][fit], beta), h1, h2, k, steps=args.steps,
                      log=lambda *_: None)
        lg = logits_of(pf, mean_f, istd_f, vec[val], h1, h2, k)
        t_val = d["times"][val]
        beta_scores[str(beta)] = geomean(t_val[np.arange(len(val)), lg.argmax(1)] / t_val.min(1))
        print(f"beta {beta}: validation slowdown {beta_scores[str(beta)]:.4f}", flush=True)
    beta = float(min(args.betas, key=lambda b_: beta_scores[str(b_)]))
    params, hist, train_ms = train(z[tr], soft_targets(d["times"][tr], beta), h1, h2, k, steps=args.steps)
    mu, calib = calibrate_margin(d, tr, beta, h1, h2, k, args.steps)
    model = sp.spmv_model_create(h1, h2, k, mean, istd, params, list(range(k)), mu)
    sp.spmv_model_save(model, os.path.join(args.out, "selector_mlp.bin"))
    report = {"train": evaluate(d, params, mean, istd, mu, h1, h2, k, tr),
              "test": evaluate(d, params, mean, istd, mu, h1, h2, k, test),
              "min_margin": mu, "margin_calibration": calib,
              "loss_history": hist, "variants": list(sp.VARIANTS),
              "beta": beta, "beta_validation_slowdown": beta_scores,
              "training_stream_ms": round(train_ms, 2),
              "training_ms_per_step": round(train_ms / max(args.steps, 1), 4),
              "network": [16, h1, h2, k]}
    with open(os.path.join(args.out, "selector_report.json"), "w") as f:
        json.dump(report, f, indent=1)
    print(json.dumps(report["test"], indent=1))
    if args.second_level:
        train_second_level(args, d, model)


if __name__ == "__main__":
    main()
