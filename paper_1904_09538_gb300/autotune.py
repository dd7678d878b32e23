"""Model-guided autotuning (Section "Assumptions and Limitations": a
calibrated model as a pruning heuristic for choosing among mathematically
equivalent kernel variants; important accuracy gains come from a few extra
on-line calibration runs).

rank_family(): for a family of variants (the 24 register-tiled SIMT matmul
tile shapes at n = 7680, the multiple of lcm(96, 256) nearest 8192; the 12
TMA-staged stencil tiles at n = 16384), first prune the variants whose
compiled form cannot pay off (register spills to local memory, or no CTA
resident per SM: pm_kernel_resources), calibrate a cost model on cheap runs
of the surviving variants at small sizes, predict them at the target size
from their exact counts, then time every variant at the target size and
report how well the predicted order matches the measured one (Spearman,
Kendall, best-variant hit, the measured time of the predicted best relative
to the true best, and whether pruning removed the true best).

tune_fit_threads(): pick the CTA size of the batched calibration kernel by
timing the plan for each candidate.
"""
import itertools
import math
import time

import numpy as np

from . import Model, FitPlan, run, resources
from .experiments import Buffers, spearman, kendall

SIMT_SHAPES = [dict(BM=bm, BN=bn, BK=bk) for bm, bn, bk in
               itertools.product((64, 96, 128, 256), (64, 128, 256), (32, 64))]

SIMT_MODEL = (
    "p_launch * f_sync_kernel_launch + p_group * f_thread_groups + p_bar * f_sync_barrier_local * f_thread_groups + "
    "(p_gv * f_mem_access_global_float32x4) * (tanh(p_edge * ((p_gv * f_mem_access_global_float32x4) - "
    "(p_madd * f_op_float32_madd + p_ls * f_mem_access_local_float32 + p_lv * f_mem_access_local_float32x4))) + 1) / 2"
    " + (p_madd * f_op_float32_madd + p_ls * f_mem_access_local_float32 + p_lv * f_mem_access_local_float32x4) * "
    "(tanh(p_edge * ((p_madd * f_op_float32_madd + p_ls * f_mem_access_local_float32 + "
    "p_lv * f_mem_access_local_float32x4) - (p_gv * f_mem_access_global_float32x4))) + 1) / 2")


# 8 outputs per work-item: the faster work-item shape for every tile with at most 2^19 tiles at n = 16384
STENCIL_SHAPES = [dict(BX=bx, BY=by, V=8) for bx in (32, 64, 128) for by in (4, 8, 16, 32)]

# linear model of Section "Finite Differences" on the tile family's features
STENCIL_MODEL = ("p_launch * f_sync_kernel_launch + p_group * f_thread_groups + "
                 "p_bar * f_sync_barrier_local * f_thread_groups + p_u * f_mem_access_tag:fdb-u + "
                 "p_res * f_mem_access_tag:fdb-res + p_lmem * f_mem_access_local_float32 + "
                 "p_add * f_op_float32_add + p_madd * f_op_float32_madd")


def prune(kernel, variants):
    """Split variants into (kept, pruned) by their compiled resources."""
    kept, pruned = [], []
    for p in variants:
        r = resources(kernel, **p)
        (pruned if r["local_bytes_per_thread"] > 0 or r["blocks_per_sm"] == 0 else kept).append((p, r))
    return kept, pruned


def _time(kernel, variants, bufs, trials, flush_l2=True):
    out = []
    for p in variants:
        tm = run(kernel, bufs.get(kernel, p), warmup=2, trials=trials, flush_l2=flush_l2, **p)
        out.append(tm["mean_ms"] * 1e-3)
    return np.array(out)


def rank_family(kernel="mm_simt", shapes=None, calib_sizes=(3072, 4608), target=7680, trials=5, seed=7,
                expr=SIMT_MODEL, flops_per_n3=2.0, bytes_fn=None):
    import torch
    shapes = shapes or SIMT_SHAPES
    dev = torch.device("cuda", torch.cuda.current_device())
    bufs = Buffers(torch, dev, seed)
    targets = [dict(s, n=target) for s in shapes]
    kept, pruned = prune(kernel, targets)
    keep_shapes = [{k: v for k, v in p.items() if k != "n"} for p, _ in kept]
    m = Model("f_wall_time", expr)
    calib = [dict(s, n=n) for n in calib_sizes for s in keep_shapes]
    Xc = np.stack([m.feature_values(kernel, **p) for p in calib])
    t0 = time.perf_counter()
    tc = _time(kernel, calib, bufs, trials)
    calib_s = time.perf_counter() - t0
    plan = FitPlan([m], [len(tc)])
    p, reps = plan.run(Xc.ravel(), tc)
    kt = [q for q, _ in kept]
    Xt = np.stack([m.feature_values(kernel, **q) for q in kt])
    pred = m.predict(p, Xt)
    t0 = time.perf_counter()
    meas = _time(kernel, kt, bufs, trials)
    meas_s = time.perf_counter() - t0
    meas_pruned = _time(kernel, [q for q, _ in pruned], bufs, trials) if pruned else np.array([])
    best_pred, best_meas = int(np.argmin(pred)), int(np.argmin(meas))
    top3 = set(np.argsort(pred)[:3].tolist())
    best_all = float(min(meas.min(), meas_pruned.min() if len(meas_pruned) else np.inf))
    rate = (lambda t: flops_per_n3 * target ** 3 / t / 1e12) if bytes_fn is None else \
        (lambda t: bytes_fn(target) / t / 1e9)
    return {
        "kernel": kernel, "target_n": target, "calib_sizes": list(calib_sizes), "n_shapes": len(shapes),
        "n_pruned": len(pruned), "pruned": [{"shape": q, "resources": r, "measured_s": float(t)}
                                            for (q, r), t in zip(pruned, meas_pruned)],
        "pruning_removed_best": bool(len(meas_pruned) and meas_pruned.min() < meas.min()),
        "params": dict(zip(m.params, [float(x) for x in p])), "fit": reps[0],
        "spearman": spearman(pred, meas), "kendall": kendall(pred, meas),
        "best_predicted": kt[best_pred], "best_measured": kt[best_meas],
        "best_hit": best_pred == best_meas, "best_in_predicted_top3": best_meas in top3,
        "slowdown_of_predicted_best": float(meas[best_pred] / best_all),
        # the model as a pruning heuristic: time only its k best predictions, keep the fastest
        "slowdown_after_timing_predicted_top_k": {str(k): float(meas[np.argsort(pred)[:k]].min() / best_all)
                                                  for k in (1, 3, 5) if k <= len(pred)},
        "best_measured_rate": rate(best_all), "rate_unit": "TFLOP/s" if bytes_fn is None else "GB/s",
        "geomean_rel_err": float(math.exp(np.mean(np.log(np.abs(pred - meas) / meas)))),
        "calibration_seconds": calib_s, "exhaustive_seconds": meas_s,
        "rows": [{"shape": q, "resources": r, "measured_s": float(a), "predicted_s": float(b)}
                 for (q, r), a, b in zip(kept, meas, pred)],
    }


def rank_stencil(target=16384, calib_sizes=(4096, 8192), trials=5, seed=7):
    """The 12 stencil tile shapes (BX x BY outputs per CTA) at n = 16384."""
    return rank_family("fd_block", STENCIL_SHAPES, calib_sizes, target, trials, seed, STENCIL_MODEL,
                       bytes_fn=lambda n: 4.0 * ((n + 2) * (n + 4) + n * n))


def tune_fit_threads(models, Xs, ts, p0s=None, candidates=(64, 128, 256, 512), reps=10):
    """Time the batched calibration plan at each CTA size; return the fastest
    and all timings (seconds per plan run)."""
    X = np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in Xs])
    t = np.concatenate([np.asarray(x, dtype=np.float64) for x in ts])
    p0 = None if p0s is None else np.concatenate([np.asarray(q, dtype=np.float64) for q in p0s])
    times = {}
    for th in candidates:
        plan = FitPlan(models, [len(x) for x in ts], p0_given=p0s is not None, threads=th)
        plan.run(X, t, p0)
        t0 = time.perf_counter()
        for _ in range(reps):
            plan.run(X, t, p0)
        times[th] = (time.perf_counter() - t0) / reps
    best = min(times, key=times.get)
    return best, times


if __name__ == "__main__":
    import json
    import sys
    out = {"mm_simt": rank_family(), "fd_block": rank_stencil()}
    json.dump(out, open(sys.argv[1], "w") if len(sys.argv) > 1 else sys.stdout, indent=1, default=str)
