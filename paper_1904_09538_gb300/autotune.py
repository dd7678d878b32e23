"""Model-guided autotuning (Section "Assumptions and Limitations": a
calibrated model as a pruning heuristic for choosing among mathematically
equivalent kernel variants; important accuracy gains come from a few extra
on-line calibration runs).

rank_family(): for a family of variants (the 24 register-tiled SIMT matmul
tile shapes), calibrate a cost model on cheap runs of every variant at a
small size, predict every variant at the target size from its exact counts,
then time the variants at the target size and report how well the predicted
order matches the measured one (Spearman, Kendall, best-variant hit, and the
measured time of the predicted best relative to the true best).

tune_fit_threads(): pick the CTA size of the batched calibration kernel by
timing the plan for each candidate.
"""
import itertools
import math
import time

import numpy as np

from . import Model, FitPlan, run
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


def _time(kernel, variants, bufs, trials, flush_l2=True):
    out = []
    for p in variants:
        tm = run(kernel, bufs.get(kernel, p), warmup=2, trials=trials, flush_l2=flush_l2, **p)
        out.append(tm["mean_ms"] * 1e-3)
    return np.array(out)


def rank_family(kernel="mm_simt", shapes=None, calib_sizes=(1536, 2304), target=7680, trials=5, seed=7,
                expr=SIMT_MODEL):
    import torch
    shapes = shapes or SIMT_SHAPES
    dev = torch.device("cuda", torch.cuda.current_device())
    bufs = Buffers(torch, dev, seed)
    m = Model("f_wall_time", expr)
    calib = [dict(s, n=n) for n in calib_sizes for s in shapes]
    Xc = np.stack([m.feature_values(kernel, **p) for p in calib])
    t0 = time.perf_counter()
    tc = _time(kernel, calib, bufs, trials)
    calib_s = time.perf_counter() - t0
    plan = FitPlan([m], [len(tc)])
    p, reps = plan.run(Xc.ravel(), tc)
    targets = [dict(s, n=target) for s in shapes]
    Xt = np.stack([m.feature_values(kernel, **q) for q in targets])
    pred = m.predict(p, Xt)
    t0 = time.perf_counter()
    meas = _time(kernel, targets, bufs, trials)
    meas_s = time.perf_counter() - t0
    best_pred, best_meas = int(np.argmin(pred)), int(np.argmin(meas))
    top3 = set(np.argsort(pred)[:3].tolist())
    flops = 2.0 * target ** 3
    return {
        "kernel": kernel, "target_n": target, "calib_sizes": list(calib_sizes), "n_shapes": len(shapes),
        "params": dict(zip(m.params, [float(x) for x in p])), "fit": reps[0],
        "spearman": spearman(pred, meas), "kendall": kendall(pred, meas),
        "best_predicted": targets[best_pred], "best_measured": targets[best_meas],
        "best_hit": best_pred == best_meas, "best_in_predicted_top3": best_meas in top3,
        "slowdown_of_predicted_best": float(meas[best_pred] / meas[best_meas]),
        "best_measured_tflops": flops / meas[best_meas] / 1e12,
        "geomean_rel_err": float(math.exp(np.mean(np.log(np.abs(pred - meas) / meas)))),
        "calibration_seconds": calib_s, "exhaustive_seconds": meas_s,
        "rows": [{"shape": q, "measured_s": float(a), "predicted_s": float(b)} for q, a, b in zip(targets, meas, pred)],
    }


def tune_fit_threads(models, Xs, ts, p0s=None, candidates=(64, 128, 256), reps=10):
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
    out = {"mm_simt": rank_family()}
    json.dump(out, open(sys.argv[1], "w") if len(sys.argv) > 1 else sys.stdout, indent=1, default=str)
