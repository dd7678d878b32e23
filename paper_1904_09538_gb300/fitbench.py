"""Time the batched calibration: python -m paper_1904_09538_gb300.fitbench
[--models K] [--reps R] [--threads T]

K models (alternately linear and tanh-overlap, 4..12 parameters, 40..400 rows each, seeded
synthetic features and model-plus-noise outputs) fitted in one batched plan
(one persistent launch in a CUDA graph), R timed replays.  Prints one JSON
line: fits per second, milliseconds per replay, status counts."""
import json
import sys
import time

import numpy as np


LAUNCH = "p_launch * f_sync_kernel_launch + p_group * f_thread_groups"
# (parameter, feature) terms the models draw from: global-memory terms and
# on-chip terms (arithmetic, local memory)
GMEM = [("p_gmem", "f_mem_access_global_float32"), ("p_g64", "f_mem_access_global_float64"),
        ("p_gld", "f_mem_access_global_float32_load"), ("p_gst", "f_mem_access_global_float32_store"),
        ("p_g16", "f_mem_access_global_bfloat16")]
ONCHIP = [("p_madd", "f_op_float32_madd"), ("p_lmem", "f_mem_access_local_float32"), ("p_add", "f_op_float32_add"),
          ("p_mul", "f_op_float32_mul"), ("p_d64", "f_op_float64_madd")]
TRUTH = {"p_launch": 5e-6, "p_group": 2e-9, "p_add": 4e-12, "p_madd": 3e-12, "p_gmem": 6e-12, "p_lmem": 2e-12,
         "p_mul": 5e-12, "p_g64": 9e-12, "p_gld": 5e-12, "p_gst": 7e-12, "p_g16": 4e-12, "p_d64": 2e-11,
         "p_edge": 3e4}


def _sum(terms):
    return " + ".join("%s * %s" % t for t in terms)


def model_expr(k):
    """Expression of problem k: even k a linear model with 4..12 parameters
    (launch and work-group terms plus 2..10 cost terms), odd k a tanh-overlap
    model (Section "Modeling Operation Overlap") with 5..12 parameters
    (launch, work-group, p_edge, and 2..9 terms split between the global and
    the on-chip cost), the parameter count cycling with k."""
    if k % 2 == 0:
        m = 4 + (k // 2) % 9
        return LAUNCH + " + " + _sum((GMEM + ONCHIP)[:m - 2])
    m = 5 + (k // 2) % 8
    n = m - 3
    cg = "(%s)" % _sum(GMEM[:(n + 1) // 2])
    co = "(%s)" % _sum(ONCHIP[:n // 2])
    return (LAUNCH + " + %s * (tanh(p_edge * (%s - %s)) + 1) / 2 + %s * (tanh(p_edge * (%s - %s)) + 1) / 2"
            % (cg, cg, co, co, co, cg))


def features(K, nfeat):
    """Seeded feature matrices of K problems (launch = 1, work-groups in
    [1e2, 1e4], other counts in [1e5, 1e7]) and their row counts."""
    import pm_inputs
    ls = pm_inputs.row_counts(K, 4242)
    Xs = []
    for k in range(K):
        l = int(ls[k])
        X = pm_inputs.integers((l, nfeat(k)), 9000 + k, 10 ** 5, 10 ** 7).astype(np.float64)
        X[:, 0] = 1.0
        X[:, 1] = pm_inputs.integers((l,), 9500 + k, 100, 10 ** 4)
        Xs.append(X)
    return Xs, ls


def synthetic_times(k, features, X):
    """Outputs the workload is made from: model k (model_expr) at the TRUTH
    parameters on the rows of X (columns named by `features`), evaluated
    here in plain NumPy from the model's term lists -- synthetic input data,
    made without the library -- times (1 + 1 % noise)."""
    import pm_inputs
    col = {f: X[:, i] for i, f in enumerate(features)}

    def cost(terms):
        return sum(TRUTH[p] * col[f] for p, f in terms)

    launch = TRUTH["p_launch"] * col["f_sync_kernel_launch"] + TRUTH["p_group"] * col["f_thread_groups"]
    if k % 2 == 0:
        m = 4 + (k // 2) % 9
        g = launch + cost((GMEM + ONCHIP)[:m - 2])
    else:
        n = 5 + (k // 2) % 8 - 3
        cg, co = cost(GMEM[:(n + 1) // 2]), cost(ONCHIP[:n // 2])
        pe = TRUTH["p_edge"]
        g = launch + cg * (np.tanh(pe * (cg - co)) + 1) / 2 + co * (np.tanh(pe * (co - cg)) + 1) / 2
    return g * (1 + 1e-2 * pm_inputs.noise((len(X),), 9900 + k))


def problem(K):
    """K seeded calibration problems: (models, feature matrices, outputs,
    start points = 1.2 x the parameters the outputs were made with)."""
    from . import Model
    models = [Model("f_wall_time", model_expr(k)) for k in range(K)]
    Xs, ls = features(K, lambda k: len(models[k].features))
    ts, p0s = [], []
    for k, (m, X) in enumerate(zip(models, Xs)):
        ts.append(synthetic_times(k, m.features, X))
        p0s.append(np.array([TRUTH[n] for n in m.params]) * 1.2)
    return models, Xs, ts, p0s, ls


def main(argv):
    import torch
    from . import FitPlan
    K, reps, threads = 64, 10, 128
    it = iter(argv)
    for a in it:
        if a == "--models":
            K = int(next(it))
        elif a == "--reps":
            reps = int(next(it))
        elif a == "--threads":
            threads = int(next(it))
    models, Xs, ts, p0s, ls = problem(K)
    plan = FitPlan(models, [len(t) for t in ts], p0_given=True, threads=threads)
    Xc = np.concatenate([x.ravel() for x in Xs])
    tc = np.concatenate(ts)
    pc = np.concatenate(p0s)
    plan.run(Xc, tc, pc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        _, out = plan.run(Xc, tc, pc)
    dt = (time.perf_counter() - t0) / reps
    st = [r["status"] for r in out]
    print(json.dumps({"models": K, "rows": [int(ls.min()), int(ls.max())], "threads": threads,
                      "ms_per_batch": dt * 1e3, "fits_per_s": K / dt,
                      "iterations_max": max(r["iterations"] for r in out),
                      "statuses": {str(s): st.count(s) for s in sorted(set(st))}}))


if __name__ == "__main__":
    main(sys.argv[1:])
