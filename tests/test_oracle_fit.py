"""Pins of the oracle's model expressions and FP64 calibration: hand-evaluated
expressions, finite differences, exact recovery of known parameters, the
normal-equation and minimum-norm properties, and the paper's printed
geometric means.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import pm_inputs
from oracle import fit as ofit
from oracle.features import features
from oracle.model import Model, step_hat, overlap_expr, linear_expr, tokenize

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def test_expression_eval_by_hand():
    m = Model("f_wall_time", "p_a * f_x + p_b * (f_y - 2) / f_z - -p_c")
    assert m.params == ["p_a", "p_b", "p_c"] and m.features == ["f_x", "f_y", "f_z"]
    v = m.eval({"p_a": 2.0, "p_b": 3.0, "p_c": 5.0}, {"f_x": 7.0, "f_y": 6.0, "f_z": 4.0})
    assert v == 2 * 7 + 3 * (6 - 2) / 4 + 5
    m2 = Model("t", "tanh(p_e * (f_a - f_b))")
    assert m2.eval({"p_e": 0.5}, {"f_a": 3.0, "f_b": 1.0}) == math.tanh(1.0)
    # a '-' glued to a name is part of the name (tags contain '-')
    assert ("name", "f_mem_access_tag:mm-PF-a") in tokenize("p_x*f_mem_access_tag:mm-PF-a")
    with pytest.raises(ValueError):
        Model("t", "p_a * (f_x + 1")


def test_step_function():
    # Section "Modeling Operation Overlap": s_hat(x) = (tanh(p_edge x) + 1) / 2
    assert step_hat(0.0, 10.0) == 0.5
    for x in (-1.0, -0.1, 0.03, 0.5, 2.0):
        assert abs(step_hat(x, 10.0) + step_hat(-x, 10.0) - 1.0) < 1e-15
    assert step_hat(1.0, 1e4) == 1.0 and step_hat(-1.0, 1e4) == 0.0
    assert step_hat(0.3, 10.0) > step_hat(0.1, 10.0)


def test_symbolic_gradient_vs_central_differences():
    expr = overlap_expr("p_k * f_k + p_g * f_g", "p_m * f_m + p_d * f_d", "p_a * f_a / f_k + sqrt(p_s * f_a)")
    m = Model("t", expr)
    f = {"f_k": 1.0, "f_g": 300.0, "f_m": 2e6, "f_d": 1e5, "f_a": 4e6}
    p = {"p_k": 1e-5, "p_g": 2e-9, "p_m": 3e-12, "p_d": 5e-12, "p_a": 7e-12, "p_s": 1e-18, "p_edge": 2e4}
    g, d = m.grad(p, f)
    assert g == m.eval(p, f)
    for i, name in enumerate(m.params):
        h = 1e-4 * abs(p[name])
        pp, pm = dict(p), dict(p)
        pp[name] += h
        pm[name] -= h
        fd = (m.eval(pp, f) - m.eval(pm, f)) / (2 * h)
        assert abs(fd - d[i]) <= 1e-6 * (abs(d[i]) + 1e-12 * abs(g) / abs(p[name])), name


def test_nonlinear_limit_is_max():
    # p_edge -> infinity: overlap model -> c_overhead + max(c_gmem, c_onchip)
    m = Model("t", overlap_expr("p_o", "p_g * f_g", "p_c * f_c"))
    for fg, fc in ((3.0, 1.0), (1.0, 3.0)):
        v = m.eval({"p_o": 0.5, "p_g": 1.0, "p_c": 1.0, "p_edge": 1e6}, {"f_g": fg, "f_c": fc})
        assert v == 0.5 + max(fg, fc)


def _synthetic_rows(l, nf, seed):
    X = pm_inputs.integers((l, nf), seed, 1, 10 ** 7).astype(np.float64)
    return X


def test_linear_exact_recovery_and_normal_equations():
    l, m = 60, 6
    X = _synthetic_rows(l, m, 11)
    p_true = pm_inputs.log_uniform((m,), 12, 1e-12, 1e-8)
    t = X @ p_true
    p, info = ofit.fit_linear(X, t)
    assert not info["rank_deficient"] and info["rank"] == m
    assert np.max(np.abs(p - p_true) / p_true) < 1e-10
    # with noise: the relative residual is orthogonal to the scaled columns
    t2 = t * (1 + 1e-2 * pm_inputs.noise((l,), 13))
    p2, _ = ofit.fit_linear(X, t2)
    A = X / t2[:, None]
    r = 1 - A @ p2
    assert np.max(np.abs(A.T @ r) / (np.linalg.norm(A, axis=0) * np.linalg.norm(r))) < 1e-10


def test_linear_rank_deficient_min_norm():
    # columns in span{n^3, n^2} (rank 2), like the matmul design on flops,
    # global, local and work-group counts
    n = np.array([256, 384, 512, 640, 768], dtype=np.float64)
    X = np.stack([2 * n ** 3, n ** 3 / 8 + n ** 2, 2 * n ** 3 + 2 * n ** 3 / 16, n ** 2 / 256], axis=1)
    t = 1e-12 * n ** 3 + 3e-10 * n ** 2
    p, info = ofit.fit_linear(X, t)
    assert info["rank"] == 2 and info["rank_deficient"]
    A = X / t[:, None]
    As = A / info["colscale"]
    q = p * info["colscale"]
    # min-norm: q is orthogonal to the null space of As
    _, s, Vt = np.linalg.svd(As)
    null = Vt[2:]
    assert np.max(np.abs(null @ q)) < 1e-8 * np.linalg.norm(q)
    # the fit is exact (t is in the column span), so predictions at a new n are unique
    assert np.max(np.abs(A @ p - 1)) < 1e-9
    n2 = 896.0
    x2 = np.array([2 * n2 ** 3, n2 ** 3 / 8 + n2 ** 2, 2 * n2 ** 3 + 2 * n2 ** 3 / 16, n2 ** 2 / 256])
    assert abs(x2 @ p / (1e-12 * n2 ** 3 + 3e-10 * n2 ** 2) - 1) < 1e-8


def test_lm_recovers_overlap_model():
    l = 80
    expr = overlap_expr("p_launch * f_sync_kernel_launch + p_group * f_thread_groups",
                        "p_gmem * f_mem_access_global_float32", "p_lmem * f_mem_access_local_float32")
    m = Model("f_wall_time", expr)
    X = _synthetic_rows(l, 3, 21)
    F = [{"f_sync_kernel_launch": 1.0, "f_thread_groups": X[k, 0] / 100,
          "f_mem_access_global_float32": X[k, 1], "f_mem_access_local_float32": X[k, 2]} for k in range(l)]
    p_true = {"p_launch": 5e-6, "p_group": 2e-9, "p_gmem": 3e-12, "p_lmem": 2e-12, "p_edge": 1e5}
    t = np.array([m.eval(p_true, f) for f in F])
    pv = np.array([p_true[n] for n in m.params])
    p, info = ofit.fit(m, F, t, p0=pv * (1 + 0.2 * np.array([1, -1, 1, -1, 1])))
    assert info["method"] == "lm"
    assert np.max(np.abs(p - pv) / pv) < 1e-8, (p, pv)
    # the start point heuristic alone also converges here
    p_auto, _ = ofit.fit(m, F, t)
    pred = ofit.predict(m, p_auto, F)
    assert np.max(np.abs(pred - t) / t) < 1e-6


def test_lm_on_linear_model_matches_linear_solution():
    l = 50
    X = _synthetic_rows(l, 3, 31)
    m = Model("t", "p_a * f_a + p_b * f_b + p_c * f_c")
    F = [{"f_a": X[k, 0], "f_b": X[k, 1], "f_c": X[k, 2]} for k in range(l)]
    t = X @ np.array([1e-9, 2e-10, 3e-11]) * (1 + 1e-2 * pm_inputs.noise((l,), 32))
    p_lin, _ = ofit.fit_linear(X, t)
    r, J = ofit.residual_and_jacobian(m, F, t)
    import scipy.optimize
    p_lm = scipy.optimize.leastsq(r, p_lin * 1.3, Dfun=J, ftol=1e-15, xtol=1e-15)[0]
    assert np.max(np.abs(p_lm - p_lin) / np.abs(p_lin)) < 1e-9


def test_illustrative_model_madd_only():
    # Section "Model Creation, Calibration, and Evaluation": t = p_madd * f_madd
    m = Model("f_wall_time", "p_f32madd * f_op_float32_madd")
    ns = [256, 384, 512, 640, 768]
    F = [{"f_op_float32_madd": float(n ** 3 // 32)} for n in ns]
    t = np.array([5.0e-12 * f["f_op_float32_madd"] for f in F])
    p, info = ofit.fit(m, F, t)
    assert info["method"] == "linear" and abs(p[0] / 5.0e-12 - 1) < 1e-14


def test_paper_geomean_rows():
    # the 'Mean' rows of the accuracy tables are geometric means over variants
    for study in ("matmul", "dg", "fd"):
        tab = GOLD["accuracy_tables"][study]
        for g in range(len(tab["gpus"])):
            vals = [v[g] for v in tab["variants"].values()]
            # each printed entry v stands for a value in [v - 0.05, v + 0.05]
            lo = ofit.geomean([v - 0.05 for v in vals])
            hi = ofit.geomean([v + 0.05 for v in vals])
            printed = tab["mean"][g]
            assert lo <= printed + 0.05 and printed - 0.05 <= hi, (study, g, lo, hi)


def test_geomean_rel_err_definition():
    meas = np.array([1.0, 2.0, 4.0])
    pred = np.array([1.1, 1.8, 4.4])      # 10 % error each
    assert abs(ofit.geomean_rel_err(pred, meas) - 0.1) < 1e-12


def test_model_features_from_counts():
    # feature assembly: the matmul illustrative model's feature from counts
    fs = features("mm_pf", n=32)
    m = Model("t", linear_expr("p_l * f_sync_kernel_launch + p_g * f_thread_groups",
                               "p_c * f_mem_access_tag:c", "p_m * f_op_float32_madd"))
    from oracle.features import feature_value
    vals = {name: feature_value(name, fs) for name in m.features}
    assert vals == {"f_sync_kernel_launch": 1, "f_thread_groups": 4, "f_mem_access_tag:c": 1024,
                    "f_op_float32_madd": 1024}


def test_fit_rows_is_fit_on_plain_data():
    # the process-pool entry point: the same fit from (expression, names,
    # matrix) as from the model and row dicts; exact recovery without noise
    expr = "p_a * f_x + p_b * f_y + p_c"
    m = Model("f_wall_time", expr)
    X = pm_inputs.integers((30, 2), 77, 1, 1000).astype(np.float64)
    truth = {"p_a": 3e-9, "p_b": 5e-10, "p_c": 2e-6}
    F = [dict(zip(m.features, r)) for r in X]
    t = np.array([m.eval(truth, f) for f in F])
    p1, _ = ofit.fit(m, F, t)
    p2, _ = ofit.fit_rows((expr, list(m.features), X, t, None))
    assert np.array_equal(p1, p2)
    assert np.allclose(p2, [truth[n] for n in m.params], rtol=1e-10, atol=0)


def test_start_point_rules():
    # linear fit of the model with every tanh switch at 1/2: exact here for
    # p_a; p_b comes out negative and becomes 1e-3 sum(t) / sum |f_y|; p_c
    # only multiplies p_a (its column is zero at the origin): the same rule on
    # its column at the point reached so far, p_a * f_z; p_edge starts at
    # 10 / median(t)
    m = Model("t", "p_a * f_x + p_b * f_y + p_c * p_a * f_z + tanh(p_edge * f_x) * 0")
    F = [{"f_x": float(x), "f_y": float(y), "f_z": 1.0} for x, y in ((1, 5), (2, 1), (3, 7), (4, 2))]
    t = np.array([1e-6 * f["f_x"] - 1e-9 * f["f_y"] for f in F])
    p0 = dict(zip(m.params, ofit.start_point(m, F, t)))
    assert p0["p_a"] == pytest.approx(1e-6, rel=1e-9)
    assert p0["p_b"] == pytest.approx(1e-3 * t.sum() / 15.0, rel=1e-12)
    assert p0["p_c"] == pytest.approx(1e-3 * t.sum() / (4 * p0["p_a"]), rel=1e-9)
    assert p0["p_edge"] == pytest.approx(10.0 / np.median(t), rel=1e-12)
