"""The paper's diagnostic experiments on the GPU, at reduced size
(experiments.diagnostics(reduced=True)): the a- versus b-pattern cost of the
prefetching matmul's fetches (Section "Data Motion Features", Table
ab_pattern), the madd-only calibration (Section "Illustrative Example"), the
overlap test choosing the linear or the tanh-overlap model per variant and
the calibration residual beside it (Section "Models Demonstrated"), and local
memory split by lid(1) stride (Section "Finite Differences").  Every
calibration in the report is refit by the oracle (FP64, SciPy) on the same
rows -- the measured times and the same kernels' counts -- and must reach
the same point: linear fits the same parameters within 1e-6, nonlinear fits
the same SSR within 1e-4."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1904_09538_gb300 as pm  # noqa: E402
from paper_1904_09538_gb300 import experiments as E  # noqa: E402
from oracle import fit as ofit  # noqa: E402
from oracle.model import Model as OModel  # noqa: E402


def refit(expr, params, rows):
    """(relative parameter difference or None, GPU SSR, oracle SSR, linear?)"""
    m = pm.Model("f_wall_time", expr)
    om = OModel("f_wall_time", expr)
    X = np.stack([m.feature_values(r["kernel"], **r["params"]) for r in rows])
    t = np.array([r["measured_s"] for r in rows])
    F = [dict(zip(om.features, x)) for x in X]
    pg = np.array([params[n] for n in om.params])
    po, info = ofit.fit(om, F, t)
    ssr_g = float(np.sum((1 - np.asarray(ofit.predict(om, pg, F)) / t) ** 2))
    ssr_o = float(np.sum((1 - np.asarray(ofit.predict(om, po, F)) / t) ** 2))
    lin = info.get("method") == "linear"
    d = None
    if lin and not info["rank_deficient"]:
        d = float(np.max(np.abs(pg - po) / np.abs(po)))
    return d, ssr_g, ssr_o, lin


def test_diagnostics_reduced_matches_oracle_refits():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rep = E.diagnostics(trials=3, reduced=True)
    ab = rep["ab_ratio"]
    assert len(ab["rows"]) >= 2 and all(r["b_over_a"] > 0 and math.isfinite(r["b_over_a"]) for r in ab["rows"])
    md = rep["madd_only"]
    assert md["fit"]["status"] == 0 and md["rate_flops"] > 0
    fits = dict(rep["calibrations"], madd_only={"expr": md["expr"], "params": md["params"], "fit": md["fit"],
                                                 "rows": md["rows"]})
    assert len(fits) >= 11, sorted(fits)
    for name, f in fits.items():
        d, ssr_g, ssr_o, lin = refit(f["expr"], f["params"], f["rows"])
        if d is not None:
            assert d <= 1e-6, (name, d)
        assert abs(ssr_g / ssr_o - 1) <= (1e-6 if lin else 1e-4), (name, ssr_g, ssr_o)
    # the overlap test and the model choice are reported for every variant
    for study, per in rep["overlap"].items():
        for v, row in per.items():
            if isinstance(row, dict) and "separate_costs_over_measured" in row:
                assert row["chosen_by_cost_sum"] in ("linear", "nonlinear")
                assert row["separate_costs_over_measured"] > 0
    assert rep["split_lmem"]["s_per_subgroup_local_access"]["T16"] > 0
