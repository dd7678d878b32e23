"""Model expressions the studies build (Section "Models Demonstrated"): the
compact overlap form and the two-level on-chip overlap of the extension study
against Eq. tanh written out, evaluated by the oracle's expression evaluator;
the library's model program accepts every study's expression."""
import numpy as np
import pytest

import paper_1904_09538_gb300 as pm
from paper_1904_09538_gb300 import experiments as E
from oracle.model import Model as OModel


def _tanh_pair(a, b, edge):
    # Eq. tanh as the paper writes it: a s(a - b) + b s(b - a)
    return "(%s * (tanh(%s * (%s - %s)) + 1) / 2 + %s * (tanh(%s * (%s - %s)) + 1) / 2)" % (
        a, edge, a, b, b, edge, b, a)


def _random_point(model, rng):
    p = {}
    for name in model.params:
        # switches over the range the fits reach (1e3 .. 1e9 per second),
        # costs over picoseconds to microseconds per unit
        p[name] = 10.0 ** rng.uniform(3, 9) if name in ("p_edge", "p_e2") else 10.0 ** rng.uniform(-13, -6)
    f = {name: float(rng.integers(0, 1 << 30)) for name in model.features}
    return p, f


def test_soft_max_equals_eq_tanh():
    rng = np.random.default_rng(11)
    compact = OModel("f_wall_time", E.soft_max("(p_a * f_x)", "(p_b * f_y)", "p_edge"))
    written = OModel("f_wall_time", _tanh_pair("(p_a * f_x)", "(p_b * f_y)", "p_edge"))
    for _ in range(200):
        p, f = _random_point(written, rng)
        g0, g1 = compact.eval(p, f), written.eval(p, f)
        assert g0 == pytest.approx(g1, rel=1e-12, abs=0.0)
        # the larger of the two when the switch is sharp, their mean when it is flat
        a, b = p["p_a"] * f["f_x"], p["p_b"] * f["f_y"]
        if p["p_edge"] * abs(a - b) > 40:
            assert g0 == pytest.approx(max(a, b), rel=1e-12)
    p = {"p_a": 2e-9, "p_b": 1e-9, "p_edge": 0.0}
    assert compact.eval(p, {"f_x": 1.0, "f_y": 1.0}) == pytest.approx(1.5e-9, rel=1e-15)


def test_overlap2_is_eq_tanh_nested():
    gm = [s for s in E.studies() if s["name"] == "matmul"][0]["gmem"]
    cg = "(%s)" % " + ".join(gm)
    written = E.OVERHEAD + " + " + _tanh_pair(cg, _tanh_pair("(%s)" % E.ARITH, "(%s)" % E.LOCAL, "p_e2"), "p_edge")
    ow, oc = OModel("f_wall_time", written), OModel("f_wall_time", E.overlap2(gm))
    assert sorted(ow.params) == sorted(oc.params) and sorted(ow.features) == sorted(oc.features)
    rng = np.random.default_rng(12)
    for _ in range(200):
        p, f = _random_point(ow, rng)
        assert oc.eval(p, f) == pytest.approx(ow.eval(p, f), rel=1e-12, abs=0.0)


def test_every_study_model_fits_the_library_program():
    # the library compiles every study's and sweep study's expression (at most
    # 16 parameters and its program's operation limit) and sees the same
    # features and parameters as the oracle
    sts = E.studies() + E.sweep_studies() + E.sweep_studies(reduced=True)
    for st in sts:
        m, om = pm.Model("f_wall_time", st["expr"]), OModel("f_wall_time", st["expr"])
        assert sorted(m.params) == sorted(om.params), st["name"]
        assert sorted(m.features) == sorted(om.features), st["name"]
    names = {st["name"] for st in sts}
    assert {"matmul", "matmul_onchip_overlap", "sweep_dg_tile", "sweep_dg_tc"} <= names


def test_dg_tile_sweep_model_is_linear_in_its_parameters():
    # both fit paths solve a model linear in p directly (one optimum), which
    # the DG tile form's sweep model relies on
    from oracle import fit as ofit
    st = [s for s in E.sweep_studies(reduced=True) if s["name"] == "sweep_dg_tile"][0]
    om = OModel("f_wall_time", st["expr"])
    m = pm.Model("f_wall_time", st["expr"])
    rows = [(k, p) for k, p in st["measure"]][:12]
    F = [dict(zip(m.features, m.feature_values(k, **p))) for k, p in rows]
    assert ofit.is_linear(om, F)
    assert "f_mem_access_tag:dgt-u" in om.features and "f_op_float32_madd" in om.features
