"""Host-side logic of bench.py and the suite's fit designs (no GPU)."""
import importlib.util
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_calibrated_rates_units(bench):
    # per-unit costs made from known rates come back as those rates
    fitted = {"fma_f32_madd": {"p_madd": 64 / 72e12}, "fma_f32_add": {"p_add": 32 / 40e12},
              "fma_f64_madd": {"p_madd": 64 / 1.2e12}, "smem_sync0": {"p_lmem": 128 / 30e12},
              "stream_f64_s1": {"p_gmem": 16 / 7000e9}, "empty": {"p_launch": 2e-6, "p_group": 1e-9},
              "barrier": {"p_bar": 5e-9}}
    r = bench.calibrated_rates(fitted, 152, 2070.0)
    assert r["fp32_peak_tflops"] == pytest.approx(152 * 256 * 2.07e9 / 1e12, rel=1e-3)
    assert r["smem_peak_tbs"] == pytest.approx(152 * 128 * 2.07e9 / 1e12, rel=1e-3)
    assert r["f32_madd_tflops"] == pytest.approx(72.0)
    assert r["f32_add_tflops"] == pytest.approx(40.0)
    assert r["f64_madd_tflops"] == pytest.approx(1.2)
    assert r["lmem_tbs"] == pytest.approx(30.0)
    assert r["gmem_f64_s1_gbs"] == pytest.approx(7000.0)
    assert r["f32_madd_frac"] == pytest.approx(72.0 / r["fp32_peak_tflops"], rel=1e-3)
    assert r["launch_us"] == pytest.approx(2.0) and r["group_ns"] == pytest.approx(1.0)
    assert r["barrier_ns_per_group"] == pytest.approx(5.0)
    # missing families and non-positive costs give null, not a division error
    assert r["f32_mul_tflops"] is None and r["gmem_f32_s1_gbs"] is None
    assert bench.calibrated_rates({"fma_f32_madd": {"p_madd": -1.0}}, 152, None)["f32_madd_tflops"] is None


def test_clock_sampler_parses_reasons(bench):
    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    cs = bench.ClockSampler(0)
    cs.proc = _Proc()
    cs.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
                "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
                "0, 2010, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                "garbage line"]
    out = bench.ClockSampler.stop(cs)
    assert out["sm_mhz"] == 2010 and out["sm_max_mhz"] == 2070 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]


def test_kernel_instance_names(bench):
    assert bench.kernel_instance("stream", dict(dtype=1, vec=1, L=4, shape=0)) == "k_stream<double2,4,0>"
    assert bench.kernel_instance("stream", dict(dtype=0, vec=0, L=2, shape=1)) == "k_stream<float,2,1>"
    assert bench.kernel_instance("fma", dict(dtype=1, op=2)) == "k_fma<double,2>"
    assert bench.kernel_instance("smem", dict(sync=1)) == "k_smem<1>"
    assert bench.kernel_instance("barrier", dict(B=4)) == "k_barrier"


def test_source_sha_tracks_one_definition(bench):
    a = bench.source_sha("pm_suite.cu", "k_stream")
    assert a is not None and len(a) == 16 and a == bench.source_sha("pm_suite.cu", "k_stream")
    assert a != bench.source_sha("pm_suite.cu", "k_fma")
    assert bench.source_sha("pm_suite.cu", "k_no_such_kernel") is None


def test_workload_config_counts_bytes(bench):
    from paper_1904_09538_gb300 import suite as S
    variants = S.generate(["suite"])
    cfg = bench.workload_config(variants, 3)
    assert cfg["variants"] == len(variants) == 230
    assert cfg["bytes_per_step"] == 3 * sum(S.algorithmic_bytes(k, p) for k, p in variants)
    assert cfg["families"] == 22 and cfg["bytes_per_step"] > 100 * 129e6   # far above L2


def test_every_suite_family_design_is_full_rank():
    # each family model is identifiable from its fitting rows (every third
    # variant is held out): no feature column is a combination of the others
    import paper_1904_09538_gb300 as pm
    from paper_1904_09538_gb300 import suite as S
    variants = S.generate(["suite"])
    fams = {}
    for idx, (k, p) in enumerate(variants):
        fams.setdefault(S.family_key(k, p), []).append(idx)
    for f, idxs in fams.items():
        m = pm.Model("f_wall_time", S.family_model(f))
        fit = [i for j, i in enumerate(idxs) if j % 3 != 2]
        X = np.stack([m.feature_values(variants[i][0], **variants[i][1]) for i in fit])
        Xs = X / np.abs(X).max(axis=0)
        assert np.linalg.matrix_rank(Xs) == X.shape[1], f
        assert np.linalg.cond(Xs) < 1e3, f


def test_tensor_core_tiles_separate_load_and_mma_costs():
    # at one tile shape the bf16 loads are a fixed multiple of the tensor
    # multiply-adds (3/256 for 128 x 256 tiles, 2/256 for 256 x 256), so only
    # a calibration over both shapes identifies both costs
    import paper_1904_09538_gb300 as pm
    from paper_1904_09538_gb300.experiments import sweep_studies
    st = [s for s in sweep_studies() if s["name"] == "sweep_tc_tiles"][0]
    m = pm.Model("f_wall_time", st["expr"])
    cols = [m.features.index("f_mem_access_global_bfloat16"), m.features.index("f_op_bfloat16_madd")]
    rows = {k: np.stack([m.feature_values(k, **p)[cols] for kk, p in st["measure"] if kk == k])
            for k in ("mm_tc", "mm_tc256")}
    for k, ratio in (("mm_tc", 3 / 256), ("mm_tc256", 2 / 256)):
        assert np.allclose(rows[k][:, 0] / rows[k][:, 1], ratio)
        assert np.linalg.matrix_rank(rows[k] / rows[k].max(axis=0)) == 1
    both = np.concatenate([rows["mm_tc"], rows["mm_tc256"]])
    assert np.linalg.matrix_rank(both / both.max(axis=0)) == 2
    assert {k for k, _ in st["modeled"]} == {"mm_tc", "mm_tc256"}


def _sig(x, digits=2):
    return float("%.*g" % (digits, x))


def test_rates_reproduce_paper_table_mm_param_vals():
    # Table mm_param_vals: each printed rate follows from the printed
    # parameter, its counting granularity and the work per work-item
    import json
    from paper_1904_09538_gb300.report import rate
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_tables.json")))["mm_param_vals"]
    assert len(g["rows"]) == 9
    for row in g["rows"]:
        work = row.get("flops_per_op", row.get("bytes"))
        r = rate(row["param"], row["mcg"], work)
        assert _sig(r) == _sig(row["rate"]), (row, r)
    assert rate(0.0, "SG", 1) is None
    with pytest.raises(ValueError):
        rate(1e-12, "WG", 1)


def test_overlap_family_model_limits():
    # the partial-overlap model reduces to Eq. overlap_max as p_edge grows
    # (p_part = 0: max of the two costs), to the linear sum of both costs
    # with p_part = 1, and equals the tanh model of the section at p_part = 0
    from oracle.model import Model as OModel, overlap_expr
    from paper_1904_09538_gb300 import suite as S
    assert S.family_model("overlap") == S.overlap_model(partial=True)
    part = OModel("f_wall_time", S.overlap_model(partial=True))
    tanh = OModel("f_wall_time", S.overlap_model(partial=False))
    ref = OModel("f_wall_time", overlap_expr("p_launch * f_sync_kernel_launch",
                                             "p_gmem * f_mem_access_global_float32",
                                             "p_lmem * f_mem_access_local_float32"))
    assert set(part.params) == set(tanh.params) | {"p_part"}
    for m_ratio in (0.25, 0.9, 1.1, 4.0):
        f = {"f_sync_kernel_launch": 1.0, "f_mem_access_global_float32": 2e6,
             "f_mem_access_local_float32": 2e6 * m_ratio}
        p = {"p_launch": 5e-6, "p_gmem": 3e-12, "p_lmem": 3e-12, "p_edge": 1e9}
        cg, co = 6e-6, 6e-6 * m_ratio
        assert tanh.eval(p, f) == pytest.approx(ref.eval(p, f), rel=1e-15)
        assert part.eval(dict(p, p_part=0.0), f) == pytest.approx(tanh.eval(p, f), rel=1e-15)
        assert part.eval(dict(p, p_part=0.0), f) == pytest.approx(5e-6 + max(cg, co), rel=1e-9)
        assert part.eval(dict(p, p_part=1.0), f) == pytest.approx(5e-6 + cg + co, rel=1e-9)
        assert part.eval(dict(p, p_part=0.5), f) == pytest.approx(5e-6 + max(cg, co) + min(cg, co) / 2, rel=1e-9)


def test_suite_roofline_fractions(bench):
    # times built from known rates come back as those fractions of the peaks
    from paper_1904_09538_gb300 import suite as S
    variants = S.generate(["suite"])
    hbm, sms, mhz = 7000.0, 152, 2000.0
    lanes = sms * 128 * mhz * 1e6
    times = []
    for k, p in variants:
        nbytes, flops, lbytes = bench.variant_work(k, p)
        if k == "stream":
            times.append(nbytes / (0.9 * hbm * 1e9))
        elif k == "fma" and p["dtype"] == 0:
            times.append(flops / (0.75 * lanes * (2 if p["op"] == 2 else 1)))
        elif k == "fma":
            times.append(flops / 1.1e12)
        elif k == "smem":
            times.append(lbytes / (0.5 * lanes))
        else:
            times.append(1e-3)
    r = bench.suite_roofline(variants, times, hbm, sms, mhz)
    big = [p for k, p in variants if k == "stream" and S.algorithmic_bytes(k, p) >= 4 * S.L2_BYTES]
    assert r["stream_ge_4x_l2"]["variants"] == len(big) > 0
    assert r["stream_ge_4x_l2"]["at_least_0.8"] == len(big)
    for v in r["stream_ge_4x_l2"]["by_stride"].values():
        assert v["min"] == v["max"] == 0.9
    assert set(r["fma_f32_vs_pipe"]) == {"add", "mul", "madd"}
    assert all(v["median"] == 0.75 for v in r["fma_f32_vs_pipe"].values())
    assert r["fma_f64_madd_tflops"]["median"] == 1.1
    assert set(r["smem_vs_bandwidth"]) == {"sync0", "sync1"}
    assert all(v["median"] == 0.5 for v in r["smem_vs_bandwidth"].values())
    # a madd variant's flops are 2 per madd from its exact counts
    k, p = [(k, p) for k, p in variants if k == "fma" and p["op"] == 2 and p["dtype"] == 0][0]
    assert bench.variant_work(k, p)[1] >= 2 * p["F"] * p["G"] * 256


def test_cpu_model_is_named(bench):
    name = bench.cpu_model()
    assert isinstance(name, str) and name


def test_overlap_model_choice_rules():
    # the overlap test: separately calibrated costs about equal to the
    # measured time -> linear; well above it -> nonlinear
    from paper_1904_09538_gb300.experiments import choose_by_residual, choose_overlap_model
    assert choose_overlap_model(0.92) == "linear"
    assert choose_overlap_model(1.05) == "linear"
    assert choose_overlap_model(1.10) == "linear"
    assert choose_overlap_model(1.18) == "nonlinear"
    assert choose_overlap_model(1.18, margin=0.2) == "linear"
    assert choose_by_residual({"linear": 0.9, "nonlinear": 0.87, "partial": 0.5}) == "nonlinear"
    assert choose_by_residual({"linear": 0.8, "nonlinear": 0.87}) == "linear"
    assert choose_by_residual({"linear": None, "nonlinear": 0.87}) == "nonlinear"
    assert choose_by_residual({}) is None


def test_experiments_cli_rejects_unknown_part():
    import subprocess
    r = subprocess.run([sys.executable, "-m", "paper_1904_09538_gb300.experiments", "--only=bogus"],
                       cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode != 0 and "unknown part 'bogus'" in r.stderr
