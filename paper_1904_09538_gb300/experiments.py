"""The paper's evaluation on this GPU (Section "Results").

For each computation -- matmul (2 variants), DG differentiation (noPF, uPF,
dmPF, dmPF-T with 16x16 work-groups; noPF, dmPF, dmPF-T with 32x8), five-point
stencil (16x16 and 18x18 tiles, direct loads) -- a model of the form
of Eq. linear_model or Eq. nonlinear_model is calibrated on a measurement
kernel set that does NOT contain the modeled kernels (microbenchmarks: the
arithmetic, local-memory, barrier, overlap, empty and global-memory pattern
kernels, plus the work-removed twins of the modeled kernels, Algorithm 3),
then predicts the modeled kernels' times at every size.  Reported: the
geometric mean and maximum relative error per variant, and how well the
predictions rank the variants (Spearman and Kendall over all sizes).

Also the illustrative case of Section "Illustrative Example" (configuration
1): a 4-parameter linear model of the prefetching matmul on n = 256..768,
predicting n = 896.

Timing: pm_run, `trials` device-timed launches after 2 warm-ups (mean, trials
above 5x the median dropped).  Inputs are seeded uniform / normal values.
"""
import math
import re

import numpy as np

from . import Model, FitPlan, kernel_buffers, run
from .suite import LAUNCH, generate

GENERIC = "p_gen * f_mem_access_global_float32_lstrides:{0:1}_afr:1"
OVERHEAD = ("p_launch * f_sync_kernel_launch + p_group * f_thread_groups + "
            "p_bar * f_sync_barrier_local * f_thread_groups")
ONCHIP = ("p_madd * f_op_float32_madd + p_add * f_op_float32_add + p_mul * f_op_float32_mul + "
          "p_lmem * f_mem_access_local_float32")


def nonlinear(gmem_terms, overhead=OVERHEAD, onchip=ONCHIP):
    cg = "(%s)" % " + ".join(gmem_terms)
    co = "(%s)" % onchip
    return ("%s + %s * (tanh(p_edge * (%s - %s)) + 1) / 2 + %s * (tanh(p_edge * (%s - %s)) + 1) / 2"
            % (overhead, cg, cg, co, co, co, cg))


def partial(gmem_terms, overhead=OVERHEAD, onchip=ONCHIP):
    """Eq. nonlinear_model with one more parameter, p_part, for partial overlap
    (the variation of Eq. tanh the paper suggests): the smaller of the two
    cost groups is added with weight p_part (0: full overlap, 1: none)."""
    cg = "(%s)" % " + ".join(gmem_terms)
    co = "(%s)" % onchip
    hi = "%s * (tanh(p_edge * (%s - %s)) + 1) / 2 + %s * (tanh(p_edge * (%s - %s)) + 1) / 2" % (cg, cg, co, co, co, cg)
    lo = "%s * (tanh(p_edge * (%s - %s)) + 1) / 2 + %s * (tanh(p_edge * (%s - %s)) + 1) / 2" % (cg, co, cg, co, cg, co)
    return "%s + %s + p_part * (%s)" % (overhead, hi, lo)


ARITH = "p_madd * f_op_float32_madd + p_add * f_op_float32_add + p_mul * f_op_float32_mul"
LOCAL = "p_lmem * f_mem_access_local_float32"


def soft_max(a, b, edge):
    """Eq. tanh's a s(a - b) + b s(b - a), s(x) = (tanh(edge x) + 1) / 2, written
    as b + (a - b) s(a - b) (equal since s(x) + s(-x) = 1), which repeats a
    and b fewer times in the model's program."""
    return "(%s + (%s - %s) * (tanh(%s * (%s - %s)) + 1) / 2)" % (b, a, b, edge, a, b)


def overlap2(gmem_terms, overhead=OVERHEAD, arith=ARITH, local=LOCAL):
    """Eq. tanh between global-memory and on-chip work, the on-chip side
    itself the same overlap of arithmetic and local memory (second switch
    p_e2) instead of their sum: on GB300 the FMA pipe and the shared-memory
    pipe issue side by side, so a kernel whose inner loop pairs every
    multiply-add with local loads (the tiled matmuls) costs about the larger
    of the two, not their sum."""
    cg = "(%s)" % " + ".join(gmem_terms)
    return "%s + %s" % (overhead, soft_max(cg, soft_max("(%s)" % arith, "(%s)" % local, "p_e2"), "p_edge"))


def linear(gmem_terms, overhead=OVERHEAD, onchip=ONCHIP):
    return "%s + %s + %s" % (overhead, " + ".join(gmem_terms), onchip)


def tagged(tag, name):
    return "p_%s * f_mem_access_tag:%s" % (name, tag)


# microbenchmarks shared by every computation's measurement set (paper Fig. mkernels_common)
def common_measurements():
    out = []
    out += generate(["ops", "dtype:0"])                       # f32 add / mul / madd loops
    out += generate(["lmem"])                                 # local memory, with and without barriers
    out += generate(["sync"])                                 # barrier kernel
    out += generate(["overlap"])                              # local/global overlap
    out += generate(["launch"])                               # empty kernels
    out += generate(["stream2d"])                             # unit-stride f32 global pattern (AFR 1)
    return out


def studies(reduced=False):
    """(name, model expression, measurement kernels, modeled kernels) per computation.
    reduced: every third modeled size and every second twin size (a bounded
    form for tests and benchmark runs)."""
    mm_sizes = list(range(512, 4096 + 1, 128))                # 29 sizes
    mm_twin_sizes = [512, 1024, 1536, 2048, 2560, 3072, 3584, 4096]
    mm_gm = [GENERIC] + [tagged(t, n) for t, n in (("mm-PF-a", "pfa"), ("mm-PF-b", "pfb"),
                                                   ("mm-noPF-a", "npa"), ("mm-noPF-b", "npb"))]
    mm = dict(
        name="matmul", gmem=mm_gm,
        expr=nonlinear(mm_gm),
        measure=common_measurements() + [(k, {"n": n}) for k in ("mm_pf_a", "mm_pf_b", "mm_nopf_a", "mm_nopf_b")
                                         for n in mm_twin_sizes],
        modeled=[(k, {"n": n}) for k in ("mm_pf", "mm_nopf") for n in mm_sizes],
    )
    # the same measurements and predictions with the on-chip side itself an
    # overlap (overlap2): an extension of the paper's model, reported beside it
    out = [mm, dict(mm, name="matmul_onchip_overlap", expr=overlap2(mm_gm), extension=True)]
    for L0, L1 in ((16, 16), (32, 8)):
        sh = "%dx%d" % (L0, L1)
        # uPF's D loads share noPF's pattern and twin; dmPF-T's D fetch shares
        # dmPF's; dmPF-T's unit-stride AFR-1 result store is covered by the
        # generic feature (a tag on it would count it twice)
        tags = [("dg-noPF-u-" + sh, "nu"), ("dg-noPF-dm-" + sh, "ndm"), ("dg-dmPF-u-" + sh, "pu"),
                ("dg-dmPF-dm-" + sh, "pdm"), ("dg-res-" + sh, "res"), ("dg-dmPFT-u-" + sh, "tu")]
        twin_k = ["dg_nopf_u", "dg_nopf_dm", "dg_dmpf_u", "dg_dmpf_dm", "dg_res", "dg_dmpft_u", "dg_dmpft_res"]
        variants = ["dg_nopf", "dg_dmpf", "dg_dmpft"]
        if L0 == L1:   # the u-prefetch variant needs a square work-group
            tags.append(("dg-uPF-u-" + sh, "uu"))
            twin_k.append("dg_upf_u")
            variants.insert(1, "dg_upf")
        twins = []
        for k in twin_k:
            for Np in (20, 35, 56, 84):
                for Nel in (1 << 14, 1 << 16, 1 << 18):
                    twins.append((k, dict(Np=Np, Nel=Nel, L0=L0, L1=L1)))
        modeled = [(k, dict(Np=Np, Nel=Nel, L0=L0, L1=L1)) for k in variants
                   for Np in (20, 35, 56, 84) for Nel in (1 << 14, 1 << 15, 1 << 16, 1 << 17, 1 << 18)]
        gm = [GENERIC] + [tagged(t, n) for t, n in tags]
        out.append(dict(name="dg_" + sh, gmem=gm, expr=nonlinear(gm),
                        measure=common_measurements() + twins, modeled=modeled))
    fd_sizes = [int(round(1024 * 2 ** (i / 7.0))) for i in range(29)]   # 1024 .. 16384, geometric
    fd_twins = [(k, {"n": n}) for k in ("fd_tile_u", "fd_tile_res", "fd_direct_u", "fd_direct_res",
                                        "fd_tile18_u", "fd_tile18_res")
                for n in (1024, 2048, 4096, 8192, 16384)]
    # the tile variants' result stores are unit-stride AFR-1 patterns, so the
    # generic feature covers them; only the overlapping tile fetches are tagged
    fd_gm = [GENERIC, tagged("fd-tile-u", "tu"), tagged("fd-tile18-u", "t18u")]
    out.append(dict(name="fd", gmem=fd_gm, expr=linear(fd_gm),
                    measure=common_measurements() + fd_twins,
                    modeled=[(k, {"n": n}) for k in ("fd_tile", "fd_tile18", "fd_direct") for n in fd_sizes]))
    if reduced:
        for st in out:
            seen = {}
            keep = []
            for k, p in st["measure"]:
                if k in TWIN_KERNELS:
                    seen[k] = seen.get(k, -1) + 1
                    if seen[k] % 2:
                        continue
                keep.append((k, p))
            st["measure"] = keep
            st["modeled"] = st["modeled"][::3]
    return out


def sweep_studies(reduced=False):
    """The cross-variant sweep: 11 modeled variants (prefetching fp32 matmul,
    BF16 tensor-core matmul with 128 x 256 and 256 x 256 tiles, DG noPF /
    uPF / dmPF / dmPF-T with 16x16 work-groups, the DG tile form and its
    tensor-core form, stencil 16x16 tile and direct) at ~30 sizes each.  Every third size is held out; each variant's
    model is calibrated on the microbenchmarks (plus its computation's twins)
    and the variant's own other sizes -- the paper's "few extra on-line
    calibration runs" -- and predicts the held-out sizes.  A tenth study
    calibrates one model on both tensor-core tiles and ranks them at the
    held-out sizes.

    reduced: a bounded form for a benchmark run -- every second size of each
    variant (so 4-5 held out per variant), matmul up to n = 3072, and the
    paper's other two modeled variants (non-prefetching matmul, 18 x 18
    stencil tile) added."""
    base = {s["name"]: s for s in studies()}
    # the A and B tile loads both scale as n^3 at a fixed tile shape, so one
    # bf16 load feature carries them
    tc_expr = nonlinear(["p_gbf * f_mem_access_global_bfloat16", tagged("tc-c", "tcc")],
                        overhead="p_launch * f_sync_kernel_launch + p_group * f_thread_groups",
                        onchip="p_tc * f_op_bfloat16_madd")
    nels = sorted({int(round(2 ** (14 + 4 * i / 7.0) / 32)) * 32 for i in range(8)})
    dg_sizes = [dict(Np=Np, Nel=Nel, L0=16, L1=16) for Np in (20, 35, 56, 84) for Nel in nels]
    tc_sizes = [{"n": n} for n in range(1024, 8192 + 1, 256)]
    # the tensor-core DG form: no microbenchmark carries its TF32 multiply-adds,
    # its TMA-box u loads or its bulk res stores, so (as for the tensor-core
    # matmul) its own sizes calibrate those costs; the empty kernels fix the
    # launch and group terms
    dgc_expr = nonlinear([tagged("dgc-u", "dcu"), tagged("dgc-res", "dcr")],
                         overhead="p_launch * f_sync_kernel_launch + p_group * f_thread_groups",
                         onchip="p_tf * f_op_tfloat32_madd + p_lm4 * f_mem_access_local_float32x4")
    # the DG tile form: its u tiles arrive by one bulk copy and its operands
    # are read as 8-byte pairs, which none of the DG study's pattern features
    # matches; its u loads and res stores have equal counts (3 Nel Np each), so
    # one cost carries both, and its shared reads grow with its multiply-adds
    # (a fit with both gave the memory term a negative cost), so the
    # multiply-adds carry the on-chip side; its own sizes calibrate them.
    # Linear: on these rows the tanh overlap's switch goes to zero (the
    # linear model's optimum) or to a local optimum that depends on the path
    dgt_expr = linear(["p_dtm * (f_mem_access_tag:dgt-u + f_mem_access_tag:dgt-res)"],
                      overhead="p_launch * f_sync_kernel_launch + p_group * f_thread_groups",
                      onchip="p_madd * f_op_float32_madd")
    plan = [("mm_pf", "matmul", None, [{"n": n} for n in range(512, 4096 + 1, 128)]),
            ("mm_tc", None, tc_expr, tc_sizes), ("mm_tc256", None, tc_expr, tc_sizes)]
    plan += [(k, "dg_16x16", None, dg_sizes) for k in ("dg_nopf", "dg_upf", "dg_dmpf", "dg_dmpft")]
    plan += [("dg_tile", "launch", dgt_expr, [dict(Np=Np, Nel=Nel) for Np in (20, 35, 56, 84) for Nel in nels])]
    plan += [("dg_tc", "launch", dgc_expr, [dict(Np=Np, Nel=Nel) for Np in (20, 35, 56, 84) for Nel in nels])]
    plan += [(k, "fd", None, [{"n": int(round(1024 * 2 ** (i / 7.0)))} for i in range(29)])
             for k in ("fd_tile", "fd_direct")]
    if reduced:
        mm_small = [{"n": n} for n in range(512, 3072 + 1, 128)]
        plan = [(k, parent, expr, mm_small if k == "mm_pf" else sizes) for k, parent, expr, sizes in plan]
        plan.insert(1, ("mm_nopf", "matmul", None, mm_small))
        plan.append(("fd_tile18", "fd", None, [{"n": int(round(1024 * 2 ** (i / 7.0)))} for i in range(29)]))
        plan = [(k, parent, expr, sizes[::2]) for k, parent, expr, sizes in plan]
        tc_sizes = tc_sizes[::2]
        base = {st["name"]: st for st in studies(reduced=True)}   # twins at every second size
    out = []
    for k, parent, expr, sizes in plan:
        fit = [(k, p) for i, p in enumerate(sizes) if i % 3 != 2]
        held = [(k, p) for i, p in enumerate(sizes) if i % 3 == 2]
        if parent == "launch":
            measure = generate(["launch"]) + fit
        else:
            measure = (base[parent]["measure"] if parent else common_measurements()) + fit
        out.append(dict(name="sweep_" + k, expr=expr or base[parent]["expr"], measure=measure, modeled=held))
    # both tensor-core tile shapes in one calibration: their bf16 loads per
    # multiply-add differ (3/256 and 2/256), which separates the load and
    # tensor-op costs; the held-out sizes then rank the two tiles
    tcs = ("mm_tc", "mm_tc256")
    out.append(dict(name="sweep_tc_tiles", expr=tc_expr,
                    measure=common_measurements() + [(k, p) for k in tcs for i, p in enumerate(tc_sizes) if i % 3 != 2],
                    modeled=[(k, p) for k in tcs for i, p in enumerate(tc_sizes) if i % 3 == 2]))
    return out


# the work-removed twins (Algorithm 3) of the modeled kernels
TWIN_KERNELS = {"mm_pf_a", "mm_pf_b", "mm_nopf_a", "mm_nopf_b", "dg_nopf_u", "dg_nopf_dm", "dg_dmpf_u",
                "dg_dmpf_dm", "dg_res", "dg_dmpft_u", "dg_dmpft_res", "dg_upf_u", "fd_tile_u", "fd_tile_res",
                "fd_direct_u", "fd_direct_res", "fd_tile18_u", "fd_tile18_res"}


class Buffers:
    """Device buffers reused across kernels (seeded uniform values in [-1, 1))."""

    def __init__(self, torch, dev, seed=1234):
        self.torch, self.dev = torch, dev
        self.gen = torch.Generator(device=dev)
        self.gen.manual_seed(seed)
        self.pool = {}

    def get(self, kernel, params):
        torch = self.torch
        out = []
        for i, b in enumerate(kernel_buffers(kernel, **params)):
            dt = torch.float64 if b["dtype"] == np.float64 else torch.float32
            key = (i, dt)
            cur = self.pool.get(key)
            if cur is None or cur.numel() < b["elems"]:
                cur = torch.rand(int(b["elems"]), device=self.dev, dtype=dt, generator=self.gen) * 2 - 1
                self.pool[key] = cur
            out.append(cur[:b["elems"]])
        return out


def measure(kernels, bufs, trials, flush_l2=True):
    times = []
    for k, p in kernels:
        tm = run(k, bufs.get(k, p), warmup=2, trials=trials, flush_l2=flush_l2, **p)
        times.append(tm["mean_ms"] * 1e-3)
    return np.array(times)


def spearman(a, b):
    ra, rb = np.argsort(np.argsort(a)), np.argsort(np.argsort(b))
    return float(np.corrcoef(ra, rb)[0, 1])


def kendall(a, b):
    n, s = len(a), 0
    for i in range(n):
        for j in range(i + 1, n):
            s += np.sign(a[i] - a[j]) * np.sign(b[i] - b[j])
    return float(2 * s / (n * (n - 1))) if n > 1 else 1.0


def geomean(x):
    x = np.maximum(np.asarray(x, dtype=np.float64), 1e-300)
    return float(math.exp(np.mean(np.log(x))))


def run_studies(trials=10, names=None, seed=1234, flush_l2=True, study_list=None, cache_path=None):
    """Calibrate each study's model on its measurement set (all studies in one
    batched fit) and predict its modeled kernels.  Returns a report dict.
    flush_l2: every timed trial starts with a cold L2 (pm_run flush_l2).
    A kernel instance shared by several studies is timed once.
    cache_path: a JSON timing cache (timings.TimingCache) read before timing
    and saved after every batch, so an interrupted run resumes."""
    import torch
    from .timings import TimingCache, device_identity
    dev = torch.device("cuda", torch.cuda.current_device())
    bufs = Buffers(torch, dev, seed)
    sts = [s for s in (study_list if study_list is not None else studies()) if names is None or s["name"] in names]
    cache = {}
    tc = TimingCache(cache_path, device_identity(torch, dev.index)) if cache_path else None

    def timed(kernels):
        todo = [(k, p) for k, p in kernels if (k, tuple(sorted(p.items()))) not in cache]
        if tc is not None:
            rest = []
            for k, p in todo:
                v = tc.get(k, p, trials, flush_l2)
                if v is None:
                    rest.append((k, p))
                else:
                    cache[(k, tuple(sorted(p.items())))] = v
            todo = rest
        for (k, p), t in zip(todo, measure(todo, bufs, trials, flush_l2) if todo else []):
            cache[(k, tuple(sorted(p.items())))] = t
            if tc is not None:
                tc.put(k, p, trials, flush_l2, t)
        if tc is not None and todo:
            tc.save()
        return np.array([cache[(k, tuple(sorted(p.items())))] for k, p in kernels])

    models, Xs, ts, info = [], [], [], []
    for s in sts:
        m = Model("f_wall_time", s["expr"])
        Xm = np.stack([m.feature_values(k, **p) for k, p in s["measure"]])
        tm = timed(s["measure"])
        Xp = np.stack([m.feature_values(k, **p) for k, p in s["modeled"]])
        tp = timed(s["modeled"])
        models.append(m)
        Xs.append(Xm)
        ts.append(tm)
        info.append((s, Xp, tp, Xm, tm))
    plan = FitPlan(models, [len(t) for t in ts])
    pvec, reps = plan.run(np.concatenate([x.ravel() for x in Xs]), np.concatenate(ts))
    report, o = {}, 0
    for m, (s, Xp, tp, Xm, tm), rep in zip(models, info, reps):
        p = pvec[o:o + len(m.params)]
        o += len(m.params)
        pred = m.predict(p, Xp)
        fitted = m.predict(p, Xm)
        err = np.abs(pred - tp) / tp
        per = {}
        for v in sorted(set(k for k, _ in s["modeled"])):
            idx = [i for i, (k, _) in enumerate(s["modeled"]) if k == v]
            per[v] = {"geomean_rel_err": geomean(err[idx]), "max_rel_err": float(err[idx].max()),
                      "n_sizes": len(idx)}
        # ranking of variants at equal sizes
        groups = {}
        for i, (k, prm) in enumerate(s["modeled"]):
            key = tuple(sorted((a, b) for a, b in prm.items()))
            groups.setdefault(key, []).append(i)
        agree = [int(np.argmin(pred[g]) == np.argmin(tp[g])) for g in groups.values() if len(g) > 1]
        report[s["name"]] = {
            "expr": s["expr"], "params": dict(zip(m.params, [float(x) for x in p])), "fit": rep,
            "n_measure": len(s["measure"]), "n_modeled": len(s["modeled"]),
            "variants": per, "geomean_rel_err": geomean(err), "max_rel_err": float(err.max()),
            "spearman": spearman(pred, tp), "kendall": kendall(pred, tp),
            "fastest_variant_identified": float(np.mean(agree)) if agree else None,
            "rows": [{"kernel": k, "params": prm, "measured_s": float(a), "predicted_s": float(b)}
                     for (k, prm), a, b in zip(s["modeled"], tp, pred)],
            "measure_rows": [{"kernel": k, "params": prm, "measured_s": float(a), "fitted_s": float(b)}
                             for (k, prm), a, b in zip(s["measure"], tm, fitted)],
            "flush_l2": flush_l2,
        }
        if tc is not None:
            report[s["name"]]["timing_cache"] = {"path": cache_path, "hits": tc.hits, "stored": tc.stored}
    return report


# relative excess of the separately calibrated costs over the measured time
# above which the overlap test reads the on-chip cost as hidden
OVERLAP_MARGIN = 0.10


def choose_overlap_model(separate_over_measured, margin=OVERLAP_MARGIN):
    """The overlap test of Section "Models Demonstrated": the work-removed
    twin's time plus the on-chip cost priced by the microbenchmarks, over the
    kernel's measured time.  About 1 means little or no overlap (the linear
    model); well above 1 means on-chip cost is hidden (the nonlinear model).
    The paper leaves "well above" open; here it is more than `margin`."""
    return "nonlinear" if separate_over_measured > 1.0 + margin else "linear"


def choose_by_residual(residuals):
    """The section's other indicator: of the calibrated models, the one with
    the smallest least-squares residual on the measurement set (a dict
    kind -> residual; the kinds compared are "linear" and "nonlinear")."""
    cand = {k: v for k, v in residuals.items() if k in ("linear", "nonlinear") and v is not None}
    return min(cand, key=cand.get) if cand else None


def diagnostics(trials=10, seed=1234, flush_l2=True, cache_path=None, reduced=False):
    """The paper's diagnostic experiments on this GPU.

    ab_ratio (Section "Data Motion Features", Table ab_pattern): average cost
    per load of the prefetching matmul's b fetch pattern over its a pattern,
    from the two work-removed twins at n = 2048 .. 3584, where overhead is
    negligible (time / tagged loads).

    madd_only (Section "Illustrative Example"): p_madd calibrated on the madd
    throughput kernels alone, as a FLOP/s rate against the FP32 peak, and the
    share of the prefetching matmul's time it accounts for.

    overlap (Section "Modeling Overlap"): per modeled variant, the sum of the
    separately calibrated costs (linear model: twins for global memory,
    microbenchmarks for on-chip work) over the measured time -- near 1 means
    no overlap, well above 1 means hidden on-chip cost -- the model that test
    chooses (Section "Models Demonstrated"), and the geomean error of the
    linear, the tanh-overlap and the partial-overlap model calibrated on the
    same measurement set; per study, each model's calibration residual and
    the model with the smaller one (the section's other indicator).

    reduced: the studies' reduced form (studies(reduced=True)), fewer a/b
    and matmul sizes: a bounded run for tests.  Every calibration in the
    report carries its measured rows, for a refit elsewhere."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    bufs = Buffers(torch, dev, seed)
    out = {}
    # -- a vs b pattern
    rows = []
    for n in range(2048, 3584 + 1, 768 if reduced else 256):
        per = {}
        for k, tag in (("mm_pf_a", "mm-PF-a"), ("mm_pf_b", "mm-PF-b")):
            loads = Model("f_wall_time", "p_x * f_mem_access_tag:%s" % tag).feature_values(k, n=n)[0]
            per[k] = measure([(k, {"n": n})], bufs, trials, flush_l2)[0] / loads
        rows.append({"n": n, "a_s_per_load": per["mm_pf_a"], "b_s_per_load": per["mm_pf_b"],
                     "b_over_a": per["mm_pf_b"] / per["mm_pf_a"]})
    out["ab_ratio"] = {"rows": rows, "mean_b_over_a": float(np.mean([r["b_over_a"] for r in rows]))}
    # -- madd-only calibration: launch, work-group and madd costs on the madd
    # throughput kernels alone (their sizes vary total work and its split)
    m = Model("f_wall_time", LAUNCH + " + p_madd * f_op_float32_madd")
    cal = generate(["flops_pattern", "dtype:0", "op:2"])
    X = np.stack([m.feature_values(k, **p) for k, p in cal])
    t = measure(cal, bufs, trials, flush_l2)
    p, rep = m.fit(X, t)
    madd_rows = [{"kernel": k, "params": q, "measured_s": float(x)} for (k, q), x in zip(cal, t)]
    sizes = [512, 1024, 2048] if reduced else [512, 1024, 1536, 2048, 3072, 4096]
    tm = measure([("mm_pf", {"n": n}) for n in sizes], bufs, trials, flush_l2)
    im = m.params.index("p_madd")
    fm = m.features.index("f_op_float32_madd")
    share = [float(p[im] * m.feature_values("mm_pf", n=n)[fm] / tt) for n, tt in zip(sizes, tm)]
    out["madd_only"] = {"expr": m.expr, "params": dict(zip(m.params, [float(x) for x in p])),
                        "p_madd_s_per_subgroup_op": float(p[im]), "rate_flops": 64.0 / float(p[im]),
                        "fit": rep, "mm_pf_sizes": sizes, "mm_pf_madd_share": share, "rows": madd_rows}
    # -- overlap analysis, linear vs tanh-overlap on the same measurement sets
    res = {}
    fits = {}
    for st in studies(reduced):
        if st.get("extension"):
            continue
        gm = st["gmem"]
        exprs = {"linear": linear(gm), "nonlinear": nonlinear(gm), "partial": partial(gm)}
        if len(set(re.findall(r"\bp_\w+", exprs["partial"]))) > 16:   # the fit's parameter limit
            del exprs["partial"]
        rep_s = run_studies(trials, seed=seed, flush_l2=flush_l2, cache_path=cache_path,
                            study_list=[dict(st, name=st["name"] + "_" + kind, expr=e) for kind, e in exprs.items()])
        per = {}
        lin = rep_s[st["name"] + "_linear"]
        resid = {kind: rep_s[st["name"] + "_" + kind]["fit"].get("residual") for kind in exprs}
        by_resid = choose_by_residual(resid)
        for v in lin["variants"]:
            ratio = [r["predicted_s"] / r["measured_s"] for r in lin["rows"] if r["kernel"] == v]
            per[v] = {"separate_costs_over_measured": geomean(ratio)}
            for kind in exprs:
                per[v][kind + "_geomean_err"] = rep_s[st["name"] + "_" + kind]["variants"][v]["geomean_rel_err"]
            choice = choose_overlap_model(per[v]["separate_costs_over_measured"])
            per[v]["chosen_by_cost_sum"] = choice
            per[v]["chosen_geomean_err"] = per[v][choice + "_geomean_err"]
        if "partial" in exprs:
            per["p_part"] = rep_s[st["name"] + "_partial"]["params"]["p_part"]
        per["calibration_residual"] = resid
        per["chosen_by_residual"] = by_resid
        res[st["name"]] = per
        for kind in exprs:
            r = rep_s[st["name"] + "_" + kind]
            fits[st["name"] + "_" + kind] = {"expr": r["expr"], "params": r["params"], "fit": r["fit"],
                                             "rows": r["measure_rows"]}
    out["overlap"] = res
    out["calibrations"] = fits
    # -- local memory split by lid(1) stride (Section "Finite Differences"): the
    # 16x16 and 18x18 stencil tiles differ in the lid(1) stride of their local
    # accesses; calibrate a per-stride correction on the 2-D local kernels
    fd = [st for st in studies(reduced) if st["name"] == "fd"][0]
    l2d = generate(["lmem2d"])
    split_onchip = ONCHIP + " + p_l18 * f_mem_access_local_float32_lstrides:{1:18}"
    sts = [dict(fd, name="fd_single_lmem", expr=linear(fd["gmem"]), measure=fd["measure"] + l2d),
           dict(fd, name="fd_split_lmem", expr=linear(fd["gmem"], onchip=split_onchip), measure=fd["measure"] + l2d)]
    rep_s = run_studies(trials, seed=seed, flush_l2=flush_l2, cache_path=cache_path, study_list=sts)
    for name in ("fd_single_lmem", "fd_split_lmem"):
        r = rep_s[name]
        fits[name] = {"expr": r["expr"], "params": r["params"], "fit": r["fit"], "rows": r["measure_rows"]}
    per_access = {}
    for T in (16, 18):
        rows = [(k, p) for k, p in l2d if p["T"] == T]
        ml = Model("f_wall_time", "p_l * f_mem_access_local_float32")
        X = np.stack([ml.feature_values(k, **p) for k, p in rows])
        t = measure(rows, bufs, trials, flush_l2)
        per_access["T%d" % T] = float(np.median(t / X[:, 0]))
    out["split_lmem"] = {
        "s_per_subgroup_local_access": per_access,
        "single": {v: r["geomean_rel_err"] for v, r in rep_s["fd_single_lmem"]["variants"].items()},
        "split": {v: r["geomean_rel_err"] for v, r in rep_s["fd_split_lmem"]["variants"].items()},
        "p_lmem": rep_s["fd_split_lmem"]["params"]["p_lmem"], "p_l18": rep_s["fd_split_lmem"]["params"]["p_l18"],
        "fastest_identified": {k: rep_s[k]["fastest_variant_identified"] for k in rep_s}}
    return out


def illustrative(trials=20, seed=1234, flush_l2=True):
    """Configuration 1: t = p_f flops + p_g gmem + p_s smem + p_l work-groups on
    the prefetching matmul at n = 256..768 (rank-2 design: minimum-norm fit),
    predict n = 896."""
    import torch
    from . import _lib  # noqa: F401
    dev = torch.device("cuda", torch.cuda.current_device())
    bufs = Buffers(torch, dev, seed)
    expr = ("p_f * f_op_float32_madd + p_g * f_mem_access_global_float32 + p_s * f_mem_access_local_float32 + "
            "p_l * f_thread_groups")
    m = Model("f_wall_time", expr)
    fit_n, test_n = [256, 384, 512, 640, 768], [896]
    X = np.stack([m.feature_values("mm_pf", n=n) for n in fit_n])
    t = measure([("mm_pf", {"n": n}) for n in fit_n], bufs, trials, flush_l2)
    p, rep = m.fit(X, t)
    Xt = np.stack([m.feature_values("mm_pf", n=n) for n in test_n])
    tt = measure([("mm_pf", {"n": n}) for n in test_n], bufs, trials, flush_l2)
    pred = m.predict(p, Xt)
    return {"expr": expr, "fit_sizes": fit_n, "fit_times_s": t.tolist(), "params": p.tolist(), "report": rep,
            "test_sizes": test_n, "measured_s": tt.tolist(), "predicted_s": pred.tolist(),
            "rel_err": (np.abs(pred - tt) / tt).tolist()}


if __name__ == "__main__":
    import json
    import sys
    flush = "--no-flush" not in sys.argv
    cache = next((a.split("=", 1)[1] for a in sys.argv[1:] if a.startswith("--cache=")), None)
    # --only=a,b runs a subset of: illustrative, studies, sweep, diagnostics
    only = next((a.split("=", 1)[1].split(",") for a in sys.argv[1:] if a.startswith("--only=")), None)
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    parts = {"illustrative": lambda: illustrative(flush_l2=flush),
             "studies": lambda: run_studies(flush_l2=flush, cache_path=cache),
             "sweep": lambda: run_studies(flush_l2=flush, study_list=sweep_studies(), cache_path=cache),
             "diagnostics": lambda: diagnostics(flush_l2=flush, cache_path=cache)}
    for name in only or []:
        if name not in parts:
            sys.exit("unknown part %r (one of %s)" % (name, ", ".join(parts)))
    out = {name: run() for name, run in parts.items() if only is None or name in only}
    sys.argv = [sys.argv[0]] + args
    json.dump(out, open(sys.argv[1], "w") if len(sys.argv) > 1 else sys.stdout, indent=1)
