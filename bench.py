#!/usr/bin/env python
"""Benchmark: one calibration pass of the performance-modeling hot path per
step, on synthetic inputs shaped like the paper's workloads.

Step = every variant of the calibration suite (global-memory stream patterns,
arithmetic loops, local memory, barriers, overlap, empty launches; ~230
variants) device-timed with `--trials` launches each (pm_run), exact features
for every variant (pm_counts), feature assembly and ONE batched calibration of
all per-family models on two thirds of the variants, and prediction of the
held-out third.  Reported value: suite GB/s = algorithmic bytes moved by the
suite's launches / step time.

Multi-GPU: replicas only (calibration is per device); each rank runs the
whole pass on its GPU, value = all ranks' bytes / max time.

--impl reference runs the CPU oracle (the plain reference implementation)
on a bounded sample of each variant and reports the same metric.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "suite GB/s & % roofline; held-out pred. rel. error; batched-fit fits/s vs plain"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--trials", type=int, default=3, help="timed launches per suite variant per step")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fit-bench", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the per-variant held-out accuracy leg")
    ap.add_argument("--no-tiles", action="store_true", help="skip the modeled computations' GB300 kernels leg")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--filter", default="suite", help="comma-separated suite filter tags")
    ap.add_argument("--dump", default=None, help="write per-variant timings of the last step (JSON)")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (read-only queries)."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- ours
def kernel_instance(kernel, p):
    """Name of the CUDA kernel instantiation a variant launches."""
    if kernel == "stream":
        t = {(0, 0): "float", (0, 1): "float4", (1, 0): "double", (1, 1): "double2"}[(p.get("dtype", 0), p.get("vec", 0))]
        return "k_stream<%s,%d,%d>" % (t, p.get("L", 1), p.get("shape", 0))
    if kernel == "fma":
        return "k_fma<%s,%d>" % ("float" if p.get("dtype", 0) == 0 else "double", p.get("op", 2))
    if kernel == "smem":
        return "k_smem<%d>" % p.get("sync", 0)
    return "k_" + kernel


def workload_config(variants, trials):
    """The workload a step covers; identical in both arms."""
    from paper_1904_09538_gb300 import suite as S
    bps = sum(S.algorithmic_bytes(k, p) for k, p in variants) * trials
    return {"workload": "calibration suite (stream, arithmetic, local-memory, barrier, overlap, empty kernels): "
                        "%d variants, %d timed launches each (%d for the empty kernels)" % (len(variants), trials,
                                                                                              10 * trials),
            "variants": len(variants), "trials_per_variant": trials,
            "families": len({S.family_key(k, p) for k, p in variants}), "bytes_per_step": bps,
            "l2": "stream variants under 2x L2 (%d) timed from a flushed L2, the others larger than L2 (arrays "
                  "up to 2 GiB; step footprint %.0f GB)" % (sum(S.cache_resident(k, p) for k, p in variants),
                                                             bps / 1e9),
            "parallelism": "replicas"}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1904_09538_gb300 as pm
    from paper_1904_09538_gb300 import suite as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks, peak_kind = load_peaks()

    variants = S.generate(args.filter.split(","))
    # device pools: 5 buffers per dtype, sized for the largest variant
    need32, need64 = 1, 1
    for k, p in variants:
        for b in pm.kernel_buffers(k, **p):
            if b["dtype"] == np.float64:
                need64 = max(need64, b["elems"])
            else:
                need32 = max(need32, b["elems"])
    gen = torch.Generator(device=dev)
    gen.manual_seed(1234 + rank)
    pool32 = [torch.rand(need32, device=dev, generator=gen) * 2 - 1 for _ in range(5)]
    pool64 = [torch.rand(need64, device=dev, generator=gen, dtype=torch.float64) * 2 - 1 for _ in range(5)]

    def bufs_for(k, p):
        out, i32, i64 = [], 0, 0
        for b in pm.kernel_buffers(k, **p):
            if b["dtype"] == np.float64:
                out.append(pool64[i64][:b["elems"]])
                i64 += 1
            else:
                out.append(pool32[i32][:b["elems"]])
                i32 += 1
        return out

    prepared = [(k, p, bufs_for(k, p), S.algorithmic_bytes(k, p), kernel_instance(k, p)) for k, p in variants]
    families = {}
    for idx, (k, p) in enumerate(variants):
        families.setdefault(S.family_key(k, p), []).append(idx)
    fam_names = sorted(families)
    models = {f: pm.Model("f_wall_time", S.family_model(f)) for f in fam_names}
    # feature rows (exact counts), fixed per variant
    rows = {}
    for f in fam_names:
        for idx in families[f]:
            k, p = variants[idx]
            rows[idx] = models[f].feature_values(k, **p)
    fit_rows = {f: [i for j, i in enumerate(families[f]) if j % 3 != 2] for f in fam_names}
    held = {f: [i for j, i in enumerate(families[f]) if j % 3 == 2] for f in fam_names}
    plan = pm.FitPlan([models[f] for f in fam_names], [len(fit_rows[f]) for f in fam_names])
    Xfit = np.concatenate([np.stack([rows[i] for i in fit_rows[f]]).ravel() for f in fam_names])

    stream = torch.cuda.current_stream()
    flushed = [S.cache_resident(k, p) for k, p in variants]
    # the empty kernels last a few microseconds: ten times the trials keep
    # their event-timing jitter out of the calibration
    ntrials = [args.trials * (10 if k == "empty" else 1) for k, p in variants]
    # variant launches, one L2-flush launch per trial of the cache-resident
    # variants, the batched fit's graph (3 kernels) and one predict per family
    launches_per_step = sum(ntrials) + sum(t for t, f in zip(ntrials, flushed) if f) + 3 + len(fam_names)

    last_times = {}

    fitted, fam_errs = {}, {}

    def fit_and_predict(times):
        # calibrate every family model on its fitting rows in one batched launch
        tfit = np.array([times[i] for f in fam_names for i in fit_rows[f]])
        pvec, reps = plan.run(Xfit, tfit)
        # predict the held-out rows
        o, errs = 0, []
        fam_errs.clear()
        for f, npar in zip(fam_names, plan.nparams):
            pf = pvec[o:o + npar]
            fitted[f] = dict(zip(models[f].params, (float(x) for x in pf)))
            o += npar
            if held[f]:
                Xh = np.stack([rows[i] for i in held[f]])
                pred = models[f].predict(pf, Xh)
                meas = np.array([times[i] for i in held[f]])
                e = list(np.abs(pred - meas) / meas)
                errs.extend(e)
                fam_errs[f] = e
        return errs, reps

    def one_step(record):
        times = last_times
        for idx, (k, p, bufs, nbytes, inst) in enumerate(prepared):
            tm = pm.run(k, bufs, warmup=0, trials=ntrials[idx], outlier_factor=0.0, flush_l2=flushed[idx], **p)
            times[idx] = tm["mean_ms"] * 1e-3
            if record is not None:
                record.append((idx, inst, nbytes, tm["mean_ms"] * ntrials[idx], ntrials[idx]))
        return fit_and_predict(times)

    for _ in range(args.warmup):
        one_step(None)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    record = []
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    all_errs, fit_status = [], []
    for _ in range(args.steps):
        errs, reps = one_step(record)
        all_errs.extend(errs)
        fit_status.extend(r["status"] for r in reps)
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    from paper_1904_09538_gb300 import replicas
    bytes_per_step = sum(x[3] for x in prepared) * args.trials
    value, elapsed = replicas.job_throughput(bytes_per_step * args.steps, t_start.elapsed_time(t_end) * 1e-3,
                                             dist, dev)
    value /= 1e9
    geo_rank = math.exp(sum(math.log(max(e, 1e-12)) for e in all_errs) / len(all_errs)) if all_errs else None
    rank_reports = replicas.gather_reports({"rank": rank, "heldout_geomean": geo_rank,
                                            "fit_status": sorted(set(fit_status))}, dist)

    # roofline of the dominant kernel instantiation (largest share of device time)
    per = {}
    for _, inst, nbytes, ms, n in record:
        a = per.setdefault(inst, [0.0, 0.0, 0])
        a[0] += nbytes * n
        a[1] += ms
        a[2] += n
    tot_ms = sum(a[1] for a in per.values())
    dom = max(per, key=lambda k: per[k][1])
    achieved = per[dom][0] / (per[dom][1] * 1e-3) / 1e9
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        try:
            tj = json.load(open(tpath))
            ent = tj.get(dom)
            if ent and ent.get("source_sha") == source_sha(ent.get("source", "pm_suite.cu"), dom.split("<")[0]):
                traffic = ent["dram_bytes_per_launch"]
        except Exception:
            traffic = None
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                "peak_source": peak_kind, "share": round(per[dom][1] / tot_ms, 4)}
    best_stream = max((a[0] / (a[1] * 1e-3) / 1e9, k) for k, a in per.items() if k.startswith("k_stream"))

    geo = math.exp(sum(math.log(max(e, 1e-12)) for e in all_errs) / len(all_errs)) if all_errs else None
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(elapsed / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
        "config": workload_config(variants, args.trials),
        "roofline": roofline,
        "best_stream_kernel": {"kernel": best_stream[1], "GB/s": round(best_stream[0], 1),
                               "frac": round(best_stream[0] / peaks["hbm_gbs"], 4)},
        "heldout_pred_rel_err": {"geomean": geo, "max": max(all_errs) if all_errs else None, "n": len(all_errs),
                                 "max_by_family_last_step": {f: round(max(e), 4) for f, e in sorted(fam_errs.items())}},
        "fit_status_counts": {str(s): fit_status.count(s) for s in sorted(set(fit_status))},
        "clocks": clk,
        "gpu_launches": launches_per_step * args.steps,
    }
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    line["calibrated"] = calibrated_rates(fitted, sm_count, clk.get("sm_mhz"))
    # per-variant roofline fractions from the mean launch time over the timed steps
    tsum, nsum = [0.0] * len(variants), [0] * len(variants)
    for idx, _, _, ms, n in record:
        tsum[idx] += ms
        nsum[idx] += n
    mean_s = [tsum[i] / nsum[i] * 1e-3 if nsum[i] else None for i in range(len(variants))]
    line["suite_roofline"] = suite_roofline(variants, mean_s, peaks["hbm_gbs"], sm_count, clk.get("sm_mhz"))
    line["suite_roofline"]["stream_bounds"] = stream_bounds(pm, torch, variants, mean_s, peaks["hbm_gbs"], sm_count,
                                                            bufs_for)
    if world > 1:
        line["ranks"] = rank_reports
    if args.dump and rank == 0:
        json.dump([{"kernel": k, "params": p, "instance": inst, "mean_s": last_times[i], "bytes": nb,
                    "GB/s": nb / last_times[i] / 1e9 if last_times[i] > 0 else None}
                   for i, (k, p, _b, nb, inst) in enumerate(prepared)], open(args.dump, "w"), indent=0)
    if not args.no_e2e:
        fit_sizes = {"models": len(fam_names), "params": sum(plan.nparams), "rows": sum(len(fit_rows[f]) for f in fam_names),
                     "features": int(Xfit.size), "heldout": sum(len(held[f]) for f in fam_names),
                     "heldout_features": sum(len(held[f]) * len(models[f].features) for f in fam_names)}
        line["e2e"] = e2e_measure(pm, S, variants, torch, args.trials, fit_and_predict, fit_sizes)
    if not args.no_fit_bench:
        line["fit"] = fit_throughput(pm, torch, dev)
        gpu_params = line["fit"].pop("_params")
        if rank == 0 and world == 1 and not args.no_cpu:
            orc = oracle_fit_rate()
            line["fit"]["max_param_rel_err_vs_oracle"] = fit_vs_oracle(gpu_params, orc.pop("_params"))
            line["fit"]["oracle_cpu"] = orc
    if not args.no_tiles:
        line["tile_kernels"] = tile_kernels_leg(pm, torch, dev, peaks, clk.get("sm_mhz"))
    if not args.no_accuracy:
        line["accuracy"] = accuracy_leg()
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(variants, seconds=12.0)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def variant_work(kernel, p):
    """(algorithmic bytes, flops, local-memory bytes) of one suite launch:
    bytes by the kernel's definition; flops and local bytes from its exact
    counts (a madd is 2 flops, a local access moves 4 bytes per work-item)."""
    import paper_1904_09538_gb300 as pm
    from paper_1904_09538_gb300 import suite as S
    flops = lbytes = 0
    if kernel in ("fma", "smem"):
        for f in pm.counts(kernel, **p):
            if f["kind"] == "op":
                flops += f["count_wi"] * (2 if f["op"] == "madd" else 1)
            elif f["kind"] == "mem" and f["mem"] == "local":
                lbytes += f["count_wi"] * f["dsize"]
    return S.algorithmic_bytes(kernel, p), flops, lbytes


def suite_roofline(variants, mean_s, hbm_gbs, sm_count, sm_mhz, l2_bytes=None):
    """Per-variant fractions of the roofline that bounds each suite kernel,
    from its mean launch time: stream variants of at least 4x the L2 size
    against the measured HBM copy rate (smaller ones are partly served by
    L2 and claim nothing), by lid(0) stride; FP32 arithmetic loops against
    SMs x 128 lanes x clock operations (x2 flops for madd); local-memory
    loops against SMs x 128 bytes x clock.  FP64 loops are reported as
    TFLOP/s (no peak is assumed for GB300's FP64 pipe)."""
    from paper_1904_09538_gb300 import suite as S
    l2 = l2_bytes or S.L2_BYTES
    clk = (sm_mhz or 2070.0) * 1e6
    lanes = sm_count * 128 * clk

    def summary(fr):
        fr = sorted(fr)
        return {"n": len(fr), "min": round(fr[0], 4), "median": round(fr[len(fr) // 2], 4),
                "max": round(fr[-1], 4)} if fr else None

    stream, fma, f64, smem = {}, {}, [], {}
    for (k, p), t in zip(variants, mean_s):
        if t is None or t <= 0:
            continue
        nbytes, flops, lbytes = variant_work(k, p)
        if k == "stream" and nbytes >= 4 * l2:
            key = "2d" if p.get("shape", 0) == 1 else "s%d" % p["s"]
            stream.setdefault(key, []).append(nbytes / t / 1e9 / hbm_gbs)
        elif k == "fma" and p["dtype"] == 0:
            op = ("add", "mul", "madd")[p["op"]]
            fma.setdefault(op, []).append(flops / t / (lanes * (2 if op == "madd" else 1)))
        elif k == "fma":
            f64.append(flops / t / 1e12)
        elif k == "smem":
            smem.setdefault("sync%d" % p["sync"], []).append(lbytes / t / lanes)
    allf = [x for v in stream.values() for x in v]
    return {
        "sm_mhz": round(clk / 1e6, 1),
        "stream_ge_4x_l2": {"variants": len(allf), "at_least_0.8": sum(x >= 0.8 for x in allf),
                            "by_stride": {k: summary(v) for k, v in sorted(stream.items())}},
        "fma_f32_vs_pipe": {k: summary(v) for k, v in sorted(fma.items())},
        "fma_f64_madd_tflops": summary(f64),
        "smem_vs_bandwidth": {k: summary(v) for k, v in sorted(smem.items())},
    }


def stream_bounds(pm, torch, variants, mean_s, hbm_gbs, sm_count, bufs_for, l2_bytes=None):
    """The bound that applies to each stream variant of at least 4x the L2
    size, the smallest of:
      hbm      the measured copy rate;
      pattern  the same kernel instantiation with its working set in L2,
               timed warm at two sizes (about 24 and 96 MiB): the marginal
               rate, bytes over time between them, is what the memory system
               delivers this access pattern with DRAM out of the way (for
               lid(0) strides of 8 or more the L2 request rate);
      little   Little's law with the unloaded HBM latency: resident
               work-items x bytes each has in flight (its L loads, then its
               store) / latency, for all SMs (pm_probe_latency on a 1 GiB
               buffer; the resident count from pm_kernel_resources).
    Returns the latencies, and per lid(0) stride / shape the fraction of the
    applicable bound (min / median / max) with the variants below 0.8."""
    from paper_1904_09538_gb300 import suite as S
    l2 = l2_bytes or S.L2_BYTES
    dev = torch.cuda.current_device()
    big = torch.empty(1 << 30, dtype=torch.uint8, device=dev)
    lat_hbm = pm.probe_latency(big, hops=100000)
    del big
    small = torch.empty(16 << 20, dtype=torch.uint8, device=dev)
    lat_l2 = pm.probe_latency(small, hops=100000)
    del small
    ceil, res_cache, per, below = {}, {}, {}, []
    for (k, p), t in zip(variants, mean_s):
        nbytes = S.algorithmic_bytes(k, p)
        if k != "stream" or t is None or t <= 0 or nbytes < 4 * l2:
            continue
        key = tuple(sorted((a, b) for a, b in p.items() if a != "N"))
        if key not in ceil:
            pts = []
            try:
                for target in (24 << 20, 96 << 20):
                    q = dict(p)
                    n = p["N"]
                    while n > 1 and S.algorithmic_bytes(k, dict(q, N=n)) > target:
                        n //= 2
                    q["N"] = n
                    tm = pm.run(k, bufs_for(k, q), warmup=3, trials=20, flush_l2=False, **q)
                    pts.append((S.algorithmic_bytes(k, q), tm["median_ms"] * 1e-3))
                (b1, t1), (b2, t2) = pts
                ceil[key] = (b2 - b1) / (t2 - t1) / 1e9 if t2 > t1 and b2 > b1 else None
            except pm.PMError:   # no valid L2-resident size of this shape
                ceil[key] = None
        if key not in res_cache:
            r = pm.resources(k, **p)
            res_cache[key] = r["blocks_per_sm"] * r["threads_per_block"]
        esize = 16 if p.get("vec", 0) else (8 if p.get("dtype", 0) else 4)
        little = sm_count * res_cache[key] * esize * (p.get("L", 1) + 1) / (lat_hbm * 1e-9) / 1e9
        cands = {"hbm": hbm_gbs, "little": little}
        if ceil[key]:
            cands["pattern"] = ceil[key]
        kind = min(cands, key=cands.get)
        got = nbytes / t / 1e9
        frac = got / cands[kind]
        skey = "2d" if p.get("shape", 0) == 1 else "s%d" % p["s"]
        per.setdefault(skey, []).append((frac, kind, cands[kind]))
        if frac < 0.8:
            below.append({"params": p, "gbs": round(got, 1), "bound": kind, "bound_gbs": round(cands[kind], 1),
                          "frac": round(frac, 3)})

    def summ(v):
        fr = sorted(x[0] for x in v)
        kinds = sorted(set(x[1] for x in v))
        return {"n": len(v), "min": round(fr[0], 3), "median": round(fr[len(fr) // 2], 3), "max": round(fr[-1], 3),
                "bounds": kinds, "bound_gbs_median": round(sorted(x[2] for x in v)[len(v) // 2], 1)}
    allf = [x[0] for v in per.values() for x in v]
    return {"hbm_latency_ns": round(lat_hbm, 1), "l2_latency_ns": round(lat_l2, 1),
            "variants": len(allf), "at_least_0.8_of_bound": sum(f >= 0.8 for f in allf),
            "by_stride": {k: summ(v) for k, v in sorted(per.items())}, "below_0.8": below}


def calibrated_rates(fitted, sm_count, sm_mhz):
    """The suite families' fitted per-unit costs as rates (the conversions of
    the paper's Table mm_param_vals), against the peaks they estimate.
    A sub-group op is 32 lanes (a madd is 2 flops), a sub-group local access
    moves 32 x 4 bytes, a stream access one 16-byte vector per work-item.
    FP32 peak = SMs x 128 lanes x 2 x clock; shared memory = SMs x 128 B x
    clock, at the sampled median SM clock (2070 MHz if none was sampled)."""
    from paper_1904_09538_gb300.report import rate as unit_rate
    clk = (sm_mhz or 2070.0) * 1e6
    fp32_peak, smem_peak = sm_count * 128 * 2 * clk, sm_count * 128 * clk

    def rate(fam, par, gran, per_wi):
        v = fitted.get(fam, {}).get(par)
        return None if v is None else unit_rate(v, gran, per_wi)

    out = {"sm_mhz": round(clk / 1e6, 1), "fp32_peak_tflops": round(fp32_peak / 1e12, 2),
           "smem_peak_tbs": round(smem_peak / 1e12, 2)}
    # (key, family, parameter, counting granularity, flops or bytes per work-item)
    for key, fam, par, gran, per_wi in (("f32_madd_tflops", "fma_f32_madd", "p_madd", "SG", 2),
                                        ("f32_mul_tflops", "fma_f32_mul", "p_mul", "SG", 1),
                                        ("f32_add_tflops", "fma_f32_add", "p_add", "SG", 1),
                                        ("f64_madd_tflops", "fma_f64_madd", "p_madd", "SG", 2),
                                        ("lmem_tbs", "smem_sync0", "p_lmem", "SG", 4),
                                        ("lmem_sync_tbs", "smem_sync1", "p_lmem", "SG", 4),
                                        ("gmem_f32_s1_gbs", "stream_f32_s1", "p_gmem", "WI", 16),
                                        ("gmem_f64_s1_gbs", "stream_f64_s1", "p_gmem", "WI", 16)):
        r = rate(fam, par, gran, per_wi)
        out[key] = round(r / (1e9 if key.endswith("gbs") else 1e12), 3) if r else None
    if out["f32_madd_tflops"]:
        out["f32_madd_frac"] = round(out["f32_madd_tflops"] * 1e12 / fp32_peak, 4)
    if out["lmem_tbs"]:
        out["lmem_frac"] = round(out["lmem_tbs"] * 1e12 / smem_peak, 4)
    emp, bar = fitted.get("empty", {}), fitted.get("barrier", {})
    out["launch_us"] = round(emp["p_launch"] * 1e6, 3) if "p_launch" in emp else None
    out["group_ns"] = round(emp["p_group"] * 1e9, 4) if "p_group" in emp else None
    out["barrier_ns_per_group"] = round(bar["p_bar"] * 1e9, 4) if "p_bar" in bar else None
    return out


def source_sha(f="pm_suite.cu", kernel="k_stream"):
    """Hash of a kernel's definition (from its __global__ line to the closing
    brace of its body): a recorded DRAM traffic figure is valid only while
    that definition is unchanged."""
    import hashlib
    import re
    src = open(os.path.join(ROOT, "paper_1904_09538_gb300", "csrc", f)).read()
    m = re.search(r"__global__[^;{]*\b%s\s*\(" % re.escape(kernel), src)
    if not m:
        return None
    i = src.index("{", m.end())
    depth, j = 0, i
    while j < len(src):
        depth += {"{": 1, "}": -1}.get(src[j], 0)
        j += 1
        if depth == 0:
            break
    return hashlib.sha256(src[m.start():j].encode()).hexdigest()[:16]


def gpu_local_cpus(torch, dev_index):
    """Host CPUs local to the GPU's PCI device (Linux sysfs), or None."""
    try:
        pr = torch.cuda.get_device_properties(dev_index)
        bus = "%04x:%02x:%02x.0" % (getattr(pr, "pci_domain_id"), getattr(pr, "pci_bus_id"), getattr(pr, "pci_device_id"))
        text = open("/sys/bus/pci/devices/%s/local_cpulist" % bus).read().strip()
        cpus = set()
        for part in text.split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        return cpus & os.sched_getaffinity(0) or None
    except Exception:
        return None


def e2e_measure(pm, S, variants, torch, trials, fit_and_predict, fit_sizes, steps=3):
    """Same step through the public API with host buffers: pm_run_host_batch
    over every variant (inputs in four pinned host buffers, each variant
    reading a prefix of them, so each buffer is one shared region that the
    batch copies to the device once per step; per variant its `trials`
    timed launches, the outputs of the measurement kernels left on the
    device), then the batched calibration and the held-out predictions from
    host arrays, their results read back.  `steps` steps, timed on the host
    clock; the copied bytes are the library's own count."""
    import numpy as np
    # staging buffers on the host memory next to the GPU: run (and first-touch
    # the pinned pages) on the GPU's local CPUs
    saved = os.sched_getaffinity(0)
    local = gpu_local_cpus(torch, torch.cuda.current_device())
    if local:
        os.sched_setaffinity(0, local)
    need = 1
    for k, p in variants:
        for b in pm.kernel_buffers(k, **p):
            need = max(need, b["elems"] * np.dtype(b["dtype"]).itemsize)
    ins = [torch.empty(need, dtype=torch.uint8, pin_memory=True) for _ in range(4)]
    for a in ins:   # values in [-1, 1) as float32 bit patterns are fine for every kernel here
        a.numpy().view(np.float32)[:] = 0.5
    nbytes = 0
    jobs = []
    for j, (k, p) in enumerate(variants):
        arrs, ii = [], 0
        for b in pm.kernel_buffers(k, **p):
            if b["role"] == "in":
                a = ins[ii].numpy().view(b["dtype"])[:b["elems"]]
                ii += 1
            else:
                a = None    # the measurement kernels' outputs stay on the device
            arrs.append(a)
        jobs.append((k, arrs, p))
        nbytes += S.algorithmic_bytes(k, p) * trials
    h2d, d2h = pm.run_host_batch_bytes(jobs)
    # the step's result read back to the host: fitted parameters, fit
    # reports (64 bytes per model) and held-out predictions; the fit's
    # inputs (features, times) go host -> device
    d2h += 8 * (fit_sizes["params"] + fit_sizes["heldout"]) + 64 * fit_sizes["models"]
    h2d += 8 * (fit_sizes["features"] + fit_sizes["rows"] + fit_sizes["heldout_features"])
    # this box's link rates (pinned 1 GiB copies, untimed), for reading copy_ms
    link = {}
    dbuf = torch.empty(1 << 30, dtype=torch.uint8, device=torch.cuda.current_device())
    hbuf = ins[0][:1 << 30] if need >= 1 << 30 else torch.empty(1 << 30, dtype=torch.uint8, pin_memory=True)
    for name, dst, src in (("h2d_gbs", dbuf, hbuf), ("d2h_gbs", hbuf, dbuf)):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for _ in range(3):
            dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        link[name] = round(3 * (1 << 30) / (time.perf_counter() - t1) / 1e9, 1)
    del dbuf
    # untimed warm-up: the largest variant sizes the reserved staging pool
    big = max(jobs, key=lambda x: sum(a.nbytes for a in x[1] if a is not None))
    pm.run_host_batch(jobs[:3] + [big, big], warmup=0, trials=1)
    torch.cuda.synchronize()
    # `steps` timed steps (the host link is shared with the machine's other
    # GPUs, so one step is a thin sample): aggregate throughput, each step kept
    step_ms, copy_list, kern_list, fit_list = [], [], [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        tms, copy_ms = pm.run_host_batch(jobs, warmup=0, trials=trials, outlier_factor=0.0)
        t1 = time.perf_counter()
        fit_and_predict({i: t["mean_ms"] * 1e-3 for i, t in enumerate(tms)})
        torch.cuda.synchronize()
        step_ms.append((time.perf_counter() - t0) * 1e3)
        fit_list.append((time.perf_counter() - t1) * 1e3)
        copy_list.append(copy_ms)
        kern_list.append(sum(t["mean_ms"] * t["n_trials"] for t in tms))
    os.sched_setaffinity(0, saved)
    dt = sum(step_ms) * 1e-3
    return {"value": round(steps * nbytes / dt / 1e9, 2), "unit": "GB/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "steps": steps, "ms_per_step": round(dt * 1e3 / steps, 2),
            "step_ms": [round(x, 1) for x in step_ms], "copy_ms": [round(x, 1) for x in copy_list],
            "kernel_ms": [round(x, 1) for x in kern_list], "fit_predict_ms": [round(x, 1) for x in fit_list],
            "other_ms": [round(a - b - c - d, 1) for a, b, c, d in zip(step_ms, copy_list, kern_list, fit_list)],
            "link": dict(link, copies_at_link_rate_ms=round((h2d / link["h2d_gbs"] + d2h / link["d2h_gbs"]) / 1e6, 1)),
            "host_cpus": len(local) if local else None}


def fit_throughput(pm, torch, dev):
    """Batched calibration (64 models of 4..12 parameters, uneven 40..400 rows,
    one persistent launch in a CUDA graph) against three per-model fits on
    the same GPU, same data, same start points, every model fitted:
      plain          host-driven LM through the autograd.Function, one model
                     at a time (library residual, adjoint, Jacobian, step and
                     update calls; one status read per trial);
      pm_fit loop    the single-model entry point called once per model (a
                     plan built, run and freed per call);
      plan per model one single-model plan per model, built before timing and
                     replayed in turn (the batching alone).
    The per-model parameter vectors of the batched and plain fits are
    returned under "_params" for the comparison with the oracle's fits."""
    import numpy as np
    from paper_1904_09538_gb300 import autograd as pag
    from paper_1904_09538_gb300.fitbench import problem
    from paper_1904_09538_gb300.autotune import tune_fit_threads
    K = 64
    models, Xs, ts, p0s, ls = problem(K)
    # the autotuner picks the fit kernel's CTA size for this batch
    threads, tune_times = tune_fit_threads(models, Xs, ts, p0s, candidates=(64, 128, 256, 512), reps=5)
    plan = pm.FitPlan(models, [len(t) for t in ts], p0_given=True, threads=threads)
    Xc = np.concatenate([x.ravel() for x in Xs])
    tc = np.concatenate(ts)
    pc = np.concatenate(p0s)
    plan.run(Xc, tc, pc)
    torch.cuda.synchronize()
    reps_n = 20
    t0 = time.perf_counter()
    for _ in range(reps_n):
        pb, reps = plan.run(Xc, tc, pc)
    dt_b = (time.perf_counter() - t0) / reps_n
    o = np.cumsum([0] + [len(p) for p in p0s])
    batched = [pb[o[k]:o[k + 1]].copy() for k in range(K)]

    def timed(fn):
        fn(0)                         # untimed: one-time initialisation
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = [fn(k) for k in range(K)]
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / K, out

    Xd = [torch.from_numpy(X).to(dev) for X in Xs]
    td = [torch.from_numpy(t).to(dev) for t in ts]
    dt_p, plain = timed(lambda k: pag.lm_fit(models[k], Xd[k], td[k], p0s[k]))
    dt_f, loop = timed(lambda k: models[k].fit(Xs[k], ts[k], p0=p0s[k]))
    singles = [pm.FitPlan([models[k]], [len(ts[k])], p0_given=True, threads=threads) for k in range(K)]
    dt_q, per_plan = timed(lambda k: singles[k].run(Xs[k].ravel(), ts[k], p0s[k]))

    def rel(a, b):
        return float(np.max(np.abs(np.asarray(a) - b) / np.abs(b)))

    fps_b = K / dt_b
    return {"models": K, "rows": [int(ls.min()), int(ls.max())], "cta_threads": threads,
            "tuned_ms": {str(k): round(v * 1e3, 3) for k, v in tune_times.items()},
            "fits_per_s_batched": round(fps_b, 1),
            "fits_per_s_plain": round(1.0 / dt_p, 2), "speedup": round(fps_b * dt_p, 1),
            "fits_per_s_pm_fit_loop": round(1.0 / dt_f, 2), "speedup_vs_pm_fit_loop": round(fps_b * dt_f, 1),
            "fits_per_s_plan_per_model": round(1.0 / dt_q, 2), "speedup_vs_plan_per_model": round(fps_b * dt_q, 1),
            "batched_ms": round(dt_b * 1e3, 3), "plain_ms_per_model": round(dt_p * 1e3, 3),
            "plain_iterations_max": max(r["iterations"] for _, r in plain),
            "max_param_rel_diff_plain_vs_batched": max(rel(pp, pbk) for (pp, _), pbk in zip(plain, batched)),
            "max_param_rel_diff_pm_fit_loop_vs_batched": max(rel(pp, pbk) for (pp, _), pbk in zip(loop, batched)),
            "statuses": {str(s): [r["status"] for r in reps].count(s) for s in set(r["status"] for r in reps)},
            "statuses_plain": {str(s): [r["status"] for _, r in plain].count(s)
                               for s in set(r["status"] for _, r in plain)},
            "_params": {"batched": batched, "plain": [pp for pp, _ in plain]}}


def tile_kernels_leg(pm, torch, dev, peaks, sm_mhz, trials=10):
    """The modeled computations' GB300 kernels against their rooflines, each
    timed alone (pm_run, L2 flushed before every trial, median of `trials`;
    every footprint is larger than L2): the DG derivative on the tensor cores
    (dg_tc) and in its SIMT tile form (dg_tile) at Np = 20, 35, 56, 84 and
    Nel = 2^20, the stencil's best tile shape at n = 16384, the 256 x 256
    BF16 tensor-core matmul at n = 8192 and the best SIMT matmul tile
    (128 x 64 x 32) at n = 7680.  Bounds: HBM = the measured copy rate for every algorithmic
    byte (DG: 4 (4 Nel Np + 3 Np^2); stencil: 4 ((n + 2)(n + 4) + n^2));
    BF16 = the measured cuBLAS burst; TF32 = that x the nominal TF32 / BF16
    ratio 1.1 / 2.25, for the multiply-adds dg_tc issues (three passes over
    the padded product, from its counts); FP32 = SMs x 128 lanes x 2 x the
    sampled SM clock.  frac = the larger of the kernel's bound times over
    its median time."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    clk = (sm_mhz or 2070.0) * 1e6
    hbm = peaks["hbm_gbs"] * 1e9
    bf16 = peaks.get("bf16_tflops", 1900.0) * 1e12
    tf32 = bf16 * 1.1 / 2.25
    fp32 = sms * 128 * 2 * clk
    gen = torch.Generator(device=dev)
    gen.manual_seed(5)

    def buffers(kernel, p):
        out = []
        for b in pm.kernel_buffers(kernel, **p):
            n = int(b["elems"])
            if getattr(b["dtype"], "__name__", "") == "uint16":   # bf16 bit patterns
                x = (torch.rand(n, device=dev, generator=gen) * 2 - 1).to(torch.bfloat16).view(torch.int16)
            else:
                x = torch.rand(n, device=dev, generator=gen) * 2 - 1
            out.append(x)
        return out

    def timed(kernel, p):
        bufs = buffers(kernel, p)
        tm = pm.run(kernel, bufs, warmup=3, trials=trials, flush_l2=True, **p)
        del bufs
        return tm["median_ms"] * 1e-3

    out = {}
    nel = 1 << 20
    for np_ in (20, 35, 56, 84):
        bts = 4.0 * (4 * nel * np_ + 3 * np_ * np_)
        fl = 6.0 * nel * np_ * np_
        for k in ("dg_tc", "dg_tile"):
            p = dict(Np=np_, Nel=nel)
            s = timed(k, p)
            rec = {"ms": round(s * 1e3, 4), "GB/s": round(bts / s / 1e9, 1), "TFLOP/s": round(fl / s / 1e12, 2),
                   "hbm_frac": round(bts / s / hbm, 3)}
            if k == "dg_tc":
                mm = sum(r["count_wi"] for r in pm.counts(k, **p) if r["kind"] == "op" and r["dtype"] == "tfloat32")
                t_tc = 2.0 * mm / tf32
                rec["tf32_bound_ms"] = round(t_tc * 1e3, 4)
                rec["bound"] = "hbm" if bts / hbm >= t_tc else "tf32"
                rec["frac"] = round(max(bts / hbm, t_tc) / s, 3)
            else:
                rec["fp32_frac"] = round(fl / s / fp32, 3)
                rec["bound"] = "hbm" if bts / hbm >= fl / fp32 else "fp32"
                rec["frac"] = round(max(bts / hbm, fl / fp32) / s, 3)
            out["%s_Np%d" % (k, np_)] = rec
    n = 16384
    p = dict(n=n, BX=32, BY=16, V=8)
    s = timed("fd_block", p)
    bts = 4.0 * ((n + 2) * (n + 4) + n * n)
    out["fd_block_32x16_v8"] = {"ms": round(s * 1e3, 4), "GB/s": round(bts / s / 1e9, 1), "bound": "hbm",
                                "frac": round(bts / s / hbm, 3)}
    n = 8192
    s = timed("mm_tc256", dict(n=n))
    out["mm_tc256"] = {"ms": round(s * 1e3, 4), "TFLOP/s": round(2.0 * n ** 3 / s / 1e12, 1), "bound": "bf16",
                       "frac": round(2.0 * n ** 3 / s / bf16, 3)}
    n = 7680
    p = dict(n=n, BM=128, BN=64, BK=32)
    s = timed("mm_simt", p)
    out["mm_simt_128x64x32"] = {"ms": round(s * 1e3, 4), "TFLOP/s": round(2.0 * n ** 3 / s / 1e12, 2),
                                 "bound": "fp32", "frac": round(2.0 * n ** 3 / s / fp32, 3)}
    out["peaks"] = {"hbm_gbs": peaks["hbm_gbs"], "bf16_tflops": peaks.get("bf16_tflops"),
                    "tf32_tflops": round(tf32 / 1e12, 1), "fp32_tflops": round(fp32 / 1e12, 2), "sm_mhz": sm_mhz}
    return out


def accuracy_leg(trials=3):
    """Time-prediction accuracy per modeled variant (Section "Results": the
    geometric mean of the relative error), bounded to well under two
    minutes: the reduced cross-variant sweep -- the paper's eight modeled
    variants (two matmul, four DG, two stencil tiles), the direct stencil,
    the DG tile form and the two tensor-core tiles, each calibrated on the
    microbenchmarks, its computation's twins and every other of its own
    sizes, predicting the sizes held out (L2 flushed before every trial) --
    and the model-guided autotuner at reduced sizes (24 SIMT matmul tiles at
    n = 3840, 12 stencil tiles at n = 8192): predicted against measured
    order.  The prefetching matmul is also reported with the on-chip costs
    themselves overlapped (mm_pf_onchip_overlap, the same measurements)."""
    from paper_1904_09538_gb300 import autotune as A
    from paper_1904_09538_gb300 import experiments as E
    t0 = time.perf_counter()
    sweep = E.sweep_studies(reduced=True)
    mm_gm = [s for s in E.studies() if s["name"] == "matmul"][0]["gmem"]
    sweep.append(dict([s for s in sweep if s["name"] == "sweep_mm_pf"][0], name="sweep_mm_pf_onchip_overlap",
                      expr=E.overlap2(mm_gm)))
    rep = E.run_studies(trials=trials, study_list=sweep, flush_l2=True)
    by = {}
    for name, r in rep.items():
        if name == "sweep_tc_tiles":
            continue
        for v, e in r["variants"].items():
            if name == "sweep_mm_pf_onchip_overlap":
                v = "mm_pf_onchip_overlap"
            by[v] = {"geomean": round(e["geomean_rel_err"], 4), "max": round(e["max_rel_err"], 4),
                     "heldout": e["n_sizes"], "fit_status": r["fit"]["status"]}
    tcr = rep["sweep_tc_tiles"]
    t1 = time.perf_counter()
    tune = {}
    for fam, r in (("mm_simt", A.rank_family(target=3840, calib_sizes=(1536, 2304), trials=trials)),
                   ("fd_block", A.rank_stencil(target=8192, calib_sizes=(2048, 4096), trials=trials))):
        tune[fam] = {"target_n": r["target_n"], "variants": r["n_shapes"] - r["n_pruned"], "pruned": r["n_pruned"],
                     "spearman": round(r["spearman"], 3), "kendall": round(r["kendall"], 3),
                     "slowdown_of_predicted_best": round(r["slowdown_of_predicted_best"], 3),
                     "slowdown_top3": round(r["slowdown_after_timing_predicted_top_k"].get("3", float("nan")), 3)}
    return {"heldout_by_variant": by, "trials": trials,
            "tc_tiles_one_model": {"geomean": round(tcr["geomean_rel_err"], 4), "max": round(tcr["max_rel_err"], 4),
                                   "spearman": round(tcr["spearman"], 3),
                                   "faster_tile_identified": tcr["fastest_variant_identified"]},
            "autotune": tune, "sweep_s": round(t1 - t0, 1), "autotune_s": round(time.perf_counter() - t1, 1)}


def fit_vs_oracle(params, oracle_params):
    """max_i |p_i - p_i*| / |p_i*| per model against the oracle's FP64 fit of
    the same problem (the parameter bar of the calibration), worst over the
    64 models, for each GPU path."""
    import numpy as np
    out = {}
    for path, ps in params.items():
        errs = [float(np.max(np.abs(np.asarray(p) - po) / np.abs(po))) for p, po in zip(ps, oracle_params)]
        out[path] = {"max": max(errs), "median": float(np.median(errs)), "models": len(errs)}
    return out


def oracle_fit_rate(seconds=5.0):
    """The oracle's FP64 fits (SciPy Levenberg-Marquardt / least squares) on
    the same 64 calibration problems: on one host core, as many as fit in
    about `seconds`, and all 64 on every host core (a spawn-started process
    pool, one fit per task): fits per second, for context beside the GPU
    fits."""
    import multiprocessing as mp
    import platform
    import numpy as np
    import pm_inputs
    from oracle import fit as ofit
    from oracle.model import Model as OModel
    from paper_1904_09538_gb300.fitbench import TRUTH, features, model_expr
    oms = [OModel("f_wall_time", model_expr(k)) for k in range(64)]
    Xs, _ = features(64, lambda k: len(oms[k].features))
    jobs = []
    for k, om in enumerate(oms):
        # outputs by the oracle's own model evaluation (the GPU legs use
        # fitbench.synthetic_times, equal within 1e-14)
        F = [dict(zip(om.features, row)) for row in Xs[k]]
        t = np.array([om.eval(TRUTH, f) for f in F]) * (1 + 1e-2 * pm_inputs.noise((len(F),), 9900 + k))
        p0 = np.array([TRUTH[n] for n in om.params]) * 1.2
        jobs.append((om.expr, list(om.features), Xs[k], t, p0))
    done, t0 = 0, time.perf_counter()
    for job in jobs:
        ofit.fit_rows(job)
        done += 1
        if time.perf_counter() - t0 > seconds:
            break
    one = done / (time.perf_counter() - t0)
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        # start-up and imports untimed; every wait bounded
        pool.map_async(ofit.fit_rows, jobs[:cores], chunksize=1).get(timeout=300)
        t1 = time.perf_counter()
        res = pool.map_async(ofit.fit_rows, jobs, chunksize=1).get(timeout=300)
        n_all = len(res)
        allc = n_all / (time.perf_counter() - t1)
    return {"fits_per_s": round(one, 2), "fits": done, "cores": 1, "kind": "oracle",
            "all_cores": {"fits_per_s": round(allc, 2), "fits": n_all, "cores": cores,
                          "machine": platform.machine(), "cpu": cpu_model()},
            "_params": [p for p, _ in res]}


_CPU_INPUTS = {}


def cpu_baseline(variants, seconds=12.0, scale=16):
    """The oracle's plain CPU reference kernels on a bounded sample of the
    same suite: every stream variant at N/`scale` (arrays still larger than a
    host's last-level cache at the larger N), every arithmetic variant at
    1/(64 `scale`) of its work-items, each oracle call repeated until the pass
    costs about `seconds` of one host core.  Inputs are made once per array
    and kept across calls; only the oracle calls are timed."""
    import numpy as np
    import pm_inputs
    from oracle import refs

    def inp(n, seed, dt):
        key = (n, seed, np.dtype(dt).str)
        if key not in _CPU_INPUTS:
            _CPU_INPUTS[key] = pm_inputs.uniform((n,), seed, dtype=dt)
        return _CPU_INPUTS[key]

    def one_pass(vs, reps):
        total_b, total_t = 0, 0.0
        for k, p in vs:
            dt = np.float32 if p.get("dtype", 0) == 0 else np.float64
            if k == "stream":
                N = max(256, p["N"] // scale)
                xs = [inp(N, 5 + a, dt) for a in range(p.get("L", 1))]
                t1 = time.perf_counter()
                for _ in range(reps):
                    refs.stream(xs)
                total_t += time.perf_counter() - t1
                total_b += reps * (p.get("L", 1) + 1) * N * np.dtype(dt).itemsize
            elif k == "fma":
                T = max(256, p["G"] * 256 // (scale * 64))
                u = inp(T, 9, dt)
                t1 = time.perf_counter()
                for _ in range(reps):
                    refs.fma(u, p["op"], p["F"])
                total_t += time.perf_counter() - t1
                total_b += reps * 2 * T * np.dtype(dt).itemsize
        return total_b, total_t

    b, t = one_pass(variants, 1)
    reps = max(1, math.ceil(seconds / t)) if t > 0 else 1
    if reps > 1:
        b, t = one_pass(variants, reps)
    # the same calls spread over a thread pool of every host core (the C
    # reference runs with the GIL released): wall time of the whole pass
    from concurrent.futures import ThreadPoolExecutor
    cores = os.cpu_count() or 1
    t1 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        ba = sum(ex.map(lambda kp: one_pass([kp], reps)[0], variants))
    ta = time.perf_counter() - t1
    return {"value": round(b / t / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle", "cpu": cpu_model(),
            "sample": "every stream variant at N/%d and every arithmetic variant at 1/%d of its work-items, "
                      "each oracle call %d times (oracle C reference, one host core, %.1f s)"
                      % (scale, scale * 64, reps, t),
            "all_cores": {"value": round(ba / ta / 1e9, 3), "cores": cores,
                          "sample": "the same calls over a %d-thread pool, %.1f s wall" % (cores, ta)}}


def cpu_model():
    """The host CPU's model name (lscpu's "Model name", else /proc/cpuinfo's
    "model name", else the machine type)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1904_09538_gb300 import suite as S
    variants = S.generate(args.filter.split(","))
    for _ in range(args.warmup):
        cpu_baseline(variants, seconds=2.0)
    vals = []
    t0 = time.perf_counter()
    last = None
    for _ in range(args.steps):
        last = cpu_baseline(variants, seconds=6.0)
        vals.append(last["value"])
    el = time.perf_counter() - t0
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
            "config": workload_config(variants, args.trials),
            "cpu_baseline": {"value": v, "unit": "GB/s", "cores": 1, "kind": "oracle", "cpu": last["cpu"],
                             "sample": last["sample"], "all_cores": last["all_cores"]},
            "e2e": {"value": v, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
