"""Tie the counts to the compiled kernels (Algorithm 1 counts the kernel's own
program; here the counts are closed forms written beside hand-written CUDA,
so they are checked against what the GPU executed).

  python -m paper_1904_09538_gb300.countcheck launch
      launches every instance of INSTANCES once on cuda:0 (run it under ncu
      with the METRICS below to collect executed-instruction counters);
  python -m paper_1904_09538_gb300.countcheck table LAUNCHES.csv
      prints, per instance, the counters beside what pm_counts implies.

Expected values from the feature records: executed warp-level global load /
store instructions with at least one lane active = the sub-group count of
the global load / store records (one instruction per access, 16-byte
vectors included); shared-memory load / store instructions = the sub-group
count of the local records; thread-level FP32 multiply-adds = the madd
work-item count (an FFMA2 instruction does two), adds and multiplies
likewise; CTAs = the work-group count.  No counter isolates barrier
instructions, so barriers are not compared."""
import csv
import json
import sys

import numpy as np

from . import counts, kernel_buffers, launch

INSTANCES = [
    ("stream", dict(N=1 << 16, s=1, L=1)), ("stream", dict(N=1 << 16, s=4, L=2)),
    ("stream", dict(N=1 << 16, s=1, L=3, vec=1)), ("stream", dict(N=1 << 16, s=8, L=1, dtype=1, vec=1)),
    ("stream", dict(N=1 << 16, shape=1, W=256, L=2)),
    ("fma", dict(F=1024, G=8, op=2)), ("fma", dict(F=1024, G=8, op=0)), ("fma", dict(F=1024, G=8, op=1)),
    ("fma", dict(F=1024, G=8, op=2, dtype=1)),
    ("smem", dict(R=256, G=8)), ("smem", dict(R=256, G=8, sync=1)), ("barrier", dict(B=64, G=8)),
    ("overlap", dict(m=4, N=1 << 16)), ("empty", dict(G=64)), ("smem2d", dict(R=256, T=16, G=8)),
    ("mm_pf", dict(n=128)), ("mm_nopf", dict(n=128)), ("mm_pf_a", dict(n=128)), ("mm_pf_b", dict(n=128)),
    ("mm_nopf_a", dict(n=128)), ("mm_nopf_b", dict(n=128)),
    ("dg_nopf", dict(Np=35, Nel=256)), ("dg_dmpf", dict(Np=35, Nel=256)), ("dg_upf", dict(Np=35, Nel=256)),
    ("dg_dmpft", dict(Np=35, Nel=256)), ("dg_nopf", dict(Np=35, Nel=256, L0=32, L1=8)),
    ("dg_nopf_u", dict(Np=35, Nel=256)), ("dg_nopf_dm", dict(Np=35, Nel=256)), ("dg_dmpf_u", dict(Np=35, Nel=256)),
    ("dg_dmpf_dm", dict(Np=35, Nel=256)), ("dg_res", dict(Np=35, Nel=256)), ("dg_upf_u", dict(Np=35, Nel=256)),
    ("dg_dmpft_u", dict(Np=35, Nel=256)), ("dg_dmpft_res", dict(Np=35, Nel=256)),
    ("dg_tile", dict(Np=35, Nel=256)), ("dg_tile", dict(Np=20, Nel=256)),
    ("dg_tc", dict(Np=20, Nel=256)), ("dg_tc", dict(Np=35, Nel=256)), ("dg_tc", dict(Np=35, Nel=256, A=0)),
    ("dg_tc", dict(Np=84, Nel=256, A=0)), ("dg_tc", dict(Np=84, Nel=256)),
    ("fd_tile", dict(n=45)), ("fd_tile18", dict(n=45)), ("fd_direct", dict(n=45)),
    ("fd_tile_u", dict(n=45)), ("fd_tile_res", dict(n=45)), ("fd_direct_u", dict(n=45)),
    ("fd_direct_res", dict(n=45)), ("fd_tile18_u", dict(n=45)), ("fd_tile18_res", dict(n=45)),
    ("fd_block", dict(n=128, BX=64, BY=8)), ("fd_block", dict(n=128, BX=32, BY=16, V=8)),
    ("mm_simt", dict(n=768, BM=128, BN=128, BK=32)), ("mm_tc", dict(n=512)), ("mm_tc256", dict(n=512)),
]

METRICS = ["launch__grid_size", "launch__block_size",
           "smsp__inst_executed_op_global_ld_pred_on_any.sum", "smsp__inst_executed_op_global_st_pred_on_any.sum",
           "smsp__inst_executed_op_shared_ld_pred_on_any.sum", "smsp__inst_executed_op_shared_st_pred_on_any.sum",
           "smsp__inst_executed_op_tma_ld.sum", "smsp__inst_executed_op_ldgsts.sum",
           "smsp__sass_thread_inst_executed_op_ffma_pred_on.sum", "smsp__sass_thread_inst_executed_op_ffma2_pred_on.sum",
           "smsp__sass_thread_inst_executed_op_fadd_pred_on.sum", "smsp__sass_thread_inst_executed_op_fadd2_pred_on.sum",
           "smsp__sass_thread_inst_executed_op_fmul_pred_on.sum", "smsp__sass_thread_inst_executed_op_fmul2_pred_on.sum",
           "smsp__sass_thread_inst_executed_op_dfma_pred_on.sum"]


def expected(kernel, params):
    """What the feature records of kernel(params) imply for the counters."""
    e = dict(gld=0, gst=0, sld=0, sst=0, ffma=0, fadd=0, fmul=0, dfma=0, ctas=0)
    for r in counts(kernel, **params):
        if r["kind"] == "mem":
            key = ("g" if r["mem"] == "global" else "s") + ("ld" if r["dir"] == "load" else "st")
            e[key] += r["count_sg"]
        elif r["kind"] == "op":
            if r["dtype"] == "float32":
                e[{"madd": "ffma", "add": "fadd", "mul": "fmul"}[r["op"]]] += r["count_wi"]
            elif r["dtype"] == "float64" and r["op"] == "madd":
                e["dfma"] += r["count_wi"]
        elif r["kind"] == "groups":
            e["ctas"] = r["count"]
    return e


def launch_all():
    import torch
    dev = torch.device("cuda:0")
    gen = torch.Generator(device=dev)
    gen.manual_seed(7)
    for kernel, params in INSTANCES:
        bufs = []
        for b in kernel_buffers(kernel, **params):
            n = int(b["elems"])
            if b["dtype"] == np.uint16:
                x = (torch.randint(0, 1 << 14, (n,), device=dev, generator=gen, dtype=torch.int32) + 0x3800).to(torch.int16)
            elif b["dtype"] == np.float64:
                x = torch.rand(n, device=dev, generator=gen, dtype=torch.float64) * 2 - 1
            else:
                x = torch.rand(n, device=dev, generator=gen) * 2 - 1
            bufs.append(x)
        launch(kernel, bufs, **params)
        torch.cuda.synchronize()
    print(json.dumps({"launched": len(INSTANCES)}))


def measured(path):
    """Per launch (in order) the metric values of an ncu --csv log."""
    rows = {}
    with open(path) as f:
        lines = [l for l in f if l.startswith('"')]
    for r in csv.DictReader(lines):
        i = int(r["ID"])
        v = r["Metric Value"].replace(",", "")
        try:
            rows.setdefault(i, {"name": r["Kernel Name"]})[r["Metric Name"]] = float(v)
        except ValueError:
            rows.setdefault(i, {"name": r["Kernel Name"]})[r["Metric Name"]] = v
    return [rows[i] for i in sorted(rows)]


def table(path):
    got = [g for g in measured(path) if "pm::" in g["name"]]   # the library's kernels, not torch's fills
    if len(got) != len(INSTANCES):
        raise SystemExit("%d launches in %s, %d instances" % (len(got), path, len(INSTANCES)))
    out = ["| kernel | params | CTAs cnt/exe | global ld cnt/exe | global st cnt/exe | shared ld cnt/exe | "
           "shared st cnt/exe | FP32 fma cnt/exe | add cnt/exe | mul cnt/exe | TMA ld |", "|" + "---|" * 11]
    for (kernel, params), g in zip(INSTANCES, got):
        e = expected(kernel, params)
        m = lambda k: int(g.get(k, 0) or 0)
        exe = dict(ctas=m("launch__grid_size"), gld=m("smsp__inst_executed_op_global_ld_pred_on_any.sum"),
                   gst=m("smsp__inst_executed_op_global_st_pred_on_any.sum"),
                   sld=m("smsp__inst_executed_op_shared_ld_pred_on_any.sum"),
                   sst=m("smsp__inst_executed_op_shared_st_pred_on_any.sum"),
                   ffma=m("smsp__sass_thread_inst_executed_op_ffma_pred_on.sum")
                   + 2 * m("smsp__sass_thread_inst_executed_op_ffma2_pred_on.sum")
                   + m("smsp__sass_thread_inst_executed_op_dfma_pred_on.sum"),
                   fadd=m("smsp__sass_thread_inst_executed_op_fadd_pred_on.sum")
                   + 2 * m("smsp__sass_thread_inst_executed_op_fadd2_pred_on.sum"),
                   fmul=m("smsp__sass_thread_inst_executed_op_fmul_pred_on.sum")
                   + 2 * m("smsp__sass_thread_inst_executed_op_fmul2_pred_on.sum"))
        e = dict(e, ffma=e["ffma"] + e["dfma"])

        def cell(k):
            return "%d / %d%s" % (e[k], exe[k], "" if e[k] == exe[k] else " **≠**")
        out.append("| %s | %s | %s | %s | %s | %s | %s | %s | %s | %s | %d |" % (
            kernel, ",".join("%s=%s" % kv for kv in params.items()), cell("ctas"), cell("gld"), cell("gst"),
            cell("sld"), cell("sst"), cell("ffma"), cell("fadd"), cell("fmul"), m("smsp__inst_executed_op_tma_ld.sum")))
    return "\n".join(out)


if __name__ == "__main__":
    if sys.argv[1:2] == ["launch"]:
        launch_all()
    elif sys.argv[1:2] == ["table"]:
        print(table(sys.argv[2]))
    else:
        raise SystemExit(__doc__)
