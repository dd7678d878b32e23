"""Measurement-kernel collection (Section "Parameterized Collection of
Kernels"): generators carry generator tags and, per argument, a list of
allowed values; a generator emits one kernel variant per element of the
Cartesian product of its argument lists.  Filter tags select generators
(match condition identical / subset / superset (default) / intersect) and
restrict argument values ("arg:v1,v2").

The default collection is the calibration suite of the GB300 build: stream
(global memory patterns), arithmetic loops, local-memory shuffle with and
without per-iteration barriers, barrier, local/global overlap and empty
kernels, plus the modeled computations and their work-removed twins.
"""
import itertools

IDENTICAL, SUBSET, SUPERSET, INTERSECT = "identical", "subset", "superset", "intersect"

SM_COUNT = 152
RESIDENT = 8 * SM_COUNT   # 256-thread work-groups resident at full occupancy
FMA_F32_PER_SM = 6        # k_fma<float> holds 32 accumulators: 37-39 registers -> 6 CTAs of 256 per SM
FMA_F64_PER_SM = 3        # k_fma<double>: 70-72 registers -> 3 CTAs of 256 per SM
L2_BYTES = 129 * 10 ** 6


class Generator:
    def __init__(self, kernel, tags, args, derive=None):
        self.kernel = kernel
        self.tags = set(tags)
        self.args = {k: list(v) for k, v in args.items()}
        self.derive = derive

    def variants(self, restrict):
        lists = []
        for k, vals in self.args.items():
            if k in restrict:
                allowed = [v for v in vals if v in restrict[k]]
                lists.append(allowed)
            else:
                lists.append(vals)
        out = []
        for combo in itertools.product(*lists):
            p = dict(zip(self.args, combo))
            if self.derive:
                p = self.derive(p)
                if p is None:
                    continue
            out.append((self.kernel, p))
        return out


def _half_on_odd(x):
    # 1 for even powers of two, 1/2 for odd ones: neighbouring variants then
    # differ in total work as well as in its split into work-groups, so the
    # per-operation and per-work-group costs are separately identifiable
    return 2 if (x.bit_length() - 1) % 2 else 1


def _fma_groups(p):
    # total work per dtype ~2^16 * 256 * RESIDENT operations for float32
    # (halved on every other F), 1/64 of that for float64 (GB300's FP64 rate
    # is far lower).  float32 grids are whole waves of FMA_F32_PER_SM CTAs per
    # SM: a last round of 2-4 CTAs per SM is placed unevenly across the SMs
    # and runs up to 25 % longer than its share of the work, which no count
    # feature sees.  The float64 loop saturates its pipe at one CTA per SM, so
    # below one wave it runs whole CTAs per SM.
    F = p["F"]
    p = dict(p)
    if p["dtype"] == 0:
        wave = FMA_F32_PER_SM * SM_COUNT
        p["G"] = wave * max(1, round((1 << 16) * RESIDENT / F / _half_on_odd(F) / wave))
    else:
        wave = FMA_F64_PER_SM * SM_COUNT
        g = (1 << 10) * RESIDENT / F / _half_on_odd(F)
        p["G"] = wave * round(g / wave) if g >= wave else SM_COUNT * max(1, round(g / SM_COUNT))
    return p


def _smem_groups(p):
    p = dict(p)
    p["G"] = max(SM_COUNT, RESIDENT * (1 << 14) // p["R"] // _half_on_odd(p["R"]))
    return p


def _barrier_groups(p):
    # B runs over even powers of two: alternate one and two full waves of
    # work-groups so the launch and per-work-group costs separate (a partial
    # wave would change the per-barrier cost: fewer resident groups hide
    # less of each barrier's latency)
    p = dict(p)
    e = p["B"].bit_length() - 1
    p["G"] = RESIDENT * (1 + (e // 2) % 2)
    return p


def _overlap_size(p):
    # alternate the global footprint with m (2^26 and 2^27 floats per array,
    # both above the L2 size) so the global and local costs are not both
    # fixed multiples of the launch
    p = dict(p)
    p["N"] = (1 << 26) * (1 + _OVERLAP_M.index(p["m"]) % 2)
    return p


_OVERLAP_M = [0, 1, 2, 4, 8, 12, 16, 24, 32]


def _smem2d_groups(p):
    # the 1-D kernel's sizing: R x G constant, at least one work-group per SM
    p = dict(p)
    p["G"] = max(SM_COUNT, RESIDENT * (1 << 14) // p["R"])
    return p


def _stream_extra(p):
    # L in {2, 3} only at stride 1
    if p["L"] in (2, 3) and p["s"] != 1:
        return None
    return p


POW = lambda lo, hi, step=1: [1 << e for e in range(lo, hi + 1, step)]  # noqa: E731

GENERATORS = [
    Generator("stream", ["gmem", "stream", "suite"],
              {"dtype": [0, 1], "vec": [1], "N": POW(20, 28, 2), "s": [1, 2, 4, 8, 16, 32], "L": [1, 2, 3, 4],
               "shape": [0]}, _stream_extra),
    Generator("stream", ["gmem", "stream2d", "suite"],
              {"dtype": [0], "vec": [0], "N": POW(20, 28, 2), "L": [1, 2, 3, 4], "shape": [1], "W": [2048]}),
    Generator("fma", ["ops", "flops_pattern", "suite"],
              {"dtype": [0], "op": [0, 1, 2], "F": POW(10, 16)}, _fma_groups),
    Generator("fma", ["ops", "flops_pattern", "fp64", "suite"],
              {"dtype": [1], "op": [2], "F": POW(10, 16)}, _fma_groups),
    Generator("smem", ["lmem", "suite"], {"R": POW(8, 14), "sync": [0, 1]}, _smem_groups),
    Generator("barrier", ["sync", "suite"], {"B": POW(4, 14, 2)}, _barrier_groups),
    Generator("smem2d", ["lmem2d"], {"R": POW(8, 14), "T": [16, 18]}, _smem2d_groups),
    Generator("overlap", ["overlap", "suite"], {"m": _OVERLAP_M}, _overlap_size),
    Generator("empty", ["launch", "suite"], {"G": POW(6, 18)}),
    Generator("mm_pf", ["matmul_sq", "modeled"], {"n": [256, 384, 512, 640, 768, 896]}),
    Generator("mm_nopf", ["matmul_sq", "modeled"], {"n": [256, 384, 512, 640, 768, 896]}),
    Generator("dg_nopf", ["dg", "modeled"], {"Np": [20, 35, 56, 84], "Nel": POW(14, 18), "L0": [16, 32]},
              lambda p: dict(p, L1=256 // p["L0"])),
    Generator("dg_dmpf", ["dg", "modeled"], {"Np": [20, 35, 56, 84], "Nel": POW(14, 18), "L0": [16, 32]},
              lambda p: dict(p, L1=256 // p["L0"])),
    Generator("dg_upf", ["dg", "modeled"], {"Np": [20, 35, 56, 84], "Nel": POW(14, 18), "L0": [16]},
              lambda p: dict(p, L1=16)),
    Generator("dg_dmpft", ["dg", "modeled"], {"Np": [20, 35, 56, 84], "Nel": POW(14, 18), "L0": [16, 32]},
              lambda p: dict(p, L1=256 // p["L0"])),
    Generator("dg_tile", ["dg", "modeled", "dg_tile"], {"Np": [20, 35, 56, 84], "Nel": POW(14, 18)}),
    Generator("dg_tc", ["dg", "modeled", "dg_tc"], {"Np": [20, 35, 56, 84], "Nel": POW(14, 18)}),
    Generator("fd_tile", ["finite_diff", "modeled"], {"n": POW(10, 14)}),
    Generator("fd_tile18", ["finite_diff", "modeled"], {"n": POW(10, 14)}),
    Generator("fd_direct", ["finite_diff", "modeled"], {"n": POW(10, 14)}),
    Generator("mm_tc", ["matmul_tc", "modeled"], {"n": POW(10, 14)}),
    Generator("mm_tc256", ["matmul_tc", "modeled"], {"n": POW(10, 14)}),
    Generator("mm_simt", ["matmul_tiles", "autotune"],
              {"n": [7680], "BM": [64, 96, 128, 256], "BN": [64, 128, 256], "BK": [32, 64]}),
    Generator("fd_block", ["stencil_tiles", "autotune"], {"n": [16384], "BX": [32, 64, 128], "BY": [4, 8, 16, 32]}),
]


def parse_filter(tags):
    gen_tags, restrict = set(), {}
    for t in tags:
        if ":" in t:
            k, vals = t.split(":", 1)
            restrict[k] = [int(v) for v in vals.split(",")]
        else:
            gen_tags.add(t)
    return gen_tags, restrict


def generate(tags, match=SUPERSET, generators=None):
    """Kernel variants [(kernel, params)] for filter tags."""
    gen_tags, restrict = parse_filter(tags)
    out = []
    for g in generators or GENERATORS:
        if match == IDENTICAL:
            ok = g.tags == gen_tags
        elif match == SUBSET:
            ok = g.tags <= gen_tags
        elif match == SUPERSET:
            ok = g.tags >= gen_tags
        else:
            ok = bool(g.tags & gen_tags)
        if ok:
            out.extend(g.variants(restrict))
    return out


def calibration_suite():
    return generate(["suite"])


def cache_resident(kernel, p):
    """Stream variants whose footprint is below twice the L2 size: repeated
    trials would find their arrays in L2, so they are timed from a flushed L2
    (the features count DRAM-bound accesses)."""
    return kernel == "stream" and algorithmic_bytes(kernel, p) < 2 * L2_BYTES


def algorithmic_bytes(kernel, p):
    """Bytes a launch must move to/from global memory by its definition."""
    if kernel == "stream":
        size = 4 if p.get("dtype", 0) == 0 else 8
        return (p.get("L", 1) + 1) * p["N"] * size
    if kernel == "fma":
        return 2 * p["G"] * 256 * (4 if p.get("dtype", 0) == 0 else 8)
    if kernel in ("smem", "barrier"):
        return 2 * p["G"] * 256 * 4
    if kernel == "overlap":
        return 2 * p["N"] * 4
    return 0


# ---------------------------------------------------------------- calibration models
LAUNCH = "p_launch * f_sync_kernel_launch + p_group * f_thread_groups"


def family_key(kernel, p):
    """Which calibration model a suite variant belongs to."""
    if kernel == "stream":
        if p.get("shape", 0) == 1:
            return "stream2d_f32"
        return "stream_%s_s%d" % ("f32" if p["dtype"] == 0 else "f64", p["s"])
    if kernel == "fma":
        return "fma_%s_%s" % ("f32" if p["dtype"] == 0 else "f64", ("add", "mul", "madd")[p["op"]])
    if kernel == "smem":
        return "smem_sync%d" % p["sync"]
    return kernel


def overlap_model(partial=True):
    """Model of the local/global overlap kernel (Section "Modeling Operation
    Overlap"): launch cost plus the tanh-weighted larger of the global and
    local costs (Eq. overlap_differentiable).  With partial=True the
    tanh-weighted smaller of the two is added with weight p_part, one of the
    variations with an extra parameter that the section proposes for partial
    overlap (p_part = 0: the smaller cost hidden entirely, 1: not at all)."""
    cg = "(p_gmem * f_mem_access_global_float32)"
    co = "(p_lmem * f_mem_access_local_float32)"
    sw = "%s * (tanh(p_edge * (%s - %s)) + 1) / 2 + %s * (tanh(p_edge * (%s - %s)) + 1) / 2"
    expr = "p_launch * f_sync_kernel_launch + " + sw % (cg, cg, co, co, co, cg)
    if partial:
        expr += " + p_part * (%s)" % (sw % (cg, co, cg, co, cg, co))
    return expr


def family_model(key):
    """(output feature, expression) of each family's model: the linear model
    of Section "Models Demonstrated" restricted to the family's features, and
    the partial-overlap variant of the tanh overlap model for the overlap
    kernel."""
    if key.startswith("stream"):
        return LAUNCH + " + p_gmem * f_mem_access_global"
    if key.startswith("fma"):
        # the mul / madd loops end in a reduction of a fixed number of adds
        # per work-group: that cost is part of p_group, not a separate term
        dt = "float32" if "_f32_" in key else "float64"
        op = key.rsplit("_", 1)[1]
        return LAUNCH + " + p_%s * f_op_%s_%s" % (op, dt, op)
    if key == "smem_sync0":
        return LAUNCH + " + p_lmem * f_mem_access_local_float32"
    if key == "smem_sync1":
        # one barrier per fixed number of local accesses: the barrier cost is
        # folded into p_lmem (the barrier kernel calibrates p_bar on its own)
        return LAUNCH + " + p_lmem * f_mem_access_local_float32"
    if key == "barrier":
        return LAUNCH + " + p_bar * f_sync_barrier_local * f_thread_groups"
    if key == "overlap":
        return overlap_model(partial=True)
    if key == "empty":
        return LAUNCH
    raise KeyError(key)
