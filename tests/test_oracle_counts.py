"""Pins of the oracle's brute-force counting against what the paper and the
mathematics fix (closed forms, worked examples, Table 'ab_pattern',
coverage invariants).  CPU only."""
import json
import os

import pytest

import oracle
from oracle.features import features, feature_value, parse_feature, matches
from oracle.quasipoly import extrapolate

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))


def by_tag(fs, tag):
    out = [f for f in fs if f["kind"] == "mem" and f["tag"] == tag]
    assert len(out) == 1, (tag, [f["name"] for f in fs])
    return out[0]


def op(fs, dtype, o, wi=False):
    for f in fs:
        if f["kind"] == "op" and f["dtype"] == dtype and f["op"] == o:
            return f["count_wi"] if wi else f["count"]
    return 0


def single(fs, kind):
    return [f for f in fs if f["kind"] == kind][0]["count"]


def test_worked_count_example():
    # Section "Gathering Kernel Statistics": |{p<=i<n, p<=j<i+1}| = (n^2+p^2-2np+n-p)/2
    for n in range(0, 41):
        for p in range(0, n + 1):
            assert 2 * oracle.count_example(n, p) == n * n + p * p - 2 * n * p + n - p


@pytest.mark.parametrize("n", [16, 32, 48, 64])
def test_mm_pf_closed_forms(n):
    fs = features("mm_pf", n=n)
    assert op(fs, "float32", "madd", wi=True) == n ** 3           # 2n^3 flops
    assert op(fs, "float32", "madd") == n ** 3 // 32               # per sub-group
    a, b = by_tag(fs, "mm-PF-a"), by_tag(fs, "mm-PF-b")
    assert a["count"] == b["count"] == n ** 3 // 16 and a["gran"] == "WI"
    # Table ab_pattern
    assert a["lstr"] == (1, n) and a["gstr"] == (0, 16 * n) and a["loopstr"] == 16
    assert b["lstr"] == (1, n) and b["gstr"] == (16, 0) and b["loopstr"] == 16 * n
    assert a["accesses"] * 16 == n * a["footprint"] and b["accesses"] * 16 == n * b["footprint"]  # AFR n/16
    # Section "Matrix Multiplication": 2n^3 local loads, 2n^3/16 local stores
    loc = [f for f in fs if f["kind"] == "mem" and f["mem"] == "local"]
    assert sum(f["count_wi"] for f in loc if f["dir"] == "load") == 2 * n ** 3
    assert sum(f["count_wi"] for f in loc if f["dir"] == "store") == 2 * n ** 3 // 16
    c = by_tag(fs, "c")
    assert c["count"] == c["footprint"] == n * n
    assert single(fs, "sync") == n // 8
    assert single(fs, "groups") == n * n // 256
    assert single(fs, "launch") == 1


@pytest.mark.parametrize("n", [16, 32, 48])
def test_mm_nopf_closed_forms(n):
    fs = features("mm_nopf", n=n)
    a, b = by_tag(fs, "mm-noPF-a"), by_tag(fs, "mm-noPF-b")
    # lid(0) stride 0: uniform, counted once per sub-group (Table mm_param_vals, MCG SG)
    assert a["lstr"][0] == 0 and a["gran"] == "SG" and a["count"] == n ** 3 // 32
    assert b["gran"] == "WI" and b["count"] == n ** 3
    # 16x fewer global loads with prefetching (Section "Matrix Multiplication")
    pf = features("mm_pf", n=n)
    assert by_tag(pf, "mm-PF-a")["count_wi"] * 16 == a["count_wi"]
    assert single(fs, "sync") == 0
    assert op(fs, "float32", "madd", wi=True) == n ** 3


def test_mm_counts_at_paper_sizes_by_interpolation():
    # Counts are polynomials in n on the class n = 0 mod 16; brute force at
    # n = 16..80 fixes them exactly; compare with the closed forms at the
    # configuration sizes.
    def cnt(n, what):
        fs = features("mm_pf", n=n)
        return {"madd": op(fs, "float32", "madd", wi=True),
                "gld": by_tag(fs, "mm-PF-a")["count"] + by_tag(fs, "mm-PF-b")["count"],
                "gst": by_tag(fs, "c")["count"], "wg": single(fs, "groups"), "bar": single(fs, "sync")}[what]
    cache = {}

    def f(what):
        def g(n):
            key = (n, what)
            if key not in cache:
                cache[key] = cnt(n, what)
            return cache[key]
        return g
    for n in (256, 768, 896):
        assert extrapolate(f("madd"), n, 16, 3, 16) == n ** 3
        assert extrapolate(f("gld"), n, 16, 3, 16) == n ** 3 // 8
        assert extrapolate(f("gst"), n, 16, 2, 16) == n ** 2
        assert extrapolate(f("wg"), n, 16, 2, 16) == n ** 2 // 256
        assert extrapolate(f("bar"), n, 16, 1, 16) == n // 8


def test_paper_constraint_features_select_a_and_b():
    # Section "Data Motion Features": pattern-based features pick the a and b loads
    n = 48
    fs = features("mm_pf", n=n)
    fa = "f_mem_access_global_float32_load_lstrides:{0:1;1:>15}_gstrides:{0:0}_afr:>1"
    fb = "f_mem_access_global_float32_load_lstrides:{0:1;1:>15}_gstrides:{0:16}_afr:>1"
    assert feature_value(fa, fs) == by_tag(fs, "mm-PF-a")["count"]
    assert feature_value(fb, fs) == by_tag(fs, "mm-PF-b")["count"]
    assert [f["tag"] for f in fs if f["kind"] == "mem" and matches(parse_feature(fa), f)] == ["mm-PF-a"]
    assert feature_value("f_mem_access_tag:mm-PF-a", fs) == n ** 3 // 16
    assert feature_value("f_mem_access_local_float32", fs) == (2 * n ** 3 + 2 * n ** 3 // 16) // 32
    assert feature_value("f_op_float32_madd", fs) == n ** 3 // 32
    with pytest.raises(ValueError):
        parse_feature("f_mem_access_float32_global")     # fields out of order


@pytest.mark.parametrize("kernel,tag,loads_per_wi", [
    ("mm_pf_a", "mm-PF-a", lambda n: n // 16), ("mm_pf_b", "mm-PF-b", lambda n: n // 16),
    ("mm_nopf_a", "mm-noPF-a", lambda n: n), ("mm_nopf_b", "mm-noPF-b", lambda n: n)])
def test_mm_twins_keep_parent_pattern(kernel, tag, loads_per_wi):
    # Algorithm 3: the kept load keeps its pattern; one add per kept load; a
    # per-work-item store of tgt is added.
    n = 32
    parent = features("mm_pf" if "_pf_" in kernel else "mm_nopf", n=n)
    twin = features(kernel, n=n)
    p, t = by_tag(parent, tag), by_tag(twin, tag)
    for key in ("lstr", "gstr", "loopstr", "count", "gran", "footprint", "accesses"):
        assert p[key] == t[key], key
    assert op(twin, "float32", "add", wi=True) == n * n * loads_per_wi(n)
    dest = by_tag(twin, "tgt_dest")
    assert dest["count"] == dest["footprint"] == n * n
    assert single(twin, "sync") == 0


@pytest.mark.parametrize("Np,Nel,L0,L1", [(20, 32, 16, 16), (35, 64, 32, 8), (32, 32, 16, 16), (56, 32, 32, 8)])
def test_dg_closed_forms(Np, Nel, L0, L1):
    sh = "%dx%d" % (L0, L1)
    for v in ("dg_nopf", "dg_dmpf"):
        fs = features(v, Np=Np, Nel=Nel, L0=L0, L1=L1)
        assert op(fs, "float32", "madd", wi=True) == 3 * Nel * Np * Np    # 6 Nel Np^2 flops
        res = by_tag(fs, "dg-res-" + sh)
        assert res["count"] == res["footprint"] == 3 * Nel * Np              # every output once
        pre = "dg-noPF" if v == "dg_nopf" else "dg-dmPF"
        u = by_tag(fs, pre + "-u-" + sh)
        assert u["count_wi"] == 3 * Nel * Np * Np and u["footprint"] == Nel * Np
        assert u["lstr"] == (Np, 0) and u["gstr"][0] == L0 * Np
        d = by_tag(fs, pre + "-dm-" + sh)
        assert d["footprint"] == 3 * Np * Np
        if v == "dg_nopf":
            assert d["lstr"][0] == 0 and d["gran"] == "SG" and d["count_wi"] == 3 * Nel * Np * Np
            assert single(fs, "sync") == 0
            if Np % (2 * 32 // L0) == 0:   # sub-groups all full
                assert d["count"] == d["count_wi"] // 32
        else:
            # each D element fetched once per k-tile: AFR = Nel / L0
            assert d["count_wi"] == 3 * Np * Np * (Nel // L0)
            assert single(fs, "sync") == 2 * 3 * (-(-Np // L0))
            loc = [f for f in fs if f["kind"] == "mem" and f["mem"] == "local"]
            assert sum(f["count_wi"] for f in loc if f["dir"] == "load") == 3 * Nel * Np * Np
            assert sum(f["count_wi"] for f in loc if f["dir"] == "store") == 3 * Np * Np * (Nel // L0)
        assert single(fs, "groups") == (Nel // L0) * (-(-Np // L1))


@pytest.mark.parametrize("Np,Nel,L0,L1", [(20, 64, 16, 16), (35, 32, 16, 16), (84, 32, 16, 16), (7, 16, 16, 16)])
def test_dg_upf_closed_forms(Np, Nel, L0, L1):
    # uPF (Section "DG"): j split by lsize1, u tile prefetched per j tile,
    # loops j tile -> j -> m with one accumulator per m
    fs = features("dg_upf", Np=Np, Nel=Nel, L0=L0, L1=L1)
    G1 = -(-Np // L1)
    assert op(fs, "float32", "madd", wi=True) == 3 * Nel * Np * Np
    u = by_tag(fs, "dg-uPF-u-16x16")
    # every u element fetched once per i-group, lid(0) runs along j (stride 1)
    assert u["count_wi"] == G1 * Nel * Np and u["footprint"] == Nel * Np
    assert u["lstr"] == (1, Np) and u["gstr"] == (L0 * Np, 0) and u["loopstr"] == L1
    d = by_tag(fs, "dg-noPF-dm-16x16")     # same pattern as noPF's D, shared twin
    assert d["lstr"][0] == 0 and d["gran"] == "SG" and d["count_wi"] == 3 * Nel * Np * Np
    assert d["loopstr"] == Np * Np           # m innermost
    loc = {f["tag"]: f for f in fs if f["kind"] == "mem" and f["mem"] == "local"}
    assert loc["u_fetch_st"]["count_wi"] == u["count_wi"]
    assert loc["u_fetch_ld"]["count_wi"] == Nel * Np * Np      # read once per (k, i, j)
    res = by_tag(fs, "dg-res-16x16")
    assert res["count"] == res["footprint"] == 3 * Nel * Np
    assert single(fs, "sync") == 2 * G1
    with pytest.raises(Exception):
        features("dg_upf", Np=Np, Nel=64, L0=32, L1=8)


@pytest.mark.parametrize("Np,Nel,L0,L1", [(20, 64, 16, 16), (35, 64, 32, 8), (56, 32, 16, 16)])
def test_dg_dmpft_closed_forms(Np, Nel, L0, L1):
    # dmPF-T: dmPF on transposed u and res, lid(0) stride 1 for both
    sh = "%dx%d" % (L0, L1)
    t = features("dg_dmpft", Np=Np, Nel=Nel, L0=L0, L1=L1)
    d = features("dg_dmpf", Np=Np, Nel=Nel, L0=L0, L1=L1)
    assert op(t, "float32", "madd", wi=True) == op(d, "float32", "madd", wi=True) == 3 * Nel * Np * Np
    u = by_tag(t, "dg-dmPFT-u-" + sh)
    assert u["lstr"] == (1, 0) and u["gstr"] == (L0, 0) and u["loopstr"] == Nel
    assert u["count_wi"] == 3 * Nel * Np * Np and u["footprint"] == Nel * Np
    r = by_tag(t, "dg-dmPFT-res-" + sh)
    assert r["lstr"] == (1, Nel) and r["count"] == r["footprint"] == 3 * Nel * Np
    for tag in ("dg-dmPF-dm-" + sh,):
        a, b = by_tag(t, tag), by_tag(d, tag)
        assert (a["count"], a["lstr"], a["gstr"], a["footprint"]) == (b["count"], b["lstr"], b["gstr"], b["footprint"])
    assert single(t, "sync") == single(d, "sync")


@pytest.mark.parametrize("n", [16, 20, 33, 48])
def test_fd_tile18_closed_forms(n):
    # 18x18 work-groups fetch 18x18 tiles, the 16x16 interior computes:
    # gid(0) stride 16 (Section "Finite Differences")
    W = n + 2
    t = features("fd_tile18", n=n)
    assert op(t, "float32", "madd", wi=True) == n * n
    assert op(t, "float32", "add", wi=True) == 3 * n * n
    u = by_tag(t, "fd-tile18-u")
    assert u["footprint"] == W * W and u["lstr"] == (1, W) and u["gstr"] == (16, 16 * W)
    G = -(-n // 16)
    per_axis = sum(min(18, W - 16 * g) for g in range(G))
    assert u["count"] == per_axis * per_axis
    if n % 16 == 0:
        assert u["count"] == 324 * G * G          # one fetch per thread of every group
    r = by_tag(t, "fd-tile18-res")
    assert r["count"] == r["footprint"] == n * n and r["gstr"] == (16, 16 * n)
    loc = [f for f in t if f["kind"] == "mem" and f["mem"] == "local"]
    assert sum(f["count_wi"] for f in loc if f["dir"] == "load") == 5 * n * n
    assert single(t, "sync") == 1 and single(t, "groups") == G * G
    # 18x18 = 324 threads: 10 full sub-groups and one of 4 lanes per group
    if n % 16 == 0:
        assert by_tag(t, "u_fetch_st")["count"] == 11 * G * G


@pytest.mark.parametrize("n", [14, 20, 33, 48])
def test_fd_closed_forms(n):
    W = n + 2
    t = features("fd_tile", n=n)
    assert op(t, "float32", "madd", wi=True) == n * n
    assert op(t, "float32", "add", wi=True) == 3 * n * n
    assert op(t, "float32", "mul", wi=True) == n * n
    r = by_tag(t, "fd-tile-res")
    assert r["count"] == r["footprint"] == n * n
    u = by_tag(t, "fd-tile-u")
    assert u["footprint"] == W * W and u["lstr"] == (1, W) and u["gstr"] == (14, 14 * W)
    G = -(-n // 14)
    per_axis = sum(min(16, W - 14 * g) for g in range(G))
    assert u["count"] == per_axis * per_axis
    loc = [f for f in t if f["kind"] == "mem" and f["mem"] == "local"]
    assert sum(f["count_wi"] for f in loc if f["dir"] == "load") == 5 * n * n
    assert single(t, "sync") == 1
    d = features("fd_direct", n=n)
    loads = [f for f in d if f["kind"] == "mem" and f["dir"] == "load"]
    assert len(loads) == 5
    for f in loads:
        assert f["count"] == f["footprint"] == n * n and f["lstr"] == (1, W) and f["gstr"] == (16, 16 * W)
    assert op(d, "float32", "madd", wi=True) == n * n


@pytest.mark.parametrize("dtype,vec,s,L,shape", [(0, 0, 1, 1, 0), (0, 1, 4, 3, 0), (1, 0, 32, 4, 0),
                                                 (1, 1, 2, 2, 0), (0, 0, 1, 2, 1), (0, 1, 1, 4, 1)])
def test_stream_pattern(dtype, vec, s, L, shape):
    N = 256 * 32 * 8 * 4
    Wd = 64
    fs = features("stream", dtype=dtype, vec=vec, N=N, s=s, L=L, shape=shape, W=Wd)
    w = (4 if dtype == 0 else 2) if vec else 1
    M = N // w
    sites = [f for f in fs if f["kind"] == "mem"]
    assert len(sites) == L + 1
    for f in sites:
        assert f["count"] == f["footprint"] == M           # AFR 1: every element once
        if shape == 0:
            assert f["lstr"] == (s,) and f["gstr"] == (1, 256 * s)
        else:
            assert f["lstr"] == (1, Wd) and f["gstr"] == (16, 16 * Wd)
    dn = "float32" if dtype == 0 else "float64"
    assert op(fs, dn, "add") == (L - 1) * N // 32


@pytest.mark.parametrize("dtype,o,F", [(0, 0, 64), (0, 1, 128), (0, 2, 1024), (1, 2, 96)])
def test_fma_counts(dtype, o, F):
    G = 3
    fs = features("fma", dtype=dtype, op=o, F=F, G=G)
    dn = "float32" if dtype == 0 else "float64"
    nsg = G * 256 // 32
    target = ("add", "mul", "madd")[o]
    adds = 32 + 31 + (F if target == "add" else 0)
    assert op(fs, dn, "add") == adds * nsg
    if target != "add":
        assert op(fs, dn, target) == F * nsg


@pytest.mark.parametrize("R,sync", [(4, 0), (256, 0), (64, 1)])
def test_smem_and_barrier_counts(R, sync):
    fs = features("smem", R=R, sync=sync, G=2)
    assert feature_value("f_mem_access_local_float32", fs) == (R + 2) * 2 * 8
    assert single(fs, "sync") == 1 + (R // 4 if sync else 0)
    b = features("barrier", B=37, G=3)
    assert single(b, "sync") == 37 and single(b, "groups") == 3
    o = features("overlap", m=5, N=1024)
    assert feature_value("f_mem_access_local_float32", o) == 2 * 5 * 1024 // 32
    e = features("empty", G=64)
    assert single(e, "groups") == 64 and single(e, "launch") == 1
    assert [f for f in e if f["kind"] == "mem"] == []


@pytest.mark.parametrize("T", [16, 18])
@pytest.mark.parametrize("R,G", [(4, 1), (64, 3)])
def test_smem2d_counts(T, R, G):
    # 2-D local shuffle: R local accesses per work-item in the loop, lid(1)
    # stride T; a T x T work-group has ceil(T^2 / 32) sub-groups
    fs = features("smem2d", R=R, T=T, G=G)
    loc = [f for f in fs if f["kind"] == "mem" and f["mem"] == "local"]
    assert sum(f["count_wi"] for f in loc) == G * T * T * (R + 2)
    sgs = G * (-(-T * T // 32))
    for f in loc:
        assert f["lstr"] == (1, T) and f["gran"] == "SG"
        assert f["count"] == sgs * (R // 4 if f["tag"] in ("s_ldA", "s_stB", "s_ldB", "s_stA") else 1)
        assert f["footprint"] == T * T
    g = by_tag(fs, "in")
    assert g["count"] == g["footprint"] == G * T * T and g["lstr"] == (1, T) and g["gstr"] == (T * T,)
    assert single(fs, "sync") == 1 and single(fs, "groups") == G


@pytest.mark.parametrize("V", [4, 8])
@pytest.mark.parametrize("n,BX,BY", [(64, 32, 4), (128, 64, 8), (96, 32, 32)])
def test_fd_block_counts(n, BX, BY, V):
    # TMA stencil tile: every output computed once (3 add + 1 mul + 1 madd),
    # the box (BY+2) x (BX+4) copied once per group, 3V + 2 shared loads and
    # V/4 vector stores per work-item
    fs = features("fd_block", n=n, BX=BX, BY=BY, V=V)
    assert op(fs, "float32", "add", wi=True) == 3 * n * n and op(fs, "float32", "madd", wi=True) == n * n
    G = (n // BX) * (n // BY)
    u = by_tag(fs, "fdb-u")
    assert u["count_wi"] == G * (BY + 2) * (BX + 4) and u["lstr"] == (0, 0) and u["footprint"] == (n + 2) * (n + 4)
    wi = G * (BX // V) * BY
    assert by_tag(fs, "t_c")["count_wi"] == wi * (V + 2) and by_tag(fs, "t_n")["count_wi"] == wi * V
    assert by_tag(fs, "t_c")["footprint"] == BY * (BX + 2) and by_tag(fs, "t_s")["footprint"] == BY * BX
    r = by_tag(fs, "fdb-res")
    assert r["count"] == r["footprint"] == n * n // 4 and r["lstr"] == (V // 4, n // 4)
    assert single(fs, "sync") == 1 and single(fs, "groups") == G


@pytest.mark.parametrize("n,BM,BN,BK", [(192, 96, 64, 32), (256, 128, 64, 64), (256, 64, 128, 32)])
def test_simt_closed_forms(n, BM, BN, BK):
    # register-tiled matmul: n^3 multiply-adds, A read n/BN times and B n/BM
    # times (16-byte vectors), every C vector stored once; the B fragment is
    # read as vectors lid0 and L0 + lid0 (lid(0) stride 1)
    fs = features("mm_simt", n=n, BM=BM, BN=BN, BK=BK)
    assert op(fs, "float32", "madd", wi=True) == n ** 3
    assert by_tag(fs, "simt-a")["count_wi"] == n ** 3 // (4 * BN)
    assert by_tag(fs, "simt-b")["count_wi"] == n ** 3 // (4 * BM)
    c = by_tag(fs, "simt-c")
    assert c["count_wi"] == c["footprint"] == n * n // 4 and c["lstr"][0] == 1 and c["loopstr"] == BN // 8
    for t in ("Bs_ld0", "Bs_ld1"):
        assert by_tag(fs, t)["lstr"] == (1, 0)
    assert single(fs, "sync") == 2 * (n // BK)


@pytest.mark.parametrize("kernel,R", [("mm_tc", 128), ("mm_tc256", 256)])
@pytest.mark.parametrize("n", [256, 512])
def test_tensor_core_closed_forms(kernel, R, n):
    # R x 256 tiles: n^3 bf16 multiply-adds; A read once per tile column
    # (n/256 times), Bt once per tile row (n/R times), by one elected thread
    # (uniform, lid(0) stride 0); every 16-byte C vector stored once, each
    # work-item writing one row (lid(0) stride n/4 vectors)
    fs = features(kernel, n=n)
    assert op(fs, "bfloat16", "madd", wi=True) == n ** 3
    a, b = by_tag(fs, "tc-a"), by_tag(fs, "tc-b")
    assert a["count_wi"] == a["count"] == n ** 3 // 256 and a["footprint"] == n * n and a["lstr"][0] == 0
    assert b["count_wi"] == n ** 3 // R and b["footprint"] == n * n
    c = by_tag(fs, "tc-c")
    assert c["count_wi"] == c["footprint"] == n * n // 4 and c["lstr"][0] == n // 4
    assert c["count"] == c["count_wi"]   # non-uniform global access: counted per work-item
    assert single(fs, "groups") == (n // 256) * (n // R) and single(fs, "sync") == 3


@pytest.mark.parametrize("Np,Nel,P,A", [(20, 260, 0, 0), (35, 256, 2, 1), (84, 388, 0, 1), (10, 132, 3, 0),
                                        (56, 128, 0, 0), (56, 260, 0, 1), (56, 516, 2, -1), (84, 132, 0, -1)])
def test_dg_tc_closed_forms(Np, Nel, P, A):
    # the tensor-core DG: every u element reaches each m-group once (TMA box
    # element by element, uniform, when Np % 4 == 0, else per work-item),
    # every result stored once (bulk copy, uniform); the multiply-adds are
    # three TF32 passes over the padded product 128 x NR x 8 KS per tile
    # (NR = 3 NP8 or NP8 rounded up to 16), at least three times the useful
    # 3 Nel Np^2; each operator element is loaded once per work-group; all
    # work-items pass the same three work-group barriers
    fs = features("dg_tc", Np=Np, Nel=Nel, P=P, A=A)
    if A < 0:
        A = 1 if (20 < Np <= 40 or Np > 64) else 0
    MS = 3 if (Np <= 40 or (A == 0 and Np <= 64)) else 1
    G, T, NP8, KS = 3 // MS, -(-Nel // 128), -(-Np // 8) * 8, -(-Np // 8)
    NR = -(-(MS * NP8) // 16) * 16
    R = 2 if (A == 0 and Np <= 20) else 1
    Pr = P if P else min(T, 152 * R // G)
    assert single(fs, "groups") == G * Pr and single(fs, "sync") == 3
    mm = op(fs, "tfloat32", "madd", wi=True)
    assert mm == G * T * KS * 3 * 128 * NR * 8 >= 3 * (3 * Nel * Np * Np)
    uu = by_tag(fs, "dgc-u")
    assert uu["count_wi"] == G * Nel * Np and uu["footprint"] == Nel * Np and uu["gstr"] == (0, 128 * Np)
    # Np % 4 == 0: TMA boxes; else A = 1: one bulk copy per tile (both uniform);
    # else per work-item loads from global memory
    bulk = Np % 4 != 0 and A == 1
    assert uu["lstr"] == ((0,) if (Np % 4 == 0 or bulk) else (Np,))
    if bulk:
        rr = by_tag(fs, "dgc-R")   # the converters' reads of the staged rows
        assert rr["count_wi"] == G * Nel * Np and rr["lstr"] == (Np,) and rr["footprint"] == min(128, Nel) * Np
    r = by_tag(fs, "dgc-res")
    assert r["count_wi"] == r["count"] == r["footprint"] == 3 * Nel * Np and r["lstr"] == (0,)
    assert r["gstr"] == ((Nel * Np if MS == 1 else 0), 128 * Np)
    d = by_tag(fs, "dgc-D")
    assert d["count_wi"] == G * Pr * MS * Np * Np and d["footprint"] == 3 * Np * Np
    # the split: one subtraction per operator and per converted u element
    adds = op(fs, "float32", "add", wi=True)
    assert adds == 4 * G * Pr * MS * NP8 * 8 * (-(-Np // 32)) + 4 * G * T * 2 * KS * 128
    assert any(f["kind"] == "mem" and f["tag"] == "dgc-Uh" for f in fs) == (A == 0)


@pytest.mark.parametrize("Np,Nel", [(20, 132), (35, 256), (84, 128), (17, 4), (56, 256)])
def test_dg_tile_closed_forms(Np, Nel):
    # the DG product, one work-group per (m, 128 elements), NB = ceil(Np/16)
    # columns per work-item over XL = ceil(Np/NB) x-lanes, j in 8-byte pairs:
    # every D row of its m loaded once per work-group (as vectors when Np is
    # even), every u element once per m (one bulk copy, uniform), every result
    # stored once; padded rows (XL NB > Np), padded j and rows of a partial
    # tile add multiply-adds (2 x 8 x NB per pair per work-item), never stores;
    # each output's even-j and odd-j running sums are combined by one add
    fs = features("dg_tile", Np=Np, Nel=Nel)
    T, NB, Q = -(-Nel // 128), -(-Np // 16), -(-Np // 2)
    XL = -(-Np // NB)
    G = 3 * T
    assert op(fs, "float32", "madd", wi=True) == G * 16 * XL * 8 * NB * 2 * Q >= 3 * Nel * Np * Np
    assert op(fs, "float32", "add", wi=True) == G * 16 * XL * 8 * NB   # even-j and odd-j sums combined
    if XL * NB == Np and Np % 2 == 0 and Nel % 128 == 0:
        assert op(fs, "float32", "madd", wi=True) == 3 * Nel * Np * Np
    d = by_tag(fs, "dgt-D")
    if Np % 2 == 0:
        assert d["dtype"] == "float32x2" and d["count_wi"] == G * Np * Np // 2 and d["lstr"] == (1, Np // 2)
        assert d["footprint"] == 3 * Np * Np // 2 and d["gstr"] == (Np * Np // 2, 0)
    else:
        assert d["dtype"] == "float32" and d["count_wi"] == G * Np * Np and d["lstr"] == (2, Np)
        assert d["footprint"] == 3 * Np * Np and d["gstr"] == (Np * Np, 0)
    uu = by_tag(fs, "dgt-u")
    assert uu["count_wi"] == uu["count"] == 3 * Nel * Np and uu["footprint"] == Nel * Np and uu["lstr"] == (0, 0)
    r = by_tag(fs, "dgt-res")
    assert r["count_wi"] == r["footprint"] == 3 * Nel * Np and r["lstr"] == (1, Np)
    assert r["gstr"] == (Nel * Np, 128 * Np)
    assert by_tag(fs, "dgt-Us")["count_wi"] == G * 16 * XL * 8 * Q
    assert by_tag(fs, "dgt-Dl")["count_wi"] == G * 16 * XL * NB * Q
    pd = by_tag(fs, "dgt-Dl")["lstr"][0] * 2
    assert pd % 32 == 2 and pd >= 2 * Q
    assert single(fs, "sync") == (1 if Np % 2 == 0 else 2) and single(fs, "groups") == G
