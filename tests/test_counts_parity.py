"""pm_counts (library closed forms) vs the oracle's brute-force enumeration:
every record bit-exact, over sizes that span several tiles, ragged tails
(guarded partial tiles), degenerate sizes, and paper-size values via exact
quasi-polynomial interpolation.  Host code only -- no GPU needed."""
import pytest

import paper_1904_09538_gb300 as pm
from oracle.features import features as ofeatures, feature_value as ofeature_value
from oracle.quasipoly import extrapolate


def _key(r):
    if r["kind"] == "op":
        return ("op", r["dtype"], r["op"])
    if r["kind"] == "mem":
        return ("mem", r["tag"], r["mem"], r["dir"])
    return (r["kind"],)


def compare(kernel, **params):
    lib = [r for r in pm.counts(kernel, **params)]
    orc = [r for r in ofeatures(kernel, **params) if r["kind"] != "grid"]
    lk = {_key(r): r for r in lib}
    ok = {_key(r): r for r in orc}
    assert len(lk) == len(lib) and len(ok) == len(orc)
    assert sorted(lk) == sorted(ok), (kernel, params, sorted(lk), sorted(ok))
    for k, o in ok.items():
        l = lk[k]
        assert l["name"] == o["name"], (kernel, params, l["name"], o["name"])
        assert l["count"] == o["count"] and l["gran"] == o["gran"], (kernel, params, k, l, o)
        if o["kind"] == "op":
            assert l["count_wi"] == o["count_wi"], (kernel, params, k)
        if o["kind"] == "mem":
            for f in ("lstr", "gstr", "loopstr", "accesses", "footprint", "count_wi", "count_sg", "dsize", "dtype"):
                assert l[f] == o[f], (kernel, params, k, f, l[f], o[f])
    return lib


@pytest.mark.parametrize("dtype,vec,s,L,shape,N,W", [
    (0, 0, 1, 1, 0, 256 * 8, 16), (0, 0, 2, 2, 0, 256 * 8, 16), (0, 1, 4, 3, 0, 4 * 256 * 16, 16),
    (1, 0, 8, 4, 0, 256 * 16, 16), (1, 1, 32, 2, 0, 2 * 256 * 64, 16), (0, 0, 1, 4, 1, 32 * 64, 32),
    (1, 1, 1, 1, 1, 2 * 16 * 48 * 3, 48)])
def test_stream(dtype, vec, s, L, shape, N, W):
    compare("stream", dtype=dtype, vec=vec, N=N, s=s, L=L, shape=shape, W=W)


@pytest.mark.parametrize("dtype,op,F,G", [(0, 0, 32, 1), (0, 1, 64, 3), (0, 2, 1024, 2), (1, 2, 96, 1), (1, 0, 64, 2)])
def test_fma(dtype, op, F, G):
    compare("fma", dtype=dtype, op=op, F=F, G=G)


@pytest.mark.parametrize("R,sync,G", [(4, 0, 1), (64, 1, 3), (256, 0, 2)])
def test_smem(R, sync, G):
    compare("smem", R=R, sync=sync, G=G)


def test_barrier_overlap_empty():
    compare("barrier", B=0, G=2)
    compare("barrier", B=17, G=3)
    for m in (0, 1, 5):
        compare("overlap", m=m, N=768)
    compare("empty", G=1)
    compare("empty", G=77)


@pytest.mark.parametrize("kernel", ["mm_pf", "mm_nopf", "mm_pf_a", "mm_pf_b", "mm_nopf_a", "mm_nopf_b"])
@pytest.mark.parametrize("n", [16, 32, 48, 80])
def test_mm(kernel, n):
    compare(kernel, n=n)


DG = ["dg_nopf", "dg_dmpf", "dg_nopf_u", "dg_nopf_dm", "dg_dmpf_u", "dg_dmpf_dm", "dg_res",
      "dg_dmpft", "dg_dmpft_u", "dg_dmpft_res", "dg_upf", "dg_upf_u"]


@pytest.mark.parametrize("kernel", DG)
@pytest.mark.parametrize("Np,Nel,L0,L1", [(20, 32, 16, 16), (35, 64, 32, 8), (56, 32, 16, 16), (84, 32, 32, 8),
                                          (1, 16, 16, 16), (7, 32, 32, 8), (16, 16, 16, 16), (33, 32, 32, 8),
                                          (84, 48, 16, 16), (17, 16, 16, 16)])
def test_dg(kernel, Np, Nel, L0, L1):
    if kernel.startswith("dg_upf") and L0 != L1:
        with pytest.raises(pm.PMError):
            pm.counts(kernel, Np=Np, Nel=Nel, L0=L0, L1=L1)
        return
    compare(kernel, Np=Np, Nel=Nel, L0=L0, L1=L1)


FD = ["fd_tile", "fd_direct", "fd_tile_u", "fd_tile_res", "fd_direct_u", "fd_direct_res",
      "fd_tile18", "fd_tile18_u", "fd_tile18_res"]


@pytest.mark.parametrize("kernel", FD)
@pytest.mark.parametrize("n", [1, 2, 13, 14, 15, 16, 17, 28, 29, 31, 32, 33, 45, 64])
def test_fd(kernel, n):
    compare(kernel, n=n)


def test_paper_sizes_by_interpolation():
    # library counts at the configuration sizes equal the oracle's exact
    # interpolation from brute-force samples on the same residue class
    def series(kernel, what, **fixed):
        cache = {}

        def f(x):
            if x not in cache:
                p = dict(fixed)
                p[what[0]] = x
                recs = ofeatures(kernel, **p)
                cache[x] = {(r["name"].split("_lstrides")[0] if r["kind"] == "mem" else r["name"]): r["count"]
                            for r in recs if r["kind"] != "grid"}
            return cache[x]
        return f

    def check(kernel, var, target, period, degree, start, **fixed):
        f = series(kernel, (var,), **fixed)
        lib = {(r["name"].split("_lstrides")[0] if r["kind"] == "mem" else r["name"]): r["count"]
               for r in pm.counts(kernel, **dict(fixed, **{var: target}))}
        for key in f(start):
            want = extrapolate(lambda x: f(x)[key], target, period, degree, start)
            assert lib[key] == want, (kernel, key, lib[key], want)

    for n in (256, 768, 896):
        check("mm_pf", "n", n, 16, 3, 16)
        check("mm_nopf", "n", n, 16, 3, 16)
    # stencil tile variant: quasi-polynomial of period 14 in n
    for n in (1024, 4096):
        check("fd_tile", "n", n, 14, 2, 14 + n % 14)
        check("fd_direct", "n", n, 16, 2, 16 + n % 16)
        check("fd_tile18", "n", n, 16, 2, 16 + n % 16)
    for n in (1000, 16383):
        check("fd_tile18", "n", n, 16, 2, 16 + n % 16)
    # DG: linear in Nel at fixed Np, shape
    for Np in (20, 35, 56, 84):
        check("dg_dmpf", "Nel", 1 << 14, 16, 1, 16, Np=Np, L0=16, L1=16)
        check("dg_nopf", "Nel", 1 << 14, 32, 1, 32, Np=Np, L0=32, L1=8)
        check("dg_upf", "Nel", 1 << 14, 16, 1, 16, Np=Np, L0=16, L1=16)
        check("dg_dmpft", "Nel", 1 << 14, 32, 1, 32, Np=Np, L0=32, L1=8)


def test_feature_values_match_oracle():
    expr = ("p_launch * f_sync_kernel_launch + p_group * f_thread_groups + "
            "p_bar * f_sync_barrier_local * f_thread_groups + "
            "p_madd * f_op_float32_madd + p_add * f_op_float32_add + p_mul * f_op_float32_mul + "
            "p_lmem * f_mem_access_local_float32 + "
            "p_g * f_mem_access_global_float32_lstrides:{0:1;1:>1}_gstrides:{0:16;1:>16}_afr:1 + "
            "p_a * f_mem_access_tag:mm-PF-a + p_b * f_mem_access_global_float32_load_gstrides:{0:16}_afr:>1 + "
            "p_v2 * f_mem_access_local_float32x2 + p_v2l * f_mem_access_local_float32x2_load + "
            "p_v4 * f_mem_access_local_float32x4 + p_du * f_mem_access_tag:dgt-u")
    m = pm.Model("f_wall_time", expr)
    for kernel, params in (("mm_pf", dict(n=48)), ("mm_nopf", dict(n=32)), ("fd_tile", dict(n=29)),
                           ("dg_dmpf", dict(Np=35, Nel=64, L0=32, L1=8)), ("stream", dict(N=4096, shape=1, W=32)),
                           ("dg_tile", dict(Np=20, Nel=300)), ("dg_tile", dict(Np=35, Nel=260)),
                           ("mm_simt", dict(n=128, BM=64, BN=64, BK=32))):
        row = m.feature_values(kernel, **params)
        recs = ofeatures(kernel, **params)
        want = [ofeature_value(f, recs) for f in m.features]
        assert list(row) == want, (kernel, list(row), want)


def test_bad_parameters_rejected():
    with pytest.raises(pm.PMError):
        pm.counts("mm_pf", n=17)
    with pytest.raises(pm.PMError):
        pm.counts("stream", N=1000)
    with pytest.raises(pm.PMError):
        pm.counts("dg_nopf", Np=20, Nel=32, L0=8, L1=32)
    with pytest.raises(pm.PMError):
        pm.counts("no_such_kernel")
    with pytest.raises(pm.PMError):
        pm.Model("t", "p_a * (f_x")
    with pytest.raises(pm.PMError):
        pm.Model("t", "p_a * f_mem_access_float32_global")


@pytest.mark.parametrize("n,BM,BN,BK", [(192, 96, 64, 32), (256, 64, 128, 64), (256, 128, 64, 32),
                                        (512, 256, 128, 32), (256, 128, 256, 64), (256, 256, 256, 32),
                                        (768, 96, 256, 64), (384, 96, 128, 32), (128, 64, 64, 64)])
def test_mm_simt(n, BM, BN, BK):
    compare("mm_simt", n=n, BM=BM, BN=BN, BK=BK)


@pytest.mark.parametrize("n", [256, 512])
def test_mm_tc(n):
    compare("mm_tc", n=n)


@pytest.mark.parametrize("n", [256, 512, 768])
def test_mm_tc256(n):
    compare("mm_tc256", n=n)


@pytest.mark.parametrize("V", [4, 8])
@pytest.mark.parametrize("n,BX,BY", [(64, 32, 4), (128, 64, 8), (128, 128, 16), (256, 128, 32), (96, 32, 32)])
def test_fd_block(n, BX, BY, V):
    compare("fd_block", n=n, BX=BX, BY=BY, V=V)


@pytest.mark.parametrize("R,T,G", [(4, 16, 1), (64, 18, 3), (256, 16, 5), (8, 18, 1)])
def test_smem2d(R, T, G):
    compare("smem2d", R=R, T=T, G=G)


@pytest.mark.parametrize("Np,Nel", [(20, 132), (35, 256), (56, 4), (84, 260), (1, 8), (16, 128), (17, 132),
                                    (96, 136)])
def test_dg_tile(Np, Nel):
    compare("dg_tile", Np=Np, Nel=Nel)


# the tensor-core DG: both operand forms, the TMA (Np % 4 == 0) and the
# direct-load paths, ragged last tiles, persistent grids smaller and larger
# than the tile count, the default grid
@pytest.mark.parametrize("Np,Nel,P,A", [(20, 260, 0, -1), (20, 132, 0, 1), (4, 8, 0, -1), (10, 300, 0, 0),
                                        (10, 300, 0, 1), (35, 256, 0, 0), (35, 260, 0, -1), (56, 132, 0, 0),
                                        (56, 516, 0, -1), (84, 388, 2, -1), (84, 132, 0, 0), (20, 1028, 3, 0),
                                        (35, 644, 2, 0), (84, 260, 5, 1), (56, 4, 0, 1)])
def test_dg_tc(Np, Nel, P, A):
    compare("dg_tc", Np=Np, Nel=Nel, P=P, A=A)
