"""Edge cases of the host-side boundary (no GPU): counts at the largest
accepted sizes (no 64-bit overflow; closed forms the paper fixes), the
PM_ECAP protocol of caller-owned output arrays, and parameter validation."""
import ctypes

import pytest

import paper_1904_09538_gb300 as pm
from paper_1904_09538_gb300 import _lib


def rec(recs, name_prefix):
    out = [r for r in recs if r["name"].startswith(name_prefix)]
    assert len(out) == 1, (name_prefix, [r["name"] for r in recs])
    return out[0]


def test_matmul_counts_at_largest_size():
    n = 32768
    r = pm.counts("mm_pf", n=n)
    assert rec(r, "f_op_float32_madd")["count_wi"] == n ** 3          # 2 n^3 flops
    assert rec(r, "f_mem_access_tag:mm-PF-a")["count"] == n ** 3 // 16
    assert rec(r, "f_thread_groups")["count"] == n * n // 256
    t = pm.counts("mm_tc", n=n)
    assert rec(t, "f_op_bfloat16_madd")["count"] == n ** 3           # one work-item issues 128x256x16 per instruction
    assert rec(t, "f_thread_groups")["count"] == (n // 256) * (n // 128)
    w = pm.counts("mm_tc256", n=n)
    assert rec(w, "f_op_bfloat16_madd")["count"] == n ** 3
    assert rec(w, "f_thread_groups")["count"] == (n // 256) ** 2
    assert rec(w, "f_mem_access_tag:tc-b")["count"] == n ** 3 // 256


@pytest.mark.parametrize("kernel", ["fd_tile", "fd_tile18", "fd_direct"])
def test_stencil_counts_at_largest_size(kernel):
    n = 46000
    r = pm.counts(kernel, n=n, c0=-4.0, c1=1.0)
    assert rec(r, "f_op_float32_madd")["count_wi"] == n * n
    assert rec(r, "f_op_float32_add")["count_wi"] == 3 * n * n
    stores = [x for x in r if x["kind"] == "mem" and x["mem"] == "global" and x["dir"] == "store"]
    assert sum(x["count_wi"] for x in stores) == n * n


def test_stream_counts_at_largest_size():
    N = (1 << 31) - 256 * 32            # largest N below 2^31 vectors of 1 element with s = 32
    N -= N % (256 * 32)
    r = pm.counts("stream", dtype=1, vec=0, N=N, s=32, L=4)
    loads = [x for x in r if x["kind"] == "mem" and x["dir"] == "load"]
    assert len(loads) == 4 and all(x["count"] == N for x in loads)
    assert rec(r, "f_op_float64_add")["count_wi"] == 3 * N


def test_counts_cap_protocol():
    k = pm.kernel_lookup("mm_pf")
    arr = (_lib.pm_param * 1)()
    arr[0].key = b"n"
    arr[0].value = 64.0
    need = ctypes.c_size_t(0)
    out = (_lib.pm_feature * 1)()
    st = pm.lib().pm_counts(k, arr, 1, out, 1, ctypes.byref(need))
    assert st == -9 and need.value > 1                                   # PM_ECAP, size needed
    out = (_lib.pm_feature * need.value)()
    n2 = ctypes.c_size_t(0)
    assert pm.lib().pm_counts(k, arr, 1, out, need.value, ctypes.byref(n2)) == 0 and n2.value == need.value


@pytest.mark.parametrize("kernel,params", [
    ("mm_pf", dict(n=0)), ("mm_pf", dict(n=17)), ("mm_tc", dict(n=384)), ("mm_tc", dict(n=512, pipe=3)),
    ("mm_tc256", dict(n=384)), ("mm_tc256", dict(n=32768 + 256)),
    ("dg_tile", dict(Np=20, Nel=130)), ("dg_tile", dict(Np=97, Nel=128)), ("dg_tile", dict(Np=20, Nel=65536 * 128)),
    ("dg_tile", dict(Np=0, Nel=128)),
    ("dg_tc", dict(Np=21, Nel=128)), ("dg_tc", dict(Np=20, Nel=130)), ("dg_tc", dict(Np=20, Nel=0)),
    ("dg_tc", dict(Np=84, Nel=(1 << 24) + 4)), ("dg_tc", dict(Np=20, Nel=128, P=-1)),
    ("dg_tc", dict(Np=20, Nel=128, P=4097)), ("dg_tc", dict(Np=20, Nel=128, A=2)),
    ("fd_block", dict(n=100, BX=64, BY=8)), ("fd_block", dict(n=256, BX=64, BY=8, V=2)),
    ("fd_tile", dict(n=0)), ("dg_upf", dict(Np=20, Nel=32, L0=32, L1=8)), ("dg_nopf", dict(Np=0, Nel=32)),
    ("smem2d", dict(R=8, T=17, G=1)), ("stream", dict(N=1000)), ("stream", dict(N=1 << 20, s=3)),
    ("mm_simt", dict(n=7680, BM=100, BN=64, BK=32)), ("empty", dict(G=0))])
def test_invalid_parameters_rejected(kernel, params):
    with pytest.raises(pm.PMError):
        pm.counts(kernel, **params)


def test_missing_and_unknown_parameters_rejected():
    with pytest.raises(pm.PMError):
        pm.counts("mm_pf")                  # n is required
    with pytest.raises(pm.PMError):
        pm.counts("mm_pf", n=64, bogus=1)
    with pytest.raises(pm.PMError):
        pm.counts("mm_pf", n=64.5)          # integer parameter


def test_dg_tc_counts_at_largest_size():
    # 2^24 elements, Np = 84 (one m per work-group, three m-groups): the
    # closed forms do not overflow; the default grid is 50 work-groups per
    # m-group (one wave of 152 SMs, one per SM)
    Np, Nel = 84, 1 << 24
    r = pm.counts("dg_tc", Np=Np, Nel=Nel)
    T = Nel // 128
    assert rec(r, "f_op_tfloat32_madd")["count"] == 3 * T * 11 * 3 * 128 * 96 * 8
    assert rec(r, "f_mem_access_tag:dgc-res")["count"] == 3 * Nel * Np
    assert rec(r, "f_mem_access_tag:dgc-u")["count"] == 3 * Nel * Np
    assert rec(r, "f_thread_groups")["count"] == 3 * 50


def test_dg_tile_counts_at_largest_size():
    # 65535 tiles of 128 elements, Np = 96: the closed forms do not overflow
    Np, Nel = 96, 65535 * 128
    r = pm.counts("dg_tile", Np=Np, Nel=Nel)
    assert rec(r, "f_op_float32_madd")["count_wi"] == 3 * Nel * Np * Np     # Np % 16 == 0, no padding
    assert rec(r, "f_mem_access_tag:dgt-res")["count"] == 3 * Nel * Np
    assert rec(r, "f_mem_access_tag:dgt-u")["count"] == 3 * Nel * Np
    assert rec(r, "f_thread_groups")["count"] == 3 * 65535
