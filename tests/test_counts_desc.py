"""pm_counts_desc: features of kernels given as loop-nest descriptions.
The descriptions in tests/descriptors/ restate eleven registry kernels (the
three modeled computations, two work-removed twins, the arithmetic, local
memory and stream microbenchmarks) from their definitions; their counts must equal the library's closed forms record
for record -- by enumeration at small sizes, by quasi-polynomial
extrapolation at large ones -- and the oracle's brute force.  CPU only."""
import os

import numpy as np
import pytest

import paper_1904_09538_gb300 as pm
from oracle.features import features as ofeatures

HERE = os.path.join(os.path.dirname(__file__), "descriptors")


def desc(name):
    return open(os.path.join(HERE, name + ".desc")).read()


FIELDS = ("count", "gran", "count_wi", "count_sg", "lstr", "gstr", "loopstr", "accesses", "footprint", "dsize")


def same(a, b):
    ka = {r["name"]: r for r in a}
    kb = {r["name"]: r for r in b if r.get("kind") != "grid"}
    assert sorted(ka) == sorted(kb), (sorted(set(ka) ^ set(kb)))
    for n, r in kb.items():
        for f in FIELDS:
            if f in r and f in ka[n]:
                assert ka[n][f] == r[f], (n, f, ka[n][f], r[f])


@pytest.mark.parametrize("n", [16, 48, 80])
def test_matmul_enumerated(n):
    same(pm.counts_desc(desc("mm_pf"), n=n), pm.counts("mm_pf", n=n))


@pytest.mark.parametrize("n", [1024, 2048, 4096])
def test_matmul_extrapolated(n):
    same(pm.counts_desc(desc("mm_pf"), interp={"n": (16, 3)}, n=n), pm.counts("mm_pf", n=n))


@pytest.mark.parametrize("n", [1, 13, 14, 29, 45])
def test_stencil_enumerated(n):
    same(pm.counts_desc(desc("fd_tile"), n=n), pm.counts("fd_tile", n=n))


@pytest.mark.parametrize("n", [1000, 4096, 16383])
def test_stencil_extrapolated(n):
    same(pm.counts_desc(desc("fd_tile"), interp={"n": (14, 2)}, n=n), pm.counts("fd_tile", n=n))


@pytest.mark.parametrize("Np", [20, 35, 56, 84])
def test_dg_extrapolated_in_elements(Np):
    same(pm.counts_desc(desc("dg_nopf"), interp={"Nel": (16, 1)}, Np=Np, Nel=1 << 18),
         pm.counts("dg_nopf", Np=Np, Nel=1 << 18, L0=16, L1=16))


@pytest.mark.parametrize("s", [1, 4, 32])
def test_stream_two_parameters(s):
    same(pm.counts_desc(desc("stream2"), N=1 << 16, s=s), pm.counts("stream", N=1 << 16, s=s, L=2))
    same(pm.counts_desc(desc("stream2"), interp={"N": (256 * s, 1)}, N=1 << 26, s=s),
         pm.counts("stream", N=1 << 26, s=s, L=2))


# the other restated registry kernels: (description, its parameters, registry
# kernel, its parameters) at small sizes, and at full size with the period and
# degree bound of the interpolated parameter derived from the description
RESTATED = [
    ("mm_nopf", dict(n=48), "mm_nopf", {}),
    ("mm_pf_a", dict(n=48), "mm_pf_a", {}),
    ("mm_pf_b", dict(n=64), "mm_pf_b", {}),
    ("fd_direct", dict(n=45), "fd_direct", {}),
    ("fd_tile18", dict(n=45), "fd_tile18", {}),
    ("fma_madd", dict(F=1024, G=3), "fma", dict(op=2, dtype=0)),
    ("smem_sync", dict(R=64, G=2), "smem", dict(sync=1)),
]


@pytest.mark.parametrize("name,params,kernel,kparams", RESTATED)
def test_restated_kernels_enumerated(name, params, kernel, kparams):
    same(pm.counts_desc(desc(name), **params), pm.counts(kernel, **dict(kparams, **params)))


@pytest.mark.parametrize("name,param,params,kernel,kparams,want", [
    ("mm_nopf", "n", dict(n=4096), "mm_nopf", {}, (16, 3)),
    ("mm_pf_a", "n", dict(n=4096), "mm_pf_a", {}, (16, 3)),
    ("fd_direct", "n", dict(n=16383), "fd_direct", {}, (16, 2)),
    ("fd_tile18", "n", dict(n=16384), "fd_tile18", {}, (16, 2)),
    ("fma_madd", "F", dict(F=65536, G=8), "fma", dict(op=2, dtype=0), (32, 1)),
    ("smem_sync", "R", dict(R=16384, G=608), "smem", dict(sync=1), (4, 1)),
])
def test_restated_kernels_extrapolated(name, param, params, kernel, kparams, want):
    assert pm.counts_desc_interp(desc(name), param, **params) == want
    same(pm.counts_desc(desc(name), interp={param: None}, **params), pm.counts(kernel, **dict(kparams, **params)))


def test_matches_oracle_brute_force():
    same(pm.counts_desc(desc("mm_pf"), n=48), ofeatures("mm_pf", n=48))
    same(pm.counts_desc(desc("fd_tile"), n=29), ofeatures("fd_tile", n=29))
    same(pm.counts_desc(desc("dg_nopf"), Np=35, Nel=32), ofeatures("dg_nopf", Np=35, Nel=32, L0=16, L1=16))
    same(pm.counts_desc(desc("fd_tile18"), n=29), ofeatures("fd_tile18", n=29))
    same(pm.counts_desc(desc("smem_sync"), R=16, G=2), ofeatures("smem", R=16, sync=1, G=2))


def test_model_rows_from_descriptions():
    m = pm.Model("f_wall_time", "p_f * f_op_float32_madd + p_a * f_mem_access_tag:mm-PF-a + "
                 "p_l * f_mem_access_local_float32 + p_g * f_thread_groups")
    a = m.feature_values_desc(desc("mm_pf"), interp={"n": (16, 3)}, n=1536)
    assert np.array_equal(a, m.feature_values("mm_pf", n=1536))


@pytest.mark.parametrize("text,params", [
    ("params n\ngrid n\ngroup 16\nstmt\n  access x global load float32 4 l0*l0\n", dict(n=4)),     # not affine
    ("params n\ngrid n\ngroup 16\nstmt\n  access x global load float32 4 l0+q\n", dict(n=4)),      # unknown name
    ("params n\ngrid n\ngroup 16\nstmt\n  access x global load float32 4 (l0\n", dict(n=4)),       # syntax
    ("params n\ngrid n\nstmt\n", dict(n=4)),                                                       # no group
    ("params n\ngrid n\ngroup 16\nbarrier\n  guard l0-8\n", dict(n=4)),                            # uneven barriers
    ("params n\ngrid n\ngroup 2048\n", dict(n=1)),                                                 # group too large
    ("params n\ngrid n\ngroup 16\n", dict(m=1)),                                                   # unknown parameter
])
def test_bad_descriptions_rejected(text, params):
    with pytest.raises(pm.PMError):
        pm.counts_desc(text, **params)


def test_wrong_degree_bound_detected():
    with pytest.raises(pm.PMError):
        pm.counts_desc(desc("mm_pf"), interp={"n": (16, 2)}, n=4096)   # madd count is cubic in n


@pytest.mark.parametrize("name,param,params,want", [
    ("mm_pf", "n", dict(n=64), (16, 3)),             # grid n/16, k loop to n/16, n*(16*g1 + l1) index
    ("fd_tile", "n", dict(n=64), (14, 2)),           # grid (n+13)/14 on both axes
    ("dg_nopf", "Nel", dict(Np=35, Nel=64), (16, 1)),
    ("dg_nopf", "Np", dict(Np=35, Nel=64), (16, 2)),  # (Np+15)/16 tiles, j loop to Np, Np*Np*m index
    ("stream2", "N", dict(N=1 << 16, s=4), (1024, 1)),   # N/(256 s) with s fixed at 4
])
def test_period_and_degree_derived(name, param, params, want):
    assert pm.counts_desc_interp(desc(name), param, **params) == want


@pytest.mark.parametrize("name,param,fixed,target,kernel,kparams", [
    ("mm_pf", "n", {}, 4096, "mm_pf", {}),
    ("fd_tile", "n", {}, 16383, "fd_tile", {}),
    ("dg_nopf", "Nel", dict(Np=84), 1 << 18, "dg_nopf", dict(Np=84, L0=16, L1=16)),
    ("stream2", "N", dict(s=8), 1 << 26, "stream", dict(s=8, L=2)),
])
def test_derived_extrapolation_matches_closed_forms(name, param, fixed, target, kernel, kparams):
    got = pm.counts_desc(desc(name), interp={param: None}, **dict(fixed, **{param: target}))
    same(got, pm.counts(kernel, **dict(kparams, **{param: target})))


def test_derived_in_two_parameters():
    # nested extrapolation, both periods and degrees derived: DG at Np = 84
    # (residue 4 of 16) and Nel = 2^18
    got = pm.counts_desc(desc("dg_nopf"), interp={"Nel": None, "Np": None}, Np=84, Nel=1 << 18)
    same(got, pm.counts("dg_nopf", Np=84, Nel=1 << 18, L0=16, L1=16))


@pytest.mark.parametrize("text,param", [
    ("params n\ngrid 4\ngroup n\nstmt\n  access x global load float32 4 l0\n", "n"),          # group extent in n
    ("params n m\ngrid n/m\ngroup 16\nstmt\n  access x global load float32 4 l0\n", "m"),    # divisor depends on m
    ("params n\ngrid 8\ngroup 16\nstmt\n  loop i 0 n/(l0+1)\n  access x global load float32 4 i\n", "n"),
])
def test_underivable_period_refused(text, param):
    with pytest.raises(pm.PMError) as e:
        pm.counts_desc_interp(text, param, n=64, m=4)
    assert "state its period and degree" in str(e.value)
