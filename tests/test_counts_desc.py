"""pm_counts_desc: features of kernels given as loop-nest descriptions.
The descriptions in tests/descriptors/ restate four registry kernels from
their definitions; their counts must equal the library's closed forms record
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


def test_matches_oracle_brute_force():
    same(pm.counts_desc(desc("mm_pf"), n=48), ofeatures("mm_pf", n=48))
    same(pm.counts_desc(desc("fd_tile"), n=29), ofeatures("fd_tile", n=29))
    same(pm.counts_desc(desc("dg_nopf"), Np=35, Nel=32), ofeatures("dg_nopf", Np=35, Nel=32, L0=16, L1=16))


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
