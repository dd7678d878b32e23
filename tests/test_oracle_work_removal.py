"""Automatic work removal (Algorithm 3) applied to the oracle's descriptors
of the modeled kernels reproduces, record for record, the counts of the
hand-written twins -- in the oracle and in the library's closed forms.
Pins each hand-written twin (and so its CUDA kernel's definition) to the
paper's transformation of its parent.  CPU only."""
import pytest

import paper_1904_09538_gb300 as pm
from oracle.features import features

MM_TAGS = {"mm_pf": ["mm-PF-a", "mm-PF-b", "c"], "mm_nopf": ["mm-noPF-a", "mm-noPF-b", "c"]}


def _dg(kind, sh):
    return {"nopf": ["dg-noPF-u-" + sh, "dg-noPF-dm-" + sh, "dg-res-" + sh],
            "dmpf": ["dg-dmPF-u-" + sh, "dg-dmPF-dm-" + sh, "dg-res-" + sh],
            "upf": ["dg-uPF-u-" + sh, "dg-noPF-dm-" + sh, "dg-res-" + sh],
            "dmpft": ["dg-dmPFT-u-" + sh, "dg-dmPF-dm-" + sh, "dg-dmPFT-res-" + sh]}[kind]


def _key(r):
    return (r["kind"], r["name"])


def same(auto, twin, **params):
    a = {_key(r): r for r in auto if r["kind"] != "grid"}
    b = {_key(r): r for r in twin if r["kind"] != "grid"}
    assert sorted(a) == sorted(b), (sorted(a), sorted(b))
    for k, r in b.items():
        for f in ("count", "count_wi", "count_sg", "lstr", "gstr", "loopstr", "footprint", "gran"):
            if f in r and f in a[k]:
                assert a[k][f] == r[f], (k, f, a[k][f], r[f])


def lib_records(kernel, **params):
    return pm.counts(kernel, **params)


# (parent, kept global tags index list, hand-written twin)
MM_CASES = [("mm_pf", [0], "mm_pf_a"), ("mm_pf", [1], "mm_pf_b"), ("mm_nopf", [0], "mm_nopf_a"),
            ("mm_nopf", [1], "mm_nopf_b")]


@pytest.mark.parametrize("parent,keep,twin", MM_CASES)
@pytest.mark.parametrize("n", [32, 48])
def test_matmul_twins(parent, keep, twin, n):
    tags = MM_TAGS[parent]
    auto = features(parent, remove=[t for i, t in enumerate(tags) if i not in keep], n=n)
    same(auto, features(twin, n=n))
    same(auto, lib_records(twin, n=n))


DG_CASES = [("dg_nopf", "nopf", [0], "dg_nopf_u"), ("dg_nopf", "nopf", [1], "dg_nopf_dm"),
            ("dg_nopf", "nopf", [2], "dg_res"), ("dg_dmpf", "dmpf", [0], "dg_dmpf_u"),
            ("dg_dmpf", "dmpf", [1], "dg_dmpf_dm"), ("dg_dmpf", "dmpf", [2], "dg_res"),
            ("dg_upf", "upf", [0], "dg_upf_u"), ("dg_upf", "upf", [2], "dg_res"),
            ("dg_dmpft", "dmpft", [0], "dg_dmpft_u"), ("dg_dmpft", "dmpft", [1], "dg_dmpf_dm"),
            ("dg_dmpft", "dmpft", [2], "dg_dmpft_res")]


@pytest.mark.parametrize("parent,kind,keep,twin", DG_CASES)
@pytest.mark.parametrize("Np,Nel,L0,L1", [(20, 32, 16, 16), (35, 64, 32, 8), (7, 16, 16, 16)])
def test_dg_twins(parent, kind, keep, twin, Np, Nel, L0, L1):
    if parent == "dg_upf" and L0 != L1:
        return
    sh = "%dx%d" % (L0, L1)
    tags = _dg(kind, sh)
    p = dict(Np=Np, Nel=Nel, L0=L0, L1=L1)
    auto = features(parent, remove=[t for i, t in enumerate(tags) if i not in keep], **p)
    same(auto, features(twin, **p))
    same(auto, lib_records(twin, **p))


FD_CASES = [("fd_tile", ["fd-tile-res"], "fd_tile_u"), ("fd_tile", ["fd-tile-u"], "fd_tile_res"),
            ("fd_tile18", ["fd-tile18-res"], "fd_tile18_u"), ("fd_tile18", ["fd-tile18-u"], "fd_tile18_res"),
            ("fd_direct", ["res"], "fd_direct_u"), ("fd_direct", ["u_c", "u_n", "u_s", "u_w", "u_e"], "fd_direct_res")]


@pytest.mark.parametrize("parent,remove,twin", FD_CASES)
@pytest.mark.parametrize("n", [13, 16, 29])
def test_stencil_twins(parent, remove, twin, n):
    auto = features(parent, remove=remove, n=n)
    same(auto, features(twin, n=n))
    same(auto, lib_records(twin, n=n))


def test_work_removal_drops_barriers_and_local_memory():
    auto = features("mm_pf", remove=["mm-PF-b", "c"], n=32)
    assert not [r for r in auto if r["kind"] == "mem" and r["mem"] == "local"]
    assert [r for r in auto if r["kind"] == "sync"][0]["count"] == 0
    assert {r["op"] for r in auto if r["kind"] == "op"} == {"add"}
