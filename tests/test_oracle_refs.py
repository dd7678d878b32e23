"""Pins of the oracle's reference outputs: exact special cases, closed forms,
invariants, and special cases that reduce to independent library routines
(NumPy).  CPU only."""
import numpy as np
import pytest

import pm_inputs
from oracle import refs
from oracle.features import features


def test_stream_exact_integer_sums():
    for L in (1, 2, 3, 4):
        xs = [pm_inputs.integers((4096,), 10 + a, -1000, 1000).astype(np.float32) for a in range(L)]
        out = refs.stream(xs)
        want = sum(x.astype(np.int64) for x in xs)
        assert np.array_equal(out.astype(np.int64), want)
    x = pm_inputs.uniform((1000,), 3)
    assert np.all(refs.stream([x, -x]) == 0.0)
    xd = pm_inputs.uniform((1000,), 4, dtype=np.float64)
    assert np.array_equal(refs.stream([xd]), xd)


def test_stream_rounding_bound():
    xs = [pm_inputs.uniform((1 << 14,), 20 + a) for a in range(4)]
    out = refs.stream(xs).astype(np.float64)
    exact = sum(x.astype(np.float64) for x in xs)
    bound = 3 * 2.0 ** -24 * sum(np.abs(x.astype(np.float64)) for x in xs)
    assert np.all(np.abs(out - exact) <= bound)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_fma_add_closed_form(dt):
    # dyadic start values keep every step exact: out = 32 u + 15.5 + R/256
    u = (pm_inputs.integers((512,), 5, -64, 64) / 128.0).astype(dt)
    for F in (32, 1024, 1 << 16):
        R = F // 32
        out = refs.fma(u, 0, F)
        assert np.array_equal(out, (32 * u.astype(np.float64) + 15.5 + R / 256.0).astype(dt))


@pytest.mark.parametrize("dt,tol", [(np.float32, 2e-5), (np.float64, 1e-13)])
def test_fma_mul_madd_closed_forms(dt, tol):
    u = pm_inputs.uniform((512,), 6, dtype=dt)
    F = 1024
    R = F // 32
    t = np.arange(32) / 32.0
    x0 = u.astype(np.float64)[:, None] + t[None, :]
    mul = (x0 * (1 - 2.0 ** -12) ** R).sum(1)
    madd = (1.0 + (x0 - 1.0) * (1 - 2.0 ** -10) ** R).sum(1)
    scale = np.abs(x0).sum(1) + 32
    assert np.all(np.abs(refs.fma(u, 1, F) - mul) <= tol * scale)
    assert np.all(np.abs(refs.fma(u, 2, F) - madd) <= tol * scale)


def test_matmul_reference():
    n = 48
    a = pm_inputs.uniform((n, n), 1)
    b = pm_inputs.uniform((n, n), 2)
    c, ca = refs.matmul(a, b)
    want = a.astype(np.float64) @ b.astype(np.float64)
    assert np.max(np.abs(c - want)) <= 1e-13 * np.max(ca)
    assert np.allclose(ca, np.abs(a.astype(np.float64)) @ np.abs(b.astype(np.float64)), rtol=1e-13)
    c_id, _ = refs.matmul(a, np.eye(n, dtype=np.float32))
    assert np.array_equal(c_id, a.astype(np.float64))


def test_matmul_rows_agrees_with_full_product():
    # rows of the product from the FP64 matrix product equal the same rows of
    # the C reference's triple loop; the identity gives A's rows back exactly
    n = 40
    a = pm_inputs.uniform((n, n), 11)
    b = pm_inputs.uniform((n, n), 12)
    c, ca = refs.matmul(a, b)
    rows = np.array([0, 7, 39])
    cr, car = refs.matmul_rows(a[rows], b)
    assert cr.shape == (3, n)
    assert np.max(np.abs(cr - c[rows])) <= 1e-13 * np.max(ca)
    assert np.allclose(car, ca[rows], rtol=1e-13)
    ci, _ = refs.matmul_rows(a[rows], np.eye(n, dtype=np.float32))
    assert np.array_equal(ci, a[rows].astype(np.float64))


def test_dg_reference():
    Np, Nel = 20, 40
    D = pm_inputs.normal((3, Np, Np), 3)
    u = pm_inputs.normal((Nel, Np), 4)
    res, ra = refs.dg(D, u)
    want = np.einsum("mij,kj->mki", D.astype(np.float64), u.astype(np.float64))
    assert np.max(np.abs(res - want)) <= 1e-13 * np.max(ra)
    # D = identity per m: res[m,k,:] = u[k,:]
    Di = np.stack([np.eye(Np, dtype=np.float32)] * 3)
    r2, _ = refs.dg(Di, u)
    assert np.array_equal(r2, np.stack([u.astype(np.float64)] * 3))


def test_stencil_reference():
    n = 30
    i = np.arange(n + 2, dtype=np.float64)
    I, J = np.meshgrid(i, i, indexing="ij")
    # discrete Laplacian (c0=-4, c1=1): constant -> 0, linear -> 0, i^2 -> 2
    for field, want in ((np.ones_like(I), 0.0), (I + 2 * J, 0.0), (I * I, 2.0)):
        r, _ = refs.stencil(field.astype(np.float32), -4.0, 1.0)
        assert np.all(r == want)
    u = pm_inputs.uniform((n + 2, n + 2), 9)
    r, ra = refs.stencil(u, 0.7, -0.3)
    U = u.astype(np.float64)
    want = 0.7 * U[1:-1, 1:-1] - 0.3 * (U[:-2, 1:-1] + U[2:, 1:-1] + U[1:-1, :-2] + U[1:-1, 2:])
    assert np.max(np.abs(r - want)) <= 1e-14 * np.max(ra)


def _loads_per_wi(kernel, **p):
    fs = features(kernel, **p)
    return sum(f["count_wi"] for f in fs if f["kind"] == "mem" and f["dir"] == "load")


@pytest.mark.parametrize("kernel", ["mm_pf_a", "mm_pf_b", "mm_nopf_a", "mm_nopf_b"])
def test_mm_twin_ones(kernel):
    n = 32
    dest = refs.mm_twin(kernel, np.ones((n, n), np.float32))
    assert dest.sum() == _loads_per_wi(kernel, n=n)
    assert np.all(dest == (n // 16 if "_pf_" in kernel else n))


@pytest.mark.parametrize("kernel", ["dg_nopf_u", "dg_nopf_dm", "dg_dmpf_u", "dg_dmpf_dm"])
@pytest.mark.parametrize("Np,L0,L1", [(20, 16, 16), (35, 32, 8)])
def test_dg_twin_ones(kernel, Np, L0, L1):
    Nel = 64
    D = np.ones((3, Np, Np), np.float32)
    u = np.ones((Nel, Np), np.float32)
    dest = refs.dg_twin(kernel, D, u, L0, L1)
    assert dest.sum() == _loads_per_wi(kernel, Np=Np, Nel=Nel, L0=L0, L1=L1)
    assert np.all(dest[Np:] == 0)


@pytest.mark.parametrize("kernel", ["dg_upf_u", "dg_dmpft_u"])
@pytest.mark.parametrize("Np", [20, 35])
def test_dg_new_twin_ones(kernel, Np):
    Nel, L0, L1 = 64, 16, 16
    D = np.ones((3, Np, Np), np.float32)
    u = np.ones((Np, Nel) if kernel == "dg_dmpft_u" else (Nel, Np), np.float32)
    dest = refs.dg_twin(kernel, D, u, L0, L1)
    assert dest.sum() == _loads_per_wi(kernel, Np=Np, Nel=Nel, L0=L0, L1=L1)
    if kernel == "dg_upf_u":     # the u fetch is not guarded by the row i
        l0 = np.arange(Nel) % L0
        assert np.all(dest == (-(-(Np - l0) // L1))[None, :])   # j tiles in which lane l0 fetches
    else:
        assert np.all(dest[:Np] == 3 * Np) and np.all(dest[Np:] == 0)


@pytest.mark.parametrize("kernel", ["fd_tile_u", "fd_direct_u", "fd_tile18_u"])
def test_fd_twin_ones(kernel):
    n = 37
    dest = refs.fd_twin(kernel, np.ones((n + 2, n + 2), np.float32))
    assert dest.sum() == _loads_per_wi(kernel, n=n)
