"""GPU parity: every kernel's output vs the CPU oracle on the same seeded
inputs, through the C ABI.  Bit-exact where the kernel's operation order is
fixed (suite kernels, work-removed twins); within 1e-5 of the FP64
reference, relative to sum |terms| (condition-aware), for matmul, DG and
stencil.  Buffers carry guard bands that must stay untouched."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import pm_inputs  # noqa: E402
import paper_1904_09538_gb300 as pm  # noqa: E402
from oracle import refs  # noqa: E402

TOL = 1e-5
GUARD = 64
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SENT = {np.float32: 1234.5, np.float64: -4321.25}


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


class Guarded:
    """Device buffer with GUARD sentinel elements on both sides."""

    def __init__(self, n, dtype, data=None):
        tdt = torch.float32 if dtype == np.float32 else torch.float64
        self.n, self.dtype = n, dtype
        self.full = torch.full((n + 2 * GUARD,), SENT[dtype], dtype=tdt, device=dev())
        self.view = self.full[GUARD:GUARD + n]
        if data is not None:
            self.view.copy_(torch.from_numpy(np.ascontiguousarray(data).ravel()))

    def check(self):
        f = self.full.cpu().numpy()
        assert np.all(f[:GUARD] == SENT[self.dtype]) and np.all(f[GUARD + self.n:] == SENT[self.dtype]), "guard hit"

    def get(self):
        return self.view.cpu().numpy()


def run_kernel(kernel, inputs, **params):
    """Allocate guarded buffers per pm_kernel_buffers, launch, return outputs."""
    dev()
    spec = pm.kernel_buffers(kernel, **params)
    bufs, it = [], iter(inputs)
    for b in spec:
        if b["role"] == "in":
            bufs.append(Guarded(b["elems"], b["dtype"], next(it)))
        else:
            bufs.append(Guarded(b["elems"], b["dtype"]))
    pm.launch(kernel, [b.view for b in bufs], **params)
    torch.cuda.synchronize()
    for b in bufs:
        b.check()
    return [b.get() for b, s in zip(bufs, spec) if s["role"] == "out"]


@pytest.mark.parametrize("dtype,vec,s,L,shape,W", [
    (0, 0, 1, 1, 0, 16), (0, 0, 2, 2, 0, 16), (0, 1, 1, 2, 0, 16), (0, 1, 32, 4, 0, 16), (1, 0, 4, 3, 0, 16),
    (1, 1, 1, 4, 0, 16), (0, 0, 1, 3, 1, 64), (1, 1, 16, 1, 0, 16), (0, 1, 8, 2, 1, 128)])
def test_stream_bitexact(dtype, vec, s, L, shape, W):
    N = 1 << 17
    dt = np.float32 if dtype == 0 else np.float64
    xs = [pm_inputs.uniform((N,), 40 + a, dtype=dt) for a in range(L)]
    (out,) = run_kernel("stream", xs, dtype=dtype, vec=vec, N=N, s=s, L=L, shape=shape, W=W)
    assert np.array_equal(out, refs.stream(xs))


@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("op", [0, 1, 2])
@pytest.mark.parametrize("F", [32, 1024, 3200])
def test_fma_bitexact(dtype, op, F):
    G = 5
    dt = np.float32 if dtype == 0 else np.float64
    seed = pm_inputs.uniform((G * 256,), 7, dtype=dt)
    (out,) = run_kernel("fma", [seed], dtype=dtype, op=op, F=F, G=G)
    assert np.array_equal(out, refs.fma(seed, op, F))


@pytest.mark.parametrize("kernel,params", [("smem", dict(R=64, sync=0, G=7)), ("smem", dict(R=256, sync=1, G=3)),
                                           ("barrier", dict(B=0, G=2)), ("barrier", dict(B=33, G=9)),
                                           ("overlap", dict(m=0, N=2048)), ("overlap", dict(m=12, N=4096))])
def test_copy_kernels(kernel, params):
    n = pm.kernel_buffers(kernel, **params)[0]["elems"]
    x = pm_inputs.uniform((n,), 3)
    (out,) = run_kernel(kernel, [x], **params)
    assert np.array_equal(out, x)


def test_empty():
    run_kernel("empty", [], G=4096)


def cond_err(out, ref, rabs):
    return float(np.max(np.abs(out.astype(np.float64) - ref) / np.maximum(rabs, 1e-300)))


@pytest.mark.parametrize("kernel", ["mm_pf", "mm_nopf"])
@pytest.mark.parametrize("n", [16, 48, 128, 768])
def test_matmul(kernel, n):
    a, b = pm_inputs.uniform((n, n), 1), pm_inputs.uniform((n, n), 2)
    (c,) = run_kernel(kernel, [a, b], n=n)
    ref, rabs = refs.matmul(a, b)
    assert cond_err(c.reshape(n, n), ref, rabs) <= TOL


@pytest.mark.parametrize("kernel", ["mm_pf_a", "mm_pf_b", "mm_nopf_a", "mm_nopf_b"])
@pytest.mark.parametrize("n", [16, 80])
def test_matmul_twins_bitexact(kernel, n):
    x = pm_inputs.uniform((n, n), 5)
    (d,) = run_kernel(kernel, [x], n=n)
    assert np.array_equal(d.reshape(n, n), refs.mm_twin(kernel, x))


DG_CASES = [(20, 64, 16, 16), (35, 96, 32, 8), (56, 32, 16, 16), (84, 64, 32, 8), (1, 16, 16, 16), (33, 64, 32, 8)]


@pytest.mark.parametrize("kernel", ["dg_nopf", "dg_dmpf"])
@pytest.mark.parametrize("Np,Nel,L0,L1", DG_CASES)
def test_dg(kernel, Np, Nel, L0, L1):
    D, u = pm_inputs.normal((3, Np, Np), 11), pm_inputs.normal((Nel, Np), 12)
    (res,) = run_kernel(kernel, [D, u], Np=Np, Nel=Nel, L0=L0, L1=L1)
    ref, rabs = refs.dg(D, u)
    assert cond_err(res.reshape(3, Nel, Np), ref, rabs) <= TOL


@pytest.mark.parametrize("kernel", ["dg_nopf_u", "dg_nopf_dm", "dg_dmpf_u", "dg_dmpf_dm"])
@pytest.mark.parametrize("Np,Nel,L0,L1", DG_CASES[:4])
def test_dg_twins_bitexact(kernel, Np, Nel, L0, L1):
    D, u = pm_inputs.normal((3, Np, Np), 13), pm_inputs.normal((Nel, Np), 14)
    ins = [u] if kernel.endswith("_u") else [D]
    (d,) = run_kernel(kernel, ins, Np=Np, Nel=Nel, L0=L0, L1=L1)
    assert np.array_equal(d.reshape(-1, Nel), refs.dg_twin(kernel, D, u, L0, L1))


def test_dg_res_twin_writes_zeros():
    (r,) = run_kernel("dg_res", [], Np=20, Nel=32, L0=16, L1=16)
    assert np.all(r == 0)
    (r,) = run_kernel("dg_dmpft_res", [], Np=35, Nel=64, L0=32, L1=8)
    assert np.all(r == 0)


@pytest.mark.parametrize("Np,Nel,L0,L1", [c for c in DG_CASES if c[2] == c[3]] + [(84, 48, 16, 16), (17, 16, 16, 16)])
def test_dg_upf(Np, Nel, L0, L1):
    D, u = pm_inputs.normal((3, Np, Np), 15), pm_inputs.normal((Nel, Np), 16)
    (res,) = run_kernel("dg_upf", [D, u], Np=Np, Nel=Nel, L0=L0, L1=L1)
    ref, rabs = refs.dg(D, u)
    assert cond_err(res.reshape(3, Nel, Np), ref, rabs) <= TOL


@pytest.mark.parametrize("Np,Nel,L0,L1", DG_CASES)
def test_dg_dmpft(Np, Nel, L0, L1):
    # transposed layouts: the kernel reads uT[j, k] and writes resT[m, i, k]
    D, u = pm_inputs.normal((3, Np, Np), 17), pm_inputs.normal((Nel, Np), 18)
    (resT,) = run_kernel("dg_dmpft", [D, np.ascontiguousarray(u.T)], Np=Np, Nel=Nel, L0=L0, L1=L1)
    ref, rabs = refs.dg(D, u)
    assert cond_err(resT.reshape(3, Np, Nel).transpose(0, 2, 1), ref, rabs) <= TOL


@pytest.mark.parametrize("kernel", ["dg_upf_u", "dg_dmpft_u"])
@pytest.mark.parametrize("Np,Nel", [(20, 64), (84, 64), (35, 32)])
def test_dg_new_twins_bitexact(kernel, Np, Nel):
    D, u = pm_inputs.normal((3, Np, Np), 19), pm_inputs.normal((Nel, Np), 20)
    uk = np.ascontiguousarray(u.T) if kernel == "dg_dmpft_u" else u
    (d,) = run_kernel(kernel, [uk], Np=Np, Nel=Nel, L0=16, L1=16)
    assert np.array_equal(d.reshape(-1, Nel), refs.dg_twin(kernel, D, uk, 16, 16))


@pytest.mark.parametrize("kernel", ["fd_tile", "fd_direct", "fd_tile18"])
@pytest.mark.parametrize("n", [1, 13, 14, 16, 29, 100, 1024])
def test_stencil(kernel, n):
    u = pm_inputs.uniform((n + 2, n + 2), 21)
    (r,) = run_kernel(kernel, [u], n=n, c0=-4.0, c1=1.0)
    ref, rabs = refs.stencil(u, -4.0, 1.0)
    assert cond_err(r.reshape(n, n), ref, rabs) <= TOL


@pytest.mark.parametrize("kernel", ["fd_tile_u", "fd_direct_u", "fd_tile18_u"])
@pytest.mark.parametrize("n", [13, 45, 100])
def test_stencil_twins_bitexact(kernel, n):
    u = pm_inputs.uniform((n + 2, n + 2), 22)
    (d,) = run_kernel(kernel, [u], n=n)
    want = refs.fd_twin(kernel, u)
    assert np.array_equal(d.reshape(want.shape), want)


@pytest.mark.parametrize("kernel", ["fd_tile_res", "fd_direct_res", "fd_tile18_res"])
def test_stencil_res_twins(kernel):
    (r,) = run_kernel(kernel, [], n=37)
    assert np.all(r == 0)


# ---------------------------------------------------------------- full sizes, sampled
def test_stream_full_size_sampled():
    d = dev()
    N = 1 << 28
    L = 2
    gen = torch.Generator(device=d)
    gen.manual_seed(77)
    xs = [torch.rand(N, device=d, generator=gen) * 2 - 1 for _ in range(L)]
    out = torch.empty(N, device=d)
    pm.launch("stream", xs + [out], N=N, L=L, vec=1)
    torch.cuda.synchronize()
    idx = torch.from_numpy(pm_inputs.integers((4096,), 5, 0, N - 1)).to(d)
    samples = [x[idx].cpu().numpy() for x in xs]
    assert np.array_equal(out[idx].cpu().numpy(), refs.stream(samples))
    del xs, out


def test_dg_full_size_sampled():
    Np, Nel = 84, 1 << 18
    D, u = pm_inputs.normal((3, Np, Np), 31), pm_inputs.normal((Nel, Np), 32)
    d = dev()
    res = torch.empty(3 * Nel * Np, device=d)
    for kernel, L0, L1 in (("dg_dmpf", 16, 16), ("dg_nopf", 32, 8), ("dg_upf", 16, 16), ("dg_dmpft", 32, 8)):
        uk = np.ascontiguousarray(u.T) if kernel == "dg_dmpft" else u
        pm.launch(kernel, [torch.from_numpy(D).to(d), torch.from_numpy(uk).to(d), res], Np=Np, Nel=Nel, L0=L0, L1=L1)
        torch.cuda.synchronize()
        ks = np.unique(pm_inputs.integers((512,), 33, 0, Nel - 1))
        ref, rabs = refs.dg(D, u[ks])
        full = res.cpu().numpy()
        got = (full.reshape(3, Np, Nel).transpose(0, 2, 1) if kernel == "dg_dmpft" else full.reshape(3, Nel, Np))[:, ks, :]
        assert cond_err(got, ref, rabs) <= TOL


def test_stencil_full_size_sampled():
    n = 16384
    d = dev()
    gen = torch.Generator(device=d)
    gen.manual_seed(5)
    u = torch.rand((n + 2) * (n + 2), device=d, generator=gen) * 2 - 1
    r = torch.empty(n * n, device=d)
    for kernel in ("fd_tile", "fd_direct", "fd_tile18"):
        pm.launch(kernel, [u, r], n=n, c0=-4.0, c1=1.0)
        torch.cuda.synchronize()
        for i0 in (0, 7777, n - 9):
            win = u.view(n + 2, n + 2)[i0:i0 + 11].cpu().numpy()
            ref, rabs = refs.stencil_rows(win, -4.0, 1.0)
            got = r.view(n, n)[i0:i0 + 9].cpu().numpy()
            assert cond_err(got, ref, rabs) <= TOL


# ---------------------------------------------------------------- timing entry points
def test_run_timing_and_host_path():
    d = dev()
    N = 1 << 20
    xs = [pm_inputs.uniform((N,), 60 + a) for a in range(2)]
    bufs = [torch.from_numpy(x).to(d) for x in xs] + [torch.empty(N, device=d)]
    tm = pm.run("stream", bufs, warmup=3, trials=60, want_trials=True, N=N, L=2)
    assert tm["n_trials"] == 60 and tm["mean_ms"] > 0 and len(tm["trials_ms"]) == 60
    assert tm["min_ms"] <= tm["median_ms"] <= tm["max_ms"]
    host_out = np.zeros(N, np.float32)
    th = pm.run_host("stream", xs + [host_out], warmup=1, trials=3, N=N, L=2)
    assert th["copy_ms"] > 0
    assert np.array_equal(host_out, refs.stream(xs))


def test_launch_errors():
    d = dev()
    x = torch.zeros(1024, device=d)
    with pytest.raises(pm.PMError):
        pm.launch("stream", [x], N=1024, L=1)               # too few buffers
    with pytest.raises(pm.PMError):
        pm.launch("stream", [x, x], N=1000, L=1)            # N not a multiple of 256
    with pytest.raises(pm.PMError):
        pm.launch("mm_pf", [x, x, x], n=24)                 # n not a multiple of 16


# ---------------------------------------------------------------- autotuning families
_MM768 = {}


def _mm768():
    if not _MM768:
        n = 768
        a, b = pm_inputs.uniform((n, n), 91), pm_inputs.uniform((n, n), 92)
        ref, rabs = refs.matmul(a, b)
        _MM768.update(a=a, b=b, ref=ref, rabs=rabs)
    return _MM768


@pytest.mark.parametrize("BM", [64, 96, 128, 256])
@pytest.mark.parametrize("BN", [64, 128, 256])
@pytest.mark.parametrize("BK", [32, 64])
def test_mm_simt_all_tiles(BM, BN, BK):
    d = _mm768()
    (c,) = run_kernel("mm_simt", [d["a"], d["b"]], n=768, BM=BM, BN=BN, BK=BK)
    assert cond_err(c.reshape(768, 768), d["ref"], d["rabs"]) <= TOL


@pytest.mark.parametrize("V", [4, 8])
@pytest.mark.parametrize("BX", [32, 64, 128])
@pytest.mark.parametrize("BY", [4, 8, 16, 32])
def test_fd_block_all_tiles(BX, BY, V):
    n = 256
    u = pm_inputs.uniform((n + 2, n + 4), 71)      # row pitch n + 4; columns n+2, n+3 are padding
    (r,) = run_kernel("fd_block", [u], n=n, BX=BX, BY=BY, V=V, c0=-4.0, c1=1.0)
    ref, rabs = refs.stencil(np.ascontiguousarray(u[:, :n + 2]), -4.0, 1.0)
    assert cond_err(r.reshape(n, n), ref, rabs) <= TOL


def test_kernel_resources_report_launch_shape():
    dev()
    r = pm.resources("mm_simt", n=768, BM=128, BN=64, BK=32)
    assert r["threads_per_block"] == (128 // 8) * (64 // 8) and r["grid_blocks"] == (768 // 64) * (768 // 128)
    assert r["dynamic_smem_bytes"] == (128 + 4 + 64) * 32 * 4 and r["blocks_per_sm"] >= 1 and r["sm_count"] > 0
    r = pm.resources("fd_block", n=1024, BX=64, BY=8)
    assert r["threads_per_block"] == 16 * 8 and r["grid_blocks"] == (1024 // 64) * (1024 // 8)
    r = pm.resources("stream", N=1 << 20, L=2, vec=1)
    assert r["threads_per_block"] == 256 and r["regs_per_thread"] > 0
    r = pm.resources("mm_tc", n=512)
    assert r["threads_per_block"] == 128 and r["grid_blocks"] == (512 // 256) * (512 // 128)


def test_suite_wave_sizes_match_residency():
    # the arithmetic suite sizes its grids in whole waves of the resident
    # CTAs per SM; the compiled kernels must have that residency
    from paper_1904_09538_gb300 import suite as S
    dev()
    for op in (0, 1, 2):
        r = pm.resources("fma", dtype=0, op=op, F=1024, G=912)
        assert r["blocks_per_sm"] == S.FMA_F32_PER_SM and r["sm_count"] == S.SM_COUNT, r
    r = pm.resources("fma", dtype=1, op=2, F=1024, G=456)
    assert r["blocks_per_sm"] == S.FMA_F64_PER_SM, r
    for k, p in S.generate(["ops"]):
        per_sm = S.FMA_F32_PER_SM if p["dtype"] == 0 else S.FMA_F64_PER_SM
        assert p["G"] % (per_sm * S.SM_COUNT) == 0 or p["G"] < per_sm * S.SM_COUNT, p
    for k, p in S.generate(["lmem"]) + S.generate(["sync"]):
        assert pm.resources(k, **p)["blocks_per_sm"] == S.RESIDENT // S.SM_COUNT, (k, p)


@pytest.mark.parametrize("T", [16, 18])
def test_smem2d_moves_values_exactly(T):
    G = 7
    x = pm_inputs.uniform((G * T * T,), 81)
    (r,) = run_kernel("smem2d", [x], R=64, T=T, G=G)
    assert np.array_equal(r, x)


def test_run_host_batch_pipelines_and_orders_aliased_buffers():
    dev()
    N = 1 << 20
    x0, x1 = pm_inputs.uniform((N,), 91), pm_inputs.uniform((N,), 92)
    o0 = np.zeros(N, np.float32)
    o1 = np.zeros(N, np.float32)
    y = [pm_inputs.uniform((N,), 93 + a) for a in range(4)]
    o2 = np.zeros(N, np.float32)
    jobs = [("stream", [x0, x1, o0], dict(N=N, L=2, vec=1)),
            ("stream", [o0, o1], dict(N=N, L=1, vec=1)),        # reads job 0's output: copies serialised
            ("stream", y + [o2], dict(N=N, L=4, vec=1))]
    tms, copy_ms = pm.run_host_batch(jobs, warmup=1, trials=3)
    want = refs.stream([x0, x1])
    assert np.array_equal(o0, want) and np.array_equal(o1, want)
    assert np.array_equal(o2, refs.stream(y))
    assert len(tms) == 3 and all(t["n_trials"] == 3 and t["mean_ms"] > 0 for t in tms) and copy_ms > 0


def test_run_host_batch_shared_input_regions():
    # several jobs read prefixes of the same host buffers (shared regions,
    # copied once); a region that an earlier job's output writes is not
    # shared, and its readers see the written values
    dev()
    N = 1 << 18
    X, Y = pm_inputs.uniform((4 * N,), 101), pm_inputs.uniform((4 * N,), 102)
    P = pm_inputs.uniform((N,), 103)
    Z = np.zeros(2 * N, np.float32)
    oa, ob, oc, o1, o2 = (np.zeros(n, np.float32) for n in (N, 2 * N, 2 * N, N, N))
    jobs = [("stream", [X[:N], Y[:N], oa], dict(N=N, L=2, vec=1)),
            ("stream", [X[:2 * N], ob], dict(N=2 * N, L=1, vec=1)),
            ("stream", [X[:4 * N], None], dict(N=4 * N, L=1, vec=1)),     # output left on the device
            ("stream", [Y[:2 * N], X[:2 * N], oc], dict(N=2 * N, L=2, vec=0)),
            ("stream", [P, Z[:N]], dict(N=N, L=1, vec=1)),               # writes the host region read next
            ("stream", [Z[:N], o1], dict(N=N, L=1, vec=1)),
            ("stream", [Z[:N], o2], dict(N=N, L=1, vec=0))]
    h2d, d2h = pm.run_host_batch_bytes(jobs)
    # X once (4N), Y once (2N), P, and Z[:N] twice (not shared)
    assert h2d == 4 * (4 * N + 2 * N + N + 2 * N) and d2h == 4 * (N + 2 * N + 2 * N + N + N + N)
    tms, copy_ms = pm.run_host_batch(jobs, warmup=1, trials=2)
    assert np.array_equal(oa, refs.stream([X[:N], Y[:N]]))
    assert np.array_equal(ob, X[:2 * N])
    assert np.array_equal(oc, refs.stream([Y[:2 * N], X[:2 * N]]))
    assert np.array_equal(Z[:N], P) and np.array_equal(o1, P) and np.array_equal(o2, P)
    assert len(tms) == 7 and all(t["n_trials"] == 2 for t in tms) and copy_ms > 0


# DG tile (128 elements per CTA, D staged transposed in shared memory, the
# u tile by one bulk copy, ceil(Np / ceil(Np / 16)) column lanes): odd Np
# (re-laid rows), Np with padded rows (33, 35, 63, 95) and ragged Nel (last
# tile of 4..124 elements), guard bands checked by run_kernel
@pytest.mark.parametrize("Np,Nel", [(20, 132), (35, 256), (56, 4), (84, 260), (1, 8), (17, 132), (96, 136),
                                    (84, 1024), (16, 384), (33, 132), (63, 200), (95, 8), (2, 12)])
def test_dg_tile(Np, Nel):
    D, u = pm_inputs.normal((3, Np, Np), 21), pm_inputs.normal((Nel, Np), 22)
    (res,) = run_kernel("dg_tile", [D, u], Np=Np, Nel=Nel)
    ref, rabs = refs.dg(D, u)
    assert cond_err(res.reshape(3, Nel, Np), ref, rabs) <= TOL


# dg_tc: the tensor-core form (TF32 head/remainder split, three passes);
# ragged last tiles, one and three CTAs per m-group (the ring and the two
# accumulators wrap many times), every supported node count
@pytest.mark.parametrize("Np,Nel,P", [(20, 132, 0), (20, 4, 0), (35, 256, 0), (56, 260, 0), (84, 1024, 0),
                                      (84, 132, 0), (4, 8, 0), (10, 300, 0), (20, 4100, 1), (35, 1028, 3),
                                      (56, 2052, 1), (84, 3076, 2), (10, 1 << 12, 1), (4, 1 << 12, 0)])
@pytest.mark.parametrize("A", [0, 1])
def test_dg_tc(Np, Nel, P, A):
    D, u = pm_inputs.normal((3, Np, Np), 21), pm_inputs.normal((Nel, Np), 22)
    (res,) = run_kernel("dg_tc", [D, u], Np=Np, Nel=Nel, P=P, A=A)
    ref, rabs = refs.dg(D, u)
    assert cond_err(res.reshape(3, Nel, Np), ref, rabs) <= TOL


@pytest.mark.parametrize("Np", [20, 35, 56, 84])
@pytest.mark.parametrize("A", [0, 1])
def test_dg_tc_full_size_sampled_and_timed(Np, A):
    Nel = 1 << 18
    D, u = pm_inputs.normal((3, Np, Np), 41), pm_inputs.normal((Nel, Np), 42)
    d = dev()
    res = torch.full((3 * Nel * Np,), float("nan"), device=d)
    bufs = [torch.from_numpy(D).to(d), torch.from_numpy(u).to(d), res]
    tm = pm.run("dg_tc", bufs, warmup=2, trials=5, Np=Np, Nel=Nel, A=A)
    ks = np.unique(np.concatenate([pm_inputs.integers((512,), 43, 0, Nel - 1), [0, Nel - 1]]))
    ref, rabs = refs.dg(D, u[ks])
    got = res.cpu().numpy().reshape(3, Nel, Np)[:, ks, :]
    assert cond_err(got, ref, rabs) <= TOL and tm["mean_ms"] > 0


@pytest.mark.parametrize("Np,launches", [(56, 40), (84, 16), (35, 16)])
def test_dg_tc_tensor_memory_form_repeated_launches_every_output(Np, launches):
    # the u operand in tensor memory, many persistent work-groups (one wave),
    # every output of every launch against the oracle: the raw stages are
    # reused from the third tile on, and a converter that frees a stage before
    # its reads are ordered against the next copy corrupts rows of that tile
    # now and then, so one launch is not enough
    Nel = 1 << 18
    D, u = pm_inputs.normal((3, Np, Np), 51), pm_inputs.normal((Nel, Np), 52)
    ref, rabs = refs.dg(D, u)
    d = dev()
    ref_d = torch.from_numpy(ref).to(d)
    inv_d = 1.0 / torch.from_numpy(np.maximum(rabs, 1e-300)).to(d)
    bufs = [torch.from_numpy(D).to(d), torch.from_numpy(u).to(d), torch.empty(3 * Nel * Np, device=d)]
    worst = 0.0
    for _ in range(launches):
        bufs[2].fill_(float("nan"))
        pm.run("dg_tc", bufs, warmup=0, trials=1, Np=Np, Nel=Nel, A=1)
        err = ((bufs[2].view(3, Nel, Np).double() - ref_d).abs() * inv_d).nan_to_num(nan=float("inf"))
        worst = max(worst, float(err.max()))
    assert worst <= TOL, worst


def test_tma_kernel_resources_as_first_cuda_call():
    # a resource query of a TMA-staged kernel encodes a tensor map; as the
    # first CUDA call of a process (no context current yet) it must work too
    dev()
    code = ("import paper_1904_09538_gb300 as pm; "
            "r = pm.resources('fd_block', n=8192, BX=64, BY=16, V=8); "
            "assert r['grid_blocks'] == (8192 // 64) * (8192 // 16), r; "
            "r = pm.resources('mm_tc', n=1024); assert r['grid_blocks'] > 0; print('ok')")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stderr[-2000:]


def test_bounded_wait_gives_up_and_reports_timeout():
    # failure detection without a GPU fault: a wait on an mbarrier phase that
    # nothing completes gives up after its poll limit through the dg_tile
    # kernel's wait and error word; the host reads PM_ETIMEOUT, clears the
    # word, and the context keeps working (a dg_tile launch afterwards is
    # exact and reports no timeout); polls out of range are refused
    dev()
    L = pm.lib()
    for polls in (1, 4096):
        assert L.pm_test_bounded_wait(polls, None) == -6, pm.lib().pm_last_error()
    assert L.pm_test_bounded_wait(0, None) == -1 and L.pm_test_bounded_wait(1 << 21, None) == -1
    D, u = pm_inputs.normal((3, 20, 20), 21), pm_inputs.normal((132, 20), 22)
    (res,) = run_kernel("dg_tile", [D, u], Np=20, Nel=132)
    ref, rabs = refs.dg(D, u)
    assert cond_err(res.reshape(3, 132, 20), ref, rabs) <= TOL
    d = dev()
    bufs = [torch.from_numpy(D).to(d), torch.from_numpy(u).to(d), torch.empty(3 * 132 * 20, device=d)]
    tm = pm.run("dg_tile", bufs, warmup=0, trials=2, Np=20, Nel=132)   # reads the error word
    assert tm["n_trials"] == 2


@pytest.mark.parametrize("Np", [20, 35, 56, 84])
def test_dg_tile_full_size_sampled_and_timed(Np):
    Nel = 1 << 18
    D, u = pm_inputs.normal((3, Np, Np), 41), pm_inputs.normal((Nel, Np), 42)
    d = dev()
    res = torch.empty(3 * Nel * Np, device=d)
    bufs = [torch.from_numpy(D).to(d), torch.from_numpy(u).to(d), res]
    tm = pm.run("dg_tile", bufs, warmup=2, trials=5, Np=Np, Nel=Nel)
    ks = np.unique(pm_inputs.integers((512,), 43, 0, Nel - 1))
    ref, rabs = refs.dg(D, u[ks])
    got = res.cpu().numpy().reshape(3, Nel, Np)[:, ks, :]
    assert cond_err(got, ref, rabs) <= TOL and tm["mean_ms"] > 0


def test_dg_tile_resources():
    dev()
    r = pm.resources("dg_tile", Np=84, Nel=1 << 18)
    # Np = 84: NB = 6 columns per thread over 14 x-lanes (no padded rows), 14 x 16 threads
    assert r["threads_per_block"] == 14 * 16 and r["grid_blocks"] == 3 * (1 << 18) // 128
    assert r["local_bytes_per_thread"] == 0 and r["blocks_per_sm"] >= 2
    assert r["dynamic_smem_bytes"] >= (128 * 84 + 84 * 98) * 4


def test_run_host_batch_outputs_left_on_device():
    # a NULL output pointer leaves that output on the device (timings only);
    # a NULL input pointer is an error
    dev()
    N = 1 << 16
    x = np.ones(N, dtype=np.float32)
    out = np.zeros(N, dtype=np.float32)
    tms, cms = pm.run_host_batch([("stream", [x, None], {"N": N}), ("stream", [x, out], {"N": N}),
                                  ("fma", [x[:256 * 4], None], {"F": 1024, "G": 4})], trials=2)
    assert len(tms) == 3 and all(t["n_trials"] == 2 and t["mean_ms"] > 0 for t in tms) and cms >= 0
    assert np.array_equal(out, x)
    with pytest.raises(pm.PMError):
        pm.run_host_batch([("stream", [None, out], {"N": N})])


# ---------------------------------------------------------------- the timed suite, every variant at its size
def test_every_suite_variant_at_timed_size_sampled():
    # each of the calibration suite's variants in the size and launch shape the
    # suite is timed in (arrays up to 2^28 elements), inputs ~U[-1, 1] from a
    # seeded device generator, outputs poisoned with NaN first: 2048 sampled
    # outputs per variant must equal the oracle's bit for bit (an element the
    # kernel never wrote stays NaN and fails)
    from paper_1904_09538_gb300 import suite as S
    d = dev()
    gen = torch.Generator(device=d)
    checked = 0
    for vi, (k, p) in enumerate(S.generate(["suite"])):
        gen.manual_seed(1000 + vi)
        spec = pm.kernel_buffers(k, **p)
        bufs = []
        for b in spec:
            tdt = torch.float32 if b["dtype"] == np.float32 else torch.float64
            if b["role"] == "in":
                bufs.append(torch.rand(b["elems"], device=d, dtype=tdt, generator=gen) * 2 - 1)
            else:
                bufs.append(torch.full((b["elems"],), float("nan"), device=d, dtype=tdt))
        pm.launch(k, bufs, **p)
        torch.cuda.synchronize()
        ins = [t for t, b in zip(bufs, spec) if b["role"] == "in"]
        outs = [t for t, b in zip(bufs, spec) if b["role"] == "out"]
        if k == "empty":
            assert not outs
            continue
        (out,) = outs
        n = out.numel()
        idx_np = np.unique(pm_inputs.integers((2048,), 2000 + vi, 0, n - 1))
        idx = torch.from_numpy(idx_np).to(d)
        got = out[idx].cpu().numpy()
        samples = [x[idx].cpu().numpy() for x in ins]
        if k == "stream":
            want = refs.stream(samples)
        elif k == "fma":
            want = refs.fma(samples[0], p["op"], p["F"])
        else:   # local-memory shuffle, barrier and overlap kernels move each value back to its place
            want = samples[0]
        assert np.array_equal(got, want), (k, p)
        checked += 1
        del bufs, ins, outs, out
    assert checked == 230 - 13   # every variant but the 13 empty kernels has an output


# ---------------------------------------------------------------- matmuls at their sweep sizes, sampled rows
def _mm_sampled(kernel, n, seed, **params):
    d = dev()
    a, b = pm_inputs.uniform((n, n), seed), pm_inputs.uniform((n, n), seed + 1)
    c = torch.full((n * n,), float("nan"), device=d)
    pm.launch(kernel, [torch.from_numpy(a).to(d), torch.from_numpy(b).to(d), c], n=n, **params)
    torch.cuda.synchronize()
    # one sampled row in each of 16 bands of the rows, all columns
    rows = np.arange(0, n, n // 16) + pm_inputs.integers((16,), seed + 2, 0, n // 16 - 1)
    ref, rabs = refs.matmul_rows(a[rows], b)
    got = c.view(n, n)[torch.from_numpy(rows).to(d)].cpu().numpy()
    return cond_err(got, ref, rabs)


@pytest.mark.parametrize("kernel", ["mm_pf", "mm_nopf"])
def test_matmul_largest_sweep_size_sampled(kernel):
    # n = 4096, the largest size of the matmul study and sweep
    assert _mm_sampled(kernel, 4096, 90) <= TOL


@pytest.mark.parametrize("BM,BN,BK", [(128, 128, 32), (96, 256, 64), (64, 64, 32)])
def test_mm_simt_autotune_size_sampled(BM, BN, BK):
    # n = 7680, the size the SIMT tile shapes are ranked at
    assert _mm_sampled("mm_simt", 7680, 95, BM=BM, BN=BN, BK=BK) <= TOL


@pytest.mark.parametrize("BX,BY,V", [(32, 16, 8), (128, 32, 8), (64, 4, 4)])
def test_fd_block_ranking_size_sampled(BX, BY, V):
    # n = 16384, the size the stencil tile shapes are ranked at (row pitch
    # n + 4 as in the ranking); three row windows, one at each edge band
    n = 16384
    d = dev()
    gen = torch.Generator(device=d)
    gen.manual_seed(9)
    u = torch.rand((n + 2) * (n + 4), device=d, generator=gen) * 2 - 1
    r = torch.full((n * n,), float("nan"), device=d)
    pm.launch("fd_block", [u, r], n=n, BX=BX, BY=BY, V=V, c0=-4.0, c1=1.0)
    torch.cuda.synchronize()
    for i0 in (0, 8191, n - 9):
        win = u.view(n + 2, n + 4)[i0:i0 + 11, :n + 2].cpu().numpy()
        ref, rabs = refs.stencil_rows(np.ascontiguousarray(win), -4.0, 1.0)
        got = r.view(n, n)[i0:i0 + 9].cpu().numpy()
        assert cond_err(got, ref, rabs) <= TOL
