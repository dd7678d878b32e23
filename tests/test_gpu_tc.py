"""BF16-in / FP32-accumulate tensor-core matmul (tcgen05, TMEM, TMA) vs the
FP64 oracle over the same bf16 inputs (uint16 bit patterns from pm_inputs):
within 1e-5 of sum_k |a_ik b_jk| per element."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import pm_inputs  # noqa: E402
import paper_1904_09538_gb300 as pm  # noqa: E402
from oracle import refs  # noqa: E402

TOL = 1e-5


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def run_tc(n, seed, pipe=1, kernel="mm_tc"):
    d = dev()
    a = pm_inputs.bf16_bits((n, n), seed)
    bt = pm_inputs.bf16_bits((n, n), seed + 1)
    ta = torch.from_numpy(a.view(np.int16)).to(d)
    tb = torch.from_numpy(bt.view(np.int16)).to(d)
    c = torch.full((n * n,), 7.5, device=d)
    if kernel == "mm_tc":
        pm.launch(kernel, [ta, tb, c], n=n, pipe=pipe)
    else:
        pm.launch(kernel, [ta, tb, c], n=n)
    torch.cuda.synchronize()
    return a, bt, c.cpu().numpy().reshape(n, n)


@pytest.mark.parametrize("pipe", [0, 1, 2])
@pytest.mark.parametrize("n", [256, 512, 1024])
def test_mm_tc_matches_oracle(n, pipe):
    a, bt, c = run_tc(n, 40 + n, pipe)
    ref, rabs = refs.matmul_bf16_tn(a, bt)
    err = np.abs(c.astype(np.float64) - ref) / rabs
    assert err.max() <= TOL, err.max()


@pytest.mark.parametrize("pipe", [0, 1, 2])
@pytest.mark.parametrize("n", [2304, 4352])
def test_mm_tc_partial_tile_groups(n, pipe):
    # 18 and 34 tile rows: the last group of 16 tile rows is partial; every
    # output row block must still be computed exactly once (sampled rows,
    # one from each tile row, all columns)
    a, bt, c = run_tc(n, 60 + n, pipe)
    rows = np.arange(0, n, 128) + pm_inputs.integers((n // 128,), 61, 0, 127)
    ref, rabs = refs.matmul_bf16_tn(a[rows], bt)
    err = np.abs(c[rows].astype(np.float64) - ref) / rabs
    assert err.max() <= TOL, err.max()


def test_mm_tc_full_size_sampled_and_timed():
    d = dev()
    n = 8192
    a = pm_inputs.bf16_bits((n, n), 3)
    bt = pm_inputs.bf16_bits((n, n), 4)
    ta = torch.from_numpy(a.view(np.int16)).to(d)
    tb = torch.from_numpy(bt.view(np.int16)).to(d)
    c = torch.empty(n * n, device=d)
    tm = pm.run("mm_tc", [ta, tb, c], warmup=2, trials=5, n=n)
    rows = np.unique(pm_inputs.integers((24,), 5, 0, n - 1))
    ref, rabs = refs.matmul_bf16_tn(a[rows][:, :], bt)  # rows of A times all of Bt: rectangular block
    got = c.view(n, n)[torch.from_numpy(rows).to(d)].cpu().numpy()
    assert np.max(np.abs(got - ref) / rabs) <= TOL
    assert tm["mean_ms"] > 0


# 256 x 256 tiles: two 128-row accumulators sharing each Bt box


@pytest.mark.parametrize("n", [256, 512, 1024])
def test_mm_tc256_matches_oracle(n):
    a, bt, c = run_tc(n, 140 + n, kernel="mm_tc256")
    ref, rabs = refs.matmul_bf16_tn(a, bt)
    err = np.abs(c.astype(np.float64) - ref) / rabs
    assert err.max() <= TOL, err.max()


@pytest.mark.parametrize("n", [2304, 4352])
def test_mm_tc256_partial_tile_groups(n):
    # 9 and 17 tile rows of 256: the last group of 8 tile rows is partial;
    # one sampled row from each 128-row half of every tile row
    a, bt, c = run_tc(n, 160 + n, kernel="mm_tc256")
    rows = np.arange(0, n, 128) + pm_inputs.integers((n // 128,), 161, 0, 127)
    ref, rabs = refs.matmul_bf16_tn(a[rows], bt)
    err = np.abs(c[rows].astype(np.float64) - ref) / rabs
    assert err.max() <= TOL, err.max()


def test_mm_tc256_full_size_sampled_and_timed():
    d = dev()
    n = 8192
    a = pm_inputs.bf16_bits((n, n), 13)
    bt = pm_inputs.bf16_bits((n, n), 14)
    ta = torch.from_numpy(a.view(np.int16)).to(d)
    tb = torch.from_numpy(bt.view(np.int16)).to(d)
    c = torch.empty(n * n, device=d)
    tm = pm.run("mm_tc256", [ta, tb, c], warmup=2, trials=5, n=n)
    rows = np.unique(pm_inputs.integers((24,), 15, 0, n - 1))
    ref, rabs = refs.matmul_bf16_tn(a[rows], bt)
    got = c.view(n, n)[torch.from_numpy(rows).to(d)].cpu().numpy()
    assert np.max(np.abs(got - ref) / rabs) <= TOL
    assert tm["mean_ms"] > 0


def test_mm_tc256_resources():
    dev()
    r = pm.resources("mm_tc256", n=8192)
    assert r["threads_per_block"] == 256 and r["blocks_per_sm"] == 1
    assert r["grid_blocks"] == (8192 // 256) ** 2
    assert r["local_bytes_per_thread"] == 0


@pytest.mark.parametrize("kernel", ["mm_tc", "mm_tc256"])
def test_tc_large_size_sampled(kernel):
    # n = 16384 (1 GiB of fp32 output): eight sampled rows, every column
    d = dev()
    n = 16384
    a = pm_inputs.bf16_bits((n, n), 23)
    bt = pm_inputs.bf16_bits((n, n), 24)
    ta = torch.from_numpy(a.view(np.int16)).to(d)
    tb = torch.from_numpy(bt.view(np.int16)).to(d)
    c = torch.empty(n * n, device=d)
    pm.launch(kernel, [ta, tb, c], n=n)
    torch.cuda.synchronize()
    rows = np.unique(pm_inputs.integers((8,), 25, 0, n - 1))
    ref, rabs = refs.matmul_bf16_tn(a[rows], bt)
    got = c.view(n, n)[torch.from_numpy(rows).to(d)].cpu().numpy()
    assert np.max(np.abs(got - ref) / rabs) <= TOL
