"""The allocation-free batched fit (pm_fit_batched_noalloc) against the
allocating one (pm_fit_batched), through the C ABI on the GPU.

Some callers cannot allocate GPU memory: processes whose device memory is
reserved by another framework's pooling allocator, and latency-critical loops
that cannot afford the device-wide synchronisation of cudaMalloc / cudaFree.
For them the library stages the fit in a static device array; this checks
that two calls in a row (different data each time, so nothing from the first
call leaks into the second) give the same parameters and statuses as the
regular entry point, and that oversized requests and non-finite start points
are refused up front."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import pm_inputs  # noqa: E402
import paper_1904_09538_gb300 as pm  # noqa: E402

TOL = 1e-6   # the parameter tolerance of the other fit tests

LIN = ("p_launch * f_sync_kernel_launch + p_group * f_thread_groups + p_add * f_op_float32_add + "
       "p_gmem * f_mem_access_global_float32")
CG = "(p_gmem * f_mem_access_global_float32)"
CO = "(p_madd * f_op_float32_madd)"
OVL = ("p_launch * f_sync_kernel_launch + %s * (tanh(p_edge * (%s - %s)) + 1) / 2 + "
       "%s * (tanh(p_edge * (%s - %s)) + 1) / 2" % (CG, CG, CO, CO, CO, CG))
TRUTH = dict(p_launch=5e-6, p_group=2e-9, p_add=4e-12, p_gmem=6e-12, p_madd=3e-12, p_edge=3e4)


def problem(seed, K=6):
    ls = pm_inputs.row_counts(K, seed, 40, 300)
    models, Xs, ts, p0s = [], [], [], []
    for k in range(K):
        m = pm.Model("f_wall_time", LIN if k % 2 == 0 else OVL)
        l = int(ls[k])
        X = pm_inputs.integers((l, len(m.features)), seed * 100 + k, 10 ** 5, 10 ** 7).astype(np.float64)
        X[:, 0] = 1.0
        if m.features[1] == "f_thread_groups":
            X[:, 1] = pm_inputs.integers((l,), seed * 100 + 50 + k, 100, 10 ** 4)
        pt = np.array([TRUTH[n] for n in m.params])
        t = m.predict(pt, X) * (1 + 1e-2 * pm_inputs.noise((l,), seed * 100 + 70 + k))
        models.append(m)
        Xs.append(X)
        ts.append(t)
        p0s.append(pt * 1.15)
    return models, Xs, ts, p0s


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b))))


def test_noalloc_matches_allocating_fit_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    for seed in (11, 12):   # two calls in a row, different data
        models, Xs, ts, p0s = problem(seed)
        ref, rrep = pm.fit_batched(models, Xs, ts, p0s, threads=128)
        got, grep = pm.fit_batched_noalloc(models, Xs, ts, p0s)
        for k in range(len(models)):
            assert grep[k]["status"] == rrep[k]["status"], (seed, k)
            assert rel(got[k], ref[k]) <= TOL, (seed, k, rel(got[k], ref[k]))
    # default start points (no p0) as well
    models, Xs, ts, _ = problem(13)
    ref, _ = pm.fit_batched(models, Xs, ts, None, threads=128)
    got, _ = pm.fit_batched_noalloc(models, Xs, ts, None)
    for k in range(len(models)):
        assert rel(got[k], ref[k]) <= TOL


def test_noalloc_rejects_oversized_request():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    m = pm.Model("f_wall_time", LIN)
    rows = pm.NOALLOC_SCRATCH_BYTES // (16 * len(m.features)) + 10
    X = np.ones((rows, len(m.features)))
    t = np.ones(rows)
    with pytest.raises(pm.PMError) as e:
        pm.fit_batched_noalloc([m], [X], [t])
    assert "limit" in str(e.value)


def test_noalloc_rejects_non_finite_start_point():
    # a NaN or an infinite start point is refused before anything is staged,
    # as pm_fit_batched refuses it; a valid call afterwards still works
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    models, Xs, ts, p0s = problem(14, K=2)
    for bad in (np.nan, np.inf):
        p0 = [p.copy() for p in p0s]
        p0[1][0] = bad
        with pytest.raises(pm.PMError) as e:
            pm.fit_batched_noalloc(models, Xs, ts, p0)
        assert e.value.status == -1 and "start point" in str(e.value)
    ref, _ = pm.fit_batched(models, Xs, ts, p0s, threads=128)
    got, _ = pm.fit_batched_noalloc(models, Xs, ts, p0s)
    for k in range(len(models)):
        assert rel(got[k], ref[k]) <= TOL
