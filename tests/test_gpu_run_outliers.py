"""pm_run's outlier rule on the GPU.  The paper excludes anomalous timings
(about ten times the usual ones, Section "Results", experimental setup)
without stating a threshold; the library drops every trial above
outlier_factor x the median of all trials (default 5) and reports how many
it dropped.  Checked here against the per-trial times pm_run returns: the
median, the kept set, the count and the statistics of the kept trials."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1904_09538_gb300 as pm  # noqa: E402


def expected(trials_ms, factor):
    tr = np.asarray(trials_ms, dtype=np.float32).astype(np.float64)
    med = float(np.median(tr))          # mean of the two middle trials for an even count
    keep = tr if factor <= 0 else tr[~(tr > factor * med)]
    return med, keep


@pytest.mark.parametrize("factor", [0.0, 1.0, 1.02, 5.0])
def test_outlier_rule_matches_returned_trials(factor):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = torch.device("cuda:0")
    N = 1 << 22
    bufs = [torch.rand(N, device=d), torch.empty(N, device=d)]
    r = pm.run("stream", bufs, warmup=2, trials=60, outlier_factor=factor, want_trials=True, N=N, L=1)
    med, keep = expected(r["trials_ms"], factor)
    assert r["n_trials"] == 60 and len(r["trials_ms"]) == 60
    assert r["median_ms"] == med
    assert r["n_dropped"] == 60 - len(keep)
    assert r["mean_ms"] == pytest.approx(float(np.mean(keep)), rel=1e-12)
    assert r["min_ms"] == keep.min() and r["max_ms"] == keep.max()
    if factor <= 0:
        assert r["n_dropped"] == 0
    if factor == 1.0:
        # every trial above the median goes; at most half of 60 can be
        assert r["n_dropped"] == int(np.sum(np.asarray(r["trials_ms"], dtype=np.float64) > med)) <= 30


def test_outlier_factor_one_drops_the_slowest_trials():
    # a factor of 1 keeps exactly the trials at or below the median, so the
    # mean of what is kept cannot exceed the median and the maximum kept
    # trial is at most the median
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = torch.device("cuda:0")
    N = 1 << 20
    bufs = [torch.rand(N, device=d), torch.rand(N, device=d), torch.empty(N, device=d)]
    r = pm.run("stream", bufs, warmup=1, trials=41, outlier_factor=1.0, want_trials=True, N=N, L=2)
    assert r["max_ms"] <= r["median_ms"] and r["mean_ms"] <= r["median_ms"]
    assert r["n_trials"] - r["n_dropped"] >= 21      # an odd count: the median trial itself is kept
