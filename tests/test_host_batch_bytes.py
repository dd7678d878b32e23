"""pm_run_host_batch_bytes: what a host-buffer batch copies (host only, no
GPU).  Input buffers that start at the same host address in several jobs are
one region, copied once at the largest extent read; a region that a host
output of the batch overlaps is copied by each reader; outputs with a NULL
host pointer are not copied back."""
import numpy as np
import pytest

import paper_1904_09538_gb300 as pm

N = 1 << 12


def stream_job(ins, out, L=1, n=N):
    return ("stream", list(ins) + [out], dict(dtype=0, vec=0, N=n, s=1, L=L, shape=0))


def test_shared_prefixes_copied_once_at_largest_extent():
    a = np.zeros(4 * N, np.float32)
    b = np.zeros(4 * N, np.float32)
    jobs = [stream_job([a[:N]], None), stream_job([a[:4 * N], b[:2 * N]], None, L=2, n=2 * N),
            stream_job([a[:2 * N]], None, n=2 * N)]
    # a job reads as many elements as its kernel's buffer holds, whatever the
    # length of the host view passed (job 1 passes a 4N view of a for a 2N buffer)
    sizes = [[buf["elems"] for buf in pm.kernel_buffers(k, **p)] for k, _, p in jobs]
    assert sizes == [[N, N], [2 * N, 2 * N, 2 * N], [2 * N, 2 * N]]
    h2d, d2h = pm.run_host_batch_bytes(jobs)
    # region a: 3 readers, largest 2N floats; b: one reader (not shared), 2N floats
    assert h2d == 4 * (2 * N) + 4 * (2 * N)
    assert d2h == 0


def test_single_readers_and_outputs():
    a = np.zeros(N, np.float32)
    b = np.zeros(N, np.float32)
    o = np.zeros(N, np.float32)
    h2d, d2h = pm.run_host_batch_bytes([stream_job([a], o), stream_job([b], None)])
    assert h2d == 2 * 4 * N and d2h == 4 * N


def test_region_overlapped_by_an_output_is_not_shared():
    a = np.zeros(2 * N, np.float32)
    o = a[N:]        # job 0 writes into the second half of a
    jobs = [stream_job([a[:N]], o), stream_job([a[:N]], None), stream_job([a[:N]], None)]
    # a[:N] does not overlap a[N:]: shared, copied once
    assert pm.run_host_batch_bytes(jobs) == (4 * N, 4 * N)
    jobs = [stream_job([a[:N]], a[N // 2:N // 2 + N]), stream_job([a[:N]], None), stream_job([a[:N]], None)]
    # now the output overlaps the region: each reader copies it
    assert pm.run_host_batch_bytes(jobs) == (3 * 4 * N, 4 * N)


def test_same_region_twice_in_one_job():
    a = np.zeros(N, np.float32)
    assert pm.run_host_batch_bytes([stream_job([a, a], None, L=2)]) == (4 * N, 0)


def test_errors_match_the_batch_call():
    a = np.zeros(N, np.float32)
    with pytest.raises(pm.PMError):
        pm.run_host_batch_bytes([("stream", [a], dict(dtype=0, vec=0, N=N, s=1, L=1, shape=0))])   # missing output
    assert pm.run_host_batch_bytes([]) == (0, 0)
