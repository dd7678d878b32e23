"""Multi-GPU as replicas.  The path does not shard: calibration is per
device (Section "Introduction": parameters are fitted for one machine), and
two measurements must not share a GPU.  N processes, one per GPU, each run
the whole step on their own device; the only exchanges are the slowest
rank's elapsed time (the job's time), the summed work, and a host-side
gather of each rank's calibration report.  No data-path collective."""


def job_time(elapsed_s, dist, device):
    """Max over ranks of the timed region (seconds); `device` is where the
    reduction tensor lives (a CUDA device under NCCL, the CPU under gloo)."""
    import torch
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(elapsed_s)
    t = torch.tensor([float(elapsed_s)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, elapsed_s, dist, device):
    """(whole-job throughput = units of all ranks / slowest rank's time, that time)."""
    import torch
    t = job_time(elapsed_s, dist, device)
    total = float(units_per_rank)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        u = torch.tensor([total], dtype=torch.float64, device=device)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        total = float(u.item())
    return total / t, t


def gather_reports(report, dist):
    """Every rank's (JSON-able) calibration report, in rank order, on every rank."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [report]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, report)
    return out
