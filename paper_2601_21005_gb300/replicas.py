"""Replica bookkeeping for one process per GPU (MC samples are independent, Sec. 2.3).

Each rank runs whole samples on its own GPU; nothing crosses ranks on the data path.  What the
ranks share is host-side: which sample indices each one draws, the slowest rank's time for the
whole-job throughput, and -- after the run, for one combined QP solve -- the per-sample rows
Sigma_i(t), X_i.  A `torch.distributed` process group (NCCL on GPUs, gloo on CPU) carries them.
"""

SAMPLE_STRIDE = 1000000


def sample_base(rank, stride=SAMPLE_STRIDE):
    """First sample index of a rank: rank r draws r * stride + i, so ranks never share a sample."""
    if rank < 0:
        raise ValueError('rank must be >= 0')
    return rank * stride


def sample_range(rank, n_samples, stride=SAMPLE_STRIDE):
    """Sample indices of a rank's n_samples draws."""
    if n_samples > stride:
        raise ValueError('n_samples exceeds the per-rank stride')
    b = sample_base(rank, stride)
    return range(b, b + n_samples)


def max_over_ranks(value, dist=None, device='cpu'):
    """The largest of the ranks' values (e.g. elapsed milliseconds); the value itself without a group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank_step, steps, world, ms):
    """Whole-job throughput: the units all ranks processed divided by the slowest rank's time."""
    if ms <= 0:
        raise ValueError('elapsed time must be positive')
    return units_per_rank_step * steps * world / (ms * 1e-3)


def gather_rows(sigma, x, dist=None):
    """Concatenate every rank's per-sample rows in rank order (after the timed run).

    sigma: [n][2N+1] complex128, x: [n] float64 (equal n on every rank).  Returns tensors on the
    inputs' device; without a group, the inputs themselves."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return sigma, x
    import torch
    w = dist.get_world_size()
    sr = torch.view_as_real(sigma.contiguous())
    parts_s = [torch.empty_like(sr) for _ in range(w)]
    parts_x = [torch.empty_like(x) for _ in range(w)]
    dist.all_gather(parts_s, sr)
    dist.all_gather(parts_x, x.contiguous())
    return torch.view_as_complex(torch.cat(parts_s).contiguous()), torch.cat(parts_x)
