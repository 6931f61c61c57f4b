"""Sample sharding of an ensemble across ranks (one GPU per rank).

The samples of an ensemble are independent (Sec. "Discrete approximation":
M IID samples advanced separately), so an ensemble of M samples splits into
contiguous sample ranges, one per rank, with no exchange during time stepping.
Only the statistics need an exchange:

  * per-sample results (E_m(t), spectra, structure functions): gathered;
  * pointwise ensemble mean / variance: each rank's (count, mean, M2) merged in
    FP64 by the pairwise update of Chan, Golub & LeVeque (1979), in rank order so
    the result does not depend on timing;
  * the one-point W1: the Q^3 restrictions (M x 12 KB at Q = 8) all-gathered.

The exchanges here are host-side (torch.distributed on CPU tensors, e.g. the gloo
backend); the data path itself has no collective.
"""
import numpy as np


def shard_range(M_total, rank, world):
    """Samples [lo, hi) of `rank`: contiguous, sizes differ by at most one."""
    base, extra = divmod(M_total, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def merge_mean_var(parts):
    """Merge per-rank (count, mean, M2) triples (M2 = sum of squared deviations) in the given
    order; returns (count, mean, unbiased variance)."""
    n, mean, m2 = None, None, None
    for cnt, mu, M2 in parts:
        cnt = int(cnt)
        if cnt == 0:
            continue
        mu = np.asarray(mu, dtype=np.float64)
        M2 = np.asarray(M2, dtype=np.float64)
        if n is None:
            n, mean, m2 = cnt, mu.copy(), M2.copy()
            continue
        tot = n + cnt
        delta = mu - mean
        mean = mean + delta * (cnt / tot)
        m2 = m2 + M2 + delta * delta * (n * cnt / tot)
        n = tot
    if n is None or n < 2:
        raise ValueError("variance needs at least two samples in total")
    return n, mean, m2 / (n - 1)


def allgather_concat(local, group=None):
    """Concatenate a per-rank numpy array along axis 0 over all ranks (rank order)."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(local))
    world = dist.get_world_size(group)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([t.shape[0]], dtype=torch.int64), group=group)
    mx = int(max(s.item() for s in sizes))
    pad = torch.zeros((mx,) + tuple(t.shape[1:]), dtype=t.dtype)
    pad[: t.shape[0]] = t
    bufs = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(bufs, pad, group=group)
    return np.concatenate([b[: int(s.item())].numpy() for b, s in zip(bufs, sizes)], axis=0)


def merged_mean_var(count, mean, var, group=None):
    """Ensemble mean / unbiased variance over all ranks from each rank's local ones."""
    m2 = np.asarray(var, dtype=np.float64) * max(count - 1, 0)
    stacked = np.concatenate([np.array([float(count)]), np.ravel(mean), np.ravel(m2)])
    allparts = allgather_concat(stacked[None, :], group)
    k = np.asarray(mean).size
    parts = [(row[0], row[1:1 + k], row[1 + k:]) for row in allparts]
    n, mu, v = merge_mean_var(parts)
    return n, mu.reshape(np.shape(mean)), v.reshape(np.shape(mean))
