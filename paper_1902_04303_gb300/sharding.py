"""Sharding of encrypted GWAS work across ranks (one process per GPU).

After the covariate phase (Alg. 9, the preamble of Alg. 11) the SNP batches
of the loop in Alg. 11 are independent: each needs only the batch-invariant
state (Dup(w), Dup(w z'), and Dup(M_j) or Dup(X_c)/Dup((XA)_c)) and its own
tau SNP columns.  A job therefore shards by batch ranges.  Rank 0 encrypts
the inputs and runs the covariate phase; its batch-invariant state (about 66
MB at the paper's shape in the factored layout) is broadcast once to the
other ranks, which import it into their own job handle (same context seed,
hence the same keys); every rank then evaluates its own contiguous range of
batches, and the decrypted per-SNP numerators and denominators are gathered
once at the end (8 bytes x 2 per SNP).  Without the broadcast every rank
would repeat the deterministic fit.  The batches' data path has no
collective.

Independent jobs (several cohorts, or one job per GPU in the benchmark) need
no coordination at all beyond the timing barrier.

torch.distributed is the transport (gloo on CPU, nccl between GPUs).
"""
from __future__ import annotations

import numpy as np


def shard_batches(n_batches: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous batch range [b0, b1) of a rank: sizes differ by at most one,
    lower ranks take the extra batches, every batch belongs to exactly one
    rank.  Ranks beyond the batch count get an empty range."""
    if world < 1 or not 0 <= rank < world or n_batches < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_batches, world)
    b0 = rank * base + min(rank, extra)
    b1 = b0 + base + (1 if rank < extra else 0)
    return b0, b1


def snp_range(b0: int, b1: int, tau: int, k: int) -> tuple[int, int]:
    """SNP columns [s0, s1) covered by batches [b0, b1) of tau SNPs each."""
    return min(b0 * tau, k), min(b1 * tau, k)


def merge_shards(shards, k: int):
    """shards: (s0, s1, num, den) per rank, num/den of length k holding that
    rank's SNP range [s0, s1).  Returns (num[k], den[k], complete); raises if
    two ranges overlap."""
    out_num = np.full(k, np.nan)
    out_den = np.full(k, np.nan)
    covered = np.zeros(k, bool)
    for a, b, num, den in shards:
        if a >= b:
            continue
        if covered[a:b].any():
            raise RuntimeError("overlapping shards")
        out_num[a:b] = num[a:b]
        out_den[a:b] = den[a:b]
        covered[a:b] = True
    return out_num, out_den, bool(covered.all())


def gather_results(num: np.ndarray, den: np.ndarray, b0: int, b1: int, tau: int, group=None,
                   device=None):
    """Merge per-rank results into the full num[k], den[k] on every rank.

    Each rank passes arrays of length k holding its own SNP range (other
    entries ignored); one all_gather of the range bounds and one of the
    values rebuild the whole.  Uses the default process group unless one is
    given; device selects where the exchange tensors live (cuda for nccl)."""
    import torch
    import torch.distributed as dist

    k = num.shape[0]
    s0, s1 = snp_range(b0, b1, tau, k)
    world = dist.get_world_size(group)
    dev = device if device is not None else "cpu"
    bounds = torch.tensor([s0, s1], dtype=torch.int64, device=dev)
    all_bounds = [torch.empty_like(bounds) for _ in range(world)]
    dist.all_gather(all_bounds, bounds, group=group)
    vals = torch.from_numpy(np.stack([num, den]).astype(np.float64)).to(dev)
    all_vals = [torch.empty_like(vals) for _ in range(world)]
    dist.all_gather(all_vals, vals, group=group)
    shards = []
    for bnd, v in zip(all_bounds, all_vals):
        a, b = (int(x) for x in bnd.cpu())
        arr = v.cpu().numpy()
        shards.append((a, b, arr[0], arr[1]))
    return merge_shards(shards, k)


def max_over_ranks(value: float, group=None, device=None) -> float:
    """The maximum of a per-rank number (e.g. a step time) over all ranks."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def broadcast_state(job, rank: int, src: int = 0, group=None, device=None):
    """One broadcast of the batch-invariant state: rank src exports its job's
    state (after its fit), every other rank imports it into its own job.
    job needs state_words(), export_state(buf) and import_state(buf); the
    buffer is an int64 tensor on `device` (cpu for gloo, cuda for nccl).
    Returns the number of 8-byte words moved."""
    import torch
    import torch.distributed as dist

    dev = device if device is not None else "cpu"
    n = torch.tensor([job.state_words() if rank == src else 0], dtype=torch.int64, device=dev)
    dist.broadcast(n, src, group=group)
    buf = torch.empty(int(n.item()), dtype=torch.int64, device=dev)
    if rank == src:
        job.export_state(buf)
    dist.broadcast(buf, src, group=group)
    if rank != src:
        job.import_state(buf)
    return int(n.item())


def run_sharded_job(ctx, job, X, A, y, S, kappa: int, rank: int, world: int, group=None,
                    device=None, share_state: bool = True):
    """One encrypted GWAS job over ranks: rank 0 encrypts the inputs and runs
    the covariate phase and its state is broadcast (share_state; otherwise
    every rank repeats the deterministic fit), every rank evaluates its own
    batch range and decrypts it, and the results are gathered on all ranks.
    Returns (num[k], den[k], (b0, b1))."""
    if share_state and world > 1:
        if rank == 0:
            job.encrypt_inputs(X, A, y)
            job.fit(kappa)
        broadcast_state(job, rank, 0, group, device)
    else:
        job.encrypt_inputs(X, A, y)
        job.fit(kappa)
    b0, b1 = shard_batches(job.layout["batches"], world, rank)
    if b1 > b0:
        job.snp_stats(S, b0, b1)
        num, den = job.decrypt_results()
    else:
        num = np.full(job.k, np.nan)
        den = np.full(job.k, np.nan)
    if world == 1:  # one rank: the whole job, nothing to gather
        return num, den, (b0, b1)
    num, den, complete = gather_results(num, den, b0, b1, job.layout["tau"], group, device)
    if not complete:
        raise RuntimeError("some SNP batches were not evaluated")
    return num, den, (b0, b1)
