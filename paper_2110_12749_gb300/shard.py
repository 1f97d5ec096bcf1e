"""Host-side sharding of independent beams across ranks (one GPU per rank).

The hot path has no exchange step: beams (and DM ranges) are independent
units, so ranks split them with no data-path collective.  The only
cross-rank operations are the timing reduction and the final concatenation
of the (small) candidate lists, both on the host side of the job.
"""
import numpy as np


def beams_for_rank(nbeams, rank, world):
    """Round-robin assignment of beam indices to a rank."""
    if not (0 <= rank < world):
        raise ValueError("rank out of range")
    return list(range(rank, nbeams, world))


def label_beam(cands, beam):
    """Copy of a candidate array with its beam field set."""
    out = np.array(cands, copy=True)
    out["beam"] = beam
    return out


def merge_candidates(parts, dtype):
    """Concatenate per-beam candidate arrays, sorted by (beam, dm_idx, t, width)."""
    parts = [p for p in parts if len(p)]
    if not parts:
        return np.zeros(0, dtype=dtype)
    allc = np.concatenate(parts).astype(dtype)
    order = np.lexsort((allc["width"], allc["t"], allc["dm_idx"], allc["beam"]))
    return allc[order]


def max_over_ranks(value, dist=None, device=None):
    """Max of a float over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_candidates(cands, dist, dtype):
    """All candidate arrays of all ranks, merged (rank 0 gets the full list)."""
    if dist is None or not dist.is_initialized():
        return merge_candidates([cands], dtype)
    parts = [None] * dist.get_world_size()
    dist.all_gather_object(parts, np.asarray(cands))
    return merge_candidates(parts, dtype)
