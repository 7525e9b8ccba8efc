"""Splitting one batch of unique samples across processes (one per GPU).

E_loc(n) of each unique sample is independent of the others (Sec. 2.4), so a
batch splits into contiguous shards with no exchange while the local energies
are computed. Each shard passes its global position as the Philox sample index
base, so the draws, and hence every E_loc, do not depend on how the batch was
split. The one exchange is the reduction of the sums that the weighted energy
and the reweighting factor B of Sec. 2.3 are made of:

    E_bar = sum_n c_n E_loc(n) / sum_n c_n
    B     = sum_n c_n f(n)^2 / sum_n c_n          (kept as log B)
    E~    = sum_n c_n f(n)^2 / B E_loc(n) / sum_n c_n

A shard's summary holds these as means over its own samples; the global values
are rebuilt from the sums, with B combined in the log domain (max-shifted) so
that large f never overflows.
"""
from __future__ import annotations

import math

import numpy as np


def shard_range(n_total: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous [lo, hi) of rank's samples; sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard request")
    q, r = divmod(n_total, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


# fields summed over shards as they are (counts of work)
_SUMMED = ("n_det", "n_draw_unique", "n_amplitudes", "span_sites", "matvecs")


def _local_terms(s: dict) -> tuple[np.ndarray, float]:
    """(sums that add across shards, log of the shard's sum c f^2)."""
    c = s["sum_counts"]
    if c > 0:
        log_cf2 = s["log_B"] + math.log(c)
    else:
        log_cf2 = -math.inf
    sums = [c * s["e_mean"], c] + [float(s[k]) for k in _SUMMED]
    return np.array(sums, np.float64), log_cf2


def combine(summaries: list[dict]) -> dict:
    """Global summary from per-shard summaries (serial form of `allreduce`)."""
    terms = [_local_terms(s) for s in summaries]
    sums = np.sum([t[0] for t in terms], axis=0)
    logs = np.array([t[1] for t in terms])
    m = np.max(logs)
    # a shard's e_tilde_mean is sum c f^2 E / (sum c f^2) over the shard, so the
    # global value is its mean weighted by each shard's sum c f^2
    et = [(s["e_tilde_mean"], lg) for s, lg in zip(summaries, logs)]
    return _finish(sums, m, np.sum(np.exp(logs - m)) if np.isfinite(m) else 0.0,
                   np.sum([a * math.exp(lg - m) for a, lg in et if np.isfinite(lg)]),
                   summaries[0])


def _finish(sums, m, scaled_cf2, scaled_et, like):
    c = sums[1]
    out = dict(like)
    out["sum_counts"] = float(c)
    out["e_mean"] = float(sums[0] / c) if c > 0 else 0.0
    for i, k in enumerate(_SUMMED):
        out[k] = int(round(sums[2 + i]))
    if c > 0 and scaled_cf2 > 0:
        # log B = log(sum c f^2) - log(sum c); E~ mean = sum c f^2 E / sum c f^2
        out["log_B"] = float(m + math.log(scaled_cf2) - math.log(c))
        out["e_tilde_mean"] = float(scaled_et / scaled_cf2)
    return out


def allreduce(summary: dict, device=None) -> dict:
    """Global summary over the default torch.distributed process group.

    Two collectives: a MAX of log(sum c f^2), then one SUM of the shard sums
    and of the max-shifted B terms.
    """
    import torch
    import torch.distributed as dist

    sums, lg = _local_terms(summary)
    t = torch.tensor([lg], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    m = float(t.item())
    w = math.exp(lg - m) if math.isfinite(lg) else 0.0
    payload = np.concatenate([sums, [w, summary["e_tilde_mean"] * w]])
    t = torch.tensor(payload, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    v = t.cpu().numpy()
    return _finish(v[:-2], m, v[-2], v[-1], summary)
