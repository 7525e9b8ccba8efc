"""The multi-process path on CPU: two gloo ranks each take a contiguous shard
of one batch (with its global Philox index base), compute their local
energies with the oracle, and reduce the summary; the result must equal the
single-process summary of the whole batch, and the concatenated per-sample
energies must equal the whole batch's bit for bit."""
import math
import os
import socket

import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_19276_gb300 import shard
from paper_2507_19276_gb300 import workloads as W


def _system():
    s = W.tiny_system(K=7, na=3, nb=3, D=4, n_hidden=5, seed=31)
    rng = np.random.default_rng(5)
    s.counts = rng.integers(1, 50, size=len(s.samples)).astype(np.float64)
    s.eps, s.n_draws, s.seed = 0.05, 40, 77
    return s


def _summary(out, counts):
    """The library's summary fields, from oracle outputs (Sec. 2.3)."""
    c = np.asarray(counts, np.float64)
    e, lf = out["e_loc"], out["log_f"]
    lw = np.log(c) + 2 * lf
    m = np.max(lw)
    cf2 = np.exp(lw - m)
    return {"e_mean": float(np.sum(c * e) / np.sum(c)), "sum_counts": float(np.sum(c)),
            "log_B": float(m + math.log(np.sum(cf2)) - math.log(np.sum(c))),
            "e_tilde_mean": float(np.sum(cf2 * e) / np.sum(cf2)),
            "n_conn": 0, "n_det": int(np.sum(out["n_det"])), "n_draw_unique": 0,
            "n_amplitudes": 0, "span_sites": 0, "matvecs": 0}


def test_shard_range_covers_the_batch_once():
    for n in [0, 1, 5, 64, 4097]:
        for w in [1, 2, 3, 8]:
            parts = [shard.shard_range(n, w, r) for r in range(w)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.shard_range(10, 2, 2)


def test_serial_combine_equals_whole_batch():
    s = _system()
    P = O.Problem(s)
    full = O.local_energy(P)
    ref = _summary(full, s.counts)
    parts = []
    for r in range(3):
        lo, hi = shard.shard_range(len(s.samples), 3, r)
        parts.append(_summary(full[lo:hi], s.counts[lo:hi]))
    got = shard.combine(parts)
    for k in ("e_mean", "log_B", "e_tilde_mean", "sum_counts"):
        assert abs(got[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), k
    assert got["n_det"] == ref["n_det"]


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = _system()
        lo, hi = shard.shard_range(len(s.samples), world, rank)
        P = O.Problem(s)
        out = O.local_energy(P, samples=s.samples[lo:hi], index=np.arange(lo, hi))
        g = shard.allreduce(_summary(out, s.counts[lo:hi]))
        np.save(os.path.join(outdir, f"e{rank}.npy"), out["e_loc"])
        np.save(os.path.join(outdir, f"g{rank}.npy"),
                np.array([g["e_mean"], g["log_B"], g["e_tilde_mean"], g["sum_counts"], g["n_det"]]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def test_two_gloo_ranks_reduce_to_the_whole_batch(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    s = _system()
    full = O.local_energy(O.Problem(s))
    ref = _summary(full, s.counts)
    e = np.concatenate([np.load(tmp_path / f"e{r}.npy") for r in range(world)])
    assert np.array_equal(e.view(np.uint64), full["e_loc"].view(np.uint64))
    for r in range(world):
        g = np.load(tmp_path / f"g{r}.npy")
        assert abs(g[0] - ref["e_mean"]) <= 1e-12 * abs(ref["e_mean"])
        assert abs(g[1] - ref["log_B"]) <= 1e-12 * max(1.0, abs(ref["log_B"]))
        assert abs(g[2] - ref["e_tilde_mean"]) <= 1e-12 * abs(ref["e_tilde_mean"])
        assert g[3] == ref["sum_counts"] and int(g[4]) == ref["n_det"]
