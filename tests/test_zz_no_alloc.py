"""The allocation-free draws entry point (nqs_draws_noalloc) against nqs_draws.

nqs_draws_noalloc exists for callers that may not allocate device memory
while they run (latency-critical loops that must not wait on an allocator,
applications that give all GPU memory to their own pool). It works in a fixed
scratch array inside the library instead of allocating. Its draws must be the
same as those of nqs_draws: the drawn indices and W are integers, so the
comparison is exact, and it is repeated on two calls in a row so that a call
cannot lean on what the previous one left in the shared scratch.
"""
import numpy as np
import pytest

from paper_2507_19276_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_19276_gb300 import nqs  # noqa: E402


def _noalloc(ctx, samples, eps, n_draws, seed):
    s_dev = torch.from_numpy(np.ascontiguousarray(samples).view(np.int64)).cuda()
    Ns = len(samples)
    r_dev = torch.full((Ns, n_draws), -7, dtype=torch.int64, device="cuda")
    w_dev = torch.full((Ns,), -7, dtype=torch.int64, device="cuda")
    nqs.nqs_draws_noalloc(ctx.h, s_dev, Ns, eps, n_draws, seed, r_dev, w_dev)
    torch.cuda.synchronize()
    return r_dev.cpu().numpy(), w_dev.cpu().numpy().view(np.uint64)


def test_noalloc_draws_equal_nqs_draws_on_two_calls_in_a_row():
    ctx = nqs.Context(0)
    try:
        calls = [
            (W.h50_chain().subset(range(8)), 1e-3, 1024, 2507192761),
            (W.small_chain(), 0.02, 257, 99),
        ]
        for sys_, eps, nd, seed in calls:
            ctx.set_system(sys_)
            ref_r, ref_w = ctx.draws(sys_.samples, eps, nd, seed)
            got_r, got_w = _noalloc(ctx, sys_.samples, eps, nd, seed)
            assert np.array_equal(got_r, ref_r)
            assert np.array_equal(got_w, ref_w)
    finally:
        ctx.close()


def test_noalloc_larger_then_smaller_batch_and_optional_outputs():
    """A batch of 30 H50 samples (most of the scratch), then a K = 64 batch
    with fewer samples but more rank chunks per sample, so the second call's
    regions overlap what the first left behind; then W alone (n_draws = 0) and
    ranks alone (w_total = None)."""
    ctx = nqs.Context(0)
    try:
        big = W.h50_chain().subset(range(30))
        ctx.set_system(big)
        ref_r, ref_w = ctx.draws(big.samples, 1e-3, 64, 11)
        got_r, got_w = _noalloc(ctx, big.samples, 1e-3, 64, 11)
        assert np.array_equal(got_r, ref_r) and np.array_equal(got_w, ref_w)

        wide = W.h50_chain(n_samples=3, K=64, D=16, n_hidden=0)
        ctx.set_system(wide)
        ref_r, ref_w = ctx.draws(wide.samples, 2e-3, 200, 5)
        got_r, got_w = _noalloc(ctx, wide.samples, 2e-3, 200, 5)
        assert np.array_equal(got_r, ref_r) and np.array_equal(got_w, ref_w)

        # W only
        s_dev = torch.from_numpy(wide.samples.view(np.int64)).cuda()
        w_dev = torch.full((3,), -7, dtype=torch.int64, device="cuda")
        nqs.nqs_draws_noalloc(ctx.h, s_dev, 3, 2e-3, 0, 5, None, w_dev)
        torch.cuda.synchronize()
        assert np.array_equal(w_dev.cpu().numpy().view(np.uint64), ref_w)
        # ranks only
        r_dev = torch.full((3, 200), -7, dtype=torch.int64, device="cuda")
        nqs.nqs_draws_noalloc(ctx.h, s_dev, 3, 2e-3, 200, 5, r_dev, None)
        torch.cuda.synchronize()
        assert np.array_equal(r_dev.cpu().numpy(), ref_r)
    finally:
        ctx.close()


def test_noalloc_rejects_batches_beyond_the_scratch_and_host_pointers():
    ctx = nqs.Context(0)
    try:
        sys_ = W.h50_chain().subset(range(64))      # needs ~1.7M scratch words
        ctx.set_system(sys_)
        s_dev = torch.from_numpy(sys_.samples.view(np.int64)).cuda()
        r_dev = torch.empty((64, 16), dtype=torch.int64, device="cuda")
        with pytest.raises(nqs.NQSError) as ei:
            nqs.nqs_draws_noalloc(ctx.h, s_dev, 64, 1e-3, 16, 1, r_dev, None)
        assert ei.value.status == 1 and "scratch" in str(ei.value)
        host = np.empty((64, 16), np.int64)
        with pytest.raises(nqs.NQSError) as ei:
            nqs.nqs_draws_noalloc(ctx.h, s_dev, 64, 1e-3, 16, 1, host, None)
        assert "device pointers" in str(ei.value)
    finally:
        ctx.close()
