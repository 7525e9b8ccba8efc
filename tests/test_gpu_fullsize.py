"""Parity at the full workload sizes, in the launch configuration the benchmark
times (whole batch in one nqs_local_energy call, device-resident buffers).

The oracle cannot recompute thousands of samples in seconds, so it recomputes
a spread of sampled ones, each with its batch position (the Philox counter of
its draws), and the whole batch is checked through properties that hold at any
size: the deterministic-set size in the summary equals the sum of the sizes
nqs_connected reports, and the summary's weighted energy is the weighted mean of
the returned local energies.
"""
import os
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_19276_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_19276_gb300 import nqs  # noqa: E402

RTOL_FP64 = 1e-12
RTOL_MIXED = 1e-6
U64 = 2.0 ** -52    # unit roundoff of FP64, both sides


@pytest.fixture(scope="module")
def ctx():
    c = nqs.Context(0)
    yield c
    c.close()


def _run_full(ctx, sys_, precision):
    ctx.set_system(sys_)
    ctx.set_precision(precision)
    s = torch.from_numpy(sys_.samples.view(np.int64)).cuda()
    c = torch.from_numpy(sys_.counts).cuda()
    e = torch.empty(len(sys_.samples), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, summ = ctx.local_energy(s, c, sys_.eps, sys_.n_draws, sys_.seed, out=e)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return e.cpu().numpy(), summ, dt


def _picked(ctx, sys_, extra, seed):
    """Spread positions, random ones, and the sample nearest a node of psi
    (smallest |psi(n)|, where every ratio is large and cancellation in psi(n)
    would show most)."""
    Ns = len(sys_.samples)
    rng = np.random.default_rng(seed)
    la, _ = ctx.amplitude(sys_.samples)
    base = [0, Ns // 3, (2 * Ns) // 3, Ns - 1, int(np.argmin(la))]
    more = rng.choice(Ns, size=extra, replace=False).tolist()
    return sorted(set(base + more))


def _check_sampled(sys_, e, idx, rtol):
    """Largest error over the bar's scale: for FP64, max(|E|, e_abs) plus the
    first-order rounding scale (U64 / rtol) e_cond; for mixed, max(|E|, e_abs)."""
    P = O.Problem(sys_)
    fp64 = rtol == RTOL_FP64
    ref = O.local_energy(P, samples=sys_.samples[idx], index=idx, threads=os.cpu_count() or 1,
                         cond=fp64)
    scale = np.maximum(np.abs(ref["e_loc"]), ref["e_abs"])
    if fp64:
        scale = scale + (U64 / rtol) * ref["e_cond"]
    err = np.abs(e[idx] - ref["e_loc"]) / scale
    print(f"  errors over scale {np.array2string(err, precision=2)}")
    return float(np.max(err)), ref


def _check_properties(ctx, sys_, e, summ):
    assert np.all(np.isfinite(e))
    c = sys_.counts
    ebar = float(np.sum(c * e) / np.sum(c))
    assert abs(summ["e_mean"] - ebar) <= 1e-12 * abs(ebar)
    off = np.zeros(len(sys_.samples) + 1, np.int64)
    nqs.nqs_connected(ctx.h, np.ascontiguousarray(sys_.samples), len(sys_.samples), sys_.eps,
                      off, None, None, None, None, 0)
    assert summ["n_det"] == int(off[-1])
    assert summ["n_conn"] == O.n_conn(sys_.K, sys_.n_alpha, sys_.n_beta)


def test_h50_full_batch_mixed_sampled_against_oracle(ctx):
    """4096 samples, D=64, N_h=100, eps=1e-3, 1024 draws: the benchmark's step."""
    sys_ = W.h50_chain()
    e, summ, dt = _run_full(ctx, sys_, nqs.NQS_PREC_MIXED)
    _check_properties(ctx, sys_, e, summ)
    idx = _picked(ctx, sys_, 2, 11)
    err, _ = _check_sampled(sys_, e, idx, RTOL_MIXED)
    print(f"h50 full mixed: {dt:.2f} s, sampled max error / max(|E|, e_abs) {err:.3e}")
    assert err < RTOL_MIXED


def test_h50_full_batch_fp64_shared_sampled_against_oracle(ctx):
    sys_ = W.h50_chain()
    e, summ, dt = _run_full(ctx, sys_, nqs.NQS_PREC_FP64_SHARED)
    _check_properties(ctx, sys_, e, summ)
    idx = _picked(ctx, sys_, 2, 12)
    err, _ = _check_sampled(sys_, e, idx, RTOL_FP64)
    print(f"h50 full fp64 shared: {dt:.2f} s, sampled max error {err:.3e}")
    assert err < RTOL_FP64


def test_fe2s2_full_batch_mixed_sampled_against_oracle(ctx):
    """8192 samples, D=256 (beyond the tensor-core tile: FP32 CUDA-core batches)."""
    sys_ = W.fe2s2_dense()
    e, summ, dt = _run_full(ctx, sys_, nqs.NQS_PREC_MIXED)
    _check_properties(ctx, sys_, e, summ)
    idx = _picked(ctx, sys_, 0, 13)
    err, _ = _check_sampled(sys_, e, idx, RTOL_MIXED)
    print(f"fe2s2 full mixed: {dt:.2f} s, sampled max error / max(|E|, e_abs) {err:.3e}")
    assert err < RTOL_MIXED


def test_h18_graph_full_batch_fp64_sampled_against_oracle(ctx):
    """16384 samples of the graph-ordered ansatz (FP64, fully deterministic)."""
    sys_ = W.h18_graph()
    e, summ, dt = _run_full(ctx, sys_, nqs.NQS_PREC_FP64)
    _check_properties(ctx, sys_, e, summ)
    idx = _picked(ctx, sys_, 4, 14)
    err, _ = _check_sampled(sys_, e, idx, RTOL_FP64)
    print(f"h18 full fp64: {dt:.2f} s, sampled max error {err:.3e}")
    assert err < RTOL_FP64


def test_h50_energy_tolerance_refinement_meets_the_bound(ctx):
    """Mixed form with energy_tolerance = 1e-6 Ha: the heaviest samples are
    re-evaluated in FP64, the weighted energy lands within the tolerance of
    the FP64 form's, the re-evaluated E_loc are the FP64 ones, and every other
    sample keeps its mixed value bit for bit."""
    sys_ = W.h50_chain()
    e64, s64, _ = _run_full(ctx, sys_, nqs.NQS_PREC_FP64_SHARED)
    emx, smx, _ = _run_full(ctx, sys_, nqs.NQS_PREC_MIXED)
    assert smx["n_refined"] == 0 and smx["e_error_bound"] == 0.0
    ctx.set_precision(nqs.NQS_PREC_MIXED, energy_tolerance=1e-6)
    try:
        s = torch.from_numpy(sys_.samples.view(np.int64)).cuda()
        c = torch.from_numpy(sys_.counts).cuda()
        out = torch.empty(len(sys_.samples), dtype=torch.float64, device="cuda")
        _, summ = ctx.local_energy(s, c, sys_.eps, sys_.n_draws, sys_.seed, out=out)
        e = out.cpu().numpy()
    finally:
        ctx.set_precision(nqs.NQS_PREC_FP64)
    k = summ["n_refined"]
    print(f"refined {k} of {len(e)}; bound {summ['e_error_bound']:.3e}; "
          f"|E_bar - E_bar_fp64| mixed {abs(smx['e_mean'] - s64['e_mean']):.3e} "
          f"refined {abs(summ['e_mean'] - s64['e_mean']):.3e}")
    assert 0 < k < len(e) and summ["e_error_bound"] <= 1e-6
    changed = e != emx
    assert changed.sum() <= k
    np.testing.assert_allclose(e[changed], e64[changed], rtol=1e-13, atol=0)
    assert np.array_equal(e[~changed], emx[~changed])
    # within the tolerance, plus the FP64 form's own rounding of the mean
    assert abs(summ["e_mean"] - s64["e_mean"]) <= 1e-6 + 1e-12 * abs(s64["e_mean"])
    assert summ["n_det"] == smx["n_det"] and summ["log_B"] == smx["log_B"]


def test_h18_graph_full_batch_mixed_sampled_against_oracle(ctx):
    """16384 samples of the graph-ordered ansatz on the tensor-core tiles
    (D = 32, up to three in-edges per vertex)."""
    sys_ = W.h18_graph()
    e, summ, dt = _run_full(ctx, sys_, nqs.NQS_PREC_MIXED)
    _check_properties(ctx, sys_, e, summ)
    idx = _picked(ctx, sys_, 4, 15)
    err, _ = _check_sampled(sys_, e, idx, RTOL_MIXED)
    print(f"h18 full mixed: {dt:.2f} s, sampled max error / max(|E|, e_abs) {err:.3e}")
    assert err < RTOL_MIXED


def test_h18_energy_tolerance_refinement_meets_the_bound(ctx):
    """The graph ansatz's mixed form with energy_tolerance = 1e-6 Ha: the
    heaviest samples are re-evaluated in the plain FP64 form, the weighted
    energy lands within the tolerance of the FP64 form's, and every other
    sample keeps its mixed value."""
    sys_ = W.h18_graph()
    e64, s64, t64 = _run_full(ctx, sys_, nqs.NQS_PREC_FP64)
    emx, smx, tmx = _run_full(ctx, sys_, nqs.NQS_PREC_MIXED)
    ctx.set_precision(nqs.NQS_PREC_MIXED, energy_tolerance=1e-6)
    try:
        s = torch.from_numpy(sys_.samples.view(np.int64)).cuda()
        c = torch.from_numpy(sys_.counts).cuda()
        out = torch.empty(len(sys_.samples), dtype=torch.float64, device="cuda")
        _, summ = ctx.local_energy(s, c, sys_.eps, sys_.n_draws, sys_.seed, out=out)
        e = out.cpu().numpy()
    finally:
        ctx.set_precision(nqs.NQS_PREC_FP64)
    k = summ["n_refined"]
    print(f"fp64 {t64:.2f} s, mixed {tmx:.2f} s; refined {k} of {len(e)}; bound "
          f"{summ['e_error_bound']:.3e}; |E_bar - E_bar_fp64| mixed "
          f"{abs(smx['e_mean'] - s64['e_mean']):.3e} refined {abs(summ['e_mean'] - s64['e_mean']):.3e}; "
          f"audit {summ['audit_rel_error']:.3e}")
    assert 0 < k < len(e) and summ["e_error_bound"] <= 1e-6
    changed = e != emx
    assert changed.sum() <= k
    np.testing.assert_allclose(e[changed], e64[changed], rtol=1e-13, atol=0)
    assert np.array_equal(e[~changed], emx[~changed])
    assert abs(summ["e_mean"] - s64["e_mean"]) <= 1e-6 + 1e-12 * abs(s64["e_mean"])
