"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Bars (from the method's statement of the problem):
  * connected lists, canonical ranks, determinants, fermionic signs, H_nm and
    deterministic-set membership: bit-exact;
  * drawn indices of the stochastic part and the total remainder weight W:
    bit-exact;
  * FP64 local energies: |E - E_oracle| <= 1e-12 max(|E|, e_abs) + 2^-52 e_cond.
    e_abs = |H_nn| + sum |H_nm r_m| is the scale rounding errors of the sums
    are bounded by (|E_loc| when nothing cancels). e_cond is the oracle's
    first-order rounding scale of the ratios (the contractions' running-error
    bound P1, weighted like the terms): near a node of psi, psi(n) itself is
    ill-conditioned, and two FP64 evaluations in different orders differ by
    up to ~u e_cond, which no implementation can remove;
  * mixed (FP32 contractions, FP64 psi(n), ratios and sums): within 1e-6 of
    max(|E|, e_abs);
  * log|psi|: within 1e-12 absolute; gradients within 1e-10 relative.
"""
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


def _cases():
    h50 = W.h50_chain()
    fe = W.fe2s2_dense()
    h18 = W.h18_graph()
    return {
        "tiny": W.tiny_system(K=6, na=3, nb=2, D=4, n_hidden=5, seed=3),
        "tiny_graph": W.tiny_system(K=6, na=3, nb=3, D=4, n_hidden=5, seed=4, graph=True),
        # the smallest bond dimension of the graph ansatz's tensor-core tiles
        "graph16": W.tiny_system(K=6, na=3, nb=3, D=16, n_hidden=5, seed=4, graph=True),
        "k8": W.small_chain(),
        # 3532: the batch's smallest |psi(n)| (E_loc ~ 1.9e6 Ha, ratios ~ 1e4):
        # the ratio denominators must not lose accuracy to cancellation
        "h50": h50.subset([0, 1, 2, 3532, 4095]),
        "fe2s2": fe.subset([0, 8191]),
        "h18": h18.subset([0, 1, 2, 3, 16380, 16381, 16382, 16383]),
    }


@pytest.fixture(scope="module")
def cases():
    return _cases()


@pytest.fixture(scope="module")
def problems(cases):
    return {k: O.Problem(v) for k, v in cases.items()}


@pytest.fixture(scope="module")
def ctx():
    c = nqs.Context(0)
    yield c
    c.close()


def _load(ctx, sys_, precision=0):
    ctx.set_system(sys_)
    ctx.set_precision(precision)


# ---------------------------------------------------------------------------
# connectivity
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["tiny", "tiny_graph", "k8", "h50", "fe2s2", "h18"])
def test_connected_lists_bit_exact(ctx, cases, problems, name):
    sys_, P = cases[name], problems[name]
    _load(ctx, sys_)
    for eps in sorted({0.0, 1e-3, 2e-2}):
        off, rank, dets, H, sg = ctx.connected(sys_.samples, eps)
        assert off[0] == 0
        for s, n in enumerate(sys_.samples):
            od, oh, os_ = O.connected(P, n)
            keep = np.nonzero(np.abs(oh) >= eps)[0]
            a, b = off[s], off[s + 1]
            assert b - a == len(keep), (name, eps, s)
            assert np.array_equal(rank[a:b], keep.astype(np.uint32))
            assert np.array_equal(dets[a:b], od[keep])
            assert np.array_equal(H[a:b].view(np.uint64), oh[keep].view(np.uint64))
            assert np.array_equal(sg[a:b], os_[keep])


def test_connected_sizes_query_and_capacity(ctx, cases):
    sys_ = cases["k8"]
    _load(ctx, sys_)
    s = np.ascontiguousarray(sys_.samples[:3])
    off = np.zeros(4, np.int64)
    nqs.nqs_connected(ctx.h, s, 3, 0.0, off, None, None, None, None, 0)
    assert off[-1] == 3 * O.n_conn(8, 4, 4)
    rank = np.empty(10, np.uint32)
    with pytest.raises(nqs.NQSError) as ei:
        nqs.nqs_connected(ctx.h, s, 3, 0.0, off, rank, None, None, None, 10)
    assert ei.value.status == 1 and "capacity" in str(ei.value)


# ---------------------------------------------------------------------------
# stochastic draws
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name,eps,nd", [("h50", 1e-3, 1024), ("tiny", 0.05, 333),
                                         ("h18", 1e-2, 100), ("fe2s2", 1e-2, 257)])
def test_draws_bit_exact(ctx, cases, problems, name, eps, nd):
    sys_, P = cases[name], problems[name]
    _load(ctx, sys_)
    seed = 2507192761
    ranks, wt = ctx.draws(sys_.samples, eps, nd, seed)
    for s, n in enumerate(sys_.samples):
        ref, Wref, _ = O.draws(P, n, s, eps, nd, seed)
        assert int(wt[s]) == Wref
        assert np.array_equal(ranks[s], ref)


def test_sample_index_base_shifts_the_draw_counter(ctx, cases, problems):
    """A shard of a batch, passed with its global position, draws what the
    whole batch draws at those positions (and its E_loc matches the oracle's
    at the same positions)."""
    sys_, P = cases["h50"], problems["h50"]
    _load(ctx, sys_)
    base = 1000
    try:
        ctx.set_precision(nqs.NQS_PREC_FP64, sample_index_base=base)
        ranks, wt = ctx.draws(sys_.samples, sys_.eps, 64, 5)
        for s, n in enumerate(sys_.samples):
            ref, Wref, _ = O.draws(P, n, base + s, sys_.eps, 64, 5)
            assert int(wt[s]) == Wref and np.array_equal(ranks[s], ref)
        sub = sys_.subset([0, 1])
        e, _ = ctx.local_energy(sub.samples, None, sys_.eps, 64, 5)
        ref = O.local_energy(P, samples=sub.samples, eps=sys_.eps, n_draws=64, seed=5,
                             index=[base, base + 1], cond=True)
        assert _rel_sum(e, ref) < RTOL_FP64
        with pytest.raises(nqs.NQSError):
            ctx.set_precision(nqs.NQS_PREC_FP64, sample_index_base=-1)
    finally:
        ctx.set_precision(nqs.NQS_PREC_FP64)


# ---------------------------------------------------------------------------
# local energy, FP64
# ---------------------------------------------------------------------------

def _rel(a, b):
    return np.max(np.abs(a - b) / np.maximum(1e-300, np.abs(b)))


U64 = 2.0 ** -52    # unit roundoff of FP64, both sides


def _rel_sum(e, ref):
    """Error of E_loc over max(|E|, e_abs) + (U64 / RTOL_FP64) e_cond, so that
    `_rel_sum(e, ref) < RTOL_FP64` is the FP64 bar."""
    scale = np.maximum(np.abs(ref["e_loc"]), ref["e_abs"]) + (U64 / RTOL_FP64) * ref["e_cond"]
    return np.max(np.abs(e - ref["e_loc"]) / scale)


def _rel_abs(e, ref):
    """Error relative to the summed-term magnitude only (reported)."""
    return np.max(np.abs(e - ref["e_loc"]) / np.maximum(np.abs(ref["e_loc"]), ref["e_abs"]))


@pytest.mark.parametrize("name", ["tiny", "tiny_graph", "k8", "h50", "fe2s2", "h18"])
def test_local_energy_fp64_matches_oracle(ctx, cases, problems, name):
    sys_, P = cases[name], problems[name]
    _load(ctx, sys_)
    e, summ = ctx.local_energy(sys_.samples, sys_.counts, sys_.eps, sys_.n_draws, sys_.seed)
    ref = O.local_energy(P, cond=True)
    # reported next to the bar: the plain relative error and the bar's scaled one
    print(f"{name}: FP64 max |dE|/|E| = {_rel(e, ref['e_loc']):.3e}, "
          f"scaled (R15) = {_rel_sum(e, ref):.3e}")
    assert _rel_sum(e, ref) < RTOL_FP64
    c = sys_.counts
    # the weighted energy: against the library's own E_loc to summation
    # rounding, and against the oracle within the count-weighted per-sample bar
    bar = RTOL_FP64 * np.maximum(np.abs(ref["e_loc"]), ref["e_abs"]) + U64 * ref["e_cond"]
    assert abs(summ["e_mean"] - np.sum(c * e) / np.sum(c)) <= 1e-13 * np.sum(c * np.abs(e)) / np.sum(c)
    ebar = np.sum(c * ref["e_loc"]) / np.sum(c)
    assert abs(summ["e_mean"] - ebar) <= np.sum(c * bar) / np.sum(c)
    assert summ["n_det"] == int(np.sum(ref["n_det"]))
    assert summ["n_conn"] == O.n_conn(sys_.K, sys_.n_alpha, sys_.n_beta)
    eb, Bs, m, et = O.summary(ref, c)
    assert abs(summ["log_B"] - (m + np.log(Bs))) < 1e-10
    etm = np.sum(c * et) / np.sum(c)
    w = np.exp(2 * ref["log_f"] - m) / Bs          # f^2 / B per sample
    assert abs(summ["e_tilde_mean"] - etm) <= 1e-10 * abs(etm) + np.sum(c * w * bar) / np.sum(c)


@pytest.mark.parametrize("name", ["tiny", "k8", "h50", "fe2s2"])
def test_local_energy_shared_prefix_fp64_matches_oracle(ctx, cases, problems, name):
    """The shared-prefix evaluation re-associates the same products: in FP64 it
    must meet the FP64 bar."""
    sys_, P = cases[name], problems[name]
    _load(ctx, sys_, nqs.NQS_PREC_FP64_SHARED)
    e, summ = ctx.local_energy(sys_.samples, sys_.counts, sys_.eps, sys_.n_draws, sys_.seed)
    ref = O.local_energy(P, cond=True)
    assert _rel_sum(e, ref) < RTOL_FP64
    assert summ["n_det"] == int(np.sum(ref["n_det"]))


# FP32 contractions: tolerance stated against the summed-term magnitude
RTOL_MIXED = 1e-6


@pytest.mark.parametrize("name", ["tiny", "k8", "h50", "fe2s2", "graph16", "h18"])
def test_local_energy_mixed_matches_oracle(ctx, cases, problems, name):
    sys_, P = cases[name], problems[name]
    _load(ctx, sys_, nqs.NQS_PREC_MIXED)
    e, summ = ctx.local_energy(sys_.samples, sys_.counts, sys_.eps, sys_.n_draws, sys_.seed)
    ref = O.local_energy(P)
    err = _rel_abs(e, ref)
    print(f"{name}: mixed max error / max(|E|, e_abs) = {err:.3e}")
    assert err < RTOL_MIXED
    assert summ["n_det"] == int(np.sum(ref["n_det"]))


def test_graph_mixed_cos_correlator(ctx, cases):
    """The graph ansatz's tensor-core form with the cos-RBM correlator (its
    ratio cos(theta + d) / cos(theta) = 1 + (cos d - 1) - tan(theta) sin d)."""
    for name in ("graph16", "h18"):
        sys_ = W.with_correlator(cases[name], 1)
        _load(ctx, sys_, nqs.NQS_PREC_MIXED)
        e, _ = ctx.local_energy(sys_.samples, sys_.counts, sys_.eps, sys_.n_draws, sys_.seed)
        err = _rel_abs(e, O.local_energy(O.Problem(sys_)))
        print(f"{name} cos-RBM: mixed max error / max(|E|, e_abs) = {err:.3e}")
        assert err < RTOL_MIXED


def test_graph_mixed_semistochastic(ctx, cases, problems):
    """Deterministic and drawn rows through the graph tiles (the drawn rows of
    a sample are a second row set with its own tiles)."""
    sys_, P = cases["graph16"], problems["graph16"]
    _load(ctx, sys_, nqs.NQS_PREC_MIXED)
    for eps, nd in [(0.02, 64), (1e3, 200)]:
        e, s = ctx.local_energy(sys_.samples, sys_.counts, eps, nd, 17)
        ref = O.local_energy(P, eps=eps, n_draws=nd, seed=17)
        err = _rel_abs(e, ref)
        print(f"eps={eps}: mixed max error / max(|E|, e_abs) = {err:.3e}")
        assert err < RTOL_MIXED
        assert s["n_det"] == int(np.sum(ref["n_det"]))


def test_graph_mixed_unsupported_cases(ctx, cases):
    """The tensor-core tiles need D in {16, 32, 64}, the linear readout, no
    tensor term and the 2cosh or cos correlator; graphs have no shared-prefix
    form. Each refusal is NQS_ERR_UNSUPPORTED with the reason."""
    def refused(sys_, prec, words):
        _load(ctx, sys_, prec)
        with pytest.raises(nqs.NQSError) as ei:
            ctx.local_energy(sys_.samples, None, 0.0, 0, 0)
        assert ei.value.status == 6 and words in str(ei.value), str(ei.value)
    refused(cases["tiny_graph"], nqs.NQS_PREC_MIXED, "bond dimension")
    refused(cases["graph16"], nqs.NQS_PREC_FP64_SHARED, "shared-prefix")
    refused(W.with_correlator(cases["graph16"], 2), nqs.NQS_PREC_MIXED, "correlator")
    g = cases["graph16"]
    refused(W.with_tensor_term(g), nqs.NQS_PREC_MIXED, "tensor term")
    ctx.set_precision(nqs.NQS_PREC_FP64)


def test_local_energy_stochastic_edge_cases(ctx, cases, problems):
    sys_, P = cases["tiny"], problems["tiny"]
    _load(ctx, sys_)
    exact = O.local_energy(P, eps=0.0, n_draws=0, cond=True)
    # eps = 0 with draws: empty remainder, E^s = 0
    e, s = ctx.local_energy(sys_.samples, None, 0.0, 64, 5)
    assert _rel_sum(e, exact) < RTOL_FP64 and s["n_draw_unique"] == 0
    # eps above every |H|: everything is drawn
    ref = O.local_energy(P, eps=1e3, n_draws=200, seed=9, cond=True)
    e, s = ctx.local_energy(sys_.samples, None, 1e3, 200, 9)
    assert s["n_det"] == 0 and _rel_sum(e, ref) < RTOL_FP64
    # no draws: deterministic part only
    ref = O.local_energy(P, eps=0.05, n_draws=0, cond=True)
    e, _ = ctx.local_energy(sys_.samples, None, 0.05, 0, 9)
    assert _rel_sum(e, ref) < RTOL_FP64
    # empty batch
    e, s = ctx.local_energy(np.zeros((0, 2), np.uint64), None, 0.0, 0, 0)
    assert len(e) == 0


def test_invalid_samples_are_rejected(ctx, cases):
    sys_ = cases["k8"]
    _load(ctx, sys_)
    bad = np.array(sys_.samples[:5], copy=True)
    bad[3, 0] = np.uint64(0b111)                     # 3 alpha electrons, 4 expected
    with pytest.raises(nqs.NQSError) as ei:
        ctx.local_energy(bad, None, 0.0, 0, 0)
    assert ei.value.status == 1 and "samples[3]" in str(ei.value)
    bad[3, 0] = np.uint64(0b1111) | np.uint64(1 << 9)
    with pytest.raises(nqs.NQSError):
        ctx.connected(bad, 0.0)
    with pytest.raises(nqs.NQSError):
        ctx.local_energy(sys_.samples, None, -1.0, 0, 0)
    with pytest.raises(nqs.NQSError):
        ctx.local_energy(sys_.samples, None, 0.0, 5000, 0)


def test_degenerate_systems(ctx):
    # one orbital pair: no excitations at all, E_loc = H_nn
    for K, na, nb in [(1, 1, 1), (2, 1, 0), (2, 2, 1), (3, 0, 3)]:
        sys_ = W.tiny_system(K=K, na=na, nb=nb, D=2, seed=K + na)
        P = O.Problem(sys_)
        _load(ctx, sys_)
        e, s = ctx.local_energy(sys_.samples, None, 0.0, 8, 1)
        ref = O.local_energy(P, eps=0.0, n_draws=8, seed=1, cond=True)
        assert _rel_sum(e, ref) < RTOL_FP64
        assert s["n_conn"] == O.n_conn(K, na, nb)


def test_device_and_host_buffers_agree(ctx, cases):
    sys_ = cases["h18"]
    _load(ctx, sys_)
    e_host, _ = ctx.local_energy(sys_.samples, sys_.counts, 0.0, 0, 0)
    s_dev = torch.from_numpy(sys_.samples.view(np.int64)).cuda()
    c_dev = torch.from_numpy(sys_.counts).cuda()
    out = torch.empty(len(sys_.samples), dtype=torch.float64, device="cuda")
    ctx.local_energy(s_dev, c_dev, 0.0, 0, 0, out=out)
    assert np.array_equal(out.cpu().numpy(), e_host)


# ---------------------------------------------------------------------------
# amplitudes and gradients
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", ["tiny", "tiny_graph", "k8", "h50", "fe2s2", "h18"])
def test_amplitude_matches_oracle(ctx, cases, problems, name):
    sys_, P = cases[name], problems[name]
    _load(ctx, sys_)
    od, _, _ = O.connected(P, sys_.samples[0])
    dets = np.concatenate([sys_.samples, od[:: max(1, len(od) // 200)]])
    la, sg = ctx.amplitude(dets)
    for d, l, s in zip(dets, la, sg):
        rl, rs, _ = O.log_psi(P, d)
        assert s == rs and abs(l - rl) < 1e-12 * max(1.0, abs(rl))


@pytest.mark.parametrize("name", ["tiny", "tiny_graph", "k8", "h18"])
def test_grad_vjp_matches_oracle(ctx, cases, problems, name):
    sys_, P = cases[name], problems[name]
    _load(ctx, sys_)
    rng = np.random.default_rng(1)
    u = rng.normal(size=len(sys_.samples))
    gT, gW, gb = ctx.grad_log_psi_vjp(sys_.samples, u)
    rT = np.zeros_like(gT)
    rW = np.zeros_like(gW) if gW is not None else None
    rb = np.zeros_like(gb) if gb is not None else None
    for ui, d in zip(u, sys_.samples):
        t, w, b = O.grad_log_psi(P, d)
        rT += ui * t
        if rW is not None:
            rW += ui * w
            rb += ui * b
    scale = np.max(np.abs(rT))
    assert np.max(np.abs(gT - rT)) < 1e-10 * scale
    if rW is not None:
        assert np.max(np.abs(gW - rW)) < 1e-10 * max(1.0, np.max(np.abs(rW)))
        assert np.max(np.abs(gb - rb)) < 1e-10 * max(1.0, np.max(np.abs(rb)))


@pytest.mark.parametrize("D", [16, 32, 48, 128, 192, 256])
def test_bond_dimensions_of_the_tensor_core_path(ctx, D):
    """Every tile shape of the shared-prefix path: D = 16..128 in one
    reduction chunk (48 through the run-time-D epilogue), 192 and 256 in
    chunks of 64; mixed against the mixed bar, FP64 shared against the FP64
    bar, with draws."""
    sys_ = W.tiny_system(K=7, na=3, nb=3, D=D, n_hidden=6, seed=60 + D, eps=0.02, n_draws=48,
                         n_samples=10)
    P = O.Problem(sys_)
    ref = O.local_energy(P, cond=True)
    try:
        for prec in (nqs.NQS_PREC_MIXED, nqs.NQS_PREC_FP64_SHARED):
            _load(ctx, sys_, prec)
            e, summ = ctx.local_energy(sys_.samples, sys_.counts, sys_.eps, sys_.n_draws, sys_.seed)
            assert summ["n_det"] == int(np.sum(ref["n_det"]))
            if prec == nqs.NQS_PREC_MIXED:
                err = _rel_abs(e, ref)
                print(f"D={D}: mixed max error / max(|E|, e_abs) = {err:.3e}")
                assert err < RTOL_MIXED
            else:
                assert _rel_sum(e, ref) < RTOL_FP64
    finally:
        ctx.set_precision(nqs.NQS_PREC_FP64)


# ---------------------------------------------------------------------------
# 64 orbitals: both occupation words full width, orbital 63 occupied
# ---------------------------------------------------------------------------

def _k64_system(D):
    """K = 64 (Sec. 3: interleaved order on two 64-bit words), 2 alpha + 1 beta
    electrons; the first samples occupy orbital 63 in one or both spins."""
    sys_ = W.tiny_system(K=64, na=2, nb=1, D=D, n_hidden=5, seed=13, chol_rank=6, n_samples=5,
                         eps=2e-3, n_draws=96)
    top = np.array([[(1 << 63) | (1 << 20), 1 << 63],
                    [(1 << 63) | (1 << 62), 1],
                    [3, 1 << 63]], np.uint64)
    keep = [i for i, d in enumerate(sys_.samples) if not any((d == t).all() for t in top)]
    samples = np.ascontiguousarray(np.concatenate([top, sys_.samples[keep]]))
    counts = np.concatenate([np.array([1.0, 2.0, 0.5]), sys_.counts[keep]])
    import dataclasses
    return dataclasses.replace(sys_, samples=samples, counts=counts)


def test_sixty_four_orbitals_lists_draws_and_energies(ctx):
    sys_ = _k64_system(D=16)
    P = O.Problem(sys_)
    try:
        _load(ctx, sys_)
        for eps in (0.0, 2e-3):
            off, rank, dets, H, sg = ctx.connected(sys_.samples, eps)
            for s, n in enumerate(sys_.samples):
                od, oh, os_ = O.connected(P, n)
                keep = np.nonzero(np.abs(oh) >= eps)[0]
                a, b = off[s], off[s + 1]
                assert b - a == len(keep)
                assert np.array_equal(rank[a:b], keep.astype(np.uint32))
                assert np.array_equal(dets[a:b], od[keep])
                assert np.array_equal(H[a:b].view(np.uint64), oh[keep].view(np.uint64))
                assert np.array_equal(sg[a:b], os_[keep])
        ranks, wt = ctx.draws(sys_.samples, sys_.eps, sys_.n_draws, sys_.seed)
        for s, n in enumerate(sys_.samples):
            ref, Wref, _ = O.draws(P, n, s, sys_.eps, sys_.n_draws, sys_.seed)
            assert int(wt[s]) == Wref and np.array_equal(ranks[s], ref)
        ref = O.local_energy(P, cond=True)
        for prec in (nqs.NQS_PREC_FP64, nqs.NQS_PREC_FP64_SHARED, nqs.NQS_PREC_MIXED):
            _load(ctx, sys_, prec)
            e, summ = ctx.local_energy(sys_.samples, sys_.counts, sys_.eps, sys_.n_draws, sys_.seed)
            assert summ["n_det"] == int(np.sum(ref["n_det"]))
            if prec == nqs.NQS_PREC_MIXED:
                assert _rel_abs(e, ref) < RTOL_MIXED
            else:
                print(f"K=64 precision {prec}: FP64 max |dE|/|E| = {_rel(e, ref['e_loc']):.3e}")
                assert _rel_sum(e, ref) < RTOL_FP64
    finally:
        ctx.set_precision(nqs.NQS_PREC_FP64)


def test_schedule_options_do_not_change_results(ctx):
    """tile_blocks_per_sm and table_mb (the autotuner's knobs) change only the
    launch shapes and the sample-batch split of the shared-prefix tables: the
    mixed and FP64-shared E_loc stay bit-identical."""
    sys_ = W.h50_chain(n_samples=48)
    try:
        for prec in (nqs.NQS_PREC_MIXED, nqs.NQS_PREC_FP64_SHARED):
            _load(ctx, sys_, prec)
            ref, _ = ctx.local_energy(sys_.samples, sys_.counts, sys_.eps, sys_.n_draws, sys_.seed)
            for bps, mb in [(2, 0), (8, 0), (4, 40)]:
                ctx.set_precision(prec, tile_blocks_per_sm=bps, table_mb=mb)
                e, _ = ctx.local_energy(sys_.samples, sys_.counts, sys_.eps, sys_.n_draws, sys_.seed)
                assert np.array_equal(e.view(np.uint64), ref.view(np.uint64)), (prec, bps, mb)
    finally:
        ctx.set_precision(nqs.NQS_PREC_FP64)
