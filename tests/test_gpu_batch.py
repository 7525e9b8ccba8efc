"""Multi-system batch (nqs_local_energy_batch): independent chains of
different K, D and batch sizes in one call, each on its own context and
stream. Every system's result must equal its own nqs_local_energy call bit
for bit, sampled positions must match the oracle, and a failing system must
not disturb the others."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_19276_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_19276_gb300 import nqs  # noqa: E402

RTOL_MIXED = 1e-6


def _systems(n=6):
    """A spread of the 64-system batch: distinct (K, D) pairs, batches cut to
    at most 1024 samples so the oracle checks stay short."""
    seen, out = set(), []
    for s in W.uneven_batch():
        if (s.K, s.D) in seen:
            continue
        seen.add((s.K, s.D))
        out.append(s.subset(range(min(len(s.samples), 1024))))
        if len(out) == n:
            break
    return out


@pytest.fixture(scope="module")
def setup():
    systems = _systems()
    streams = [torch.cuda.Stream() for _ in systems]
    ctxs = []
    for s, st in zip(systems, streams):
        c = nqs.Context(0, stream=st.cuda_stream)
        c.set_system(s)
        c.set_precision(nqs.NQS_PREC_MIXED)
        ctxs.append(c)
    yield systems, ctxs, streams
    for c in ctxs:
        c.close()


def _args(s):
    return {"samples": s.samples, "counts": s.counts, "eps": s.eps, "n_draws": s.n_draws,
            "seed": s.seed}


def test_batch_equals_per_system_calls_and_the_oracle(setup):
    systems, ctxs, _ = setup
    print("systems:", [(s.K, s.D, len(s.samples)) for s in systems])
    got = nqs.local_energy_batch(ctxs, [_args(s) for s in systems], n_workers=4)
    for s, c, (e, summ) in zip(systems, ctxs, got):
        ref, rs = c.local_energy(s.samples, s.counts, s.eps, s.n_draws, s.seed)
        assert np.array_equal(e.view(np.uint64), ref.view(np.uint64)), s.name
        assert summ["e_mean"] == rs["e_mean"] and summ["n_det"] == rs["n_det"]
        idx = [0, len(s.samples) // 2, len(s.samples) - 1]
        o = O.local_energy(O.Problem(s), samples=s.samples[idx], index=idx,
                           threads=os.cpu_count() or 1)
        err = np.max(np.abs(e[idx] - o["e_loc"]) / np.maximum(np.abs(o["e_loc"]), o["e_abs"]))
        assert err < RTOL_MIXED, (s.name, err)


def test_batch_reports_the_failing_system_and_finishes_the_others(setup):
    systems, ctxs, _ = setup
    args = [_args(s) for s in systems]
    bad = np.array(systems[2].samples, copy=True)
    bad[5, 0] = np.uint64(0)                          # wrong alpha electron count
    args[2] = dict(args[2], samples=bad)
    with pytest.raises(nqs.NQSError) as ei:
        nqs.local_energy_batch(ctxs, args, n_workers=3)
    assert "system 2" in str(ei.value) and ei.value.status == 1
    # the others still give their own results
    ok = nqs.local_energy_batch(ctxs[:2] + ctxs[3:], args[:2] + args[3:])
    for (e, _), s, c in zip(ok, systems[:2] + systems[3:], ctxs[:2] + ctxs[3:]):
        ref, _ = c.local_energy(s.samples, s.counts, s.eps, s.n_draws, s.seed)
        assert np.array_equal(e, ref)


def test_batch_rejects_a_context_shared_by_two_systems(setup):
    systems, ctxs, _ = setup
    with pytest.raises(nqs.NQSError):
        nqs.local_energy_batch([ctxs[0], ctxs[0]], [_args(systems[0])] * 2)


def test_full_batch_every_system_at_full_size():
    """All 64 systems of the uneven batch at their full sample counts (the
    benchmark's launch configuration): every system equals its own
    nqs_local_energy call bit for bit, and two sampled positions per system
    (one drawn at random, the last) match the oracle at their batch positions."""
    systems = W.uneven_batch()
    streams = [torch.cuda.Stream() for _ in systems]
    ctxs = []
    try:
        for s, st in zip(systems, streams):
            c = nqs.Context(0, stream=st.cuda_stream)
            c.set_system(s)
            c.set_precision(nqs.NQS_PREC_MIXED)
            ctxs.append(c)
        got = nqs.local_energy_batch(ctxs, [_args(s) for s in systems], n_workers=8)
        rng = np.random.default_rng(64)
        picks, worst = [], 0.0
        for s, c, (e, summ) in zip(systems, ctxs, got):
            ref, rs = c.local_energy(s.samples, s.counts, s.eps, s.n_draws, s.seed)
            assert np.array_equal(e.view(np.uint64), ref.view(np.uint64)), s.name
            assert summ["e_mean"] == rs["e_mean"] and summ["n_det"] == rs["n_det"]
            picks.append(([int(rng.integers(len(s.samples) - 1)), len(s.samples) - 1], e))
        for s, (idx, e) in zip(systems, picks):
            o = O.local_energy(O.Problem(s), samples=s.samples[idx], index=idx,
                               threads=os.cpu_count() or 1)
            err = np.max(np.abs(e[idx] - o["e_loc"]) / np.maximum(np.abs(o["e_loc"]), o["e_abs"]))
            worst = max(worst, err)
            assert err < RTOL_MIXED, (s.name, err)
        print(f"64 systems, {sum(len(s.samples) for s in systems)} samples: "
              f"max mixed error / max(|E|, e_abs) at the sampled positions = {worst:.3e}")
    finally:
        for c in ctxs:
            c.close()


def test_batch_energy_gradient_equals_per_system_calls(setup):
    """With gradient outputs, each system of the batch runs nqs_energy_gradient
    (E_loc, u_n on the device, the VJP): bit-equal to its own call."""
    systems, ctxs, _ = setup
    sel = [0, 3, 5]
    got = nqs.local_energy_batch([ctxs[i] for i in sel], [dict(_args(systems[i]), grad=True) for i in sel],
                                 n_workers=3)
    for i, (e, summ, (gT, gW, gb)) in zip(sel, got):
        s, c = systems[i], ctxs[i]
        rT, rW, rb, _, re, rs = c.energy_gradient(s.samples, s.counts, s.eps, s.n_draws, s.seed)
        assert np.array_equal(e, re) and summ["e_mean"] == rs["e_mean"]
        assert np.array_equal(gT, rT)
        assert (gW is None and rW is None) or np.array_equal(gW, rW)
