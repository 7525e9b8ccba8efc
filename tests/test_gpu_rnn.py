"""GPU parity of the normalised MPS-RNN / BDG-RNN readout (Sec. 2.2), the
cos-RBM and Ising-RBM correlators (Sec. 2.3), the autoregressive sampler
(Sec. 2.1, Sec. 3), the outer-product gradient kernels and the energy
gradient (Eq. egrad, Sec. 2.3), through the C ABI, against the CPU oracle.

Bars: log|psi| within 1e-12 absolute; FP64 E_loc within 1e-12 of max(|E|,
e_abs) (plus the first-order ratio-rounding scale 2^-52 e_cond for the linear
readout, as in test_gpu_parity); sampled determinants and counts bit-exact;
gradients within 1e-10 of their largest entry."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_19276_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2507_19276_gb300 import nqs  # noqa: E402

RTOL = 1e-12


def _rnn_cases():
    h50 = W.h50_rnn(n_samples=6, eps=0.01, n_draws=100)
    h18 = W.with_readout(W.h18_graph(n_samples=4), seed=2)
    return {
        "tiny_chain": W.with_readout(W.tiny_system(K=6, na=3, nb=2, D=4, seed=3), seed=3),
        "tiny_graph_cos": W.with_correlator(
            W.with_readout(W.tiny_system(K=6, na=3, nb=3, D=4, n_hidden=5, seed=4, graph=True), seed=4), 1),
        "h50_rnn": h50,
        "h18_rnn_ising": W.with_correlator(h18, 2, seed=1),
    }


@pytest.fixture(scope="module")
def ctx():
    c = nqs.Context(0)
    yield c
    c.close()


def _scale(ref):
    s = np.maximum(np.abs(ref["e_loc"]), ref["e_abs"])
    return s + (2.0 ** -52 / RTOL) * ref["e_cond"]


@pytest.mark.parametrize("name", ["tiny_chain", "tiny_graph_cos", "h50_rnn", "h18_rnn_ising"])
def test_readout_amplitudes_and_local_energy(ctx, name):
    sys_ = _rnn_cases()[name]
    P = O.Problem(sys_)
    ctx.set_system(sys_)
    ctx.set_precision(nqs.NQS_PREC_FP64)
    od, _, _ = O.connected(P, sys_.samples[0])
    dets = np.concatenate([sys_.samples, od[:: max(1, len(od) // 100)]])
    la, sg = ctx.amplitude(dets)
    for d, l, s in zip(dets, la, sg):
        rl, rs, _ = O.log_psi(P, d)
        assert s == rs and (rs == 0 or abs(l - rl) < 1e-12 * max(1.0, abs(rl))), (name, l, rl)
    e, summ = ctx.local_energy(sys_.samples, sys_.counts, sys_.eps, sys_.n_draws, sys_.seed)
    ref = O.local_energy(P, cond=True)
    err = np.max(np.abs(e - ref["e_loc"]) / _scale(ref))
    print(f"{name}: FP64 max |dE| / max(|E|, e_abs) = {err:.3e}")
    assert err < RTOL
    assert summ["n_det"] == int(np.sum(ref["n_det"]))
    # the shared-prefix forms do not evaluate this readout
    ctx.set_precision(nqs.NQS_PREC_MIXED)
    with pytest.raises(nqs.NQSError) as ei:
        ctx.local_energy(sys_.samples, sys_.counts, sys_.eps, sys_.n_draws, sys_.seed)
    assert ei.value.status == 6
    ctx.set_precision(nqs.NQS_PREC_FP64)


@pytest.mark.parametrize("corr", [1, 2])
def test_correlators_on_the_linear_readout(ctx, corr):
    """cos-RBM and Ising-RBM with the chain and graph tensor networks (FP64
    plain form) on the K8-, H50- and H18-shaped systems."""
    cases = [W.with_correlator(W.tiny_system(K=6, na=3, nb=2, D=4, n_hidden=7, seed=8), corr, seed=2),
             W.with_correlator(W.h50_chain(n_samples=3, D=16, n_hidden=20), corr, seed=3),
             W.with_correlator(W.h18_graph(n_samples=4), corr, seed=4)]
    for sys_ in cases:
        P = O.Problem(sys_)
        ctx.set_system(sys_)
        ctx.set_precision(nqs.NQS_PREC_FP64)
        e, _ = ctx.local_energy(sys_.samples, sys_.counts, sys_.eps, sys_.n_draws, sys_.seed)
        ref = O.local_energy(P, cond=True)
        err = np.max(np.abs(e - ref["e_loc"]) / _scale(ref))
        print(f"{sys_.name}: FP64 max scaled error {err:.3e}")
        assert err < RTOL
        la, sg = ctx.amplitude(sys_.samples)
        for d, l, s in zip(sys_.samples, la, sg):
            rl, rs, _ = O.log_psi(P, d)
            assert s == rs and abs(l - rl) < 1e-12 * max(1.0, abs(rl))


@pytest.mark.parametrize("name,n", [("tiny_chain", 100000), ("tiny_graph_cos", 100000), ("h50_rnn", 20000),
                                    ("h18_rnn_ising", 20000)])
def test_sampler_matches_the_oracle(ctx, name, n):
    """Unique determinants and counts bit-exact against the oracle's
    breadth-first sampler (same Philox stream, same prefix order)."""
    sys_ = _rnn_cases()[name]
    ctx.set_system(sys_)
    got, cnt = ctx.sample(n, 2507192761)
    ref, rcnt, nu = O.sample(O.Problem(sys_), n, 2507192761)
    assert len(got) == nu
    assert np.array_equal(got, ref) and np.array_equal(cnt, rcnt)
    assert cnt.sum() == n
    # every sample is a valid determinant of the system
    pa = np.array([bin(int(a)).count("1") for a in got[:, 0]])
    pb = np.array([bin(int(b)).count("1") for b in got[:, 1]])
    assert (pa == sys_.n_alpha).all() and (pb == sys_.n_beta).all()


def test_sampler_capacity_and_state_errors(ctx):
    sys_ = _rnn_cases()["tiny_chain"]
    ctx.set_system(sys_)
    s = np.empty((2, 2), np.uint64)
    c = np.empty(2, np.float64)
    with pytest.raises(nqs.NQSError) as ei:
        nqs.nqs_sample(ctx.h, 5000, 1, s, c, 2)
    assert ei.value.status == 1 and ei.value.n_unique > 2
    ctx.set_system(W.tiny_system(K=6, na=3, nb=2, D=4, seed=3))    # linear readout
    with pytest.raises(nqs.NQSError) as ei:
        nqs.nqs_sample(ctx.h, 10, 1, s, c, 2)
    assert ei.value.status == 2


def _oracle_vjp(P, sys_, u, corr):
    rT = rW = rb = rW2 = None
    for ui, d in zip(u, sys_.samples):
        t, w, b = O.grad_log_psi(P, d)
        rT = ui * t if rT is None else rT + ui * t
        if w is not None:
            rW = ui * w if rW is None else rW + ui * w
            rb = ui * b if rb is None else rb + ui * b
        if corr == 2:
            g2 = O.grad_corr_W2(P, d)
            rW2 = ui * g2 if rW2 is None else rW2 + ui * g2
    return rT, rW, rb, rW2


def _close(a, b):
    return np.max(np.abs(a - b)) <= 1e-10 * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("corr", [0, 1, 2])
def test_vjp_with_the_correlator_kinds_and_chunked_environments(ctx, corr):
    """The outer-product site-tensor gradient and the correlator gradients
    (W, b, W2) against the oracle; grad_chunk = 3 (environments of three
    samples at a time) gives the same result to rounding."""
    base = W.h18_graph(n_samples=7)
    sys_ = W.with_correlator(base, corr, seed=5) if corr else base
    P = O.Problem(sys_)
    ctx.set_system(sys_)
    u = np.random.default_rng(3).normal(size=len(sys_.samples))
    rT, rW, rb, rW2 = _oracle_vjp(P, sys_, u, corr)
    for chunk in (0, 3):
        ctx.set_precision(nqs.NQS_PREC_FP64, grad_chunk=chunk)
        gT = np.empty_like(rT)
        gW, gb = np.empty_like(rW), np.empty_like(rb)
        gW2 = np.empty_like(rW2) if corr == 2 else None
        nqs.nqs_grad_log_psi_vjp2(ctx.h, np.ascontiguousarray(sys_.samples), u, len(u), gT, gW, gb, gW2)
        assert _close(gT, rT) and _close(gW, rW) and _close(gb, rb)
        if corr == 2:
            assert _close(gW2, rW2)
    ctx.set_precision(nqs.NQS_PREC_FP64)


@pytest.mark.parametrize("reweighted", [False, True])
def test_energy_gradient_matches_the_oracle(ctx, reweighted):
    """nqs_energy_gradient = VJP with u_n = 2 c_n (E_loc - E)/sum c (Eq. egrad),
    or with u_n = 2 c_n f~_n^2 (E_loc - E_theta)/sum c (Sec. 2.3), E_loc and the
    weights computed on the device; the oracle's E_loc and per-sample
    gradients give the reference."""
    sys_ = W.with_correlator(W.tiny_system(K=6, na=3, nb=2, D=4, n_hidden=5, seed=9, eps=0.02, n_draws=40,
                                           n_samples=30), 1, seed=6)
    P = O.Problem(sys_)
    ctx.set_system(sys_)
    ctx.set_precision(nqs.NQS_PREC_FP64)
    gT, gW, gb, _, e, summ = ctx.energy_gradient(sys_.samples, sys_.counts, sys_.eps, sys_.n_draws,
                                                 sys_.seed, reweighted=reweighted)
    ref = O.local_energy(P, cond=True)
    c = sys_.counts
    if reweighted:
        ebar, Bs, m, et = O.summary(ref, c)
        f2 = np.exp(2 * ref["log_f"] - m) / Bs
        etheta = np.sum(c * et) / np.sum(c)
        u = 2 * c * f2 * (ref["e_loc"] - etheta) / np.sum(c)
    else:
        u = 2 * c * (ref["e_loc"] - np.sum(c * ref["e_loc"]) / np.sum(c)) / np.sum(c)
    rT, rW, rb, _ = _oracle_vjp(P, sys_, u, 1)
    assert np.max(np.abs(e - ref["e_loc"]) / _scale(ref)) < RTOL
    assert _close(gT, rT) and _close(gW, rW) and _close(gb, rb)


def test_tensor_term_graph_linear_and_normalised_readouts(ctx):
    """BDG-TensorRNN (Eq. bdg-rnn-update with the Tucker tensor term) on the
    H18-shaped graph: amplitudes and FP64 E_loc with the linear readout, and
    with the normalised readout (plus its sampler), against the oracle."""
    base = W.with_tensor_term(W.h18_graph(n_samples=4), seed=3)
    for sys_ in (base, W.with_readout(base, seed=6)):
        P = O.Problem(sys_)
        ctx.set_system(sys_)
        ctx.set_precision(nqs.NQS_PREC_FP64)
        la, sg = ctx.amplitude(sys_.samples)
        for d, l, s in zip(sys_.samples, la, sg):
            rl, rs, _ = O.log_psi(P, d)
            assert s == rs and abs(l - rl) < 1e-12 * max(1.0, abs(rl))
        e, _ = ctx.local_energy(sys_.samples, sys_.counts, sys_.eps, sys_.n_draws, sys_.seed)
        ref = O.local_energy(P, cond=True)
        err = np.max(np.abs(e - ref["e_loc"]) / _scale(ref))
        print(f"{sys_.name}: FP64 max |dE| / max(|E|, e_abs) = {err:.3e}")
        assert err < RTOL
    got, cnt = ctx.sample(5000, 11)
    ref, rcnt, _ = O.sample(O.Problem(W.with_readout(base, seed=6)), 5000, 11)
    assert np.array_equal(got, ref) and np.array_equal(cnt, rcnt)
    # the site-tensor gradient does not cover the tensor term
    with pytest.raises(nqs.NQSError) as ei:
        ctx.grad_log_psi_vjp(W.with_readout(base, seed=6).samples, np.ones(4))
    assert ei.value.status == 6
