"""Pins of the oracle's normalised readout, correlators and autoregressive
sampler (Sec. 2.1-2.3, Sec. 3, Sec. 4.1), each against something other than
the oracle's own formula: the squared norm of a matrix product (isometric site
tensors), normalisation and marginal consistency by brute force over every
determinant, a forced constraint, the paper's parameter counts, special cases
that reduce one correlator to another, central finite differences, the
variational identity on the full K = 6 space, and a chi-square test of the
sampler against the exact |Phi|^2."""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2507_19276_gb300 import workloads as W
from tests import brute_fci as B


def _rnn(K=5, na=2, nb=2, D=3, seed=3, graph=False, n_hidden=0, corr=0):
    s = W.with_readout(W.tiny_system(K=K, na=na, nb=nb, D=D, seed=seed, graph=graph,
                                     n_hidden=n_hidden), seed=seed)
    return W.with_correlator(s, corr, seed=seed) if corr else s


def _phi2(P, dets):
    return np.array([np.exp(2 * O.log_psi(P, d)[0]) for d in dets])


@pytest.mark.parametrize("graph", [False, True])
def test_readout_is_normalised_over_the_constrained_space(graph):
    """sum_n |Phi(n)|^2 = 1 (Sec. 2.3: Phi is normalised) over every
    determinant with N_alpha, N_beta electrons, chain and graph."""
    for K, na, nb in [(5, 2, 2), (6, 3, 1), (4, 0, 2)]:
        s = _rnn(K, na, nb, D=3, seed=K + na, graph=graph)
        total = _phi2(O.Problem(s), W.all_dets(K, na, nb)).sum()
        assert abs(total - 1.0) < 1e-13, (K, na, nb, total)


def test_conditionals_are_the_marginals_of_phi_squared():
    """Autoregressive property: for every prefix, the sum of |Phi|^2 over its
    completions equals the product of the conditionals along the prefix."""
    K, na, nb = 5, 2, 3
    s = _rnn(K, na, nb, D=2, seed=11, graph=True)
    P = O.Problem(s)
    dets = W.all_dets(K, na, nb)
    p2 = _phi2(P, dets)
    sig = lambda d, i: int((int(d[0]) >> i) & 1) + 2 * int((int(d[1]) >> i) & 1)
    for L in range(1, K + 1):
        groups = {}
        for d, v in zip(dets, p2):
            key = tuple(sig(d, i) for i in range(L))
            groups.setdefault(key, [0.0, d])[0] += v
        for key, (mass, d) in groups.items():
            cond = O.rnn_conditionals(P, d)
            prod = np.prod([cond[i, key[i]] for i in range(L)])
            assert abs(mass - prod) < 1e-14, (L, key)


def test_isometric_tensors_give_the_matrix_product_norm():
    """Without the particle-number constraint, v = 0, eta = 1 and site tensors
    with sum_s A_s^T A_s = I (the blocks of an orthonormal 4D x D matrix), the
    site normalisers telescope: |Phi(n)|^2 = |A^{s_{K-1}} ... A^{s_0} e_0|^2,
    and with w = e_0, c = 0 the sign is the product of the signs of the first
    component of the partial products."""
    K, D = 4, 3
    rng = np.random.default_rng(5)
    base = W.tiny_system(K=K, na=2, nb=2, D=D, seed=5)
    T = np.empty((K, 4, D, D))
    for t in range(K):
        q, _ = np.linalg.qr(rng.normal(size=(4 * D, D)))
        T[t] = q.reshape(4, D, D)
    w = np.zeros((K, D)); w[:, 0] = 1.0
    s = W.dataclasses.replace(base, tensors=T, rnn=(np.zeros((K, 4, D)), np.ones((K, D)), w, np.zeros(K)))
    P = O.Problem(s)
    P.ans.n_alpha = -1                      # every local state allowed
    total = 0.0
    for sig in itertools.product(range(4), repeat=K):
        det = np.array([sum(((x & 1) << i) for i, x in enumerate(sig)),
                        sum(((x >> 1) << i) for i, x in enumerate(sig))], np.uint64)
        h = np.eye(D)[:, 0]
        sign = 1
        for t, x in enumerate(sig):
            h = T[t, x] @ h
            sign *= -1 if h[0] < 0 else 1
        la, sg, _ = O.log_psi(P, det)
        assert abs(np.exp(2 * la) - h @ h) < 1e-14
        assert sg == sign
        total += np.exp(2 * la)
    assert abs(total - 1.0) < 1e-13


def test_a_forced_constraint_leaves_probability_one():
    """N_alpha = K, N_beta = 0: every vertex must hold one alpha electron, so
    the only determinant has |Phi| = 1 whatever the parameters."""
    s = _rnn(K=4, na=4, nb=0, D=3, seed=9)
    la, sg, _ = O.log_psi(O.Problem(s), np.array([0b1111, 0], np.uint64))
    assert abs(la) < 1e-15 and sg in (-1, 1)


def test_parameter_count_of_the_paper():
    """Sec. 4.1: BDG(1) at chi = 10, 20, 30 on H50 has 46100, 172100 and 378100
    (complex) parameters: 2K (4 chi^2 + 6 chi + 1) = M, v, eta, w, c per site;
    cos-RBM(alpha = 2) adds 20200 (tests/golden/rbm_param_count.txt)."""
    for chi, want in [(10, 46100), (20, 172100), (30, 378100)]:
        s = W.h50_rnn(n_samples=2, D=chi)
        v, eta, w, c = s.rnn
        assert 2 * (s.tensors.size + v.size + eta.size + w.size + c.size) == want
    s = W.h50_chain(n_samples=2, D=8, n_hidden=200)
    assert s.rbm_W.size + s.rbm_b.size == 20200


def test_ising_with_diagonal_couplings_is_a_cos_rbm():
    """n_s^2 = n_s: an Ising-RBM whose W2 is diagonal equals the cos-RBM with
    W + diag(W2)/2; and cos(theta + pi) = -cos(theta): shifting every b_k by pi
    flips the sign of f by (-1)^N_h and keeps |f|."""
    base = W.tiny_system(K=4, na=2, nb=1, D=2, n_hidden=5, seed=21)
    ising = W.with_correlator(base, 2, seed=3)
    N = 2 * base.K
    diag = np.stack([np.diag(np.diag(x)) for x in ising.rbm_W2])
    ising = W.dataclasses.replace(ising, rbm_W2=diag)
    cosr = W.dataclasses.replace(base, corr=1,
                                 rbm_W=base.rbm_W + 0.5 * np.stack([np.diag(x) for x in diag]))
    shifted = W.dataclasses.replace(cosr, rbm_b=cosr.rbm_b + np.pi)
    Pi, Pc, Ps = O.Problem(ising), O.Problem(cosr), O.Problem(shifted)
    for d in W.all_dets(4, 2, 1):
        li, si, fi = O.log_psi(Pi, d)
        lc, sc, fc = O.log_psi(Pc, d)
        ls, ss, fs = O.log_psi(Ps, d)
        assert abs(fi - fc) < 1e-12 and si == sc
        assert abs(fs - fc) < 1e-12 and ss == sc * (-1) ** base.n_hidden
    assert N == 8


@pytest.mark.parametrize("corr", [0, 1, 2])
def test_correlator_gradients_match_central_differences(corr):
    base = W.tiny_system(K=4, na=2, nb=2, D=2, n_hidden=3, seed=31)
    s = W.with_correlator(base, corr, seed=1) if corr else base
    P = O.Problem(s)
    d = W.all_dets(4, 2, 2)[7]
    _, gW, gb = O.grad_log_psi(P, d)
    h = 1e-6

    def lf(sys_):
        return O.log_psi(O.Problem(sys_), d)[2]

    for k in range(3):
        bp, bm = s.rbm_b.copy(), s.rbm_b.copy()
        bp[k] += h; bm[k] -= h
        fd = (lf(W.dataclasses.replace(s, rbm_b=bp)) - lf(W.dataclasses.replace(s, rbm_b=bm))) / (2 * h)
        assert abs(fd - gb[k]) < 1e-8
        for q in range(8):
            Wp, Wm = s.rbm_W.copy(), s.rbm_W.copy()
            Wp[k, q] += h; Wm[k, q] -= h
            fd = (lf(W.dataclasses.replace(s, rbm_W=Wp)) - lf(W.dataclasses.replace(s, rbm_W=Wm))) / (2 * h)
            assert abs(fd - gW[k, q]) < 1e-8
    if corr == 2:
        g2 = O.grad_corr_W2(P, d)
        for k, q, r in [(0, 0, 2), (1, 3, 3), (2, 5, 1), (2, 6, 7)]:
            Wp, Wm = s.rbm_W2.copy(), s.rbm_W2.copy()
            Wp[k, q, r] += h; Wm[k, q, r] -= h
            fd = (lf(W.dataclasses.replace(s, rbm_W2=Wp)) - lf(W.dataclasses.replace(s, rbm_W2=Wm))) / (2 * h)
            assert abs(fd - g2[k, q, r]) < 1e-8


@pytest.mark.parametrize("kind", ["rnn_chain", "rnn_graph_cos", "ising"])
def test_variational_identity_on_the_full_space(kind):
    """sum_n |psi|^2 E_loc(n) / sum_n |psi|^2 = <psi|H|psi> / <psi|psi> with the
    exact E_loc (eps = 0) and H from brute-force second quantisation."""
    if kind == "rnn_chain":
        s = _rnn(K=5, na=2, nb=2, D=3, seed=41)
    elif kind == "rnn_graph_cos":
        s = _rnn(K=5, na=2, nb=3, D=3, seed=42, graph=True, n_hidden=4, corr=1)
    else:
        s = W.with_correlator(W.tiny_system(K=5, na=2, nb=2, D=3, seed=43, n_hidden=4), 2, seed=2)
    dets = W.all_dets(s.K, s.n_alpha, s.n_beta)
    s = W.dataclasses.replace(s, samples=dets, counts=np.ones(len(dets)))
    P = O.Problem(s)
    out = O.local_energy(P, eps=0.0, n_draws=0)
    la = out["log_abs_psi"]
    sg = out["sign_psi"].astype(np.float64)
    psi = sg * np.exp(la - la.max())
    H = B.hamiltonian(s.h1e, P.eri, s.K, dets, s.e_core)
    rq = psi @ H @ psi / (psi @ psi)
    wmean = np.sum(psi ** 2 * out["e_loc"]) / np.sum(psi ** 2)
    assert abs(rq - wmean) < 1e-11 * max(1.0, abs(rq))


def test_sampler_counts_follow_phi_squared():
    """Counts sum to the number of draws, every sample is a distinct valid
    determinant, and the histogram passes a chi-square test against the exact
    |Phi|^2 (Sec. 2.1: autoregressive sampling is exact)."""
    K, na, nb = 5, 2, 2
    s = _rnn(K, na, nb, D=3, seed=51, graph=True)
    P = O.Problem(s)
    dets = W.all_dets(K, na, nb)
    p2 = _phi2(P, dets)
    N = 200000
    got, cnt, n = O.sample(P, N, 2507192761)
    assert n == len(got) and cnt.sum() == N
    assert len({(int(a), int(b)) for a, b in got}) == n
    for a, b in got:
        assert bin(int(a)).count("1") == na and bin(int(b)).count("1") == nb
    index = {(int(a), int(b)): i for i, (a, b) in enumerate(dets)}
    obs = np.zeros(len(dets))
    for (a, b), c in zip(got, cnt):
        obs[index[(int(a), int(b))]] = c
    exp = N * p2
    keep = exp > 5
    chi2 = np.sum((obs[keep] - exp[keep]) ** 2 / exp[keep])
    dof = keep.sum() - 1
    assert chi2 < dof + 6 * np.sqrt(2 * dof), (chi2, dof)
    # a different seed gives a different but equally valid histogram
    got2, cnt2, _ = O.sample(P, N, 7)
    assert cnt2.sum() == N and not (len(got2) == len(got) and np.array_equal(cnt2, cnt))


def _three_vertex_graph(D=3, seed=71):
    """Vertices 0 <- l, 1 <- 0, 2 <- {0, 1}: vertex 2 carries the tensor term."""
    base = W.tiny_system(K=3, na=1, nb=1, D=D, seed=seed)
    rng = np.random.default_rng(seed)
    ptr = np.array([0, 1, 2, 4], np.int32)
    idx = np.array([-1, 0, 0, 1], np.int32)
    T = rng.normal(0.0, 0.7, size=(4, 4, D, D))
    return W.with_tensor_term(W.dataclasses.replace(base, tensors=T, pred_ptr=ptr, pred_idx=idx), seed=seed,
                              core_std=0.8)


def test_tensor_term_equals_the_dense_tucker_reconstruction():
    """Eq. (bdg-rnn-update) with the Tucker form of Sec. 2.2: the factored
    contraction of the oracle equals the full tensor T^s = U^s x Kout x K_1 x
    K_2 rebuilt with numpy.einsum and applied to the source cells, for every
    local-state string of a three-vertex graph (linear readout)."""
    s = _three_vertex_graph()
    D = s.D
    ranks, params = s.tucker
    assert list(ranks) == [0, 0, 3]          # ceil(3^(2/3)) = 3 for the two-edge vertex
    r = 3
    U = params[:4 * r ** 3].reshape(4, r, r, r)
    Kout, K1, K2 = params[4 * r ** 3:].reshape(3, D, r)
    Tfull = np.einsum("sopq,ao,bp,cq->sabc", U, Kout, K1, K2)
    P = O.Problem(s)
    e0 = np.eye(D)[:, 0]
    for sig in itertools.product(range(4), repeat=3):
        det = np.array([sum(((x & 1) << i) for i, x in enumerate(sig)),
                        sum(((x >> 1) << i) for i, x in enumerate(sig))], np.uint64)
        h0 = s.tensors[0, sig[0]] @ e0
        h1 = s.tensors[1, sig[1]] @ h0
        h2 = s.tensors[2, sig[2]] @ h0 + s.tensors[3, sig[2]] @ h1 + np.einsum("abc,b,c->a", Tfull[sig[2]], h0, h1)
        la, sg, _ = O.log_psi(P, det)
        if h2[0] == 0.0:
            assert sg == 0
        else:
            assert sg == (1 if h2[0] > 0 else -1)
            assert abs(la - np.log(abs(h2[0]))) < 1e-12


def test_tensor_term_keeps_the_readout_normalised():
    """BDG-TensorRNN with the normalised readout: sum |Phi|^2 = 1."""
    s = W.with_readout(_three_vertex_graph(D=4, seed=72), seed=5)
    s = W.dataclasses.replace(s, n_alpha=1, n_beta=2)
    total = _phi2(O.Problem(s), W.all_dets(3, 1, 2)).sum()
    assert abs(total - 1.0) < 1e-13


def test_tensor_term_rounding_scale_is_psi_for_nonnegative_parameters():
    """With the tensor term the rounding scale P1 is the contraction evaluated
    with absolute values: for nonnegative tensors, factors and cores it is
    psi_TN itself; with signs it can only be larger."""
    s = _three_vertex_graph(D=3, seed=73)
    pos = W.dataclasses.replace(s, tensors=np.abs(s.tensors), tucker=(s.tucker[0], np.abs(s.tucker[1])))
    Pp, Ps = O.Problem(pos), O.Problem(s)
    for sig in itertools.product(range(4), repeat=3):
        det = np.array([sum(((x & 1) << i) for i, x in enumerate(sig)),
                        sum(((x >> 1) << i) for i, x in enumerate(sig))], np.uint64)
        la, sg, _ = O.log_psi(Pp, det)
        assert sg == 1 and abs(O.log_psi_p1(Pp, det) - la) < 1e-12
        la_s, _, _ = O.log_psi(Ps, det)
        assert O.log_psi_p1(Ps, det) >= la_s - 1e-12
