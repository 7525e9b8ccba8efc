"""Pins of the oracle's ansatz, local energy, stochastic part and gradient.

Sec. 2.1 (Eq. exactElocal, Eq. egrad), Sec. 2.2-2.3 (tensor network, RBM
correlator, reweighting), Sec. 2.4 (semistochastic estimator). Each check
compares the oracle with something it does not share code with.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sps
import scipy.sparse.linalg as spla

from oracle import oracle as O
from paper_2507_19276_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# helpers (independent numpy restatements)
# --------------------------------------------------------------------------

def sigmas(det, K):
    a, b = int(det[0]), int(det[1])
    return [((a >> p) & 1) + 2 * ((b >> p) & 1) for p in range(K)]


def psi_tn_paths(sys_, det):
    """Brute-force sum over all source->sink paths of the DAG of the product
    of edge matrices (the unrolled linear recursion of Eq. bdg-rnn-update)."""
    K, D = sys_.K, sys_.D
    sg = sigmas(det, K)
    if sys_.pred_ptr is None:
        preds = {i: [(i - 1, i)] for i in range(K)}
    else:
        preds = {i: [(int(sys_.pred_idx[e]), e) for e in range(sys_.pred_ptr[i], sys_.pred_ptr[i + 1])]
                 for i in range(K)}
    e0 = np.zeros(D); e0[0] = 1.0

    def walk(i):  # all paths ending at vertex i, returned as a summed vector
        total = np.zeros(D)
        for j, e in preds[i]:
            M = sys_.tensors[e, sg[i]]
            total += M @ (e0 if j < 0 else walk(j))
        return total
    return walk(K - 1)[0]


def log_f_numpy(sys_, det):
    if sys_.rbm_W is None:
        return 0.0
    K = sys_.K
    n = np.array([((int(det[s % 2]) >> (s // 2)) & 1) for s in range(2 * K)], float)
    th = sys_.rbm_b + sys_.rbm_W @ n
    return float(np.sum(np.log(2 * np.cosh(th))))


def sparse_oracle_H(P, dets):
    key = {(int(a), int(b)): i for i, (a, b) in enumerate(dets)}
    rows, cols, vals = [], [], []
    for j, d in enumerate(dets):
        rows.append(j); cols.append(j); vals.append(O.diag(P, d))
        md, hv, _ = O.connected(P, d)
        for m, v in zip(md, hv):
            rows.append(key[(int(m[0]), int(m[1]))]); cols.append(j); vals.append(v)
    N = len(dets)
    return sps.csr_matrix((vals, (rows, cols)), shape=(N, N))


def psi_vector(P, dets):
    out = np.empty(len(dets))
    for i, d in enumerate(dets):
        la, sg, _ = O.log_psi(P, d)
        out[i] = sg * np.exp(la)
    return out


# --------------------------------------------------------------------------
# Philox (counter-based generator keyed by (seed, sample, draw))
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed,s,d", [(0, 0, 1), (2507192761, 17, 5), (2**63 + 5, 4095, 1023),
                                      (123, 2**40, 2**33)])
def test_philox_matches_numpy(seed, s, d):
    # numpy's Philox increments its 256-bit counter before each block, so the
    # block for counter c is the first output of a generator started at c-1.
    bg = np.random.Philox(key=np.array([seed, 0], np.uint64),
                          counter=np.array([d - 1, s, 0, 0], np.uint64))
    ref = bg.random_raw(4).astype(np.uint64)
    got = O.philox4x64_10(np.array([d, s, 0, 0], np.uint64), np.array([seed, 0], np.uint64))
    assert np.array_equal(ref, got)


# --------------------------------------------------------------------------
# Ansatz
# --------------------------------------------------------------------------

def test_chain_amplitude_is_the_matrix_product():
    sys_ = W.small_chain()
    P = O.Problem(sys_)
    for det in sys_.samples[:20]:
        sg = sigmas(det, sys_.K)
        v = np.zeros(sys_.D); v[0] = 1.0
        for t in range(sys_.K):
            v = sys_.tensors[t, sg[t]] @ v
        la, s, _ = O.log_psi(P, det)
        assert s == np.sign(v[0])
        assert abs(la - np.log(abs(v[0]))) < 1e-12


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_graph_amplitude_is_the_path_sum(seed):
    sys_ = W.tiny_system(K=6, na=3, nb=2, D=4, seed=seed, graph=True, n_hidden=5)
    assert sys_.pred_idx is not None and len(sys_.pred_idx) > sys_.K
    P = O.Problem(sys_)
    for det in sys_.samples[::13]:
        ref = psi_tn_paths(sys_, det)
        la, s, lf = O.log_psi(P, det)
        assert s == np.sign(ref)
        assert abs((la - lf) - np.log(abs(ref))) < 1e-12
        assert abs(lf - log_f_numpy(sys_, det)) < 1e-12


def test_chain_as_graph_is_bitwise_equal():
    sys_ = W.small_chain()
    g = W.System(**{**sys_.__dict__})
    g.pred_ptr = np.arange(sys_.K + 1, dtype=np.int32)
    g.pred_idx = np.arange(-1, sys_.K - 1, dtype=np.int32)
    P, Pg = O.Problem(sys_), O.Problem(g)
    for det in sys_.samples[:32]:
        assert O.log_psi(P, det) == O.log_psi(Pg, det)


def p1_paths(sys_, det):
    """First-order rounding bound by plain recursion over the DAG (no scaling):
    h(j) = sum of paths from the boundary to j, g(i) = d psi / d h_i = sum of
    transposed paths from the readout back to i, then
    P1 = sum over edges e = (j -> i) of |g(i)|^T |M_e| |h(j)|."""
    K, D = sys_.K, sys_.D
    sg = sigmas(det, K)
    if sys_.pred_ptr is None:
        edges = [(i - 1, i, i) for i in range(K)]
    else:
        edges = [(int(sys_.pred_idx[e]), i, e) for i in range(K)
                 for e in range(sys_.pred_ptr[i], sys_.pred_ptr[i + 1])]
    e0 = np.zeros(D); e0[0] = 1.0

    def h(j):
        if j < 0:
            return e0
        return sum(sys_.tensors[e, sg[i]] @ h(jj) for jj, i, e in edges if i == j)

    def g(i):
        if i == K - 1:
            return e0
        return sum(sys_.tensors[e, sg[k]].T @ g(k) for j, k, e in edges if j == i)

    return sum(np.abs(g(i)) @ np.abs(sys_.tensors[e, sg[i]]) @ np.abs(h(j)) for j, i, e in edges)


@pytest.mark.parametrize("graph", [False, True])
def test_first_order_bound_is_the_path_recursion(graph):
    sys_ = W.tiny_system(K=6, na=3, nb=2, D=4, seed=9, graph=graph)
    P = O.Problem(sys_)
    for det in sys_.samples[::11]:
        ref = p1_paths(sys_, det)
        assert abs(O.log_psi_p1(P, det) - np.log(ref)) < 1e-12
        la, _, lf = O.log_psi(P, det)
        assert O.log_psi_p1(P, det) >= (la - lf) - 1e-12


def test_first_order_bound_closed_form_for_nonnegative_chain():
    """No cancellation: every edge term equals psi, so P1 = K psi_TN."""
    sys_ = W.small_chain()
    pos = W.System(**{**sys_.__dict__})
    pos.tensors = np.abs(sys_.tensors)
    P = O.Problem(pos)
    for det in sys_.samples[:16]:
        la, s, lf = O.log_psi(P, det)
        assert s == 1
        assert abs(O.log_psi_p1(P, det) - (la - lf + np.log(sys_.K))) < 1e-12


def test_condition_scale_closed_form_for_nonnegative_tensors():
    """With nonnegative tensors kappa_n = K and P1(m) = K psi_TN(m), so each
    term contributes 2K |a_m r_m|: e_cond = 2K (e_abs - |H_nn|)."""
    sys_ = W.tiny_system(K=6, na=3, nb=3, D=4, n_hidden=5, seed=12, eps=0.02, n_draws=50)
    pos = W.System(**{**sys_.__dict__})
    pos.tensors = np.abs(sys_.tensors)
    out = O.local_energy(O.Problem(pos), cond=True)
    hd = np.abs(out["h_diag"])
    assert np.allclose(out["e_cond"], 2 * sys_.K * (out["e_abs"] - hd), rtol=1e-12, atol=0)
    signed = O.local_energy(O.Problem(sys_), cond=True)
    assert np.all(signed["e_cond"] >= 2 * (signed["e_abs"] - np.abs(signed["h_diag"])) * (1 - 1e-14))
    assert np.all(O.local_energy(O.Problem(sys_))["e_cond"] == 0.0)


def test_rbm_param_count_matches_paper():
    """Sec. 4.1: cos-RBM(alpha=2) adds 20200 parameters to the H50 ansatz,
    i.e. N_h*N_v + N_h with N_v = 2K spin orbitals and N_h = alpha*N_v."""
    fx = dict(l.split("=") for l in open(os.path.join(GOLDEN, "rbm_param_count.txt"))
              if "=" in l and not l.startswith("#"))
    K, alpha, count = int(fx["K"]), int(fx["alpha"]), int(fx["extra_parameters"])
    sys_ = W.h50_chain(n_samples=4, K=K, n_hidden=alpha * 2 * K)
    assert sys_.rbm_W.size + sys_.rbm_b.size == count


# --------------------------------------------------------------------------
# Exact local energy and its invariants (Eq. exactElocal)
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def small_space():
    sys_ = W.small_chain()
    P = O.Problem(sys_)
    dets = W.all_dets(sys_.K, sys_.n_alpha, sys_.n_beta)
    H = sparse_oracle_H(P, dets)
    psi = psi_vector(P, dets)
    return sys_, P, dets, H, psi


def test_exact_eloc_is_H_psi_over_psi(small_space):
    sys_, P, dets, H, psi = small_space
    key = {(int(a), int(b)): i for i, (a, b) in enumerate(dets)}
    out = O.local_energy(P, eps=0.0, n_draws=0)
    idx = np.array([key[(int(a), int(b))] for a, b in sys_.samples])
    ref = (H @ psi)[idx] / psi[idx]
    assert np.all(out["n_rem"] == 0) and np.all(out["e_stoch"] == 0.0)
    assert np.max(np.abs(out["e_loc"] - ref) / np.maximum(1.0, np.abs(ref))) < 1e-10


def test_weighted_mean_of_eloc_is_rayleigh_quotient(small_space):
    sys_, P, dets, H, psi = small_space
    out = O.local_energy(P, samples=dets, eps=0.0, n_draws=0)
    w = psi ** 2
    lhs = np.sum(w * out["e_loc"]) / np.sum(w)
    rhs = psi @ (H @ psi) / (psi @ psi)
    assert abs(lhs - rhs) < 1e-10 * abs(rhs)


def tt_svd_chain(vec, dets, K, tol=1e-13):
    """Exact MPS (TT-SVD) of a determinant-space vector, local dim 4, written
    into this library's chain layout tensors[t][sigma][out][in]."""
    T = np.zeros((4,) * K)
    for v, d in zip(vec, dets):
        T[tuple(sigmas(d, K))] = v
    cores, r = [], 1
    M = T.reshape(1, -1)
    for t in range(K - 1):
        M = M.reshape(r * 4, -1)
        U, S, Vt = np.linalg.svd(M, full_matrices=False)
        keep = max(1, int(np.sum(S > tol * S[0])))
        cores.append(U[:, :keep].reshape(r, 4, keep))
        M = S[:keep, None] * Vt[:keep]
        r = keep
    cores.append(M.reshape(r, 4, 1))
    D = max(c.shape[2] for c in cores[:-1])
    A = np.zeros((K, 4, D, D))
    for t, c in enumerate(cores):
        for s in range(4):
            A[t, s, :c.shape[2], :c.shape[0]] = c[:, s, :].T
    return A, D


@pytest.mark.slow
def test_eloc_is_constant_for_the_exact_eigenvector(small_space):
    sys_, P, dets, H, psi = small_space
    e0, v0 = spla.eigsh(H, k=1, which="SA", tol=1e-14)
    e0, v0 = float(e0[0]), v0[:, 0]
    A, D = tt_svd_chain(v0, dets, sys_.K)
    g = W.System(**{**sys_.__dict__})
    g.tensors, g.D = A, D
    Pg = O.Problem(g, eri=P.eri)
    out = O.local_energy(Pg, samples=sys_.samples[:24], eps=0.0, n_draws=0)
    assert np.max(np.abs(out["e_loc"] - e0)) < 1e-9


def test_reweighted_energy_identity():
    """Sec. 2.3: with B over |Phi|^2, <E~_loc>_{|Phi|^2} = <Psi|H|Psi>/<Psi|Psi>."""
    sys_ = W.tiny_system(K=5, na=2, nb=2, D=3, n_hidden=4, seed=9)
    P = O.Problem(sys_)
    dets = sys_.samples
    H = sparse_oracle_H(P, dets)
    psi = psi_vector(P, dets)
    lf = np.array([O.log_psi(P, d)[2] for d in dets])
    phi = psi / np.exp(lf)
    out = O.local_energy(P, eps=0.0, n_draws=0)
    c = phi ** 2
    ebar, Bs, m, et = O.summary(out, c)
    lhs = np.sum(c * et) / np.sum(c)
    rhs = psi @ (H @ psi) / (psi @ psi)
    assert abs(lhs - rhs) < 1e-10 * abs(rhs)
    assert abs(ebar - np.sum(c * out["e_loc"]) / np.sum(c)) < 1e-14 * abs(ebar)


# --------------------------------------------------------------------------
# Semistochastic part (Sec. 2.4)
# --------------------------------------------------------------------------

@pytest.fixture(scope="module")
def h50_small():
    sys_ = W.h50_chain(n_samples=2, K=14, D=4, n_hidden=6, eps=2e-2, n_draws=64)
    return sys_, O.Problem(sys_)


def test_draw_index_is_first_prefix_above_target(h50_small):
    """Integer inverse CDF vs a linear scan over the remainder."""
    sys_, P = h50_small
    n = sys_.samples[0]
    _, H, _ = O.connected(P, n)
    ranks, Wt, sh = O.draws(P, n, 0, sys_.eps, 200, sys_.seed)
    rem = np.nonzero(~(np.abs(H) >= sys_.eps))[0]
    w = np.array([int(np.ceil(np.ldexp(abs(H[r]), sh))) for r in rem], dtype=object)
    assert sum(w) == Wt and Wt < 2 ** 63 and Wt > 2 ** 55
    for d in range(200):
        x = int(O.philox4x64_10(np.array([d, 0, 0, 0], np.uint64),
                                np.array([sys_.seed, 0], np.uint64))[0])
        t = (x * Wt) >> 64
        run = 0
        for r, wi in zip(rem, w):
            run += wi
            if run > t:
                break
        assert ranks[d] == r


def test_draw_histogram_follows_abs_H(h50_small):
    """Chi-square of the draw frequencies against P_n(m) ~ |H_nm| (Sec. 2.4)."""
    sys_, P = h50_small
    n = sys_.samples[1]
    _, H, _ = O.connected(P, n)
    rem = np.nonzero(~(np.abs(H) >= sys_.eps))[0]
    p = np.abs(H[rem]) / np.sum(np.abs(H[rem]))
    # bucket the remainder into 20 groups of equal probability
    order = np.argsort(-p)
    edges = np.searchsorted(np.cumsum(p[order]), np.linspace(0, 1, 21)[1:-1])
    groups = np.zeros(len(rem), int)
    for g, e in enumerate(edges):
        groups[order[e:]] = g + 1
    pos = {r: i for i, r in enumerate(rem)}
    counts = np.zeros(21)
    total = 0
    for s in range(60):
        ranks, _, _ = O.draws(P, n, 1, sys_.eps, 400, sys_.seed + 7919 * s)
        for r in ranks:
            counts[groups[pos[r]]] += 1
        total += len(ranks)
    expect = np.array([p[groups == g].sum() for g in range(21)]) * total
    ok = expect > 0
    chi2 = np.sum((counts[ok] - expect[ok]) ** 2 / expect[ok])
    assert chi2 < 60.0  # 20 dof: P(chi2 > 60) ~ 5e-6


def test_stochastic_estimate_is_unbiased(h50_small):
    """E_loc(n, eps, N_eps) averaged over seeds -> the exact E_loc (Sec. 2.4)."""
    sys_, P = h50_small
    exact = O.local_energy(P, eps=0.0, n_draws=0)["e_loc"]
    S = 300
    vals = np.array([O.local_energy(P, eps=sys_.eps, n_draws=16, seed=1000 + s)["e_loc"]
                     for s in range(S)])
    mean, sd = vals.mean(0), vals.std(0, ddof=1)
    assert np.all(np.abs(mean - exact) < 4.5 * sd / np.sqrt(S) + 1e-12)
    # the deterministic part alone (N_eps = 0) is biased (Sec. 4.1): it misses
    # the remainder's whole contribution
    det_only = O.local_energy(P, eps=sys_.eps, n_draws=0)["e_loc"]
    assert np.all(np.abs(det_only - exact) > 1e-3)


def test_batch_index_selects_the_draw_counter(h50_small):
    """A sample recomputed alone with its batch position gives the batch's
    value bit for bit; at another position it draws other determinants."""
    sys_, P = h50_small
    full = O.local_energy(P)
    one = O.local_energy(P, samples=sys_.samples[1:2], index=[1])
    assert one["e_loc"][0] == full["e_loc"][1] and one["e_stoch"][0] == full["e_stoch"][1]
    other = O.local_energy(P, samples=sys_.samples[1:2], index=[0])
    assert other["e_det"][0] == full["e_det"][1]
    assert other["e_stoch"][0] != full["e_stoch"][1]


def test_zero_eps_has_no_stochastic_part(h50_small):
    sys_, P = h50_small
    out = O.local_energy(P, eps=0.0, n_draws=32)
    assert np.all(out["n_rem"] == 0) and np.all(out["e_stoch"] == 0.0)
    nc = O.n_conn(sys_.K, sys_.n_alpha, sys_.n_beta)
    assert np.all(out["n_det"] == nc)


# --------------------------------------------------------------------------
# Gradient (Eq. egrad)
# --------------------------------------------------------------------------

def _perturbed(sys_, which, idx, h):
    g = W.System(**{**sys_.__dict__})
    arr = getattr(sys_, which).copy()
    arr[idx] += h
    setattr(g, which, arr)
    return g


@pytest.mark.parametrize("graph", [False, True])
def test_grad_log_psi_central_differences(graph):
    sys_ = W.tiny_system(K=6, na=3, nb=3, D=4, n_hidden=5, seed=21, graph=graph)
    P = O.Problem(sys_)
    rng = np.random.default_rng(0)
    h = 1e-6
    for det in sys_.samples[::50]:
        gt, gW, gb = O.grad_log_psi(P, det)
        for which, g in (("tensors", gt), ("rbm_W", gW), ("rbm_b", gb)):
            for _ in range(12):
                idx = tuple(rng.integers(0, s) for s in g.shape)
                if which == "tensors":  # pick the sigma the determinant uses at that vertex
                    K = sys_.K
                    e = idx[0]
                    v = e if sys_.pred_ptr is None else int(np.searchsorted(sys_.pred_ptr, e, "right") - 1)
                    idx = (e, sigmas(det, K)[v]) + idx[2:]
                lp = O.log_psi(O.Problem(_perturbed(sys_, which, idx, h)), det)[0]
                lm = O.log_psi(O.Problem(_perturbed(sys_, which, idx, -h)), det)[0]
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g[idx]) < 1e-6 * max(1.0, abs(fd))


def test_energy_gradient_formula_matches_rayleigh_quotient_derivative():
    """Eq. egrad over the full space with |psi|^2 weights equals the finite-
    difference derivative of <psi|H|psi>/<psi|psi>."""
    sys_ = W.tiny_system(K=4, na=2, nb=2, D=3, n_hidden=3, seed=5)
    P = O.Problem(sys_)
    dets = sys_.samples
    H = sparse_oracle_H(P, dets).toarray()

    def energy(s):
        q = O.Problem(s, eri=P.eri)
        v = psi_vector(q, dets)
        return v @ H @ v / (v @ v)

    psi = psi_vector(P, dets)
    w = psi ** 2 / np.sum(psi ** 2)
    out = O.local_energy(P, samples=dets, eps=0.0, n_draws=0)
    ebar = np.sum(w * out["e_loc"])
    grads = [O.grad_log_psi(P, d) for d in dets]
    h = 1e-6
    for which, k, idx in (("tensors", 0, (2, 1, 0, 0)), ("tensors", 0, (1, 3, 2, 1)),
                          ("rbm_W", 1, (1, 3)), ("rbm_b", 2, (2,))):
        g_formula = 2 * np.sum(w * (out["e_loc"] - ebar) * np.array([g[k][idx] for g in grads]))
        fd = (energy(_perturbed(sys_, which, idx, h)) - energy(_perturbed(sys_, which, idx, -h))) / (2 * h)
        assert abs(g_formula - fd) < 1e-6 * max(1.0, abs(fd))
