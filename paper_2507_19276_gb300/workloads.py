"""Seeded synthetic inputs for the semistochastic local-energy path.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no integrals are combined, no matrix element, amplitude
or energy is formed here). Both the CUDA library's tests/benchmark and the CPU
oracle's tests take their inputs from here.

Shapes follow the paper's workloads (Sec. 4): an H50-like chain (Sec. 4.1), a
Fe2S2-like dense CAS(30e,20o) active space (Sec. 4.2) and a 3x3x2 H18-like
cluster with a graph-ordered ansatz (Sec. 4.3). The molecular integrals,
FCIDUMP files and trained parameters of the paper are not available, so
seeded random stand-ins with the same sizes and decay structure are used.

Conventions (shared with the library and the oracle):
  * spatial orbitals p = 0..K-1; spin orbital index s = 2p + spin (alpha 0,
    beta 1), the interleaved order of Sec. 3;
  * a determinant is two uint64 words [alpha bits, beta bits], bit p of each
    word is the occupation of spatial orbital p with that spin;
  * local state sigma_p = n_{p,alpha} + 2 n_{p,beta} in {0,1,2,3};
  * Cholesky vectors L[x][p][q] (symmetric in p,q), (pq|rs) = sum_x L_pq L_rs;
  * tensor-network edges: tensors[e][sigma][a][b], h_i = sum_e M_e^{sigma_i} h_j
    (column convention, Eq. (MPS-RNN-1D) with v = 0); pred_idx = -1 marks the
    boundary vector l = e_0; the read-out vector is r = e_0;
  * RBM correlator W[k][s] over the 2K interleaved spin orbitals, b[k];
    `corr` selects 2cosh (0), cos (1) or Ising-cos (2, with W2[k][s][t]);
  * `rnn` = (v [K][4][D], eta [K][D], w [K][D], c [K]) switches the readout to
    the normalised MPS-RNN / BDG-RNN of Sec. 2.2 (None: the linear readout).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

BASE_SEED = 2507192760


@dataclasses.dataclass
class System:
    """One molecule-shaped problem: Hamiltonian, ansatz and a sample batch."""
    name: str
    K: int
    n_alpha: int
    n_beta: int
    h1e: np.ndarray            # [K][K] float64, symmetric
    chol: np.ndarray           # [n_chol][K][K] float64, symmetric in the last two
    e_core: float
    D: int
    tensors: np.ndarray        # [E][4][D][D] float64
    pred_ptr: Optional[np.ndarray]  # [K+1] int32, None for a chain
    pred_idx: Optional[np.ndarray]  # [E] int32 (-1 = boundary), None for a chain
    rbm_W: Optional[np.ndarray]     # [N_h][2K] float64
    rbm_b: Optional[np.ndarray]     # [N_h] float64
    samples: np.ndarray        # [Ns][2] uint64, unique
    counts: np.ndarray         # [Ns] float64
    eps: float                 # deterministic threshold epsilon
    n_draws: int               # N_epsilon
    seed: int                  # Philox key for the stochastic part
    rnn: Optional[tuple] = None          # (v, eta, w, c): normalised readout
    corr: int = 0                        # 0 2cosh, 1 cos-RBM, 2 Ising-RBM
    rbm_W2: Optional[np.ndarray] = None  # [N_h][2K][2K] (Ising-RBM)
    tucker: Optional[tuple] = None       # (ranks [K], packed parameters): tensor term

    @property
    def n_hidden(self) -> int:
        return 0 if self.rbm_W is None else int(self.rbm_W.shape[0])

    @property
    def n_edges(self) -> int:
        return int(self.tensors.shape[0])

    def subset(self, idx) -> "System":
        """Same system with only the samples at positions ``idx``."""
        idx = np.asarray(idx)
        return dataclasses.replace(self, samples=np.ascontiguousarray(self.samples[idx]),
                                   counts=np.ascontiguousarray(self.counts[idx]))


def _sym_chol(rng, n_chol, K, std, decay):
    """Cholesky-like vectors, symmetric in (p,q): L = N(0,std) * decay(p,q)."""
    g = rng.normal(0.0, std, size=(n_chol, K, K))
    g = np.triu(g) + np.transpose(np.triu(g, 1), (0, 2, 1))
    return np.ascontiguousarray(g * decay[None, :, :])


def _banded_h(rng, K, decay):
    g = rng.normal(0.0, 1.0, size=(K, K))
    h = -decay * (1.0 + 0.1 * g)
    return np.ascontiguousarray(0.5 * (h + h.T))


def _mps_tensors(rng, n_edges, D, identity_mask=None):
    """A = I + G/sqrt(D), G ~ N(0,1): 'N(0,1/D) plus identity'."""
    t = rng.normal(0.0, 1.0, size=(n_edges, 4, D, D)) / math.sqrt(D)
    eye = np.eye(D)
    for e in range(n_edges):
        if identity_mask is None or identity_mask[e]:
            t[e] += eye[None, :, :]
    return np.ascontiguousarray(t)


def random_dets(rng, K, na, nb, n):
    """``n`` unique determinants drawn uniformly over fixed N_alpha, N_beta."""
    seen = set()
    out = []
    while len(out) < n:
        a = rng.choice(K, size=na, replace=False)
        b = rng.choice(K, size=nb, replace=False)
        wa = int(np.sum(np.left_shift(np.uint64(1), a.astype(np.uint64))))
        wb = int(np.sum(np.left_shift(np.uint64(1), b.astype(np.uint64))))
        key = (wa, wb)
        if key in seen:
            continue
        seen.add(key)
        out.append(key)
    return np.array(out, dtype=np.uint64).reshape(n, 2)


def all_dets(K, na, nb):
    """Every determinant with N_alpha, N_beta electrons (small K only)."""
    from itertools import combinations
    wa = [sum(1 << p for p in c) for c in combinations(range(K), na)]
    wb = [sum(1 << p for p in c) for c in combinations(range(K), nb)]
    return np.array([(a, b) for a in wa for b in wb], dtype=np.uint64).reshape(-1, 2)


def _zipf_counts(rng, n):
    return rng.zipf(1.2, size=n).astype(np.float64)


def _decay_1d(K, length):
    p = np.arange(K)
    return np.exp(-np.abs(p[:, None] - p[None, :]) / length)


# ----------------------------------------------------------------------------
# The five workloads
# ----------------------------------------------------------------------------

def small_chain(seed_offset=0, n_samples=256):
    """K=8, 4a+4b, rank-16 Cholesky, MPS D=8, no correlator, deterministic."""
    rng = np.random.Generator(np.random.PCG64(BASE_SEED + 0 + seed_offset))
    K, na, nb, D = 8, 4, 4, 8
    dec = _decay_1d(K, 2.0)
    h = _banded_h(rng, K, dec)
    L = _sym_chol(rng, 16, K, 0.3, dec)
    T = _mps_tensors(rng, K, D)
    s = random_dets(rng, K, na, nb, n_samples)
    return System("k8_d8", K, na, nb, h, L, 0.0, D, T, None, None, None, None, s,
                  np.ones(n_samples), 0.0, 0, BASE_SEED + 0 + seed_offset)


def h50_chain(n_samples=4096, seed_offset=0, K=50, D=64, n_hidden=100, eps=1e-3,
              n_draws=1024):
    """H50-shaped chain: K=50, 25a+25b, decay length 2, rank 100, MPS D=64,
    RBM with 100 hidden units, Zipf(1.2) counts, eps=1e-3, 1024 draws."""
    rng = np.random.Generator(np.random.PCG64(BASE_SEED + 1 + seed_offset))
    na = nb = K // 2
    dec = _decay_1d(K, 2.0)
    h = _banded_h(rng, K, dec)
    L = _sym_chol(rng, 2 * K, K, 0.3, dec)
    T = _mps_tensors(rng, K, D)
    W = rng.normal(0.0, 0.01, size=(n_hidden, 2 * K)) if n_hidden else None
    b = rng.normal(0.0, 0.1, size=n_hidden) if n_hidden else None
    s = random_dets(rng, K, na, nb, n_samples)
    c = _zipf_counts(rng, n_samples)
    return System("h50", K, na, nb, h, L, 0.0, D, T, None, None, W, b, s, c, eps,
                  n_draws, BASE_SEED + 1 + seed_offset)


def fe2s2_dense(n_samples=8192, seed_offset=0, D=256):
    """Fe2S2-shaped CAS(30e,20o): dense undecayed integrals, rank 80, MPS
    D=256, RBM with 40 hidden units, Zipf counts, fully deterministic."""
    rng = np.random.Generator(np.random.PCG64(BASE_SEED + 2 + seed_offset))
    K, na, nb = 20, 15, 15
    g = rng.normal(0.0, 0.5, size=(K, K))
    h = np.ascontiguousarray(0.5 * (g + g.T))
    L = _sym_chol(rng, 80, K, 0.2, np.ones((K, K)))
    T = _mps_tensors(rng, K, D)
    W = rng.normal(0.0, 0.01, size=(40, 2 * K))
    b = rng.normal(0.0, 0.1, size=40)
    s = random_dets(rng, K, na, nb, n_samples)
    c = _zipf_counts(rng, n_samples)
    return System("fe2s2", K, na, nb, h, L, 0.0, D, T, None, None, W, b, s, c, 0.0, 0,
                  BASE_SEED + 2 + seed_offset)


def grid_graph(shape=(3, 3, 2), length=1.5, max_in=3):
    """Orbital order and bounded-in-degree DAG for a grid cluster.

    Sites sit on an integer grid. They are ordered by the Fiedler vector of
    the graph Laplacian with weights exp(-d/length) (ties by index), the
    ordering step of Sec. 2.2. Vertex i then takes i-1 and the earlier grid
    neighbours at Manhattan distance 1, keeping at most ``max_in`` of them by
    largest weight. Returns (positions [K][3] in the new order, pred_ptr,
    pred_idx, chain_edge mask).
    """
    pos = np.array([(x, y, z) for x in range(shape[0]) for y in range(shape[1])
                    for z in range(shape[2])], dtype=np.float64)
    K = len(pos)
    d = np.sqrt(((pos[:, None, :] - pos[None, :, :]) ** 2).sum(-1))
    w = np.exp(-d / length)
    np.fill_diagonal(w, 0.0)
    lap = np.diag(w.sum(1)) - w
    evals, evecs = np.linalg.eigh(lap)
    f = evecs[:, 1]
    if f[np.argmax(np.abs(f))] < 0:
        f = -f
    order = sorted(range(K), key=lambda i: (round(float(f[i]), 12), i))
    pos = pos[order]
    d = np.sqrt(((pos[:, None, :] - pos[None, :, :]) ** 2).sum(-1))
    man = np.abs(pos[:, None, :] - pos[None, :, :]).sum(-1)
    ptr = [0]
    idx: List[int] = []
    chain = []
    for i in range(K):
        if i == 0:
            preds = [-1]
        else:
            cand = [j for j in range(i - 1) if man[i, j] == 1.0]
            cand.sort(key=lambda j: (-float(np.exp(-d[i, j] / length)), j))
            preds = [i - 1] + cand[: max_in - 1]
            preds.sort()
        for j in preds:
            idx.append(j)
            chain.append(j == i - 1 or j == -1)
        ptr.append(len(idx))
    return pos, np.array(ptr, np.int32), np.array(idx, np.int32), np.array(chain, bool)


def h18_graph(n_samples=16384, seed_offset=0, D=32, n_hidden=36):
    """H18 3x3x2-shaped: integrals decaying as exp(-d/1.5) in grid distance,
    rank 36, graph-ordered TN with <=3 predecessors, D=32, RBM with 36 hidden
    units, deterministic E_loc (plus the backward pass)."""
    rng = np.random.Generator(np.random.PCG64(BASE_SEED + 3 + seed_offset))
    pos, ptr, idx, chain = grid_graph()
    K, na, nb = 18, 9, 9
    d = np.sqrt(((pos[:, None, :] - pos[None, :, :]) ** 2).sum(-1))
    dec = np.exp(-d / 1.5)
    h = _banded_h(rng, K, dec)
    L = _sym_chol(rng, 36, K, 0.3, dec)
    T = _mps_tensors(rng, len(idx), D, identity_mask=chain)
    W = rng.normal(0.0, 0.01, size=(n_hidden, 2 * K))
    b = rng.normal(0.0, 0.1, size=n_hidden)
    s = random_dets(rng, K, na, nb, n_samples)
    c = _zipf_counts(rng, n_samples)
    return System("h18", K, na, nb, h, L, 0.0, D, T, ptr, idx, W, b, s, c, 0.0, 0,
                  BASE_SEED + 3 + seed_offset)


def uneven_batch(n_systems=64, seed_offset=0, max_samples=4096, min_samples=512):
    """64 independent chains: K uniform over the even numbers 12..40, half
    filling, decay length 2, Cholesky rank 2K, D in {16,32,64}, 512-4096
    samples each, eps=1e-3, 1024 draws."""
    rng = np.random.Generator(np.random.PCG64(BASE_SEED + 4 + seed_offset))
    out = []
    for sidx in range(n_systems):
        K = int(rng.choice(np.arange(12, 41, 2)))
        D = int(rng.choice([16, 32, 64]))
        ns = int(rng.integers(min_samples, max_samples + 1))
        na = nb = K // 2
        dec = _decay_1d(K, 2.0)
        h = _banded_h(rng, K, dec)
        L = _sym_chol(rng, 2 * K, K, 0.3, dec)
        T = _mps_tensors(rng, K, D)
        s = random_dets(rng, K, na, nb, ns)
        c = _zipf_counts(rng, ns)
        out.append(System(f"batch{sidx}_k{K}_d{D}", K, na, nb, h, L, 0.0, D, T, None,
                          None, None, None, s, c, 1e-3, 1024,
                          BASE_SEED + 4 + seed_offset + 1000 * (sidx + 1)))
    return out


def tiny_system(K=4, na=2, nb=2, D=3, n_hidden=0, seed=7, graph=False, chol_rank=None,
                decay=2.0, eps=0.0, n_draws=0, n_samples=None):
    """Small random system for brute-force pins (all determinants as samples)."""
    rng = np.random.Generator(np.random.PCG64(BASE_SEED + 100 + seed))
    dec = _decay_1d(K, decay)
    h = _banded_h(rng, K, dec)
    L = _sym_chol(rng, chol_rank or 2 * K, K, 0.3, dec)
    if graph:
        ptr, idx = [0], []
        chain = []
        for i in range(K):
            preds = [-1] if i == 0 else sorted(set([i - 1] + [j for j in range(i - 1)
                                                             if rng.random() < 0.5][:2]))
            for j in preds:
                idx.append(j)
                chain.append(j == i - 1 or j == -1)
            ptr.append(len(idx))
        ptr = np.array(ptr, np.int32)
        idx = np.array(idx, np.int32)
        T = _mps_tensors(rng, len(idx), D, identity_mask=np.array(chain))
    else:
        ptr = idx = None
        T = _mps_tensors(rng, K, D)
    W = rng.normal(0.0, 0.3, size=(n_hidden, 2 * K)) if n_hidden else None
    b = rng.normal(0.0, 0.3, size=n_hidden) if n_hidden else None
    s = all_dets(K, na, nb)
    if n_samples is not None:
        s = s[rng.permutation(len(s))[:n_samples]]
    c = rng.uniform(0.5, 2.0, size=len(s))
    return System(f"tiny_k{K}", K, na, nb, h, L, 0.0, D, T, ptr, idx, W, b,
                  np.ascontiguousarray(s), c, eps, n_draws, BASE_SEED + 100 + seed)


CONFIGS = {
    "k8_d8": small_chain,
    "h50": h50_chain,
    "fe2s2": fe2s2_dense,
    "h18": h18_graph,
}


def rnn_params(rng, K, D, v_std=0.1):
    """Parameters of the normalised readout (Sec. 2.2): v [K][4][D] ~ N(0, v_std),
    eta [K][D] ~ U(0.5, 1.5), w [K][D] ~ N(0, 1/sqrt(D)), c [K] ~ N(0, 0.1)."""
    v = rng.normal(0.0, v_std, size=(K, 4, D))
    eta = rng.uniform(0.5, 1.5, size=(K, D))
    w = rng.normal(0.0, 1.0 / math.sqrt(D), size=(K, D))
    c = rng.normal(0.0, 0.1, size=K)
    return (v, eta, w, c)


def with_readout(sys_, seed=0, v_std=0.1):
    """The same system with the normalised MPS-RNN / BDG-RNN readout of Sec. 2.2
    (site tensors unchanged; v, eta, w, c drawn from their own seeded stream)."""
    rng = np.random.Generator(np.random.PCG64(BASE_SEED + 300 + seed))
    return dataclasses.replace(sys_, rnn=rnn_params(rng, sys_.K, sys_.D, v_std), name=sys_.name + "_rnn")


def with_correlator(sys_, corr, seed=0, w2_std=0.005):
    """The same system with the cos-RBM (corr 1) or Ising-RBM (corr 2)
    correlator of Sec. 2.3: the same W and b; for corr 2 a symmetric
    W2 [N_h][2K][2K] with entries N(0, w2_std)."""
    W2 = None
    if corr == 2:
        rng = np.random.Generator(np.random.PCG64(BASE_SEED + 400 + seed))
        N = 2 * sys_.K
        W2 = rng.normal(0.0, w2_std, size=(sys_.n_hidden, N, N))
        W2 = 0.5 * (W2 + W2.transpose(0, 2, 1))
    return dataclasses.replace(sys_, corr=corr, rbm_W2=W2,
                               name=sys_.name + ("_cosrbm" if corr == 1 else "_isingrbm"))


def tucker_ranks(pred_ptr, D):
    """chi' = ceil(chi^(2/(d+1))) for every vertex with d >= 2 in-edges (Sec. 2.2),
    0 for the others. Integer arithmetic: the smallest r with r^(d+1) >= chi^2."""
    ranks = []
    for i in range(len(pred_ptr) - 1):
        d = int(pred_ptr[i + 1] - pred_ptr[i])
        r = 0
        if d >= 2:
            r = 1
            while r ** (d + 1) < D * D:
                r += 1
        ranks.append(r)
    return np.array(ranks, np.int32)


def with_tensor_term(sys_, seed=0, core_std=0.3):
    """The same graph system with the BDG-TensorRNN tensor term (Sec. 2.2):
    per vertex with d >= 2 in-edges and rank r = ceil(D^(2/(d+1))), a core
    U [4][r^(d+1)] ~ N(0, core_std) and factor matrices Kout, K_1..K_d
    [D][r] ~ N(0, 1/sqrt(D)), packed in vertex order."""
    rng = np.random.Generator(np.random.PCG64(BASE_SEED + 500 + seed))
    ranks = tucker_ranks(sys_.pred_ptr, sys_.D)
    parts = []
    for i, r in enumerate(ranks):
        if r == 0:
            continue
        d = int(sys_.pred_ptr[i + 1] - sys_.pred_ptr[i])
        parts.append(rng.normal(0.0, core_std, size=4 * r ** (d + 1)))
        parts.append(rng.normal(0.0, 1.0 / math.sqrt(sys_.D), size=(d + 1) * sys_.D * r))
    params = np.concatenate(parts) if parts else np.zeros(0)
    return dataclasses.replace(sys_, tucker=(ranks, params), name=sys_.name + "_tensor")


def h50_rnn(n_samples=4096, seed_offset=0, K=50, D=10, n_hidden=0, eps=0.01, n_draws=100):
    """H50-shaped chain with the paper's BDG(1)-RNN readout at chi = 10 and its
    semistochastic setting eps = 0.01, N_eps = 100 (Sec. 4.1, Fig. 3a): the
    Hamiltonian of h50_chain, site tensors I + G/sqrt(D), v, eta, w, c from
    rnn_params; unique samples uniform over fixed N_alpha / N_beta (the bench
    draws its samples autoregressively instead)."""
    base = h50_chain(n_samples=n_samples, seed_offset=seed_offset, K=K, D=D, n_hidden=n_hidden,
                     eps=eps, n_draws=n_draws)
    return with_readout(base, seed=seed_offset)
