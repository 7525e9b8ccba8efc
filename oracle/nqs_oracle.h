/*
 * nqs_oracle.h -- CPU oracle for the semistochastic local energy.
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow FP64 restatement of the
 * method of "Hybrid tensor network and neural network quantum states for
 * quantum chemistry" (Wu, Zhang, Fang, Li): Eq. (Ham), Eq. (exactElocal),
 * Sec. 2.1-2.4. It exists to check the CUDA library and is only called from
 * tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg. It shares
 * no code, header, table or helper with the CUDA library.
 *
 * Conventions (readings of the paper where it is silent or ambiguous):
 *  - K spatial orbitals, spin orbital s = 2p + spin (alpha=0, beta=1),
 *    the interleaved order of Sec. 3.
 *  - determinant = uint64 [alpha word, beta word]; bit p = orbital p.
 *  - |n> = a+_{s1} a+_{s2} ... |0> with s1 < s2 < ...; an operator on spin
 *    orbital s picks up (-1)^(number of occupied s' < s).
 *  - eri[((p*K+q)*K+r)*K+s] = (pq|rs), chemists' notation; the spin-orbital
 *    integral of Eq. (Ham) is <pq||rs> = (pr|qs) d(sp,sr) d(sq,ss)
 *    - (ps|qr) d(sp,ss) d(sq,sr), d(.,.) comparing spins.
 *  - tensors[e][sigma][a][b]; h_i = sum_{edges e=(j->i)} M_e^{sigma_i} h_j,
 *    h_{-1} = l = e_0, psi_TN = e_0 . h_{K-1} (Eq. MPS-RNN-1D with v = 0;
 *    Eq. bdg-rnn-update without the tensor term for a graph).
 *  - RBM correlator f = prod_k 2 cosh(b_k + sum_s W[k][s] n_s) (Eq. RBM).
 *
 * Parity status: every function here is pinned by tests under tests/ (brute
 * force, closed forms, invariants, an independent Philox implementation).
 */
#ifndef NQS_ORACLE_H
#define NQS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int K, n_alpha, n_beta;
    const double* h1e;   /* [K][K] */
    const double* eri;   /* [K^4] (pq|rs) */
    double e_core;
} or_ham;

typedef struct {
    int K, D;
    int n_edges;
    const int* pred_ptr;     /* [K+1], NULL = chain (edge i joins i-1 -> i) */
    const int* pred_idx;     /* [n_edges], -1 = boundary vector l */
    const double* tensors;   /* [n_edges][4][D][D] */
    int n_hidden;            /* 0 = no correlator */
    const double* rbm_W;     /* [n_hidden][2K] */
    const double* rbm_b;     /* [n_hidden] */
    /* Readout of Sec. 2.2. 0: linear, psi_TN = (h_{K-1})_0 (as above).
     * 1: the normalised MPS-RNN / BDG-RNN of Eq. (MPS-RNN-1D) and
     * Eq. (bdg-rnn-update) without the tensor term: at vertex i (vertices in
     * computation order; vertex i is spatial orbital i) the candidate cells
     * h_i^s = sum_{e=(j->i)} M_e^s h_j + v_i^s, with h_j the cells of the local
     * states already chosen (h_{-1} = e_0), give P_i(s) = sum_a eta_i[a]
     * (h_i^s[a])^2; P~_i(s) = P_i(s) / sum over the local states s' still
     * allowed by the N_alpha / N_beta constraint of Sec. 3 (0 for the others);
     * Phi(n) = prod_i sqrt(P~_i(s_i)) * prod_i sign(w_i . h_i^{s_i} + c_i)
     * (real parameters: the phase arg(.) is a sign; a zero argument counts +). */
    int readout;
    int n_alpha, n_beta;     /* the constraint (readout 1); n_alpha < 0: none,
                                every local state allowed everywhere */
    const double* rnn_v;     /* [K][4][D] */
    const double* rnn_eta;   /* [K][D], >= 0 */
    const double* rnn_w;     /* [K][D] */
    const double* rnn_c;     /* [K] */
    /* Correlator of Sec. 2.3. 0: f = prod_k 2 cosh(theta_k) (Eq. RBM);
     * 1: cos-RBM, f = prod_k cos(theta_k); 2: Ising-RBM, f = prod_k
     * cos(theta_k + 1/2 sum_{s,t} W2[k][s][t] n_s n_t); theta_k = b_k +
     * sum_s W[k][s] n_s over the 2K interleaved spin orbitals. */
    int corr;
    const double* rbm_W2;    /* [n_hidden][2K][2K] (corr 2) */
    /* Tensor term of Eq. (bdg-rnn-update) (the BDG-TensorRNN of Sec. 2.2) with
     * the Tucker factors: for a vertex i with d >= 2 in-edges and rank
     * r = tucker_rank[i] > 0 the cell gains
     *   t_i^s[a] = sum_{i'} Kout[a][i'] sum_{a_1'..a_d'} U^s[i'][a_1']..[a_d'] prod_k z_k[a_k'],
     *   z_k[a'] = sum_b K_k[b][a'] h_{j_k}[b]
     * (j_k the source of the k-th in-edge in edge order, h_{-1} = e_0): the core
     * U^s contracted with the factor matrices Kout, K_1 .. K_d (each D x r) on
     * every mode. Parameters per such vertex, in vertex order: U [4][r^(d+1)]
     * (index order i', a_1', .., a_d'), Kout [D][r], then K_k [D][r] for each
     * in-edge k. */
    const int* tucker_rank;  /* [K] (NULL: no tensor term) */
    const double* tucker;    /* the packed parameters */
} or_ansatz;

typedef struct {
    double e_loc, e_det, e_stoch, h_diag;
    double e_abs;            /* |H_nn| + sum |terms| of E^d and E^s: the scale
                                that rounding errors of the sums are relative to */
    double e_cond;           /* (with_cond only, else 0) first-order rounding scale
                                of the ratios: sum |a_m| (P1(m) f(m) + kappa_n
                                |psi(m)|) / |psi(n)|, a_m the term's coefficient,
                                P1 the first-order bound of the contraction (see
                                or_log_psi_p1) and kappa_n = P1(n)/|psi_TN(n)|: to
                                first order in the unit roundoff u, evaluating every
                                ratio in precision u moves E_loc by at most about
                                u e_cond (times the length of a mat-vec row) */
    double log_abs_psi;      /* log|psi(n)| (TN x correlator) */
    double log_f;            /* log f(n) */
    int sign_psi;
    int64_t n_det;           /* |H_nm| >= eps, off-diagonal */
    int64_t n_rem;
    uint64_t w_total;        /* W: sum of remainder integer weights */
    int w_shift;             /* s in w = ceil(|H| 2^s) */
} or_sample_out;

/* (pq|rs) = sum_x L[x][p][q] L[x][r][s], ascending x, with fused multiply-add. */
void or_build_eri(int K, int n_chol, const double* L, double* eri);

/* Number of single and double excitations that conserve N_alpha, N_beta. */
int64_t or_n_conn(int K, int n_alpha, int n_beta);

/* <n|H|n> (includes e_core). */
double or_diag(const or_ham* ham, const uint64_t* n);

/* All connected m of n in canonical order: rank[i] = i, m determinant, H_mn
 * and the fermionic sign gamma. Returns the count (= or_n_conn). Any output
 * pointer may be NULL. */
int64_t or_connected(const or_ham* ham, const uint64_t* n, uint64_t* dets,
                     double* H, int8_t* sign);

/* Philox4x64 with 10 rounds (Salmon et al., SC'11). */
void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

/* log|psi| and sign for one determinant, full K-site product (no caching). */
void or_log_psi(const or_ansatz* a, const uint64_t* det, double* log_abs, int* sign,
                double* log_f);

/* log P1(det), P1 = sum over edges e = (j -> i) of |g_i|^T |M_e^{sigma_i}| |h_j|,
 * with h_j the forward states of Sec. 2.2 (h_{-1} = e_0) and g_i = d psi_TN /
 * d h_i the exact adjoints. Each mat-vec h_i = sum_e M_e h_j rounded in precision
 * u errs by at most ~u |M_e| |h_j| per entry, and that error reaches psi_TN
 * through g_i, so u P1 bounds the rounding error of psi_TN to first order
 * (running-error analysis; Higham, Accuracy and Stability of Numerical
 * Algorithms, 2nd ed., Ch. 3). For a chain it is
 * sum_t |R_{t+1}|^T |A_t^{sigma_t}| |L_{t-1}|, which grows linearly in K.
 * With the tensor term (multilinear in the sources) it is instead the whole
 * contraction evaluated with the absolute values of every parameter: psi_TN
 * is a sum of products, and its rounding error is at most about (depth) u
 * times that value (ibid.). */
double or_log_psi_p1(const or_ansatz* a, const uint64_t* det);

/* Draw indices (canonical rank) of the stochastic part for sample n with
 * batch index `sample_index`; returns W and the shift through the pointers. */
int or_draws(const or_ham* ham, const uint64_t* n, int64_t sample_index, double eps,
             int n_draws, uint64_t seed, int64_t* ranks, uint64_t* w_total, int* shift);

/* Semistochastic local energy for a batch (OpenMP over samples). Sample s
 * draws with Philox counter index `index[s]` (NULL: s itself), so that a few
 * samples of a larger batch can be recomputed with their batch positions. */
int or_local_energy(const or_ham* ham, const or_ansatz* a, const uint64_t* samples,
                    int64_t Ns, double eps, int n_draws, uint64_t seed,
                    or_sample_out* out, int n_threads, const int64_t* index, int with_cond);

/* d log|psi(n)| / d theta for one determinant: grad_t [n_edges][4][D][D],
 * grad_W [n_hidden][2K], grad_b [n_hidden] (any may be NULL). The tensor
 * part needs the linear readout (readout 0) without the tensor term. */
void or_grad_log_psi(const or_ansatz* a, const uint64_t* det, double* grad_t,
                     double* grad_W, double* grad_b);

/* d log|f(n)| / d W2 [n_hidden][2K][2K] of the Ising-RBM correlator (corr 2). */
void or_grad_corr_W2(const or_ansatz* a, const uint64_t* det, double* grad_W2);

/* Conditional probabilities of the normalised readout (readout 1) along
 * `det`: P~_i(s) for every vertex i and local state s, [K][4]. */
void or_rnn_conditionals(const or_ansatz* a, const uint64_t* det, double* probs);

/* Autoregressive sampling from |Phi|^2 (readout 1; Sec. 2.1, Sec. 3),
 * breadth-first over the vertices. A node of level i is a prefix (the local
 * states of vertices < i) holding `c` of the n_samples draws at offsets
 * o .. o+c-1 (nodes of a level tile [0, n_samples) in prefix order). At vertex
 * i, draw j of a node takes the first allowed local state s with
 * u_j Z < sum_{allowed s' <= s} P_i(s') (Z the sum over the allowed states;
 * the last allowed state if rounding leaves none), where u_j = (x >> 11) 2^-53
 * and x is the first output of Philox4x64-10 with key (seed, 0) and counter
 * (j, i, 1, 0); the children keep the node's offsets in the order of s.
 * Writes up to `capacity` unique determinants and their counts in prefix
 * order and returns how many there are. */
int64_t or_sample(const or_ansatz* a, int64_t n_samples, uint64_t seed, uint64_t* dets,
                  double* counts, int64_t capacity);

#ifdef __cplusplus
}
#endif
#endif
