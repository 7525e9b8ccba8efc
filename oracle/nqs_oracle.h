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
 * sum_t |R_{t+1}|^T |A_t^{sigma_t}| |L_{t-1}|, which grows linearly in K. */
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
 * grad_W [n_hidden][2K], grad_b [n_hidden] (any may be NULL). */
void or_grad_log_psi(const or_ansatz* a, const uint64_t* det, double* grad_t,
                     double* grad_W, double* grad_b);

#ifdef __cplusplus
}
#endif
#endif
