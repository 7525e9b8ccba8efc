/*
 * nqs_oracle.c -- CPU oracle for the semistochastic local energy.
 *
 * TEST INFRASTRUCTURE ONLY (see nqs_oracle.h). Plain FP64 loops that follow
 * the paper's definitions step by step. Compile with -ffp-contract=off so
 * that every a*b+c is rounded twice unless fma() is written out.
 */
#include "nqs_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ERI(K, eri, p, q, r, s) ((eri)[((((size_t)(p)) * (K) + (q)) * (K) + (r)) * (K) + (s)])

/* ------------------------------------------------------------------------ */
/* Integrals (Eq. Ham): (pq|rs) from Cholesky-like vectors                   */
/* ------------------------------------------------------------------------ */

void or_build_eri(int K, int n_chol, const double* L, double* eri)
{
    const size_t KK = (size_t)K * K;
    for (int p = 0; p < K; ++p)
        for (int q = 0; q < K; ++q)
            for (int r = 0; r < K; ++r)
                for (int s = 0; s < K; ++s) {
                    double acc = 0.0;
                    for (int x = 0; x < n_chol; ++x)
                        acc = fma(L[x * KK + (size_t)p * K + q], L[x * KK + (size_t)r * K + s], acc);
                    ERI(K, eri, p, q, r, s) = acc;
                }
}

/* ------------------------------------------------------------------------ */
/* Occupation numbers and fermionic operators (Sec. 2.1, Sec. 3 ordering)    */
/* ------------------------------------------------------------------------ */

static void unpack(int K, const uint64_t* det, int* occ)
{
    for (int p = 0; p < K; ++p) {
        occ[2 * p] = (int)((det[0] >> p) & 1u);
        occ[2 * p + 1] = (int)((det[1] >> p) & 1u);
    }
}

static void pack(int K, const int* occ, uint64_t* det)
{
    det[0] = det[1] = 0;
    for (int p = 0; p < K; ++p) {
        if (occ[2 * p]) det[0] |= (uint64_t)1 << p;
        if (occ[2 * p + 1]) det[1] |= (uint64_t)1 << p;
    }
}

/* a_s acting on an occupied s: returns the phase, empties s. */
static int annihilate(int* occ, int s)
{
    int c = 0;
    for (int t = 0; t < s; ++t) c += occ[t];
    occ[s] = 0;
    return (c & 1) ? -1 : 1;
}

/* a+_s acting on an empty s: returns the phase, fills s. */
static int create(int* occ, int s)
{
    int c = 0;
    for (int t = 0; t < s; ++t) c += occ[t];
    occ[s] = 1;
    return (c & 1) ? -1 : 1;
}

static int64_t binom2(int64_t n) { return n * (n - 1) / 2; }

int64_t or_n_conn(int K, int na, int nb)
{
    int64_t va = K - na, vb = K - nb;
    int64_t sa = (int64_t)na * va, sb = (int64_t)nb * vb;
    return sa + sb + binom2(na) * binom2(va) + binom2(nb) * binom2(vb) + sa * sb;
}

double or_diag(const or_ham* h, const uint64_t* n)
{
    const int K = h->K;
    int occ[128];
    unpack(K, n, occ);
    double e = h->e_core;
    for (int s = 0; s < 2 * K; ++s)
        if (occ[s]) e += h->h1e[(s / 2) * K + s / 2];
    for (int s = 0; s < 2 * K; ++s) {
        if (!occ[s]) continue;
        for (int t = 0; t < 2 * K; ++t) {
            if (!occ[t]) continue;
            double v = ERI(K, h->eri, s / 2, s / 2, t / 2, t / 2);
            if ((s & 1) == (t & 1)) v -= ERI(K, h->eri, s / 2, t / 2, t / 2, s / 2);
            e += 0.5 * v;
        }
    }
    return e;
}

/* One excitation: spin orbitals i (,j) emptied and a (,b) filled. For a
 * double, m = a+_a a+_b a_j a_i |n> up to the phase gamma. */
typedef struct { int kind, i, j, a, b; } exc_t;

/* The canonical order: blocks [S_alpha, S_beta, D_alphaalpha, D_betabeta,
 * D_alphabeta]; inside a block, positions among the occupied / empty
 * orbitals of that spin in ascending order, pairs lexicographic. */
static int64_t list_excitations(int K, const uint64_t* n, exc_t* out)
{
    int occ[2][64], vir[2][64], no[2] = {0, 0}, nv[2] = {0, 0};
    for (int sp = 0; sp < 2; ++sp)
        for (int p = 0; p < K; ++p) {
            if ((n[sp] >> p) & 1u) occ[sp][no[sp]++] = p;
            else vir[sp][nv[sp]++] = p;
        }
    int64_t c = 0;
    for (int sp = 0; sp < 2; ++sp)
        for (int io = 0; io < no[sp]; ++io)
            for (int ao = 0; ao < nv[sp]; ++ao) {
                exc_t e = {1, 2 * occ[sp][io] + sp, -1, 2 * vir[sp][ao] + sp, -1};
                out[c++] = e;
            }
    for (int sp = 0; sp < 2; ++sp)
        for (int io = 0; io < no[sp]; ++io)
            for (int jo = io + 1; jo < no[sp]; ++jo)
                for (int ao = 0; ao < nv[sp]; ++ao)
                    for (int bo = ao + 1; bo < nv[sp]; ++bo) {
                        exc_t e = {2, 2 * occ[sp][io] + sp, 2 * occ[sp][jo] + sp,
                                   2 * vir[sp][ao] + sp, 2 * vir[sp][bo] + sp};
                        out[c++] = e;
                    }
    for (int io = 0; io < no[0]; ++io)
        for (int ao = 0; ao < nv[0]; ++ao)
            for (int jo = 0; jo < no[1]; ++jo)
                for (int bo = 0; bo < nv[1]; ++bo) {
                    exc_t e = {2, 2 * occ[0][io], 2 * occ[1][jo] + 1, 2 * vir[0][ao],
                               2 * vir[1][bo] + 1};
                    out[c++] = e;
                }
    return c;
}

/* Slater-Condon matrix element <m|H|n> and the phase, Eq. (Ham) applied to n. */
static double matrix_element(const or_ham* h, const int* occ_n, const exc_t* e, int* occ_m,
                             int* gamma)
{
    const int K = h->K;
    memcpy(occ_m, occ_n, sizeof(int) * 2 * K);
    int g;
    double v;
    const int I = e->i / 2, A = e->a / 2;
    if (e->kind == 1) {
        g = annihilate(occ_m, e->i);
        g *= create(occ_m, e->a);
        /* h_ai + sum_{j common} (ai|jj) - sum_{j common, same spin} (aj|ji) */
        v = h->h1e[A * K + I];
        for (int s = 0; s < 2 * K; ++s)
            if (occ_n[s] && s != e->i) v = v + ERI(K, h->eri, A, I, s / 2, s / 2);
        for (int s = 0; s < 2 * K; ++s)
            if (occ_n[s] && s != e->i && (s & 1) == (e->i & 1))
                v = v - ERI(K, h->eri, A, s / 2, s / 2, I);
    } else {
        const int J = e->j / 2, B = e->b / 2;
        g = annihilate(occ_m, e->i);
        g *= annihilate(occ_m, e->j);
        g *= create(occ_m, e->b);
        g *= create(occ_m, e->a);
        /* <ab||ij> = (ai|bj) - (aj|bi) [second term only for equal spins] */
        v = ERI(K, h->eri, A, I, B, J);
        if ((e->i & 1) == (e->j & 1)) v = v - ERI(K, h->eri, A, J, B, I);
    }
    *gamma = g;
    return g < 0 ? -v : v;
}

int64_t or_connected(const or_ham* h, const uint64_t* n, uint64_t* dets, double* H,
                     int8_t* sign)
{
    const int K = h->K;
    int64_t nc = or_n_conn(K, h->n_alpha, h->n_beta);
    exc_t* ex = (exc_t*)malloc(sizeof(exc_t) * (size_t)(nc > 0 ? nc : 1));
    int64_t c = list_excitations(K, n, ex);
    int occ_n[128], occ_m[128];
    unpack(K, n, occ_n);
    for (int64_t r = 0; r < c; ++r) {
        int g;
        double v = matrix_element(h, occ_n, &ex[r], occ_m, &g);
        if (dets) pack(K, occ_m, &dets[2 * r]);
        if (H) H[r] = v;
        if (sign) sign[r] = (int8_t)g;
    }
    free(ex);
    return c;
}

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11)                         */
/* ------------------------------------------------------------------------ */

static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo)
{
    unsigned __int128 p = (unsigned __int128)a * b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void or_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, x0, &hi0, &lo0);
        mulhilo64(M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------ */
/* Ansatz: tensor network (Eq. MPS-RNN-1D / bdg-rnn-update, v = 0) x RBM     */
/* ------------------------------------------------------------------------ */

/* Edges into vertex i as [begin, end) of pred_idx; a chain has edge i: i-1 -> i. */
static void edges_of(const or_ansatz* a, int i, int* e0, int* e1)
{
    if (a->pred_ptr) { *e0 = a->pred_ptr[i]; *e1 = a->pred_ptr[i + 1]; }
    else { *e0 = i; *e1 = i + 1; }
}

static int edge_src(const or_ansatz* a, int e) { return a->pred_ptr ? a->pred_idx[e] : e - 1; }

static const double* tensor(const or_ansatz* a, int e, int sigma)
{
    return a->tensors + ((size_t)e * 4 + sigma) * a->D * a->D;
}

/* Parameters of vertex i's tensor term (NULL when it has none): *d in-edges,
 * rank *r; the blocks of the vertices before i are skipped in order. */
static const double* tucker_block(const or_ansatz* a, int i, int* d, int* r)
{
    if (!a->tucker_rank || !a->pred_ptr) return NULL;
    const double* p = a->tucker;
    for (int v = 0; v <= i; ++v) {
        const int dv = a->pred_ptr[v + 1] - a->pred_ptr[v], rv = a->tucker_rank[v];
        if (dv < 2 || rv <= 0) continue;
        if (v == i) { *d = dv; *r = rv; return p; }
        size_t core = 1;
        for (int k = 0; k <= dv; ++k) core *= (size_t)rv;
        p += 4 * core + (size_t)(dv + 1) * a->D * rv;
    }
    return NULL;
}

/* Tensor term t_i^s of vertex i for the in-edge sources src[k] (length D
 * each): added to out[0..D). With absval, every parameter enters by its
 * absolute value (the sources are passed as absolute values by the caller):
 * the magnitude scale of the same expression (see or_log_psi_p1). */
static void tensor_term_x(const or_ansatz* a, int i, int s, const double* const* src, double* out, int absval)
{
    int d = 0, r = 0;
    const double* blk = tucker_block(a, i, &d, &r);
    if (!blk) return;
    const int D = a->D;
    size_t core = 1;
    for (int k = 0; k < d; ++k) core *= (size_t)r;          /* r^d entries per output index */
    const double* U = blk + (size_t)s * core * r;
    const double* Kout = blk + 4 * core * r;
    double* z = (double*)malloc(sizeof(double) * d * r);
    for (int k = 0; k < d; ++k) {
        const double* Kk = Kout + (size_t)(k + 1) * D * r;
        for (int q = 0; q < r; ++q) {
            double acc = 0.0;
            for (int b = 0; b < D; ++b) {
                const double kk = Kk[(size_t)b * r + q];
                acc += (absval ? fabs(kk) : kk) * src[k][b];
            }
            z[k * r + q] = acc;
        }
    }
    double* y = (double*)calloc(r, sizeof(double));
    for (int o = 0; o < r; ++o) {
        double acc = 0.0;
        for (size_t m = 0; m < core; ++m) {
            /* digits of m: a_1' (most significant) .. a_d' */
            double prod = absval ? fabs(U[(size_t)o * core + m]) : U[(size_t)o * core + m];
            size_t rem = m;
            for (int k = d - 1; k >= 0; --k) {
                prod *= z[k * r + (int)(rem % (size_t)r)];
                rem /= (size_t)r;
            }
            acc += prod;
        }
        y[o] = acc;
    }
    for (int q = 0; q < D; ++q) {
        double acc = 0.0;
        for (int o = 0; o < r; ++o) {
            const double ko = Kout[(size_t)q * r + o];
            acc += (absval ? fabs(ko) : ko) * y[o];
        }
        out[q] += acc;
    }
    free(z);
    free(y);
}

static void tensor_term(const or_ansatz* a, int i, int s, const double* const* src, double* out)
{
    tensor_term_x(a, i, s, src, out, 0);
}

/* Rescale v by a power of two so that max|v| is in [0.5, 1); returns the exponent. */
static int renorm(double* v, int D)
{
    double m = 0.0;
    for (int k = 0; k < D; ++k) if (fabs(v[k]) > m) m = fabs(v[k]);
    if (m == 0.0) return 0;
    int e;
    frexp(m, &e);
    for (int k = 0; k < D; ++k) v[k] = ldexp(v[k], -e);
    return e;
}

/* Forward states h_i (scaled, exponents ex[i]) for sigma[0..K-1]; with
 * absval every parameter enters by its absolute value (the magnitude scale of
 * the same contraction, see or_log_psi_p1). */
static void forward_states_x(const or_ansatz* a, const int* sigma, double* hs, int* ex, int absval)
{
    const int K = a->K, D = a->D;
    double* tmp = (double*)malloc(sizeof(double) * D);
    double* e0v = (double*)calloc(D, sizeof(double));
    e0v[0] = 1.0;
    for (int i = 0; i < K; ++i) {
        int e0, e1;
        edges_of(a, i, &e0, &e1);
        int eref = -100000;
        for (int e = e0; e < e1; ++e) {
            int j = edge_src(a, e);
            int ej = j < 0 ? 0 : ex[j];
            if (ej > eref) eref = ej;
        }
        /* the tensor term scales with the product of its sources: exponent sum */
        int dt = 0, rt = 0, et = 0;
        const int has_t = tucker_block(a, i, &dt, &rt) != NULL;
        if (has_t) {
            for (int e = e0; e < e1; ++e) { int j = edge_src(a, e); et += j < 0 ? 0 : ex[j]; }
            if (et > eref) eref = et;
        }
        double* hi = hs + (size_t)i * D;
        for (int k = 0; k < D; ++k) hi[k] = 0.0;
        for (int e = e0; e < e1; ++e) {
            int j = edge_src(a, e);
            const double* M = tensor(a, e, sigma[i]);
            for (int r = 0; r < D; ++r) {
                double s = 0.0;
                for (int c = 0; c < D; ++c) {
                    double hj = (j < 0) ? (c == 0 ? 1.0 : 0.0) : hs[(size_t)j * D + c];
                    s += (absval ? fabs(M[r * D + c]) : M[r * D + c]) * hj;
                }
                tmp[r] = s;
            }
            int ej = j < 0 ? 0 : ex[j];
            for (int r = 0; r < D; ++r) hi[r] += ldexp(tmp[r], ej - eref);
        }
        if (has_t) {
            const double* src[8];
            for (int e = e0; e < e1; ++e) {
                int j = edge_src(a, e);
                src[e - e0] = j < 0 ? e0v : hs + (size_t)j * D;
            }
            for (int r = 0; r < D; ++r) tmp[r] = 0.0;
            tensor_term_x(a, i, sigma[i], src, tmp, absval);
            for (int r = 0; r < D; ++r) hi[r] += ldexp(tmp[r], et - eref);
        }
        ex[i] = eref + renorm(hi, D);
    }
    free(tmp);
    free(e0v);
}

static void forward_states(const or_ansatz* a, const int* sigma, double* hs, int* ex)
{
    forward_states_x(a, sigma, hs, ex, 0);
}

static void sigma_of(int K, const uint64_t* det, int* sigma)
{
    for (int p = 0; p < K; ++p)
        sigma[p] = (int)((det[0] >> p) & 1u) + 2 * (int)((det[1] >> p) & 1u);
}

/* log(2 cosh x) without overflow. */
static double log2cosh(double x)
{
    double ax = fabs(x);
    return ax + log1p(exp(-2.0 * ax));
}

/* theta_k(n) of the correlator (Sec. 2.3): b_k + sum_s W[k][s] n_s, plus
 * 1/2 sum_{s,t} W2[k][s][t] n_s n_t for the Ising-RBM. */
static double corr_theta(const or_ansatz* a, const int* occ, int k)
{
    const int N = 2 * a->K;
    double th = a->rbm_b[k];
    for (int s = 0; s < N; ++s)
        if (occ[s]) th += a->rbm_W[(size_t)k * N + s];
    if (a->corr == 2) {
        double q = 0.0;
        for (int s = 0; s < N; ++s)
            for (int t = 0; t < N; ++t)
                if (occ[s] && occ[t]) q += a->rbm_W2[((size_t)k * N + s) * N + t];
        th += 0.5 * q;
    }
    return th;
}

/* log|f(n)| and the sign of f (Eq. RBM, cos-RBM and Ising-RBM of Sec. 2.3). */
static double rbm_log_f(const or_ansatz* a, const uint64_t* det, int* sign_f)
{
    *sign_f = 1;
    if (a->n_hidden <= 0) return 0.0;
    const int K = a->K;
    int occ[128];
    unpack(K, det, occ);
    double lf = 0.0;
    for (int k = 0; k < a->n_hidden; ++k) {
        const double th = corr_theta(a, occ, k);
        if (a->corr == 0) {
            lf += log2cosh(th);
        } else {
            const double c = cos(th);
            if (c < 0.0) *sign_f = -*sign_f;
            lf += log(fabs(c));
        }
    }
    if (isinf(lf) && lf < 0) *sign_f = 0;
    return lf;
}

/* Local state s = n_alpha + 2 n_beta at vertex i is allowed when, after it,
 * neither spin exceeds its electron count and the vertices after i can still
 * hold the electrons left (the N_alpha / N_beta constraint of Sec. 3). */
static int state_allowed(const or_ansatz* a, int i, int na_done, int nb_done, int s)
{
    if (a->n_alpha < 0) return 1;        /* no particle-number constraint */
    const int ea = na_done + (s & 1), eb = nb_done + (s >> 1), left = a->K - 1 - i;
    return ea <= a->n_alpha && eb <= a->n_beta && a->n_alpha - ea <= left && a->n_beta - eb <= left;
}

/* Candidate cells cand[s][r] = v_i^s[r] + sum_{e=(j->i)} sum_c M_e^s[r][c] h_j[c]
 * for the four local states of vertex i, and P_i(s) = sum_r eta_i[r] cand[s][r]^2
 * (Eq. MPS-RNN-1D / bdg-rnn-update without the tensor term, Sec. 2.2). */
static void rnn_candidates(const or_ansatz* a, int i, const double* hs, double* cand, double* P)
{
    const int D = a->D;
    int e0, e1;
    edges_of(a, i, &e0, &e1);
    for (int s = 0; s < 4; ++s) {
        double* h = cand + (size_t)s * D;
        for (int r = 0; r < D; ++r) {
            double acc = a->rnn_v[((size_t)i * 4 + s) * D + r];
            for (int e = e0; e < e1; ++e) {
                const int j = edge_src(a, e);
                const double* M = tensor(a, e, s);
                for (int c = 0; c < D; ++c) {
                    const double hj = (j < 0) ? (c == 0 ? 1.0 : 0.0) : hs[(size_t)j * D + c];
                    acc += M[r * D + c] * hj;
                }
            }
            h[r] = acc;
        }
        int dt = 0, rt = 0;
        if (tucker_block(a, i, &dt, &rt)) {
            double* e0v = (double*)calloc(D, sizeof(double));
            e0v[0] = 1.0;
            const double* src[8];
            for (int e = e0; e < e1; ++e) {
                const int j = edge_src(a, e);
                src[e - e0] = j < 0 ? e0v : hs + (size_t)j * D;
            }
            tensor_term(a, i, s, src, h);
            free(e0v);
        }
        double p = 0.0;
        for (int r = 0; r < D; ++r) p += a->rnn_eta[(size_t)i * D + r] * h[r] * h[r];
        P[s] = p;
    }
}

/* log|Phi(n)| of the normalised readout; the chosen cells go to hs [K][D],
 * the conditionals P~_i(s) to probs [K][4] (may be NULL). */
static double rnn_log_phi(const or_ansatz* a, const int* sigma, double* hs, int* sign, double* probs)
{
    const int K = a->K, D = a->D;
    double* cand = (double*)malloc(sizeof(double) * 4 * D);
    double lp = 0.0;
    int sg = 1, na_done = 0, nb_done = 0;
    for (int i = 0; i < K; ++i) {
        double P[4], Z = 0.0;
        rnn_candidates(a, i, hs, cand, P);
        for (int s = 0; s < 4; ++s)
            if (state_allowed(a, i, na_done, nb_done, s)) Z += P[s];
        if (probs)
            for (int s = 0; s < 4; ++s)
                probs[i * 4 + s] = state_allowed(a, i, na_done, nb_done, s) && Z > 0.0 ? P[s] / Z : 0.0;
        const int s = sigma[i];
        if (!state_allowed(a, i, na_done, nb_done, s) || P[s] == 0.0 || Z == 0.0) { sg = 0; lp = -INFINITY; }
        if (sg != 0) {
            lp += 0.5 * (log(P[s]) - log(Z));
            double ph = a->rnn_c[i];
            for (int r = 0; r < D; ++r) ph += a->rnn_w[(size_t)i * D + r] * cand[(size_t)s * D + r];
            if (ph < 0.0) sg = -sg;
        }
        for (int r = 0; r < D; ++r) hs[(size_t)i * D + r] = cand[(size_t)s * D + r];
        na_done += s & 1;
        nb_done += s >> 1;
    }
    free(cand);
    *sign = sg;
    return lp;
}

void or_rnn_conditionals(const or_ansatz* a, const uint64_t* det, double* probs)
{
    int sigma[64], sg;
    sigma_of(a->K, det, sigma);
    double* hs = (double*)malloc(sizeof(double) * (size_t)a->K * a->D);
    rnn_log_phi(a, sigma, hs, &sg, probs);
    free(hs);
}

void or_log_psi(const or_ansatz* a, const uint64_t* det, double* log_abs, int* sign,
                double* log_f)
{
    const int K = a->K, D = a->D;
    int sigma[64];
    sigma_of(K, det, sigma);
    double* hs = (double*)malloc(sizeof(double) * (size_t)K * D);
    double la_tn;
    int sg_tn;
    if (a->readout == 1) {
        la_tn = rnn_log_phi(a, sigma, hs, &sg_tn, NULL);
    } else {
        int* ex = (int*)malloc(sizeof(int) * K);
        forward_states(a, sigma, hs, ex);
        const double mant = hs[(size_t)(K - 1) * D + 0];
        sg_tn = mant == 0.0 ? 0 : (mant < 0 ? -1 : 1);
        la_tn = mant == 0.0 ? -INFINITY : log(fabs(mant)) + (double)ex[K - 1] * M_LN2;
        free(ex);
    }
    free(hs);
    int sg_f;
    double lf = rbm_log_f(a, det, &sg_f);
    if (log_f) *log_f = lf;
    if (sg_tn == 0 || sg_f == 0) { *sign = 0; *log_abs = -INFINITY; return; }
    *sign = sg_tn * sg_f;
    *log_abs = la_tn + lf;
}

int64_t or_sample(const or_ansatz* a, int64_t n_samples, uint64_t seed, uint64_t* dets,
                  double* counts, int64_t capacity)
{
    const int K = a->K, D = a->D;
    if (n_samples <= 0) return 0;
    /* nodes of the current level: prefix words, offset, count, cells [K][D] */
    int64_t n = 1, cap = 1;
    uint64_t* pa = (uint64_t*)calloc(cap, 8);
    uint64_t* pb = (uint64_t*)calloc(cap, 8);
    int64_t* off = (int64_t*)calloc(cap, 8);
    int64_t* cnt = (int64_t*)calloc(cap, 8);
    double* cells = (double*)calloc((size_t)cap * K * D, 8);
    cnt[0] = n_samples;
    double* cand = (double*)malloc(sizeof(double) * 4 * D);
    for (int i = 0; i < K; ++i) {
        const int64_t ncap = n * 4;
        uint64_t* qa = (uint64_t*)calloc(ncap, 8);
        uint64_t* qb = (uint64_t*)calloc(ncap, 8);
        int64_t* qo = (int64_t*)calloc(ncap, 8);
        int64_t* qc = (int64_t*)calloc(ncap, 8);
        double* qcells = (double*)calloc((size_t)ncap * K * D, 8);
        int64_t m = 0;
        for (int64_t q = 0; q < n; ++q) {
            double* hs = cells + (size_t)q * K * D;
            double P[4];
            rnn_candidates(a, i, hs, cand, P);
            const int na_done = __builtin_popcountll(pa[q]), nb_done = __builtin_popcountll(pb[q]);
            int ok[4], last = -1;
            double Z = 0.0;
            for (int s = 0; s < 4; ++s) {
                ok[s] = state_allowed(a, i, na_done, nb_done, s);
                if (ok[s]) { Z += P[s]; last = s; }
            }
            int64_t hist[4] = {0, 0, 0, 0};
            for (int64_t j = off[q]; j < off[q] + cnt[q]; ++j) {
                const uint64_t ctr[4] = {(uint64_t)j, (uint64_t)i, 1, 0}, key[2] = {seed, 0};
                uint64_t x[4];
                or_philox4x64_10(ctr, key, x);
                const double u = (double)(x[0] >> 11) * 0x1.0p-53;
                const double t = u * Z;
                double cum = 0.0;
                int pick = last;
                for (int s = 0; s < 4; ++s) {
                    if (!ok[s]) continue;
                    cum += P[s];
                    if (t < cum) { pick = s; break; }
                }
                if (pick >= 0) hist[pick] += 1;
            }
            int64_t o = off[q];
            for (int s = 0; s < 4; ++s) {
                if (hist[s] == 0) continue;
                qa[m] = pa[q] | ((uint64_t)(s & 1) << i);
                qb[m] = pb[q] | ((uint64_t)(s >> 1) << i);
                qo[m] = o;
                qc[m] = hist[s];
                double* dst = qcells + (size_t)m * K * D;
                memcpy(dst, hs, sizeof(double) * (size_t)K * D);
                memcpy(dst + (size_t)i * D, cand + (size_t)s * D, sizeof(double) * D);
                o += hist[s];
                ++m;
            }
        }
        free(pa); free(pb); free(off); free(cnt); free(cells);
        pa = qa; pb = qb; off = qo; cnt = qc; cells = qcells;
        n = m;
    }
    for (int64_t q = 0; q < n && q < capacity; ++q) {
        dets[2 * q] = pa[q];
        dets[2 * q + 1] = pb[q];
        counts[q] = (double)cnt[q];
    }
    free(pa); free(pb); free(off); free(cnt); free(cells); free(cand);
    return n;
}

/* S 2^Se += v 2^e, keeping the larger exponent */
static void add_scaled(double* S, int* Se, double v, int e)
{
    if (v == 0.0) return;
    if (*S == 0.0) { *S = v; *Se = e; }
    else if (e > *Se) { *S = ldexp(*S, *Se - e) + v; *Se = e; }
    else *S += ldexp(v, e - *Se);
    int k;
    *S = frexp(*S, &k);
    *Se += k;
}

double or_log_psi_p1(const or_ansatz* a, const uint64_t* det)
{
    const int K = a->K, D = a->D;
    int sigma[64];
    sigma_of(K, det, sigma);
    double* hs = (double*)malloc(sizeof(double) * (size_t)K * D);
    int* ex = (int*)malloc(sizeof(int) * K);
    if (a->tucker_rank) {
        /* with the (multilinear) tensor term: the whole contraction evaluated with
         * absolute values of every parameter -- a sum of products whose rounding
         * error is at most ~(depth) u times this value (Higham, Ch. 3) */
        forward_states_x(a, sigma, hs, ex, 1);
        const double v = hs[(size_t)(K - 1) * D];
        const int e = ex[K - 1];
        free(hs);
        free(ex);
        return v > 0.0 ? log(v) + (double)e * M_LN2 : -INFINITY;
    }
    forward_states(a, sigma, hs, ex);
    /* adjoints g_i = d psi_TN / d h_i, scaled with exponents gx */
    double* gs = (double*)calloc((size_t)K * D, sizeof(double));
    int* gx = (int*)calloc(K, sizeof(int));
    int* gset = (int*)calloc(K, sizeof(int));
    double* tmp = (double*)malloc(sizeof(double) * D);
    gs[(size_t)(K - 1) * D + 0] = 1.0;
    gset[K - 1] = 1;
    double S = 0.0;
    int Se = 0;
    for (int i = K - 1; i >= 0; --i) {        /* every successor of i is done */
        if (!gset[i]) continue;               /* i does not reach the readout */
        const double* g = gs + (size_t)i * D;
        int e0, e1;
        edges_of(a, i, &e0, &e1);
        for (int e = e0; e < e1; ++e) {
            const int j = edge_src(a, e);
            const double* M = tensor(a, e, sigma[i]);
            /* |g_i|^T |M_e| |h_j| (h_{-1} = e_0) */
            double t = 0.0;
            for (int r = 0; r < D; ++r) {
                double s = 0.0;
                for (int q = 0; q < D; ++q) {
                    double hj = (j < 0) ? (q == 0 ? 1.0 : 0.0) : hs[(size_t)j * D + q];
                    s += fabs(M[r * D + q]) * fabs(hj);
                }
                t += fabs(g[r]) * s;
            }
            add_scaled(&S, &Se, t, gx[i] + (j < 0 ? 0 : ex[j]));
            if (j < 0) continue;
            /* g_j += M_e^T g_i */
            for (int q = 0; q < D; ++q) {
                double s = 0.0;
                for (int r = 0; r < D; ++r) s += M[r * D + q] * g[r];
                tmp[q] = s;
            }
            double* gj = gs + (size_t)j * D;
            if (!gset[j]) {
                for (int q = 0; q < D; ++q) gj[q] = tmp[q];
                gx[j] = gx[i];
                gset[j] = 1;
            } else {
                const int em = gx[j] > gx[i] ? gx[j] : gx[i];
                for (int q = 0; q < D; ++q) gj[q] = ldexp(gj[q], gx[j] - em) + ldexp(tmp[q], gx[i] - em);
                gx[j] = em;
            }
            gx[j] += renorm(gj, D);
        }
    }
    free(hs); free(ex); free(gs); free(gx); free(gset); free(tmp);
    return S > 0.0 ? log(S) + (double)Se * M_LN2 : -INFINITY;
}

/* ------------------------------------------------------------------------ */
/* Semistochastic local energy (Sec. 2.4)                                    */
/* ------------------------------------------------------------------------ */

static int bit_length(uint64_t x)
{
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

/* Remainder weights w = ceil(|H| 2^s) (P_n(m) proportional to |H_nm|, Sec.
 * 2.4, as exact integers) with s = 62 - e - bitlen(n_conn), eps = f 2^e,
 * f in [0.5, 1): every remainder |H| < eps, so sum w < 2^62. */
static int weight_shift(double eps, int64_t nconn)
{
    int e = 0;
    if (eps > 0.0) frexp(eps, &e);
    return 62 - e - bit_length((uint64_t)nconn);
}

static uint64_t weight_of(double H, int shift)
{
    return (uint64_t)ceil(ldexp(fabs(H), shift));
}

/* t = floor(x * W / 2^64): the uniform target in [0, W). */
static uint64_t draw_target(uint64_t x, uint64_t W)
{
    return (uint64_t)(((unsigned __int128)x * W) >> 64);
}

typedef struct {
    int64_t nc, nrem;
    double* H;
    uint64_t* dets;
    int64_t* rem_rank;   /* canonical ranks of the remainder */
    uint64_t* prefix;    /* inclusive prefix sums of remainder weights */
    uint64_t W;
    int shift;
} split_t;

static void split_build(const or_ham* h, const uint64_t* n, double eps, split_t* sp)
{
    int64_t nc = or_n_conn(h->K, h->n_alpha, h->n_beta);
    sp->nc = nc;
    sp->H = (double*)malloc(sizeof(double) * (size_t)(nc + 1));
    sp->dets = (uint64_t*)malloc(sizeof(uint64_t) * 2 * (size_t)(nc + 1));
    or_connected(h, n, sp->dets, sp->H, NULL);
    int64_t nrem = 0;
    for (int64_t r = 0; r < nc; ++r)
        if (!(fabs(sp->H[r]) >= eps)) ++nrem;
    sp->nrem = nrem;
    sp->rem_rank = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nrem + 1));
    sp->prefix = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nrem + 1));
    sp->W = 0;
    sp->shift = 0;
    if (nrem == 0) return;
    sp->shift = weight_shift(eps, nc);
    uint64_t run = 0;
    int64_t c = 0;
    for (int64_t r = 0; r < nc; ++r)
        if (!(fabs(sp->H[r]) >= eps)) {
            run += weight_of(sp->H[r], sp->shift);
            sp->rem_rank[c] = r;
            sp->prefix[c] = run;
            ++c;
        }
    sp->W = run;
}

static void split_free(split_t* sp)
{
    free(sp->H); free(sp->dets); free(sp->rem_rank); free(sp->prefix);
}

/* Draw d of sample `si`: the first remainder element whose inclusive prefix
 * weight exceeds the target t (inverse CDF of P_n(m) = w_m / W). */
static int64_t draw_one(const split_t* sp, int64_t si, int d, uint64_t seed)
{
    uint64_t ctr[4] = {(uint64_t)d, (uint64_t)si, 0, 0}, key[2] = {seed, 0}, out[4];
    or_philox4x64_10(ctr, key, out);
    uint64_t t = draw_target(out[0], sp->W);
    int64_t lo = 0, hi = sp->nrem - 1;     /* smallest c with prefix[c] > t */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (sp->prefix[mid] > t) hi = mid; else lo = mid + 1;
    }
    return lo;
}

int or_draws(const or_ham* h, const uint64_t* n, int64_t si, double eps, int n_draws,
             uint64_t seed, int64_t* ranks, uint64_t* w_total, int* shift)
{
    split_t sp;
    split_build(h, n, eps, &sp);
    if (w_total) *w_total = sp.W;
    if (shift) *shift = sp.shift;
    for (int d = 0; d < n_draws; ++d)
        ranks[d] = sp.W ? sp.rem_rank[draw_one(&sp, si, d, seed)] : -1;
    split_free(&sp);
    return 0;
}

/* |a| (P1(m) f(m) + kappa_n |psi(m)|) / |psi(n)| for one term (see e_cond) */
static double cond_term(const or_ansatz* a, const uint64_t* m, double coef, double la_m,
                        double lf_m, double la_n, double kappa_n)
{
    const double lp = or_log_psi_p1(a, m);
    return fabs(coef) * (exp(lp + lf_m - la_n) + kappa_n * exp(la_m - la_n));
}

static void one_sample(const or_ham* h, const or_ansatz* a, const uint64_t* n, int64_t si,
                       double eps, int n_draws, uint64_t seed, or_sample_out* o, int with_cond)
{
    memset(o, 0, sizeof(*o));
    /* the first-order bound P1 describes the linear readout's contraction */
    if (a->readout != 0) with_cond = 0;
    double la_n, lf_n;
    int sg_n;
    or_log_psi(a, n, &la_n, &sg_n, &lf_n);
    o->log_abs_psi = la_n;
    o->sign_psi = sg_n;
    o->log_f = lf_n;
    o->h_diag = or_diag(h, n);
    if (sg_n == 0) { o->e_loc = NAN; return; }
    /* kappa_n = P1(n) / |psi_TN(n)| */
    const double kappa_n = with_cond ? exp(or_log_psi_p1(a, n) - (la_n - lf_n)) : 0.0;
    double econd = 0.0;

    split_t sp;
    split_build(h, n, eps, &sp);
    o->n_rem = sp.nrem;
    o->w_total = sp.W;
    o->w_shift = sp.shift;

    /* deterministic part: sum over |H_nm| >= eps in canonical order */
    double ed = 0.0, eabs = fabs(o->h_diag);
    int64_t ndet = 0;
    for (int64_t r = 0; r < sp.nc; ++r) {
        if (!(fabs(sp.H[r]) >= eps)) continue;
        ++ndet;
        double la_m, lf_m;
        int sg_m;
        or_log_psi(a, &sp.dets[2 * r], &la_m, &sg_m, &lf_m);
        double ratio = (double)(sg_m * sg_n) * exp(la_m - la_n);
        ed += sp.H[r] * ratio;
        eabs += fabs(sp.H[r] * ratio);
        if (with_cond) econd += cond_term(a, &sp.dets[2 * r], sp.H[r], la_m, lf_m, la_n, kappa_n);
    }
    o->n_det = ndet;
    o->e_det = ed;

    /* stochastic part: N_eps draws m' ~ w/W, estimator H/P * psi(m')/psi(n) */
    double es = 0.0;
    if (n_draws > 0 && sp.W > 0) {
        for (int d = 0; d < n_draws; ++d) {
            int64_t c = draw_one(&sp, si, d, seed);
            int64_t r = sp.rem_rank[c];
            uint64_t w = c == 0 ? sp.prefix[0] : sp.prefix[c] - sp.prefix[c - 1];
            double la_m, lf_m;
            int sg_m;
            or_log_psi(a, &sp.dets[2 * r], &la_m, &sg_m, &lf_m);
            double ratio = (double)(sg_m * sg_n) * exp(la_m - la_n);
            es += sp.H[r] * ((double)sp.W / (double)w) * ratio;
            eabs += fabs(sp.H[r] * ((double)sp.W / (double)w) * ratio) / (double)n_draws;
            if (with_cond)
                econd += cond_term(a, &sp.dets[2 * r], sp.H[r] * ((double)sp.W / (double)w) / (double)n_draws,
                                   la_m, lf_m, la_n, kappa_n);
        }
        es /= (double)n_draws;
    }
    o->e_stoch = es;
    o->e_abs = eabs;
    o->e_cond = with_cond ? econd : 0.0;
    o->e_loc = o->h_diag + ed + es;
    split_free(&sp);
}

int or_local_energy(const or_ham* h, const or_ansatz* a, const uint64_t* samples, int64_t Ns,
                    double eps, int n_draws, uint64_t seed, or_sample_out* out, int n_threads,
                    const int64_t* index, int with_cond)
{
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t s = 0; s < Ns; ++s)
        one_sample(h, a, &samples[2 * s], index ? index[s] : s, eps, n_draws, seed, &out[s], with_cond);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Gradient of log|psi| (Eq. egrad needs d ln Psi / d theta)                */
/* ------------------------------------------------------------------------ */

void or_grad_log_psi(const or_ansatz* a, const uint64_t* det, double* grad_t, double* grad_W,
                     double* grad_b)
{
    const int K = a->K, D = a->D;
    int sigma[64];
    sigma_of(K, det, sigma);
    double* hs = (double*)malloc(sizeof(double) * (size_t)K * D);
    int* ex = (int*)malloc(sizeof(int) * K);
    forward_states(a, sigma, hs, ex);
    double mant = hs[(size_t)(K - 1) * D];
    int emant = ex[K - 1];

    if (grad_t) {
        memset(grad_t, 0, sizeof(double) * (size_t)a->n_edges * 4 * D * D);
        /* adjoints g_i = d psi_TN / d h_i, scaled like the states */
        double* gs = (double*)calloc((size_t)K * D, sizeof(double));
        int* gx = (int*)malloc(sizeof(int) * K);
        int* gset = (int*)calloc(K, sizeof(int));
        gs[(size_t)(K - 1) * D] = 1.0;       /* r = e_0 */
        gx[K - 1] = 0;
        gset[K - 1] = 1;
        double* tmp = (double*)malloc(sizeof(double) * D);
        for (int i = K - 1; i >= 0; --i) {
            if (!gset[i]) continue;
            int ge = renorm(gs + (size_t)i * D, D);
            gx[i] += ge;
            const double* g = gs + (size_t)i * D;
            int e0, e1;
            edges_of(a, i, &e0, &e1);
            for (int e = e0; e < e1; ++e) {
                int j = edge_src(a, e);
                const double* M = tensor(a, e, sigma[i]);
                /* d log|psi| / d M[r][c] = g[r] h_j[c] / psi_TN */
                double* G = grad_t + ((size_t)e * 4 + sigma[i]) * D * D;
                int ej = j < 0 ? 0 : ex[j];
                for (int r = 0; r < D; ++r)
                    for (int c = 0; c < D; ++c) {
                        double hj = (j < 0) ? (c == 0 ? 1.0 : 0.0) : hs[(size_t)j * D + c];
                        G[r * D + c] += ldexp(g[r] * hj / mant, gx[i] + ej - emant);
                    }
                if (j < 0) continue;
                /* g_j += g_i M (row vector times matrix) */
                for (int c = 0; c < D; ++c) {
                    double s = 0.0;
                    for (int r = 0; r < D; ++r) s += g[r] * M[r * D + c];
                    tmp[c] = s;
                }
                double* gj = gs + (size_t)j * D;
                if (!gset[j]) {
                    for (int c = 0; c < D; ++c) gj[c] = tmp[c];
                    gx[j] = gx[i];
                    gset[j] = 1;
                } else {
                    int eref = gx[j] > gx[i] ? gx[j] : gx[i];
                    for (int c = 0; c < D; ++c)
                        gj[c] = ldexp(gj[c], gx[j] - eref) + ldexp(tmp[c], gx[i] - eref);
                    gx[j] = eref;
                }
            }
        }
        free(tmp); free(gs); free(gx); free(gset);
    }
    if (a->n_hidden > 0 && (grad_W || grad_b)) {
        int occ[128];
        unpack(K, det, occ);
        for (int k = 0; k < a->n_hidden; ++k) {
            /* d log|f| / d theta_k: tanh (2 cosh), -tan (cos, Ising) */
            const double th = corr_theta(a, occ, k);
            const double t = a->corr == 0 ? tanh(th) : -tan(th);
            if (grad_b) grad_b[k] = t;
            if (grad_W)
                for (int s = 0; s < 2 * K; ++s) grad_W[(size_t)k * 2 * K + s] = occ[s] ? t : 0.0;
        }
    }
    free(hs);
    free(ex);
}

void or_grad_corr_W2(const or_ansatz* a, const uint64_t* det, double* grad_W2)
{
    const int K = a->K, N = 2 * K;
    int occ[128];
    unpack(K, det, occ);
    for (int k = 0; k < a->n_hidden; ++k) {
        const double t = a->corr == 0 ? tanh(corr_theta(a, occ, k)) : -tan(corr_theta(a, occ, k));
        for (int s = 0; s < N; ++s)
            for (int u = 0; u < N; ++u)
                grad_W2[((size_t)k * N + s) * N + u] = (a->corr == 2 && occ[s] && occ[u]) ? 0.5 * t : 0.0;
    }
}
