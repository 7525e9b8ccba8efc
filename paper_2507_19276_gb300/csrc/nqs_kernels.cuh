// nqs_kernels.cuh -- argument blocks and launchers of every kernel of the
// local-energy path (host orchestration lives in nqs_api.cu).
#pragma once

#include <vector>

#include "nqs_internal.cuh"

namespace nqs {

// Allow a kernel the largest dynamic shared memory the device permits next
// to its static shared memory. The attribute is process-wide per function, so
// setting each launch's exact size would race between host threads launching
// with different sizes; this value is the same for every caller, and occupancy
// still follows the size each launch requests.
template <typename F>
inline void allow_max_smem(F* kernel)
{
    int dev = 0, mx = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, kernel);
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx - (int)fa.sharedSizeBytes);
}


// ---- enumeration (nqs_enum.cu) ---------------------------------------------

struct EnumArgs {
    HamView h;
    const uint64_t* samples;
    int s0;                              // first sample of this launch (set by the launcher)
    uint64_t eps_bits;                   // bits of |eps|
    uint32_t n_chunks;                   // ceil(n_conn / 32)
    uint32_t* chunk_cnt;                 // [Ns][n_chunks] entries with |H| >= eps (count pass
                                         // writes; the write pass skips chunks without any)
    uint32_t* chunk_mask;                // [Ns][n_chunks] ballot of |H| >= eps (count pass writes
                                         // if non-NULL; the write pass needs it)
    int shift;                           // remainder weights w = ceil(|H| 2^shift)
    const uint32_t* chunk_off;           // write pass: exclusive prefix of chunk_cnt per sample
    const int64_t* det_off;              // [Ns+1] start of each sample's list (NULL: no list)
    uint32_t* out_rank;
    double* out_H;
    uint64_t* out_det;
    int8_t* out_sign;
    uint64_t* chunk_w;                   // count pass: [Ns][n_chunks] remainder weight sums
                                         // (NULL: skip)
};
int launch_enum(const EnumArgs& a, int64_t Ns, bool write, cudaStream_t st);

struct DrawArgs {
    HamView h;
    const uint64_t* samples;
    int64_t Ns;
    uint64_t eps_bits;
    uint32_t n_chunks;
    const uint64_t* chunk_pre;           // [Ns][n_chunks] inclusive prefix of weights
    int shift;                           // remainder weight shift
    int n_draws;
    uint64_t seed;
    int64_t index_base;                  // Philox sample counter of samples[0]
    const int64_t* index;                // per-sample Philox counters (NULL: index_base + s)
    int64_t* out_rank;                   // [Ns][n_draws]
};
int launch_draws(const DrawArgs& a, cudaStream_t st);

struct DedupArgs {
    HamView h;
    const uint64_t* samples;
    const int64_t* ranks;                // [Ns][n_draws]
    int n_draws;
    int pow2;                            // next power of two >= n_draws
    int shift;                           // remainder weight shift
    const uint64_t* W;                   // [Ns] total remainder weight
    uint32_t* out_rank;                  // [Ns][n_draws] unique ranks (first n_unique)
    double* out_coef;                    // [Ns][n_draws]
    int64_t* n_unique;                   // [Ns]
};
int launch_dedup(const DedupArgs& a, int64_t Ns, cudaStream_t st);

int launch_validate(const uint64_t* samples, int64_t Ns, int K, int na, int nb, DevError* err,
                     cudaStream_t st);

// ---- utilities (nqs_util.cu) -----------------------------------------------

int launch_build_eri(const double* L, int n_chol, int K, double* eri, cudaStream_t st);
int launch_swap_eri(const double* in, int K, double* eri, cudaStream_t st);
// per sample: exclusive scan of u32 chunk counts -> chunk_off, totals -> n_det
int launch_scan_chunks_u32(const uint32_t* cnt, uint32_t* off, int64_t* total, int64_t Ns,
                            uint32_t n_chunks, cudaStream_t st);
// per sample: inclusive scan of u64 chunk weights (in place), totals -> W
int launch_scan_chunks_u64(uint64_t* w, uint64_t* total, int64_t Ns, uint32_t n_chunks,
                            cudaStream_t st);
// exclusive scan of n values -> out[0..n] (out[n] = total); single block
int launch_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st);
// the same over many blocks for large n; tmp holds scan_i64_tmp_elems(n) values
inline int64_t scan_i64_tmp_elems(int64_t n) { return 2 * (n / 4096 + 2); }
int launch_scan_i64_wide(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t st);
// chunk bases for row sets: out[s] = sum_{s'<s} ceil(cnt[s'] / rows), out[Ns] total
int launch_chunk_base(const int64_t* cnt, int rows, int64_t* out, int64_t Ns, cudaStream_t st);

struct FinalArgs {
    int64_t Ns;
    const double* h_diag;                // [Ns]
    const double* part_det;              // partial sums of det rows
    const int64_t* base_det;             // [Ns+1] chunk bases of det rows
    const double* part_draw;
    const int64_t* base_draw;            // NULL when there are no draws
    const double* counts;                // [Ns] or NULL
    const double* log_f;                 // [Ns]
    const int64_t* det_off;              // [Ns+1] (NULL: the summary skips the work counts)
    const int64_t* n_unique;             // [Ns] or NULL
    double* e_loc;                       // [Ns]
    double* e_det;                       // [Ns] (optional)
    double* e_stoch;                     // [Ns] (optional)
    const int64_t* span_det;             // [chunks] from the amplitude kernels
    const int64_t* span_draw;
    double* summary;                     // [8] e_mean, sum_c, log_B, e_tilde_mean, n_det, n_uniq, span
    const double* part_det_abs;          // chunk sums of |term| (NULL: no e_abs)
    const double* part_draw_abs;
    double* e_abs;                       // [Ns] |H_nn| + sum |terms| (optional)
    const int64_t* mv_det;               // [chunks] in-edge products of the rows (graph
    const int64_t* mv_draw;              // ansatz; NULL: summary[7] = 0)
};
int launch_finalize(const FinalArgs& a, cudaStream_t st);
int launch_summary(const FinalArgs& a, cudaStream_t st);     // the summary alone
// re-evaluation of picked samples: gather (words, counts, base + position), scatter
int launch_gather_picked(const int64_t* idx, int64_t n, const uint64_t* samples, const double* counts,
                         int64_t base, uint64_t* out_s, double* out_c, int64_t* out_pos, cudaStream_t st);
int launch_scatter_picked(const int64_t* idx, int64_t n, const double* v, double* out, cudaStream_t st);

// ---- FP64 ansatz (nqs_fp64.cu) ---------------------------------------------

struct AnsatzView {
    int K, D, n_edges;
    int chain;                           // 1: pred(i) = {i-1}
    const int* pred_ptr;                 // [K+1] (graph)
    const int* pred_idx;                 // [E]
    const double* A;                     // [E][4][D][D]  A[e][s][a][b]
    const double* AT;                    // [E][4][D][D]  AT[e][s][b][a]
    int n_hidden;
    const double* W;                     // [n_hidden][2K]
    const double* b;                     // [n_hidden]
    // readout (Sec. 2.2): 0 linear psi_TN = (h_{K-1})_0; 1 the normalised
    // MPS-RNN / BDG-RNN: candidate cells h_i^s = sum_e M_e^s h_j + v_i^s,
    // P_i(s) = sum_a eta_i[a] (h_i^s[a])^2 normalised over the local states
    // the N_alpha / N_beta constraint allows, sign of w_i . h_i^{s_i} + c_i
    int readout;
    int mask_na, mask_nb;                // the constraint's electron counts (mask_na < 0: none)
    const double* rv;                    // [K][4][D]
    const double* reta;                  // [K][D]
    const double* rw;                    // [K][D]
    const double* rc;                    // [K]
    // correlator (Sec. 2.3): 0 prod 2cosh(theta_k); 1 cos-RBM prod cos(theta_k);
    // 2 Ising-RBM, theta_k + 1/2 sum_{s,t} W2[k][s][t] n_s n_t inside the cos
    int corr;
    const double* W2;                    // [n_hidden][2K][2K] (corr 2)
    // tensor term of Eq. (bdg-rnn-update) with Tucker factors (graph ansatz):
    // vertex i with d >= 2 in-edges and rank r = tk_rank[i] > 0 owns, at
    // tk[tk_off[i]], U [4][r^(d+1)] then Kout [D][r] then K_k [D][r] per in-edge
    const int* tk_rank;                  // [K] (NULL: no tensor term)
    const long long* tk_off;             // [K] (-1: none)
    const double* tk;
    int tk_zy;                           // scratch doubles per evaluation: max (d + 4) r
};

// D x D products a graph amplitude that first changes at vertex p performs:
// the in-edges with a vertex source of the vertices p..K-1
__device__ __forceinline__ int graph_matvecs(const AnsatzView& an, int p)
{
    int n = 0;
    for (int e = an.pred_ptr[p]; e < an.pred_ptr[an.K]; ++e) n += an.pred_idx[e] >= 0;
    return n;
}

// sum_k AT[k][c] x[k] (AT row-major D x D) with four interleaved partial sums:
// independent FMA chains that hide the FP64 pipe's latency, combined as
// (s0 + s1) + (s2 + s3)
__device__ __forceinline__ double dot_col4(const double* AT, const double* x, int D, int c)
{
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int k = 0;
    for (; k + 3 < D; k += 4) {
        s0 = fma(__ldg(AT + (size_t)k * D + c), x[k], s0);
        s1 = fma(__ldg(AT + (size_t)(k + 1) * D + c), x[k + 1], s1);
        s2 = fma(__ldg(AT + (size_t)(k + 2) * D + c), x[k + 2], s2);
        s3 = fma(__ldg(AT + (size_t)(k + 3) * D + c), x[k + 3], s3);
    }
    for (; k < D; ++k) s0 = fma(__ldg(AT + (size_t)k * D + c), x[k], s0);
    return (s0 + s1) + (s2 + s3);
}

// ---- tensor term (Tucker form), shared by the FP64 kernels ------------------
// t_i^s[a] = sum_o Kout[a][o] y[o],  y[o] = sum_{a_1'..a_d'} U^s[o][a_1']..[a_d']
// prod_k z_k[a_k'],  z_k[q] = sum_b K_k[b][q] h_{j_k}[b] (h_{-1} = e_0).

__device__ __forceinline__ int tk_degree(const AnsatzView& an, int i)
{
    return an.chain ? 1 : an.pred_ptr[i + 1] - an.pred_ptr[i];
}

__device__ __forceinline__ bool tk_has(const AnsatzView& an, int i)
{
    return an.tk_rank && an.tk_off[i] >= 0;
}

// z [d][r] for the in-edge sources of vertex i; threads tid, tid + nt, ...
template <class Src>
__device__ __forceinline__ void tk_project(const AnsatzView& an, int i, const Src& src, double* z, int tid, int nt)
{
    const int d = tk_degree(an, i), r = an.tk_rank[i], D = an.D;
    size_t core = 1;
    for (int k = 0; k <= d; ++k) core *= (size_t)r;
    const double* K1 = an.tk + an.tk_off[i] + 4 * core + (size_t)D * r;   // K_1, then K_2, ...
    for (int q = tid; q < d * r; q += nt) {
        const int k = q / r, c = q - k * r;
        const int j = an.pred_idx[an.pred_ptr[i] + k];
        const double* Kk = K1 + (size_t)k * D * r;
        double acc;
        if (j < 0) acc = __ldg(Kk + c);                        // K_k^T e_0 = row 0 of K_k
        else {
            const double* h = src(j);
            acc = 0.0;
            for (int b = 0; b < D; ++b) acc = fma(__ldg(Kk + (size_t)b * r + c), h[b], acc);
        }
        z[q] = acc;
    }
}

// y [r] for local state s from z
__device__ __forceinline__ void tk_core(const AnsatzView& an, int i, int s, const double* z, double* y, int tid, int nt)
{
    const int d = tk_degree(an, i), r = an.tk_rank[i];
    size_t cd = 1;
    for (int k = 0; k < d; ++k) cd *= (size_t)r;
    const double* U = an.tk + an.tk_off[i] + (size_t)s * cd * r;
    for (int o = tid; o < r; o += nt) {
        double acc = 0.0;
        for (size_t m = 0; m < cd; ++m) {
            double prod = __ldg(U + (size_t)o * cd + m);
            size_t rem = m;
            for (int k = d - 1; k >= 0; --k) {
                prod *= z[k * r + (int)(rem % (size_t)r)];
                rem /= (size_t)r;
            }
            acc += prod;
        }
        y[o] = acc;
    }
}

// component a of the tensor term from y
__device__ __forceinline__ double tk_out(const AnsatzView& an, int i, int a, const double* y)
{
    const int d = tk_degree(an, i), r = an.tk_rank[i];
    size_t core = 1;
    for (int k = 0; k <= d; ++k) core *= (size_t)r;
    const double* Kout = an.tk + an.tk_off[i] + 4 * core;
    double acc = 0.0;
    for (int o = 0; o < r; ++o) acc = fma(__ldg(Kout + (size_t)a * r + o), y[o], acc);
    return acc;
}

struct EnvArgs {
    AnsatzView an;
    HamView h;
    const uint64_t* samples;
    int64_t Ns;
    double* Lenv; int* Lexp;             // chain: [Ns][K+1][D] (index t+1 = after site t)
    double* Renv; int* Rexp;             // chain: [Ns][K+1][D] (index t = sites t..K-1)
    double* Hst; int* Hexp;              // graph: forward states [Ns][K][D]
    double* Gst; int* Gexp;              // adjoints [Ns][K][D] (graph; NULL to skip)
    double* theta;                       // [Ns][n_hidden] b + W n
    double* lc;                          // [Ns][n_hidden] log 2cosh(theta)
    double* log_f;                       // [Ns]
    double* psi_mant; int* psi_exp;      // [Ns] psi_TN = mant 2^exp
    double* h_diag;                      // [Ns]
    int tn;                              // 0: skip the tensor-network part; 1: psi(n) and the
                                         // environments; 2 (chain): psi(n) only; 3 (chain):
                                         // psi(n) only, in double-FP32 arithmetic (ATdf)
    const float2* ATdf;                  // tn == 3: AT as FP32 (hi, lo) pairs, hi + lo = AT
};
int launch_env_fp64(const EnvArgs& a, cudaStream_t st);

struct RowSet {
    const uint32_t* rank;                // canonical ranks, or site words (see nqs_family.cu)
    int sites;                           // when set
    const double* coef;
    const int64_t* begin;                // [Ns] first row of each sample (NULL: s * stride)
    int64_t stride;
    const int64_t* count;                // [Ns] rows of each sample (NULL: from begin diff)
    const int64_t* chunk_base;           // [Ns+1] from launch_chunk_base
    int64_t max_chunks;                  // grid upper bound
};

struct AmpArgs {
    AnsatzView an;
    HamView h;
    const uint64_t* samples;
    int64_t Ns;
    RowSet rows;
    int rows_per_block;
    const double* Lenv; const int* Lexp;
    const double* Renv; const int* Rexp;
    const double* Hst; const int* Hexp;
    const double* theta; const double* lc;
    const double* psi_mant; const int* psi_exp;
    double* partial;                     // [chunks]
    int64_t* span;                       // [chunks] sites recomputed per chunk
    int64_t* mv;                         // [chunks] in-edge products (graph; optional)
};
int amp_fp64_rows_per_block(const AnsatzView& an);
size_t amp_fp64_smem(const AnsatzView& an, int rows);
int launch_amp_fp64(const AmpArgs& a, cudaStream_t st);

// ---- mixed form of the graph ansatz on the tensor cores (nqs_graph.cu) ------

constexpr int kGtMaxSlots = 16;          // vertex states a tile keeps at once
constexpr int kGtMaxDeg = 8;             // in-degree bound of the graph ansatz

struct GraphTcPlan {
    std::vector<unsigned char> img;      // [E][4] split images of M_e^sigma (hi, lo)
    std::vector<int> bexp;               // [E][4] power of two taken out of each image
    std::vector<float> col0;             // [E][4][D] column 0 of each matrix (e_0 sources)
    std::vector<int> slot;               // [K] state slot of each vertex (-1: never read)
    std::vector<int> last_use;           // [K] last vertex reading each state (-1: none)
    int n_slots = 0, max_deg = 0;
    int nbuf = 1;                        // matrix-image buffers that fit next to the slots
};
// false (with the reason) when the graph does not fit the tile kernel
bool graph_tc_plan(const double* A, const int* ptr, const int* idx, int K, int D, int n_hidden,
                   GraphTcPlan& p, const char** why);
size_t graph_tiles_smem(int D, int K, int n_slots, int max_deg, int n_hidden, int nbuf);

struct GraphTcArgs {
    AnsatzView an;
    HamView h;
    const uint64_t* samples;
    int64_t Ns;
    RowSet rows;                         // chunk_base over 128-row tiles
    const double* Hst; const int* Hexp;  // h_j(n) and their powers of two (FP64 pass)
    unsigned char* simg;                 // [Ns][K][4D] bytes: split images of h_j(n) (written here)
    float* tts;                          // [Ns][np] tanh (cos form: tan) of theta_k(n) (written here)
    const double* theta;                 // [Ns][n_hidden]
    const double* psi_mant; const int* psi_exp;
    const unsigned char* bimg;           // GraphTcPlan::img on the device
    const int* bexp;
    const float* col0;
    const int* slot;
    const int* last_use;
    int n_slots, max_deg, nbuf;
    uint32_t tmem_cols;                  // power of two >= max_deg * 4 * D
    const float* WT;                     // [2K][np] FP32 correlator weights, transposed
    int np;
    double* partial;                     // [tiles] sum of the terms
    double* partial_abs;                 // [tiles] sum of their magnitudes (optional)
    int64_t* span;                       // [tiles] vertices re-run
    int64_t* mv;                         // [tiles] in-edge D x D products of the rows (optional)
    DevError* err;
};
int launch_graph_tiles(const GraphTcArgs& a, int n_sm, cudaStream_t st);
// each sample's rows (rank, coefficient) stably sorted by their first changed vertex
int launch_graph_sort(const HamView& h, const uint64_t* samples, const RowSet& in, int64_t Ns, int K,
                      uint32_t* out_rank, double* out_coef, cudaStream_t st);

// full K-site product for arbitrary determinants (nqs_amplitude)
int launch_full_amp_fp64(const AnsatzView& an, const uint64_t* dets, int64_t n, double* log_abs,
                          int8_t* sign, cudaStream_t st);

struct GradArgs {
    AnsatzView an;
    const uint64_t* samples;
    int64_t Ns;
    const double* u;
    const double* Lenv; const int* Lexp;  // chain
    const double* Renv; const int* Rexp;
    const double* Hst; const int* Hexp;   // graph
    const double* Gst; const int* Gexp;
    const double* psi_mant; const int* psi_exp;
    const double* theta;
    double* grad_sites;                   // [E][4][D][D]
    double* grad_W;
    double* grad_b;
    double* grad_W2;                      // [n_hidden][2K][2K] (Ising-RBM; NULL: skip)
    int accumulate;                       // 0: overwrite the outputs; 1: add to them
    // scratch of the tensor part (see grad_scratch_bytes): per vertex the
    // sample indices grouped by local state, and per chunk of samples the
    // partial outer-product sums
    int32_t* sidx;                        // [K][Ns]
    int64_t* soff;                        // [K][5]
    double* part;                         // [n_chunks][E][4][D][D]
};
// scratch bytes of the tensor-part gradient for Ns samples
size_t grad_scratch_bytes(const AnsatzView& an, int64_t Ns);
int launch_grad_fp64(const GradArgs& a, cudaStream_t st);

// d log|f| / d theta_k of the correlator: tanh (2cosh), -tan (cos, Ising)
__device__ __forceinline__ double corr_dlog(int corr, double theta)
{
    return corr == 0 ? tanh(theta) : -tan(theta);
}

// log|factor_k| of the correlator at angle theta: log 2cosh or log|cos|
__device__ __forceinline__ double corr_log_factor(int corr, double theta)
{
    return corr == 0 ? log2cosh(theta) : log(fabs(cos(theta)));
}

// theta_k(n) = b_k + sum_s W[k][s] n_s (+ 1/2 sum_{s,t} W2[k][s][t] n_s n_t for
// the Ising-RBM), spin orbitals s = 2p + spin
// cosh d - 1 and sinh d for |d| <= 1 from their Taylor series in z = d^2
// (terms up to d^10 and d^11; the first omitted term is below 2^-28 of the sum)
__device__ __forceinline__ void cosh_sinh_small(float d, float& ch1, float& sh)
{
    const float z = d * d;
    ch1 = z * fmaf(z, fmaf(z, fmaf(z, fmaf(z, 1.f / 3628800.f, 1.f / 40320.f), 1.f / 720.f), 1.f / 24.f), 0.5f);
    sh = fmaf(d * z, fmaf(z, fmaf(z, fmaf(z, fmaf(z, 1.f / 39916800.f, 1.f / 362880.f), 1.f / 5040.f),
                                 1.f / 120.f), 1.f / 6.f), d);
}

__device__ __forceinline__ double corr_theta(const AnsatzView& an, int k, uint64_t na, uint64_t nb)
{
    const int K = an.K, N = 2 * K;
    const double* Wk = an.W + (size_t)k * N;
    double th = an.b[k];
    for (int p = 0; p < K; ++p) {
        if ((na >> p) & 1ull) th += __ldg(Wk + 2 * p);
        if ((nb >> p) & 1ull) th += __ldg(Wk + 2 * p + 1);
    }
    if (an.corr == 2) {
        const double* W2 = an.W2 + (size_t)k * N * N;
        double q = 0.0;
        for (int s = 0; s < N; ++s) {
            if (!(((s & 1) ? nb : na) >> (s >> 1) & 1ull)) continue;
            for (int t = 0; t < N; ++t)
                if ((((t & 1) ? nb : na) >> (t >> 1)) & 1ull) q += __ldg(W2 + (size_t)s * N + t);
        }
        th += 0.5 * q;
    }
    return th;
}

// Ising-RBM: 1/2 sum_{s,t in occ(m)} W2 - 1/2 sum_{s,t in occ(n)} W2 for the
// flips fs[] (sign +1 created, -1 removed): the cross terms with the spin
// orbitals occupied in both, and the pairs inside the created / removed sets.
__device__ __forceinline__ double ising_dq(const AnsatzView& an, int k, uint64_t na, uint64_t nb,
                                           const int* fs, const int* sg, int nf)
{
    const int N = 2 * an.K;
    const double* Wk = an.W2 + (size_t)k * N * N;
    uint64_t ra = 0, rb = 0;                 // removed spin orbitals
    for (int f = 0; f < nf; ++f)
        if (sg[f] < 0) { if (fs[f] & 1) rb |= 1ull << (fs[f] >> 1); else ra |= 1ull << (fs[f] >> 1); }
    double q = 0.0;
    for (int f = 0; f < nf; ++f) {
        const int s = fs[f];
        double x = 0.0;
        for (uint64_t w = na & ~ra; w; w &= w - 1) {
            const int t = 2 * (__ffsll((long long)w) - 1);
            x += __ldg(Wk + (size_t)s * N + t) + __ldg(Wk + (size_t)t * N + s);
        }
        for (uint64_t w = nb & ~rb; w; w &= w - 1) {
            const int t = 2 * (__ffsll((long long)w) - 1) + 1;
            x += __ldg(Wk + (size_t)s * N + t) + __ldg(Wk + (size_t)t * N + s);
        }
        q += sg[f] * x;
        for (int g = 0; g < nf; ++g)
            if (sg[g] == sg[f]) q += sg[f] * __ldg(Wk + (size_t)s * N + fs[g]);
    }
    return 0.5 * q;
}

// log|f(m) / f(n)| for the spin orbitals flipped between n and m, one warp,
// the result on every lane; *neg = 1 when the ratio is negative (cos forms).
__device__ __forceinline__ double corr_log_ratio_warp(const AnsatzView& an, int64_t s,
                                                      const double* theta, const double* lc,
                                                      uint64_t na, uint64_t nb, uint64_t ma,
                                                      uint64_t mb, int lane, int* neg)
{
    *neg = 0;
    const int NH = an.n_hidden;
    if (NH == 0) return 0.0;
    int fs[4], sg[4], nf = 0;
    uint64_t da = na ^ ma, db = nb ^ mb;
    while (da && nf < 4) { const int p = __ffsll((long long)da) - 1; fs[nf] = 2 * p; sg[nf] = ((ma >> p) & 1ull) ? 1 : -1; ++nf; da &= da - 1; }
    while (db && nf < 4) { const int p = __ffsll((long long)db) - 1; fs[nf] = 2 * p + 1; sg[nf] = ((mb >> p) & 1ull) ? 1 : -1; ++nf; db &= db - 1; }
    const int K2 = 2 * an.K;
    double acc = 0.0;
    int odd = 0;
    for (int k = lane; k < NH; k += 32) {
        double d = 0.0;
        for (int f = 0; f < nf; ++f) d += sg[f] * __ldg(an.W + (size_t)k * K2 + fs[f]);
        if (an.corr == 2) d += ising_dq(an, k, na, nb, fs, sg, nf);
        const double th = theta[(size_t)s * NH + k];
        if (an.corr == 0) {
            acc += log2cosh(th + d) - lc[(size_t)s * NH + k];
        } else {
            const double cm = cos(th + d);
            acc += log(fabs(cm)) - lc[(size_t)s * NH + k];
            odd ^= (cm < 0.0) ^ (cos(th) < 0.0);
        }
    }
    for (int o = 16; o; o >>= 1) {
        acc += __shfl_xor_sync(kFull, acc, o);
        odd ^= __shfl_xor_sync(kFull, odd, o);
    }
    *neg = odd;
    return acc;
}

// ---- normalised readout and autoregressive sampling (nqs_rnn.cu) -----------

struct RnnEnvArgs {
    AnsatzView an;
    const uint64_t* samples;
    int64_t Ns;
    double* cells;                        // [Ns][K][D] chosen cells h_i(n)
    double* lp;                           // [Ns][K] 1/2 log P~_i(s_i(n))
    int8_t* sg;                           // [Ns][K] sign of w_i . h_i + c_i
    const double* log_f;                  // [Ns] log|f(n)| (from the correlator pass)
    double* psi_mant;                     // [Ns] sign of Phi(n) f(n) (0: psi(n) = 0)
    int* psi_exp;                         // [Ns] 0
};
int launch_rnn_env(const RnnEnvArgs& a, cudaStream_t st);

struct RnnAmpArgs {
    AnsatzView an;
    HamView h;
    const uint64_t* samples;
    int64_t Ns;
    RowSet rows;
    int rows_per_block;
    const double* cells; const double* lp; const int8_t* sg;
    const double* theta; const double* lc;
    double* partial;                      // [chunks]
    int64_t* span;                        // [chunks] vertices recomputed per chunk
};
int rnn_rows_per_block();
int launch_rnn_amp(const RnnAmpArgs& a, cudaStream_t st);
int launch_rnn_full(const AnsatzView& an, const uint64_t* dets, int64_t n, double* log_abs,
                    int8_t* sign, cudaStream_t st);

// breadth-first autoregressive sampling, one level (vertex i) per call pair.
// A node of level l holds a prefix of the local states of vertices < l; the
// cell of vertex j of a level-l node lives at level j + 1, reached through
// the parent links of levels l, l-1, ..., j + 2.
struct SampleLevel {
    AnsatzView an;
    int level;                            // vertex i (nodes of level i)
    int64_t n_nodes;
    const uint64_t* pa; const uint64_t* pb;   // [n] prefix words
    const int64_t* off; const int64_t* cnt;   // [n] draw offsets and counts
    const int32_t* const* parents;        // device table [K+1]: level l >= 1 -> parent index per node
    const double* const* cells;           // device table [K+1]: level l >= 1 -> [nodes][D], vertex l-1
    double* cand;                         // [n][4][D] candidate cells of vertex i
    int64_t* child_cnt;                   // [n][4] draws per local state
    int64_t* child_flag;                  // [n][4] 1 where a child exists (its draws > 0)
    uint64_t seed;
};
int launch_sample_level(const SampleLevel& a, cudaStream_t st);
struct SampleChildren {
    int level, D;
    int64_t n_nodes;
    const uint64_t* pa; const uint64_t* pb; const int64_t* off;
    const double* cand; const int64_t* child_cnt;
    const int64_t* child_pos;             // [n*4+1] exclusive scan of the child flags
    uint64_t* qa; uint64_t* qb; int64_t* qoff; int64_t* qcnt; int32_t* qparent; double* qcell;
};
int launch_sample_children(const SampleChildren& a, cudaStream_t st);
int launch_sample_output(const uint64_t* pa, const uint64_t* pb, const int64_t* cnt, int64_t n,
                         uint64_t* dets, double* counts, cudaStream_t st);
// u_n of the energy gradient (nqs_grad.cu)
int launch_energy_weights(const double* e_loc, const double* counts, const double* log_f, int64_t Ns,
                          double e_mean, double sum_c, double log_B, bool reweighted, double* u,
                          cudaStream_t st);

}  // namespace nqs
