// nqs_kernels.cuh -- argument blocks and launchers of every kernel of the
// local-energy path (host orchestration lives in nqs_api.cu).
#pragma once

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
};

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
                                         // environments; 2 (chain): psi(n) only
};
int launch_env_fp64(const EnvArgs& a, cudaStream_t st);

struct RowSet {
    const uint32_t* rank;
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
};
int amp_fp64_rows_per_block(const AnsatzView& an);
size_t amp_fp64_smem(const AnsatzView& an, int rows);
int launch_amp_fp64(const AmpArgs& a, cudaStream_t st);

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
};
int launch_grad_fp64(const GradArgs& a, cudaStream_t st);

}  // namespace nqs
