// nqs_family.cuh -- shared-prefix amplitude evaluation for chain ansaetze
// (see nqs_family.cu for the decomposition).
#pragma once

#include <vector>

#include "nqs_kernels.cuh"

namespace nqs {

template <typename T>
struct FamArgs {
    HamView h;
    int K, D;
    FastDiv div3K, div9K;     // / 3K, / 9K (cluster key fields)
    int split;                // blocks per sample of the correlator-factor kernel
    int nmax;                 // vectors per block-wide mat-vec batch
    size_t batch_bytes;       // shared memory of one batch (see fam_batch_bytes)
    int tc;                   // 1: tensor-core batches (FP32; D % 16 == 0 up to 128, or 192 / 256)
    int tc_cols;              // tensor-memory columns allocated per block
    const uint4* tc_mats;     // [2][K][4] split-FP16 operand images, see fam_tc_images
    const int* tc_exp;        // [2][K][4] power-of-two scale of each image
    DevError* err;
    const T* A;               // [K][4][D][D] site tensors in T, A[a][b]
    const T* AT;              // transposed copy, AT[b][a]
    int df;                   // FP64 tables only: CUDA-core mat-vecs in double-FP32 arithmetic
    const float2* Adf;        // with df: A and AT as FP32 (hi, lo) pairs, hi + lo = the FP64 entry
    const float2* ATdf;
    const uint64_t* samples;  // all samples of the call
    int64_t s0, s1;           // batch = samples [s0, s1)
    // table pool of the batch: rows of D elements (and one exponent each) for the
    // G families, then the H families, the TL entries and the TR rows
    T* pool; int* pool_e;
    int64_t row_H, row_TL, row_TR;   // first pool row of the H, TL and TR tables
    // per batch sample b (= s - s0)
    T* G; int* Ge;            // [b][3][K][K][D]: G_{s,a}(t) at ((a*K+s)*K+t), t >= s
    T* H; int* He;            // [b][3][K][K][D]: H_{s,a}(t) at ((a*K+s)*K+t), t <= s
    const double* pm; const int* pe;   // psi_TN(n) = pm 2^pe (FP64, batch-relative)
    int* tl_end;              // [b][K*K*9] last site a TL cluster is needed at (-1: unused)
    int* tl_idx;              // [b][K*K*9] entry offset of the cluster in the packed TL table
    int* tl_ci;               // [b][K*K*9] cluster index of a TL key
    int* tl_list;             // [b][K*K*9] TL keys in ascending order
    int* tr_idx;              // [b][K*K*9] marks, then row index in the packed TR table
    int* tr_list;             // [b][K*K*9] TR keys in ascending order
    int* tl_total; int* tl_count; int* tr_total;      // [b] TL entries, TL clusters, TR rows
    const int64_t* tl_base; const int64_t* tr_base;   // [b] batch offsets (entries)
    T* TL; int* TLe;          // packed TL entries
    T* TR; int* TRe;          // packed TR rows
    // correlator
    int n_hidden;
    const float4* csite;      // [K][4][3][NP] per-site correlator factors, FP32 (fam_corr_sites)
    const double4_32a* csite64;   // the same in FP64
    const double* theta;      // [Ns][n_hidden] (all samples)
    T* rbl; T* rbr;           // per-object correlator factors (see nqs_family.cu)
    const int64_t* rbl_base; const int64_t* rbr_base;   // [b] object offsets
};

// marks of the clusters the rows need; words (may be NULL) receives each row's
// site word in place of its rank (rows.rank may point to the same array)
template <typename T> int fam_launch_mark(const FamArgs<T>& f, const RowSet& rows, int nb, uint32_t* words,
                                          cudaStream_t st);
template <typename T> int fam_launch_compact(const FamArgs<T>& f, int nb, cudaStream_t st);
// grid = upper bound of the batch's row chunks (128 rows each); blocks map to
// rows.chunk_base[s0] + blockIdx.x. partial_abs (may be NULL) gets each chunk's
// sum of |term|.
template <typename T> int fam_launch_rows(const FamArgs<T>& f, const RowSet& rows, int64_t grid,
                                          double* partial, int64_t* span, double* partial_abs,
                                          cudaStream_t st);

// ---- site-synchronous tables (tensor-core path) ----------------------------
// The boundary vectors and the families at their first site are formed per
// sample on the CUDA cores (k_site_boundary); every other
// vector update of the tables of a sample batch -- one-change families past
// their first site, TL creation and propagation, TR rows -- is one item. The
// items of site step tau fall into 8 groups (side x local state of the
// matrix), each one matrix image, and one launch per step runs 128-row tiles
// over all samples' items.
// One product of a site step: row `src` of the table pool times the step's
// site matrix into row `dst` (rows of D elements; each row's exponent at the
// same index of the exponent pool).
struct SiteItem {
    uint32_t src, dst;
};
struct SiteBufs {
    int64_t* counts;    // [K][8][nbb] items per (step, group, sample)
    int64_t* offs;      // [K*8*nbb + 1] exclusive prefix of counts
    int64_t* bounds;    // [K*8 + 1] first item of each (step, group)
    void* items;        // SiteItem[total]
    int64_t* scan_tmp;  // scan_i64_tmp_elems(K*8*nbb) values
};
// boundary vectors and first-site families, then the item counts, their
// prefix and the (step, group) bounds (device); returns launches
// Tiles: 128-row tensor-core batches (FP32 with images), else f.nmax-row
// CUDA-core batches (FP64, or FP32 without images).
template <typename T> int fam_site_count(const FamArgs<T>& f, const SiteBufs& b, int nbb, cudaStream_t st);
// write the items (after the counts)
template <typename T> int fam_site_fill(const FamArgs<T>& f, const SiteBufs& b, int nbb, cudaStream_t st);
// run the tiles of step tau; bounds: host copy of SiteBufs::bounds
template <typename T> int fam_site_step(const FamArgs<T>& f, const SiteBufs& b, int tau,
                                        const int64_t* bounds, int max_ctas, cudaStream_t st);
// the correlator factors alone (the site-synchronous path builds the tables)
template <typename T> int fam_launch_rbm(const FamArgs<T>& f, int nb, cudaStream_t st);
// per-site correlator factors from W [n_hidden][2K] (device, FP64), in FP32
// (out) and FP64 (out64): [((p * 4 + own) * 3 + a) * NP + k] = {tanh d,
// cosh d - 1, d, 0}, d = the change of theta_k when site p goes from local
// state own to its a-th alternative; NP = n_hidden rounded up to 4 (zero rows
// past n_hidden); returns launches
int fam_corr_sites(const double* W, int K, int n_hidden, float4* out, double4_32a* out64, cudaStream_t st);

// shared memory of the batch buffers of the site tiles
// width of the reduction chunks of a tensor-core batch: the whole D up to 128,
// else 64 (the operands of one chunk then fit shared memory)
__host__ __device__ inline int fam_tc_kc(int D) { return D <= 128 ? D : 64; }
__host__ __device__ inline size_t fam_batch_bytes(int D, int nmax, size_t elem, bool tc)
{
    if (!tc) return (size_t)2 * nmax * D * elem;
    const size_t kc = (size_t)fam_tc_kc(D);
    return (size_t)4 * 128 * kc + (size_t)4 * D * kc + 2 * 128 * 4;
}

// Split-FP16 operand images of the chain's site tensors for the tensor-core
// batches: for side 0 the matrix A_t^s, for side 1 its transpose, each scaled
// by 2^-e (max |entry| in [0.5, 1)). Each image is D / kc reduction chunks
// (kc = fam_tc_kc(D)), each chunk its hi then its lo half, D rows x kc columns
// in the K-major core-matrix layout. images holds 2*K*4 blocks of 4*D*D bytes;
// exps the e.
void fam_tc_images(const double* A, int K, int D, std::vector<unsigned char>& images, std::vector<int>& exps);

// bytes of the per-sample tables (G, H, their exponents, cluster maps)
// elements of one correlator-factor row: N_h rounded up to 4, one more for the
// product term, rounded up to 32
__host__ __device__ inline int rbm_row_len(int NH) { return ((((NH + 3) & ~3) + 1) + 31) & ~31; }

inline size_t fam_bytes_per_sample(int K, int D, size_t elem)
{
    const size_t KK = (size_t)K * K;
    return 2 * (3 * KK * D * elem + 3 * KK * 4) + 6 * KK * 9 * 4 + 64;
}

}  // namespace nqs
