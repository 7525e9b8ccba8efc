// nqs_util.cu -- integral build, prefix scans, per-sample reductions and the
// energy summary (Sec. 2.1 weighted mean, Sec. 2.3 B and E~_loc).
#include "nqs_kernels.cuh"

namespace nqs {

// (pq|rs) = sum_x L[x][p][q] L[x][r][s], ascending x, fused multiply-add,
// stored at [p][q][s][r] (the layout eri_at reads).
__global__ void k_build_eri(const double* L, int n_chol, int K, double* eri)
{
    const int64_t KK = (int64_t)K * K;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= KK * KK) return;
    const int64_t pq = idx / KK, sr = idx - pq * KK;
    const int64_t s = sr / K, r = sr - s * K, rs = r * K + s;
    double acc = 0.0;
    for (int x = 0; x < n_chol; ++x)
        acc = __fma_rn(__ldg(L + x * KK + pq), __ldg(L + x * KK + rs), acc);
    eri[idx] = acc;
}

int launch_build_eri(const double* L, int n_chol, int K, double* eri, cudaStream_t st)
{
    const int64_t n = (int64_t)K * K * K * K;
    k_build_eri<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(L, n_chol, K, eri);
    return 1;
}

// a full (pq|rs) table [p][q][r][s] into the layout eri_at reads, [p][q][s][r]
__global__ void k_swap_eri(const double* in, int K, double* eri)
{
    const int64_t KK = (int64_t)K * K;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= KK * KK) return;
    const int64_t pq = idx / KK, sr = idx - pq * KK;
    const int64_t s = sr / K, r = sr - s * K;
    eri[idx] = in[pq * KK + r * K + s];
}

int launch_swap_eri(const double* in, int K, double* eri, cudaStream_t st)
{
    const int64_t n = (int64_t)K * K * K * K;
    k_swap_eri<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(in, K, eri);
    return 1;
}

// Block-wide inclusive scan of one value per thread (blockDim multiple of 32).
template <typename T>
__device__ T block_incl_scan(T v, T* warp_tot)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? warp_tot[lane] : T(0);
        for (int o = 1; o < 32; o <<= 1) {
            T t = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += t;
        }
        if (lane < nw) warp_tot[lane] = w;
    }
    __syncthreads();
    if (warp) v += warp_tot[warp - 1];
    __syncthreads();
    return v;
}

__global__ void k_scan_chunks_u32(const uint32_t* cnt, uint32_t* off, int64_t* total,
                                  uint32_t n_chunks)
{
    __shared__ uint32_t wt[32];
    const size_t row = (size_t)blockIdx.x * n_chunks;
    uint32_t carry = 0;
    for (uint32_t t0 = 0; t0 < n_chunks; t0 += blockDim.x) {
        const uint32_t i = t0 + threadIdx.x;
        const uint32_t v = i < n_chunks ? cnt[row + i] : 0u;
        const uint32_t inc = block_incl_scan<uint32_t>(v, wt);
        if (i < n_chunks) off[row + i] = carry + inc - v;
        carry += wt[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) total[blockIdx.x] = carry;
}

int launch_scan_chunks_u32(const uint32_t* cnt, uint32_t* off, int64_t* total, int64_t Ns,
                           uint32_t n_chunks, cudaStream_t st)
{
    if (Ns == 0) return 0;
    k_scan_chunks_u32<<<(unsigned)Ns, 256, 0, st>>>(cnt, off, total, n_chunks);
    return 1;
}

__global__ void k_scan_chunks_u64(uint64_t* w, uint64_t* total, uint32_t n_chunks)
{
    __shared__ uint64_t wt[32];
    const size_t row = (size_t)blockIdx.x * n_chunks;
    uint64_t carry = 0;
    for (uint32_t t0 = 0; t0 < n_chunks; t0 += blockDim.x) {
        const uint32_t i = t0 + threadIdx.x;
        const uint64_t v = i < n_chunks ? w[row + i] : 0ull;
        const uint64_t inc = block_incl_scan<uint64_t>(v, wt);
        if (i < n_chunks) w[row + i] = carry + inc;
        carry += wt[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) total[blockIdx.x] = carry;
}

int launch_scan_chunks_u64(uint64_t* w, uint64_t* total, int64_t Ns, uint32_t n_chunks,
                           cudaStream_t st)
{
    if (Ns == 0) return 0;
    k_scan_chunks_u64<<<(unsigned)Ns, 256, 0, st>>>(w, total, n_chunks);
    return 1;
}

__global__ void __launch_bounds__(1024) k_scan_i64(const int64_t* in, int64_t* out, int64_t n, int rows)
{
    __shared__ int64_t wt[32];
    int64_t carry = 0;
    for (int64_t t0 = 0; t0 < n; t0 += blockDim.x) {
        const int64_t i = t0 + threadIdx.x;
        int64_t v = i < n ? in[i] : 0;
        if (rows > 0) v = (v + rows - 1) / rows;
        const int64_t inc = block_incl_scan<int64_t>(v, wt);
        if (i < n) out[i] = carry + inc - v;
        carry += wt[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = carry;
}

int launch_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t st)
{
    k_scan_i64<<<1, 1024, 0, st>>>(in, out, n, 0);
    return 1;
}

// Multi-block exclusive scan: sums of 4096-element tiles, one block scans the
// sums, then every tile rescans its elements from its offset (integers: the
// result does not depend on the tiling).
constexpr int kScanTile = 4096;   // 1024 threads x 4 elements

__global__ void __launch_bounds__(1024) k_scan_tile_sums(const int64_t* in, int64_t n, int64_t* sums)
{
    __shared__ int64_t wt[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t v = 0;
    #pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t i = base + k * 1024 + threadIdx.x;
        if (i < n) v += in[i];
    }
    v = block_incl_scan<int64_t>(v, wt);
    if (threadIdx.x == blockDim.x - 1) sums[blockIdx.x] = v;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(const int64_t* in, int64_t* out, int64_t n,
                                                      const int64_t* tile_off)
{
    __shared__ int64_t wt[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + 4 * (int64_t)threadIdx.x;
    int64_t x[4], s = 0;
    #pragma unroll
    for (int k = 0; k < 4; ++k) {
        x[k] = base + k < n ? in[base + k] : 0;
        s += x[k];
    }
    const int64_t inc = block_incl_scan<int64_t>(s, wt);
    int64_t run = tile_off[blockIdx.x] + inc - s;
    #pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < n) out[base + k] = run;
        run += x[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = run;
}

int launch_scan_i64_wide(const int64_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t st)
{
    if (n <= 16 * kScanTile || !tmp) return launch_scan_i64(in, out, n, st);
    const int64_t nt = (n + kScanTile - 1) / kScanTile;
    int64_t* sums = tmp;
    int64_t* offs = tmp + nt + 1;
    k_scan_tile_sums<<<(unsigned)nt, 1024, 0, st>>>(in, n, sums);
    k_scan_i64<<<1, 1024, 0, st>>>(sums, offs, nt, 0);
    k_scan_tiles<<<(unsigned)nt, 1024, 0, st>>>(in, out, n, offs);
    return 3;
}

int launch_chunk_base(const int64_t* cnt, int rows, int64_t* out, int64_t Ns, cudaStream_t st)
{
    k_scan_i64<<<1, 1024, 0, st>>>(cnt, out, Ns, rows);
    return 1;
}

// ---------------------------------------------------------------------------
// E_loc per sample = H_nn + sum of det-row partials + sum of draw-row partials
// (fixed order), then the weighted summary in one block (fixed tree order).
// ---------------------------------------------------------------------------

__global__ void k_final_samples(FinalArgs a)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.Ns) return;
    double ed = 0.0, es = 0.0;
    for (int64_t b = a.base_det[s]; b < a.base_det[s + 1]; ++b) ed += a.part_det[b];
    if (a.base_draw)
        for (int64_t b = a.base_draw[s]; b < a.base_draw[s + 1]; ++b) es += a.part_draw[b];
    a.e_loc[s] = a.h_diag[s] + ed + es;
    if (a.e_abs) {
        double ea = fabs(a.h_diag[s]);
        for (int64_t b = a.base_det[s]; b < a.base_det[s + 1]; ++b) ea += a.part_det_abs[b];
        if (a.base_draw && a.part_draw_abs)
            for (int64_t b = a.base_draw[s]; b < a.base_draw[s + 1]; ++b) ea += a.part_draw_abs[b];
        a.e_abs[s] = ea;
    }
    if (a.e_det) a.e_det[s] = ed;
    if (a.e_stoch) a.e_stoch[s] = es;
}

__device__ double block_reduce_sum(double v, double* sh)
{
    v = warp_sum_f64(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
    __syncthreads();
    return r;   // valid in thread 0
}

__global__ void __launch_bounds__(256) k_summary(FinalArgs a)
{
    __shared__ double sh[32];
    __shared__ double bc;
    double m = -INFINITY;
    for (int64_t s = threadIdx.x; s < a.Ns; s += blockDim.x) m = fmax(m, 2.0 * a.log_f[s]);
    m = warp_max_f64(m);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = -INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = fmax(mm, sh[w]);
        bc = mm;
    }
    __syncthreads();
    m = bc;
    __syncthreads();
    double sc = 0.0, sce = 0.0, scf = 0.0, ndet = 0.0, nu = 0.0;
    for (int64_t s = threadIdx.x; s < a.Ns; s += blockDim.x) {
        const double c = a.counts ? a.counts[s] : 1.0;
        sc += c;
        sce += c * a.e_loc[s];
        scf += c * exp(2.0 * a.log_f[s] - m);
        if (a.det_off) ndet += (double)(a.det_off[s + 1] - a.det_off[s]);
        if (a.n_unique) nu += (double)a.n_unique[s];
    }
    double sp = 0.0;
    if (a.span_det)
        for (int64_t b = threadIdx.x; b < a.base_det[a.Ns]; b += blockDim.x) sp += (double)a.span_det[b];
    if (a.span_draw && a.base_draw)
        for (int64_t b = threadIdx.x; b < a.base_draw[a.Ns]; b += blockDim.x) sp += (double)a.span_draw[b];
    double mv = 0.0;
    if (a.mv_det)
        for (int64_t b = threadIdx.x; b < a.base_det[a.Ns]; b += blockDim.x) mv += (double)a.mv_det[b];
    if (a.mv_draw && a.base_draw)
        for (int64_t b = threadIdx.x; b < a.base_draw[a.Ns]; b += blockDim.x) mv += (double)a.mv_draw[b];
    sp = block_reduce_sum(sp, sh);
    mv = block_reduce_sum(mv, sh);
    sc = block_reduce_sum(sc, sh);
    sce = block_reduce_sum(sce, sh);
    scf = block_reduce_sum(scf, sh);
    ndet = block_reduce_sum(ndet, sh);
    nu = block_reduce_sum(nu, sh);
    if (threadIdx.x == 0) bc = m + log(scf / sc);
    __syncthreads();
    const double logB = bc;
    double set = 0.0;
    for (int64_t s = threadIdx.x; s < a.Ns; s += blockDim.x) {
        const double c = a.counts ? a.counts[s] : 1.0;
        set += c * exp(2.0 * a.log_f[s] - logB) * a.e_loc[s];
    }
    set = block_reduce_sum(set, sh);
    if (threadIdx.x == 0) {
        a.summary[0] = sce / sc;
        a.summary[1] = sc;
        a.summary[2] = logB;
        a.summary[3] = set / sc;
        a.summary[4] = ndet;
        a.summary[5] = nu;
        a.summary[6] = sp;
        a.summary[7] = mv;
    }
}

int launch_summary(const FinalArgs& a, cudaStream_t st)
{
    if (a.Ns == 0 || !a.summary) return 0;
    k_summary<<<1, 256, 0, st>>>(a);
    return 1;
}

// samples picked for re-evaluation: their words, counts and global positions
__global__ void k_gather_picked(const int64_t* idx, int64_t n, const uint64_t* samples,
                                const double* counts, int64_t base, uint64_t* out_s, double* out_c,
                                int64_t* out_pos)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t s = idx[j];
    out_s[2 * j] = samples[2 * s];
    out_s[2 * j + 1] = samples[2 * s + 1];
    out_c[j] = counts ? counts[s] : 1.0;
    out_pos[j] = base + s;
}

__global__ void k_scatter_picked(const int64_t* idx, int64_t n, const double* v, double* out)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[idx[j]] = v[j];
}

int launch_gather_picked(const int64_t* idx, int64_t n, const uint64_t* samples, const double* counts,
                         int64_t base, uint64_t* out_s, double* out_c, int64_t* out_pos, cudaStream_t st)
{
    if (n == 0) return 0;
    k_gather_picked<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(idx, n, samples, counts, base, out_s,
                                                                 out_c, out_pos);
    return 1;
}

int launch_scatter_picked(const int64_t* idx, int64_t n, const double* v, double* out, cudaStream_t st)
{
    if (n == 0) return 0;
    k_scatter_picked<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(idx, n, v, out);
    return 1;
}

int launch_finalize(const FinalArgs& a, cudaStream_t st)
{
    if (a.Ns == 0) return 0;
    k_final_samples<<<(unsigned)((a.Ns + 255) / 256), 256, 0, st>>>(a);
    if (a.summary) k_summary<<<1, 256, 0, st>>>(a);
    return a.summary ? 2 : 1;
}

}  // namespace nqs
