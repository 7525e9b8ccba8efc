// nqs_enum.cu -- enumeration of connected determinants, the eps split, the
// remainder weights and the Philox draws (Sec. 2.4, Sec. 3).
//
// Work unit: a "chunk" of 32 consecutive canonical ranks of one sample, one
// warp-wide evaluation. The count pass records, per chunk, the ballot mask of
// the entries with |H| >= eps, their number and the sum of the integer
// remainder weights (their shift depends only on eps and n_conn, so one pass
// suffices); the write pass evaluates only the deterministic entries, packed
// densely into warps by the masks; the draw pass inverts the per-sample prefix
// of the weight sums and re-evaluates one chunk per draw.
#include "nqs_kernels.cuh"

namespace nqs {

constexpr int kEnumWarps = 8;       // warps per block
constexpr int kChunksPerWarp = 16;  // consecutive chunks per warp (amortises the block's list build)

__global__ void __launch_bounds__(kEnumWarps * 32) k_enum(EnumArgs a)
{
    __shared__ OrbLists lists;
    const int s = a.s0 + blockIdx.y;
    const uint64_t na = a.samples[2 * s], nb = a.samples[2 * s + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool ok = sample_ok(a.h, na, nb);   // else: empty chunks, nothing decoded
    if (warp == 0 && ok) build_lists_warp(na, nb, a.h.K, lists, lane);
    __syncthreads();
    const HamView& h = a.h;
    const size_t srow = (size_t)s * a.n_chunks;
    const uint32_t c_beg = (blockIdx.x * kEnumWarps + warp) * kChunksPerWarp;
    // the chunk's ballot of |H| >= eps, its count and its remainder weight sum
    auto record = [&](uint32_t c, bool valid, double H) {
        const bool det = valid && is_det(H, a.eps_bits);
        const unsigned bal = __ballot_sync(kFull, det);
        if (lane == 0) {
            a.chunk_cnt[srow + c] = __popc(bal);
            if (a.chunk_mask) a.chunk_mask[srow + c] = bal;
        }
        if (a.chunk_w) {
            uint64_t w = (valid && !det) ? weight_of(H, a.shift) : 0ull;
            w = a.h.bitlen_nconn >= 15 ? warp_sum_sliced2(w) : warp_sum_sliced(w);
            if (lane == 0) a.chunk_w[srow + c] = w;
        }
    };
    if (ok && c_beg * 32 >= h.blk[4] && h.blk[4] < h.n_conn) {
        // every rank of this warp is an alpha-beta double (or past the end):
        // decode the first rank, then step the indices by 32 ranks per chunk.
        // H = (ai|bj) with i, a alpha and j, b beta, as in matrix_element.
        const uint32_t x = c_beg * 32 + lane - h.blk[4];
        const uint32_t ia = fdiv(x, h.div_sb), jb = x - ia * h.div_sb.d;
        int io = (int)fdiv(ia, h.div_nv[0]), ao = (int)ia - io * h.nv[0];
        int jo = (int)fdiv(jb, h.div_nv[1]), bo = (int)jb - jo * h.nv[1];
        for (int k = 0; k < kChunksPerWarp; ++k) {
            const uint32_t c = c_beg + k;
            if (c >= a.n_chunks) break;
            const bool valid = c * 32 + lane < h.n_conn;
            double H = 0.0;
            if (valid)
                H = eri_at(h, lists.vir[0][ao], lists.occ[0][io], lists.vir[1][bo], lists.occ[1][jo]);
            record(c, valid, H);
            bo += 32;
            while (bo >= h.nv[1]) {          // nv_beta >= 1 when the block is not empty
                bo -= h.nv[1];
                if (++jo == h.no[1]) { jo = 0; if (++ao == h.nv[0]) { ao = 0; ++io; } }
            }
        }
        return;
    }
    for (int k = 0; k < kChunksPerWarp; ++k) {
        const uint32_t c = c_beg + k;
        if (c >= a.n_chunks) break;
        const uint32_t r = c * 32 + lane;
        const bool valid = ok && r < h.n_conn;
        double H = 0.0;
        if (valid) {
            uint64_t ma, mb;
            int odd;
            // the split and the weights depend on |H| only: no phase here
            Exc e = decode_rank<false>(h, lists, r);
            H = matrix_element(h, na, nb, e, ma, mb, odd);
        }
        record(c, valid, H);
    }
}

// Write pass: the deterministic entries of 8 consecutive chunks per warp,
// dealt out one per lane through the chunks' ballot masks (about 30 per warp
// on H50 instead of 8 live lanes out of 32 per chunk). Entry j of the group
// lies in the chunk whose mask prefix brackets j; its list position is that
// chunk's offset plus its rank among the chunk's set bits, so the lists stay
// in canonical order.
constexpr int kWriteChunks = 8;
constexpr int kWriteGroups = 4;     // groups of kWriteChunks chunks per warp

// position of the (k+1)-th set bit of m (k < popc(m)), by halving with popc
__device__ __forceinline__ int nth_set_bit(uint32_t m, int k)
{
    int pos = 0;
    #pragma unroll
    for (int w = 16; w >= 2; w >>= 1) {
        const int c = __popc(m & ((1u << w) - 1u));
        if (k >= c) { k -= c; m >>= w; pos += w; }
    }
    return pos + (k >= (int)(m & 1u) ? 1 : 0);
}

__global__ void __launch_bounds__(kEnumWarps * 32, 5) k_write_dets(EnumArgs a)
{
    __shared__ OrbLists lists;
    const int s = a.s0 + blockIdx.y;
    const uint64_t na = a.samples[2 * s], nb = a.samples[2 * s + 1];
    if (!sample_ok(a.h, na, nb)) return;     // block-uniform: no list to write
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (warp == 0) build_lists_warp(na, nb, a.h.K, lists, lane);
    __syncthreads();
    const HamView& h = a.h;
    const size_t srow = (size_t)s * a.n_chunks;
    for (int grp = 0; grp < kWriteGroups; ++grp) {
        const uint32_t c0 = ((blockIdx.x * kEnumWarps + warp) * kWriteGroups + grp) * kWriteChunks;
        if (c0 >= a.n_chunks) break;
        uint32_t m = 0, co = 0;
        if (lane < kWriteChunks && c0 + lane < a.n_chunks) {
            m = a.chunk_mask[srow + c0 + lane];
            co = a.chunk_off[srow + c0 + lane];
        }
        const int cnt = __popc(m);
        int incl = cnt;
        for (int o = 1; o < kWriteChunks; o <<= 1) {
            const int u = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += u;
        }
        int ex[kWriteChunks];
        uint32_t mk[kWriteChunks], cof[kWriteChunks];
        #pragma unroll
        for (int k = 0; k < kWriteChunks; ++k) {
            ex[k] = __shfl_sync(kFull, incl - cnt, k);
            mk[k] = __shfl_sync(kFull, m, k);
            cof[k] = __shfl_sync(kFull, co, k);
        }
        const int64_t base = a.det_off[s];
        const int total = __shfl_sync(kFull, incl, kWriteChunks - 1);
        for (int j = lane; j < total; j += 32) {
            int k = 0, e0 = ex[0];                       // chunk of entry j, selected with
            uint32_t bits = mk[0], off = cof[0];         // static indices (no local memory)
            #pragma unroll
            for (int q = 1; q < kWriteChunks; ++q)
                if (ex[q] <= j) { k = q; e0 = ex[q]; bits = mk[q]; off = cof[q]; }
            const int idx = j - e0;                      // rank among the chunk's set bits
            const uint32_t r = (c0 + k) * 32 + (uint32_t)nth_set_bit(bits, idx);
            uint64_t ma, mb;
            int odd;
            const Exc e = decode_rank(h, lists, r);
            const double H = matrix_element(h, na, nb, e, ma, mb, odd);
            const int64_t pos = base + off + idx;
            if (a.out_rank) a.out_rank[pos] = r;
            if (a.out_H) a.out_H[pos] = H;
            if (a.out_det) { a.out_det[2 * pos] = ma; a.out_det[2 * pos + 1] = mb; }
            if (a.out_sign) a.out_sign[pos] = odd ? -1 : 1;
        }
    }
}

int launch_enum(const EnumArgs& args, int64_t Ns, bool write, cudaStream_t st)
{
    const uint32_t per_block = kEnumWarps * (write ? kWriteChunks * kWriteGroups : kChunksPerWarp);
    const uint32_t gx = (args.n_chunks + per_block - 1) / per_block;
    if (gx == 0) return 0;
    int n = 0;
    for (int64_t s0 = 0; s0 < Ns; s0 += 65535, ++n) {
        EnumArgs a = args;
        a.s0 = (int)s0;
        dim3 grid(gx, (unsigned)((Ns - s0) < 65535 ? (Ns - s0) : 65535));
        if (write) k_write_dets<<<grid, kEnumWarps * 32, 0, st>>>(a);
        else k_enum<<<grid, kEnumWarps * 32, 0, st>>>(a);
    }
    return n;
}

// ---------------------------------------------------------------------------
// Draws: one warp per (sample, draw)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_draws(DrawArgs a)
{
    __shared__ OrbLists lists[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t g = (int64_t)blockIdx.x * 8 + warp;
    if (g >= a.Ns * (int64_t)a.n_draws) return;
    const int64_t s = g / a.n_draws;
    const int d = (int)(g - s * a.n_draws);
    const size_t srow = (size_t)s * a.n_chunks;
    const uint64_t W = a.n_chunks ? a.chunk_pre[srow + a.n_chunks - 1] : 0ull;
    const uint64_t na = a.samples[2 * s], nb = a.samples[2 * s + 1];
    if (W == 0 || !sample_ok(a.h, na, nb)) {
        if (lane == 0) a.out_rank[g] = -1;
        return;
    }
    build_lists_warp(na, nb, a.h.K, lists[warp], lane);
    __syncwarp();
    // target t = floor(x W / 2^64), then the first chunk whose inclusive prefix > t
    const uint64_t x = philox_first((uint64_t)d, (uint64_t)(a.index ? a.index[s] : a.index_base + s), a.seed);
    const uint64_t t = __umul64hi(x, W);
    // first chunk whose inclusive prefix exceeds t, by a 32-way search: each
    // round the lanes probe 32 evenly spaced chunks of [lo, hi] (the prefix is
    // nondecreasing and its last entry W > t, so the answer stays in range)
    uint32_t lo = 0, hi = a.n_chunks - 1;
    while (hi - lo >= 32) {
        const uint32_t span = hi - lo + 1;
        const uint32_t p = lo + (uint32_t)(((uint64_t)span * (lane + 1)) / 32) - 1;   // p <= hi
        const unsigned above = __ballot_sync(kFull, a.chunk_pre[srow + p] > t);
        // the first probe above t bounds the answer from above, the one before from below
        const int f = __ffs(above) - 1;                 // above != 0: lane 31 probes hi
        const uint32_t nhi = (uint32_t)__shfl_sync(kFull, p, f);
        const uint32_t nlo = f ? (uint32_t)__shfl_sync(kFull, p, f - 1) + 1 : lo;
        __syncwarp();
        lo = nlo;
        hi = nhi;
    }
    {
        const uint32_t p = lo + lane;
        const bool in = p <= hi;
        const unsigned above = __ballot_sync(kFull, in && a.chunk_pre[srow + p] > t);
        lo = lo + (uint32_t)(__ffs(above) - 1);
    }
    const uint32_t c = lo;
    const uint32_t r = c * 32 + lane;
    uint64_t w = 0;
    if (r < a.h.n_conn) {
        Exc e = decode_rank<false>(a.h, lists[warp], r);     // weights need |H| only
        uint64_t ma, mb;
        int odd;
        const double H = matrix_element(a.h, na, nb, e, ma, mb, odd);
        if (!is_det(H, a.eps_bits)) w = weight_of(H, a.shift);
    }
    const uint64_t incl = warp_incl_scan_u64(w, lane);
    const uint64_t base = c ? a.chunk_pre[srow + c - 1] : 0ull;
    const unsigned hit = __ballot_sync(kFull, base + incl > t);
    if (lane == 0) a.out_rank[g] = hit ? (int64_t)(c * 32 + (__ffs(hit) - 1)) : -1;
}

int launch_draws(const DrawArgs& a, cudaStream_t st)
{
    const int64_t n = a.Ns * (int64_t)a.n_draws;
    if (n == 0) return 0;
    k_draws<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(a);
    return 1;
}

// ---------------------------------------------------------------------------
// Dedup of the draws of a sample: sort, unique, multiplicity -> amplitude rows
// with coefficient mult/N_eps * H * W / w.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(1024) k_dedup(DedupArgs a)
{
    extern __shared__ uint32_t keys[];      // [P] padded to a power of two
    __shared__ int head_scan[1024];
    __shared__ OrbLists lists;
    const int s = blockIdx.x;
    const int P = a.pow2;
    const int64_t base = (int64_t)s * a.n_draws;
    if (!sample_ok(a.h, a.samples[2 * s], a.samples[2 * s + 1])) {   // block-uniform
        if (threadIdx.x == 0) a.n_unique[s] = 0;
        return;
    }
    for (int i = threadIdx.x; i < P; i += blockDim.x)
        keys[i] = i < a.n_draws && a.ranks[base + i] >= 0 && a.ranks[base + i] < (int64_t)a.h.n_conn
                      ? (uint32_t)a.ranks[base + i] : 0xffffffffu;
    const uint64_t na = a.samples[2 * s], nb = a.samples[2 * s + 1];
    if (threadIdx.x < 32) build_lists_warp(na, nb, a.h.K, lists, threadIdx.x);
    __syncthreads();
    // bitonic sort, ascending
    for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                int l = i ^ j;
                if (l > i) {
                    uint32_t x = keys[i], y = keys[l];
                    bool up = (i & k) == 0;
                    if ((x > y) == up) { keys[i] = y; keys[l] = x; }
                }
            }
            __syncthreads();
        }
    // heads of runs; each thread owns a contiguous slice of `per` entries
    const int per = (P + blockDim.x - 1) / blockDim.x;
    const int i0 = threadIdx.x * per;
    int cnt = 0;
    for (int i = i0; i < i0 + per && i < P; ++i)
        if (keys[i] != 0xffffffffu && (i == 0 || keys[i] != keys[i - 1])) ++cnt;
    head_scan[threadIdx.x] = cnt;
    __syncthreads();
    for (int o = 1; o < (int)blockDim.x; o <<= 1) {
        int v = threadIdx.x >= (unsigned)o ? head_scan[threadIdx.x - o] : 0;
        __syncthreads();
        head_scan[threadIdx.x] += v;
        __syncthreads();
    }
    int u = head_scan[threadIdx.x] - cnt;   // exclusive
    const int total = head_scan[blockDim.x - 1];
    const uint64_t W = a.W[s];
    for (int i = i0; i < i0 + per && i < P; ++i) {
        if (keys[i] == 0xffffffffu || (i > 0 && keys[i] == keys[i - 1])) continue;
        int e = i + 1;
        while (e < P && keys[e] == keys[i]) ++e;
        const uint32_t r = keys[i];
        Exc ex = decode_rank(a.h, lists, r);
        uint64_t ma, mb;
        int odd;
        const double H = matrix_element(a.h, na, nb, ex, ma, mb, odd);
        uint64_t w = weight_of(H, a.shift);
        double coef = ((double)(e - i) / (double)a.n_draws) * H * ((double)W / (double)w);
        a.out_rank[base + u] = r;
        a.out_coef[base + u] = coef;
        ++u;
    }
    if (threadIdx.x == 0) a.n_unique[s] = total;
}

int launch_dedup(const DedupArgs& a, int64_t Ns, cudaStream_t st)
{
    if (Ns == 0) return 0;
    const int threads = a.pow2 >= 1024 ? 1024 : (a.pow2 < 32 ? 32 : a.pow2);
    k_dedup<<<(unsigned)Ns, threads, a.pow2 * sizeof(uint32_t), st>>>(a);
    return 1;
}

// ---------------------------------------------------------------------------
// Validation of the input determinants
// ---------------------------------------------------------------------------

__global__ void k_validate(const uint64_t* samples, int64_t Ns, int K, int na, int nb,
                           DevError* err)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= Ns) return;
    const uint64_t a = samples[2 * s], b = samples[2 * s + 1];
    const uint64_t outside = K >= 64 ? 0ull : ~((1ull << K) - 1ull);
    if ((a & outside) || (b & outside)) report(err, 1, 1, s);
    else if (__popcll(a) != na || __popcll(b) != nb) report(err, 1, 2, s);
}

int launch_validate(const uint64_t* samples, int64_t Ns, int K, int na, int nb, DevError* err,
                    cudaStream_t st)
{
    if (Ns == 0) return 0;
    k_validate<<<(unsigned)((Ns + 255) / 256), 256, 0, st>>>(samples, Ns, K, na, nb, err);
    return 1;
}

}  // namespace nqs
