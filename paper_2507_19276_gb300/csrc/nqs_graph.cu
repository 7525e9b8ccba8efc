// nqs_graph.cu -- the mixed (tensor-core) form of the graph-ordered ansatz.
//
// psi_TN(m) follows Eq. (bdg-rnn-update) with the linear readout and without
// the tensor term: h_i(m) = sum_{e in in(i)} M_e^{s_i(m)} h_{j(e)}(m), with
// h_{-1} = e_0 and psi_TN(m) = (h_{K-1}(m))_0. A connected row m of sample n
// first differs from n at site p, so h_j(m) = h_j(n) for j < p and only the
// vertices p..K-1 are re-run; h_j(n) comes from the FP64 environment pass.
//
// One CTA takes 128 rows of one sample at a time (a tile) and walks the
// vertices in order. For each vertex, each in-edge e with a vertex source j,
// and each local state sigma that an active row of the tile takes there, the
// tile's states h_j (128 rows x D, split into FP16 hi + lo in shared memory)
// are multiplied on the tensor cores by the split image of M_e^sigma
// (hi*hi + lo*hi + hi*lo, FP32 accumulation in tensor memory, one accumulator
// of D columns per (edge, sigma)). Thread r, which owns tensor-memory lane r,
// then adds its row's accumulators for its own sigma, each scaled by the power
// of two of its source, renormalises the sum to a maximum in [0.5, 1) (the
// per-site log-scale of the mixed form) and splits it into the vertex's state
// slot; a row whose first change comes later copies h_i(n) instead. A slot
// is reused once the last vertex reading its state has run.
//
// The ratio psi(m)/psi(n) = psi_TN(m)/psi_TN(n) f(m)/f(n) is formed in FP64
// from the FP32 result, with the correlator ratio of Eq. (RBM) (2cosh, or the
// cos form) as a product over hidden units of cosh(theta + d)/cosh(theta) =
// 1 + (cosh d - 1) + tanh(theta) sinh d (cos: 1 + (cos d - 1) - tan(theta)
// sin d) in FP32, carried as P - 1. Per tile the terms H_nm psi(m)/psi(n)
// and their magnitudes are summed in a fixed order.
#include "nqs_kernels.cuh"
#include "nqs_tc.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace nqs {

namespace {

constexpr int kGtRows = 128;

// the largest s with base[s] <= b, for b not below base[s0]: a galloping
// search forward from s0 (a CTA's tiles ascend, so its sample index does too)
__device__ __forceinline__ int64_t gt_next_sample(const int64_t* base, int64_t Ns, int64_t s0, int64_t b)
{
    int64_t lo = s0, step = 1;
    while (lo + step < Ns && base[lo + step] <= b) { lo += step; step <<= 1; }
    int64_t hi = lo + step < Ns ? lo + step - 1 : Ns - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (base[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// 2^d for d <= 0 in FP32 (0 below the normal range)
__device__ __forceinline__ float pow2_neg(int d)
{
    return d >= -126 ? __int_as_float((127 + d) << 23) : 0.f;
}

// cos d - 1 and sin d for |d| <= 1 from their Taylor series in z = d^2 (the
// first omitted terms are below 2^-28 of the sums)
__device__ __forceinline__ void cos_sin_small(float d, float& c1, float& sn)
{
    const float z = d * d;
    c1 = -z * fmaf(z, fmaf(z, fmaf(z, fmaf(z, 1.f / 3628800.f, -1.f / 40320.f), 1.f / 720.f), -1.f / 24.f), 0.5f);
    sn = fmaf(d * z, fmaf(z, fmaf(z, fmaf(z, fmaf(z, -1.f / 39916800.f, 1.f / 362880.f), -1.f / 5040.f),
                                 1.f / 120.f), -1.f / 6.f), d);
}

// x 2^e, exact: an exponent-field add while the result stays a normal number,
// ldexp otherwise
__device__ __forceinline__ double gt_scale_pow2(double x, int e)
{
    const long long bits = __double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    const int ne = ex + e;
    if (ex != 0 && ex != 0x7FF && ne > 0 && ne < 0x7FF)
        return __longlong_as_double(bits + ((long long)e << 52));
    return ldexp(x, e);
}

// Per sample, once per launch: the split images of the states h_j(n)
// (FP64 -> FP32 -> FP16 hi + lo, [K][hi D | lo D]) and tanh theta_k(n) (cos
// form: tan theta_k(n)) in FP32, [np] per sample, zero-padded.
__global__ void k_graph_prep(const double* __restrict__ Hst, const double* __restrict__ theta, int64_t Ns,
                             int K, int D, int NH, int NP, int corr, unsigned char* __restrict__ simg,
                             float* __restrict__ tts)
{
    const int64_t n1 = Ns * K * D, n2 = Ns * NP;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n1 + n2;
         q += (int64_t)gridDim.x * blockDim.x) {
        if (q < n1) {
            const int64_t si = q / D;                  // (sample, vertex)
            const int c = (int)(q - si * D);
            const float v = (float)Hst[q];
            const __half hv = __float2half_rn(v);
            __half* row = (__half*)(simg + si * 4 * D);
            row[c] = hv;
            row[D + c] = __float2half_rn(v - __half2float(hv));
        } else {
            const int64_t t = q - n1, s = t / NP;
            const int k = (int)(t - s * NP);
            float x = 0.f;
            if (k < NH) {
                const double th = theta[s * NH + k];
                x = (float)(corr == 1 ? tan(th) : tanh(th));
            }
            tts[t] = x;
        }
    }
}

// Thread layout: 256 threads, two per row. Thread t owns row r = 32 (w % 4) +
// lane of tensor-memory lane quadrant w % 4 (warp w) and the half h = w / 4 of
// the row's D columns. Thread 0 also waits for the matrix images and issues
// and waits for the MMAs; with two image buffers thread 32 streams in the next
// vertex's images meanwhile, and the other threads advance their rows'
// correlator products.
constexpr int kGtThreads = 2 * kGtRows;
constexpr int kGtMaxEdges = kMaxOrb * kGtMaxDeg;

template <int D>
__global__ void __launch_bounds__(kGtThreads, 1) k_graph_tiles(GraphTcArgs a)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t mb_mma, mb_b[2], mb_s;   // MMAs done, images landed, sample data landed
    __shared__ OrbLists lists;
    __shared__ int rx[kGtMaxSlots][kGtRows];      // power of two of each slot's rows
    __shared__ int sx[kMaxOrb];                   // powers of two of h_j(n)
    __shared__ int t_ptr[kMaxOrb + 1], t_slot[kMaxOrb], t_last[kMaxOrb], t_msuf[kMaxOrb + 1];
    __shared__ int t_idx[kGtMaxEdges];
    __shared__ short t_bexp[kGtMaxEdges * 4];
    __shared__ int s_pmin;
    __shared__ long long s_sample;
    __shared__ double s_rpsi;                     // 1 / mantissa of psi(n)
    __shared__ float s_max[2][kGtRows];           // per half: the row's largest |entry|
    __shared__ float s_X[kGtRows];                // the odd hidden units' correlator product - 1
    __shared__ double wsum[4], wabs[4];
    __shared__ long long wspan[4], wmv[4];
    constexpr int H = D / 2;                      // columns per row thread
    constexpr int SPT = D <= 32 ? 2 : 1;          // local states per tensor-memory round trip
    constexpr uint32_t kSlot = kGtRows * D * 4;   // hi then lo, 128 x D FP16 each
    constexpr uint32_t kLo = kGtRows * D * 2;
    constexpr uint32_t kImg = 16 * D * D;         // one edge's image: hi [4D][D], then lo [4D][D]
    const int K = a.an.K, NH = a.an.n_hidden, NP = a.np;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool mmat = tid == 0;                   // the MMA thread
    const bool bt = tid == (a.nbuf == 2 ? 32 : 0);   // the image-copy thread
    const int r = 32 * (warp & 3) + lane, h = warp >> 2;
    unsigned char* const slots = smraw;
    unsigned char* const Bs = slots + (size_t)a.n_slots * kSlot;
    unsigned char* const simg = Bs + (size_t)a.nbuf * a.max_deg * kImg; // [K][hi D | lo D]
    float* const WTs = (float*)(simg + (size_t)K * 4 * D);              // [NH][2K]
    float* const tts = WTs + (((size_t)2 * K * NH + 3) & ~(size_t)3);   // [NP] tanh / tan theta
    if (warp == 0) { tc::tmem_alloc(&tmem_slot, a.tmem_cols); tc::tmem_relinquish(); }
    if (mmat) {
        tc::mbar_init(&mb_mma, 1); tc::mbar_init(&mb_b[0], 1); tc::mbar_init(&mb_b[1], 1);
        tc::mbar_init(&mb_s, 1);
    }
    // correlator weights as [unit][spin orbital]: the lanes of a warp read one
    // unit's weights of their rows' different flips
    for (int q = tid; q < 2 * K * NH; q += kGtThreads) {
        const int k = q / (2 * K), f = q - k * 2 * K;
        WTs[q] = a.WT[(size_t)f * NP + k];
    }
    // the graph's tables
    const int E = a.an.pred_ptr[K];
    for (int q = tid; q <= K; q += kGtThreads) t_ptr[q] = a.an.pred_ptr[q];
    for (int q = tid; q < K; q += kGtThreads) { t_slot[q] = a.slot[q]; t_last[q] = a.last_use[q]; }
    for (int q = tid; q < E; q += kGtThreads) t_idx[q] = a.an.pred_idx[q];
    for (int q = tid; q < 4 * E; q += kGtThreads) t_bexp[q] = (short)a.bexp[q];
    __syncthreads();
    if (tid == 0) {
        // D x D products of a row whose first change is p: vertex-source in-edges of p..K-1
        int n = 0;
        t_msuf[K] = 0;
        for (int i = K - 1; i >= 0; --i) {
            for (int e = t_ptr[i]; e < t_ptr[i + 1]; ++e) n += t_idx[e] >= 0;
            t_msuf[i] = n;
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t tlane = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(h * H);
    const uint32_t idesc = tc::idesc_f16(kGtRows, 4 * D);
    uint32_t ph_mma = 0, ph_b0 = 0, ph_b1 = 0, ph_s = 0;
    bool ok = true;
    const int64_t* cb = a.rows.chunk_base;
    const int64_t nblk = cb[a.Ns];
    constexpr uint32_t kPoll = 1u << 24;

    // the matrix images of vertex i's in-edges into image buffer `buf` (copy
    // engine), completing on that buffer's mbarrier
    auto issue_B = [&](int i, int buf) {
        const int e0 = t_ptr[i], e1 = t_ptr[i + 1];
        int nv = 0;
        for (int e = e0; e < e1; ++e) nv += t_idx[e] >= 0;
        unsigned char* dst = Bs + (size_t)buf * a.max_deg * kImg;
        tc::mbar_expect_tx(&mb_b[buf], (uint32_t)nv * kImg);
        for (int e = e0; e < e1; ++e)
            if (t_idx[e] >= 0) tc::bulk_g2s(dst + (size_t)(e - e0) * kImg, a.bimg + (size_t)e * kImg, kImg, &mb_b[buf]);
    };
    // this thread's half of a D-vector's split image into row r of a slot
    auto put_half = [&](unsigned char* slot, const unsigned char* src) {
        #pragma unroll
        for (int c8 = h * (H / 8); c8 < (h + 1) * (H / 8); ++c8) {
            const uint32_t off = tc::op_offset(r, 8 * c8, D);
            *(uint4*)(slot + off) = *(const uint4*)(src + 16 * c8);
            *(uint4*)(slot + kLo + off) = *(const uint4*)(src + 2 * D + 16 * c8);
        }
    };

    int64_t s = 0;
    for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        if (mmat) {
            // the tile's sample, its split states and correlator angles (the copy
            // engine overwrites what the row threads read in the previous tile)
            s = gt_next_sample(cb, a.Ns, s, blk);
            s_sample = s;
            tc::fence_proxy_async();
            const uint32_t bs = (uint32_t)K * 4 * D, bt = (uint32_t)NP * 4;
            tc::mbar_expect_tx(&mb_s, bs + bt);
            tc::bulk_g2s(simg, a.simg + (size_t)s * bs, bs, &mb_s);
            if (bt) tc::bulk_g2s(tts, a.tts + (size_t)s * NP, bt, &mb_s);
            s_pmin = K;
            s_rpsi = 1.0 / a.psi_mant[s];
        }
        __syncthreads();
        s = s_sample;
        const int64_t jb = blk - cb[s];
        const int64_t beg = a.rows.begin ? a.rows.begin[s] : s * a.rows.stride;
        const int64_t left = a.rows.count[s] - jb * kGtRows;
        const int nr = (int)(left < kGtRows ? left : kGtRows);
        const int64_t r0 = beg + jb * kGtRows;
        const uint64_t na = a.samples[2 * s], nb = a.samples[2 * s + 1];
        if (warp == 0) build_lists_warp(na, nb, a.h.K, lists, lane);
        if (tid < K) sx[tid] = a.Hexp[s * K + tid];
        __syncthreads();
        // both threads of a row decode it: the determinant m and its first changed site
        int p = K;
        double coef = 0.0;
        uint64_t ma = na, mb = nb;
        if (r < nr) {
            const Exc e = decode_rank<false>(a.h, lists, a.rows.rank[r0 + r]);
            flip(ma, mb, e.i); flip(ma, mb, e.a);
            if (e.kind == 2) { flip(ma, mb, e.j); flip(ma, mb, e.b); }
            const uint64_t ch = (na ^ ma) | (nb ^ mb);
            p = ch ? __ffsll((long long)ch) - 1 : K - 1;
            coef = a.rows.coef[r0 + r];
        }
        if (warp < 4) {
            const unsigned pm = __reduce_min_sync(kFull, (unsigned)p);
            if (lane == 0) atomicMin(&s_pmin, (int)pm);
        }
        __syncthreads();
        const int pmin = s_pmin;
        if (mmat) {
            issue_B(pmin, 0);
            ok = tc::mbar_wait(&mb_s, ph_s, kPoll) && ok;
        }
        ph_s ^= 1u;
        __syncthreads();
        // the states before pmin that a later vertex reads, in every row
        for (int j = 0; j < pmin; ++j) {
            if (t_last[j] < pmin) continue;
            const int sl = t_slot[j];
            put_half(slots + (size_t)sl * kSlot, simg + (size_t)j * 4 * D);
            if (h == 0) rx[sl][r] = sx[j];
        }
        // the row's correlator ratio, computed in the MMA waits: the flipped
        // spin orbitals (at most four, +1 where m occupies them); each half
        // takes every other hidden unit
        int fi[4];
        float fs[4];
        {
            uint64_t da = na ^ ma, db = nb ^ mb;
            #pragma unroll
            for (int q = 0; q < 4; ++q) {
                fi[q] = 0;
                fs[q] = 0.f;
                if (da) {
                    const int b = __ffsll((long long)da) - 1;
                    da &= da - 1;
                    fi[q] = 2 * b; fs[q] = ((ma >> b) & 1ull) ? 1.f : -1.f;
                } else if (db) {
                    const int b = __ffsll((long long)db) - 1;
                    db &= db - 1;
                    fi[q] = 2 * b + 1; fs[q] = ((mb >> b) & 1ull) ? 1.f : -1.f;
                }
            }
        }
        float X = 0.f;                            // prod_k (1 + x_k) - 1
        int kc = h;                               // next hidden unit
        const bool cos_kind = a.an.corr == 1;
        auto corr_units = [&](int n) {
            for (int u = 0; u < n && kc < NH; ++u, kc += 2) {
                float d = 0.f;
                #pragma unroll
                for (int q = 0; q < 4; ++q) d = fmaf(fs[q], WTs[kc * 2 * K + fi[q]], d);
                float x;
                if (!cos_kind) {
                    float ch1, sh;
                    if (fabsf(d) <= 1.f) {
                        cosh_sinh_small(d, ch1, sh);
                    } else {
                        const float em = expm1f(d), inv = 1.f / (1.f + em);
                        ch1 = 0.5f * em * em * inv;
                        sh = 0.5f * em * (1.f + inv);
                    }
                    x = fmaf(tts[kc], sh, ch1);
                } else {
                    float c1, sn;
                    if (fabsf(d) <= 1.f) {
                        cos_sin_small(d, c1, sn);
                    } else {
                        const float hs = sinf(0.5f * d);
                        c1 = -2.f * hs * hs;
                        sn = sinf(d);
                    }
                    x = fmaf(-tts[kc], sn, c1);
                }
                X = fmaf(X, x, X + x);
            }
        };
        const int per_vertex = (NH / 2 + (K - pmin) - 1) / (K - pmin) + 1;
        float mant = 0.f;
        int mex = 0;
        for (int i = pmin; i < K; ++i) {
            tc::fence_proxy_async();            // the slot rows written by the threads, for the MMAs
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            const int e0 = t_ptr[i], deg = t_ptr[i + 1] - e0;
            const bool any = t_msuf[i] > t_msuf[i + 1];
            const int buf = a.nbuf == 2 ? ((i - pmin) & 1) : 0;
            if (mmat) {
                ok = tc::mbar_wait(&mb_b[buf], buf ? ph_b1 : ph_b0, kPoll) && ok;   // this vertex's images
                if (any) {
                    // one N = 4D group per in-edge (all four local states). The
                    // descriptors hold the start address >> 4 in their low bits:
                    // the k-th 16-wide slice of K is desc + 16 k, the lo half
                    // desc + offset >> 4
                    const uint64_t d0 = tc::desc(0, 128, 16 * D);
                    const uint64_t bbase = tc::smem_addr(Bs + (size_t)buf * a.max_deg * kImg) >> 4;
                    for (int k = 0; k < deg; ++k) {
                        const int j = t_idx[e0 + k];
                        if (j < 0) continue;
                        const uint64_t dA = d0 + (tc::smem_addr(slots + (size_t)t_slot[j] * kSlot) >> 4);
                        const uint64_t dB = d0 + bbase + (uint64_t)k * (kImg >> 4);
                        const uint32_t dc = tmem + (uint32_t)(k * 4 * D);
                        #pragma unroll
                        for (int term = 0; term < 3; ++term)
                            #pragma unroll
                            for (int ks = 0; ks < D / 16; ++ks) {
                                const uint64_t ao = term == 1 ? (kLo >> 4) : 0;
                                const uint64_t bo = term == 2 ? ((8u * D * D) >> 4) : 0;
                                tc::mma_f16(dc, dA + ao + 16 * ks, dB + bo + 16 * ks, idesc, (term | ks) ? 1u : 0u);
                            }
                    }
                    tc::mma_commit(&mb_mma);
                    ok = tc::mbar_wait(&mb_mma, ph_mma, kPoll) && ok;
                }
                // one buffer: the next vertex's images once these MMAs are done
                if (a.nbuf == 1 && i + 1 < K) issue_B(i + 1, 0);
            } else {
                // two buffers: the next vertex's images into the other one (its
                // last reader, the previous vertex's MMAs, has completed)
                if (bt && i + 1 < K) issue_B(i + 1, buf ^ 1);
                if (r < nr) corr_units(per_vertex);   // while the MMAs run
            }
            if (buf) ph_b1 ^= 1u; else ph_b0 ^= 1u;
            if (any) ph_mma ^= 1u;
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            const bool act = i >= p;
            const int sg = sigma_at(ma, mb, i);
            int es[kGtMaxDeg];
            int eref = -(1 << 30);
            #pragma unroll
            for (int k = 0; k < kGtMaxDeg; ++k) {
                es[k] = 0;
                if (k < deg) {
                    const int j = t_idx[e0 + k];
                    es[k] = j < 0 ? 0 : rx[t_slot[j]][r] + t_bexp[(e0 + k) * 4 + sg];
                    eref = es[k] > eref ? es[k] : eref;
                }
            }
            float y[H];
            #pragma unroll
            for (int c = 0; c < H; ++c) y[c] = 0.f;
            if (any) {
                // the local states this warp's active rows take: the tensor-memory
                // loads are warp-wide, so a warp reads only those accumulators
                const int wmsk = (int)__reduce_or_sync(kFull, act ? 1u << sg : 0u);
                int svs[4], nsv = 0;
                #pragma unroll
                for (int sv = 0; sv < 4; ++sv)
                    if ((wmsk >> sv) & 1) svs[nsv++] = sv;
                // SPT local states x three edges per tensor-memory round trip
                for (int g = 0; g < nsv; g += SPT) {
                    #pragma unroll
                    for (int k0 = 0; k0 < kGtMaxDeg; k0 += 3) {
                        if (k0 >= deg) break;
                        uint32_t v[SPT][3][H];
                        #pragma unroll
                        for (int t = 0; t < SPT; ++t) {
                            if (g + t >= nsv) break;
                            const int sv = svs[g + t];
                            #pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                const int k = k0 + q;
                                if (k < deg && t_idx[e0 + k] >= 0) {
                                    const uint32_t ta = tlane + (uint32_t)((k * 4 + sv) * D);
                                    if constexpr (H >= 16) {
                                        #pragma unroll
                                        for (int c0 = 0; c0 < H; c0 += 16) tc::tmem_ld16(ta + c0, v[t][q] + c0);
                                    } else {
                                        tc::tmem_ld8u(ta, v[t][q]);
                                    }
                                }
                            }
                        }
                        tc::tmem_wait_ld();
                        #pragma unroll
                        for (int t = 0; t < SPT; ++t) {
                            if (g + t >= nsv) break;
                            const int sv = svs[g + t];
                            #pragma unroll
                            for (int q = 0; q < 3; ++q) {
                                const int k = k0 + q;
                                if (k < deg && t_idx[e0 + k] >= 0) {
                                    const float f = (act && sg == sv) ? pow2_neg(es[k] - eref) : 0.f;
                                    #pragma unroll
                                    for (int c = 0; c < H; ++c) y[c] = fmaf(__uint_as_float(v[t][q][c]), f, y[c]);
                                }
                            }
                        }
                    }
                }
            }
            float mx = 0.f;
            if (act) {
                #pragma unroll
                for (int k = 0; k < kGtMaxDeg; ++k) {
                    if (k >= deg) break;
                    if (t_idx[e0 + k] >= 0) continue;
                    // M e_0: column 0 of the matrix
                    const float f = pow2_neg(-eref);
                    const float* col = a.col0 + ((size_t)(e0 + k) * 4 + sg) * D + h * H;
                    #pragma unroll
                    for (int c = 0; c < H; ++c) y[c] = fmaf(__ldg(col + c), f, y[c]);
                }
                #pragma unroll
                for (int c = 0; c < H; ++c) mx = fmaxf(mx, fabsf(y[c]));
            }
            s_max[h][r] = mx;
            __syncthreads();                      // the two halves of each row meet
            const int si = t_slot[i];
            if (act) {
                mx = fmaxf(s_max[0][r], s_max[1][r]);
                int ge = 0;
                if (mx > 0.f) frexpf(mx, &ge);
                const bool pw = ge >= -126 && ge <= 126;
                const float sc = pw ? __int_as_float((127 - ge) << 23) : 0.f;
                #pragma unroll
                for (int c = 0; c < H; ++c) y[c] = pw ? y[c] * sc : ldexpf(y[c], -ge);
                const int ex = eref + ge;
                if (i == K - 1) {
                    mant = y[0];
                    mex = ex;
                } else if (si >= 0) {
                    unsigned char* sl = slots + (size_t)si * kSlot;
                    #pragma unroll
                    for (int c8 = 0; c8 < H / 8; ++c8) {
                        __align__(16) __half2 hi[4], lo[4];
                        #pragma unroll
                        for (int q = 0; q < 4; ++q)
                            tc::split_half2(y[8 * c8 + 2 * q], y[8 * c8 + 2 * q + 1], hi[q], lo[q]);
                        const uint32_t off = tc::op_offset(r, h * H + 8 * c8, D);
                        *(uint4*)(sl + off) = *(const uint4*)hi;
                        *(uint4*)(sl + kLo + off) = *(const uint4*)lo;
                    }
                    if (h == 0) rx[si][r] = ex;
                }
            } else if (si >= 0) {
                put_half(slots + (size_t)si * kSlot, simg + (size_t)i * 4 * D);
                if (h == 0) rx[si][r] = sx[i];
            }
        }
        // the rest of the correlator units, then the halves' products meet
        if (r < nr) corr_units(NH);
        if (h == 1) s_X[r] = X;
        __syncthreads();
        // the row's term: coefficient x psi_TN ratio x correlator ratio
        double term = 0.0, ab = 0.0;
        long long sp = 0, mv = 0;
        if (warp < 4 && r < nr) {
            const float X1 = s_X[r];
            X = fmaf(X, X1, X + X1);
            const double tn = gt_scale_pow2((double)mant * s_rpsi, mex - a.psi_exp[s]);
            term = coef * tn * (1.0 + (double)X);
            ab = fabs(term);
            sp = K - p;
            mv = t_msuf[p];
        }
        if (warp < 4) {
            for (int o = 16; o; o >>= 1) {
                term += __shfl_xor_sync(kFull, term, o);
                ab += __shfl_xor_sync(kFull, ab, o);
                sp += __shfl_xor_sync(kFull, sp, o);
                mv += __shfl_xor_sync(kFull, mv, o);
            }
            if (lane == 0) { wsum[warp] = term; wabs[warp] = ab; wspan[warp] = sp; wmv[warp] = mv; }
        }
        __syncthreads();
        if (tid == 0) {
            double t = 0.0, ta = 0.0;
            long long st = 0, sm = 0;
            for (int w = 0; w < 4; ++w) { t += wsum[w]; ta += wabs[w]; st += wspan[w]; sm += wmv[w]; }
            a.partial[blk] = t;
            if (a.partial_abs) a.partial_abs[blk] = ta;
            if (a.span) a.span[blk] = st;
            if (a.mv) a.mv[blk] = sm;
        }
    }
    if (!ok && mmat) report(a.err, 5, 6, (long long)blockIdx.x);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, a.tmem_cols);
}

}  // namespace

size_t graph_tiles_smem(int D, int K, int n_slots, int max_deg, int n_hidden, int nbuf)
{
    const size_t np = (size_t)((n_hidden + 3) & ~3);
    return (size_t)n_slots * kGtRows * D * 4 + (size_t)nbuf * max_deg * 16 * D * D + (size_t)K * 4 * D +
           (((size_t)2 * K * n_hidden + 3) & ~(size_t)3) * 4 + np * 4;
}

bool graph_tc_plan(const double* A, const int* ptr, const int* idx, int K, int D, int n_hidden,
                   GraphTcPlan& p, const char** why)
{
    *why = nullptr;
    if (D != 16 && D != 32 && D != 64) { *why = "bond dimension must be 16, 32 or 64"; return false; }
    int max_deg = 0;
    for (int i = 0; i < K; ++i) max_deg = std::max(max_deg, ptr[i + 1] - ptr[i]);
    if (max_deg > kGtMaxDeg || max_deg * 4 * D > 512) {
        *why = "in-degree x 4 x bond dimension must fit 512 tensor-memory columns";
        return false;
    }
    // last reader of each state; slots by greedy interval colouring (the MMAs of
    // vertex i read its sources before its epilogue writes h_i, so a source
    // whose last reader is i frees its slot for h_i)
    p.last_use.assign(K, -1);
    for (int i = 0; i < K; ++i)
        for (int e = ptr[i]; e < ptr[i + 1]; ++e)
            if (idx[e] >= 0) p.last_use[idx[e]] = std::max(p.last_use[idx[e]], i);
    p.slot.assign(K, -1);
    std::vector<int> busy;       // busy[s]: vertex holding slot s (-1 free)
    for (int i = 0; i < K; ++i) {
        for (size_t s = 0; s < busy.size(); ++s)
            if (busy[s] >= 0 && p.last_use[busy[s]] <= i) busy[s] = -1;
        if (p.last_use[i] <= i) continue;
        size_t s = 0;
        while (s < busy.size() && busy[s] >= 0) ++s;
        if (s == busy.size()) busy.push_back(-1);
        busy[s] = i;
        p.slot[i] = (int)s;
    }
    p.n_slots = std::max<int>(1, (int)busy.size());
    p.max_deg = max_deg;
    if (p.n_slots > kGtMaxSlots) { *why = "more live vertex states than the tile's slots"; return false; }
    int dev = 0, mx = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // two image buffers (the next vertex's images stream in during the MMAs)
    // when they fit, else one
    const size_t margin = 24576;            // the kernel's static shared memory and more
    p.nbuf = 2;
    if (mx > 0 && graph_tiles_smem(D, K, p.n_slots, max_deg, n_hidden, 2) + margin > (size_t)mx) p.nbuf = 1;
    if (mx > 0 && graph_tiles_smem(D, K, p.n_slots, max_deg, n_hidden, 1) + margin > (size_t)mx) {
        *why = "the tile's states and matrix images exceed the shared memory";
        return false;
    }
    // split images of every M_e^sigma scaled by 2^-x (max |M| 2^-x in [0.5, 1)):
    // per edge B[sigma D + n][k] = M_e^sigma[n][k] in the K-major core-matrix
    // layout (4D rows), hi then lo; column 0 in FP32 for the e_0 sources
    const int E = ptr[K];
    const size_t img = (size_t)16 * D * D;
    p.img.assign((size_t)E * img, 0);
    p.bexp.assign((size_t)E * 4, 0);
    p.col0.assign((size_t)E * 4 * D, 0.f);
    for (int e = 0; e < E; ++e)
        for (int sg = 0; sg < 4; ++sg) {
            const double* M = A + ((size_t)e * 4 + sg) * D * D;
            double m = 0.0;
            for (size_t q = 0; q < (size_t)D * D; ++q) m = std::max(m, std::fabs(M[q]));
            int x = 0;
            if (m > 0.0) std::frexp(m, &x);
            const size_t id = (size_t)e * 4 + sg;
            p.bexp[id] = x;
            unsigned char* hi = p.img.data() + (size_t)e * img + (size_t)sg * 2 * D * D;
            unsigned char* lo = hi + (size_t)8 * D * D;
            for (int n = 0; n < D; ++n) {
                p.col0[id * D + n] = (float)M[(size_t)n * D];
                for (int k = 0; k < D; ++k) {
                    const float v = (float)std::ldexp(M[(size_t)n * D + k], -x);
                    const __half h = __float2half_rn(v);
                    const __half l = __float2half_rn(v - __half2float(h));
                    const size_t off = ((size_t)(n >> 3) * (D >> 3) + (k >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2;
                    std::memcpy(hi + off, &h, 2);
                    std::memcpy(lo + off, &l, 2);
                }
            }
        }
    return true;
}

namespace {

// first changed vertex of the row with canonical rank r of sample (na, nb)
__device__ __forceinline__ int gt_first_change(const HamView& h, const OrbLists& L, uint64_t na, uint64_t nb,
                                               uint32_t r, int K)
{
    const Exc e = decode_rank<false>(h, L, r);
    uint64_t ma = na, mb = nb;
    flip(ma, mb, e.i); flip(ma, mb, e.a);
    if (e.kind == 2) { flip(ma, mb, e.j); flip(ma, mb, e.b); }
    const uint64_t ch = (na ^ ma) | (nb ^ mb);
    return ch ? __ffsll((long long)ch) - 1 : K - 1;
}

// Stable counting sort of each sample's rows by their first changed vertex
// (rows with the same one keep their canonical order), one block of 256
// threads per sample: a tile then holds rows that re-run the same vertices.
__global__ void __launch_bounds__(256) k_graph_sort(HamView h, const uint64_t* samples, RowSet in, int K,
                                                    uint32_t* out_rank, double* out_coef)
{
    __shared__ OrbLists lists;
    __shared__ int off[kMaxOrb];                  // next output position of each vertex
    __shared__ int wc[8][kMaxOrb];                // per-warp counts of the current 256 rows
    const int64_t s = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t beg = in.begin ? in.begin[s] : s * in.stride;
    const int cnt = (int)in.count[s];
    const uint64_t na = samples[2 * s], nb = samples[2 * s + 1];
    if (warp == 0) build_lists_warp(na, nb, h.K, lists, lane);
    for (int q = tid; q < 8 * kMaxOrb; q += 256) (&wc[0][0])[q] = 0;
    if (tid < kMaxOrb) off[tid] = 0;
    __syncthreads();
    for (int r = tid; r < cnt; r += 256) atomicAdd(&off[gt_first_change(h, lists, na, nb, in.rank[beg + r], K)], 1);
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int v = 0; v < K; ++v) { const int c = off[v]; off[v] = acc; acc += c; }
    }
    __syncthreads();
    const unsigned below = (1u << lane) - 1u;
    for (int c0 = 0; c0 < cnt; c0 += 256) {
        const int r = c0 + tid;
        const bool valid = r < cnt;
        uint32_t rk = 0;
        double cf = 0.0;
        int p = K;                                // past every vertex: no bucket
        if (valid) {
            rk = in.rank[beg + r];
            cf = in.coef[beg + r];
            p = gt_first_change(h, lists, na, nb, rk, K);
        }
        const unsigned m = __match_any_sync(kFull, p);
        if (valid && lane == __ffs(m) - 1) wc[warp][p] = __popc(m);
        __syncthreads();
        if (valid) {
            int pos = off[p] + __popc(m & below);
            for (int w = 0; w < warp; ++w) pos += wc[w][p];
            out_rank[beg + pos] = rk;
            out_coef[beg + pos] = cf;
        }
        __syncthreads();
        if (tid < K) {
            int t = 0;
            for (int w = 0; w < 8; ++w) { t += wc[w][tid]; wc[w][tid] = 0; }
            off[tid] += t;
        }
        __syncthreads();
    }
}

}  // namespace

int launch_graph_sort(const HamView& h, const uint64_t* samples, const RowSet& in, int64_t Ns, int K,
                      uint32_t* out_rank, double* out_coef, cudaStream_t st)
{
    if (Ns == 0) return 0;
    k_graph_sort<<<(unsigned)Ns, 256, 0, st>>>(h, samples, in, K, out_rank, out_coef);
    return 1;
}

int launch_graph_tiles(const GraphTcArgs& a, int n_sm, cudaStream_t st)
{
    if (a.rows.max_chunks == 0) return 0;
    size_t smem = graph_tiles_smem(a.an.D, a.an.K, a.n_slots, a.max_deg, a.an.n_hidden, a.nbuf);
    // one CTA per multiprocessor: each holds all the tensor-memory columns it
    // allocates for the whole persistent loop
    smem = std::max<size_t>(smem, 120 * 1024);
    const int64_t grid = std::min<int64_t>(n_sm, a.rows.max_chunks);
    k_graph_prep<<<4 * n_sm, 256, 0, st>>>(a.Hst, a.theta, a.Ns, a.an.K, a.an.D, a.an.n_hidden, a.np, a.an.corr,
                                           a.simg, a.tts);
    switch (a.an.D) {
    case 16:
        allow_max_smem(k_graph_tiles<16>);
        k_graph_tiles<16><<<(unsigned)grid, kGtThreads, smem, st>>>(a);
        break;
    case 32:
        allow_max_smem(k_graph_tiles<32>);
        k_graph_tiles<32><<<(unsigned)grid, kGtThreads, smem, st>>>(a);
        break;
    default:
        allow_max_smem(k_graph_tiles<64>);
        k_graph_tiles<64><<<(unsigned)grid, kGtThreads, smem, st>>>(a);
        break;
    }
    return 2;
}

}  // namespace nqs
