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

__device__ __forceinline__ int64_t gt_find_sample(const int64_t* base, int64_t Ns, int64_t b)
{
    int64_t lo = 0, hi = Ns - 1;       // largest s with base[s] <= b
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

// copy a D-vector's split image (hi [D], lo [D], FP16) into row r of a slot
template <int D>
__device__ __forceinline__ void put_row(unsigned char* slot, const unsigned char* src, int r)
{
    constexpr uint32_t kLo = kGtRows * D * 2;
    #pragma unroll
    for (int c8 = 0; c8 < D / 8; ++c8) {
        const uint32_t off = tc::op_offset(r, 8 * c8, D);
        *(uint4*)(slot + off) = *(const uint4*)(src + 16 * c8);
        *(uint4*)(slot + kLo + off) = *(const uint4*)(src + 2 * D + 16 * c8);
    }
}

template <int D>
__global__ void __launch_bounds__(kGtRows, 1) k_graph_tiles(GraphTcArgs a)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ OrbLists lists;
    __shared__ int rx[kGtMaxSlots][kGtRows];      // power of two of each slot's rows
    __shared__ int vmask[kMaxOrb];                // local states of the active rows per vertex
    __shared__ int sx[kMaxOrb];                   // powers of two of h_j(n)
    __shared__ int s_pmin;
    __shared__ double wsum[kGtRows / 32], wabs[kGtRows / 32];
    __shared__ long long wspan[kGtRows / 32], wmv[kGtRows / 32];
    constexpr uint32_t kSlot = kGtRows * D * 4;   // hi then lo, 128 x D FP16 each
    constexpr uint32_t kLo = kGtRows * D * 2;
    constexpr uint32_t kImg = 4 * D * D;          // one (edge, sigma) matrix image: hi then lo
    const int K = a.an.K, NH = a.an.n_hidden, NP = a.np;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned char* const slots = smraw;
    unsigned char* const Bs = slots + (size_t)a.n_slots * kSlot;
    unsigned char* const simg = Bs + (size_t)a.max_deg * 4 * kImg;      // [K][hi D | lo D]
    float* const WTs = (float*)(simg + (size_t)K * 4 * D);              // [2K][NP]
    float* const tts = WTs + (size_t)2 * K * NP;                        // [NH] tanh / tan theta
    if (warp == 0) { tc::tmem_alloc(&tmem_slot, a.tmem_cols); tc::tmem_relinquish(); }
    if (tid == 0) tc::mbar_init(&mbar, 1);
    for (int q = tid; q < 2 * K * NP; q += kGtRows) WTs[q] = a.WT[q];
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t tlane = tmem + ((uint32_t)(32 * warp) << 16);
    const uint32_t idesc = tc::idesc_f16(kGtRows, D);
    const int* __restrict__ pptr = a.an.pred_ptr;
    const int* __restrict__ pidx = a.an.pred_idx;
    uint32_t phase = 0;
    bool ok = true;
    const int64_t* cb = a.rows.chunk_base;
    const int64_t nblk = cb[a.Ns];

    // the matrix images of vertex i for the local states present, into Bs
    auto load_B = [&](int i) {
        const int e0 = pptr[i], e1 = pptr[i + 1], msk = vmask[i];
        for (int e = e0; e < e1; ++e) {
            if (pidx[e] < 0) continue;
            for (int sg = 0; sg < 4; ++sg) {
                if (!((msk >> sg) & 1)) continue;
                const unsigned char* src = a.bimg + ((size_t)e * 4 + sg) * kImg;
                unsigned char* dst = Bs + ((size_t)(e - e0) * 4 + sg) * kImg;
                for (int q = tid; q < (int)(kImg / 16); q += kGtRows) tc::cp_async16(dst + 16 * q, src + 16 * q);
            }
        }
        tc::cp_async_commit();
    };

    for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const int64_t s = gt_find_sample(cb, a.Ns, blk);
        const int64_t jb = blk - cb[s];
        const int64_t beg = a.rows.begin ? a.rows.begin[s] : s * a.rows.stride;
        const int64_t left = a.rows.count[s] - jb * kGtRows;
        const int nr = (int)(left < kGtRows ? left : kGtRows);
        const int64_t r0 = beg + jb * kGtRows;
        const uint64_t na = a.samples[2 * s], nb = a.samples[2 * s + 1];
        if (warp == 0) build_lists_warp(na, nb, a.h.K, lists, lane);
        if (tid < K) { vmask[tid] = 0; sx[tid] = a.Hexp[s * K + tid]; }
        if (tid == 0) s_pmin = K;
        // the sample's states h_j(n), FP64 -> FP32 -> FP16 hi + lo
        for (int q = tid; q < K * D; q += kGtRows) {
            const int i = q / D, c = q - i * D;
            const float v = (float)a.Hst[(size_t)s * K * D + q];
            const __half h = __float2half_rn(v);
            __half* row = (__half*)(simg + (size_t)i * 4 * D);
            row[c] = h;
            row[D + c] = __float2half_rn(v - __half2float(h));
        }
        for (int k = tid; k < NH; k += kGtRows) {
            const double th = a.theta[(size_t)s * NH + k];
            tts[k] = (float)(a.an.corr == 1 ? tan(th) : tanh(th));
        }
        __syncthreads();
        // each thread decodes its row: the determinant m and its first changed site
        const int r = tid;
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
        // per vertex, the local states the active rows take there (a warp
        // reduction, then one shared atomic per warp)
        for (int i = 0; i < K; ++i) {
            const unsigned m = __reduce_or_sync(kFull, i >= p ? 1u << sigma_at(ma, mb, i) : 0u);
            if (lane == 0 && m) atomicOr(&vmask[i], (int)m);
        }
        {
            const unsigned pm = __reduce_min_sync(kFull, (unsigned)p);
            if (lane == 0) atomicMin(&s_pmin, (int)pm);
        }
        __syncthreads();
        const int pmin = s_pmin;
        // the states before pmin that a later vertex reads, in every row
        for (int j = 0; j < pmin; ++j) {
            if (__ldg(a.last_use + j) < pmin) continue;
            const int sl = __ldg(a.slot + j);
            put_row<D>(slots + (size_t)sl * kSlot, simg + (size_t)j * 4 * D, r);
            rx[sl][r] = sx[j];
        }
        load_B(pmin);
        float mant = 0.f;
        int mex = 0;
        for (int i = pmin; i < K; ++i) {
            tc::cp_async_wait<0>();
            tc::fence_proxy_async();            // the slot rows written by the threads, for the MMAs
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            const int e0 = pptr[i], e1 = pptr[i + 1], deg = e1 - e0, msk = vmask[i];
            bool any = false;
            for (int e = e0; e < e1; ++e) any = any || pidx[e] >= 0;
            if (any) {
                if (tid == 0) {
                    for (int e = e0; e < e1; ++e) {
                        const int j = pidx[e];
                        if (j < 0) continue;
                        const uint32_t A0 = tc::smem_addr(slots + (size_t)__ldg(a.slot + j) * kSlot);
                        for (int sg = 0; sg < 4; ++sg) {
                            if (!((msk >> sg) & 1)) continue;
                            const uint32_t B0 = tc::smem_addr(Bs + ((size_t)(e - e0) * 4 + sg) * kImg);
                            const uint32_t dcol = tmem + (uint32_t)(((e - e0) * 4 + sg) * D);
                            const uint32_t As[3] = {A0, A0 + kLo, A0};
                            const uint32_t Bv[3] = {B0, B0, B0 + 2 * D * D};
                            uint32_t acc = 0;
                            for (int term = 0; term < 3; ++term)
                                for (int ks = 0; ks < D / 16; ++ks) {
                                    tc::mma_f16(dcol, tc::desc(As[term] + ks * 256, 128, 16 * D),
                                                tc::desc(Bv[term] + ks * 256, 128, 16 * D), idesc, acc);
                                    acc = 1;
                                }
                        }
                    }
                    tc::mma_commit(&mbar);
                }
                ok = tc::mbar_wait(&mbar, phase, 1u << 24) && ok;
                phase ^= 1u;
                tc::fence_after_sync();
            }
            // the next vertex's images stream in while the rows are finished
            if (i + 1 < K) load_B(i + 1);
            const bool act = i >= p;
            const int sg = sigma_at(ma, mb, i);
            int es[kGtMaxDeg];
            int eref = -(1 << 30);
            #pragma unroll
            for (int k = 0; k < kGtMaxDeg; ++k) {
                es[k] = 0;
                if (k < deg) {
                    const int j = pidx[e0 + k];
                    es[k] = j < 0 ? 0 : rx[__ldg(a.slot + j)][r] + __ldg(a.bexp + (e0 + k) * 4 + sg);
                    eref = es[k] > eref ? es[k] : eref;
                }
            }
            float y[D];
            #pragma unroll
            for (int c = 0; c < D; ++c) y[c] = 0.f;
            if (any) {
                for (int sv = 0; sv < 4; ++sv) {          // warp-uniform: every lane loads
                    if (!((msk >> sv) & 1)) continue;
                    for (int k = 0; k < deg; ++k) {
                        if (pidx[e0 + k] < 0) continue;
                        uint32_t v[D];
                        #pragma unroll
                        for (int c0 = 0; c0 < D; c0 += 16)
                            tc::tmem_ld16(tlane + (uint32_t)((k * 4 + sv) * D + c0), v + c0);
                        tc::tmem_wait_ld();
                        if (act && sg == sv) {
                            const float f = pow2_neg(es[k] - eref);
                            #pragma unroll
                            for (int c = 0; c < D; ++c) y[c] = fmaf(__uint_as_float(v[c]), f, y[c]);
                        }
                    }
                }
            }
            if (act) {
                for (int k = 0; k < deg; ++k) {
                    if (pidx[e0 + k] >= 0) continue;
                    // M e_0: column 0 of the matrix
                    const float f = pow2_neg(-eref);
                    const float* col = a.col0 + ((size_t)(e0 + k) * 4 + sg) * D;
                    #pragma unroll
                    for (int c = 0; c < D; ++c) y[c] = fmaf(__ldg(col + c), f, y[c]);
                }
                float mx = 0.f;
                #pragma unroll
                for (int c = 0; c < D; ++c) mx = fmaxf(mx, fabsf(y[c]));
                int ge = 0;
                if (mx > 0.f) frexpf(mx, &ge);
                const bool pw = ge >= -126 && ge <= 126;
                const float sc = pw ? __int_as_float((127 - ge) << 23) : 0.f;
                #pragma unroll
                for (int c = 0; c < D; ++c) y[c] = pw ? y[c] * sc : ldexpf(y[c], -ge);
                const int ex = eref + ge;
                const int si = __ldg(a.slot + i);
                if (i == K - 1) {
                    mant = y[0];
                    mex = ex;
                } else if (si >= 0) {
                    unsigned char* sl = slots + (size_t)si * kSlot;
                    #pragma unroll
                    for (int c8 = 0; c8 < D / 8; ++c8) {
                        __align__(16) __half2 hi[4], lo[4];
                        #pragma unroll
                        for (int q = 0; q < 4; ++q)
                            tc::split_half2(y[8 * c8 + 2 * q], y[8 * c8 + 2 * q + 1], hi[q], lo[q]);
                        const uint32_t off = tc::op_offset(r, 8 * c8, D);
                        *(uint4*)(sl + off) = *(const uint4*)hi;
                        *(uint4*)(sl + kLo + off) = *(const uint4*)lo;
                    }
                    rx[si][r] = ex;
                }
            } else {
                const int si = __ldg(a.slot + i);
                if (si >= 0) {
                    put_row<D>(slots + (size_t)si * kSlot, simg + (size_t)i * 4 * D, r);
                    rx[si][r] = sx[i];
                }
            }
            tc::fence_before_sync();
        }
        // the row's term: coefficient x psi_TN ratio x correlator ratio
        double term = 0.0;
        if (r < nr) {
            float X = 0.f;                        // prod_k (1 + x_k) - 1
            if (NH > 0) {
                int fi[4];
                float fs[4];
                int nf = 0;
                uint64_t da = na ^ ma, db = nb ^ mb;
                while (da && nf < 4) {
                    const int q = __ffsll((long long)da) - 1;
                    da &= da - 1;
                    fi[nf] = 2 * q; fs[nf] = ((ma >> q) & 1ull) ? 1.f : -1.f; ++nf;
                }
                while (db && nf < 4) {
                    const int q = __ffsll((long long)db) - 1;
                    db &= db - 1;
                    fi[nf] = 2 * q + 1; fs[nf] = ((mb >> q) & 1ull) ? 1.f : -1.f; ++nf;
                }
                const bool cosf_kind = a.an.corr == 1;
                for (int k = 0; k < NH; ++k) {
                    float d = 0.f;
                    #pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (q < nf) d = fmaf(fs[q], WTs[fi[q] * NP + k], d);
                    float x;
                    if (!cosf_kind) {
                        float ch1, sh;
                        if (fabsf(d) <= 1.f) {
                            cosh_sinh_small(d, ch1, sh);
                        } else {
                            const float em = expm1f(d), inv = 1.f / (1.f + em);
                            ch1 = 0.5f * em * em * inv;
                            sh = 0.5f * em * (1.f + inv);
                        }
                        x = fmaf(tts[k], sh, ch1);
                    } else {
                        float c1, sn;
                        if (fabsf(d) <= 1.f) {
                            cos_sin_small(d, c1, sn);
                        } else {
                            const float h = sinf(0.5f * d);
                            c1 = -2.f * h * h;
                            sn = sinf(d);
                        }
                        x = fmaf(-tts[k], sn, c1);
                    }
                    X = fmaf(X, x, X + x);
                }
            }
            const double tn = ldexp((double)mant / a.psi_mant[s], mex - a.psi_exp[s]);
            term = coef * tn * (1.0 + (double)X);
        }
        double ab = fabs(term);
        long long sp = r < nr ? (long long)(K - p) : 0;
        long long mv = r < nr ? (long long)graph_matvecs(a.an, p) : 0;
        for (int o = 16; o; o >>= 1) {
            term += __shfl_xor_sync(kFull, term, o);
            ab += __shfl_xor_sync(kFull, ab, o);
            sp += __shfl_xor_sync(kFull, sp, o);
            mv += __shfl_xor_sync(kFull, mv, o);
        }
        if (lane == 0) { wsum[warp] = term; wabs[warp] = ab; wspan[warp] = sp; wmv[warp] = mv; }
        __syncthreads();
        if (tid == 0) {
            double t = 0.0, ta = 0.0;
            long long st = 0, sm = 0;
            for (int w = 0; w < kGtRows / 32; ++w) {
                t += wsum[w]; ta += wabs[w]; st += wspan[w]; sm += wmv[w];
            }
            a.partial[blk] = t;
            if (a.partial_abs) a.partial_abs[blk] = ta;
            if (a.span) a.span[blk] = st;
            if (a.mv) a.mv[blk] = sm;
        }
        __syncthreads();
    }
    tc::cp_async_wait<0>();
    if (!ok && tid == 0) report(a.err, 5, 6, (long long)blockIdx.x);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, a.tmem_cols);
}

}  // namespace

size_t graph_tiles_smem(int D, int K, int n_slots, int max_deg, int n_hidden)
{
    const size_t np = (size_t)((n_hidden + 3) & ~3);
    return (size_t)n_slots * kGtRows * D * 4 + (size_t)max_deg * 16 * D * D + (size_t)K * 4 * D +
           (size_t)2 * K * np * 4 + (size_t)n_hidden * 4;
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
    if (mx > 0 && graph_tiles_smem(D, K, p.n_slots, max_deg, n_hidden) + 16384 > (size_t)mx) {
        *why = "the tile's states and matrix images exceed the shared memory";
        return false;
    }
    // split images of every M_e^sigma scaled by 2^-x (max |M| 2^-x in [0.5, 1)):
    // B[n][k] = M[n][k] in the K-major core-matrix layout, hi then lo; column 0
    // in FP32 for the e_0 sources
    const int E = ptr[K];
    const size_t img = (size_t)4 * D * D;
    p.img.assign((size_t)E * 4 * img, 0);
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
            unsigned char* hi = p.img.data() + id * img;
            unsigned char* lo = hi + (size_t)2 * D * D;
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

int launch_graph_tiles(const GraphTcArgs& a, int n_sm, cudaStream_t st)
{
    if (a.rows.max_chunks == 0) return 0;
    size_t smem = graph_tiles_smem(a.an.D, a.an.K, a.n_slots, a.max_deg, a.an.n_hidden);
    // one CTA per multiprocessor: each holds all the tensor-memory columns it
    // allocates for the whole persistent loop
    smem = std::max<size_t>(smem, 120 * 1024);
    const int64_t grid = std::min<int64_t>(n_sm, a.rows.max_chunks);
    switch (a.an.D) {
    case 16:
        allow_max_smem(k_graph_tiles<16>);
        k_graph_tiles<16><<<(unsigned)grid, kGtRows, smem, st>>>(a);
        break;
    case 32:
        allow_max_smem(k_graph_tiles<32>);
        k_graph_tiles<32><<<(unsigned)grid, kGtRows, smem, st>>>(a);
        break;
    default:
        allow_max_smem(k_graph_tiles<64>);
        k_graph_tiles<64><<<(unsigned)grid, kGtRows, smem, st>>>(a);
        break;
    }
    return 1;
}

}  // namespace nqs
