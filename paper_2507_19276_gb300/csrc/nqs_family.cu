// nqs_family.cu -- shared-prefix evaluation of the connected amplitudes of a
// chain tensor network (Eq. MPS-RNN-1D with v = 0) times the RBM correlator.
//
// For a sample n and a connected m that changes the local states of the sorted
// sites s1 < s2 (< s3 (< s4)), psi_TN(m) = r^T A_{K-1} ... A_0 l with the
// changed sites' matrices replaced. The product is re-associated so that the
// partial products shared by the many m of one n are formed once:
//   one-change left families  G_{s,a}(t) = A_t ... A_{s+1} A_s^{a} L_{s-1}, t >= s
//   one-change right families H_{s,a}(t) = R_{s+1} A_s^{a} A_{s-1} ... A_t,  t <= s
//   two-change left clusters  TL_{s1a1,s2a2}(t) = A_t ... A_{s2+1} A_{s2}^{a2} G_{s1,a1}(s2-1)
//   two-change right clusters TR_{sAaA,sBaB} = H_{sB,aB}(sA+1) A_{sA}^{aA}
// where A_t = A_t^{sigma_t(n)} and A_s^{a} is the a-th local state other than
// sigma_s(n) (ascending). Then
//   2 sites: psi_TN(m) = G_{s1,a1}(s2-1) . H_{s2,a2}(s2)
//   3 sites: psi_TN(m) = G_{s1,a1}(s2-1) . TR_{s2a2,s3a3}
//   4 sites: psi_TN(m) = TL_{s1a1,s2a2}(s3-1) . TR_{s3a3,s4a4}
// The correlator ratio (Eq. RBM) splits the same way: with theta_k(n), the
// left part's spin-orbital flips dL and the right part's dR,
//   f(m)/f(n) = prod_k cosh(theta_k + dL_k + dR_k) / cosh(theta_k)
//             = PL * PR * prod_k (1 + tanh(theta_k + dL_k) tanh(dR_k)),
//   PL = prod_k cosh(theta_k + dL_k) / cosh(theta_k),  PR = prod_k cosh(dR_k)
// (cosh(x + y) = cosh x cosh y (1 + tanh x tanh y)), so every left object
// stores tanh(theta + dL) and PL - 1, every right object tanh(dR) and PR - 1:
// a row reads one value per hidden unit from each side. Every vector carries a
// power-of-two exponent; T is the arithmetic type of the contractions.
#include "nqs_family.cuh"
#include "nqs_tc.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

namespace nqs {

// alternative index of local state `sg` at a site whose own state is `own`
__device__ __forceinline__ int alt_of(int sg, int own) { return sg - (sg > own ? 1 : 0); }
__device__ __forceinline__ int sig_of_alt(int a, int own) { return a + (a >= own ? 1 : 0); }

template <typename T>
__device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }

template <typename T> struct Vec4;
template <> struct Vec4<float> { typedef float4 type; };
template <> struct Vec4<double> { typedef double4_32a type; };

// Block-wide: y_i = M x_i for nv vectors in shared memory; MT[b][a] = M[a][b].
// Each thread owns two outputs (a, a + D/2) of four vectors.
template <typename T>
__device__ void mv_block(const T* __restrict__ MT, int D, const T* X, T* Y, int nv)
{
    if ((D & 3) != 0 || D < 4) {
        const int a = threadIdx.x % D, g = threadIdx.x / D, G = blockDim.x / D;
        if (g >= G) return;
        for (int i = g; i < nv; i += G) {
            T acc = T(0);
            for (int b = 0; b < D; ++b) acc = fma(__ldg(MT + (size_t)b * D + a), X[(size_t)i * D + b], acc);
            Y[(size_t)i * D + a] = acc;
        }
        return;
    }
    typedef typename Vec4<T>::type V4;
    const int H = D >> 1;
    const int a = threadIdx.x % H, g = threadIdx.x / H, G = blockDim.x / H;
    if (g >= G) return;
    for (int i = g * 4; i < nv; i += G * 4) {
        const int n4 = nv - i < 4 ? nv - i : 4;
        T acc0[4] = {T(0), T(0), T(0), T(0)}, acc1[4] = {T(0), T(0), T(0), T(0)};
        for (int b = 0; b < D; b += 4) {
            T m0[4], m1[4];
            #pragma unroll
            for (int u = 0; u < 4; ++u) {
                m0[u] = __ldg(MT + (size_t)(b + u) * D + a);
                m1[u] = __ldg(MT + (size_t)(b + u) * D + a + H);
            }
            #pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (q < n4) {
                    const V4 x = *(const V4*)(X + (size_t)(i + q) * D + b);
                    acc0[q] = fma(m0[0], x.x, acc0[q]); acc1[q] = fma(m1[0], x.x, acc1[q]);
                    acc0[q] = fma(m0[1], x.y, acc0[q]); acc1[q] = fma(m1[1], x.y, acc1[q]);
                    acc0[q] = fma(m0[2], x.z, acc0[q]); acc1[q] = fma(m1[2], x.z, acc1[q]);
                    acc0[q] = fma(m0[3], x.w, acc0[q]); acc1[q] = fma(m1[3], x.w, acc1[q]);
                }
            }
        }
        for (int q = 0; q < n4; ++q) {
            Y[(size_t)(i + q) * D + a] = acc0[q];
            Y[(size_t)(i + q) * D + a + H] = acc1[q];
        }
    }
}

// Block-wide y_i = M x_i as mv_block, in double-FP32 arithmetic: M as (hi, lo)
// float pairs (MT[b][a] = M[a][b]), x_i split into float halves Xh + Xl, one
// output per thread and pass accumulated as an unnormalised pair (the
// error-free product by FMA and Knuth's two-sum, as in the double-double
// algorithms of Hida, Li and Bailey; relative error about D 2^-48).
__device__ void mv_block_df(const float2* __restrict__ MT, int D, const float* Xh, const float* Xl,
                            double* Y, int nv)
{
    const int G = (int)blockDim.x >= D ? (int)blockDim.x / D : 1;
    for (int q = threadIdx.x; q < G * D; q += blockDim.x) {
        const int a = q % D, g = q / D;
        for (int i = g; i < nv; i += G) {
            float hi = 0.f, lo = 0.f;
            const float* xh = Xh + (size_t)i * D;
            const float* xl = Xl + (size_t)i * D;
            for (int b = 0; b < D; ++b) {
                const float2 m = __ldg(MT + (size_t)b * D + a);
                const float p = m.x * xh[b];
                const float pe = fmaf(m.x, xh[b], -p) + fmaf(m.x, xl[b], m.y * xh[b]);
                const float u = hi + p, z = u - hi;
                lo += ((hi - (u - z)) + (p - z)) + pe;
                hi = u;
            }
            Y[(size_t)i * D + a] = (double)hi + (double)lo;
        }
    }
}

// Rescale each of nv vectors (length D) in shared memory to max|v| in [0.5, 1);
// exponent increments go to ex[i]. One warp per vector.
template <typename T>
__device__ void renorm_rows(T* Y, int D, int nv, int* ex)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < nv; i += nw) {
        T* y = Y + (size_t)i * D;
        T m = T(0);
        for (int c = lane; c < D; c += 32) m = fmax(m, tabs(y[c]));
        for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
        int e = 0;
        if (m > T(0)) frexp(m, &e);
        for (int c = lane; c < D; c += 32) y[c] = ldexp(y[c], -e);
        if (lane == 0) ex[i] = e;
    }
}

// Cluster keys: TL sorted by (s2, a2, s1, a1), TR by (sA, aA, sB, aB), so that the
// clusters created with one matrix form contiguous runs.
__device__ __forceinline__ int tl_key(int K, int s1, int a1, int s2, int a2)
{
    return ((s2 * 3 + a2) * K + s1) * 3 + a1;
}

__device__ __forceinline__ int tr_key(int K, int sA, int aA, int sB, int aB)
{
    return ((sA * 3 + aA) * K + sB) * 3 + aB;
}

// ---------------------------------------------------------------------------
// Batches of block-wide matrix-vector products y_i = M x_i: x_i gathered from
// global memory, y_i rescaled by a power of two and scattered back. M is
// A_t^{sg} (side 0, column convention) or its transpose (side 1, row vectors).
//  - FP32 with tensor-core images: tcgen05 MMAs, M = 128 rows, N = D,
//    operands split into FP16 hi + lo (x_hi M_hi + x_lo M_hi + x_hi M_lo),
//    FP32 accumulation in tensor memory (tc_apply);
//  - otherwise: shared-memory CUDA-core products (mv_block).
// ---------------------------------------------------------------------------

template <typename T>
struct BatchSmem {
    T* X; T* Y;                        // CUDA-core path: [nmax][D] each
    unsigned char* Ah; unsigned char* Al; unsigned char* Bh;   // tensor path operands
    float* rmax;                       // [2][128]
    uint64_t* mbar;
    uint32_t tmem;
    uint32_t phase;
    int cur_mat;
};

template <typename T>
__device__ __forceinline__ bool use_tc(const FamArgs<T>& f)
{
    return std::is_same<T, float>::value && f.tc;
}

// One tensor-core batch (T = float) of n <= 128 rows through the matrix image
// `mat`: y_r = M x_r with x_r = acc.src(r), y_r rescaled by a power of two and
// written to acc.dst(r), acc.set_exp(r, e) receiving the exponent added (the
// row's power of two plus the image's). Row sources and destinations come
// from the accessor; results per row do not depend on the other rows of the
// tile. The scaled rows leave through shared memory (see the epilogue).
template <class Acc>
__device__ void tc_apply(const FamArgs<float>& f, BatchSmem<float>& sm, const Acc& acc, int n, int mat)
{
    const int D = f.D;
    // The reduction runs over D / KC chunks of KC columns (one chunk up to
    // D = 128): per chunk the batch rows' columns are gathered and split
    // into FP16 hi / lo, the matrix image's chunk is staged, and the MMAs
    // accumulate into the same tensor-memory columns.
    const int KC = fam_tc_kc(D), nck = D / KC;
    const int cpr = KC >> 3;                      // 8-element units per row of a chunk
    const int nun = n * cpr;
    bool ok = true;
    for (int ck = 0; ck < nck; ++ck) {
        // gather: each thread takes up to 2 units per round and issues all
        // their loads before splitting any (latency-bound otherwise)
        for (int u0 = 0; u0 < nun; u0 += 2 * blockDim.x) {
            float4 v4[2][2];
            #pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int u = u0 + k * blockDim.x + threadIdx.x;
                if (u < nun) {
                    const int r = u / cpr, c = u - r * cpr;
                    const float4* p = (const float4*)(acc.src(r) + ck * KC + 8 * c);
                    v4[k][0] = p[0];
                    v4[k][1] = p[1];
                }
            }
            #pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int u = u0 + k * blockDim.x + threadIdx.x;
                if (u < nun) {
                    const int r = u / cpr, c = u - r * cpr;
                    const float xs[8] = {v4[k][0].x, v4[k][0].y, v4[k][0].z, v4[k][0].w,
                                         v4[k][1].x, v4[k][1].y, v4[k][1].z, v4[k][1].w};
                    __align__(16) __half hi[8], lo[8];
                    #pragma unroll
                    for (int j = 0; j < 8; ++j) tc::split_half(xs[j], hi[j], lo[j]);
                    const uint32_t off = tc::op_offset(r, 8 * c, KC);
                    *(uint4*)(sm.Ah + off) = *(const uint4*)hi;
                    *(uint4*)(sm.Al + off) = *(const uint4*)lo;
                }
            }
        }
        // the image chunk (kept across batches when one chunk holds the matrix)
        if (nck > 1 || mat != sm.cur_mat) {
            const int nimg = 4 * D * KC / 16;
            const uint4* __restrict__ g = f.tc_mats + (size_t)mat * (4 * D * D / 16) + (size_t)ck * nimg;
            uint4* d = (uint4*)sm.Bh;
            for (int i0 = 0; i0 < nimg; i0 += 4 * blockDim.x) {
                uint4 w[4];
                #pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int i = i0 + k * blockDim.x + threadIdx.x;
                    if (i < nimg) w[k] = __ldg(g + i);
                }
                #pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int i = i0 + k * blockDim.x + threadIdx.x;
                    if (i < nimg) d[i] = w[k];
                }
            }
            sm.cur_mat = nck > 1 ? -1 : mat;
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (threadIdx.x == 0) {
            tc::fence_after_sync();
            const uint32_t idesc = tc::idesc_f16(128, D);
            const uint32_t lbo = 128, sbo = 16 * KC;
            const unsigned char* Bl = sm.Bh + 2 * D * KC;
            const unsigned char* As[3] = {sm.Ah, sm.Al, sm.Ah};
            const unsigned char* Bs[3] = {sm.Bh, sm.Bh, Bl};
            uint32_t acc = ck > 0 ? 1u : 0u;
            for (int term = 0; term < 3; ++term)
                for (int ks = 0; ks < KC / 16; ++ks) {
                    tc::mma_f16(sm.tmem, tc::desc(tc::smem_addr(As[term]) + ks * 256, lbo, sbo),
                                tc::desc(tc::smem_addr(Bs[term]) + ks * 256, lbo, sbo), idesc, acc);
                    acc = 1;
                }
            tc::mma_commit(sm.mbar);
        }
        // the chunk's operands may be overwritten once its MMAs are done (one
        // warp polls the mbarrier, the others wait at the barrier)
        if (threadIdx.x < 32) ok = tc::mbar_wait(sm.mbar, sm.phase, 1u << 24) && ok;
        sm.phase ^= 1u;
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    if (!ok && threadIdx.x == 0) report(f.err, 5, 4, (long long)f.s0);
    // tensor memory -> registers, twice (row maximum, then the scaled row), 8
    // columns at a time so that nothing indexed by D lives in local memory.
    // Warp w reads lanes 32 (w % 4) .. +31 and half (w / 4) of the columns.
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp & 3, h = warp >> 2, half = D >> 1;
    const int r = 32 * q + lane;
    const uint32_t trow = sm.tmem + ((uint32_t)(32 * q) << 16) + h * half;
    if (warp < 8) {
        float m = 0.f;
        for (int c0 = 0; c0 < half; c0 += 8) {
            float v[8];
            tc::tmem_ld8(trow + c0, v);
            tc::tmem_wait_ld();
            #pragma unroll
            for (int j = 0; j < 8; ++j) m = fmaxf(m, fabsf(v[j]));
        }
        sm.rmax[h * 128 + r] = m;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    // the scaled rows leave through shared memory in column slices of up to 64
    // (row stride 272 bytes: 8 consecutive rows fill the 32 banks), copied out
    // row by row so that a warp's stores fill whole lines. The slice buffer
    // overlays the operands (free now that the MMAs completed); for D > 128 it
    // reaches into the matrix image, which is reloaded per chunk there anyway.
    constexpr int kSRS = 272;
    float mm = 0.f;
    int e = 0;
    if (warp < 8) {
        mm = fmaxf(sm.rmax[r], sm.rmax[128 + r]);
        if (mm > 0.f) frexpf(mm, &e);
        if (h == 0 && r < n) acc.set_exp(r, e + f.tc_exp[mat]);
    }
    const bool pw = e >= -126 && e <= 126;
    const float sc2 = pw ? __int_as_float((127 - e) << 23) : 0.f;
    unsigned char* slice = sm.Ah;
    for (int cs = 0; cs < D; cs += 64) {
        const int sw = D - cs < 64 ? D - cs : 64, hw = sw >> 1;
        if (warp < 8) {
            float* o = (float*)(slice + r * kSRS) + h * hw;
            const uint32_t tr = sm.tmem + ((uint32_t)(32 * q) << 16) + cs + h * hw;
            for (int c0 = 0; c0 < hw; c0 += 8) {
                float v[8];
                tc::tmem_ld8(tr + c0, v);   // every lane of the warp takes part
                tc::tmem_wait_ld();
                #pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = pw ? v[j] * sc2 : ldexpf(v[j], -e);
                *(float4*)(o + c0) = make_float4(v[0], v[1], v[2], v[3]);
                *(float4*)(o + c0 + 4) = make_float4(v[4], v[5], v[6], v[7]);
            }
        }
        __syncthreads();
        const int qpr = sw >> 2;                  // 16-byte pieces per row of the slice
        for (int v = threadIdx.x; v < n * qpr; v += blockDim.x) {
            const int rr = v / qpr, qq = v - rr * qpr;
            *(float4*)(acc.dst(rr) + cs + 4 * qq) = *(const float4*)(slice + rr * kSRS + qq * 16);
        }
        __syncthreads();
    }
    if (128 * kSRS > 4 * 128 * KC) sm.cur_mat = -1;   // the slice reached into the image
    tc::fence_before_sync();
    __syncthreads();
}

template <typename T>
__device__ void batch_init(const FamArgs<T>& f, BatchSmem<T>& sm, unsigned char* base, uint32_t* tmem_slot,
                           uint64_t* mbar)
{
    const int D = f.D;
    if (!use_tc(f)) {
        sm.X = (T*)base;
        sm.Y = sm.X + (size_t)f.nmax * D;
        return;
    }
    unsigned char* p = base;
    const size_t kc = (size_t)fam_tc_kc(D);
    sm.Ah = p; p += (size_t)128 * kc * 2;
    sm.Al = p; p += (size_t)128 * kc * 2;
    sm.Bh = p; p += (size_t)4 * D * kc;
    sm.rmax = (float*)p;
    sm.mbar = mbar;
    sm.cur_mat = -1;
    sm.phase = 0;
    if ((threadIdx.x >> 5) == 0) { tc::tmem_alloc(tmem_slot, f.tc_cols); tc::tmem_relinquish(); }
    if (threadIdx.x == 0) tc::mbar_init(mbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    sm.tmem = *tmem_slot;
}

template <typename T>
__device__ void batch_fini(const FamArgs<T>& f, BatchSmem<T>& sm)
{
    if (!use_tc(f)) return;
    tc::fence_before_sync();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(sm.tmem, f.tc_cols);
}

// fields of a key: first site, its alternative, second site, its alternative
template <typename T>
__device__ __forceinline__ void key_fields(const FamArgs<T>& f, int key, int& site_hi, int& alt_hi,
                                           int& site_lo, int& alt_lo)
{
    // key = ((site_hi * 3 + alt_hi) * K + site_lo) * 3 + alt_lo, key < 9 K^2 <= 36864
    const uint32_t k = (uint32_t)key;
    const uint32_t q9 = fdiv(k, f.div9K), r9 = k - q9 * f.div9K.d;
    const uint32_t q3 = fdiv(r9, f.div3K), r3 = r9 - q3 * f.div3K.d;
    site_hi = (int)q9;
    alt_hi = (int)q3;
    site_lo = (int)(r3 / 3u);
    alt_lo = (int)(r3 - 3u * (r3 / 3u));
}

// padded correlator-factor row lengths (multiples of 4 elements)
__device__ __forceinline__ int nh_pad(int NH) { return (NH + 3) & ~3; }

// ---------------------------------------------------------------------------
// Row decomposition (shared by the marking and the evaluation passes)
// ---------------------------------------------------------------------------

struct RowParts {
    int nsite;           // 2, 3 or 4 changed sites
    int s[4], a[4];      // sites ascending and alternative indices
    int last;            // the last changed site
    uint64_t ma, mb;
};

__device__ __forceinline__ RowParts row_parts(const HamView& h, const OrbLists& L, uint64_t na,
                                              uint64_t nb, uint32_t rank)
{
    const Exc e = decode_rank<false>(h, L, rank);     // sites only: the phase is in the row's coefficient
    RowParts r;
    uint64_t ma = na, mb = nb;
    flip(ma, mb, e.i); flip(ma, mb, e.a);
    if (e.kind == 2) { flip(ma, mb, e.j); flip(ma, mb, e.b); }
    uint64_t ch = (na ^ ma) | (nb ^ mb);
    r.nsite = 0;
    r.last = 0;
    #pragma unroll
    for (int q = 0; q < 4; ++q) {          // static indices: the parts stay in registers
        r.s[q] = 0; r.a[q] = 0;
        if (ch) {
            const int p = __ffsll((long long)ch) - 1;
            r.s[q] = p;
            r.a[q] = alt_of(sigma_at(ma, mb, p), sigma_at(na, nb, p));
            r.nsite = q + 1;
            r.last = p;
            ch &= ch - 1;
        }
    }
    r.ma = ma;
    r.mb = mb;
    return r;
}

// Site word of a row: its changed sites in ascending order, 6 bits each at
// bits 0, 6, 12, 18 (a 2- or 3-site change repeats its last site), and at bits
// 24 + 2q the index of site q's new local state among the three states other
// than n's. The marking pass replaces the deterministic rows' ranks by these
// words, so that the row kernel reads the parts instead of decoding them.
__device__ __forceinline__ uint32_t site_word(const RowParts& p)
{
    uint32_t w = 0;
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int qq = q < p.nsite ? q : p.nsite - 1;
        w |= ((uint32_t)p.s[qq] << (6 * q)) | ((uint32_t)(q < p.nsite ? p.a[q] : 0) << (24 + 2 * q));
    }
    return w;
}

// the parts of row `idx` of a row set: from its site word, or by decoding its
// canonical rank
__device__ __forceinline__ RowParts row_parts_of(const HamView& h, const OrbLists& L, uint64_t na,
                                                 uint64_t nb, const RowSet& rows, int64_t idx)
{
    if (!rows.sites) return row_parts(h, L, na, nb, rows.rank[idx]);
    const uint32_t x = rows.rank[idx];
    RowParts r;
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
        r.s[q] = (int)((x >> (6 * q)) & 63u);
        r.a[q] = (int)((x >> (24 + 2 * q)) & 3u);
    }
    r.nsite = 2 + (r.s[2] != r.s[1] ? 1 : 0) + (r.s[3] != r.s[2] ? 1 : 0);
    r.last = r.s[3];
    r.ma = r.mb = 0;
    return r;
}

// F2: mark the clusters the rows need (TL end site, TR use)
template <typename T>
__global__ void k_fam_mark(FamArgs<T> f, RowSet rows, uint32_t* words)
{
    __shared__ OrbLists lists;
    const int b = blockIdx.y;
    const int64_t s = f.s0 + b;
    const int64_t beg = rows.begin ? rows.begin[s] : s * rows.stride;
    const int64_t cnt = rows.count[s];
    const uint64_t na = f.samples[2 * s], nb = f.samples[2 * s + 1];
    if (threadIdx.x < 32 && !rows.sites) build_lists_warp(na, nb, f.h.K, lists, threadIdx.x);
    __syncthreads();
    const int K = f.K;
    const size_t nk = (size_t)K * K * 9;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < cnt;
         r += (int64_t)gridDim.x * blockDim.x) {
        const RowParts p = row_parts_of(f.h, lists, na, nb, rows, beg + r);
        if (words) words[beg + r] = site_word(p);      // in place of the rank just read
        if (p.nsite == 3) {
            f.tr_idx[(size_t)b * nk + tr_key(K, p.s[1], p.a[1], p.s[2], p.a[2])] = 1;
        } else if (p.nsite == 4) {
            atomicMax(&f.tl_end[(size_t)b * nk + tl_key(K, p.s[0], p.a[0], p.s[1], p.a[1])], p.s[2] - 1);
            f.tr_idx[(size_t)b * nk + tr_key(K, p.s[2], p.a[2], p.s[3], p.a[3])] = 1;
        }
    }
}

// Block-wide exclusive scan of one int per thread; returns the total.
__device__ int block_excl_scan(int v, int* ex, int* wt)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) { const int u = __shfl_up_sync(kFull, x, o); if (lane >= o) x += u; }
    if (lane == 31) wt[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? wt[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) { const int u = __shfl_up_sync(kFull, w, o); if (lane >= o) w += u; }
        if (lane < nw) wt[lane] = w;
    }
    __syncthreads();
    *ex = x - v + (warp ? wt[warp - 1] : 0);
    const int tot = wt[nw - 1];
    __syncthreads();
    return tot;
}

// F3: per-sample compaction of the marks, keys in ascending order:
//   tl_idx[key] = entry offset of (cluster, t = s2) in the packed TL table,
//   tl_ci[key]  = cluster index (TL list position), tl_list[ci] = key,
//   tr_idx[key] = TR row index, tr_list[row] = key; -1 where unused.
template <typename T>
__global__ void __launch_bounds__(1024, 2) k_fam_compact(FamArgs<T> f)
{
    __shared__ int wt[32];
    const int b = blockIdx.x, K = f.K;
    const size_t nk = (size_t)K * K * 9;
    const int* te = f.tl_end + (size_t)b * nk;
    int* tl = f.tl_idx + (size_t)b * nk;
    int* tci = f.tl_ci + (size_t)b * nk;
    int* tr = f.tr_idx + (size_t)b * nk;
    int* tll = f.tl_list + (size_t)b * nk;
    int* trl = f.tr_list + (size_t)b * nk;
    int carry_e = 0, carry_c = 0, carry_r = 0;
    // two consecutive keys per thread and pass: local prefixes, then one
    // block scan of the thread totals per quantity
    constexpr int Q = 2;
    for (size_t k0 = 0; k0 < nk; k0 += (size_t)Q * blockDim.x) {
        const size_t kb = k0 + (size_t)Q * threadIdx.x;
        int end[Q], flag[Q], ce = 0, cc = 0, cr = 0;
        #pragma unroll
        for (int j = 0; j < Q; ++j) {
            const size_t k = kb + j;
            end[j] = -1; flag[j] = 0;
            if (k < nk) { end[j] = te[k]; flag[j] = tr[k]; }
            const int s2 = (int)(k / (9 * (size_t)K));
            ce += end[j] >= 0 ? end[j] - s2 + 1 : 0;
            cc += end[j] >= 0 ? 1 : 0;
            cr += flag[j] > 0 ? 1 : 0;
        }
        int xe, xc, xr;
        const int te_tot = block_excl_scan(ce, &xe, wt);
        const int tc_tot = block_excl_scan(cc, &xc, wt);
        const int tr_tot = block_excl_scan(cr, &xr, wt);
        int pe = carry_e + xe, pc = carry_c + xc, pr = carry_r + xr;
        #pragma unroll
        for (int j = 0; j < Q; ++j) {
            const size_t k = kb + j;
            if (k >= nk) break;
            const int s2 = (int)(k / (9 * (size_t)K));
            tl[k] = end[j] >= 0 ? pe : -1;
            tci[k] = end[j] >= 0 ? pc : -1;
            if (end[j] >= 0) { tll[pc] = (int)k; pe += end[j] - s2 + 1; ++pc; }
            tr[k] = flag[j] > 0 ? pr : -1;
            if (flag[j] > 0) { trl[pr] = (int)k; ++pr; }
        }
        carry_e += te_tot;
        carry_c += tc_tot;
        carry_r += tr_tot;
    }
    if (threadIdx.x == 0) {
        f.tl_total[b] = carry_e;
        f.tl_count[b] = carry_c;
        f.tr_total[b] = carry_r;
    }
}

// ---------------------------------------------------------------------------
// F4c: correlator factors of the left and right objects of a sample.
//   left  objects: G families (s, a) [3K] then TL clusters [tl_count]
//   right objects: H families (s, a) [3K] then TR rows [tr_total]
// left:  tanh(theta_k + dL_k) for k < N_h, then PL - 1 at index NP
// right: tanh(dR_k) for k < N_h, then PR - 1 at index NP
// (NP = N_h rounded up to 4, zero padding in between; rows of rbm_row_len
// elements, a multiple of 32, so that every row starts on a 128-byte line)
// ---------------------------------------------------------------------------

// A correlator factor evaluated directly from theta + d: the rare units whose
// addition-formula denominator is below 1/2 (out of line, so that the common
// path keeps few registers)
__device__ __noinline__ void rbm_direct(bool left, float th, float t, float d, float& val, float& y)
{
    const float em = expm1f(d);
    const float inv = 1.f / (1.f + em);
    const float ch1 = 0.5f * em * em * inv, sh = 0.5f * em * (1.f + inv);
    val = left ? tanhf(th + d) : sh / (1.f + ch1);
    y = left ? ch1 + t * sh : ch1;
}
__device__ __noinline__ void rbm_direct(bool left, double th, double t, double d, double& val, double& y)
{
    const double em = expm1(d);
    const double inv = 1.0 / (1.0 + em);
    const double ch1 = 0.5 * em * em * inv, sh = 0.5 * em * (1.0 + inv);
    val = left ? tanh(th + d) : sh / (1.0 + ch1);
    y = left ? ch1 + t * sh : ch1;
}

__device__ __forceinline__ float div_fast(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double div_fast(double a, double b) { return a / b; }
__device__ __forceinline__ const float4* site_table(const FamArgs<float>& f) { return f.csite; }
__device__ __forceinline__ const double4_32a* site_table(const FamArgs<double>& f) { return f.csite64; }

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2) k_fam_rbm(FamArgs<T> f)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    T* th_s = (T*)smraw;               // theta_k(n)
    T* tt_s = th_s + f.n_hidden;       // tanh theta_k(n)
    const int b = blockIdx.y, K = f.K, NH = f.n_hidden, NP = nh_pad(NH);
    const int64_t s = f.s0 + b;
    const uint64_t na = f.samples[2 * s], nb = f.samples[2 * s + 1];
    for (int k = threadIdx.x; k < NH; k += blockDim.x) {
        th_s[k] = (T)f.theta[s * NH + k];
        tt_s[k] = (T)tanh(f.theta[s * NH + k]);
    }
    __syncthreads();
    const size_t nk = (size_t)K * K * 9;
    const int nleft = 3 * K + f.tl_count[b], nright = 3 * K + f.tr_total[b];
    const int64_t lbase = f.rbl_base[b], rbase = f.rbr_base[b];
    const int nobj = nleft + nright;
    // two objects per warp, one per half-warp (16 lanes over the hidden units)
    const int lane = threadIdx.x & 31, hl = lane & 15;
    for (int ob = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 2; ob < nobj;
         ob += gridDim.x * (blockDim.x >> 5) * 2) {
        const int o = ob + (lane >> 4);
        const bool valid = o < nobj;
        const bool left = o < nleft;
        const int oi = left ? o : o - nleft;
        // the object's changed sites (one for a family, two for a cluster)
        int ns = 0, s_hi = 0, a_hi = 0, s_lo = 0, a_lo = 0;
        if (!valid) {
        } else if (oi < 3 * K) {
            ns = 1; s_hi = oi / 3; a_hi = oi % 3;
        } else {
            const int key = left ? f.tl_list[(size_t)b * nk + (oi - 3 * K)]
                                 : f.tr_list[(size_t)b * nk + (oi - 3 * K)];
            key_fields(f, key, s_hi, a_hi, s_lo, a_lo);
            ns = 2;
        }
        // products of (1 + y_k) are carried as P - 1 (X <- X + y + X y), exact
        // for P near 1 and free of a logarithm per unit
        const int RL = rbm_row_len(NH);
        T* out = (left ? f.rbl + (size_t)(lbase + oi) * RL : f.rbr + (size_t)(rbase + oi) * RL);
        T pm1 = T(0);
        // The object's change of theta is the sum of its sites' changes d1 (+ d2),
        // whose tanh u and cosh - 1 c come from the per-site table (FP32 or FP64
        // as T). With t = tanh theta, s = u1 + u2, p = u1 u2 (0 for one site):
        //   cosh(theta + d1 + d2) / (cosh theta cosh d1 cosh d2) = 1 + p + t s =: den
        //   tanh(theta + d1 + d2) = (t + s + t p) / den,  tanh(d1 + d2) = s / (1 + p)
        //   PL factor - 1 = (1 + e)(1 + p + t s) - 1,  PR factor - 1 = (1 + e)(1 + p) - 1
        // with e = (1 + c1)(1 + c2) - 1. A denominator below 1/2 (|theta| and
        // |d| both large) would lose bits to cancellation: such units take tanh
        // and expm1 of theta + d directly. One loop per kind of object (left /
        // right, one / two sites), each with only its own arithmetic.
        typedef typename Vec4<T>::type V4;
        const V4* tab = site_table(f);
        const V4* r1 = tab + ((size_t)(s_hi * 4 + sigma_at(na, nb, s_hi)) * 3 + a_hi) * NP;
        const V4* r2 = tab + ((size_t)(s_lo * 4 + sigma_at(na, nb, s_lo)) * 3 + a_lo) * NP;
        if (!valid) {
        } else if (left && ns == 2) {
            for (int k = hl; k < NH; k += 16) {
                const V4 u = r1[k], v = r2[k];
                const T t = tt_s[k];
                const T sx = u.x + v.x, px = u.x * v.x;
                const T e = fma(u.y, v.y, u.y + v.y);
                const T den = fma(t, sx, T(1) + px);
                T val, y;
                if (den >= T(0.5)) {
                    const T g = fma(t, sx, px);
                    val = div_fast(fma(t, px, t + sx), den);
                    y = fma(e, g, e + g);
                } else {
                    rbm_direct(true, th_s[k], t, u.z + v.z, val, y);
                }
                out[k] = val;
                pm1 = fma(pm1, y, pm1 + y);
            }
        } else if (left) {
            for (int k = hl; k < NH; k += 16) {
                const V4 u = r1[k];
                const T t = tt_s[k];
                const T den = fma(t, u.x, T(1));
                T val, y;
                if (den >= T(0.5)) {
                    const T g = t * u.x;
                    val = div_fast(t + u.x, den);
                    y = fma(u.y, g, u.y + g);
                } else {
                    rbm_direct(true, th_s[k], t, u.z, val, y);
                }
                out[k] = val;
                pm1 = fma(pm1, y, pm1 + y);
            }
        } else if (ns == 2) {
            for (int k = hl; k < NH; k += 16) {
                const V4 u = r1[k], v = r2[k];
                const T sx = u.x + v.x, px = u.x * v.x;
                const T e = fma(u.y, v.y, u.y + v.y);
                const T den = T(1) + px;
                T val, y;
                if (den >= T(0.5)) {
                    val = div_fast(sx, den);
                    y = fma(e, px, e + px);
                } else {
                    rbm_direct(false, th_s[k], tt_s[k], u.z + v.z, val, y);
                }
                out[k] = val;
                pm1 = fma(pm1, y, pm1 + y);
            }
        } else {
            for (int k = hl; k < NH; k += 16) {          // tanh d1 and cosh d1 - 1 as stored
                const V4 u = r1[k];
                out[k] = u.x;
                pm1 = fma(pm1, u.y, pm1 + u.y);
            }
        }
        for (int k = NH + ((hl - NH) % 16 + 16) % 16; valid && k < NP; k += 16) out[k] = T(0);
        for (int o2 = 8; o2; o2 >>= 1) {
            const T z = __shfl_xor_sync(kFull, pm1, o2);
            pm1 = fma(pm1, z, pm1 + z);
        }
        if (valid && hl == 0) out[NP] = pm1;
        if (valid && hl < 3) out[NP + 1 + hl] = T(0);
    }
}

// per-site factors of the FP32 correlator path (see fam_corr_sites)
template <typename V4>
__global__ void k_corr_sites(const double* __restrict__ W, int K, int NH, int NP, V4* out)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= K * 12 * NP) return;
    const int k = idx % NP, row = idx / NP;
    const int p = row / 12, own = (row % 12) / 3, a = row % 3;
    const int to = sig_of_alt(a, own);
    double d = 0.0;
    if (k < NH) {
        if ((own ^ to) & 1) d += (to & 1) ? W[(size_t)k * 2 * K + 2 * p] : -W[(size_t)k * 2 * K + 2 * p];
        if ((own ^ to) & 2) d += (to & 2) ? W[(size_t)k * 2 * K + 2 * p + 1] : -W[(size_t)k * 2 * K + 2 * p + 1];
    }
    // em = e^d - 1, inv = e^-d: cosh d - 1 = em^2 inv / 2, sinh d = em (1 + inv) / 2
    const double em = expm1(d), inv = 1.0 / (1.0 + em);
    const double ch1 = 0.5 * em * em * inv, sh = 0.5 * em * (1.0 + inv);
    V4 o;
    o.x = sh / (1.0 + ch1); o.y = ch1; o.z = d; o.w = 0.0;
    out[idx] = o;
}

int fam_corr_sites(const double* W, int K, int n_hidden, float4* out, double4_32a* out64, cudaStream_t st)
{
    const int NP = (n_hidden + 3) & ~3, n = K * 12 * NP;
    if (n_hidden <= 0) return 0;
    k_corr_sites<float4><<<(n + 255) / 256, 256, 0, st>>>(W, K, n_hidden, NP, out);
    k_corr_sites<double4_32a><<<(n + 255) / 256, 256, 0, st>>>(W, K, n_hidden, NP, out64);
    return 2;
}

// ---------------------------------------------------------------------------
// Site-synchronous tables (tensor-core path). Step tau advances the left side
// through site tau and the right side through site K-1-tau for every sample
// of the batch at once; the items of a step read only what earlier steps wrote.
// Groups: g = side * 4 + sigma, the local state whose matrix the item applies.
// ---------------------------------------------------------------------------

template <typename T, bool FILL>
__global__ void __launch_bounds__(256) k_site_build(FamArgs<T> f, SiteBufs sb)
{
    __shared__ int cnt[kMaxOrb * 8];               // counts, then fill cursors
    __shared__ int own[kMaxOrb];
    const int b = blockIdx.x, K = f.K, D = f.D;
    const int nbb = (int)(f.s1 - f.s0);
    const int64_t s = f.s0 + b;
    const uint64_t na = f.samples[2 * s], nb = f.samples[2 * s + 1];
    for (int i = threadIdx.x; i < K; i += blockDim.x) own[i] = sigma_at(na, nb, i);
    __syncthreads();
    // the 3 tau one-change families of each side that step tau advances take
    // the first slots of their group (part 1 below); the other items follow
    for (int i = threadIdx.x; i < K * 8; i += blockDim.x) {
        const int tau = i >> 3, g = i & 7, side = g >> 2;
        const int t = side == 0 ? tau : K - 1 - tau;
        cnt[i] = (g & 3) == own[t] ? 3 * tau : 0;
    }
    __syncthreads();
    const size_t nk = (size_t)K * K * 9;
    // pool rows of this sample's G and H families
    const int64_t Gr = (int64_t)b * 3 * K * K, Hr = f.row_H + (int64_t)b * 3 * K * K;
    auto put = [&](int tau, int g, int64_t src, int64_t dst) {
        const int slot = atomicAdd(&cnt[tau * 8 + g], 1);
        if (FILL) {
            const int64_t at = sb.offs[((int64_t)tau * 8 + g) * nbb + b] + slot;
            SiteItem it;
            it.src = (uint32_t)src; it.dst = (uint32_t)dst;
            ((SiteItem*)sb.items)[at] = it;
        }
    };
    // (1) families created before the step (k_site_boundary makes the new ones
    // at their first site): family (j, a) of step tau at slot 3 j + a of its
    // group, one (side, step, j) per thread, so that a warp's items are adjacent
    for (int q = threadIdx.x; FILL && q < 2 * K * K; q += blockDim.x) {
        const int side = q / (K * K), rem = q - side * K * K, tau = rem / K, j = rem - tau * K;
        if (j >= tau) continue;
        const int t = side == 0 ? tau : K - 1 - tau;
        const int64_t Tr = side == 0 ? Gr : Hr;
        const int tp = side == 0 ? t - 1 : t + 1;      // the family's previous site
        const int sf = side == 0 ? j : K - 1 - j;
        const int64_t at = sb.offs[((int64_t)tau * 8 + side * 4 + own[t]) * nbb + b] + 3 * j;
        for (int a = 0; a < 3; ++a) {
            const int64_t base = Tr + ((int64_t)a * K + sf) * K;
            SiteItem it;
            it.src = (uint32_t)(base + tp); it.dst = (uint32_t)(base + t);
            ((SiteItem*)sb.items)[at + a] = it;
        }
    }
    // (2) TL clusters: creation at s2 with A_{s2}^{a2}, then A_t^{own} up to the last use
    const int ncl = f.tl_count[b];
    const int* tll = f.tl_list + (size_t)b * nk;
    const int64_t TLr = f.row_TL + f.tl_base[b];
    for (int c = threadIdx.x; c < ncl; c += blockDim.x) {
        const int key = tll[c];
        int s2, a2, s1, a1;
        key_fields(f, key, s2, a2, s1, a1);
        const int off = f.tl_idx[(size_t)b * nk + key];
        const int end = f.tl_end[(size_t)b * nk + key];
        const int64_t gi = Gr + ((int64_t)a1 * K + s1) * K + (s2 - 1);
        put(s2, sig_of_alt(a2, own[s2]), gi, TLr + off);
        for (int t = s2 + 1; t <= end; ++t) {
            const int64_t q = TLr + off + (t - s2);
            put(t, own[t], q - 1, q);
        }
    }
    // (3) TR rows: H_{sB,aB}(sA+1) A_{sA}^{aA} at the right step of site sA
    const int ntr = f.tr_total[b];
    const int* trl = f.tr_list + (size_t)b * nk;
    const int64_t TRr = f.row_TR + f.tr_base[b];
    for (int i = threadIdx.x; i < ntr; i += blockDim.x) {
        const int key = trl[i];
        int sA, aA, sB, aB;
        key_fields(f, key, sA, aA, sB, aB);
        const int64_t hi = Hr + ((int64_t)aB * K + sB) * K + sA + 1;
        put(K - 1 - sA, 4 + sig_of_alt(aA, own[sA]), hi, TRr + i);
    }
    if (!FILL) {
        __syncthreads();
        for (int i = threadIdx.x; i < K * 8; i += blockDim.x)
            sb.counts[(int64_t)i * nbb + b] = cnt[i];
    }
}

// Boundary vectors L_t (R_t) of each sample and side and the three families
// that start at each site, on the CUDA cores (in the arithmetic type of the
// tables; FP32 for the tensor-core form, whose split-FP16 products would put
// their error into every vector built on the boundary). One block per side and
// group of S samples, steps in order: at each site the four matrices
// [A^0; A^1; A^2; A^3] are read once per block and applied to the S samples'
// vectors (every sample needs all four: its three alternatives and its own
// state), one output row per thread and pass with an fma over the input index
// in ascending order (the order of mv_block, so the results are the same bit
// for bit).
template <typename T, int S>
__global__ void __launch_bounds__(256) k_site_boundary(FamArgs<T> f)
{
    extern __shared__ __align__(16) unsigned char smb[];
    __shared__ int eo[S * 4];
    __shared__ int eL[S];
    __shared__ int own_s[S];
    const int nbb = (int)(f.s1 - f.s0);
    const int side = blockIdx.x & 1, g0 = (blockIdx.x >> 1) * S;
    const int ns = nbb - g0 < S ? nbb - g0 : S;
    const int K = f.K, D = f.D;
    T* X = (T*)smb;                               // [S][D] the samples' vectors
    T* Z = X + (size_t)S * D;                     // [S][4][D] their four products
    const T* Mats = side == 0 ? f.AT : f.A;       // column convention left, row vectors right
    for (int q = threadIdx.x; q < S * D; q += blockDim.x) X[q] = (q % D) == 0 ? T(1) : T(0);
    if (threadIdx.x < S) eL[threadIdx.x] = 0;
    __syncthreads();
    for (int step = 0; step < K; ++step) {
        const int t = side == 0 ? step : K - 1 - step;
        if (threadIdx.x < ns) {
            const int64_t s = f.s0 + g0 + threadIdx.x;
            own_s[threadIdx.x] = sigma_at(f.samples[2 * s], f.samples[2 * s + 1], t);
        }
        for (int q = threadIdx.x; q < 4 * D; q += blockDim.x) {
            const int sg = q / D, r = q - sg * D;
            const T* MT = Mats + ((size_t)t * 4 + sg) * D * D;
            T acc[S];
            #pragma unroll
            for (int j = 0; j < S; ++j) acc[j] = T(0);
            for (int c = 0; c < D; ++c) {
                const T m = __ldg(MT + (size_t)c * D + r);
                #pragma unroll
                for (int j = 0; j < S; ++j) acc[j] = fma(m, X[j * D + c], acc[j]);
            }
            #pragma unroll
            for (int j = 0; j < S; ++j)
                if (j < ns) Z[((size_t)j * 4 + sg) * D + r] = acc[j];
        }
        __syncthreads();
        renorm_rows<T>(Z, D, ns * 4, eo);
        __syncthreads();
        // the three alternatives' families at their first site, then the own
        // state's product as the next boundary vector
        for (int q = threadIdx.x; q < ns * 3 * D; q += blockDim.x) {
            const int j = q / (3 * D), ac = q - j * 3 * D, a = ac / D, c = ac - a * D;
            const int sg = sig_of_alt(a, own_s[j]);
            T* Tb = (side == 0 ? f.G : f.H) + (size_t)(g0 + j) * 3 * K * K * D;
            Tb[(((size_t)a * K + t) * K + t) * D + c] = Z[((size_t)j * 4 + sg) * D + c];
        }
        for (int q = threadIdx.x; q < ns * 3; q += blockDim.x) {
            const int j = q / 3, a = q - 3 * j;
            int* Te = (side == 0 ? f.Ge : f.He) + (size_t)(g0 + j) * 3 * K * K;
            Te[((size_t)a * K + t) * K + t] = eL[j] + eo[j * 4 + sig_of_alt(a, own_s[j])];
        }
        for (int q = threadIdx.x; q < ns * D; q += blockDim.x) {
            const int j = q / D, c = q - j * D;
            X[q] = Z[((size_t)j * 4 + own_s[j]) * D + c];
        }
        __syncthreads();
        if (threadIdx.x < ns) eL[threadIdx.x] += eo[threadIdx.x * 4 + own_s[threadIdx.x]];
        __syncthreads();
    }
}

// first item of every (step, group): bounds[i] = offs[i * nbb], bounds[K*8] = total
__global__ void k_site_bounds(const int64_t* offs, int n, int nbb, int64_t* bounds)
{
    for (int i = threadIdx.x; i <= n; i += blockDim.x) bounds[i] = offs[(int64_t)i * nbb];
}

struct SiteStep {
    int64_t gbeg[8], gend[8];   // item range of each group
    int tbeg[9];                // first tile of each group; tbeg[8] = tiles of the step
    int mat[8];                 // matrix image of each group
    int rows;                   // rows per tile
};

template <typename T>
__global__ void __launch_bounds__(256, 4) k_site_tiles(FamArgs<T> f, const SiteItem* items, SiteStep st)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ const T* s_src[128];
    __shared__ T* s_dst[128];
    __shared__ const int* s_se[128];
    __shared__ int* s_de[128];
    __shared__ int s_eo[128];
    BatchSmem<T> sm;
    batch_init(f, sm, smraw, &tmem_slot, &mbar);
    const bool tc = use_tc(f);
    const int rows = st.rows, D = f.D;
    const int ntiles = st.tbeg[8];
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        int g = 0;
        while (g < 7 && tile >= st.tbeg[g + 1]) ++g;
        const int64_t i0 = st.gbeg[g] + (int64_t)(tile - st.tbeg[g]) * rows;
        const int64_t left = st.gend[g] - i0;
        const int n = (int)(left < rows ? left : rows);
        for (int r = threadIdx.x; r < n; r += blockDim.x) {
            const SiteItem it = items[i0 + r];
            s_src[r] = f.pool + (size_t)it.src * D; s_dst[r] = f.pool + (size_t)it.dst * D;
            s_se[r] = f.pool_e + it.src; s_de[r] = f.pool_e + it.dst;
        }
        __syncthreads();
        const int mat = st.mat[g];
        if constexpr (std::is_same<T, float>::value) {
            if (tc) {
                struct Acc {
                    const float* const* s; float* const* d; const int* const* se; int* const* de;
                    __device__ const float* src(int r) const { return s[r]; }
                    __device__ float* dst(int r) const { return d[r]; }
                    __device__ void set_exp(int r, int x) const { *de[r] = *se[r] + x; }
                } acc{s_src, s_dst, s_se, s_de};
                tc_apply(f, sm, acc, n, mat);          // ends with a block barrier
                continue;
            }
        }
        // CUDA-core batch: gather, y = M x with the FP32/FP64 matrices, rescale, scatter
        const int side = mat / (4 * f.K), t = (mat >> 2) % f.K, sg = mat & 3;
        for (int q = threadIdx.x; q < n * D; q += blockDim.x) {
            const int i = q / D, c = q - i * D;
            sm.X[q] = s_src[i][c];
        }
        __syncthreads();
        if constexpr (std::is_same<T, double>::value) {
            if (f.df) {
                // the gathered rows as float halves in Y, the products back into X
                float* Xh = (float*)sm.Y;
                float* Xl = Xh + (size_t)n * D;
                for (int q = threadIdx.x; q < n * D; q += blockDim.x) {
                    const float h = (float)sm.X[q];
                    Xh[q] = h;
                    Xl[q] = (float)(sm.X[q] - (double)h);
                }
                __syncthreads();
                mv_block_df((side == 0 ? f.ATdf : f.Adf) + ((size_t)t * 4 + sg) * D * D, D, Xh, Xl, sm.X, n);
                __syncthreads();
                for (int q = threadIdx.x; q < n * D; q += blockDim.x) sm.Y[q] = sm.X[q];
            } else {
                mv_block<T>((side == 0 ? f.AT : f.A) + ((size_t)t * 4 + sg) * D * D, D, sm.X, sm.Y, n);
            }
        } else {
            mv_block<T>((side == 0 ? f.AT : f.A) + ((size_t)t * 4 + sg) * D * D, D, sm.X, sm.Y, n);
        }
        __syncthreads();
        renorm_rows<T>(sm.Y, D, n, s_eo);
        __syncthreads();
        for (int q = threadIdx.x; q < n * D; q += blockDim.x) {
            const int i = q / D, c = q - i * D;
            s_dst[i][c] = sm.Y[q];
        }
        for (int i = threadIdx.x; i < n; i += blockDim.x) *s_de[i] = *s_se[i] + s_eo[i];
        __syncthreads();
    }
    batch_fini(f, sm);
}

// ---------------------------------------------------------------------------
// Pipelined tensor-core site step (FP32 tables, D <= 64: one reduction chunk).
// A block walks a contiguous range of tiles (one matrix image for most of
// them) with two row stages: while tile i is split into
// FP16 hi / lo, multiplied and written back, the rows of tile i+1 stream into
// the other stage with cp.async and the items of tile i+2 are read into
// registers, so that each SM keeps two tiles' gathers in flight. A stage holds
// the raw FP32 rows (stride 4D + 16 bytes, so that the split's reads fall on
// distinct banks) and, once split in place, the A operand (hi then lo, in the
// core-matrix layout). Per row the arithmetic is that of tc_apply (same split,
// same MMAs in the same order, same rescaling), so the results are bitwise
// those of the unpipelined kernel.
// ---------------------------------------------------------------------------
constexpr int kPipeRows = 128;

inline size_t pipe_stage_bytes(int D)
{
    const size_t raw = (size_t)kPipeRows * (4 * D + 16);
    return (raw + 1023) & ~(size_t)1023;
}
inline size_t pipe_smem_bytes(int D) { return 2 * pipe_stage_bytes(D) + (size_t)4 * D * D; }

__global__ void __launch_bounds__(256, 2) k_site_tiles_pipe(FamArgs<float> f, const SiteItem* items, SiteStep st,
                                                           uint32_t stage_bytes)
{
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_src[3][kPipeRows];          // pool rows of the items
    __shared__ uint32_t s_dst[3][kPipeRows];
    __shared__ int s_sev[2][kPipeRows];
    __shared__ float s_rmax[2][kPipeRows];
    const int D = f.D, tid = threadIdx.x;
    const int RS = 4 * D + 16;                         // stage row stride, bytes
    unsigned char* const stage0 = smraw;
    unsigned char* const Bh = smraw + 2 * (size_t)stage_bytes;
    const int ntiles = st.tbeg[8];
    // this block's tiles: [t_beg, t_end), non-empty as the grid never exceeds the tiles
    const int t_beg = (int)((int64_t)blockIdx.x * ntiles / gridDim.x);
    const int t_end = (int)((int64_t)(blockIdx.x + 1) * ntiles / gridDim.x);
    if (tid < 32) { tc::tmem_alloc(&tmem_slot, f.tc_cols); tc::tmem_relinquish(); }
    if (tid == 0) tc::mbar_init(&mbar, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    // tile -> (group, first item, rows); the group search starts from g, as a
    // block's tiles ascend
    auto tile_info = [&](int tile, int& g, int64_t& i0, int& n) {
        while (g < 7 && tile >= st.tbeg[g + 1]) ++g;
        i0 = st.gbeg[g] + (int64_t)(tile - st.tbeg[g]) * kPipeRows;
        const int64_t left = st.gend[g] - i0;
        n = (int)(left < kPipeRows ? left : kPipeRows);
    };
    auto put_item = [&](int slot, int r, const SiteItem& it) {
        s_src[slot][r] = it.src; s_dst[slot][r] = it.dst;
    };
    // rows and source exponents of the tile in item slot `slot` into stage `buf`
    // piece v = tid + 256 j of a tile is row v / qpr, 16-byte piece v % qpr
    const int qpr = D >> 2;
    const int f_r0 = tid / qpr, f_q0 = tid - f_r0 * qpr;
    const int f_dr = 256 / qpr, f_dq = 256 - f_dr * qpr;
    auto fetch = [&](int slot, int buf, int n) {
        unsigned char* sg = stage0 + (size_t)buf * stage_bytes;
        int r = f_r0, q = f_q0;
        while (r < n) {
            tc::cp_async16(sg + r * RS + q * 16, f.pool + (size_t)s_src[slot][r] * D + 4 * q);
            r += f_dr; q += f_dq;
            if (q >= qpr) { q -= qpr; ++r; }
        }
        if (tid < n) tc::cp_async4(&s_sev[buf][tid], f.pool_e + s_src[slot][tid]);
    };
    // (group, rows) of tiles i, i+1, i+2 of the loop, carried forward
    int g0 = 0, g1 = 0, g2 = 0, n0 = 0, n1 = 0;
    {
        int64_t i0;
        tile_info(t_beg, g0, i0, n0);
        if (tid < n0) put_item(0, tid, items[i0 + tid]);
        g1 = g0;
        if (t_beg + 1 < t_end) {
            tile_info(t_beg + 1, g1, i0, n1);
            if (tid < n1) put_item(1, tid, items[i0 + tid]);
        }
        g2 = g1;
        __syncthreads();
        fetch(0, 0, n0);
        tc::cp_async_commit();
    }
    // the split's units (8 columns of one row) of this thread: stage read and
    // operand write offsets, the same for every tile
    const int cpr = D >> 3, nun = kPipeRows * cpr;
    int rd_off[4];
    uint32_t wr_off[4];
    #pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int u = tid + k * 256;
        const int r8 = u & 7, rest = u >> 3, c = rest % cpr, rg = rest / cpr;
        rd_off[k] = (8 * rg + r8) * RS + 32 * c;
        wr_off[k] = tc::op_offset(8 * rg + r8, 8 * c, D);
    }
    int cur_mat = -1, mat_exp = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int i = 0, tile = t_beg; tile < t_end; ++i, ++tile) {
        const int cur = i & 1, ri = i % 3;
        unsigned char* const sc = stage0 + (size_t)cur * stage_bytes;
        const int g = g0, n = n0;
        // (1) the next tile's rows into the other stage (its last reader, the
        // MMAs of tile i-1, completed before the previous epilogue)
        if (tile + 1 < t_end) fetch((i + 1) % 3, cur ^ 1, n1);
        tc::cp_async_commit();
        // (2) the items of the tile after next, into registers
        SiteItem nx{};
        int n2 = 0;
        if (tile + 2 < t_end) {
            int64_t i2;
            tile_info(tile + 2, g2, i2, n2);
            if (tid < n2) nx = items[i2 + tid];
        }
        // (3) this tile's rows have landed
        tc::cp_async_wait<1>();
        __syncthreads();
        // (4) split in place: every read before any write. Unit u = 8 columns
        // of one row; the 8 lanes of a unit group take the 8 rows of one
        // core matrix, so each group's stores fill one 128-byte core matrix.
        float xv[4][8];
        #pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (tid + k * 256 < nun) {
                const float4* p = (const float4*)(sc + rd_off[k]);
                const float4 a = p[0], b = p[1];
                xv[k][0] = a.x; xv[k][1] = a.y; xv[k][2] = a.z; xv[k][3] = a.w;
                xv[k][4] = b.x; xv[k][5] = b.y; xv[k][6] = b.z; xv[k][7] = b.w;
            }
        }
        __syncthreads();
        #pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (tid + k * 256 < nun) {
                __align__(16) __half2 hi[4], lo[4];
                #pragma unroll
                for (int j = 0; j < 4; ++j) tc::split_half2(xv[k][2 * j], xv[k][2 * j + 1], hi[j], lo[j]);
                const uint32_t off = wr_off[k];
                *(uint4*)(sc + off) = *(const uint4*)hi;
                *(uint4*)(sc + (size_t)kPipeRows * D * 2 + off) = *(const uint4*)lo;
            }
        }
        // (5) the matrix image (and its scale) when the group's matrix changes
        const int mat = st.mat[g];
        if (mat != cur_mat) {
            const int nimg = 4 * D * D / 16;
            const uint4* __restrict__ gsrc = f.tc_mats + (size_t)mat * nimg;
            for (int q = tid; q < nimg; q += blockDim.x) ((uint4*)Bh)[q] = __ldg(gsrc + q);
            mat_exp = f.tc_exp[mat];
            cur_mat = mat;
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        // (6) x_hi M_hi + x_lo M_hi + x_hi M_lo into tensor memory
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t idesc = tc::idesc_f16(128, D);
            const uint32_t lbo = 128, sbo = 16 * D;
            const unsigned char* As[3] = {sc, sc + (size_t)kPipeRows * D * 2, sc};
            const unsigned char* Bs[3] = {Bh, Bh, Bh + 2 * D * D};
            uint32_t acc = 0;
            for (int term = 0; term < 3; ++term)
                for (int ks = 0; ks < D / 16; ++ks) {
                    tc::mma_f16(tmem, tc::desc(tc::smem_addr(As[term]) + ks * 256, lbo, sbo),
                                tc::desc(tc::smem_addr(Bs[term]) + ks * 256, lbo, sbo), idesc, acc);
                    acc = 1;
                }
            tc::mma_commit(&mbar);
        }
        // (7) the items fetched in (2) replace those of tile i-1
        if (tid < n2) put_item((i + 2) % 3, tid, nx);
        ok = tc::mbar_wait(&mbar, phase, 1u << 24) && ok;
        phase ^= 1u;
        tc::fence_after_sync();
        // (8) two passes over tensor memory, 8 columns at a time
        const int warp = tid >> 5, lane = tid & 31;
        const int q = warp & 3, h = warp >> 2, half = D >> 1;
        const int r = 32 * q + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + h * half;
        {
            float m = 0.f;
            for (int c0 = 0; c0 < half; c0 += 8) {
                float v[8];
                tc::tmem_ld8(trow + c0, v);
                tc::tmem_wait_ld();
                #pragma unroll
                for (int j = 0; j < 8; ++j) m = fmaxf(m, fabsf(v[j]));
            }
            s_rmax[h][r] = m;
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        {
            // the scaled rows go to the stage (free since the MMAs completed;
            // stride RS, so 8 consecutive rows fill the 32 banks), then leave
            // it row by row with coalesced stores
            const float mm = fmaxf(s_rmax[0][r], s_rmax[1][r]);
            int e = 0;
            if (mm > 0.f) frexpf(mm, &e);
            float* o = (float*)(sc + r * RS) + h * half;
            const bool pw = e >= -126 && e <= 126;
            const float sc2 = pw ? __int_as_float((127 - e) << 23) : 0.f;
            for (int c0 = 0; c0 < half; c0 += 8) {
                float v[8];
                tc::tmem_ld8(trow + c0, v);
                tc::tmem_wait_ld();
                #pragma unroll
                for (int j = 0; j < 8; ++j) v[j] = pw ? v[j] * sc2 : ldexpf(v[j], -e);
                *(float4*)(o + c0) = make_float4(v[0], v[1], v[2], v[3]);
                *(float4*)(o + c0 + 4) = make_float4(v[4], v[5], v[6], v[7]);
            }
            if (h == 0 && r < n) f.pool_e[s_dst[ri][r]] = s_sev[cur][r] + e + mat_exp;
        }
        tc::fence_before_sync();
        __syncthreads();
        {
            int rr = f_r0, qq = f_q0;             // the fetch's piece order: lanes along a row
            while (rr < n) {
                const float4 w = *(const float4*)(sc + rr * RS + qq * 16);
                *(float4*)(f.pool + (size_t)s_dst[ri][rr] * D + 4 * qq) = w;
                rr += f_dr; qq += f_dq;
                if (qq >= qpr) { qq -= qpr; ++rr; }
            }
        }
        __syncthreads();
        g0 = g1; n0 = n1;
        g1 = g2; n1 = n2;
    }
    tc::cp_async_wait<0>();
    if (!ok && tid == 0) report(f.err, 5, 4, (long long)f.s0);
    tc::fence_before_sync();
    __syncthreads();
    if (tid < 32) tc::tmem_dealloc(tmem, f.tc_cols);
}

template <typename T>
int fam_site_count(const FamArgs<T>& f, const SiteBufs& b, int nbb, cudaStream_t st)
{
    const int n = f.K * 8;
    // eight samples per block when the batch fills the GPU with them (the
    // matrices are then read once per eight samples), else one (small calls
    // keep one short chain per block)
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (nbb >= 8 * n_sm) {
        const size_t smem = (size_t)5 * 8 * f.D * sizeof(T);
        allow_max_smem(k_site_boundary<T, 8>);
        k_site_boundary<T, 8><<<(unsigned)((nbb + 7) / 8) * 2, 256, smem, st>>>(f);
    } else {
        k_site_boundary<T, 1><<<(unsigned)nbb * 2, 256, (size_t)5 * f.D * sizeof(T), st>>>(f);
    }
    k_site_build<T, false><<<nbb, 256, 0, st>>>(f, b);
    const int ns = launch_scan_i64_wide(b.counts, b.offs, (int64_t)n * nbb, b.scan_tmp, st);
    k_site_bounds<<<1, 256, 0, st>>>(b.offs, n, nbb, b.bounds);
    return 3 + ns;
}

template <typename T>
int fam_site_fill(const FamArgs<T>& f, const SiteBufs& b, int nbb, cudaStream_t st)
{
    k_site_build<T, true><<<nbb, 256, 0, st>>>(f, b);
    return 1;
}

template <typename T>
int fam_site_step(const FamArgs<T>& f, const SiteBufs& b, int tau, const int64_t* bounds,
                  int max_ctas, cudaStream_t st)
{
    const bool tc = std::is_same<T, float>::value && f.tc;
    // tensor-core tiles are 128 rows; CUDA-core tiles shrink (to 4 rows) when a
    // step has few items, so that they still spread over about half the CTAs
    // (an FP64 tile is slow on one SM)
    int rows = 128;
    if (!tc) {
        const int64_t items = bounds[tau * 8 + 8] - bounds[tau * 8];
        const int64_t want = (items + max_ctas / 2 - 1) / (max_ctas / 2 > 0 ? max_ctas / 2 : 1);
        rows = (int)std::min<int64_t>(f.nmax, std::max<int64_t>(4, (want + 3) / 4 * 4));
    }
    SiteStep ss{};
    ss.rows = rows;
    int tiles = 0;
    for (int g = 0; g < 8; ++g) {
        ss.gbeg[g] = bounds[tau * 8 + g];
        ss.gend[g] = bounds[tau * 8 + g + 1];
        ss.tbeg[g] = tiles;
        tiles += (int)((ss.gend[g] - ss.gbeg[g] + rows - 1) / rows);
        const int side = g >> 2;
        const int t = side == 0 ? tau : f.K - 1 - tau;
        ss.mat[g] = (side * f.K + t) * 4 + (g & 3);
    }
    ss.tbeg[8] = tiles;
    if (tiles == 0) return 0;
    if constexpr (std::is_same<T, float>::value) {
        if (tc && f.D <= 64) {
            // two blocks per SM, each with two tiles' rows in flight
            allow_max_smem(k_site_tiles_pipe);
            cudaFuncSetAttribute(k_site_tiles_pipe, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
            const int grid = tiles < max_ctas / 2 ? tiles : max_ctas / 2;
            k_site_tiles_pipe<<<grid, 256, pipe_smem_bytes(f.D), st>>>(
                f, (const SiteItem*)b.items, ss, (uint32_t)pipe_stage_bytes(f.D));
            return 1;
        }
    }
    allow_max_smem(k_site_tiles<T>);
    const size_t smem = f.batch_bytes;
    const int grid = tiles < max_ctas ? tiles : max_ctas;
    k_site_tiles<T><<<grid, 256, smem, st>>>(f, (const SiteItem*)b.items, ss);
    return 1;
}

// F5: psi_TN(m) as a dot product of a left state and a right covector, the
// factorised correlator ratio, coefficient x ratio; block partial sums in a
// fixed order. Each lane decodes one row; then each warp evaluates its 32 rows
// one at a time with coalesced loads (lanes split the vectors and the hidden
// units), a compensated tree for the dot product and a tree for the product.
constexpr int kFamRows = 128;
constexpr int kFamRowsMB64 = 8;          // blocks per SM of the compile-time-D row kernels

template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T& s, T& e)
{
    s = a + b;
    const T z = s - a;
    e = (a - (s - z)) + (b - z);
}

// x 2^e, exact: an exponent-field add while the result stays a normal number
// (integer ALU work instead of the thin FP64 pipe), ldexp otherwise
__device__ __forceinline__ double scale_pow2(double x, int e)
{
    const long long bits = __double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7FF);
    const int ne = ex + e;
    if (ex != 0 && ex != 0x7FF && ne > 0 && ne < 0x7FF)
        return __longlong_as_double(bits + ((long long)e << 52));
    return ldexp(x, e);
}

// DT > 0: the bond dimension at compile time. Each lane group then issues
// all of its row's loads (left / right vector pieces, correlator groups) before
// the arithmetic, with fully unrolled loops; more registers per thread, fewer
// blocks per SM (MB), more loads in flight per warp. The arithmetic and its
// order are those of the general path (DT = 0).
template <typename T, int DT, int MB>
__global__ void __launch_bounds__(kFamRows, MB) k_fam_rows(FamArgs<T> f, RowSet rows, double* partial,
                                                           int64_t* span, double* partial_abs)
{
    __shared__ OrbLists lists;
    __shared__ T s_ratio[kFamRows];                  // each row's ratio in the contraction type
    __shared__ __align__(16) const T* s_ptr[kFamRows][4];   // each row's L, R and correlator rows
    __shared__ double s_coef[kFamRows];              // each row's coefficient, exponent and span,
    __shared__ int s_ex[kFamRows], s_nmv[kFamRows];  // kept out of registers during the evaluation
    __shared__ double wsum[kFamRows / 32];
    __shared__ double wabs[kFamRows / 32];
    __shared__ long long wspan[kFamRows / 32];
    __shared__ double s_inv_pm;
    const int64_t* cb = rows.chunk_base;
    const int64_t blk = cb[f.s0] + blockIdx.x;
    if (blk >= cb[f.s1]) return;
    int64_t lo = f.s0, hi = f.s1 - 1;          // largest s with cb[s] <= blk
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (cb[mid] <= blk) lo = mid; else hi = mid - 1;
    }
    const int64_t s = lo;
    const int b = (int)(s - f.s0), K = f.K, D = f.D;
    const int64_t j = blk - cb[s];
    const int64_t beg = rows.begin ? rows.begin[s] : s * rows.stride;
    const int64_t cnt = rows.count[s];
    const int64_t r0 = beg + j * kFamRows;
    const int nr = (int)((cnt - j * kFamRows) < kFamRows ? (cnt - j * kFamRows) : kFamRows);
    const uint64_t na = f.samples[2 * s], nb = f.samples[2 * s + 1];
    const int NH = f.n_hidden, NP = nh_pad(NH);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0 && !rows.sites) build_lists_warp(na, nb, f.h.K, lists, lane);
    if (threadIdx.x == 32) s_inv_pm = 1.0 / f.pm[b];
    __syncthreads();
    const size_t nk = (size_t)K * K * 9;
    // ---- per-lane decode of one row
    const T* Lv = nullptr;
    const T* Rv = nullptr;
    const T* lt = nullptr;
    const T* rs = nullptr;
    int ex = 0, nmv = 0;
    double coef = 0.0;
    const int myrow = (int)threadIdx.x;
    if (myrow < nr) {
        const RowParts p = row_parts_of(f.h, lists, na, nb, rows, r0 + myrow);
        const T* G = f.G + (size_t)b * 3 * K * K * D;
        const int* Ge = f.Ge + (size_t)b * 3 * K * K;
        const T* H = f.H + (size_t)b * 3 * K * K * D;
        const int* He = f.He + (size_t)b * 3 * K * K;
        int eL, eR, lobj, robj;
        if (p.nsite == 4) {
            const int key = tl_key(K, p.s[0], p.a[0], p.s[1], p.a[1]);
            const int off = f.tl_idx[(size_t)b * nk + key] + (p.s[2] - 1 - p.s[1]);
            const int ti = f.tr_idx[(size_t)b * nk + tr_key(K, p.s[2], p.a[2], p.s[3], p.a[3])];
            Lv = f.TL + ((size_t)f.tl_base[b] + off) * D;
            eL = f.TLe[f.tl_base[b] + off];
            Rv = f.TR + ((size_t)f.tr_base[b] + ti) * D;
            eR = f.TRe[f.tr_base[b] + ti];
            lobj = 3 * K + f.tl_ci[(size_t)b * nk + key];
            robj = 3 * K + ti;
        } else {
            const size_t gi = ((size_t)p.a[0] * K + p.s[0]) * K + p.s[1] - 1;
            Lv = G + gi * D;
            eL = Ge[gi];
            lobj = 3 * p.s[0] + p.a[0];
            if (p.nsite == 2) {
                const size_t hi2 = ((size_t)p.a[1] * K + p.s[1]) * K + p.s[1];
                Rv = H + hi2 * D;
                eR = He[hi2];
                robj = 3 * p.s[1] + p.a[1];
            } else {
                const int ti = f.tr_idx[(size_t)b * nk + tr_key(K, p.s[1], p.a[1], p.s[2], p.a[2])];
                Rv = f.TR + ((size_t)f.tr_base[b] + ti) * D;
                eR = f.TRe[f.tr_base[b] + ti];
                robj = 3 * K + ti;
            }
        }
        ex = eL + eR;
        nmv = p.last - p.s[0] + 1;
        coef = rows.coef[r0 + myrow];
        if (NH > 0) {
            lt = f.rbl + (size_t)(f.rbl_base[b] + lobj) * rbm_row_len(NH);
            rs = f.rbr + (size_t)(f.rbr_base[b] + robj) * rbm_row_len(NH);
        }
    }
    s_ptr[myrow][0] = Lv; s_ptr[myrow][1] = Rv; s_ptr[myrow][2] = lt; s_ptr[myrow][3] = rs;
    s_coef[myrow] = coef; s_ex[myrow] = ex; s_nmv[myrow] = nmv;
    __syncwarp();                                   // a warp reads only its own rows' values
    const double inv_pm = s_inv_pm;
    const int pe = f.pe[b];
    // ---- evaluation: 8 lanes per row, 4 rows of the warp at a time
    const int wbase = warp * 32;
    const int wrows = nr - wbase < 32 ? (nr - wbase > 0 ? nr - wbase : 0) : 32;
    const int g = lane >> 3, sub = lane & 7;
    for (int q0 = 0; q0 < wrows; q0 += 4) {
        const int q = q0 + g;                       // the row this lane group evaluates (< 32)
        const ulonglong2 p01 = *(const ulonglong2*)&s_ptr[wbase + q][0];
        const ulonglong2 p23 = *(const ulonglong2*)&s_ptr[wbase + q][2];
        const T* Lq = (const T*)p01.x;
        const T* Rq = (const T*)p01.y;
        const T* ltq = (const T*)p23.x;
        const T* rsq = (const T*)p23.y;
        const bool live = q < wrows;
        T ratio;
        if constexpr (DT > 0) {
            typedef typename Vec4<T>::type V4;
            constexpr int NV = DT / 4, PER = (NV + 7) / 8;
            const int NG = NP / 4 + 1;           // correlator groups, the last holding P - 1
            V4 xv[PER], yv[PER], tv[4], uv[4];
            if (live) {
                #pragma unroll
                for (int u = 0; u < PER; ++u)
                    if (sub + 8 * u < NV) { xv[u] = ((const V4*)Lq)[sub + 8 * u]; yv[u] = ((const V4*)Rq)[sub + 8 * u]; }
                if (NH > 0) {
                    #pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (sub + 8 * u < NG) {
                            tv[u] = ((const V4*)ltq)[sub + 8 * u];
                            uv[u] = ((const V4*)rsq)[sub + 8 * u];
                        }
                }
            }
            T sum = T(0), comp = T(0);
            if (live) {
                #pragma unroll
                for (int u = 0; u < PER; ++u) {
                    if (sub + 8 * u < NV) {
                        const T xs[4] = {xv[u].x, xv[u].y, xv[u].z, xv[u].w};
                        const T ys[4] = {yv[u].x, yv[u].y, yv[u].z, yv[u].w};
                        #pragma unroll
                        for (int w = 0; w < 4; ++w) {
                            const T pr = xs[w] * ys[w];
                            const T pe2 = fma(xs[w], ys[w], -pr);
                            T t, e;
                            two_sum(sum, pr, t, e);
                            sum = t;
                            comp += e + pe2;
                        }
                    }
                }
            }
            for (int o = 4; o; o >>= 1) {
                const T so = __shfl_xor_sync(kFull, sum, o);
                const T co = __shfl_xor_sync(kFull, comp, o);
                T t, e;
                two_sum(sum, so, t, e);
                sum = t;
                comp += co + e;
            }
            ratio = sum + comp;
            if (NH > 0) {
                T X = T(0);                        // product of (1 + x_k) minus 1
                if (live) {
                    auto group = [&](const V4& t, const V4& u, bool last) {
                        T x;
                        // the last group holds PL - 1 and PR - 1 (then zeros): (1 + a)(1 + b) - 1
                        x = last ? fma(t.x, u.x, t.x + u.x) : t.x * u.x; X = fma(X, x, X + x);
                        x = t.y * u.y; X = fma(X, x, X + x);
                        x = t.z * u.z; X = fma(X, x, X + x);
                        x = t.w * u.w; X = fma(X, x, X + x);
                    };
                    #pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (sub + 8 * u < NG) group(tv[u], uv[u], sub + 8 * u == NG - 1);
                    for (int k4 = sub + 32; k4 < NG; k4 += 8)
                        group(((const V4*)ltq)[k4], ((const V4*)rsq)[k4], k4 == NG - 1);
                }
                for (int o = 4; o; o >>= 1) {
                    const T Y = __shfl_xor_sync(kFull, X, o);
                    X = fma(X, Y, X + Y);
                }
                if (live) ratio *= T(1) + X;
            }
        } else {
            // dot product: FP32 with error-free product / sum transformations; FP64
            // with plain fused multiply-adds (its rounding, ~D 2^-53 of sum |x y|,
            // is far inside the FP64 forms' bar)
            constexpr bool dbl = std::is_same<T, double>::value;
            auto acc = [&](T x, T y, T& sum, T& comp) {
                if constexpr (dbl) {
                    sum = fma(x, y, sum);
                } else {
                    const T pr = x * y;
                    const T pe2 = fma(x, y, -pr);
                    T t, e;
                    two_sum(sum, pr, t, e);
                    sum = t;
                    comp += e + pe2;
                }
            };
            T sum = T(0), comp = T(0);
            if (live) {
                if ((D & 3) == 0) {
                    typedef typename Vec4<T>::type V4;
                    for (int c4 = sub; c4 < D / 4; c4 += 8) {
                        const V4 x = ((const V4*)Lq)[c4], y = ((const V4*)Rq)[c4];
                        acc(x.x, y.x, sum, comp);
                        acc(x.y, y.y, sum, comp);
                        acc(x.z, y.z, sum, comp);
                        acc(x.w, y.w, sum, comp);
                    }
                } else {
                    for (int c = sub; c < D; c += 8) acc(Lq[c], Rq[c], sum, comp);
                }
            }
            for (int o = 4; o; o >>= 1) {
                const T so = __shfl_xor_sync(kFull, sum, o);
                if constexpr (dbl) {
                    sum += so;
                } else {
                    const T co = __shfl_xor_sync(kFull, comp, o);
                    T t, e;
                    two_sum(sum, so, t, e);
                    sum = t;
                    comp += co + e;
                }
            }
            ratio = sum + comp;
            if (NH > 0) {
                typedef typename Vec4<T>::type V4;
                T X = T(0);                            // product of (1 + x_k) minus 1
                if (live) {
                    const V4* l4 = (const V4*)ltq;
                    const V4* r4 = (const V4*)rsq;
                    for (int k4 = sub; k4 <= NP / 4; k4 += 8) {
                        const V4 t = l4[k4], u = r4[k4];
                        T x;
                        // the last group holds PL - 1 and PR - 1 (then zeros): (1 + a)(1 + b) - 1
                        x = k4 == NP / 4 ? fma(t.x, u.x, t.x + u.x) : t.x * u.x; X = fma(X, x, X + x);
                        x = t.y * u.y; X = fma(X, x, X + x);
                        x = t.z * u.z; X = fma(X, x, X + x);
                        x = t.w * u.w; X = fma(X, x, X + x);
                    }
                }
                for (int o = 4; o; o >>= 1) {
                    const T Y = __shfl_xor_sync(kFull, X, o);
                    X = fma(X, Y, X + Y);
                }
                if (live) ratio *= T(1) + X;
            }
        }
        if (live && sub == 0) s_ratio[wbase + q] = ratio;
    }
    __syncwarp();
    // the FP64 epilogue once per row, by the lane that decoded it: H_nm (or the
    // draw weight) / psi(n) and the power of two of the row's scaled vectors
    double acc = 0.0, aacc = 0.0;
    if (myrow < nr) {
        acc = scale_pow2(s_coef[myrow] * ((double)s_ratio[myrow] * inv_pm), s_ex[myrow] - pe);
        if (partial_abs) aacc = fabs(acc);
    }
    long long sp = s_nmv[myrow];
    for (int o = 16; o; o >>= 1) {
        acc += __shfl_xor_sync(kFull, acc, o);
        sp += __shfl_xor_sync(kFull, sp, o);
        if (partial_abs) aacc += __shfl_xor_sync(kFull, aacc, o);
    }
    if (lane == 0) { wsum[warp] = acc; wspan[warp] = sp; wabs[warp] = aacc; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0, ta = 0.0;
        long long st = 0;
        for (int w = 0; w < kFamRows / 32; ++w) { t += wsum[w]; st += wspan[w]; ta += wabs[w]; }
        partial[blk] = t;
        if (span) span[blk] = st;
        if (partial_abs) partial_abs[blk] = ta;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

template <typename T>
int fam_launch_mark(const FamArgs<T>& f, const RowSet& rows, int nb, uint32_t* words, cudaStream_t st)
{
    dim3 grid(16, nb);
    k_fam_mark<T><<<grid, 256, 0, st>>>(f, rows, words);
    return 1;
}

template <typename T>
int fam_launch_compact(const FamArgs<T>& f, int nb, cudaStream_t st)
{
    k_fam_compact<T><<<nb, 1024, 0, st>>>(f);
    return 1;
}

template <typename T>
int fam_launch_rbm(const FamArgs<T>& f, int nb, cudaStream_t st)
{
    if (f.n_hidden <= 0) return 0;
    dim3 grid(8 * f.split, nb);
    k_fam_rbm<T><<<grid, 256, 2 * f.n_hidden * sizeof(T), st>>>(f);
    return 1;
}

template <typename T>
int fam_launch_rows(const FamArgs<T>& f, const RowSet& rows, int64_t grid, double* partial,
                    int64_t* span, double* partial_abs, cudaStream_t st)
{
    if (grid <= 0) return 0;
    if constexpr (std::is_same<T, float>::value) {
        if (f.D == 64) {
            k_fam_rows<T, 64, kFamRowsMB64><<<(unsigned)grid, kFamRows, 0, st>>>(f, rows, partial, span, partial_abs);
            return 1;
        }
        if (f.D == 32) {
            k_fam_rows<T, 32, kFamRowsMB64><<<(unsigned)grid, kFamRows, 0, st>>>(f, rows, partial, span, partial_abs);
            return 1;
        }
    }
    k_fam_rows<T, 0, 12><<<(unsigned)grid, kFamRows, 0, st>>>(f, rows, partial, span, partial_abs);
    return 1;
}

void fam_tc_images(const double* A, int K, int D, std::vector<unsigned char>& images, std::vector<int>& exps)
{
    const size_t blk = (size_t)4 * D * D;
    images.assign((size_t)2 * K * 4 * blk, 0);
    exps.assign((size_t)2 * K * 4, 0);
    for (int side = 0; side < 2; ++side)
        for (int t = 0; t < K; ++t)
            for (int sg = 0; sg < 4; ++sg) {
                const double* M = A + ((size_t)t * 4 + sg) * D * D;
                double mx = 0.0;
                for (size_t i = 0; i < (size_t)D * D; ++i) mx = std::max(mx, std::fabs(M[i]));
                int e = 0;
                if (mx > 0.0) std::frexp(mx, &e);
                const size_t id = ((size_t)side * K + t) * 4 + sg;
                exps[id] = e;
                const int kc = fam_tc_kc(D);
                const size_t chunk = (size_t)4 * D * kc;     // hi + lo of one reduction chunk
                for (int n = 0; n < D; ++n)
                    for (int k = 0; k < D; ++k) {
                        // B[n][k]: side 0 -> M[n][k] (y = M x), side 1 -> M[k][n] (y = x^T M)
                        const double m = std::ldexp(side == 0 ? M[(size_t)n * D + k] : M[(size_t)k * D + n], -e);
                        const float mf = (float)m;
                        const __half h = __float2half_rn(mf);
                        const __half l = __float2half_rn(mf - __half2float(h));
                        const int ck = k / kc, kk = k - ck * kc;
                        unsigned char* hi = images.data() + id * blk + (size_t)ck * chunk;
                        unsigned char* lo = hi + (size_t)2 * D * kc;
                        const size_t off = ((size_t)(n >> 3) * (kc >> 3) + (kk >> 3)) * 128 + (n & 7) * 16 + (kk & 7) * 2;
                        std::memcpy(hi + off, &h, 2);
                        std::memcpy(lo + off, &l, 2);
                    }
            }
}

#define NQS_FAM_INST(T)                                                                    \
    template int fam_launch_mark<T>(const FamArgs<T>&, const RowSet&, int, uint32_t*, cudaStream_t);  \
    template int fam_launch_compact<T>(const FamArgs<T>&, int, cudaStream_t);              \
    template int fam_launch_rbm<T>(const FamArgs<T>&, int, cudaStream_t);                  \
    template int fam_site_count<T>(const FamArgs<T>&, const SiteBufs&, int, cudaStream_t);  \
    template int fam_site_fill<T>(const FamArgs<T>&, const SiteBufs&, int, cudaStream_t);   \
    template int fam_site_step<T>(const FamArgs<T>&, const SiteBufs&, int, const int64_t*,  \
                                  int, cudaStream_t);                                       \
    template int fam_launch_rows<T>(const FamArgs<T>&, const RowSet&, int64_t, double*,    \
                                    int64_t*, double*, cudaStream_t);
NQS_FAM_INST(float)
NQS_FAM_INST(double)

}  // namespace nqs
