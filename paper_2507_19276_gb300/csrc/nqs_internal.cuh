// nqs_internal.cuh -- device-side building blocks of the local-energy path.
//
// Excitation decoding by closed-form unranking, fermionic phases by popcount,
// Slater-Condon matrix elements (Eq. Ham, Sec. 3), integer remainder weights
// and Philox4x64-10 draws (Sec. 2.4). Everything here works on packed uint64
// determinants [alpha word, beta word]; spin orbital s = 2p + spin.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nqs {

constexpr int kMaxOrb = 64;
constexpr unsigned kFull = 0xffffffffu;

// q = n / d for n * d < 2^32 using one wide multiply (m = ceil(2^32 / d)).
struct FastDiv {
    uint64_t m;
    uint32_t d;
};

inline FastDiv make_fastdiv(uint32_t d)
{
    FastDiv f;
    f.d = d ? d : 1;
    f.m = ((1ull << 32) + f.d - 1) / f.d;
    return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f)
{
    return (uint32_t)(((uint64_t)n * f.m) >> 32);
}

// Problem description passed by value to every kernel.
struct HamView {
    int K, na, nb;
    int no[2], nv[2];
    uint32_t blk[6];          // block starts: Sa, Sb, Daa, Dbb, Dab, end (= n_conn)
    FastDiv div_nv[2];        // / nv_sigma
    FastDiv div_vpair[2];     // / C(nv_sigma, 2)
    FastDiv div_sb;           // / (no_b * nv_b)
    uint32_t n_conn;
    int bitlen_nconn;
    const double* h1e;        // [K][K]
    const double* eri;        // [K^4] (pq|rs)
    const uint16_t* pairs;    // unranking tables, see pair_table()
    uint32_t pair_off[4];     // offsets of the occ-a, occ-b, vir-a, vir-b tables
    double e_core;
};

// Per-determinant orbital lists: positions of occupied / empty orbitals, and
// for each listed orbital the number of occupied spin orbitals of n with a
// smaller interleaved index (the count a creation or annihilation operator
// there picks up in n).
struct OrbLists {
    uint8_t occ[2][kMaxOrb];
    uint8_t vir[2][kMaxOrb];
    uint8_t ocb[2][kMaxOrb];
    uint8_t vcb[2][kMaxOrb];
};

// Spin-orbital excitation: i (,j) emptied, a (,b) filled; m = a+_a a+_b a_j a_i n.
struct Exc {
    int kind;          // 1 single, 2 double
    int i, j, a, b;    // spin-orbital indices 2p+spin (j, b = -1 for singles)
    int odd;           // parity of the fermionic phase of <m| a+_a a+_b a_j a_i |n>
};

__device__ __forceinline__ uint64_t low_mask(int p)
{
    return p >= 64 ? ~0ull : ((1ull << p) - 1ull);
}

// Number of occupied spin orbitals with interleaved index < s in (wa, wb).
__device__ __forceinline__ int count_below(uint64_t wa, uint64_t wb, int s)
{
    const int p = s >> 1;
    if (s & 1) return __popcll(wa & low_mask(p + 1)) + __popcll(wb & low_mask(p));
    return __popcll(wa & low_mask(p)) + __popcll(wb & low_mask(p));
}

__device__ __forceinline__ void flip(uint64_t& wa, uint64_t& wb, int s)
{
    if (s & 1) wb ^= 1ull << (s >> 1);
    else wa ^= 1ull << (s >> 1);
}

// Fill `L` for determinant (wa, wb); called by one warp (lanes cover 2 sites each).
__device__ __forceinline__ void build_lists_warp(uint64_t wa, uint64_t wb, int K, OrbLists& L,
                                                 int lane)
{
    for (int p = lane; p < K; p += 32) {
        for (int sp = 0; sp < 2; ++sp) {
            uint64_t w = sp ? wb : wa;
            int below = __popcll(w & low_mask(p));
            const uint8_t c = (uint8_t)count_below(wa, wb, 2 * p + sp);
            if ((w >> p) & 1ull) { L.occ[sp][below] = (uint8_t)p; L.ocb[sp][below] = c; }
            else { L.vir[sp][p - below] = (uint8_t)p; L.vcb[sp][p - below] = c; }
        }
    }
}

// A sample the enumeration may decode: N_alpha and N_beta electrons and no
// occupied orbital at or above K. Kernels that run before the host has read
// the validation error word skip other samples, so the orbital lists they
// decode from are always fully written (their results are discarded with
// the call's NQS_ERR_INVALID_ARG).
__device__ __forceinline__ bool sample_ok(const HamView& h, uint64_t na, uint64_t nb)
{
    const uint64_t outside = h.K >= 64 ? 0ull : ~((1ull << h.K) - 1ull);
    return !((na | nb) & outside) && __popcll(na) == h.na && __popcll(nb) == h.nb;
}

// The operators of a double act on n in the order a_i, a_j, a+_b, a+_a; each
// picks up the occupied spin orbitals below it in the determinant it meets,
// which differs from n by the operators already applied:
//   c = cb(i) + cb(j) - [i<j] + cb(b) - [i<b] - [j<b] + cb(a) - [i<a] - [j<a] + [b<a]
// with cb() counted in n. Only the parity matters, so the signs of the order
// terms drop out. (A single: c = cb(i) + cb(a) - [i<a].)
__device__ __forceinline__ int double_order(const Exc& e)
{
    return (e.i < e.j) + (e.i < e.b) + (e.j < e.b) + (e.i < e.a) + (e.j < e.a) + (e.b < e.a);
}

// Canonical rank -> excitation (with its phase parity; kPhase = false leaves
// odd = 0 for callers that need only |H|, such as the count pass).
template <bool kPhase = true>
__device__ __forceinline__ Exc decode_rank(const HamView& h, const OrbLists& L, uint32_t r)
{
    Exc e;
    e.odd = 0;
    if (r < h.blk[2]) {                         // singles
        int sp = r >= h.blk[1];
        uint32_t x = r - h.blk[sp];
        uint32_t io = fdiv(x, h.div_nv[sp]);
        uint32_t ao = x - io * h.nv[sp];
        e.kind = 1;
        e.i = 2 * L.occ[sp][io] + sp;
        e.a = 2 * L.vir[sp][ao] + sp;
        e.j = e.b = -1;
        if (kPhase) e.odd = (L.ocb[sp][io] + L.vcb[sp][ao] + (e.i < e.a)) & 1;
    } else if (r < h.blk[4]) {                  // same-spin doubles
        int sp = r >= h.blk[3];
        uint32_t x = r - h.blk[2 + sp];
        uint32_t po = fdiv(x, h.div_vpair[sp]);
        uint32_t pv = x - po * (uint32_t)h.div_vpair[sp].d;
        uint16_t to = h.pairs[h.pair_off[sp] + po];
        uint16_t tv = h.pairs[h.pair_off[2 + sp] + pv];
        e.kind = 2;
        e.i = 2 * L.occ[sp][to & 0xff] + sp;
        e.j = 2 * L.occ[sp][to >> 8] + sp;
        e.a = 2 * L.vir[sp][tv & 0xff] + sp;
        e.b = 2 * L.vir[sp][tv >> 8] + sp;
        if (kPhase)
            e.odd = (L.ocb[sp][to & 0xff] + L.ocb[sp][to >> 8] + L.vcb[sp][tv & 0xff] +
                     L.vcb[sp][tv >> 8] + double_order(e)) & 1;
    } else {                                    // alpha-beta doubles
        uint32_t x = r - h.blk[4];
        uint32_t ia = fdiv(x, h.div_sb);
        uint32_t jb = x - ia * (uint32_t)h.div_sb.d;
        uint32_t io = fdiv(ia, h.div_nv[0]);
        uint32_t ao = ia - io * h.nv[0];
        uint32_t jo = fdiv(jb, h.div_nv[1]);
        uint32_t bo = jb - jo * h.nv[1];
        e.kind = 2;
        e.i = 2 * L.occ[0][io];
        e.a = 2 * L.vir[0][ao];
        e.j = 2 * L.occ[1][jo] + 1;
        e.b = 2 * L.vir[1][bo] + 1;
        if (kPhase)
            e.odd = (L.ocb[0][io] + L.vcb[0][ao] + L.ocb[1][jo] + L.vcb[1][bo] + double_order(e)) & 1;
    }
    return e;
}

// (pq|rs): the table keeps the last two indices swapped, [p][q][s][r], so that
// the doubles' reads (pq|rs) over consecutive virtual orbitals r of one warp
// fall on consecutive words
__device__ __forceinline__ double eri_at(const HamView& h, int p, int q, int r, int s)
{
    const uint32_t K = (uint32_t)h.K;          // K <= 64: K^4 <= 2^24
    return __ldg(h.eri + ((((uint32_t)p * K + (uint32_t)q) * K + (uint32_t)s) * K + (uint32_t)r));
}

// <m|H|n> for m = gamma a+_a (a+_b a_j) a_i |n>; writes m and the phase bit
// (e.odd, from decode_rank). Singles: F = h_ai + sum_{common occ s'} (ai|jj) -
// sum_{common occ s', same spin} (aj|ji), added in ascending s'. Doubles:
// (ai|bj) - [same spin] (aj|bi).
__device__ __forceinline__ double matrix_element(const HamView& h, uint64_t na, uint64_t nb,
                                                 const Exc& e, uint64_t& ma, uint64_t& mb,
                                                 int& odd)
{
    uint64_t wa = na, wb = nb;
    flip(wa, wb, e.i);
    flip(wa, wb, e.a);
    double v;
    const int I = e.i >> 1, A = e.a >> 1;
    if (e.kind == 1) {
        v = __ldg(h.h1e + A * h.K + I);
        // Coulomb part over common occupied spin orbitals, ascending s' = 2p+spin
        const uint64_t ca = (e.i & 1) ? na : (na & ~(1ull << I));
        const uint64_t cb = (e.i & 1) ? (nb & ~(1ull << I)) : nb;
        for (int p = 0; p < h.K; ++p) {
            if ((ca >> p) & 1ull) v = v + eri_at(h, A, I, p, p);
            if ((cb >> p) & 1ull) v = v + eri_at(h, A, I, p, p);
        }
        const uint64_t cs = (e.i & 1) ? cb : ca;
        for (int p = 0; p < h.K; ++p)
            if ((cs >> p) & 1ull) v = v - eri_at(h, A, p, p, I);
    } else {
        flip(wa, wb, e.j);
        flip(wa, wb, e.b);
        const int J = e.j >> 1, B = e.b >> 1;
        v = eri_at(h, A, I, B, J);
        if ((e.i & 1) == (e.j & 1)) v = v - eri_at(h, A, J, B, I);
    }
    ma = wa;
    mb = wb;
    odd = e.odd;
    // the phase as a sign-bit flip (integer ALU, not the FP64 pipe)
    return __longlong_as_double(__double_as_longlong(v) ^ ((long long)odd << 63));
}

// |H| >= eps on the bit patterns (eps finite, >= 0; H not NaN).
__device__ __forceinline__ bool is_det(double H, uint64_t eps_bits)
{
    return ((uint64_t)__double_as_longlong(H) & 0x7fffffffffffffffull) >= eps_bits;
}

// ceil(|H| * 2^shift) in exact integer arithmetic on the IEEE fields.
__device__ __forceinline__ uint64_t weight_of(double H, int shift)
{
    const uint64_t bits = (uint64_t)__double_as_longlong(H) & 0x7fffffffffffffffull;
    if (bits == 0) return 0;
    const int ef = (int)(bits >> 52);
    const uint64_t frac = bits & ((1ull << 52) - 1ull);
    const uint64_t M = ef ? (frac | (1ull << 52)) : frac;
    const int E = (ef ? ef - 1075 : -1074) + shift;   // value = M * 2^E
    if (E >= 0) return M << E;
    if (E <= -64) return 1;
    const int s = -E;
    const uint64_t q = M >> s;
    return q + ((M & ((1ull << s) - 1ull)) != 0 ? 1ull : 0ull);
}

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): first output word for
// counter (c0, c1, c2, 0) and key (k0, 0).
__device__ __forceinline__ uint64_t philox_first4(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t k0)
{
    uint64_t x0 = c0, x1 = c1, x2 = c2, x3 = 0, k1 = 0;
    #pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B97F4A7C15ull; k1 += 0xBB67AE8584CAA73Bull; }
        const uint64_t lo0 = 0xD2E7470EE14C6C93ull * x0, hi0 = __umul64hi(0xD2E7470EE14C6C93ull, x0);
        const uint64_t lo1 = 0xCA5A826395121157ull * x2, hi1 = __umul64hi(0xCA5A826395121157ull, x2);
        const uint64_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
        x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
    }
    return x0;
}

// The same with counter (c0, c1, 0, 0): the draws of the stochastic part.
__device__ __forceinline__ uint64_t philox_first(uint64_t c0, uint64_t c1, uint64_t k0)
{
    uint64_t x0 = c0, x1 = c1, x2 = 0, x3 = 0, k1 = 0;
    #pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B97F4A7C15ull; k1 += 0xBB67AE8584CAA73Bull; }
        const uint64_t lo0 = 0xD2E7470EE14C6C93ull * x0, hi0 = __umul64hi(0xD2E7470EE14C6C93ull, x0);
        const uint64_t lo1 = 0xCA5A826395121157ull * x2, hi1 = __umul64hi(0xCA5A826395121157ull, x2);
        const uint64_t y0 = hi1 ^ x1 ^ k0, y2 = hi0 ^ x3 ^ k1;
        x0 = y0; x1 = lo1; x2 = y2; x3 = lo0;
    }
    return x0;
}

// Local state sigma_p of a determinant.
__device__ __forceinline__ int sigma_at(uint64_t wa, uint64_t wb, int p)
{
    return (int)((wa >> p) & 1ull) + 2 * (int)((wb >> p) & 1ull);
}

// Warp reductions.
// Exact warp sum of 64-bit values whose total stays below 2^64, on every
// lane: three 24-bit slices summed by the warp-reduce unit (slice sums < 2^29).
__device__ __forceinline__ uint64_t warp_sum_sliced(uint64_t v)
{
    const unsigned s0 = __reduce_add_sync(kFull, (unsigned)(v & 0xFFFFFFu));
    const unsigned s1 = __reduce_add_sync(kFull, (unsigned)((v >> 24) & 0xFFFFFFu));
    const unsigned s2 = __reduce_add_sync(kFull, (unsigned)(v >> 48));
    return (uint64_t)s0 + ((uint64_t)s1 << 24) + ((uint64_t)s2 << 48);
}

// The same for v < 2^48 (the remainder weights when n_conn >= 2^14, each at
// most 2^(62 - bitlen(n_conn))): two 24-bit slices.
__device__ __forceinline__ uint64_t warp_sum_sliced2(uint64_t v)
{
    const unsigned s0 = __reduce_add_sync(kFull, (unsigned)(v & 0xFFFFFFu));
    const unsigned s1 = __reduce_add_sync(kFull, (unsigned)(v >> 24));
    return (uint64_t)s0 + ((uint64_t)s1 << 24);
}

__device__ __forceinline__ double warp_sum_f64(double v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ double warp_max_f64(double v)
{
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// Inclusive scan of a uint64 across the warp.
__device__ __forceinline__ uint64_t warp_incl_scan_u64(uint64_t v, int lane)
{
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// log(2 cosh x) without overflow.
__device__ __forceinline__ double log2cosh(double x)
{
    const double ax = fabs(x);
    return ax + log1p(exp(-2.0 * ax));
}

// Device error word: the first failing sample index (or a code) is kept.
struct DevError {
    int code;          // 0 ok, else nqs_status
    int detail;        // which check
    long long index;   // offending index
};

__device__ __forceinline__ void report(DevError* err, int code, int detail, long long idx)
{
    if (atomicCAS(&err->code, 0, code) == 0) {
        err->detail = detail;
        err->index = idx;
    }
}

}  // namespace nqs
