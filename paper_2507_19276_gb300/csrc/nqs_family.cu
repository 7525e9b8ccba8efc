// nqs_family.cu -- shared-prefix evaluation of the connected amplitudes of a
// chain tensor network (Eq. MPS-RNN-1D with v = 0).
//
// For a sample n and a connected m that changes the local states of the sorted
// sites s1 < s2 (< s3 (< s4)), psi(m) = R^T A_{K-1} ... A_0 l with the changed
// sites' matrices replaced. The product is re-associated so that partial
// products are shared between the many m of one n:
//   one-change left families  G_{s,a}(t) = A_t ... A_{s+1} A_s^{a} L_{s-1}, t >= s
//   one-change right families H_{s,a}(t) = R_{s+1} A_s^{a} A_{s-1} ... A_t,  t <= s
//   two-change left clusters  TL_{s1a1,s2a2}(t) = A_t ... A_{s2+1} A_{s2}^{a2} G_{s1,a1}(s2-1)
//   two-change right clusters TR_{sAaA,sBaB} = H_{sB,aB}(sA+1) A_{sA}^{aA}
// where A_t = A_t^{sigma_t(n)} and A_s^{a} is the a-th local state other than
// sigma_s(n). Then
//   2 sites: psi(m) = G_{s1,a1}(s2-1) . H_{s2,a2}(s2)
//   3 sites: psi(m) = G_{s1,a1}(s2-1) . TR_{s2a2,s3a3}
//   4 sites: psi(m) = TL_{s1a1,s2a2}(s3-1) . TR_{s3a3,s4a4}
// Every vector carries a power-of-two exponent; T is the arithmetic type.
#include "nqs_family.cuh"

namespace nqs {

// alternative index of local state `sg` at a site whose own state is `own`
__device__ __forceinline__ int alt_of(int sg, int own) { return sg - (sg > own ? 1 : 0); }
__device__ __forceinline__ int sig_of_alt(int a, int own) { return a + (a >= own ? 1 : 0); }

template <typename T>
__device__ __forceinline__ T tabs(T x) { return x < T(0) ? -x : x; }

// Block-wide: y_i = M x_i for vectors in shared memory; MT[b][a] = M[a][b].
template <typename T>
__device__ void mv_block(const T* __restrict__ MT, int D, const T* X, T* Y, int nv)
{
    const int a = threadIdx.x % D, g = threadIdx.x / D, G = blockDim.x / D;
    if (g >= G) return;
    for (int i = g * 4; i < nv; i += G * 4) {
        const int n4 = nv - i < 4 ? nv - i : 4;
        T acc[4] = {T(0), T(0), T(0), T(0)};
        for (int b = 0; b < D; ++b) {
            const T m = __ldg(MT + (size_t)b * D + a);
            #pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q < n4) acc[q] = fma(m, X[(size_t)(i + q) * D + b], acc[q]);
        }
        for (int q = 0; q < n4; ++q) Y[(size_t)(i + q) * D + a] = acc[q];
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

// ---------------------------------------------------------------------------
// F1: left and right family sweeps, one block per sample. L (or R) stays in
// shared memory; the families are read back from the tables in batches.
// ---------------------------------------------------------------------------

template <typename T>
__global__ void k_fam_sweep(FamArgs<T> f)
{
    extern __shared__ unsigned char smraw[];
    T* X = (T*)smraw;                           // [nmax][D]
    T* Y = X + (size_t)f.nmax * f.D;            // [nmax][D]
    int* eo = (int*)(Y + (size_t)f.nmax * f.D); // [nmax]
    int* pos = eo + f.nmax;                     // [nmax] table positions
    T* Lv = (T*)(pos + f.nmax);                 // [D] (aligned: nmax multiple of 4)
    __shared__ int eL;
    const int b = blockIdx.x, K = f.K, D = f.D;
    const int64_t s = f.s0 + b;
    const uint64_t na = f.samples[2 * s], nb = f.samples[2 * s + 1];
    for (int side = 0; side < 2; ++side) {
        T* Tb = (side == 0 ? f.G : f.H) + (size_t)b * 3 * K * K * D;
        int* Te = (side == 0 ? f.Ge : f.He) + (size_t)b * 3 * K * K;
        const T* Mats = side == 0 ? f.AT : f.A;   // column convention left, row vectors right
        for (int c = threadIdx.x; c < D; c += blockDim.x) Lv[c] = c == 0 ? T(1) : T(0);
        if (threadIdx.x == 0) eL = 0;
        __syncthreads();
        for (int step = 0; step < K; ++step) {
            const int t = side == 0 ? step : K - 1 - step;
            const int own = sigma_at(na, nb, t);
            // (a) the boundary vector and the three families that start at t
            for (int q = threadIdx.x; q < D; q += blockDim.x) X[q] = Lv[q];
            __syncthreads();
            for (int a = 0; a < 4; ++a) {
                const int sg = a == 3 ? own : sig_of_alt(a, own);
                mv_block<T>(Mats + ((size_t)t * 4 + sg) * D * D, D, X, Y + (size_t)a * D, 1);
            }
            __syncthreads();
            renorm_rows<T>(Y, D, 4, eo);
            __syncthreads();
            const int e_in = eL;
            const int eL_new = e_in + eo[3];
            for (int q = threadIdx.x; q < 3 * D; q += blockDim.x) {
                const int a = q / D, c = q - a * D;
                Tb[(((size_t)a * K + t) * K + t) * D + c] = Y[q];
            }
            for (int a = threadIdx.x; a < 3; a += blockDim.x) Te[((size_t)a * K + t) * K + t] = e_in + eo[a];
            for (int c = threadIdx.x; c < D; c += blockDim.x) Lv[c] = Y[3 * D + c];
            __syncthreads();
            if (threadIdx.x == 0) eL = eL_new;
            // (b) existing families: s < t (left) or s > t (right)
            const int nfam = 3 * step;
            for (int c0 = 0; c0 < nfam; c0 += f.nmax) {
                const int n = nfam - c0 < f.nmax ? nfam - c0 : f.nmax;
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    const int j = (c0 + i) / 3, a = (c0 + i) % 3;
                    const int sf = side == 0 ? j : K - 1 - j;
                    pos[i] = (a * K + sf) * K;     // + t later
                }
                __syncthreads();
                const int tprev = side == 0 ? t - 1 : t + 1;
                for (int q = threadIdx.x; q < n * D; q += blockDim.x) {
                    const int i = q / D, c = q - i * D;
                    X[q] = Tb[((size_t)pos[i] + tprev) * D + c];
                }
                __syncthreads();
                mv_block<T>(Mats + ((size_t)t * 4 + own) * D * D, D, X, Y, n);
                __syncthreads();
                renorm_rows<T>(Y, D, n, eo);
                __syncthreads();
                for (int q = threadIdx.x; q < n * D; q += blockDim.x) {
                    const int i = q / D, c = q - i * D;
                    Tb[((size_t)pos[i] + t) * D + c] = Y[q];
                }
                for (int i = threadIdx.x; i < n; i += blockDim.x)
                    Te[pos[i] + t] = Te[pos[i] + tprev] + eo[i];
                __syncthreads();
            }
        }
        if (side == 0 && threadIdx.x == 0) { f.pm[b] = (double)Lv[0]; f.pe[b] = eL; }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Row decomposition (shared by the marking and the evaluation passes)
// ---------------------------------------------------------------------------

struct RowParts {
    int nsite;           // 2, 3 or 4 changed sites
    int s[4], a[4];      // sites ascending and alternative indices
    uint64_t ma, mb;
};

__device__ __forceinline__ RowParts row_parts(const HamView& h, const OrbLists& L, uint64_t na,
                                              uint64_t nb, uint32_t rank)
{
    const Exc e = decode_rank(h, L, rank);
    RowParts r;
    uint64_t ma = na, mb = nb;
    flip(ma, mb, e.i); flip(ma, mb, e.a);
    if (e.kind == 2) { flip(ma, mb, e.j); flip(ma, mb, e.b); }
    uint64_t ch = (na ^ ma) | (nb ^ mb);
    r.nsite = 0;
    while (ch && r.nsite < 4) {
        const int p = __ffsll((long long)ch) - 1;
        r.s[r.nsite] = p;
        r.a[r.nsite] = alt_of(sigma_at(ma, mb, p), sigma_at(na, nb, p));
        ++r.nsite;
        ch &= ch - 1;
    }
    r.ma = ma;
    r.mb = mb;
    return r;
}

__device__ __forceinline__ int tl_key(int K, int s1, int a1, int s2, int a2)
{
    return ((s2 * K + s1) * 3 + a1) * 3 + a2;
}

__device__ __forceinline__ int tr_key(int K, int sA, int aA, int sB, int aB)
{
    return ((sA * K + sB) * 3 + aA) * 3 + aB;
}

// F2: mark the clusters the rows need (TL end site, TR use)
template <typename T>
__global__ void k_fam_mark(FamArgs<T> f, RowSet rows)
{
    __shared__ OrbLists lists;
    const int b = blockIdx.y;
    const int64_t s = f.s0 + b;
    const int64_t beg = rows.begin ? rows.begin[s] : s * rows.stride;
    const int64_t cnt = rows.count[s];
    const uint64_t na = f.samples[2 * s], nb = f.samples[2 * s + 1];
    if (threadIdx.x < 32) build_lists_warp(na, nb, f.h.K, lists, threadIdx.x);
    __syncthreads();
    const int K = f.K;
    const size_t nk = (size_t)K * K * 9;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < cnt;
         r += (int64_t)gridDim.x * blockDim.x) {
        const RowParts p = row_parts(f.h, lists, na, nb, rows.rank[beg + r]);
        if (p.nsite == 3) {
            f.tr_idx[(size_t)b * nk + tr_key(K, p.s[1], p.a[1], p.s[2], p.a[2])] = 1;
        } else if (p.nsite == 4) {
            atomicMax(&f.tl_end[(size_t)b * nk + tl_key(K, p.s[0], p.a[0], p.s[1], p.a[1])], p.s[2] - 1);
            f.tr_idx[(size_t)b * nk + tr_key(K, p.s[2], p.a[2], p.s[3], p.a[3])] = 1;
        }
    }
}

// F3: per-sample compaction of the marks: tl_idx[key] = entry offset of
// (cluster, t = s2) in the packed TL table (or -1), tr_idx[key] = TR row.
template <typename T>
__global__ void k_fam_compact(FamArgs<T> f)
{
    __shared__ int wt[32];
    const int b = blockIdx.x, K = f.K;
    const size_t nk = (size_t)K * K * 9;
    const int* te = f.tl_end + (size_t)b * nk;
    int* tl = f.tl_idx + (size_t)b * nk;
    int* tr = f.tr_idx + (size_t)b * nk;
    int carry_l = 0, carry_r = 0;
    for (size_t k0 = 0; k0 < nk; k0 += blockDim.x) {
        const size_t k = k0 + threadIdx.x;
        int cl = 0, cr = 0, end = -1, flag = 0, s2 = 0;
        if (k < nk) {
            end = te[k];
            flag = tr[k];
            s2 = (int)(k / 9) / K;
            cl = end >= 0 ? end - s2 + 1 : 0;
            cr = flag > 0 ? 1 : 0;
        }
        // two block scans (lengths, flags)
        int v = cl;
        for (int o = 1; o < 32; o <<= 1) { int u = __shfl_up_sync(kFull, v, o); if ((threadIdx.x & 31) >= o) v += u; }
        if ((threadIdx.x & 31) == 31) wt[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x < 32) {
            int w = threadIdx.x < (blockDim.x >> 5) ? wt[threadIdx.x] : 0;
            for (int o = 1; o < 32; o <<= 1) { int u = __shfl_up_sync(kFull, w, o); if (threadIdx.x >= o) w += u; }
            wt[threadIdx.x] = w;
        }
        __syncthreads();
        const int incl_l = v + ((threadIdx.x >> 5) ? wt[(threadIdx.x >> 5) - 1] : 0);
        const int tot_l = wt[(blockDim.x >> 5) - 1];
        __syncthreads();
        v = cr;
        for (int o = 1; o < 32; o <<= 1) { int u = __shfl_up_sync(kFull, v, o); if ((threadIdx.x & 31) >= o) v += u; }
        if ((threadIdx.x & 31) == 31) wt[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x < 32) {
            int w = threadIdx.x < (blockDim.x >> 5) ? wt[threadIdx.x] : 0;
            for (int o = 1; o < 32; o <<= 1) { int u = __shfl_up_sync(kFull, w, o); if (threadIdx.x >= o) w += u; }
            wt[threadIdx.x] = w;
        }
        __syncthreads();
        const int incl_r = v + ((threadIdx.x >> 5) ? wt[(threadIdx.x >> 5) - 1] : 0);
        const int tot_r = wt[(blockDim.x >> 5) - 1];
        __syncthreads();
        if (k < nk) {
            tl[k] = end >= 0 ? carry_l + incl_l - cl : -1;
            tr[k] = flag > 0 ? carry_r + incl_r - 1 : -1;
        }
        carry_l += tot_l;
        carry_r += tot_r;
    }
    if (threadIdx.x == 0) { f.tl_total[b] = carry_l; f.tr_total[b] = carry_r; }
}

// F4a: TR_{sA aA, sB aB} = H_{sB,aB}(sA+1) A_{sA}^{aA}, one block per sample,
// sites sA ascending; the needed (sB, aB) of a (sA, aA) are gathered first.
template <typename T>
__global__ void k_fam_tr(FamArgs<T> f)
{
    extern __shared__ unsigned char smraw[];
    T* X = (T*)smraw;
    T* Y = X + (size_t)f.nmax * f.D;
    int* eo = (int*)(Y + (size_t)f.nmax * f.D);
    int* ei = eo + f.nmax;
    int* dst = ei + f.nmax;
    __shared__ int cnt;
    const int b = blockIdx.x, K = f.K, D = f.D;
    const int64_t s = f.s0 + b;
    const uint64_t na = f.samples[2 * s], nb = f.samples[2 * s + 1];
    const size_t nk = (size_t)K * K * 9;
    const int* tr = f.tr_idx + (size_t)b * nk;
    const T* H = f.H + (size_t)b * 3 * K * K * D;
    const int* He = f.He + (size_t)b * 3 * K * K;
    T* TR = f.TR + (size_t)f.tr_base[b] * D;
    int* TRe = f.TRe + f.tr_base[b];
    for (int sA = 0; sA < K - 1; ++sA) {
        const int own = sigma_at(na, nb, sA);
        for (int aA = 0; aA < 3; ++aA) {
            // candidates (sB, aB), sB > sA, processed in batches of nmax
            const int ncand = 3 * (K - 1 - sA);
            for (int c0 = 0; c0 < ncand; c0 += f.nmax) {
                if (threadIdx.x == 0) cnt = 0;
                __syncthreads();
                for (int c = c0 + threadIdx.x; c < ncand && c < c0 + f.nmax; c += blockDim.x) {
                    const int sB = sA + 1 + c / 3, aB = c % 3;
                    const int idx = tr[tr_key(K, sA, aA, sB, aB)];
                    if (idx >= 0) {
                        const int slot = atomicAdd(&cnt, 1);
                        dst[slot] = idx;
                        ei[slot] = ((aB * K + sB) * K + sA + 1);   // H table position
                    }
                }
                __syncthreads();
                const int n = cnt;
                if (n == 0) { __syncthreads(); continue; }
                for (int q = threadIdx.x; q < n * D; q += blockDim.x) {
                    const int i = q / D, cc = q - i * D;
                    X[q] = H[(size_t)ei[i] * D + cc];
                }
                __syncthreads();
                mv_block<T>(f.A + ((size_t)sA * 4 + sig_of_alt(aA, own)) * D * D, D, X, Y, n);
                __syncthreads();
                renorm_rows<T>(Y, D, n, eo);
                __syncthreads();
                for (int q = threadIdx.x; q < n * D; q += blockDim.x) {
                    const int i = q / D, cc = q - i * D;
                    TR[(size_t)dst[i] * D + cc] = Y[q];
                }
                for (int i = threadIdx.x; i < n; i += blockDim.x) TRe[dst[i]] = eo[i] + He[ei[i]];
                __syncthreads();
            }
        }
    }
}

// F4b: TL clusters: created at t = s2 from G_{s1,a1}(s2-1), propagated with
// A_t^{sigma_t(n)} up to their last use; every step is stored.
template <typename T>
__global__ void k_fam_tl(FamArgs<T> f)
{
    extern __shared__ unsigned char smraw[];
    T* X = (T*)smraw;
    T* Y = X + (size_t)f.nmax * f.D;
    int* eo = (int*)(Y + (size_t)f.nmax * f.D);
    int* ei = eo + f.nmax;
    int* src = ei + f.nmax;
    int* dst = src + f.nmax;
    __shared__ int cnt;
    const int b = blockIdx.x, K = f.K, D = f.D;
    const int64_t s = f.s0 + b;
    const uint64_t na = f.samples[2 * s], nb = f.samples[2 * s + 1];
    const size_t nk = (size_t)K * K * 9;
    const int* tl = f.tl_idx + (size_t)b * nk;
    const int* tl_end = f.tl_end + (size_t)b * nk;
    const T* G = f.G + (size_t)b * 3 * K * K * D;
    const int* Ge = f.Ge + (size_t)b * 3 * K * K;
    T* TL = f.TL + (size_t)f.tl_base[b] * D;
    int* TLe = f.TLe + f.tl_base[b];
    for (int t = 1; t < K; ++t) {
        const int own = sigma_at(na, nb, t);
        // (1) creation at s2 = t from G_{s1,a1}(t-1), per alternative a2
        for (int a2 = 0; a2 < 3; ++a2) {
            const int ncand = 3 * t;      // (s1 < t, a1)
            for (int c0 = 0; c0 < ncand; c0 += f.nmax) {
                if (threadIdx.x == 0) cnt = 0;
                __syncthreads();
                for (int c = c0 + threadIdx.x; c < ncand && c < c0 + f.nmax; c += blockDim.x) {
                    const int s1 = c / 3, a1 = c % 3;
                    const int key = tl_key(K, s1, a1, t, a2);
                    const int off = tl[key];
                    if (off >= 0) {
                        const int slot = atomicAdd(&cnt, 1);
                        dst[slot] = off;
                        src[slot] = (a1 * K + s1) * K + (t - 1);
                    }
                }
                __syncthreads();
                const int n = cnt;
                if (n == 0) { __syncthreads(); continue; }
                for (int q = threadIdx.x; q < n * D; q += blockDim.x) {
                    const int i = q / D, cc = q - i * D;
                    X[q] = G[(size_t)src[i] * D + cc];
                }
                __syncthreads();
                mv_block<T>(f.AT + ((size_t)t * 4 + sig_of_alt(a2, own)) * D * D, D, X, Y, n);
                __syncthreads();
                renorm_rows<T>(Y, D, n, eo);
                __syncthreads();
                for (int q = threadIdx.x; q < n * D; q += blockDim.x) {
                    const int i = q / D, cc = q - i * D;
                    TL[(size_t)dst[i] * D + cc] = Y[q];
                }
                for (int i = threadIdx.x; i < n; i += blockDim.x) TLe[dst[i]] = eo[i] + Ge[src[i]];
                __syncthreads();
            }
        }
        // (2) propagation of clusters with s2 < t <= end
        const int nkeys_t = t * K * 9;            // keys with s2 < t come first (s2-major)
        for (int c0 = 0; c0 < nkeys_t; c0 += f.nmax) {
            if (threadIdx.x == 0) cnt = 0;
            __syncthreads();
            for (int c = c0 + threadIdx.x; c < nkeys_t && c < c0 + f.nmax; c += blockDim.x) {
                const int off = tl[c];
                if (off < 0) continue;
                const int s2 = (c / 9) / K;
                if (t > tl_end[c]) continue;
                const int slot = atomicAdd(&cnt, 1);
                src[slot] = off + (t - 1 - s2);
                dst[slot] = off + (t - s2);
            }
            __syncthreads();
            const int n = cnt;
            if (n == 0) { __syncthreads(); continue; }
            for (int q = threadIdx.x; q < n * D; q += blockDim.x) {
                const int i = q / D, cc = q - i * D;
                X[q] = TL[(size_t)src[i] * D + cc];
            }
            __syncthreads();
            mv_block<T>(f.AT + ((size_t)t * 4 + own) * D * D, D, X, Y, n);
            __syncthreads();
            renorm_rows<T>(Y, D, n, eo);
            __syncthreads();
            for (int q = threadIdx.x; q < n * D; q += blockDim.x) {
                const int i = q / D, cc = q - i * D;
                TL[(size_t)dst[i] * D + cc] = Y[q];
            }
            for (int i = threadIdx.x; i < n; i += blockDim.x) TLe[dst[i]] = eo[i] + TLe[src[i]];
            __syncthreads();
        }
    }
}

// F5: one thread per row: psi(m) as a dot product of a left state and a right
// covector, the RBM ratio, coefficient x ratio; block partial sums in order.
constexpr int kFamRows = 128;
constexpr int kFamMaxHidden = 512;

template <typename T>
__global__ void __launch_bounds__(kFamRows) k_fam_rows(FamArgs<T> f, RowSet rows, double* partial,
                                                       int64_t* span)
{
    __shared__ OrbLists lists;
    __shared__ double contrib[kFamRows];
    __shared__ T tanh_s[kFamMaxHidden];
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
    const int NH = f.n_hidden;
    if (threadIdx.x < 32) build_lists_warp(na, nb, f.h.K, lists, threadIdx.x);
    for (int k = threadIdx.x; k < NH; k += blockDim.x) tanh_s[k] = (T)tanh(f.theta[s * NH + k]);
    __syncthreads();
    const size_t nk = (size_t)K * K * 9;
    double val = 0.0;
    int nmv = 0;
    if ((int)threadIdx.x < nr) {
        const RowParts p = row_parts(f.h, lists, na, nb, rows.rank[r0 + threadIdx.x]);
        const T* G = f.G + (size_t)b * 3 * K * K * D;
        const int* Ge = f.Ge + (size_t)b * 3 * K * K;
        const T* H = f.H + (size_t)b * 3 * K * K * D;
        const int* He = f.He + (size_t)b * 3 * K * K;
        const T* Lv;
        const T* Rv;
        int eL, eR;
        if (p.nsite == 4) {
            const int key = tl_key(K, p.s[0], p.a[0], p.s[1], p.a[1]);
            const int off = f.tl_idx[(size_t)b * nk + key] + (p.s[2] - 1 - p.s[1]);
            const int ti = f.tr_idx[(size_t)b * nk + tr_key(K, p.s[2], p.a[2], p.s[3], p.a[3])];
            Lv = f.TL + ((size_t)f.tl_base[b] + off) * D;
            eL = f.TLe[f.tl_base[b] + off];
            Rv = f.TR + ((size_t)f.tr_base[b] + ti) * D;
            eR = f.TRe[f.tr_base[b] + ti];
        } else {
            const size_t gi = ((size_t)p.a[0] * K + p.s[0]) * K + p.s[1] - 1;
            Lv = G + gi * D;
            eL = Ge[gi];
            if (p.nsite == 2) {
                const size_t hi2 = ((size_t)p.a[1] * K + p.s[1]) * K + p.s[1];
                Rv = H + hi2 * D;
                eR = He[hi2];
            } else {
                const int ti = f.tr_idx[(size_t)b * nk + tr_key(K, p.s[1], p.a[1], p.s[2], p.a[2])];
                Rv = f.TR + ((size_t)f.tr_base[b] + ti) * D;
                eR = f.TRe[f.tr_base[b] + ti];
            }
        }
        nmv = p.s[p.nsite - 1] - p.s[0] + 1;
        // dot product with error-free product / sum transformations
        T sum = T(0), comp = T(0);
        for (int c = 0; c < D; ++c) {
            const T x = Lv[c], y = Rv[c];
            const T pr = x * y;
            const T pe = fma(x, y, -pr);
            const T t = sum + pr;
            const T z = t - sum;
            comp += ((sum - (t - z)) + (pr - z)) + pe;
            sum = t;
        }
        const double dot = (double)sum + (double)comp;
        double ratio = ldexp(dot / f.pm[b], eL + eR - f.pe[b]);
        // RBM: prod_k cosh(theta_k + d_k) / cosh(theta_k) = prod_k (1 + (cosh d_k - 1) + tanh(theta_k) sinh d_k)
        if (NH > 0) {
            int fs[4], sg[4], nf = 0;
            uint64_t da = na ^ p.ma, db = nb ^ p.mb;
            while (da && nf < 4) { const int q = __ffsll((long long)da) - 1; fs[nf] = 2 * q; sg[nf] = ((p.ma >> q) & 1ull) ? 1 : -1; ++nf; da &= da - 1; }
            while (db && nf < 4) { const int q = __ffsll((long long)db) - 1; fs[nf] = 2 * q + 1; sg[nf] = ((p.mb >> q) & 1ull) ? 1 : -1; ++nf; db &= db - 1; }
            T lsum = T(0);
            for (int k = 0; k < NH; ++k) {
                const T* Wk = f.W + (size_t)k * 2 * K;
                T d = T(0);
                for (int q = 0; q < nf; ++q) d += sg[q] > 0 ? Wk[fs[q]] : -Wk[fs[q]];
                const T em = expm1(d);                       // e^d - 1
                const T inv = T(1) / (T(1) + em);            // e^-d
                const T sh = T(0.5) * em * (T(1) + inv);      // sinh d
                const T c1 = T(0.5) * em * em * inv;          // cosh d - 1
                lsum += log1p(c1 + tanh_s[k] * sh);
            }
            ratio *= exp((double)lsum);
        }
        val = rows.coef[r0 + threadIdx.x] * ratio;
    }
    contrib[threadIdx.x] = val;
    __shared__ int spsum[kFamRows];
    spsum[threadIdx.x] = nmv;
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = 0.0;
        int64_t sp = 0;
        for (int r = 0; r < nr; ++r) { acc += contrib[r]; sp += spsum[r]; }
        partial[blk] = acc;
        if (span) span[blk] = sp;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

template <typename T>
int fam_launch_sweep(const FamArgs<T>& f, int nb, cudaStream_t st)
{
    const size_t smem = (size_t)(2 * f.nmax + 1) * f.D * sizeof(T) + 2 * f.nmax * sizeof(int);
    cudaFuncSetAttribute(k_fam_sweep<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_fam_sweep<T><<<nb, f.threads, smem, st>>>(f);
    return 1;
}

template <typename T>
int fam_launch_mark(const FamArgs<T>& f, const RowSet& rows, int nb, cudaStream_t st)
{
    dim3 grid(16, nb);
    k_fam_mark<T><<<grid, 256, 0, st>>>(f, rows);
    return 1;
}

template <typename T>
int fam_launch_compact(const FamArgs<T>& f, int nb, cudaStream_t st)
{
    k_fam_compact<T><<<nb, 1024, 0, st>>>(f);
    return 1;
}

template <typename T>
int fam_launch_tables(const FamArgs<T>& f, int nb, cudaStream_t st)
{
    const size_t smem = (size_t)2 * f.nmax * f.D * sizeof(T) + 4 * f.nmax * sizeof(int);
    cudaFuncSetAttribute(k_fam_tr<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(k_fam_tl<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_fam_tr<T><<<nb, f.threads, smem, st>>>(f);
    k_fam_tl<T><<<nb, f.threads, smem, st>>>(f);
    return 2;
}

template <typename T>
int fam_launch_rows(const FamArgs<T>& f, const RowSet& rows, int64_t grid, double* partial,
                    int64_t* span, cudaStream_t st)
{
    if (grid <= 0) return 0;
    k_fam_rows<T><<<(unsigned)grid, kFamRows, 0, st>>>(f, rows, partial, span);
    return 1;
}

#define NQS_FAM_INST(T)                                                                    \
    template int fam_launch_sweep<T>(const FamArgs<T>&, int, cudaStream_t);                \
    template int fam_launch_mark<T>(const FamArgs<T>&, const RowSet&, int, cudaStream_t);  \
    template int fam_launch_compact<T>(const FamArgs<T>&, int, cudaStream_t);              \
    template int fam_launch_tables<T>(const FamArgs<T>&, int, cudaStream_t);               \
    template int fam_launch_rows<T>(const FamArgs<T>&, const RowSet&, int64_t, double*,    \
                                    int64_t*, cudaStream_t);
NQS_FAM_INST(float)
NQS_FAM_INST(double)

}  // namespace nqs
