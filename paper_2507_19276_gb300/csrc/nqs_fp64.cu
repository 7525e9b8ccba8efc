// nqs_fp64.cu -- the FP64 ("plain") form of the ansatz on CUDA cores.
//
// psi = psi_TN * f: psi_TN from Eq. (MPS-RNN-1D) with v = 0 (chain) or
// Eq. (bdg-rnn-update) without the tensor term (graph), f the RBM correlator
// of Eq. (RBM) in 2cosh form. Every vector carries a power-of-two exponent so
// that long products neither overflow nor underflow; the scaling is exact.
//
// Environments (per sample n): left states L_t = A_t^{s_t(n)} ... A_0 l and
// right covectors R_t = r^T A_{K-1} ... A_t (chain), forward states h_i(n) and
// adjoints g_i(n) = d psi_TN / d h_i (graph). An amplitude psi(m) for m that
// differs from n on sites p..q is R_{q+1} A_q^{s_q(m)} ... A_p^{s_p(m)} L_{p-1}
// (chain), or the graph recursion re-run from the first changed vertex p with
// the stored h_j(n), j < p.
#include "nqs_kernels.cuh"

namespace nqs {

// ---------------------------------------------------------------------------
// block helpers
// ---------------------------------------------------------------------------

__device__ double block_max_abs(const double* v, int n, double* sh)
{
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(v[i]));
    m = warp_max_f64(m);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, sh[w]);
        sh[32] = r;
    }
    __syncthreads();
    double r = sh[32];
    __syncthreads();
    return r;
}

// Scale v (length n, in shared memory) by 2^-e so that max|v| is in [0.5, 1).
__device__ int block_renorm(double* v, int n, double* sh)
{
    const double m = block_max_abs(v, n, sh);
    if (m == 0.0) return 0;
    int e;
    frexp(m, &e);
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = ldexp(v[i], -e);
    __syncthreads();
    return e;
}

__device__ __forceinline__ int warp_renorm(double* v, int n, int lane)
{
    double m = 0.0;
    for (int i = lane; i < n; i += 32) m = fmax(m, fabs(v[i]));
    m = warp_max_f64(m);
    if (m == 0.0) return 0;
    int e;
    frexp(m, &e);
    for (int i = lane; i < n; i += 32) v[i] = ldexp(v[i], -e);
    return e;
}

__device__ __forceinline__ const double* tens(const double* base, int e, int sg, int D)
{
    return base + ((size_t)e * 4 + sg) * D * D;
}

// ---------------------------------------------------------------------------
// Environments, psi(n), RBM angles, H_nn
// ---------------------------------------------------------------------------

__global__ void k_env_fp64(EnvArgs a)
{
    extern __shared__ double sm[];
    const int D = a.an.D, K = a.an.K;
    double* x = sm;
    double* y = sm + D;
    double* sh = sm + 2 * D;            // 33 doubles
    int* gx = (int*)(sh + 34);          // [K] adjoint exponents
    int* gset = gx + kMaxOrb;           // [K]
    double* tkz = (double*)(gset + kMaxOrb);   // tensor-term scratch: z [d][r], then y [r]
    const int64_t s = blockIdx.x;
    const uint64_t na = a.samples[2 * s], nb = a.samples[2 * s + 1];

    if (!a.tn) {
        // tensor-network part done elsewhere
    } else if (a.an.chain && a.tn == 3) {
        // psi(n) alone in double-FP32 arithmetic (the error-free product by FMA
        // and Knuth's two-sum, as in the double-double algorithms of Hida, Li and
        // Bailey), on the FP32 pipe: the state as (hi, lo) float pairs in place of
        // x, the site matrices as pairs, each output accumulated as an
        // unnormalised pair (relative error about D 2^-48), then rounded to FP64
        // for the exact power-of-two rescaling and split again
        float* xh = (float*)x;
        float* xl = xh + D;
        for (int i = threadIdx.x; i < D; i += blockDim.x) { xh[i] = i == 0 ? 1.f : 0.f; xl[i] = 0.f; }
        int ex = 0;
        __syncthreads();
        for (int t = 0; t < K; ++t) {
            const float2* M = a.ATdf + ((size_t)t * 4 + sigma_at(na, nb, t)) * D * D;
            for (int r = threadIdx.x; r < D; r += blockDim.x) {
                float hi = 0.f, lo = 0.f;
                for (int c = 0; c < D; ++c) {
                    const float2 m = __ldg(M + (size_t)c * D + r);
                    const float ah = xh[c], al = xl[c];
                    const float ph = m.x * ah;
                    const float pl = fmaf(m.x, ah, -ph) + fmaf(m.x, al, m.y * ah);
                    const float u = hi + ph, z = u - hi;
                    lo += ((hi - (u - z)) + (ph - z)) + pl;
                    hi = u;
                }
                y[r] = (double)hi + (double)lo;
            }
            __syncthreads();
            ex += block_renorm(y, D, sh);
            for (int i = threadIdx.x; i < D; i += blockDim.x) {
                const float h = (float)y[i];
                xh[i] = h;
                xl[i] = (float)(y[i] - (double)h);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) { a.psi_mant[s] = (double)xh[0] + (double)xl[0]; a.psi_exp[s] = ex; }
        __syncthreads();
    } else if (a.an.chain) {
        const bool keep = a.tn == 1;    // store the environments
        double* Ls = keep ? a.Lenv + (size_t)s * (K + 1) * D : nullptr;
        int* Le = keep ? a.Lexp + (size_t)s * (K + 1) : nullptr;
        for (int i = threadIdx.x; i < D; i += blockDim.x) { x[i] = i == 0 ? 1.0 : 0.0; if (keep) Ls[i] = x[i]; }
        if (keep && threadIdx.x == 0) Le[0] = 0;
        int ex = 0;
        __syncthreads();
        for (int t = 0; t < K; ++t) {
            const double* AT = tens(a.an.AT, t, sigma_at(na, nb, t), D);
            for (int r = threadIdx.x; r < D; r += blockDim.x) {
                double acc = 0.0;
                for (int c = 0; c < D; ++c) acc = fma(__ldg(AT + c * D + r), x[c], acc);
                y[r] = acc;
            }
            __syncthreads();
            ex += block_renorm(y, D, sh);
            for (int i = threadIdx.x; i < D; i += blockDim.x) {
                x[i] = y[i];
                if (keep) Ls[(size_t)(t + 1) * D + i] = y[i];
            }
            if (keep && threadIdx.x == 0) Le[t + 1] = ex;
            __syncthreads();
        }
        if (threadIdx.x == 0) { a.psi_mant[s] = x[0]; a.psi_exp[s] = ex; }
        __syncthreads();
        if (keep) {
            double* Rs = a.Renv + (size_t)s * (K + 1) * D;
            int* Re = a.Rexp + (size_t)s * (K + 1);
            for (int i = threadIdx.x; i < D; i += blockDim.x) { x[i] = i == 0 ? 1.0 : 0.0; Rs[(size_t)K * D + i] = x[i]; }
            if (threadIdx.x == 0) Re[K] = 0;
            ex = 0;
            __syncthreads();
            for (int t = K - 1; t >= 0; --t) {
                const double* A = tens(a.an.A, t, sigma_at(na, nb, t), D);
                for (int c = threadIdx.x; c < D; c += blockDim.x) {
                    double acc = 0.0;
                    for (int r = 0; r < D; ++r) acc = fma(x[r], __ldg(A + r * D + c), acc);
                    y[c] = acc;
                }
                __syncthreads();
                ex += block_renorm(y, D, sh);
                for (int i = threadIdx.x; i < D; i += blockDim.x) { x[i] = y[i]; Rs[(size_t)t * D + i] = y[i]; }
                if (threadIdx.x == 0) Re[t] = ex;
                __syncthreads();
            }
        }
    } else {
        double* Hs = a.Hst + (size_t)s * K * D;
        int* He = a.Hexp + (size_t)s * K;
        for (int i = 0; i < K; ++i) {
            const int e0 = a.an.pred_ptr[i], e1 = a.an.pred_ptr[i + 1];
            int eref = -1000000, et = 0;
            for (int e = e0; e < e1; ++e) {
                const int j = a.an.pred_idx[e];
                const int ej = j < 0 ? 0 : He[j];
                eref = ej > eref ? ej : eref;
                et += ej;
            }
            const int sg = sigma_at(na, nb, i);
            const bool tk = tk_has(a.an, i);
            if (tk) {
                // the tensor term scales with the product of its sources (exponent sum)
                eref = et > eref ? et : eref;
                tk_project(a.an, i, [&](int j) { return (const double*)(Hs + (size_t)j * D); }, tkz,
                           threadIdx.x, blockDim.x);
                __syncthreads();
                tk_core(a.an, i, sg, tkz, tkz + tk_degree(a.an, i) * a.an.tk_rank[i], threadIdx.x, blockDim.x);
                __syncthreads();
            }
            for (int r = threadIdx.x; r < D; r += blockDim.x) {
                double acc = 0.0;
                for (int e = e0; e < e1; ++e) {
                    const int j = a.an.pred_idx[e];
                    const double* AT = tens(a.an.AT, e, sg, D);
                    double t = 0.0;
                    if (j < 0) t = __ldg(AT + r);              // M e_0 = column 0
                    else {
                        const double* hj = Hs + (size_t)j * D;
                        for (int c = 0; c < D; ++c) t = fma(__ldg(AT + c * D + r), hj[c], t);
                    }
                    acc += ldexp(t, (j < 0 ? 0 : He[j]) - eref);
                }
                if (tk)
                    acc += ldexp(tk_out(a.an, i, r, tkz + tk_degree(a.an, i) * a.an.tk_rank[i]), et - eref);
                y[r] = acc;
            }
            __syncthreads();
            const int ge = block_renorm(y, D, sh);
            for (int r = threadIdx.x; r < D; r += blockDim.x) Hs[(size_t)i * D + r] = y[r];
            if (threadIdx.x == 0) He[i] = eref + ge;
            __syncthreads();
        }
        if (threadIdx.x == 0) { a.psi_mant[s] = Hs[(size_t)(K - 1) * D]; a.psi_exp[s] = He[K - 1]; }
        __syncthreads();
        if (a.Gst) {
            double* Gs = a.Gst + (size_t)s * K * D;
            int* Ge = a.Gexp + (size_t)s * K;
            for (int i = threadIdx.x; i < K; i += blockDim.x) { gset[i] = 0; gx[i] = 0; }
            for (int r = threadIdx.x; r < D; r += blockDim.x) Gs[(size_t)(K - 1) * D + r] = r == 0 ? 1.0 : 0.0;
            __syncthreads();
            if (threadIdx.x == 0) gset[K - 1] = 1;
            __syncthreads();
            for (int i = K - 1; i >= 0; --i) {
                if (!gset[i]) continue;
                for (int r = threadIdx.x; r < D; r += blockDim.x) x[r] = Gs[(size_t)i * D + r];
                __syncthreads();
                const int ge = block_renorm(x, D, sh);
                for (int r = threadIdx.x; r < D; r += blockDim.x) Gs[(size_t)i * D + r] = x[r];
                if (threadIdx.x == 0) { gx[i] += ge; Ge[i] = gx[i]; }
                __syncthreads();
                const int sg = sigma_at(na, nb, i);
                for (int e = a.an.pred_ptr[i]; e < a.an.pred_ptr[i + 1]; ++e) {
                    const int j = a.an.pred_idx[e];
                    if (j < 0) continue;
                    const double* A = tens(a.an.A, e, sg, D);
                    for (int c = threadIdx.x; c < D; c += blockDim.x) {
                        double acc = 0.0;
                        for (int r = 0; r < D; ++r) acc = fma(x[r], __ldg(A + r * D + c), acc);
                        y[c] = acc;
                    }
                    __syncthreads();
                    double* gj = Gs + (size_t)j * D;
                    if (!gset[j]) {
                        for (int c = threadIdx.x; c < D; c += blockDim.x) gj[c] = y[c];
                        __syncthreads();
                        if (threadIdx.x == 0) { gx[j] = gx[i]; gset[j] = 1; }
                    } else {
                        const int eref = gx[j] > gx[i] ? gx[j] : gx[i];
                        for (int c = threadIdx.x; c < D; c += blockDim.x)
                            gj[c] = ldexp(gj[c], gx[j] - eref) + ldexp(y[c], gx[i] - eref);
                        __syncthreads();
                        if (threadIdx.x == 0) gx[j] = eref;
                    }
                    __syncthreads();
                }
            }
        }
    }

    // correlator angles theta_k(n) (Sec. 2.3) and log|f(n)|
    const int NH = a.an.n_hidden;
    if (NH > 0) {
        for (int k = threadIdx.x; k < NH; k += blockDim.x) {
            const double th = corr_theta(a.an, k, na, nb);
            a.theta[(size_t)s * NH + k] = th;
            a.lc[(size_t)s * NH + k] = corr_log_factor(a.an.corr, th);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double lf = 0.0;
            for (int k = 0; k < NH; ++k) lf += a.lc[(size_t)s * NH + k];
            a.log_f[s] = lf;
        }
    } else if (threadIdx.x == 0) {
        a.log_f[s] = 0.0;
    }

    // H_nn = e_core + sum_occ h_ii + 1/2 sum_{s,t occ} [(ss|tt) - d(spin) (st|ts)]
    double part = 0.0;
    const int n2 = 2 * K;
    for (int q = threadIdx.x; q < n2 * n2; q += blockDim.x) {
        const int si = q / n2, ti = q - si * n2;
        const uint64_t ws = (si & 1) ? nb : na, wt = (ti & 1) ? nb : na;
        if (!((ws >> (si >> 1)) & 1ull) || !((wt >> (ti >> 1)) & 1ull)) continue;
        double v = eri_at(a.h, si >> 1, si >> 1, ti >> 1, ti >> 1);
        if ((si & 1) == (ti & 1)) v -= eri_at(a.h, si >> 1, ti >> 1, ti >> 1, si >> 1);
        part += 0.5 * v;
    }
    for (int p = threadIdx.x; p < K; p += blockDim.x) {
        const double hp = __ldg(a.h.h1e + p * K + p);
        if ((na >> p) & 1ull) part += hp;
        if ((nb >> p) & 1ull) part += hp;
    }
    part = warp_sum_f64(part);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = a.h.e_core;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) e += sh[w];
        a.h_diag[s] = e;
    }
}

int launch_env_fp64(const EnvArgs& a, cudaStream_t st)
{
    if (a.Ns == 0) return 0;
    const int threads = a.an.D >= 256 ? 256 : (a.an.D > 64 ? 128 : 64);
    const size_t smem = (2 * a.an.D + 34 + a.an.tk_zy) * sizeof(double) + 2 * kMaxOrb * sizeof(int);
    k_env_fp64<<<(unsigned)a.Ns, threads, smem, st>>>(a);
    return 1;
}

// ---------------------------------------------------------------------------
// Span-limited amplitudes of the connected rows, FP64
// ---------------------------------------------------------------------------

int amp_fp64_rows_per_block(const AnsatzView& an)
{
    if (an.chain) {
        int r = 4096 / an.D;
        return r < 4 ? 4 : (r > 64 ? 64 : r);
    }
    // rows of the states kept in shared memory ([R][K][D] doubles): about 32 KB,
    // so that several blocks share an SM and their FMA chains overlap
    int r = 4096 / (an.K * an.D);
    return r < 1 ? 1 : (r > 32 ? 32 : r);
}

size_t amp_fp64_smem(const AnsatzView& an, int R)
{
    size_t st = an.chain ? (size_t)2 * R * an.D : (size_t)R * an.K * an.D;
    size_t ints = (size_t)R * (an.chain ? 1 : an.K);
    ints = (ints + 1) & ~(size_t)1;                       // the tensor-term scratch after is 8-byte aligned
    return st * sizeof(double) + ints * sizeof(int) + (size_t)R * an.tk_zy * sizeof(double);
}

struct RowInfo {
    uint64_t ma, mb;
    double coef, tn;
    int p, q, ex;
};

__device__ __forceinline__ int64_t find_sample(const int64_t* base, int64_t Ns, int64_t b)
{
    int64_t lo = 0, hi = Ns - 1;       // largest s with base[s] <= b
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        if (base[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Correlator ratio f(m)/f(n) (one warp): its log magnitude and sign.
__device__ double rbm_log_ratio_warp(const AnsatzView& an, int64_t s, const double* theta,
                                     const double* lc, uint64_t na, uint64_t nb, uint64_t ma,
                                     uint64_t mb, int lane, double* sign)
{
    int neg;
    const double lr = corr_log_ratio_warp(an, s, theta, lc, na, nb, ma, mb, lane, &neg);
    *sign = neg ? -1.0 : 1.0;
    return lr;
}

__global__ void k_amp_chain_fp64(AmpArgs a)
{
    extern __shared__ double sm[];
    __shared__ OrbLists lists;
    __shared__ RowInfo info[64];
    __shared__ int s_range[2];
    const int R = a.rows_per_block, D = a.an.D;
    const int64_t b = blockIdx.x;
    const int64_t* cb = a.rows.chunk_base;
    if (b >= cb[a.Ns]) return;
    const int64_t s = find_sample(cb, a.Ns, b);
    const int64_t j = b - cb[s];
    const int64_t beg = a.rows.begin ? a.rows.begin[s] : s * a.rows.stride;
    const int64_t cnt = a.rows.count[s];
    const int64_t r0 = beg + j * R;
    const int nr = (int)((cnt - j * R) < R ? (cnt - j * R) : R);
    const uint64_t na = a.samples[2 * s], nb = a.samples[2 * s + 1];
    double* X = sm;
    double* Y = sm + (size_t)R * D;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (warp == 0) build_lists_warp(na, nb, a.h.K, lists, lane);
    if (threadIdx.x == 0) { s_range[0] = 1 << 30; s_range[1] = -1; }
    __syncthreads();
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        const Exc e = decode_rank<false>(a.h, lists, a.rows.rank[r0 + r]);   // sites only
        uint64_t ma = na, mb = nb;
        flip(ma, mb, e.i); flip(ma, mb, e.a);
        if (e.kind == 2) { flip(ma, mb, e.j); flip(ma, mb, e.b); }
        const uint64_t ch = (na ^ ma) | (nb ^ mb);
        RowInfo ri;
        ri.ma = ma; ri.mb = mb;
        ri.coef = a.rows.coef[r0 + r];
        ri.tn = 0.0;
        ri.p = __ffsll((long long)ch) - 1;
        ri.q = 63 - __clzll((long long)ch);
        ri.ex = 0;
        info[r] = ri;
        atomicMin(&s_range[0], ri.p);
        atomicMax(&s_range[1], ri.q);
    }
    __syncthreads();
    const int tmin = s_range[0], tmax = s_range[1];
    const double mant_n = a.psi_mant[s];
    const int exp_n = a.psi_exp[s];
    const int K = a.an.K;
    const double* Ls = a.Lenv + (size_t)s * (K + 1) * D;
    const double* Rs = a.Renv + (size_t)s * (K + 1) * D;
    for (int t = tmin; t <= tmax; ++t) {
        // rows entering at t start from L_{t-1}(n)
        for (int q = threadIdx.x; q < nr * D; q += blockDim.x) {
            const int r = q / D, c = q - r * D;
            if (info[r].p == t) X[(size_t)r * D + c] = Ls[(size_t)t * D + c];
        }
        for (int r = threadIdx.x; r < nr; r += blockDim.x)
            if (info[r].p == t) info[r].ex = a.Lexp[(size_t)s * (K + 1) + t];
        __syncthreads();
        for (int q = threadIdx.x; q < nr * D; q += blockDim.x) {
            const int r = q / D, c = q - r * D;
            if (t < info[r].p || t > info[r].q) continue;
            const double* AT = tens(a.an.AT, t, sigma_at(info[r].ma, info[r].mb, t), D);
            const double* x = X + (size_t)r * D;
            const double acc = dot_col4(AT, x, D, c);
            Y[(size_t)r * D + c] = acc;
        }
        __syncthreads();
        for (int r = warp; r < nr; r += nw) {
            if (t < info[r].p || t > info[r].q) continue;
            double* y = Y + (size_t)r * D;
            const int e = warp_renorm(y, D, lane);
            const int exn = info[r].ex + e;
            __syncwarp();
            for (int c = lane; c < D; c += 32) X[(size_t)r * D + c] = y[c];
            if (lane == 0) info[r].ex = exn;
            if (t == info[r].q) {
                double dot = 0.0;
                for (int c = lane; c < D; c += 32) dot = fma(Rs[(size_t)(t + 1) * D + c], y[c], dot);
                dot = warp_sum_f64(dot);
                if (lane == 0) {
                    const int em = exn + a.Rexp[(size_t)s * (K + 1) + t + 1];
                    info[r].tn = ldexp(dot / mant_n, em - exp_n);
                }
            }
        }
        __syncthreads();
    }
    for (int r = warp; r < nr; r += nw) {
        double fsg;
        const double lr = rbm_log_ratio_warp(a.an, s, a.theta, a.lc, na, nb, info[r].ma, info[r].mb, lane, &fsg);
        if (lane == 0) info[r].tn = info[r].coef * info[r].tn * (fsg * exp(lr));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = 0.0;
        int64_t sp = 0;
        for (int r = 0; r < nr; ++r) { acc += info[r].tn; sp += info[r].q - info[r].p + 1; }
        a.partial[b] = acc;
        if (a.span) a.span[b] = sp;
    }
}

__global__ void k_amp_graph_fp64(AmpArgs a)
{
    extern __shared__ double sm[];
    __shared__ OrbLists lists;
    __shared__ RowInfo info[32];
    __shared__ int s_min;
    const int R = a.rows_per_block, D = a.an.D, K = a.an.K;
    const int64_t b = blockIdx.x;
    const int64_t* cb = a.rows.chunk_base;
    if (b >= cb[a.Ns]) return;
    const int64_t s = find_sample(cb, a.Ns, b);
    const int64_t j = b - cb[s];
    const int64_t beg = a.rows.begin ? a.rows.begin[s] : s * a.rows.stride;
    const int64_t cnt = a.rows.count[s];
    const int64_t r0 = beg + j * R;
    const int nr = (int)((cnt - j * R) < R ? (cnt - j * R) : R);
    const uint64_t na = a.samples[2 * s], nb = a.samples[2 * s + 1];
    double* S = sm;                                   // [R][K][D]
    int* SX = (int*)(sm + (size_t)R * K * D);         // [R][K]
    double* TK = (double*)(SX + (((size_t)R * K + 1) & ~(size_t)1));   // [R][tk_zy] tensor-term scratch
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (warp == 0) build_lists_warp(na, nb, a.h.K, lists, lane);
    if (threadIdx.x == 0) s_min = 1 << 30;
    __syncthreads();
    for (int r = threadIdx.x; r < nr; r += blockDim.x) {
        const Exc e = decode_rank<false>(a.h, lists, a.rows.rank[r0 + r]);   // sites only
        uint64_t ma = na, mb = nb;
        flip(ma, mb, e.i); flip(ma, mb, e.a);
        if (e.kind == 2) { flip(ma, mb, e.j); flip(ma, mb, e.b); }
        const uint64_t ch = (na ^ ma) | (nb ^ mb);
        RowInfo ri;
        ri.ma = ma; ri.mb = mb;
        ri.coef = a.rows.coef[r0 + r];
        ri.tn = 0.0;
        ri.p = __ffsll((long long)ch) - 1;
        ri.q = K - 1;
        ri.ex = 0;
        info[r] = ri;
        atomicMin(&s_min, ri.p);
    }
    __syncthreads();
    const double* Hs = a.Hst + (size_t)s * K * D;
    const int* He = a.Hexp + (size_t)s * K;
    for (int i = s_min; i < K; ++i) {
        const int e0 = a.an.pred_ptr[i], e1 = a.an.pred_ptr[i + 1];
        const bool tk = tk_has(a.an, i);
        const int dr = tk ? tk_degree(a.an, i) * a.an.tk_rank[i] : 0;
        if (tk) {
            // tensor term per row: project the sources, contract the core (one warp per row)
            for (int r = warp; r < nr; r += nw) {
                const int p = info[r].p;
                if (i < p) continue;
                double* z = TK + (size_t)r * a.an.tk_zy;
                tk_project(a.an, i, [&](int jj) {
                    return (const double*)(jj < p ? Hs + (size_t)jj * D : S + ((size_t)r * K + jj) * D); },
                    z, lane, 32);
                __syncwarp();
                tk_core(a.an, i, sigma_at(info[r].ma, info[r].mb, i), z, z + dr, lane, 32);
            }
            __syncthreads();
        }
        for (int q = threadIdx.x; q < nr * D; q += blockDim.x) {
            const int r = q / D, c = q - r * D;
            const int p = info[r].p;
            if (i < p) continue;
            const int sg = sigma_at(info[r].ma, info[r].mb, i);
            int eref = -1000000, et = 0;
            for (int e = e0; e < e1; ++e) {
                const int jj = a.an.pred_idx[e];
                const int ej = jj < 0 ? 0 : (jj < p ? He[jj] : SX[r * K + jj]);
                eref = ej > eref ? ej : eref;
                et += ej;
            }
            if (tk) eref = et > eref ? et : eref;
            double acc = 0.0;
            for (int e = e0; e < e1; ++e) {
                const int jj = a.an.pred_idx[e];
                const double* AT = tens(a.an.AT, e, sg, D);
                double t = 0.0;
                int ej = 0;
                if (jj < 0) t = __ldg(AT + c);
                else {
                    const double* hj = jj < p ? Hs + (size_t)jj * D : S + ((size_t)r * K + jj) * D;
                    ej = jj < p ? He[jj] : SX[r * K + jj];
                    t = dot_col4(AT, hj, D, c);
                }
                acc += ldexp(t, ej - eref);
            }
            if (tk) acc += ldexp(tk_out(a.an, i, c, TK + (size_t)r * a.an.tk_zy + dr), et - eref);
            S[((size_t)r * K + i) * D + c] = acc;
            if (c == 0) SX[r * K + i] = eref;     // exponent before renorm
        }
        __syncthreads();
        for (int r = warp; r < nr; r += nw) {
            if (i < info[r].p) continue;
            const int e = warp_renorm(S + ((size_t)r * K + i) * D, D, lane);
            if (lane == 0) SX[r * K + i] += e;
        }
        __syncthreads();
    }
    const double mant_n = a.psi_mant[s];
    const int exp_n = a.psi_exp[s];
    for (int r = warp; r < nr; r += nw) {
        double fsg;
        const double lr = rbm_log_ratio_warp(a.an, s, a.theta, a.lc, na, nb, info[r].ma, info[r].mb, lane, &fsg);
        if (lane == 0) {
            const double mm = S[((size_t)r * K + K - 1) * D];
            const double tn = ldexp(mm / mant_n, SX[r * K + K - 1] - exp_n);
            info[r].tn = info[r].coef * tn * (fsg * exp(lr));
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = 0.0;
        int64_t sp = 0, mv = 0;
        for (int r = 0; r < nr; ++r) {
            acc += info[r].tn;
            sp += K - info[r].p;
            mv += graph_matvecs(a.an, info[r].p);
        }
        a.partial[b] = acc;
        if (a.span) a.span[b] = sp;
        if (a.mv) a.mv[b] = mv;
    }
}

int launch_amp_fp64(const AmpArgs& a, cudaStream_t st)
{
    if (a.rows.max_chunks == 0) return 0;
    const size_t smem = amp_fp64_smem(a.an, a.rows_per_block);
    if (a.an.chain) {
        allow_max_smem(k_amp_chain_fp64);
        k_amp_chain_fp64<<<(unsigned)a.rows.max_chunks, 256, smem, st>>>(a);
    } else {
        allow_max_smem(k_amp_graph_fp64);
        k_amp_graph_fp64<<<(unsigned)a.rows.max_chunks, 256, smem, st>>>(a);
    }
    return 1;
}

// ---------------------------------------------------------------------------
// Full K-site product for arbitrary determinants (one block per determinant)
// ---------------------------------------------------------------------------

__global__ void k_full_amp_fp64(AnsatzView an, const uint64_t* dets, int64_t n, double* log_abs,
                                int8_t* sign)
{
    extern __shared__ double sm[];
    const int D = an.D, K = an.K;
    const int64_t id = blockIdx.x;
    if (id >= n) return;
    const uint64_t na = dets[2 * id], nb = dets[2 * id + 1];
    double* sh = sm;                          // 34
    double* st = sm + 34;                     // chain: [2][D]; graph: [K][D]
    __shared__ int ex[kMaxOrb];
    if (an.chain) {
        double* x = st;
        double* y = st + D;
        for (int i = threadIdx.x; i < D; i += blockDim.x) x[i] = i == 0 ? 1.0 : 0.0;
        int e = 0;
        __syncthreads();
        for (int t = 0; t < K; ++t) {
            const double* AT = tens(an.AT, t, sigma_at(na, nb, t), D);
            for (int r = threadIdx.x; r < D; r += blockDim.x) {
                double acc = 0.0;
                for (int c = 0; c < D; ++c) acc = fma(__ldg(AT + c * D + r), x[c], acc);
                y[r] = acc;
            }
            __syncthreads();
            e += block_renorm(y, D, sh);
            for (int i = threadIdx.x; i < D; i += blockDim.x) x[i] = y[i];
            __syncthreads();
        }
        if (threadIdx.x == 0) { ex[K - 1] = e; sh[33] = x[0]; }
    } else {
        double* tkz = st + (size_t)K * D;         // tensor-term scratch
        for (int i = 0; i < K; ++i) {
            const int e0 = an.pred_ptr[i], e1 = an.pred_ptr[i + 1];
            int eref = -1000000, et = 0;
            for (int e = e0; e < e1; ++e) {
                const int j = an.pred_idx[e];
                const int ej = j < 0 ? 0 : ex[j];
                eref = ej > eref ? ej : eref;
                et += ej;
            }
            const int sg = sigma_at(na, nb, i);
            const bool tk = tk_has(an, i);
            const int dr = tk ? tk_degree(an, i) * an.tk_rank[i] : 0;
            if (tk) {
                eref = et > eref ? et : eref;
                tk_project(an, i, [&](int j) { return (const double*)(st + (size_t)j * D); }, tkz,
                           threadIdx.x, blockDim.x);
                __syncthreads();
                tk_core(an, i, sg, tkz, tkz + dr, threadIdx.x, blockDim.x);
                __syncthreads();
            }
            for (int r = threadIdx.x; r < D; r += blockDim.x) {
                double acc = 0.0;
                for (int e = e0; e < e1; ++e) {
                    const int j = an.pred_idx[e];
                    const double* AT = tens(an.AT, e, sg, D);
                    double t = 0.0;
                    if (j < 0) t = __ldg(AT + r);
                    else for (int c = 0; c < D; ++c) t = fma(__ldg(AT + c * D + r), st[(size_t)j * D + c], t);
                    acc += ldexp(t, (j < 0 ? 0 : ex[j]) - eref);
                }
                if (tk) acc += ldexp(tk_out(an, i, r, tkz + dr), et - eref);
                st[(size_t)i * D + r] = acc;
            }
            __syncthreads();
            const int ge = block_renorm(st + (size_t)i * D, D, sh);
            if (threadIdx.x == 0) ex[i] = eref + ge;
            __syncthreads();
        }
        if (threadIdx.x == 0) sh[33] = st[(size_t)(K - 1) * D];
    }
    __syncthreads();
    const double mant = sh[33];
    __syncthreads();
    // correlator log|f| and the parity of its negative factors (cos forms)
    double lf = 0.0;
    int odd = 0;
    for (int k = threadIdx.x; k < an.n_hidden; k += blockDim.x) {
        const double th = corr_theta(an, k, na, nb);
        lf += corr_log_factor(an.corr, th);
        if (an.corr != 0) odd ^= cos(th) < 0.0;
    }
    const int nodd = __syncthreads_count(odd);
    lf = warp_sum_f64(lf);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = lf;
    __syncthreads();
    if (threadIdx.x == 0) {
        double l = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) l += sh[w];
        const double m = mant;
        if (m == 0.0 || l == -INFINITY) { sign[id] = 0; log_abs[id] = -INFINITY; }
        else {
            sign[id] = ((m < 0) ^ (nodd & 1)) ? -1 : 1;
            log_abs[id] = log(fabs(m)) + (double)ex[K - 1] * 0.69314718055994530942 + l;
        }
    }
}

int launch_full_amp_fp64(const AnsatzView& an, const uint64_t* dets, int64_t n, double* log_abs,
                         int8_t* sign, cudaStream_t st)
{
    if (n == 0) return 0;
    int launches = 0;
    const size_t smem = (34 + (an.chain ? 2 * (size_t)an.D : (size_t)an.K * an.D + an.tk_zy)) * sizeof(double);
    allow_max_smem(k_full_amp_fp64);
    const int threads = an.D >= 256 ? 256 : (an.D > 64 ? 128 : 64);
    for (int64_t i0 = 0; i0 < n; i0 += (1ll << 30)) {
        const int64_t m = (n - i0) < (1ll << 30) ? (n - i0) : (1ll << 30);
        k_full_amp_fp64<<<(unsigned)m, threads, smem, st>>>(an, dets + 2 * i0, m, log_abs + i0, sign + i0);
        ++launches;
    }
    return launches;
}

}  // namespace nqs
