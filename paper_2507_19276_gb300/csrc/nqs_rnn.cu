// nqs_rnn.cu -- the normalised MPS-RNN / BDG-RNN readout of Sec. 2.2 and the
// autoregressive sampling it allows (Sec. 2.1, Sec. 3), in FP64 on CUDA cores.
//
// Vertex i (= spatial orbital i, the computation order) forms four candidate
// memory cells h_i^s = sum_{e=(j->i)} M_e^s h_j + v_i^s from the cells of the
// local states already chosen (Eq. MPS-RNN-1D; Eq. bdg-rnn-update without the
// tensor term), h_{-1} = e_0. P_i(s) = sum_a eta_i[a] (h_i^s[a])^2 is
// normalised over the local states the N_alpha / N_beta constraint of Sec. 3
// still allows, and Phi(n) = prod_i sqrt(P~_i(s_i)) sign(w_i . h_i^{s_i} + c_i).
//
// Local energy: a connected m shares n's prefix up to its first changed
// vertex p, so its cells and conditionals agree with n's below p; the kernel
// re-runs vertices p..K-1 for m (one warp per row) and divides by n's suffix
// of conditionals and signs. The normalisers depend on the whole prefix, so
// there is no right environment: the cost per amplitude is (K - p) x 4 cell
// products.
//
// Sampling: breadth first over the vertices. A node of level i is a distinct
// prefix holding `cnt` of the batch's draws at offsets off..off+cnt-1 (the
// nodes of a level tile the draws in prefix order). Draw j picks local state
// s at vertex i with u_j = Philox4x64-10(key (seed, 0), counter (j, i, 1, 0))
// as the first allowed s with u_j Z < sum_{allowed s' <= s} P_i(s') (the last
// allowed state when rounding leaves none); the children keep the offsets in
// the order of s, so the result does not depend on how nodes are scheduled.
#include "nqs_kernels.cuh"

namespace nqs {

namespace {

__device__ __forceinline__ double warp_allsum(double v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ bool rnn_allowed(const AnsatzView& an, int i, int nad, int nbd, int s)
{
    if (an.mask_na < 0) return true;
    const int ea = nad + (s & 1), eb = nbd + (s >> 1), left = an.K - 1 - i;
    return ea <= an.mask_na && eb <= an.mask_nb && an.mask_na - ea <= left && an.mask_nb - eb <= left;
}

// One warp: the four candidate cells of vertex i into cand[4][D] (shared
// memory) and P_i(s) on every lane. src(j) gives the cell of vertex j >= 0;
// the boundary source j = -1 is e_0 (M e_0 = column 0 of M).
template <class Src>
__device__ void rnn_vertex_warp(const AnsatzView& an, int i, const Src& src, double* cand,
                                double P[4], int lane, double* tkz)
{
    const int D = an.D;
    const int e0 = an.chain ? i : an.pred_ptr[i];
    const int e1 = an.chain ? i + 1 : an.pred_ptr[i + 1];
    // tensor term (BDG-TensorRNN): the sources' projections once, the core of
    // every local state, z [d][r] then y [4][r] in the scratch
    const bool tk = tk_has(an, i);
    const int rk = tk ? an.tk_rank[i] : 0;
    const int dr = tk ? tk_degree(an, i) * rk : 0;
    if (tk) {
        tk_project(an, i, src, tkz, lane, 32);
        __syncwarp();
        for (int s = 0; s < 4; ++s) tk_core(an, i, s, tkz, tkz + dr + s * rk, lane, 32);
        __syncwarp();
    }
    // the 4 D candidate entries spread over the lanes (local state, component)
    for (int q = lane; q < 4 * D; q += 32) {
        const int s = q / D, r = q - s * D;
        double acc = __ldg(an.rv + ((size_t)i * 4 + s) * D + r);
        for (int e = e0; e < e1; ++e) {
            const int j = an.chain ? e - 1 : an.pred_idx[e];
            const double* AT = an.AT + ((size_t)e * 4 + s) * D * D;    // AT[c][r] = M[r][c]
            if (j < 0) {
                acc += __ldg(AT + r);
            } else {
                acc += dot_col4(AT, src(j), D, r);
            }
        }
        if (tk) acc += tk_out(an, i, r, tkz + dr + s * rk);
        cand[q] = acc;
    }
    __syncwarp();                       // cand visible to every lane
    for (int s = 0; s < 4; ++s) {
        double p = 0.0;
        for (int r = lane; r < D; r += 32) {
            const double h = cand[s * D + r];
            p = fma(__ldg(an.reta + (size_t)i * D + r) * h, h, p);
        }
        P[s] = warp_allsum(p);
    }
}

// The conditional of local state `sg` at vertex i and the sign of its phase:
// returns 1/2 log P~_i(sg), -inf where the state is not allowed or has zero
// weight; *neg = (w_i . h + c_i < 0).
__device__ __forceinline__ double rnn_pick(const AnsatzView& an, int i, int nad, int nbd, int sg,
                                           const double* cand, const double P[4], int lane, int* neg)
{
    const int D = an.D;
    double Z = 0.0;
    for (int q = 0; q < 4; ++q)
        if (rnn_allowed(an, i, nad, nbd, q)) Z += P[q];
    double ph = 0.0;
    for (int r = lane; r < D; r += 32) ph = fma(__ldg(an.rw + (size_t)i * D + r), cand[sg * D + r], ph);
    ph = warp_allsum(ph) + __ldg(an.rc + i);
    *neg = ph < 0.0;
    if (!rnn_allowed(an, i, nad, nbd, sg) || !(P[sg] > 0.0) || !(Z > 0.0)) return -INFINITY;
    return 0.5 * (log(P[sg]) - log(Z));
}

}  // namespace

// ---------------------------------------------------------------------------
// psi(n): cells, conditionals and phase signs of every vertex (one warp per sample)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_rnn_env(RnnEnvArgs a)
{
    extern __shared__ double sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t s = (int64_t)blockIdx.x * 8 + warp;
    if (s >= a.Ns) return;
    const AnsatzView& an = a.an;
    const int K = an.K, D = an.D;
    double* cand = sm + (size_t)warp * (4 * D + an.tk_zy);
    double* tkz = cand + 4 * D;
    const uint64_t na = a.samples[2 * s], nb = a.samples[2 * s + 1];
    double* cells = a.cells + (size_t)s * K * D;
    int nad = 0, nbd = 0, sign = 1;
    for (int i = 0; i < K; ++i) {
        double P[4];
        rnn_vertex_warp(an, i, [&](int j) { return (const double*)(cells + (size_t)j * D); }, cand, P, lane, tkz);
        const int sg = sigma_at(na, nb, i);
        int neg;
        const double lp = rnn_pick(an, i, nad, nbd, sg, cand, P, lane, &neg);
        if (lane == 0) {
            a.lp[(size_t)s * K + i] = lp;
            a.sg[(size_t)s * K + i] = neg ? -1 : 1;
        }
        if (lp == -INFINITY) sign = 0;
        else if (neg) sign = -sign;
        for (int r = lane; r < D; r += 32) cells[(size_t)i * D + r] = cand[sg * D + r];
        __syncwarp();
        nad += sg & 1;
        nbd += sg >> 1;
    }
    if (lane == 0) {
        const double lf = a.log_f[s];
        a.psi_mant[s] = (lf == -INFINITY) ? 0.0 : (double)sign;
        a.psi_exp[s] = 0;
    }
}

int launch_rnn_env(const RnnEnvArgs& a, cudaStream_t st)
{
    if (a.Ns == 0) return 0;
    const size_t smem = (size_t)8 * (4 * a.an.D + a.an.tk_zy) * sizeof(double);
    allow_max_smem(k_rnn_env);
    k_rnn_env<<<(unsigned)((a.Ns + 7) / 8), 256, smem, st>>>(a);
    return 1;
}

// ---------------------------------------------------------------------------
// Connected amplitudes: vertices p..K-1 re-run for m, one warp per row
// ---------------------------------------------------------------------------

constexpr int kRnnRows = 32;      // rows per block (one chunk of the row set)

int rnn_rows_per_block() { return kRnnRows; }

static int rnn_warps(const AnsatzView& an)
{
    const size_t per = ((size_t)(an.K + 4) * an.D + an.tk_zy) * sizeof(double);
    int w = (int)((200u << 10) / per);
    return w < 1 ? 1 : (w > 8 ? 8 : w);
}

__global__ void __launch_bounds__(256) k_rnn_amp(RnnAmpArgs a)
{
    extern __shared__ double sm[];
    __shared__ OrbLists lists;
    __shared__ double s_term[kRnnRows];
    __shared__ int s_span[kRnnRows];
    const AnsatzView& an = a.an;
    const int K = an.K, D = an.D;
    const int64_t b = blockIdx.x;
    const int64_t* cb = a.rows.chunk_base;
    if (b >= cb[a.Ns]) return;
    int64_t lo = 0, hi = a.Ns - 1;                  // largest s with cb[s] <= b
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (cb[mid] <= b) lo = mid; else hi = mid - 1;
    }
    const int64_t s = lo;
    const int64_t j = b - cb[s];
    const int64_t beg = a.rows.begin ? a.rows.begin[s] : s * a.rows.stride;
    const int64_t cnt = a.rows.count[s];
    const int64_t r0 = beg + j * kRnnRows;
    const int nr = (int)((cnt - j * kRnnRows) < kRnnRows ? (cnt - j * kRnnRows) : kRnnRows);
    const uint64_t na = a.samples[2 * s], nb = a.samples[2 * s + 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (warp == 0) build_lists_warp(na, nb, a.h.K, lists, lane);
    __syncthreads();
    double* wc = sm + (size_t)warp * ((K + 4) * D + an.tk_zy);   // this warp's cells of m, [K][D]
    double* cand = wc + (size_t)K * D;
    double* tkz = cand + 4 * D;
    const double* cn = a.cells + (size_t)s * K * D;  // n's cells
    for (int r = warp; r < nr; r += nw) {
        const Exc e = decode_rank<false>(a.h, lists, a.rows.rank[r0 + r]);   // sites only
        uint64_t ma = na, mb = nb;
        flip(ma, mb, e.i); flip(ma, mb, e.a);
        if (e.kind == 2) { flip(ma, mb, e.j); flip(ma, mb, e.b); }
        const int p = __ffsll((long long)((na ^ ma) | (nb ^ mb))) - 1;
        int nad = __popcll(na & low_mask(p)), nbd = __popcll(nb & low_mask(p));
        double lpm = 0.0;
        int odd = 0;
        bool ok = true;
        for (int i = p; i < K; ++i) {
            double P[4];
            rnn_vertex_warp(an, i, [&](int jj) { return (const double*)(jj < p ? cn + (size_t)jj * D : wc + (size_t)jj * D); },
                            cand, P, lane, tkz);
            const int sg = sigma_at(ma, mb, i);
            int neg;
            const double lp = rnn_pick(an, i, nad, nbd, sg, cand, P, lane, &neg);
            if (lp == -INFINITY) ok = false;
            else { lpm += lp; odd ^= neg; }
            for (int c = lane; c < D; c += 32) wc[(size_t)i * D + c] = cand[sg * D + c];
            __syncwarp();
            nad += sg & 1;
            nbd += sg >> 1;
        }
        // n's suffix of conditionals and signs
        double lpn = 0.0;
        int oddn = 0;
        for (int i = p + lane; i < K; i += 32) {
            lpn += a.lp[(size_t)s * K + i];
            oddn ^= a.sg[(size_t)s * K + i] < 0;
        }
        for (int o = 16; o; o >>= 1) {
            lpn += __shfl_xor_sync(kFull, lpn, o);
            oddn ^= __shfl_xor_sync(kFull, oddn, o);
        }
        int negf;
        const double lr = corr_log_ratio_warp(an, s, a.theta, a.lc, na, nb, ma, mb, lane, &negf);
        if (lane == 0) {
            double t = 0.0;
            if (ok) {
                t = a.rows.coef[r0 + r] * exp(lpm - lpn + lr);
                if (odd ^ oddn ^ negf) t = -t;
            }
            s_term[r] = t;
            s_span[r] = K - p;
        }
        __syncwarp();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double acc = 0.0;
        int64_t sp = 0;
        for (int r = 0; r < nr; ++r) { acc += s_term[r]; sp += s_span[r]; }
        a.partial[b] = acc;
        if (a.span) a.span[b] = sp;
    }
}

// Chain readout, the block's 32 rows in lockstep over the vertices: per vertex
// the four site matrices are staged once in shared memory for every row, the
// 4 D candidate entries of all rows spread over the block (four independent
// FMA chains each), then one thread per (row, local state) forms P and one
// thread per row the normaliser, the choice and the phase. The arithmetic of
// each row is that of k_rnn_amp up to the order of the sums.
constexpr int kRnnChainMaxD = 32;

__global__ void __launch_bounds__(256) k_rnn_amp_chain(RnnAmpArgs a)
{
    extern __shared__ double sm[];
    __shared__ OrbLists lists;
    __shared__ uint64_t s_ma[kRnnRows], s_mb[kRnnRows];
    __shared__ int s_p[kRnnRows], s_nad[kRnnRows], s_nbd[kRnnRows], s_odd[kRnnRows], s_ok[kRnnRows];
    __shared__ int s_sig[kRnnRows];
    __shared__ double s_lpm[kRnnRows], s_term[kRnnRows];
    __shared__ int s_tmin;
    const AnsatzView& an = a.an;
    const int K = an.K, D = an.D;
    const int64_t b = blockIdx.x;
    const int64_t* cb = a.rows.chunk_base;
    if (b >= cb[a.Ns]) return;
    int64_t lo = 0, hi = a.Ns - 1;                  // largest s with cb[s] <= b
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (cb[mid] <= b) lo = mid; else hi = mid - 1;
    }
    const int64_t s = lo;
    const int64_t j = b - cb[s];
    const int64_t beg = a.rows.begin ? a.rows.begin[s] : s * a.rows.stride;
    const int64_t cnt = a.rows.count[s];
    const int64_t r0 = beg + j * kRnnRows;
    const int nr = (int)((cnt - j * kRnnRows) < kRnnRows ? (cnt - j * kRnnRows) : kRnnRows);
    const uint64_t na = a.samples[2 * s], nb = a.samples[2 * s + 1];
    const int tid = threadIdx.x, nt = blockDim.x;
    double* AT4 = sm;                                // [4][D][D]: AT4[s][c][a] = M_t^s[a][c]
    double* cell = AT4 + (size_t)4 * D * D;          // [R][D] each row's previous cell
    double* cand = cell + (size_t)kRnnRows * D;      // [R][4][D]
    double* Pv = cand + (size_t)kRnnRows * 4 * D;    // [R][4]
    if (tid < 32) build_lists_warp(na, nb, a.h.K, lists, tid);
    if (tid == 0) s_tmin = K;
    __syncthreads();
    if (tid < nr) {
        const Exc e = decode_rank<false>(a.h, lists, a.rows.rank[r0 + tid]);   // sites only
        uint64_t ma = na, mb = nb;
        flip(ma, mb, e.i); flip(ma, mb, e.a);
        if (e.kind == 2) { flip(ma, mb, e.j); flip(ma, mb, e.b); }
        const int p = __ffsll((long long)((na ^ ma) | (nb ^ mb))) - 1;
        s_ma[tid] = ma; s_mb[tid] = mb; s_p[tid] = p;
        s_nad[tid] = __popcll(na & low_mask(p));
        s_nbd[tid] = __popcll(nb & low_mask(p));
        s_odd[tid] = 0; s_ok[tid] = 1; s_lpm[tid] = 0.0;
        atomicMin(&s_tmin, p);
    }
    __syncthreads();
    const double* cn = a.cells + (size_t)s * K * D;  // n's cells
    for (int t = s_tmin; t < K; ++t) {
        // the site matrices of vertex t, and the previous cell of the rows entering at t
        const double* ATg = an.AT + (size_t)t * 4 * D * D;
        for (int q = tid; q < 4 * D * D; q += nt) AT4[q] = __ldg(ATg + q);
        for (int q = tid; q < nr * D; q += nt) {
            const int r = q / D, c = q - r * D;
            if (s_p[r] == t) cell[q] = t == 0 ? (c == 0 ? 1.0 : 0.0) : cn[(size_t)(t - 1) * D + c];
        }
        __syncthreads();
        for (int q = tid; q < nr * 4 * D; q += nt) {
            const int r = q / (4 * D), sa = q - r * 4 * D, sg = sa / D, c = sa - sg * D;
            if (t < s_p[r]) continue;
            const double* M = AT4 + (size_t)sg * D * D;
            const double* h = cell + (size_t)r * D;
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
            int k = 0;
            for (; k + 3 < D; k += 4) {
                s0 = fma(M[(size_t)k * D + c], h[k], s0);
                s1 = fma(M[(size_t)(k + 1) * D + c], h[k + 1], s1);
                s2 = fma(M[(size_t)(k + 2) * D + c], h[k + 2], s2);
                s3 = fma(M[(size_t)(k + 3) * D + c], h[k + 3], s3);
            }
            for (; k < D; ++k) s0 = fma(M[(size_t)k * D + c], h[k], s0);
            cand[q] = __ldg(an.rv + ((size_t)t * 4 + sg) * D + c) + ((s0 + s1) + (s2 + s3));
        }
        __syncthreads();
        for (int q = tid; q < nr * 4; q += nt) {
            const int r = q >> 2, sg = q & 3;
            if (t < s_p[r]) continue;
            const double* h = cand + (size_t)(r * 4 + sg) * D;
            double p = 0.0;
            for (int c = 0; c < D; ++c) p = fma(__ldg(an.reta + (size_t)t * D + c) * h[c], h[c], p);
            Pv[q] = p;
        }
        __syncthreads();
        if (tid < nr && t >= s_p[tid]) {
            const int r = tid, sg = sigma_at(s_ma[r], s_mb[r], t);
            double Z = 0.0;
            for (int q = 0; q < 4; ++q)
                if (rnn_allowed(an, t, s_nad[r], s_nbd[r], q)) Z += Pv[r * 4 + q];
            const double P = Pv[r * 4 + sg];
            double ph = __ldg(an.rc + t);
            const double* h = cand + (size_t)(r * 4 + sg) * D;
            for (int c = 0; c < D; ++c) ph = fma(__ldg(an.rw + (size_t)t * D + c), h[c], ph);
            if (!rnn_allowed(an, t, s_nad[r], s_nbd[r], sg) || !(P > 0.0) || !(Z > 0.0)) s_ok[r] = 0;
            else {
                s_lpm[r] += 0.5 * (log(P) - log(Z));
                s_odd[r] ^= ph < 0.0;
            }
            s_sig[r] = sg;
            s_nad[r] += sg & 1;
            s_nbd[r] += sg >> 1;
        }
        __syncthreads();
        for (int q = tid; q < nr * D; q += nt) {
            const int r = q / D, c = q - r * D;
            if (t >= s_p[r]) cell[q] = cand[(size_t)(r * 4 + s_sig[r]) * D + c];
        }
        __syncthreads();
    }
    // n's suffix of conditionals and signs, the correlator ratio, the term (one warp per row)
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    for (int r = warp; r < nr; r += nw) {
        const int p = s_p[r];
        double lpn = 0.0;
        int oddn = 0;
        for (int i = p + lane; i < K; i += 32) {
            lpn += a.lp[(size_t)s * K + i];
            oddn ^= a.sg[(size_t)s * K + i] < 0;
        }
        for (int o = 16; o; o >>= 1) {
            lpn += __shfl_xor_sync(kFull, lpn, o);
            oddn ^= __shfl_xor_sync(kFull, oddn, o);
        }
        int negf;
        const double lr = corr_log_ratio_warp(an, s, a.theta, a.lc, na, nb, s_ma[r], s_mb[r], lane, &negf);
        if (lane == 0) {
            double tv = 0.0;
            if (s_ok[r]) {
                tv = a.rows.coef[r0 + r] * exp(s_lpm[r] - lpn + lr);
                if (s_odd[r] ^ oddn ^ negf) tv = -tv;
            }
            s_term[r] = tv;
        }
    }
    __syncthreads();
    if (tid == 0) {
        double acc = 0.0;
        int64_t sp = 0;
        for (int r = 0; r < nr; ++r) { acc += s_term[r]; sp += K - s_p[r]; }
        a.partial[b] = acc;
        if (a.span) a.span[b] = sp;
    }
}

int launch_rnn_amp(const RnnAmpArgs& a, cudaStream_t st)
{
    if (a.rows.max_chunks == 0) return 0;
    if (a.an.chain && a.an.D <= kRnnChainMaxD) {
        const int D = a.an.D;
        const size_t smem = ((size_t)4 * D * D + (size_t)kRnnRows * D * 5 + (size_t)kRnnRows * 4) * sizeof(double);
        allow_max_smem(k_rnn_amp_chain);
        k_rnn_amp_chain<<<(unsigned)a.rows.max_chunks, 256, smem, st>>>(a);
        return 1;
    }
    const int w = rnn_warps(a.an);
    const size_t smem = (size_t)w * ((a.an.K + 4) * a.an.D + a.an.tk_zy) * sizeof(double);
    allow_max_smem(k_rnn_amp);
    k_rnn_amp<<<(unsigned)a.rows.max_chunks, 32 * w, smem, st>>>(a);
    return 1;
}

// ---------------------------------------------------------------------------
// Full evaluation of arbitrary determinants (nqs_amplitude), one warp each
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256) k_rnn_full(AnsatzView an, const uint64_t* dets, int64_t n,
                                                  double* log_abs, int8_t* sign)
{
    extern __shared__ double sm[];
    const int K = an.K, D = an.D;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int64_t id = (int64_t)blockIdx.x * nw + warp;
    if (id >= n) return;
    double* wc = sm + (size_t)warp * ((K + 4) * D + an.tk_zy);
    double* cand = wc + (size_t)K * D;
    double* tkz = cand + 4 * D;
    const uint64_t na = dets[2 * id], nb = dets[2 * id + 1];
    int nad = 0, nbd = 0, odd = 0;
    bool ok = true;
    double lp_sum = 0.0;
    for (int i = 0; i < K; ++i) {
        double P[4];
        rnn_vertex_warp(an, i, [&](int jj) { return (const double*)(wc + (size_t)jj * D); }, cand, P, lane, tkz);
        const int sg = sigma_at(na, nb, i);
        int neg;
        const double lp = rnn_pick(an, i, nad, nbd, sg, cand, P, lane, &neg);
        if (lp == -INFINITY) ok = false;
        else { lp_sum += lp; odd ^= neg; }
        for (int c = lane; c < D; c += 32) wc[(size_t)i * D + c] = cand[sg * D + c];
        __syncwarp();
        nad += sg & 1;
        nbd += sg >> 1;
    }
    // correlator log|f| and its sign
    double lf = 0.0;
    int oddf = 0;
    for (int k = lane; k < an.n_hidden; k += 32) {
        const double th = corr_theta(an, k, na, nb);
        lf += corr_log_factor(an.corr, th);
        if (an.corr != 0) oddf ^= cos(th) < 0.0;
    }
    for (int o = 16; o; o >>= 1) {
        lf += __shfl_xor_sync(kFull, lf, o);
        oddf ^= __shfl_xor_sync(kFull, oddf, o);
    }
    if (lane == 0) {
        if (!ok || lf == -INFINITY) { sign[id] = 0; log_abs[id] = -INFINITY; }
        else { sign[id] = (odd ^ oddf) ? -1 : 1; log_abs[id] = lp_sum + lf; }
    }
}

int launch_rnn_full(const AnsatzView& an, const uint64_t* dets, int64_t n, double* log_abs,
                    int8_t* sign, cudaStream_t st)
{
    if (n == 0) return 0;
    const int w = rnn_warps(an);
    const size_t smem = (size_t)w * ((an.K + 4) * an.D + an.tk_zy) * sizeof(double);
    allow_max_smem(k_rnn_full);
    int launches = 0;
    const int64_t per = (int64_t)w * 65535 * 1024;
    for (int64_t i0 = 0; i0 < n; i0 += per) {
        const int64_t m = (n - i0) < per ? (n - i0) : per;
        k_rnn_full<<<(unsigned)((m + w - 1) / w), 32 * w, smem, st>>>(an, dets + 2 * i0, m, log_abs + i0,
                                                                     sign + i0);
        ++launches;
    }
    return launches;
}

// ---------------------------------------------------------------------------
// Autoregressive sampling, one level per launch pair
// ---------------------------------------------------------------------------

// Per node of level i (one warp): the candidate cells of vertex i from the
// node's prefix, then every draw of the node picks a local state.
__global__ void __launch_bounds__(256) k_sample_level(SampleLevel a)
{
    const AnsatzView& an = a.an;
    const int D = an.D, i = a.level;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * 8 + warp;
    if (q >= a.n_nodes) return;
    double* cand = a.cand + (size_t)q * 4 * D;
    extern __shared__ double sm[];
    double* tkz = sm + (size_t)warp * an.tk_zy;         // tensor-term scratch of this warp
    // cell of vertex jj (< i) of this node: level jj + 1 through the parent links
    auto src = [&](int jj) {
        int64_t idx = q;
        for (int l = i; l > jj + 1; --l) idx = a.parents[l][idx];
        return (const double*)(a.cells[jj + 1] + (size_t)idx * D);
    };
    double P[4];
    rnn_vertex_warp(an, i, src, cand, P, lane, tkz);
    const int nad = __popcll(a.pa[q]), nbd = __popcll(a.pb[q]);
    bool ok[4];
    int last = -1;
    double Z = 0.0;
    for (int s = 0; s < 4; ++s) {
        ok[s] = rnn_allowed(an, i, nad, nbd, s);
        if (ok[s]) { Z += P[s]; last = s; }
    }
    int64_t hist[4] = {0, 0, 0, 0};
    const int64_t o = a.off[q], c = a.cnt[q];
    for (int64_t j0 = 0; j0 < c; j0 += 32) {
        int pick = -1;
        if (j0 + lane < c) {
            const uint64_t x = philox_first4((uint64_t)(o + j0 + lane), (uint64_t)i, 1ull, a.seed);
            const double u = (double)(x >> 11) * 0x1.0p-53;
            const double t = u * Z;
            double cum = 0.0;
            pick = last;
            for (int s = 0; s < 4; ++s) {
                if (!ok[s]) continue;
                cum += P[s];
                if (t < cum) { pick = s; break; }
            }
        }
        for (int s = 0; s < 4; ++s) hist[s] += __popc(__ballot_sync(kFull, pick == s));
    }
    if (lane < 4) {
        a.child_cnt[(size_t)q * 4 + lane] = hist[lane];
        a.child_flag[(size_t)q * 4 + lane] = hist[lane] > 0 ? 1 : 0;
    }
}

int launch_sample_level(const SampleLevel& a, cudaStream_t st)
{
    if (a.n_nodes == 0) return 0;
    k_sample_level<<<(unsigned)((a.n_nodes + 7) / 8), 256, (size_t)8 * a.an.tk_zy * sizeof(double), st>>>(a);
    return 1;
}

// The children of level i's nodes: one per (node, local state) with draws,
// at the position of the exclusive scan of the counts (prefix order).
__global__ void k_sample_children(SampleChildren a)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n_nodes * 4) return;
    const int64_t c = a.child_cnt[g];
    if (c == 0) return;
    const int64_t q = g >> 2;
    const int s = (int)(g & 3);
    const int64_t pos = a.child_pos[g];
    int64_t before = 0;
    for (int t = 0; t < s; ++t) before += a.child_cnt[q * 4 + t];
    a.qa[pos] = a.pa[q] | ((uint64_t)(s & 1) << a.level);
    a.qb[pos] = a.pb[q] | ((uint64_t)(s >> 1) << a.level);
    a.qoff[pos] = a.off[q] + before;
    a.qcnt[pos] = c;
    a.qparent[pos] = (int32_t)q;
    for (int r = 0; r < a.D; ++r) a.qcell[(size_t)pos * a.D + r] = a.cand[((size_t)q * 4 + s) * a.D + r];
}

int launch_sample_children(const SampleChildren& a, cudaStream_t st)
{
    if (a.n_nodes == 0) return 0;
    const int64_t n = a.n_nodes * 4;
    k_sample_children<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
    return 1;
}

// The last level's nodes as determinants [n][2] and counts (as doubles).
__global__ void k_sample_output(const uint64_t* pa, const uint64_t* pb, const int64_t* cnt, int64_t n,
                                uint64_t* dets, double* counts)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    dets[2 * q] = pa[q];
    dets[2 * q + 1] = pb[q];
    counts[q] = (double)cnt[q];
}

int launch_sample_output(const uint64_t* pa, const uint64_t* pb, const int64_t* cnt, int64_t n,
                         uint64_t* dets, double* counts, cudaStream_t st)
{
    if (n == 0) return 0;
    k_sample_output<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(pa, pb, cnt, n, dets, counts);
    return 1;
}

}  // namespace nqs
