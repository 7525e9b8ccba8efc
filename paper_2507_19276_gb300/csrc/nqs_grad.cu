// nqs_grad.cu -- the backward pass: sum_n u_n d log|psi(n)| / d theta (the
// vector-Jacobian product of Eq. egrad: with u_n = 2 c_n (E_loc(n) - E) / sum c
// it is the energy gradient; Sec. 2.3 gives the weights of the reweighted form).
//
// Tensor network (linear readout): with the forward cells h and the adjoints
// g = d psi_TN / d h of sample n, d psi_TN(n) / d M_e^s[a][b] = [s = s_i(n)]
// g_i(n)[a] h_j(n)[b] for the edge e = (j -> i) (chain: h_j = L_{i-1},
// g_i = R_{i+1}), so
//   grad_e^s = sum_{n : s_i(n) = s} w_n g_i(n) h_j(n)^T,   w_n = u_n / psi_TN(n),
// one outer-product sum (a GEMM with the samples as the reduction axis) per
// edge and local state. Per vertex the samples are grouped by local state with
// a stable counting sort; each block sums one chunk of one group into a 64 x 64
// output tile (4 x 4 accumulators per thread, operand rows staged in shared
// memory); the chunk partials are added in chunk order, so the result does not
// depend on the schedule. FP64 throughout (the check form of the gradient).
//
// Correlator: d log|f| / d b_k = t_k, d / d W[k][s] = t_k n_s, d / d W2[k][s][t]
// = t_k n_s n_t / 2, with t_k = tanh(theta_k) (2cosh) or -tan(theta_k) (cos,
// Ising); one thread per parameter sums over the samples in index order.
#include "nqs_kernels.cuh"

namespace nqs {

namespace {

constexpr int kGradChunk = 256;   // samples per block (one chunk of a local-state group)
constexpr int kTile = 64;         // output tile edge
constexpr int kStage = 16;        // samples staged per round

int64_t grad_chunks(int64_t Ns) { return (Ns + kGradChunk - 1) / kGradChunk; }

}  // namespace

size_t grad_scratch_bytes(const AnsatzView& an, int64_t Ns)
{
    return (size_t)an.K * Ns * 4 + (size_t)an.K * 5 * 8 + 512 +     // two 256-byte alignments
           (size_t)grad_chunks(Ns) * an.n_edges * 4 * an.D * an.D * 8;
}

// Stable grouping of the sample indices of vertex i (blockIdx.x) by local state.
__global__ void __launch_bounds__(1024) k_grad_sort(GradArgs a)
{
    __shared__ int wsum[32];
    __shared__ int64_t base;
    const int i = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int32_t* out = a.sidx + (size_t)i * a.Ns;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int sg = 0; sg < 4; ++sg) {
        if (threadIdx.x == 0) a.soff[(size_t)i * 5 + sg] = base;
        for (int64_t t0 = 0; t0 < a.Ns; t0 += blockDim.x) {
            const int64_t s = t0 + threadIdx.x;
            const bool f = s < a.Ns && sigma_at(a.samples[2 * s], a.samples[2 * s + 1], i) == sg;
            const unsigned bal = __ballot_sync(kFull, f);
            if (lane == 0) wsum[warp] = __popc(bal);
            __syncthreads();
            int before = 0, total = 0;
            for (int w = 0; w < nw; ++w) { if (w < warp) before += wsum[w]; total += wsum[w]; }
            if (f) out[base + before + __popc(bal & ((1u << lane) - 1u))] = (int32_t)s;
            __syncthreads();
            if (threadIdx.x == 0) base += total;
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) a.soff[(size_t)i * 5 + 4] = base;
}

// One (edge, local state, chunk, output tile): partial sum over the chunk's samples.
__global__ void __launch_bounds__(256) k_grad_tn(GradArgs a, int n_tiles)
{
    __shared__ double gS[kStage][kTile];
    __shared__ double hS[kStage][kTile];
    __shared__ int32_t sid[kStage];
    const int D = a.an.D, K = a.an.K;
    const int e = blockIdx.z >> 2, sg = blockIdx.z & 3;
    const int chunk = blockIdx.y;
    const int ta = blockIdx.x / n_tiles, tb = blockIdx.x - ta * n_tiles;
    int i, j;
    if (a.an.chain) { i = e; j = e - 1; }
    else {
        j = a.an.pred_idx[e];
        int lo = 0;
        while (a.an.pred_ptr[lo + 1] <= e) ++lo;
        i = lo;
    }
    const int64_t g0 = a.soff[(size_t)i * 5 + sg], g1 = a.soff[(size_t)i * 5 + sg + 1];
    const int64_t c0 = g0 + (int64_t)chunk * kGradChunk;
    if (c0 >= g1) return;                              // beyond this group's chunks
    const int64_t c1 = c0 + kGradChunk < g1 ? c0 + kGradChunk : g1;
    const int a0 = ta * kTile, b0 = tb * kTile;
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    double acc[4][4];
    #pragma unroll
    for (int u = 0; u < 4; ++u)
        #pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
    for (int64_t k0 = c0; k0 < c1; k0 += kStage) {
        const int nk = (int)(c1 - k0 < kStage ? c1 - k0 : kStage);
        if (threadIdx.x < kStage) sid[threadIdx.x] = threadIdx.x < nk ? a.sidx[(size_t)i * a.Ns + k0 + threadIdx.x] : 0;
        __syncthreads();
        for (int q = threadIdx.x; q < kStage * kTile; q += blockDim.x) {
            const int k = q / kTile, c = q - k * kTile;
            double gv = 0.0, hv = 0.0;
            if (k < nk) {
                const int64_t s = sid[k];
                const double* g;
                const double* h;
                int eg, eh;
                if (a.an.chain) {
                    g = a.Renv + ((size_t)s * (K + 1) + i + 1) * D;
                    eg = a.Rexp[(size_t)s * (K + 1) + i + 1];
                    h = a.Lenv + ((size_t)s * (K + 1) + i) * D;
                    eh = a.Lexp[(size_t)s * (K + 1) + i];
                } else {
                    g = a.Gst + ((size_t)s * K + i) * D;
                    eg = a.Gexp[(size_t)s * K + i];
                    h = j < 0 ? nullptr : a.Hst + ((size_t)s * K + j) * D;
                    eh = j < 0 ? 0 : a.Hexp[(size_t)s * K + j];
                }
                const double w = ldexp(a.u[s] / a.psi_mant[s], eg + eh - a.psi_exp[s]);
                if (a0 + c < D) gv = w * g[a0 + c];
                if (b0 + c < D) hv = h ? h[b0 + c] : (b0 + c == 0 ? 1.0 : 0.0);
            }
            gS[k][c] = gv;
            hS[k][c] = hv;
        }
        __syncthreads();
        for (int k = 0; k < nk; ++k) {
            double gr[4], hr[4];
            #pragma unroll
            for (int u = 0; u < 4; ++u) { gr[u] = gS[k][ty * 4 + u]; hr[u] = hS[k][tx * 4 + u]; }
            #pragma unroll
            for (int u = 0; u < 4; ++u)
                #pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(gr[u], hr[v], acc[u][v]);
        }
        __syncthreads();
    }
    double* out = a.part + (((size_t)chunk * a.an.n_edges + e) * 4 + sg) * D * D;
    #pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int ra = a0 + ty * 4 + u;
        if (ra >= D) continue;
        #pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int cb = b0 + tx * 4 + v;
            if (cb < D) out[(size_t)ra * D + cb] = acc[u][v];
        }
    }
}

// grad[e][s] = sum over the group's chunks, in chunk order.
__global__ void k_grad_reduce(GradArgs a)
{
    const int D = a.an.D;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)4 * D * D;
    if (q >= (int64_t)a.an.n_edges * per) return;
    const int e = (int)(q / per);
    const int sg = (int)((q - e * per) / ((int64_t)D * D));
    int i;
    if (a.an.chain) i = e;
    else { int lo = 0; while (a.an.pred_ptr[lo + 1] <= e) ++lo; i = lo; }
    const int64_t n = a.soff[(size_t)i * 5 + sg + 1] - a.soff[(size_t)i * 5 + sg];
    const int64_t nck = (n + kGradChunk - 1) / kGradChunk;
    double acc = a.accumulate ? a.grad_sites[q] : 0.0;
    for (int64_t c = 0; c < nck; ++c) acc += a.part[(size_t)c * a.an.n_edges * per + q];
    a.grad_sites[q] = acc;
}

__global__ void k_grad_rbm(GradArgs a)
{
    const int k = blockIdx.x, K = a.an.K, NH = a.an.n_hidden;
    const int col = threadIdx.x;             // 0..2K-1: W[k][col]; 2K: b[k]
    if (col > 2 * K) return;
    double acc = 0.0;
    for (int64_t s = 0; s < a.Ns; ++s) {
        const double t = corr_dlog(a.an.corr, a.theta[(size_t)s * NH + k]);
        if (col == 2 * K) acc += a.u[s] * t;
        else {
            const uint64_t w = a.samples[2 * s + (col & 1)];
            if ((w >> (col >> 1)) & 1ull) acc += a.u[s] * t;
        }
    }
    if (col == 2 * K) { if (a.grad_b) a.grad_b[k] = (a.accumulate ? a.grad_b[k] : 0.0) + acc; }
    else if (a.grad_W) {
        double* g = a.grad_W + (size_t)k * 2 * K + col;
        *g = (a.accumulate ? *g : 0.0) + acc;
    }
}

__global__ void k_grad_w2(GradArgs a)
{
    const int k = blockIdx.x, K = a.an.K, NH = a.an.n_hidden, N = 2 * K;
    for (int q = threadIdx.x; q < N * N; q += blockDim.x) {
        const int s1 = q / N, s2 = q - s1 * N;
        double acc = 0.0;
        for (int64_t s = 0; s < a.Ns; ++s) {
            const uint64_t w1 = a.samples[2 * s + (s1 & 1)], w2 = a.samples[2 * s + (s2 & 1)];
            if (((w1 >> (s1 >> 1)) & 1ull) && ((w2 >> (s2 >> 1)) & 1ull))
                acc += a.u[s] * (0.5 * corr_dlog(a.an.corr, a.theta[(size_t)s * NH + k]));
        }
        double* g = a.grad_W2 + ((size_t)k * N + s1) * N + s2;
        *g = (a.accumulate ? *g : 0.0) + acc;
    }
}

// Per-sample weights of the energy gradient: u_n = 2 c_n (E_loc(n) - E) / sum c
// (Eq. egrad); reweighted (Sec. 2.3): u_n = 2 c_n f~_n^2 (E_loc(n) - E) / sum c
// with f~^2 = f^2 / B = exp(2 log|f(n)| - log B) and E the mean of E~_loc.
__global__ void k_energy_weights(const double* e_loc, const double* counts, const double* log_f,
                                 int64_t Ns, double e_mean, double sum_c, double log_B, int reweighted,
                                 double* u)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= Ns) return;
    const double cn = counts ? counts[s] : 1.0;
    double w = 2.0 * cn / sum_c;
    if (reweighted) w *= exp(2.0 * log_f[s] - log_B);
    u[s] = w * (e_loc[s] - e_mean);
}

int launch_energy_weights(const double* e_loc, const double* counts, const double* log_f, int64_t Ns,
                          double e_mean, double sum_c, double log_B, bool reweighted, double* u,
                          cudaStream_t st)
{
    if (Ns == 0) return 0;
    k_energy_weights<<<(unsigned)((Ns + 255) / 256), 256, 0, st>>>(e_loc, counts, log_f, Ns, e_mean, sum_c,
                                                                   log_B, reweighted ? 1 : 0, u);
    return 1;
}

int launch_grad_fp64(const GradArgs& a, cudaStream_t st)
{
    const int D = a.an.D;
    int n = 0;
    if (a.grad_sites && a.Ns > 0) {
        k_grad_sort<<<a.an.K, 1024, 0, st>>>(a);
        const int nt = (D + kTile - 1) / kTile;
        dim3 grid((unsigned)(nt * nt), (unsigned)grad_chunks(a.Ns), (unsigned)(a.an.n_edges * 4));
        k_grad_tn<<<grid, 256, 0, st>>>(a, nt);
        const int64_t tot = (int64_t)a.an.n_edges * 4 * D * D;
        k_grad_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(a);
        n += 3;
    }
    if (a.an.n_hidden > 0 && (a.grad_W || a.grad_b)) {
        k_grad_rbm<<<a.an.n_hidden, ((2 * a.an.K + 1 + 31) / 32) * 32, 0, st>>>(a);
        ++n;
    }
    if (a.an.n_hidden > 0 && a.grad_W2 && a.an.corr == 2) {
        k_grad_w2<<<a.an.n_hidden, 256, 0, st>>>(a);
        ++n;
    }
    return n;
}

}  // namespace nqs
