// nqs_api.cu -- the C ABI of include/nqs.h: context, parameter upload,
// host/device pointer staging, and the order of the kernels of each call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/nqs.h"
#include "nqs_kernels.cuh"
#include "nqs_family.cuh"

using namespace nqs;

namespace {

// mixed form with an energy tolerance: samples re-evaluated in FP64 each call
// to check the per-sample error factor (nqs_options.audit_samples = 0)
constexpr int kDefaultAudit = 4;

struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
};

}  // namespace

struct nqs_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    char err[1024] = {0};
    int precision = NQS_PREC_FP64;

    bool has_ham = false;
    int K = 0, na = 0, nb = 0;
    int64_t n_conn = 0;
    double e_core = 0.0;
    HamView hv{};
    DevBuf h1e, eri, pairs, chol;

    bool has_ans = false;
    AnsatzView av{};
    DevBuf A, AT, W, b, pred_ptr, pred_idx;
    DevBuf Af, ATf;           // FP32 copies for the shared-prefix FP32 path
    DevBuf WTf;               // W transposed in FP32, [2K][n_hidden rounded up to 4], zero-padded
                              // (the graph tiles' correlator)
    DevBuf csite, csite64;    // per-site correlator factors, FP32 and FP64 (fam_corr_sites)
    DevBuf ATdf, Adf;         // chain: AT and A as FP32 (hi, lo) pairs (double-FP32 arithmetic)
    bool refine_df = false;   // FP64 tables of the error-budgeted re-evaluation: double-FP32 mat-vecs
    DevBuf tc_img, tc_exps;   // split-FP16 operand images for the tensor-core batches
    bool has_tc = false;

    // staging and workspace
    DevBuf st_samples, st_counts, st_u, st_out0, st_out1, st_out2, st_out3, st_out4;
    DevBuf chunk_cnt, chunk_mask, chunk_off, chunk_w, det_tot, det_off, det_rank, det_coef;
    DevBuf Lenv, Lexp, Renv, Rexp, Hst, Hexp, Gst, Gexp, theta, lc, logf, pmant, pexp, hdiag;
    DevBuf Wtot, draw_rank64, draw_rank, draw_coef, n_unique;
    DevBuf base_det, base_draw, part_det, part_draw, eloc, edet, estoch, summary, derr;
    DevBuf span_det, span_draw;
    // shared-prefix path
    DevBuf fpool, fpoole;      // table rows (G, H, TL, TR of a batch) and their exponents
    DevBuf ftl_end, ftl_idx, ftr_idx, ftl_tot, ftr_tot, ftl_base,
        ftr_base, ftl_ci, ftl_list, ftr_list, ftl_cnt, frbl, frbr, frbl_base,
        frbr_base;
    std::vector<int64_t> det_off_h;
    int64_t fam_matvecs = 0;   // work of the last shared-prefix pass

    // stage accounting (nqs_stage_times)
    int timing = 0;
    int64_t index_base = 0;    // Philox sample counter of samples[0]
    int n_sm = 152;            // multiprocessors of the device
    size_t fam_budget = 0;     // cap on the shared-prefix tables (0: none beyond free/3)
    DevBuf site_cnt, site_offs, site_bounds, site_items, site_scan;
    double energy_tol = 0.0;   // mixed form: re-evaluate heavy samples in FP64 to this bound
    DevBuf part_det_abs, part_draw_abs, eabs, logf_save, summary2, ref_idx, ref_s, ref_c, ref_pos,
        ref_e;
    double stage_ms[NQS_N_STAGES] = {0};
    int64_t stage_launch[NQS_N_STAGES] = {0};
    unsigned long long* noalloc_addr = nullptr;   // device address of the fixed draw scratch
    // normalised readout, correlator kind, gradient and audit options
    DevBuf rv, reta, rw, rc, W2, rnn_cells, rnn_lp, rnn_sg, grad_scr, u_dev, ebar_dev;
    DevBuf tk_rank, tk_off, tk;   // tensor term (Tucker form) of the graph ansatz
    // mixed form of the graph ansatz: matrix images, e_0 columns, state slots
    DevBuf g_img, g_bexp, g_col0, g_slot, g_last, mv_det, mv_draw, g_simg, g_tts, g_rank, g_coef;
    int g_slots = 0, g_maxdeg = 0, g_nbuf = 1;
    bool has_gtc = false;
    char gtc_why[160] = {0};   // why the graph does not fit the tensor-core tiles
    int grad_chunk = 0;        // samples whose environments live at once in the gradient (0: all)
    int audit = 4;             // mixed form: samples re-evaluated in FP64 to check the error factor
    double audit_rel = 0.0, err_factor = 0.0;
    int64_t n_audited = 0;
    const double* last_logf = nullptr;   // log|f| of the last nqs_local_energy batch
    int tile_bps = 4;          // site-step tile launch: blocks per multiprocessor
    int table_mb = 0;          // cap on one sample batch's shared-prefix tables (0: none)
    // autoregressive sampler levels
    std::vector<DevBuf> smp_pa, smp_pb, smp_off, smp_cnt, smp_par, smp_cell;
    DevBuf smp_cand, smp_ccnt, smp_cpos, smp_tabs;
    struct Pending { int stage; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> free_events;
    cudaEvent_t open_event[NQS_N_STAGES] = {nullptr};
};

namespace {

int set_err(nqs_ctx* c, int code, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
    return code;
}

#define CK(call)                                                                        \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return set_err(c, e_ == cudaErrorMemoryAllocation ? NQS_ERR_OOM : NQS_ERR_CUDA, \
                           "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),      \
                           __FILE__, __LINE__);                                         \
    } while (0)

#define TRY(expr)                  \
    do {                           \
        int r_ = (expr);           \
        if (r_ != NQS_OK) return r_; \
    } while (0)

int ensure(nqs_ctx* c, DevBuf& b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.n >= bytes) return NQS_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
    size_t want = bytes + bytes / 8;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return set_err(c, NQS_ERR_OOM, "cudaMalloc(%zu bytes) failed: %s", want,
                       cudaGetErrorString(e));
    }
    b.n = want;
    return NQS_OK;
}

void release(DevBuf& b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.n = 0;
}

bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
int stage_in(nqs_ctx* c, DevBuf& buf, const T* p, size_t n, const T** out)
{
    if (!p || is_device_ptr(p)) {
        *out = p;
        return NQS_OK;
    }
    TRY(ensure(c, buf, n * sizeof(T)));
    if (n) CK(cudaMemcpyAsync(buf.p, p, n * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    *out = (const T*)buf.p;
    return NQS_OK;
}

// Output: device pointer as is, host pointer -> staging buffer copied back later.
template <typename T>
int stage_out(nqs_ctx* c, DevBuf& buf, T* p, size_t n, T** dev, bool* host)
{
    *host = false;
    if (!p) {
        *dev = nullptr;
        return NQS_OK;
    }
    if (is_device_ptr(p)) {
        *dev = p;
        return NQS_OK;
    }
    TRY(ensure(c, buf, n * sizeof(T)));
    *dev = (T*)buf.p;
    *host = true;
    return NQS_OK;
}

template <typename T>
int copy_back(nqs_ctx* c, T* host, const T* dev, size_t n, bool is_host)
{
    if (is_host && n) CK(cudaMemcpyAsync(host, dev, n * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
    return NQS_OK;
}

int bit_length(uint64_t x)
{
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

int64_t binom2(int64_t n) { return n * (n - 1) / 2; }

int check_ready(nqs_ctx* c, bool need_ansatz)
{
    if (!c) return NQS_ERR_INVALID_ARG;
    if (!c->has_ham) return set_err(c, NQS_ERR_STATE, "nqs_set_hamiltonian has not been called");
    if (need_ansatz && !c->has_ans) return set_err(c, NQS_ERR_STATE, "nqs_set_ansatz has not been called");
    return NQS_OK;
}

int read_dev_error(nqs_ctx* c)
{
    DevError e;
    CK(cudaMemcpyAsync(&e, c->derr.p, sizeof(e), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (e.code == 0) return NQS_OK;
    const char* what = "device check failed";
    if (e.detail == 1) what = "sample has an occupied orbital >= n_orb";
    else if (e.detail == 2) what = "sample has the wrong number of alpha or beta electrons";
    else if (e.detail == 3) what = "psi(n) = 0 for sample";
    else if (e.detail == 4) what = "device wait gave up";
    return set_err(c, e.code, "%s (samples[%lld])", what, (long long)e.index);
}

int reset_dev_error(nqs_ctx* c)
{
    TRY(ensure(c, c->derr, sizeof(DevError)));
    CK(cudaMemsetAsync(c->derr.p, 0, sizeof(DevError), c->stream));
    return NQS_OK;
}

cudaEvent_t get_event(nqs_ctx* c)
{
    if (!c->free_events.empty()) {
        cudaEvent_t e = c->free_events.back();
        c->free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void stage_begin(nqs_ctx* c, int id)
{
    if (!c->timing) return;
    c->open_event[id] = get_event(c);
    cudaEventRecord(c->open_event[id], c->stream);
}

void stage_end(nqs_ctx* c, int id)
{
    if (!c->timing || !c->open_event[id]) return;
    cudaEvent_t b = get_event(c);
    cudaEventRecord(b, c->stream);
    c->pending.push_back({id, c->open_event[id], b});
    c->open_event[id] = nullptr;
}

struct StageScope {
    nqs_ctx* c;
    int id;
    StageScope(nqs_ctx* c_, int id_) : c(c_), id(id_) { stage_begin(c, id); }
    ~StageScope() { stage_end(c, id); }
};

#define LAUNCH(stage, expr) (c->stage_launch[(stage)] += (expr))

__global__ void k_check_psi(const double* mant, int64_t Ns, DevError* err, int64_t offset = 0)
{
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < Ns && mant[s] == 0.0) report(err, NQS_ERR_INVALID_ARG, 3, s + offset);
}

int eps_bits(nqs_ctx* c, double eps, uint64_t* bits)
{
    if (!(eps >= 0.0) || !std::isfinite(eps))
        return set_err(c, NQS_ERR_INVALID_ARG, "det_threshold must be finite and >= 0 (got %g)", eps);
    memcpy(bits, &eps, sizeof(eps));
    return NQS_OK;
}

// Remainder weights w = ceil(|H| 2^shift) (Sec. 2.4: P_n(m) proportional to
// |H_nm|, as exact integers). Every remainder element has |H| < eps = f 2^e with
// f in [0.5, 1), so shift = 62 - e - bitlen(n_conn) keeps every per-sample sum
// below 2^62 and fixes the shift before any element is evaluated.
int weight_shift(const nqs_ctx* c, uint64_t eps_bits)
{
    double eps;
    memcpy(&eps, &eps_bits, sizeof(eps));
    int e = 0;
    if (eps > 0.0) std::frexp(eps, &e);
    return 62 - e - c->hv.bitlen_nconn;
}

// Count pass + per-sample scans: det_off (device) and the total on the host;
// with `weights`, also the remainder weight sums per chunk, their per-sample
// inclusive prefix (chunk_w) and totals (Wtot).
int count_pass(nqs_ctx* c, const uint64_t* samples, int64_t Ns, uint64_t eb, int64_t* total,
               bool weights)
{
    const uint32_t nch = (uint32_t)((c->n_conn + 31) / 32);
    TRY(ensure(c, c->chunk_cnt, (size_t)Ns * nch * 4));
    TRY(ensure(c, c->chunk_mask, (size_t)Ns * nch * 4));
    TRY(ensure(c, c->chunk_off, (size_t)Ns * nch * 4));
    TRY(ensure(c, c->det_tot, (size_t)Ns * 8));
    TRY(ensure(c, c->det_off, (size_t)(Ns + 1) * 8));
    if (weights) {
        TRY(ensure(c, c->chunk_w, (size_t)Ns * nch * 8));
        TRY(ensure(c, c->Wtot, (size_t)Ns * 8));
    }
    EnumArgs a{};
    a.h = c->hv;
    a.samples = samples;
    a.eps_bits = eb;
    a.n_chunks = nch;
    a.chunk_cnt = (uint32_t*)c->chunk_cnt.p;
    a.chunk_mask = (uint32_t*)c->chunk_mask.p;
    a.shift = weight_shift(c, eb);
    a.chunk_w = weights ? (uint64_t*)c->chunk_w.p : nullptr;
    StageScope sc(c, NQS_STAGE_COUNT);
    LAUNCH(NQS_STAGE_COUNT, launch_enum(a, Ns, false, c->stream));
    CK(cudaGetLastError());
    if (weights)
        LAUNCH(NQS_STAGE_COUNT, launch_scan_chunks_u64((uint64_t*)c->chunk_w.p, (uint64_t*)c->Wtot.p,
                                                       Ns, nch, c->stream));
    LAUNCH(NQS_STAGE_COUNT, launch_scan_chunks_u32((uint32_t*)c->chunk_cnt.p, (uint32_t*)c->chunk_off.p,
                                                   (int64_t*)c->det_tot.p, Ns, nch, c->stream));
    LAUNCH(NQS_STAGE_COUNT, launch_scan_i64((int64_t*)c->det_tot.p, (int64_t*)c->det_off.p, Ns, c->stream));
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(total, (int64_t*)c->det_off.p + Ns, 8, cudaMemcpyDeviceToHost, c->stream));
    return NQS_OK;
}

// Cells, conditionals and phase signs of the normalised readout for every
// sample (after env_pass with tn = 0, which leaves the correlator and H_nn).
int rnn_env_pass(nqs_ctx* c, const uint64_t* samples, int64_t Ns)
{
    const int K = c->K, D = c->av.D;
    TRY(ensure(c, c->rnn_cells, (size_t)Ns * K * D * 8));
    TRY(ensure(c, c->rnn_lp, (size_t)Ns * K * 8));
    TRY(ensure(c, c->rnn_sg, (size_t)Ns * K));
    RnnEnvArgs r{};
    r.an = c->av;
    r.samples = samples;
    r.Ns = Ns;
    r.cells = (double*)c->rnn_cells.p;
    r.lp = (double*)c->rnn_lp.p;
    r.sg = (int8_t*)c->rnn_sg.p;
    r.log_f = (const double*)c->logf.p;
    r.psi_mant = (double*)c->pmant.p;
    r.psi_exp = (int*)c->pexp.p;
    LAUNCH(NQS_STAGE_ENV, launch_rnn_env(r, c->stream));
    CK(cudaGetLastError());
    return NQS_OK;
}

// tn: 1 = psi(n) and the environments; 2 = psi(n) only (chain, shared-prefix
// path: its FP64 value is the denominator of every ratio of the sample);
// 0 = no tensor-network part (the normalised readout has its own pass)
int env_pass(nqs_ctx* c, const uint64_t* samples, int64_t Ns, bool adjoints, int tn = 1)
{
    const int K = c->K, D = c->av.D, NH = c->av.n_hidden;
    EnvArgs e{};
    e.an = c->av;
    e.h = c->hv;
    e.samples = samples;
    e.Ns = Ns;
    e.tn = tn;
    e.ATdf = (const float2*)c->ATdf.p;
    if (tn == 2 || tn == 3 || tn == 0) {
        // psi(n) only
    } else if (c->av.chain) {
        TRY(ensure(c, c->Lenv, (size_t)Ns * (K + 1) * D * 8));
        TRY(ensure(c, c->Renv, (size_t)Ns * (K + 1) * D * 8));
        TRY(ensure(c, c->Lexp, (size_t)Ns * (K + 1) * 4));
        TRY(ensure(c, c->Rexp, (size_t)Ns * (K + 1) * 4));
        e.Lenv = (double*)c->Lenv.p; e.Lexp = (int*)c->Lexp.p;
        e.Renv = (double*)c->Renv.p; e.Rexp = (int*)c->Rexp.p;
    } else {
        TRY(ensure(c, c->Hst, (size_t)Ns * K * D * 8));
        TRY(ensure(c, c->Hexp, (size_t)Ns * K * 4));
        e.Hst = (double*)c->Hst.p; e.Hexp = (int*)c->Hexp.p;
        if (adjoints) {
            TRY(ensure(c, c->Gst, (size_t)Ns * K * D * 8));
            TRY(ensure(c, c->Gexp, (size_t)Ns * K * 4));
            e.Gst = (double*)c->Gst.p; e.Gexp = (int*)c->Gexp.p;
        }
    }
    TRY(ensure(c, c->theta, (size_t)Ns * (NH ? NH : 1) * 8));
    TRY(ensure(c, c->lc, (size_t)Ns * (NH ? NH : 1) * 8));
    TRY(ensure(c, c->logf, (size_t)Ns * 8));
    TRY(ensure(c, c->pmant, (size_t)Ns * 8));
    TRY(ensure(c, c->pexp, (size_t)Ns * 4));
    TRY(ensure(c, c->hdiag, (size_t)Ns * 8));
    e.theta = (double*)c->theta.p;
    e.lc = (double*)c->lc.p;
    e.log_f = (double*)c->logf.p;
    e.psi_mant = (double*)c->pmant.p;
    e.psi_exp = (int*)c->pexp.p;
    e.h_diag = (double*)c->hdiag.p;
    LAUNCH(NQS_STAGE_ENV, launch_env_fp64(e, c->stream));
    CK(cudaGetLastError());
    return NQS_OK;
}

// Amplitudes over one row set, accumulated into per-chunk partial sums.
// gtc: the mixed form of the graph ansatz (tensor-core tiles of 128 rows),
// which also sums the magnitudes of the terms into *pabs when it is non-NULL.
int amp_pass(nqs_ctx* c, const uint64_t* samples, int64_t Ns, RowSet rows, int64_t total_rows,
             const int64_t* count_dev, DevBuf& base, DevBuf& part, DevBuf& span,
             int64_t max_rows_per_sample, int stage, bool gtc = false, DevBuf* pabs = nullptr,
             DevBuf* mvb = nullptr)
{
    StageScope sc(c, stage);
    const bool rnn = c->av.readout == 1;
    const int R = gtc ? 128 : (rnn ? rnn_rows_per_block() : amp_fp64_rows_per_block(c->av));
    int64_t max_chunks = total_rows / R + Ns;
    if (max_rows_per_sample >= 0) max_chunks = Ns * ((max_rows_per_sample + R - 1) / R);
    TRY(ensure(c, base, (size_t)(Ns + 1) * 8));
    TRY(ensure(c, part, (size_t)(max_chunks ? max_chunks : 1) * 8));
    TRY(ensure(c, span, (size_t)(max_chunks ? max_chunks : 1) * 8));
    LAUNCH(stage, launch_chunk_base(count_dev, R, (int64_t*)base.p, Ns, c->stream));
    rows.count = count_dev;
    rows.chunk_base = (const int64_t*)base.p;
    rows.max_chunks = max_chunks;
    if (mvb) TRY(ensure(c, *mvb, (size_t)(max_chunks ? max_chunks : 1) * 8));
    if (gtc) {
        if (pabs) TRY(ensure(c, *pabs, (size_t)(max_chunks ? max_chunks : 1) * 8));
        // rows with the same first changed vertex side by side: a tile re-runs
        // the vertices its rows need, not those of its earliest row
        const size_t span_rows = rows.begin ? (size_t)total_rows : (size_t)Ns * rows.stride;
        TRY(ensure(c, c->g_rank, (span_rows ? span_rows : 1) * 4));
        TRY(ensure(c, c->g_coef, (span_rows ? span_rows : 1) * 8));
        LAUNCH(stage, launch_graph_sort(c->hv, samples, rows, Ns, c->K, (uint32_t*)c->g_rank.p,
                                        (double*)c->g_coef.p, c->stream));
        rows.rank = (const uint32_t*)c->g_rank.p;
        rows.coef = (const double*)c->g_coef.p;
        GraphTcArgs g{};
        g.an = c->av;
        g.h = c->hv;
        g.samples = samples;
        g.Ns = Ns;
        g.rows = rows;
        g.Hst = (const double*)c->Hst.p; g.Hexp = (const int*)c->Hexp.p;
        TRY(ensure(c, c->g_simg, (size_t)Ns * c->K * 4 * c->av.D));
        TRY(ensure(c, c->g_tts, (size_t)Ns * (((c->av.n_hidden + 3) & ~3) ? ((c->av.n_hidden + 3) & ~3) : 1) * 4));
        g.simg = (unsigned char*)c->g_simg.p;
        g.tts = (float*)c->g_tts.p;
        g.theta = (const double*)c->theta.p;
        g.psi_mant = (const double*)c->pmant.p;
        g.psi_exp = (const int*)c->pexp.p;
        g.bimg = (const unsigned char*)c->g_img.p;
        g.bexp = (const int*)c->g_bexp.p;
        g.col0 = (const float*)c->g_col0.p;
        g.slot = (const int*)c->g_slot.p;
        g.last_use = (const int*)c->g_last.p;
        g.n_slots = c->g_slots;
        g.max_deg = c->g_maxdeg;
        g.nbuf = c->g_nbuf;
        uint32_t cols = 32;
        while (cols < (uint32_t)(c->g_maxdeg * 4 * c->av.D)) cols <<= 1;
        g.tmem_cols = cols;
        g.WT = c->av.n_hidden ? (const float*)c->WTf.p : nullptr;
        g.np = (c->av.n_hidden + 3) & ~3;
        g.partial = (double*)part.p;
        g.partial_abs = pabs ? (double*)pabs->p : nullptr;
        g.span = (int64_t*)span.p;
        g.mv = mvb ? (int64_t*)mvb->p : nullptr;
        g.err = (DevError*)c->derr.p;
        LAUNCH(stage, launch_graph_tiles(g, c->n_sm, c->stream));
        CK(cudaGetLastError());
        return NQS_OK;
    }
    if (rnn) {
        RnnAmpArgs r{};
        r.an = c->av;
        r.h = c->hv;
        r.samples = samples;
        r.Ns = Ns;
        r.rows = rows;
        r.rows_per_block = R;
        r.cells = (const double*)c->rnn_cells.p;
        r.lp = (const double*)c->rnn_lp.p;
        r.sg = (const int8_t*)c->rnn_sg.p;
        r.theta = (const double*)c->theta.p;
        r.lc = (const double*)c->lc.p;
        r.partial = (double*)part.p;
        r.span = (int64_t*)span.p;
        LAUNCH(stage, launch_rnn_amp(r, c->stream));
        CK(cudaGetLastError());
        return NQS_OK;
    }
    AmpArgs a{};
    a.an = c->av;
    a.h = c->hv;
    a.samples = samples;
    a.Ns = Ns;
    a.rows = rows;
    a.rows_per_block = R;
    a.Lenv = (const double*)c->Lenv.p; a.Lexp = (const int*)c->Lexp.p;
    a.Renv = (const double*)c->Renv.p; a.Rexp = (const int*)c->Rexp.p;
    a.Hst = (const double*)c->Hst.p; a.Hexp = (const int*)c->Hexp.p;
    a.theta = (const double*)c->theta.p;
    a.lc = (const double*)c->lc.p;
    a.psi_mant = (const double*)c->pmant.p;
    a.psi_exp = (const int*)c->pexp.p;
    a.partial = (double*)part.p;
    a.span = (int64_t*)span.p;
    a.mv = mvb ? (int64_t*)mvb->p : nullptr;
    LAUNCH(stage, launch_amp_fp64(a, c->stream));
    CK(cudaGetLastError());
    return NQS_OK;
}

// Site-synchronous families, TL clusters and TR rows of one sample batch
// (tensor-core path): boundary vectors and first-site families per sample,
// then count the items per (step, group, sample), read the per-step group
// bounds back, write the items, and one launch per site step.
template <typename T>
int site_tables(nqs_ctx* c, const FamArgs<T>& f, int nbb)
{
    const int K = f.K;
    const int64_t ncnt = (int64_t)K * 8 * nbb;
    TRY(ensure(c, c->site_cnt, (size_t)ncnt * 8));
    TRY(ensure(c, c->site_offs, (size_t)(ncnt + 1) * 8));
    TRY(ensure(c, c->site_bounds, ((size_t)K * 8 + 1) * 8));
    TRY(ensure(c, c->site_scan, (size_t)scan_i64_tmp_elems(ncnt) * 8));
    SiteBufs sb{};
    sb.scan_tmp = (int64_t*)c->site_scan.p;
    sb.counts = (int64_t*)c->site_cnt.p;
    sb.offs = (int64_t*)c->site_offs.p;
    sb.bounds = (int64_t*)c->site_bounds.p;
    LAUNCH(NQS_STAGE_TABLES, fam_site_count(f, sb, nbb, c->stream));
    std::vector<int64_t> bounds((size_t)K * 8 + 1);
    CK(cudaMemcpyAsync(bounds.data(), c->site_bounds.p, bounds.size() * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    TRY(ensure(c, c->site_items, (size_t)(bounds.back() + 1) * sizeof(SiteItem)));
    sb.items = c->site_items.p;
    LAUNCH(NQS_STAGE_TABLES, fam_site_fill(f, sb, nbb, c->stream));
    for (int tau = 0; tau < K; ++tau)
        LAUNCH(NQS_STAGE_TABLES, fam_site_step(f, sb, tau, bounds.data(), c->tile_bps * c->n_sm, c->stream));
    CK(cudaGetLastError());
    return NQS_OK;
}

// Shared-prefix amplitudes of the deterministic and drawn rows (chain ansatz),
// samples processed in batches whose tables fit the memory budget.
template <typename T>
int family_pass(nqs_ctx* c, const uint64_t* ds, int64_t Ns, int64_t total_det, int n_draws,
                bool want_abs)
{
    const int K = c->K, D = c->av.D;
    const size_t nk = (size_t)K * K * 9;
    constexpr int kRows = 128;
    c->fam_matvecs = 0;
    // row chunk bases (128 rows per chunk) over all samples
    TRY(ensure(c, c->base_det, (size_t)(Ns + 1) * 8));
    const int64_t max_det_chunks = total_det / kRows + Ns;
    TRY(ensure(c, c->part_det, (size_t)(max_det_chunks + 1) * 8));
    TRY(ensure(c, c->span_det, (size_t)(max_det_chunks + 1) * 8));
    if (want_abs) TRY(ensure(c, c->part_det_abs, (size_t)(max_det_chunks + 1) * 8));
    LAUNCH(NQS_STAGE_AMP_DET, launch_chunk_base((const int64_t*)c->det_tot.p, kRows, (int64_t*)c->base_det.p, Ns, c->stream));
    const int64_t per_draw = n_draws > 0 ? (n_draws + kRows - 1) / kRows : 0;
    if (n_draws > 0) {
        TRY(ensure(c, c->base_draw, (size_t)(Ns + 1) * 8));
        TRY(ensure(c, c->part_draw, (size_t)(Ns * per_draw + 1) * 8));
        TRY(ensure(c, c->span_draw, (size_t)(Ns * per_draw + 1) * 8));
        if (want_abs) TRY(ensure(c, c->part_draw_abs, (size_t)(Ns * per_draw + 1) * 8));
        LAUNCH(NQS_STAGE_AMP_DET, launch_chunk_base((const int64_t*)c->n_unique.p, kRows, (int64_t*)c->base_draw.p, Ns, c->stream));
    }
    // batch size from a memory budget
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    // the table cap (table_mb, or 32 GiB), never more than a third of the free memory
    const size_t cap = c->table_mb > 0 ? (size_t)c->table_mb << 20 : (size_t)32 << 30;
    size_t budget = std::min<size_t>(cap, free_b / 3);
    if (c->fam_budget > 0) budget = std::min(budget, c->fam_budget);
    const size_t per = fam_bytes_per_sample(K, D, sizeof(T));
    int64_t nb = (int64_t)std::max<size_t>(1, budget / per);
    if (nb > 65535) nb = 65535;
    // equal batches (a short last batch would run its site steps on few items)
    if (nb < Ns) nb = (Ns + (Ns + nb - 1) / nb - 1) / ((Ns + nb - 1) / nb);
    if (nb > Ns) nb = Ns;
    TRY(ensure(c, c->ftl_end, nb * nk * 4));
    TRY(ensure(c, c->ftl_idx, nb * nk * 4));
    TRY(ensure(c, c->ftr_idx, nb * nk * 4));
    TRY(ensure(c, c->ftl_ci, nb * nk * 4));
    TRY(ensure(c, c->ftl_list, nb * nk * 4));
    TRY(ensure(c, c->ftr_list, nb * nk * 4));
    TRY(ensure(c, c->ftl_cnt, nb * 4));
    TRY(ensure(c, c->frbl_base, (nb + 1) * 8));
    TRY(ensure(c, c->frbr_base, (nb + 1) * 8));
    TRY(ensure(c, c->ftl_tot, nb * 8));
    TRY(ensure(c, c->ftr_tot, nb * 8));
    TRY(ensure(c, c->ftl_base, (nb + 1) * 8));
    TRY(ensure(c, c->ftr_base, (nb + 1) * 8));
    const bool dbl = sizeof(T) == 8;
    FamArgs<T> f{};
    f.h = c->hv;
    f.K = K;
    f.div3K = make_fastdiv((uint32_t)(3 * K));
    f.div9K = make_fastdiv((uint32_t)(9 * K));
    f.D = D;
    f.tc = (sizeof(T) == 4 && c->has_tc) ? 1 : 0;
    if (f.tc) {
        f.nmax = 128;                                  // one M = 128 tensor-core tile
        int cols = 32;
        while (cols < D) cols <<= 1;
        f.tc_cols = cols;
        f.tc_mats = (const uint4*)c->tc_img.p;
        f.tc_exp = (const int*)c->tc_exps.p;
    } else {
        // vectors staged per block-wide batch: two [nmax][D] buffers within ~180 KB
        int nm = (int)((180 * 1024) / (2 * (size_t)D * sizeof(T)));
        nm = nm / 4 * 4;
        f.nmax = nm < 4 ? 4 : (nm > 64 ? 64 : nm);
    }
    f.batch_bytes = fam_batch_bytes(D, f.nmax, sizeof(T), f.tc != 0);
    f.err = (DevError*)c->derr.p;
    f.A = (const T*)(dbl ? c->A.p : c->Af.p);
    f.AT = (const T*)(dbl ? c->AT.p : c->ATf.p);
    f.df = (dbl && c->refine_df) ? 1 : 0;
    f.Adf = (const float2*)c->Adf.p;
    f.ATdf = (const float2*)c->ATdf.p;
    f.samples = ds;
    f.n_hidden = c->av.n_hidden;
    f.csite = (const float4*)c->csite.p;
    f.csite64 = (const double4_32a*)c->csite64.p;
    f.theta = (const double*)c->theta.p;
    const int NH = c->av.n_hidden;
    RowSet rd{};
    rd.rank = (const uint32_t*)c->det_rank.p;
    rd.sites = 1;                                   // site words once marked (k_fam_mark)
    rd.coef = (const double*)c->det_coef.p;
    rd.begin = (const int64_t*)c->det_off.p;
    rd.count = (const int64_t*)c->det_tot.p;
    rd.chunk_base = (const int64_t*)c->base_det.p;
    RowSet rs{};
    if (n_draws > 0) {
        rs.rank = (const uint32_t*)c->draw_rank.p;
        rs.coef = (const double*)c->draw_coef.p;
        rs.begin = nullptr;
        rs.stride = n_draws;
        rs.count = (const int64_t*)c->n_unique.p;
        rs.chunk_base = (const int64_t*)c->base_draw.p;
    }
    for (int64_t s0 = 0; s0 < Ns; s0 += nb) {
        const int64_t s1 = std::min(Ns, s0 + nb);
        const int nbb = (int)(s1 - s0);
        f.s0 = s0;
        f.s1 = s1;
        // few samples (a small call, FP64 re-evaluation): spread each sample's
        // correlator factors over several blocks so that about two blocks per SM run
        f.split = nbb >= 2 * c->n_sm ? 1 : std::min(32, (2 * c->n_sm + nbb - 1) / nbb);
        f.pm = (const double*)c->pmant.p + s0; f.pe = (const int*)c->pexp.p + s0;
        f.tl_end = (int*)c->ftl_end.p;
        f.tl_idx = (int*)c->ftl_idx.p;
        f.tr_idx = (int*)c->ftr_idx.p;
        f.tl_total = (int*)c->ftl_tot.p;
        f.tr_total = (int*)c->ftr_tot.p;
        f.tl_ci = (int*)c->ftl_ci.p;
        f.tl_list = (int*)c->ftl_list.p;
        f.tr_list = (int*)c->ftr_list.p;
        f.tl_count = (int*)c->ftl_cnt.p;
        stage_begin(c, NQS_STAGE_TABLES);
        CK(cudaMemsetAsync(c->ftl_end.p, 0xff, (size_t)nbb * nk * 4, c->stream));
        CK(cudaMemsetAsync(c->ftr_idx.p, 0, (size_t)nbb * nk * 4, c->stream));
        // (the families are built with TL and TR, site-synchronously, below)
        {
            // the deterministic rows: marks, and their ranks replaced by site words
            RowSet rk = rd;
            rk.sites = 0;
            LAUNCH(NQS_STAGE_TABLES, fam_launch_mark<T>(f, rk, nbb, (uint32_t*)c->det_rank.p, c->stream));
        }
        if (n_draws > 0) LAUNCH(NQS_STAGE_TABLES, fam_launch_mark<T>(f, rs, nbb, nullptr, c->stream));
        LAUNCH(NQS_STAGE_TABLES, fam_launch_compact<T>(f, nbb, c->stream));
        // packed table offsets per sample of the batch
        {
            std::vector<int> tl(nbb), tr(nbb), tn(nbb);
            CK(cudaMemcpyAsync(tl.data(), c->ftl_tot.p, (size_t)nbb * 4, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaMemcpyAsync(tr.data(), c->ftr_tot.p, (size_t)nbb * 4, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaMemcpyAsync(tn.data(), c->ftl_cnt.p, (size_t)nbb * 4, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            std::vector<int64_t> tlb(nbb + 1), trb(nbb + 1), lb(nbb + 1), rb(nbb + 1);
            tlb[0] = trb[0] = lb[0] = rb[0] = 0;
            for (int i = 0; i < nbb; ++i) {
                tlb[i + 1] = tlb[i] + tl[i];
                trb[i + 1] = trb[i] + tr[i];
                lb[i + 1] = lb[i] + 3 * K + tn[i];
                rb[i + 1] = rb[i] + 3 * K + tr[i];
            }
            CK(cudaMemcpyAsync(c->frbl_base.p, lb.data(), (size_t)(nbb + 1) * 8, cudaMemcpyHostToDevice, c->stream));
            CK(cudaMemcpyAsync(c->frbr_base.p, rb.data(), (size_t)(nbb + 1) * 8, cudaMemcpyHostToDevice, c->stream));
            if (NH > 0) {
                const size_t rl = (size_t)rbm_row_len(NH);
                TRY(ensure(c, c->frbl, (size_t)lb[nbb] * rl * sizeof(T)));
                TRY(ensure(c, c->frbr, (size_t)rb[nbb] * rl * sizeof(T)));
            }
            // work: both family sides (4 + 3t products at step t), every TL entry, every TR row
            c->fam_matvecs += (int64_t)nbb * 2 * (4 * (int64_t)K + 3 * (int64_t)K * (K - 1) / 2) +
                              tlb[nbb] + trb[nbb];
            CK(cudaMemcpyAsync(c->ftl_base.p, tlb.data(), (size_t)(nbb + 1) * 8, cudaMemcpyHostToDevice, c->stream));
            CK(cudaMemcpyAsync(c->ftr_base.p, trb.data(), (size_t)(nbb + 1) * 8, cudaMemcpyHostToDevice, c->stream));
            // one pool of table rows: G families, H families, TL entries, TR rows
            const int64_t fam_rows = (int64_t)nbb * 3 * K * K;
            f.row_H = fam_rows;
            f.row_TL = 2 * fam_rows;
            f.row_TR = f.row_TL + tlb[nbb] + 1;
            const int64_t rows_total = f.row_TR + trb[nbb] + 1;
            if (rows_total >= ((int64_t)1 << 32))
                return set_err(c, NQS_ERR_UNSUPPORTED, "shared-prefix tables of %lld rows exceed 2^32",
                               (long long)rows_total);
            TRY(ensure(c, c->fpool, (size_t)rows_total * D * sizeof(T)));
            TRY(ensure(c, c->fpoole, (size_t)rows_total * 4));
            CK(cudaStreamSynchronize(c->stream));   // the host vectors above must outlive the copies
        }
        f.pool = (T*)c->fpool.p;
        f.pool_e = (int*)c->fpoole.p;
        f.G = f.pool; f.Ge = f.pool_e;
        f.H = f.pool + (size_t)f.row_H * D; f.He = f.pool_e + f.row_H;
        f.tl_base = (const int64_t*)c->ftl_base.p;
        f.tr_base = (const int64_t*)c->ftr_base.p;
        f.TL = f.pool + (size_t)f.row_TL * D; f.TLe = f.pool_e + f.row_TL;
        f.TR = f.pool + (size_t)f.row_TR * D; f.TRe = f.pool_e + f.row_TR;
        f.rbl = (T*)c->frbl.p; f.rbr = (T*)c->frbr.p;
        f.rbl_base = (const int64_t*)c->frbl_base.p;
        f.rbr_base = (const int64_t*)c->frbr_base.p;
        TRY(site_tables(c, f, nbb));
        LAUNCH(NQS_STAGE_TABLES, fam_launch_rbm<T>(f, nbb, c->stream));
        stage_end(c, NQS_STAGE_TABLES);
        stage_begin(c, NQS_STAGE_AMP_DET);
        const int64_t det_rows = c->det_off_h[s1] - c->det_off_h[s0];
        LAUNCH(NQS_STAGE_AMP_DET, fam_launch_rows<T>(f, rd, det_rows / kRows + nbb, (double*)c->part_det.p,
                                                     (int64_t*)c->span_det.p,
                                                     want_abs ? (double*)c->part_det_abs.p : nullptr,
                                                     c->stream));
        stage_end(c, NQS_STAGE_AMP_DET);
        stage_begin(c, NQS_STAGE_AMP_DRAW);
        if (n_draws > 0)
            LAUNCH(NQS_STAGE_AMP_DRAW, fam_launch_rows<T>(f, rs, (int64_t)nbb * per_draw, (double*)c->part_draw.p,
                                                          (int64_t*)c->span_draw.p,
                                                          want_abs ? (double*)c->part_draw_abs.p : nullptr,
                                                          c->stream));
        stage_end(c, NQS_STAGE_AMP_DRAW);
        CK(cudaGetLastError());
    }
    return NQS_OK;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================

extern "C" int nqs_create(nqs_ctx** out, int device, void* cuda_stream)
{
    if (!out) return NQS_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return NQS_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(device) != cudaSuccess) return NQS_ERR_CUDA;
    nqs_ctx* c = new nqs_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device);
    c->stream = (cudaStream_t)cuda_stream;
    *out = c;
    return NQS_OK;
}

extern "C" int nqs_destroy(nqs_ctx* c)
{
    if (!c) return NQS_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    DevBuf* bufs[] = {&c->h1e, &c->eri, &c->pairs, &c->chol, &c->A, &c->AT, &c->W, &c->b,
                      &c->pred_ptr, &c->pred_idx, &c->st_samples, &c->st_counts,
                      &c->st_u, &c->st_out0, &c->st_out1, &c->st_out2, &c->st_out3, &c->st_out4,
                      &c->chunk_cnt, &c->chunk_mask, &c->chunk_off, &c->chunk_w, &c->det_tot,
                      &c->det_off, &c->det_rank, &c->det_coef, &c->Lenv, &c->Lexp, &c->Renv,
                      &c->Rexp, &c->Hst, &c->Hexp, &c->Gst, &c->Gexp, &c->theta, &c->lc,
                      &c->logf, &c->pmant, &c->pexp, &c->hdiag, &c->Wtot, &c->draw_rank64,
                      &c->draw_rank, &c->draw_coef, &c->n_unique, &c->base_det, &c->base_draw,
                      &c->part_det, &c->part_draw, &c->eloc, &c->edet, &c->estoch, &c->summary,
                      &c->derr, &c->span_det, &c->span_draw, &c->Af, &c->ATf,
                      &c->WTf, &c->csite, &c->csite64, &c->ATdf, &c->Adf, &c->fpool, &c->fpoole, &c->ftl_end,
                      &c->ftl_idx, &c->ftr_idx, &c->ftl_tot, &c->ftr_tot, &c->ftl_base,
                      &c->ftr_base, &c->ftl_ci,
                      &c->ftl_list, &c->ftr_list, &c->ftl_cnt, &c->frbl, &c->frbr, &c->frbl_base,
                      &c->frbr_base, &c->tc_img, &c->tc_exps, &c->part_det_abs,
                      &c->part_draw_abs, &c->eabs, &c->logf_save, &c->summary2, &c->ref_idx,
                      &c->ref_s, &c->ref_c, &c->ref_pos, &c->ref_e, &c->site_cnt,
                      &c->site_offs, &c->site_bounds, &c->site_items, &c->site_scan};
    for (DevBuf* b : bufs) release(*b);
    DevBuf* more[] = {&c->rv, &c->reta, &c->rw, &c->rc, &c->W2, &c->rnn_cells, &c->rnn_lp, &c->rnn_sg,
                      &c->grad_scr, &c->u_dev, &c->ebar_dev, &c->smp_cand, &c->smp_ccnt, &c->smp_cpos,
                      &c->smp_tabs, &c->tk_rank, &c->tk_off, &c->tk, &c->g_img, &c->g_bexp,
                      &c->g_col0, &c->g_slot, &c->g_last, &c->mv_det, &c->mv_draw, &c->g_simg,
                      &c->g_tts, &c->g_rank, &c->g_coef};
    for (DevBuf* b : more) release(*b);
    for (auto* v : {&c->smp_pa, &c->smp_pb, &c->smp_off, &c->smp_cnt, &c->smp_par, &c->smp_cell})
        for (DevBuf& b : *v) release(b);
    for (auto& p : c->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (cudaEvent_t e : c->free_events) cudaEventDestroy(e);
    delete c;
    return NQS_OK;
}

extern "C" const char* nqs_last_error(const nqs_ctx* c) { return c ? c->err : "null context"; }

static_assert(sizeof(nqs_options) == 64, "nqs_options layout");

extern "C" int nqs_set_options(nqs_ctx* c, const nqs_options* o)
{
    if (!c || !o) return NQS_ERR_INVALID_ARG;
    c->err[0] = 0;
    if (o->precision != NQS_PREC_FP64 && o->precision != NQS_PREC_MIXED &&
        o->precision != NQS_PREC_FP64_SHARED)
        return set_err(c, NQS_ERR_INVALID_ARG, "unknown precision %d", o->precision);
    for (int i = 0; i < 6; ++i)
        if (o->reserved[i]) return set_err(c, NQS_ERR_INVALID_ARG, "nqs_options.reserved[%d] != 0", i);
    if (o->tile_blocks_per_sm < 0 || o->tile_blocks_per_sm > 32)
        return set_err(c, NQS_ERR_INVALID_ARG, "nqs_options.tile_blocks_per_sm outside 0..32");
    if (o->table_mb < 0) return set_err(c, NQS_ERR_INVALID_ARG, "nqs_options.table_mb < 0");
    c->tile_bps = o->tile_blocks_per_sm ? o->tile_blocks_per_sm : 4;
    c->table_mb = o->table_mb;
    if (o->sample_index_base < 0)
        return set_err(c, NQS_ERR_INVALID_ARG, "nqs_options.sample_index_base < 0");
    if (!(o->energy_tolerance >= 0.0) || !std::isfinite(o->energy_tolerance))
        return set_err(c, NQS_ERR_INVALID_ARG, "nqs_options.energy_tolerance must be finite and >= 0");
    if (o->grad_chunk < 0) return set_err(c, NQS_ERR_INVALID_ARG, "nqs_options.grad_chunk < 0");
    if (o->audit_samples < -1) return set_err(c, NQS_ERR_INVALID_ARG, "nqs_options.audit_samples < -1");
    c->precision = o->precision;
    c->index_base = o->sample_index_base;
    c->energy_tol = o->energy_tolerance;
    c->timing = o->timing ? 1 : 0;
    c->grad_chunk = o->grad_chunk;
    c->audit = o->audit_samples == 0 ? kDefaultAudit : (o->audit_samples < 0 ? 0 : o->audit_samples);
    return NQS_OK;
}

extern "C" int nqs_stage_times(nqs_ctx* c, double* ms, int64_t* launches, int n)
{
    if (!c || n < 0 || n > NQS_N_STAGES) return NQS_ERR_INVALID_ARG;
    c->err[0] = 0;
    cudaSetDevice(c->device);
    CK(cudaStreamSynchronize(c->stream));
    for (auto& p : c->pending) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) c->stage_ms[p.stage] += t;
        else cudaGetLastError();
        c->free_events.push_back(p.a);
        c->free_events.push_back(p.b);
    }
    c->pending.clear();
    for (int i = 0; i < n; ++i) {
        if (ms) ms[i] = c->stage_ms[i];
        if (launches) launches[i] = c->stage_launch[i];
    }
    for (int i = 0; i < NQS_N_STAGES; ++i) { c->stage_ms[i] = 0.0; c->stage_launch[i] = 0; }
    return NQS_OK;
}

extern "C" int nqs_set_hamiltonian(nqs_ctx* c, const double* h1e, const double* cholesky_or_eri,
                                   int n_chol, int K, int na, int nb, double e_core)
{
    if (!c) return NQS_ERR_INVALID_ARG;
    c->err[0] = 0;
    cudaSetDevice(c->device);
    if (K < 1 || K > kMaxOrb) return set_err(c, NQS_ERR_INVALID_ARG, "n_orb = %d outside 1..64", K);
    if (na < 0 || na > K || nb < 0 || nb > K)
        return set_err(c, NQS_ERR_INVALID_ARG, "n_alpha = %d, n_beta = %d outside 0..n_orb", na, nb);
    if (!h1e || !cholesky_or_eri) return set_err(c, NQS_ERR_INVALID_ARG, "null integral pointer");
    if (n_chol < 0) return set_err(c, NQS_ERR_INVALID_ARG, "n_chol = %d < 0", n_chol);
    c->has_ham = false;
    const size_t KK = (size_t)K * K;
    const double* dh;
    TRY(stage_in(c, c->st_out0, h1e, KK, &dh));
    TRY(ensure(c, c->h1e, KK * 8));
    CK(cudaMemcpyAsync(c->h1e.p, dh, KK * 8, cudaMemcpyDeviceToDevice, c->stream));
    TRY(ensure(c, c->eri, KK * KK * 8));
    if (n_chol > 0) {
        const double* dl;
        TRY(stage_in(c, c->st_out1, cholesky_or_eri, (size_t)n_chol * KK, &dl));
        LAUNCH(NQS_STAGE_OTHER, launch_build_eri(dl, n_chol, K, (double*)c->eri.p, c->stream));
        CK(cudaGetLastError());
    } else {
        const double* de;
        TRY(stage_in(c, c->st_out1, cholesky_or_eri, KK * KK, &de));
        LAUNCH(NQS_STAGE_OTHER, launch_swap_eri(de, K, (double*)c->eri.p, c->stream));
        CK(cudaGetLastError());
    }
    // blocks of the canonical order and the pair-unranking tables
    HamView h{};
    h.K = K; h.na = na; h.nb = nb;
    h.no[0] = na; h.no[1] = nb; h.nv[0] = K - na; h.nv[1] = K - nb;
    const int64_t Sa = (int64_t)h.no[0] * h.nv[0], Sb = (int64_t)h.no[1] * h.nv[1];
    const int64_t Daa = binom2(h.no[0]) * binom2(h.nv[0]), Dbb = binom2(h.no[1]) * binom2(h.nv[1]);
    const int64_t nconn = Sa + Sb + Daa + Dbb + Sa * Sb;
    if (nconn >= (1ll << 21))
        return set_err(c, NQS_ERR_UNSUPPORTED, "n_conn = %lld too large", (long long)nconn);
    h.blk[0] = 0; h.blk[1] = (uint32_t)Sa; h.blk[2] = (uint32_t)(Sa + Sb);
    h.blk[3] = (uint32_t)(Sa + Sb + Daa); h.blk[4] = (uint32_t)(Sa + Sb + Daa + Dbb);
    h.blk[5] = (uint32_t)nconn;
    h.div_nv[0] = make_fastdiv(h.nv[0]); h.div_nv[1] = make_fastdiv(h.nv[1]);
    h.div_vpair[0] = make_fastdiv((uint32_t)binom2(h.nv[0]));
    h.div_vpair[1] = make_fastdiv((uint32_t)binom2(h.nv[1]));
    h.div_sb = make_fastdiv((uint32_t)Sb);
    h.n_conn = (uint32_t)nconn;
    h.bitlen_nconn = bit_length((uint64_t)nconn);
    std::vector<uint16_t> tab;
    const int ns[4] = {h.no[0], h.no[1], h.nv[0], h.nv[1]};
    for (int t = 0; t < 4; ++t) {
        h.pair_off[t] = (uint32_t)tab.size();
        for (int i = 0; i < ns[t]; ++i)
            for (int j = i + 1; j < ns[t]; ++j) tab.push_back((uint16_t)(i | (j << 8)));
    }
    if (tab.empty()) tab.push_back(0);
    TRY(ensure(c, c->pairs, tab.size() * 2));
    CK(cudaMemcpyAsync(c->pairs.p, tab.data(), tab.size() * 2, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    h.h1e = (const double*)c->h1e.p;
    h.eri = (const double*)c->eri.p;
    h.pairs = (const uint16_t*)c->pairs.p;
    h.e_core = e_core;
    c->hv = h;
    c->K = K; c->na = na; c->nb = nb;
    c->n_conn = nconn;
    c->e_core = e_core;
    c->has_ham = true;
    if (c->has_ans && c->av.K != K) c->has_ans = false;
    return NQS_OK;
}

extern "C" int nqs_set_ansatz(nqs_ctx* c, const double* site_tensors, int n_edges, int D,
                              const int* pred_ptr, const int* pred_idx, const double* rbm_W,
                              const double* rbm_b, int n_hidden)
{
    if (!c) return NQS_ERR_INVALID_ARG;
    c->err[0] = 0;
    cudaSetDevice(c->device);
    TRY(check_ready(c, false));
    const int K = c->K;
    if (D < 1 || D > 256) return set_err(c, NQS_ERR_INVALID_ARG, "bond_dim = %d outside 1..256", D);
    if (!site_tensors) return set_err(c, NQS_ERR_INVALID_ARG, "site_tensors is NULL");
    if ((pred_ptr == nullptr) != (pred_idx == nullptr))
        return set_err(c, NQS_ERR_INVALID_ARG, "pred_ptr and pred_idx must both be given or both NULL");
    if (n_hidden < 0 || (n_hidden > 0 && (!rbm_W || !rbm_b)))
        return set_err(c, NQS_ERR_INVALID_ARG, "n_hidden = %d with missing rbm_W / rbm_b", n_hidden);
    const bool chain = pred_ptr == nullptr;
    std::vector<int> ptr, idx;
    if (chain) {
        if (n_edges != K) return set_err(c, NQS_ERR_INVALID_ARG, "chain needs n_edges = n_orb (%d), got %d", K, n_edges);
    } else {
        ptr.resize(K + 1);
        if (is_device_ptr(pred_ptr)) cudaMemcpy(ptr.data(), pred_ptr, (K + 1) * 4, cudaMemcpyDeviceToHost);
        else memcpy(ptr.data(), pred_ptr, (K + 1) * 4);
        if (ptr[0] != 0 || ptr[K] != n_edges)
            return set_err(c, NQS_ERR_INVALID_ARG, "pred_ptr must start at 0 and end at n_edges");
        idx.resize(n_edges > 0 ? n_edges : 1);
        if (is_device_ptr(pred_idx)) cudaMemcpy(idx.data(), pred_idx, n_edges * 4, cudaMemcpyDeviceToHost);
        else memcpy(idx.data(), pred_idx, (size_t)n_edges * 4);
        for (int i = 0; i < K; ++i) {
            const int deg = ptr[i + 1] - ptr[i];
            if (deg < 1 || deg > 8)
                return set_err(c, NQS_ERR_INVALID_ARG, "vertex %d has in-degree %d (need 1..8)", i, deg);
            for (int e = ptr[i]; e < ptr[i + 1]; ++e)
                if (idx[e] < -1 || idx[e] >= i)
                    return set_err(c, NQS_ERR_INVALID_ARG, "pred_idx[%d] = %d is not -1 or an earlier vertex of %d", e, idx[e], i);
        }
    }
    c->has_ans = false;
    const size_t nt = (size_t)n_edges * 4 * D * D;
    std::vector<double> hA(nt), hAT(nt);
    if (is_device_ptr(site_tensors)) CK(cudaMemcpy(hA.data(), site_tensors, nt * 8, cudaMemcpyDeviceToHost));
    else memcpy(hA.data(), site_tensors, nt * 8);
    for (size_t m = 0; m < (size_t)n_edges * 4; ++m)
        for (int r = 0; r < D; ++r)
            for (int q = 0; q < D; ++q) hAT[m * D * D + (size_t)q * D + r] = hA[m * D * D + (size_t)r * D + q];
    TRY(ensure(c, c->A, nt * 8));
    TRY(ensure(c, c->AT, nt * 8));
    CK(cudaMemcpy(c->A.p, hA.data(), nt * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->AT.p, hAT.data(), nt * 8, cudaMemcpyHostToDevice));
    if (!chain) {
        TRY(ensure(c, c->pred_ptr, (K + 1) * 4));
        TRY(ensure(c, c->pred_idx, (size_t)n_edges * 4));
        CK(cudaMemcpy(c->pred_ptr.p, ptr.data(), (K + 1) * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->pred_idx.p, idx.data(), (size_t)n_edges * 4, cudaMemcpyHostToDevice));
    }
    if (n_hidden > 0) {
        const size_t nw = (size_t)n_hidden * 2 * K;
        TRY(ensure(c, c->W, nw * 8));
        TRY(ensure(c, c->b, (size_t)n_hidden * 8));
        CK(cudaMemcpy(c->W.p, rbm_W, nw * 8, cudaMemcpyDefault));
        CK(cudaMemcpy(c->b.p, rbm_b, (size_t)n_hidden * 8, cudaMemcpyDefault));
    }
    {
        std::vector<float> fA(nt), fAT(nt);
        for (size_t i = 0; i < nt; ++i) { fA[i] = (float)hA[i]; fAT[i] = (float)hAT[i]; }
        TRY(ensure(c, c->Af, nt * 4));
        TRY(ensure(c, c->ATf, nt * 4));
        CK(cudaMemcpy(c->Af.p, fA.data(), nt * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->ATf.p, fAT.data(), nt * 4, cudaMemcpyHostToDevice));
        if (chain) {
            // (hi, lo) with hi = fl32(x), lo = fl32(x - hi): 48 of the entry's 53 bits
            std::vector<float2> dAT(nt), dA(nt);
            for (size_t i = 0; i < nt; ++i) {
                const float h = (float)hAT[i], g = (float)hA[i];
                dAT[i] = make_float2(h, (float)(hAT[i] - (double)h));
                dA[i] = make_float2(g, (float)(hA[i] - (double)g));
            }
            TRY(ensure(c, c->ATdf, nt * 8));
            TRY(ensure(c, c->Adf, nt * 8));
            CK(cudaMemcpy(c->ATdf.p, dAT.data(), nt * 8, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(c->Adf.p, dA.data(), nt * 8, cudaMemcpyHostToDevice));
        }
        if (n_hidden > 0) {
            // transposed FP32 copy for the graph tiles' correlator: lanes over hidden
            // units read consecutive words of one spin-orbital's column
            const size_t nw = (size_t)n_hidden * 2 * K, np = (size_t)((n_hidden + 3) & ~3);
            std::vector<double> hW(nw);
            CK(cudaMemcpy(hW.data(), c->W.p, nw * 8, cudaMemcpyDeviceToHost));
            std::vector<float> fWT((size_t)2 * K * np, 0.0f);
            for (int k = 0; k < n_hidden; ++k)
                for (int q = 0; q < 2 * K; ++q) fWT[(size_t)q * np + k] = (float)hW[(size_t)k * 2 * K + q];
            TRY(ensure(c, c->WTf, fWT.size() * 4));
            CK(cudaMemcpy(c->WTf.p, fWT.data(), fWT.size() * 4, cudaMemcpyHostToDevice));
            TRY(ensure(c, c->csite, (size_t)K * 12 * np * 16));
            TRY(ensure(c, c->csite64, (size_t)K * 12 * np * 32));
            fam_corr_sites((const double*)c->W.p, K, n_hidden, (float4*)c->csite.p, (double4_32a*)c->csite64.p,
                           c->stream);
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(c->stream));
        }
    }
    AnsatzView a{};
    a.K = K; a.D = D; a.n_edges = n_edges; a.chain = chain ? 1 : 0;
    a.pred_ptr = chain ? nullptr : (const int*)c->pred_ptr.p;
    a.pred_idx = chain ? nullptr : (const int*)c->pred_idx.p;
    a.A = (const double*)c->A.p;
    a.AT = (const double*)c->AT.p;
    a.n_hidden = n_hidden;
    a.W = n_hidden ? (const double*)c->W.p : nullptr;
    a.b = n_hidden ? (const double*)c->b.p : nullptr;
    a.readout = 0;                 // linear readout and 2cosh correlator until set otherwise
    a.mask_na = c->na;
    a.mask_nb = c->nb;
    a.corr = 0;
    c->av = a;
    c->has_tc = false;
    // tensor-core batches: D % 16 == 0 up to 128 in one reduction chunk, or
    // 192 / 256 in chunks of 64 (N = D <= 256 accumulator columns)
    if (chain && D % 16 == 0 && (D <= 128 || (D % 64 == 0 && D <= 256))) {
        std::vector<unsigned char> img;
        std::vector<int> ex;
        fam_tc_images(hA.data(), K, D, img, ex);
        TRY(ensure(c, c->tc_img, img.size()));
        TRY(ensure(c, c->tc_exps, ex.size() * 4));
        CK(cudaMemcpy(c->tc_img.p, img.data(), img.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->tc_exps.p, ex.data(), ex.size() * 4, cudaMemcpyHostToDevice));
        c->has_tc = true;
    }
    c->has_gtc = false;
    c->gtc_why[0] = 0;
    if (!chain) {
        GraphTcPlan gp;
        const char* why = nullptr;
        if (graph_tc_plan(hA.data(), ptr.data(), idx.data(), K, D, n_hidden, gp, &why)) {
            TRY(ensure(c, c->g_img, gp.img.size()));
            TRY(ensure(c, c->g_bexp, gp.bexp.size() * 4));
            TRY(ensure(c, c->g_col0, gp.col0.size() * 4));
            TRY(ensure(c, c->g_slot, (size_t)K * 4));
            TRY(ensure(c, c->g_last, (size_t)K * 4));
            CK(cudaMemcpy(c->g_img.p, gp.img.data(), gp.img.size(), cudaMemcpyHostToDevice));
            CK(cudaMemcpy(c->g_bexp.p, gp.bexp.data(), gp.bexp.size() * 4, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(c->g_col0.p, gp.col0.data(), gp.col0.size() * 4, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(c->g_slot.p, gp.slot.data(), (size_t)K * 4, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(c->g_last.p, gp.last_use.data(), (size_t)K * 4, cudaMemcpyHostToDevice));
            c->g_slots = gp.n_slots;
            c->g_maxdeg = gp.max_deg;
            c->g_nbuf = gp.nbuf;
            c->has_gtc = true;
        } else {
            snprintf(c->gtc_why, sizeof(c->gtc_why), "%s", why ? why : "unsupported graph");
        }
    }
    CK(cudaStreamSynchronize(c->stream));
    c->has_ans = true;
    return NQS_OK;
}

extern "C" int nqs_set_readout(nqs_ctx* c, const double* v, const double* eta, const double* w,
                               const double* cst, int constrained)
{
    if (!c) return NQS_ERR_INVALID_ARG;
    c->err[0] = 0;
    cudaSetDevice(c->device);
    TRY(check_ready(c, true));
    const int K = c->K, D = c->av.D;
    if (!v && !eta && !w && !cst) {
        c->av.readout = 0;
        return NQS_OK;
    }
    if (!v || !eta || !w || !cst)
        return set_err(c, NQS_ERR_INVALID_ARG, "nqs_set_readout: v, eta, w and c must all be given (or all NULL)");
    std::vector<double> he((size_t)K * D);
    CK(cudaMemcpy(he.data(), eta, he.size() * 8, cudaMemcpyDefault));
    for (size_t q = 0; q < he.size(); ++q)
        if (!(he[q] >= 0.0) || !std::isfinite(he[q]))
            return set_err(c, NQS_ERR_INVALID_ARG, "nqs_set_readout: eta[%zu] = %g is not finite and >= 0", q, he[q]);
    TRY(ensure(c, c->rv, (size_t)K * 4 * D * 8));
    TRY(ensure(c, c->reta, (size_t)K * D * 8));
    TRY(ensure(c, c->rw, (size_t)K * D * 8));
    TRY(ensure(c, c->rc, (size_t)K * 8));
    CK(cudaMemcpy(c->rv.p, v, (size_t)K * 4 * D * 8, cudaMemcpyDefault));
    CK(cudaMemcpy(c->reta.p, he.data(), (size_t)K * D * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->rw.p, w, (size_t)K * D * 8, cudaMemcpyDefault));
    CK(cudaMemcpy(c->rc.p, cst, (size_t)K * 8, cudaMemcpyDefault));
    c->av.rv = (const double*)c->rv.p;
    c->av.reta = (const double*)c->reta.p;
    c->av.rw = (const double*)c->rw.p;
    c->av.rc = (const double*)c->rc.p;
    c->av.mask_na = constrained ? c->na : -1;
    c->av.mask_nb = constrained ? c->nb : -1;
    c->av.readout = 1;
    return NQS_OK;
}

extern "C" int nqs_set_correlator(nqs_ctx* c, int kind, const double* W2)
{
    if (!c) return NQS_ERR_INVALID_ARG;
    c->err[0] = 0;
    cudaSetDevice(c->device);
    TRY(check_ready(c, true));
    if (kind < NQS_CORR_COSH || kind > NQS_CORR_ISING)
        return set_err(c, NQS_ERR_INVALID_ARG, "unknown correlator kind %d", kind);
    if (kind == NQS_CORR_ISING && c->av.n_hidden > 0 && !W2)
        return set_err(c, NQS_ERR_INVALID_ARG, "the Ising-RBM correlator needs W2");
    if (kind == NQS_CORR_ISING && c->av.n_hidden > 0) {
        const size_t n = (size_t)c->av.n_hidden * 4 * c->K * c->K;
        TRY(ensure(c, c->W2, n * 8));
        CK(cudaMemcpy(c->W2.p, W2, n * 8, cudaMemcpyDefault));
        c->av.W2 = (const double*)c->W2.p;
    }
    c->av.corr = kind;
    return NQS_OK;
}

extern "C" int nqs_set_tensor_term(nqs_ctx* c, const int* ranks, const double* params, int64_t n_params)
{
    if (!c) return NQS_ERR_INVALID_ARG;
    c->err[0] = 0;
    cudaSetDevice(c->device);
    TRY(check_ready(c, true));
    const int K = c->K, D = c->av.D;
    if (!ranks) {
        c->av.tk_rank = nullptr;
        c->av.tk_off = nullptr;
        c->av.tk = nullptr;
        c->av.tk_zy = 0;
        return NQS_OK;
    }
    if (c->av.chain) return set_err(c, NQS_ERR_INVALID_ARG, "the tensor term needs a graph ansatz (in-degree >= 2)");
    std::vector<int> rk((size_t)K), ptr((size_t)K + 1);
    CK(cudaMemcpy(rk.data(), ranks, (size_t)K * 4, cudaMemcpyDefault));
    CK(cudaMemcpy(ptr.data(), c->pred_ptr.p, (size_t)(K + 1) * 4, cudaMemcpyDeviceToHost));
    std::vector<long long> off((size_t)K, -1);
    long long total = 0;
    int zy = 0;
    for (int i = 0; i < K; ++i) {
        const int d = ptr[i + 1] - ptr[i], r = rk[(size_t)i];
        if (r < 0 || r > 64) return set_err(c, NQS_ERR_INVALID_ARG, "tensor-term rank %d of vertex %d outside 0..64", r, i);
        if (r == 0 || d < 2) continue;
        double core = 1.0;
        for (int k = 0; k <= d; ++k) core *= r;
        if (core > 1e8) return set_err(c, NQS_ERR_INVALID_ARG, "tensor-term core of vertex %d has %g entries", i, core);
        off[(size_t)i] = total;
        total += 4 * (long long)core + (long long)(d + 1) * D * r;
        zy = std::max(zy, (d + 4) * r);      // z [d][r] and y of the four local states
    }
    if (n_params != total)
        return set_err(c, NQS_ERR_INVALID_ARG, "n_params = %lld, the ranks and in-degrees need %lld",
                       (long long)n_params, total);
    TRY(ensure(c, c->tk_rank, (size_t)K * 4));
    TRY(ensure(c, c->tk_off, (size_t)K * 8));
    TRY(ensure(c, c->tk, (size_t)(total ? total : 1) * 8));
    CK(cudaMemcpy(c->tk_rank.p, rk.data(), (size_t)K * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->tk_off.p, off.data(), (size_t)K * 8, cudaMemcpyHostToDevice));
    if (total) CK(cudaMemcpy(c->tk.p, params, (size_t)total * 8, cudaMemcpyDefault));
    c->av.tk_rank = (const int*)c->tk_rank.p;
    c->av.tk_off = (const long long*)c->tk_off.p;
    c->av.tk = (const double*)c->tk.p;
    c->av.tk_zy = zy;
    return NQS_OK;
}

extern "C" int nqs_connected(nqs_ctx* c, const uint64_t* samples, int64_t Ns, double eps,
                             int64_t* offsets, uint32_t* rank, uint64_t* dets, double* H,
                             int8_t* sign, int64_t capacity)
{
    if (!c) return NQS_ERR_INVALID_ARG;
    c->err[0] = 0;
    cudaSetDevice(c->device);
    TRY(check_ready(c, false));
    if (Ns < 0 || (Ns > 0 && !samples) || !offsets)
        return set_err(c, NQS_ERR_INVALID_ARG, "bad samples / offsets arguments");
    uint64_t eb;
    TRY(eps_bits(c, eps, &eb));
    if (Ns == 0) {
        int64_t z = 0;
        if (is_device_ptr(offsets)) CK(cudaMemcpy(offsets, &z, 8, cudaMemcpyHostToDevice));
        else offsets[0] = 0;
        return NQS_OK;
    }
    const uint64_t* ds;
    TRY(stage_in(c, c->st_samples, samples, (size_t)Ns * 2, &ds));
    TRY(reset_dev_error(c));
    LAUNCH(NQS_STAGE_OTHER, launch_validate(ds, Ns, c->K, c->na, c->nb, (DevError*)c->derr.p, c->stream));
    int64_t total = 0;
    TRY(count_pass(c, ds, Ns, eb, &total, false));
    TRY(read_dev_error(c));
    int64_t* doff;
    bool hoff;
    TRY(stage_out(c, c->st_out4, offsets, (size_t)Ns + 1, &doff, &hoff));
    CK(cudaMemcpyAsync(doff, c->det_off.p, (size_t)(Ns + 1) * 8, cudaMemcpyDeviceToDevice, c->stream));
    TRY(copy_back(c, offsets, doff, (size_t)Ns + 1, hoff));
    const bool want = rank || dets || H || sign;
    if (want && capacity < total) {
        CK(cudaStreamSynchronize(c->stream));
        return set_err(c, NQS_ERR_INVALID_ARG, "capacity %lld < %lld entries", (long long)capacity, (long long)total);
    }
    if (want && total > 0) {
        uint32_t* drank; uint64_t* ddet; double* dH; int8_t* dsg;
        bool h0, h1, h2, h3;
        TRY(stage_out(c, c->st_out0, rank, (size_t)total, &drank, &h0));
        TRY(stage_out(c, c->st_out1, dets, (size_t)total * 2, &ddet, &h1));
        TRY(stage_out(c, c->st_out2, H, (size_t)total, &dH, &h2));
        TRY(stage_out(c, c->st_out3, sign, (size_t)total, &dsg, &h3));
        EnumArgs a{};
        a.h = c->hv;
        a.samples = ds;
        a.eps_bits = eb;
        a.n_chunks = (uint32_t)((c->n_conn + 31) / 32);
        a.chunk_cnt = (uint32_t*)c->chunk_cnt.p;
        a.chunk_mask = (uint32_t*)c->chunk_mask.p;
        a.chunk_off = (const uint32_t*)c->chunk_off.p;
        a.det_off = (const int64_t*)c->det_off.p;
        a.out_rank = drank; a.out_det = ddet; a.out_H = dH; a.out_sign = dsg;
        LAUNCH(NQS_STAGE_WRITE, launch_enum(a, Ns, true, c->stream));
        CK(cudaGetLastError());
        TRY(copy_back(c, rank, drank, (size_t)total, h0));
        TRY(copy_back(c, dets, ddet, (size_t)total * 2, h1));
        TRY(copy_back(c, H, dH, (size_t)total, h2));
        TRY(copy_back(c, sign, dsg, (size_t)total, h3));
    }
    CK(cudaStreamSynchronize(c->stream));
    return NQS_OK;
}

extern "C" int nqs_amplitude(nqs_ctx* c, const uint64_t* dets, int64_t n, double* log_abs,
                             int8_t* sign)
{
    if (!c) return NQS_ERR_INVALID_ARG;
    c->err[0] = 0;
    cudaSetDevice(c->device);
    TRY(check_ready(c, true));
    if (n < 0 || (n > 0 && (!dets || !log_abs || !sign)))
        return set_err(c, NQS_ERR_INVALID_ARG, "bad dets / outputs");
    if (n == 0) return NQS_OK;
    const uint64_t* dd;
    TRY(stage_in(c, c->st_samples, dets, (size_t)n * 2, &dd));
    TRY(reset_dev_error(c));
    LAUNCH(NQS_STAGE_OTHER, launch_validate(dd, n, c->K, c->na, c->nb, (DevError*)c->derr.p, c->stream));
    double* dla; int8_t* dsg;
    bool h0, h1;
    TRY(stage_out(c, c->st_out0, log_abs, (size_t)n, &dla, &h0));
    TRY(stage_out(c, c->st_out1, sign, (size_t)n, &dsg, &h1));
    TRY(read_dev_error(c));
    if (c->av.readout == 1) LAUNCH(NQS_STAGE_OTHER, launch_rnn_full(c->av, dd, n, dla, dsg, c->stream));
    else LAUNCH(NQS_STAGE_OTHER, launch_full_amp_fp64(c->av, dd, n, dla, dsg, c->stream));
    CK(cudaGetLastError());
    TRY(copy_back(c, log_abs, dla, (size_t)n, h0));
    TRY(copy_back(c, sign, dsg, (size_t)n, h1));
    if (h0 || h1) CK(cudaStreamSynchronize(c->stream));
    return NQS_OK;
}

namespace {

// Steps shared by nqs_draws and nqs_local_energy: weights, prefix, draws.
// Steps after the count pass (which made the weights when draws follow):
// the deterministic lists, then the draws.
int draw_pass(nqs_ctx* c, const uint64_t* ds, int64_t Ns, uint64_t eb, int n_draws,
              uint64_t seed, int64_t* rank_out, bool write_dets, const int64_t* index = nullptr)
{
    const uint32_t nch = (uint32_t)((c->n_conn + 31) / 32);
    if (write_dets) {
        EnumArgs a{};
        a.h = c->hv;
        a.samples = ds;
        a.eps_bits = eb;
        a.n_chunks = nch;
        a.chunk_cnt = (uint32_t*)c->chunk_cnt.p;
        a.chunk_mask = (uint32_t*)c->chunk_mask.p;
        a.chunk_off = (const uint32_t*)c->chunk_off.p;
        a.det_off = (const int64_t*)c->det_off.p;
        a.out_rank = (uint32_t*)c->det_rank.p;
        a.out_H = (double*)c->det_coef.p;
        StageScope sc(c, NQS_STAGE_WRITE);
        LAUNCH(NQS_STAGE_WRITE, launch_enum(a, Ns, true, c->stream));
        CK(cudaGetLastError());
    }
    if (n_draws > 0) {
        StageScope sc(c, NQS_STAGE_DRAW);
        DrawArgs d{};
        d.h = c->hv;
        d.samples = ds;
        d.Ns = Ns;
        d.eps_bits = eb;
        d.n_chunks = nch;
        d.chunk_pre = (const uint64_t*)c->chunk_w.p;
        d.shift = weight_shift(c, eb);
        d.n_draws = n_draws;
        d.seed = seed;
        d.index_base = c->index_base;
        d.index = index;
        d.out_rank = rank_out;
        LAUNCH(NQS_STAGE_DRAW, launch_draws(d, c->stream));
    }
    CK(cudaGetLastError());
    return NQS_OK;
}

}  // namespace

extern "C" int nqs_draws(nqs_ctx* c, const uint64_t* samples, int64_t Ns, double eps,
                         int n_draws, uint64_t seed, int64_t* ranks, uint64_t* w_total)
{
    if (!c) return NQS_ERR_INVALID_ARG;
    c->err[0] = 0;
    cudaSetDevice(c->device);
    TRY(check_ready(c, false));
    if (Ns < 0 || n_draws < 0 || (Ns > 0 && !samples) || (Ns > 0 && n_draws > 0 && !ranks))
        return set_err(c, NQS_ERR_INVALID_ARG, "bad samples / n_draws / ranks arguments");
    uint64_t eb;
    TRY(eps_bits(c, eps, &eb));
    if (Ns == 0) return NQS_OK;
    const uint64_t* ds;
    TRY(stage_in(c, c->st_samples, samples, (size_t)Ns * 2, &ds));
    TRY(reset_dev_error(c));
    LAUNCH(NQS_STAGE_OTHER, launch_validate(ds, Ns, c->K, c->na, c->nb, (DevError*)c->derr.p, c->stream));
    int64_t total = 0;
    TRY(count_pass(c, ds, Ns, eb, &total, n_draws > 0 || w_total != nullptr));
    TRY(read_dev_error(c));
    int64_t* dr = nullptr;
    bool hr = false;
    if (n_draws > 0) TRY(stage_out(c, c->st_out0, ranks, (size_t)Ns * n_draws, &dr, &hr));
    TRY(draw_pass(c, ds, Ns, eb, n_draws, seed, dr, false));
    if (n_draws > 0) TRY(copy_back(c, ranks, dr, (size_t)Ns * n_draws, hr));
    if (w_total) {
        uint64_t* dw;
        bool hw;
        TRY(stage_out(c, c->st_out1, w_total, (size_t)Ns, &dw, &hw));
        CK(cudaMemcpyAsync(dw, c->Wtot.p, (size_t)Ns * 8, cudaMemcpyDeviceToDevice, c->stream));
        TRY(copy_back(c, w_total, dw, (size_t)Ns, hw));
    }
    CK(cudaStreamSynchronize(c->stream));
    return NQS_OK;
}

namespace {

// Per-sample error of the mixed form relative to max(|E_loc|, e_abs) that the
// refinement starts from: the bound the parity tests hold it to (measured 1.3e-7
// to 2e-7 on the benchmark workloads, up to 6.8e-7 at D = 256, where the FP32
// accumulations are longest); each call checks it on an FP64 audit sample.
constexpr double kMixedRelError = 1e-6;

// The local-energy pipeline on device-resident samples in precision `prec`:
// E_loc into de, |H_nn| + sum |terms| into deabs (shared-prefix forms only; may
// be NULL), the summary into c->summary when want_summary. `dindex` (may be
// NULL) gives each sample's Philox counter.
int le_core(nqs_ctx* c, const uint64_t* ds, const double* dc, int64_t Ns, uint64_t eb, int n_draws,
            uint64_t seed, int prec, const int64_t* dindex, double* de, double* deabs,
            bool want_summary)
{
    TRY(reset_dev_error(c));
    const bool rnn = c->av.readout == 1;
    const bool shared = c->av.chain && (prec == NQS_PREC_MIXED || prec == NQS_PREC_FP64_SHARED);
    const bool gtc = !c->av.chain && prec == NQS_PREC_MIXED;
    const bool graph = !c->av.chain && !rnn;
    if (!c->av.chain && prec == NQS_PREC_FP64_SHARED)
        return set_err(c, NQS_ERR_UNSUPPORTED,
                       "graph ansatze have no shared-prefix form (NQS_PREC_FP64 or NQS_PREC_MIXED)");
    if (gtc && !c->has_gtc)
        return set_err(c, NQS_ERR_UNSUPPORTED, "mixed form of this graph ansatz: %s", c->gtc_why);
    if (gtc && (rnn || c->av.tk_rank || c->av.corr == NQS_CORR_ISING))
        return set_err(c, NQS_ERR_UNSUPPORTED,
                       "the mixed form of a graph ansatz needs the linear readout, no tensor term and "
                       "the 2cosh or cos correlator; use NQS_PREC_FP64");
    if (shared && (rnn || c->av.corr != NQS_CORR_COSH))
        return set_err(c, NQS_ERR_UNSUPPORTED,
                       "the shared-prefix forms need the linear readout and the 2cosh correlator; "
                       "use NQS_PREC_FP64");
    if (shared && c->av.n_hidden > 512)
        return set_err(c, NQS_ERR_UNSUPPORTED, "shared-prefix path supports n_hidden <= 512");
    if (deabs && !shared && !gtc) return set_err(c, NQS_ERR_STATE, "e_abs needs a mixed or shared-prefix form");
    {
        StageScope sc(c, NQS_STAGE_ENV);
        LAUNCH(NQS_STAGE_ENV, launch_validate(ds, Ns, c->K, c->na, c->nb, (DevError*)c->derr.p, c->stream));
        // the mixed form takes psi(n) in double-FP32 arithmetic, the FP64 forms in FP64
        TRY(env_pass(c, ds, Ns, false, rnn ? 0 : (shared ? (prec == NQS_PREC_MIXED ? 3 : 2) : 1)));
        if (rnn) TRY(rnn_env_pass(c, ds, Ns));
        k_check_psi<<<(unsigned)((Ns + 255) / 256), 256, 0, c->stream>>>((const double*)c->pmant.p, Ns,
                                                                       (DevError*)c->derr.p);
        LAUNCH(NQS_STAGE_ENV, 1);
    }
    int64_t total = 0;
    TRY(count_pass(c, ds, Ns, eb, &total, n_draws > 0));
    if (shared) {
        c->det_off_h.resize(Ns + 1);
        CK(cudaMemcpyAsync(c->det_off_h.data(), c->det_off.p, (size_t)(Ns + 1) * 8, cudaMemcpyDeviceToHost, c->stream));
    }
    TRY(read_dev_error(c));
    TRY(ensure(c, c->det_rank, (size_t)total * 4));
    TRY(ensure(c, c->det_coef, (size_t)total * 8));
    if (n_draws > 0) {
        TRY(ensure(c, c->draw_rank64, (size_t)Ns * n_draws * 8));
        TRY(ensure(c, c->draw_rank, (size_t)Ns * n_draws * 4));
        TRY(ensure(c, c->draw_coef, (size_t)Ns * n_draws * 8));
        TRY(ensure(c, c->n_unique, (size_t)Ns * 8));
    }
    TRY(draw_pass(c, ds, Ns, eb, n_draws, seed, (int64_t*)c->draw_rank64.p, true, dindex));
    if (n_draws > 0) {
        StageScope sc(c, NQS_STAGE_DRAW);
        DedupArgs d{};
        d.h = c->hv;
        d.samples = ds;
        d.ranks = (const int64_t*)c->draw_rank64.p;
        d.n_draws = n_draws;
        int p2 = 1;
        while (p2 < n_draws) p2 <<= 1;
        d.pow2 = p2;
        d.shift = weight_shift(c, eb);
        d.W = (const uint64_t*)c->Wtot.p;
        d.out_rank = (uint32_t*)c->draw_rank.p;
        d.out_coef = (double*)c->draw_coef.p;
        d.n_unique = (int64_t*)c->n_unique.p;
        LAUNCH(NQS_STAGE_DRAW, launch_dedup(d, Ns, c->stream));
        CK(cudaGetLastError());
    }
    if (shared) {
        if (prec == NQS_PREC_MIXED) TRY(family_pass<float>(c, ds, Ns, total, n_draws, deabs != nullptr));
        else TRY(family_pass<double>(c, ds, Ns, total, n_draws, deabs != nullptr));
    } else {
        // amplitudes: deterministic rows, then the distinct drawn rows
        RowSet rd{};
        rd.rank = (const uint32_t*)c->det_rank.p;
        rd.coef = (const double*)c->det_coef.p;
        rd.begin = (const int64_t*)c->det_off.p;
        TRY(amp_pass(c, ds, Ns, rd, total, (const int64_t*)c->det_tot.p, c->base_det, c->part_det,
                     c->span_det, -1, NQS_STAGE_AMP_DET, gtc, deabs ? &c->part_det_abs : nullptr,
                     graph ? &c->mv_det : nullptr));
        if (n_draws > 0) {
            RowSet rs{};
            rs.rank = (const uint32_t*)c->draw_rank.p;
            rs.coef = (const double*)c->draw_coef.p;
            rs.begin = nullptr;
            rs.stride = n_draws;
            TRY(amp_pass(c, ds, Ns, rs, (int64_t)Ns * n_draws, (const int64_t*)c->n_unique.p,
                         c->base_draw, c->part_draw, c->span_draw, n_draws, NQS_STAGE_AMP_DRAW, gtc,
                         deabs ? &c->part_draw_abs : nullptr, graph ? &c->mv_draw : nullptr));
        }
    }
    TRY(ensure(c, c->summary, 8 * 8));
    FinalArgs f{};
    f.Ns = Ns;
    f.h_diag = (const double*)c->hdiag.p;
    f.part_det = (const double*)c->part_det.p;
    f.base_det = (const int64_t*)c->base_det.p;
    f.part_draw = n_draws > 0 ? (const double*)c->part_draw.p : nullptr;
    f.base_draw = n_draws > 0 ? (const int64_t*)c->base_draw.p : nullptr;
    f.counts = dc;
    f.log_f = (const double*)c->logf.p;
    f.det_off = (const int64_t*)c->det_off.p;
    f.n_unique = n_draws > 0 ? (const int64_t*)c->n_unique.p : nullptr;
    f.e_loc = de;
    f.span_det = (const int64_t*)c->span_det.p;
    f.span_draw = n_draws > 0 ? (const int64_t*)c->span_draw.p : nullptr;
    f.summary = want_summary ? (double*)c->summary.p : nullptr;
    f.e_abs = deabs;
    f.part_det_abs = deabs ? (const double*)c->part_det_abs.p : nullptr;
    f.part_draw_abs = deabs && n_draws > 0 ? (const double*)c->part_draw_abs.p : nullptr;
    f.mv_det = graph ? (const int64_t*)c->mv_det.p : nullptr;
    f.mv_draw = graph && n_draws > 0 ? (const int64_t*)c->mv_draw.p : nullptr;
    {
        StageScope sc(c, NQS_STAGE_FINAL);
        LAUNCH(NQS_STAGE_FINAL, launch_finalize(f, c->stream));
    }
    CK(cudaGetLastError());
    if (shared || gtc) TRY(read_dev_error(c));
    return NQS_OK;
}

// FP64 re-evaluation (the shared-prefix form for chains, the plain form for
// graphs) of the samples `pick` (ascending) of a mixed-form result: their E_loc in de are replaced; the FP64 values also go
// to `fp64` (host, same order as pick) when it is non-NULL.
int reevaluate(nqs_ctx* c, const uint64_t* ds, const double* dc, const std::vector<int64_t>& pick,
               uint64_t eb, int n_draws, uint64_t seed, double* de, std::vector<double>* fp64)
{
    const int64_t k = (int64_t)pick.size();
    if (k == 0) return NQS_OK;
    TRY(ensure(c, c->ref_idx, (size_t)k * 8));
    TRY(ensure(c, c->ref_s, (size_t)k * 16));
    TRY(ensure(c, c->ref_c, (size_t)k * 8));
    TRY(ensure(c, c->ref_pos, (size_t)k * 8));
    TRY(ensure(c, c->ref_e, (size_t)k * 8));
    CK(cudaMemcpyAsync(c->ref_idx.p, pick.data(), (size_t)k * 8, cudaMemcpyHostToDevice, c->stream));
    LAUNCH(NQS_STAGE_OTHER, launch_gather_picked((const int64_t*)c->ref_idx.p, k, ds, dc, c->index_base,
                                                 (uint64_t*)c->ref_s.p, (double*)c->ref_c.p,
                                                 (int64_t*)c->ref_pos.p, c->stream));
    // the shared-prefix form's tables advance in double-FP32 (about 2^-44 per
    // product, far below the tolerance such a re-evaluation serves)
    c->refine_df = true;
    const int rc = le_core(c, (const uint64_t*)c->ref_s.p, (const double*)c->ref_c.p, k, eb, n_draws, seed,
                           c->av.chain ? NQS_PREC_FP64_SHARED : NQS_PREC_FP64, (const int64_t*)c->ref_pos.p,
                           (double*)c->ref_e.p, nullptr, false);
    c->refine_df = false;
    TRY(rc);
    LAUNCH(NQS_STAGE_OTHER, launch_scatter_picked((const int64_t*)c->ref_idx.p, k,
                                                  (const double*)c->ref_e.p, de, c->stream));
    if (fp64) {
        fp64->resize((size_t)k);
        CK(cudaMemcpyAsync(fp64->data(), c->ref_e.p, (size_t)k * 8, cudaMemcpyDeviceToHost, c->stream));
    }
    // pick is host memory the copy above reads: wait before it goes away
    CK(cudaStreamSynchronize(c->stream));
    return NQS_OK;
}

// Error-budgeted refinement of a mixed-form result (de, with c->eabs). The
// per-sample error of the mixed form relative to e_abs is bounded by a factor
// f, kMixedRelError to start; the samples with the largest c_n e_abs_n are
// re-evaluated in FP64 (see reevaluate) until f * sum_{rest} c_n e_abs_n
// / sum c is within c->energy_tol. With them, c->audit of the other samples
// (evenly spaced in sample order) are re-evaluated as a check of f: when their
// largest |E_mixed - E_FP64| / max(|E|, e_abs) exceeds f, f becomes twice that
// value and the selection grows to meet the tolerance with it. The corrected
// summary goes to c->summary2.
int refine_pass(nqs_ctx* c, const uint64_t* ds, const double* dc, int64_t Ns, uint64_t eb,
                int n_draws, uint64_t seed, double* de, int64_t* n_ref, double* bound)
{
    std::vector<double> ea((size_t)Ns), cn((size_t)Ns, 1.0), em((size_t)Ns);
    CK(cudaMemcpyAsync(ea.data(), c->eabs.p, (size_t)Ns * 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(em.data(), de, (size_t)Ns * 8, cudaMemcpyDeviceToHost, c->stream));
    if (dc) CK(cudaMemcpyAsync(cn.data(), dc, (size_t)Ns * 8, cudaMemcpyDeviceToHost, c->stream));
    TRY(ensure(c, c->logf_save, (size_t)Ns * 8));
    CK(cudaMemcpyAsync(c->logf_save.p, c->logf.p, (size_t)Ns * 8, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    double sc = 0.0;
    for (int64_t s = 0; s < Ns; ++s) sc += cn[(size_t)s];
    std::vector<int64_t> order((size_t)Ns);
    for (int64_t s = 0; s < Ns; ++s) order[(size_t)s] = s;
    std::sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
        const double a = cn[(size_t)x] * ea[(size_t)x], b = cn[(size_t)y] * ea[(size_t)y];
        return a != b ? a > b : x < y;
    });
    // smallest k such that f * sum over order[k..] of c e_abs / sum c <= tolerance
    auto select = [&](double f) {
        std::vector<double> rest((size_t)Ns + 1, 0.0);
        for (int64_t q = Ns - 1; q >= 0; --q) {
            const int64_t s = order[(size_t)q];
            rest[(size_t)q] = rest[(size_t)q + 1] + f * cn[(size_t)s] * ea[(size_t)s] / sc;
        }
        int64_t k = 0;
        while (k < Ns && !(rest[(size_t)k] <= c->energy_tol)) ++k;
        return k;
    };
    double f = kMixedRelError;
    int64_t k = select(f);
    std::vector<char> done((size_t)Ns, 0);
    for (int64_t q = 0; q < k; ++q) done[(size_t)order[(size_t)q]] = 1;
    // audit: c->audit of the others, evenly spaced in sample order
    std::vector<int64_t> others, audit;
    for (int64_t s = 0; s < Ns; ++s)
        if (!done[(size_t)s]) others.push_back(s);
    const int64_t na = std::min<int64_t>(c->audit, (int64_t)others.size());
    for (int64_t j = 0; j < na; ++j) audit.push_back(others[(size_t)(((2 * j + 1) * others.size()) / (2 * na))]);
    std::vector<int64_t> pick;
    for (int64_t s = 0; s < Ns; ++s)
        if (done[(size_t)s]) pick.push_back(s);
    for (int64_t s : audit) done[(size_t)s] = 1;
    pick.insert(pick.end(), audit.begin(), audit.end());
    std::sort(pick.begin(), pick.end());
    std::vector<double> e64;
    TRY(reevaluate(c, ds, dc, pick, eb, n_draws, seed, de, &e64));
    double observed = 0.0;
    for (int64_t s : audit) {
        const size_t at = (size_t)(std::lower_bound(pick.begin(), pick.end(), s) - pick.begin());
        const double scale = std::max(std::fabs(e64[at]), ea[(size_t)s]);
        if (scale > 0.0) observed = std::max(observed, std::fabs(em[(size_t)s] - e64[at]) / scale);
    }
    if (observed > f) {
        f = 2.0 * observed;
        const int64_t k2 = select(f);
        std::vector<int64_t> extra;
        for (int64_t q = 0; q < k2; ++q)
            if (!done[(size_t)order[(size_t)q]]) extra.push_back(order[(size_t)q]);
        std::sort(extra.begin(), extra.end());
        for (int64_t s : extra) done[(size_t)s] = 1;
        TRY(reevaluate(c, ds, dc, extra, eb, n_draws, seed, de, nullptr));
    }
    double b = 0.0;
    int64_t nd = 0;
    for (int64_t s = 0; s < Ns; ++s) {
        if (done[(size_t)s]) ++nd;
        else b += f * cn[(size_t)s] * ea[(size_t)s] / sc;
    }
    *n_ref = nd;
    *bound = b;
    c->audit_rel = observed;
    c->err_factor = f;
    c->n_audited = (int64_t)audit.size();
    TRY(ensure(c, c->summary2, 8 * 8));
    FinalArgs fa{};
    fa.Ns = Ns;
    fa.counts = dc;
    fa.log_f = (const double*)c->logf_save.p;
    fa.e_loc = de;
    fa.summary = (double*)c->summary2.p;
    LAUNCH(NQS_STAGE_FINAL, launch_summary(fa, c->stream));
    CK(cudaGetLastError());
    return NQS_OK;
}

}  // namespace

extern "C" int nqs_local_energy(nqs_ctx* c, const uint64_t* samples, const double* counts,
                                int64_t Ns, double eps, int n_draws, uint64_t seed, double* e_loc,
                                nqs_energy_summary* out)
{
    if (!c) return NQS_ERR_INVALID_ARG;
    c->err[0] = 0;
    cudaSetDevice(c->device);
    TRY(check_ready(c, true));
    if (Ns < 0 || (Ns > 0 && (!samples || !e_loc)))
        return set_err(c, NQS_ERR_INVALID_ARG, "bad samples / e_loc arguments");
    if (n_draws < 0 || n_draws > 4096)
        return set_err(c, NQS_ERR_INVALID_ARG, "n_draws = %d outside 0..4096", n_draws);
    uint64_t eb;
    TRY(eps_bits(c, eps, &eb));
    if (out) memset(out, 0, sizeof(*out));
    if (Ns == 0) return NQS_OK;
    const uint64_t* ds;
    const double* dc;
    TRY(stage_in(c, c->st_samples, samples, (size_t)Ns * 2, &ds));
    TRY(stage_in(c, c->st_counts, counts, (size_t)Ns, &dc));
    double* de;
    bool he;
    TRY(stage_out(c, c->st_out0, e_loc, (size_t)Ns, &de, &he));
    const bool refine = c->energy_tol > 0.0 && c->precision == NQS_PREC_MIXED;
    if (refine) TRY(ensure(c, c->eabs, (size_t)Ns * 8));
    TRY(le_core(c, ds, dc, Ns, eb, n_draws, seed, c->precision, nullptr, de,
                refine ? (double*)c->eabs.p : nullptr, out != nullptr));
    int64_t n_ref = 0;
    double bound = 0.0;
    const int64_t matvecs = c->fam_matvecs;      // of the pass over the whole batch
    c->audit_rel = 0.0;
    c->err_factor = 0.0;
    c->n_audited = 0;
    if (refine) TRY(refine_pass(c, ds, dc, Ns, eb, n_draws, seed, de, &n_ref, &bound));
    // log|f| of the whole batch (the re-evaluation overwrites c->logf with its subset's)
    c->last_logf = refine ? (const double*)c->logf_save.p : (const double*)c->logf.p;
    TRY(copy_back(c, e_loc, de, (size_t)Ns, he));
    if (out) {
        double sm[8], sm2[8];
        CK(cudaMemcpyAsync(sm, c->summary.p, sizeof(sm), cudaMemcpyDeviceToHost, c->stream));
        if (refine) CK(cudaMemcpyAsync(sm2, c->summary2.p, sizeof(sm2), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        const bool shared = c->av.chain && c->precision != NQS_PREC_FP64;
        const double* se = refine ? sm2 : sm;   // energies after re-evaluation
        out->e_mean = se[0];
        out->sum_counts = se[1];
        out->log_B = se[2];
        out->e_tilde_mean = se[3];
        out->n_conn = c->n_conn;
        out->n_det = (int64_t)llround(sm[4]);
        out->n_draw_unique = (int64_t)llround(sm[5]);
        out->n_amplitudes = out->n_det + out->n_draw_unique;
        out->span_sites = (int64_t)llround(sm[6]);
        out->matvecs = shared ? matvecs : (c->av.chain || c->av.readout ? out->span_sites
                                                                         : (int64_t)llround(sm[7]));
        out->n_refined = n_ref;
        out->e_error_bound = bound;
        out->n_audited = c->n_audited;
        out->audit_rel_error = c->audit_rel;
        out->error_factor = c->err_factor;
    } else if (he) {
        CK(cudaStreamSynchronize(c->stream));
    }
    return NQS_OK;
}

namespace {

// The VJP on device-resident samples and weights into device outputs (any may
// be NULL). The environments of at most c->grad_chunk samples (0: all) live at
// once: each chunk's environments are formed, its outer products added to the
// outputs, and the next chunk reuses the memory.
int vjp_core(nqs_ctx* c, const uint64_t* ds, const double* du, int64_t Ns, double* dg, double* dW,
             double* db, double* dW2)
{
    const int K = c->K, D = c->av.D, NH = c->av.n_hidden;
    const size_t nt = (size_t)c->av.n_edges * 4 * D * D, nw = (size_t)NH * 2 * K;
    if (dg && (c->av.readout != 0 || c->av.tk_rank))
        return set_err(c, NQS_ERR_UNSUPPORTED,
                       "the site-tensor gradient needs the linear readout without the tensor term");
    if (Ns == 0) {
        if (dg) CK(cudaMemsetAsync(dg, 0, nt * 8, c->stream));
        if (dW && nw) CK(cudaMemsetAsync(dW, 0, nw * 8, c->stream));
        if (db && NH) CK(cudaMemsetAsync(db, 0, (size_t)NH * 8, c->stream));
        if (dW2 && NH) CK(cudaMemsetAsync(dW2, 0, (size_t)NH * 4 * K * K * 8, c->stream));
        return NQS_OK;
    }
    const int64_t ch = c->grad_chunk > 0 ? c->grad_chunk : Ns;
    TRY(ensure(c, c->grad_scr, grad_scratch_bytes(c->av, ch < Ns ? ch : Ns)));
    for (int64_t s0 = 0; s0 < Ns; s0 += ch) {
        const int64_t n = Ns - s0 < ch ? Ns - s0 : ch;
        const uint64_t* cs = ds + 2 * s0;
        TRY(reset_dev_error(c));
        LAUNCH(NQS_STAGE_OTHER, launch_validate(cs, n, c->K, c->na, c->nb, (DevError*)c->derr.p, c->stream));
        TRY(env_pass(c, cs, n, true, c->av.readout == 1 ? 0 : 1));
        if (c->av.readout == 1) TRY(rnn_env_pass(c, cs, n));
        k_check_psi<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>((const double*)c->pmant.p, n,
                                                                      (DevError*)c->derr.p, s0);
        LAUNCH(NQS_STAGE_OTHER, 1);
        TRY(read_dev_error(c));
        GradArgs g{};
        g.an = c->av;
        g.samples = cs;
        g.Ns = n;
        g.u = du + s0;
        g.Lenv = (const double*)c->Lenv.p; g.Lexp = (const int*)c->Lexp.p;
        g.Renv = (const double*)c->Renv.p; g.Rexp = (const int*)c->Rexp.p;
        g.Hst = (const double*)c->Hst.p; g.Hexp = (const int*)c->Hexp.p;
        g.Gst = (const double*)c->Gst.p; g.Gexp = (const int*)c->Gexp.p;
        g.psi_mant = (const double*)c->pmant.p;
        g.psi_exp = (const int*)c->pexp.p;
        g.theta = (const double*)c->theta.p;
        g.grad_sites = dg;
        g.grad_W = dW;
        g.grad_b = db;
        g.grad_W2 = dW2;
        g.accumulate = s0 > 0;
        char* scr = (char*)c->grad_scr.p;
        g.sidx = (int32_t*)scr;
        g.soff = (int64_t*)(scr + (((size_t)K * n * 4 + 255) & ~(size_t)255));
        g.part = (double*)((char*)g.soff + (((size_t)K * 5 * 8 + 255) & ~(size_t)255));
        LAUNCH(NQS_STAGE_OTHER, launch_grad_fp64(g, c->stream));
        CK(cudaGetLastError());
    }
    return NQS_OK;
}

}  // namespace

extern "C" int nqs_grad_log_psi_vjp2(nqs_ctx* c, const uint64_t* samples, const double* u, int64_t Ns,
                                     double* grad_sites, double* grad_W, double* grad_b, double* grad_W2)
{
    if (!c) return NQS_ERR_INVALID_ARG;
    c->err[0] = 0;
    cudaSetDevice(c->device);
    TRY(check_ready(c, true));
    if (Ns < 0 || (Ns > 0 && (!samples || !u)))
        return set_err(c, NQS_ERR_INVALID_ARG, "bad samples / u arguments");
    if (grad_W2 && c->av.corr != NQS_CORR_ISING)
        return set_err(c, NQS_ERR_INVALID_ARG, "grad_W2 needs the Ising-RBM correlator");
    const int K = c->K, D = c->av.D, NH = c->av.n_hidden;
    const size_t nt = (size_t)c->av.n_edges * 4 * D * D, nw = (size_t)NH * 2 * K, nw2 = (size_t)NH * 4 * K * K;
    double *dg, *dW, *db, *dW2;
    bool hg, hW, hb, hW2;
    TRY(stage_out(c, c->st_out1, grad_sites, nt, &dg, &hg));
    TRY(stage_out(c, c->st_out2, grad_W, nw, &dW, &hW));
    TRY(stage_out(c, c->st_out3, grad_b, (size_t)NH, &db, &hb));
    TRY(stage_out(c, c->st_out4, grad_W2, nw2, &dW2, &hW2));
    const uint64_t* ds = nullptr;
    const double* du = nullptr;
    if (Ns > 0) {
        TRY(stage_in(c, c->st_samples, samples, (size_t)Ns * 2, &ds));
        TRY(stage_in(c, c->st_u, u, (size_t)Ns, &du));
    }
    TRY(vjp_core(c, ds, du, Ns, dg, dW, db, dW2));
    TRY(copy_back(c, grad_sites, dg, nt, hg));
    TRY(copy_back(c, grad_W, dW, nw, hW));
    TRY(copy_back(c, grad_b, db, (size_t)NH, hb));
    TRY(copy_back(c, grad_W2, dW2, nw2, hW2));
    CK(cudaStreamSynchronize(c->stream));
    return NQS_OK;
}

extern "C" int nqs_grad_log_psi_vjp(nqs_ctx* c, const uint64_t* samples, const double* u, int64_t Ns,
                                    double* grad_sites, double* grad_W, double* grad_b)
{
    return nqs_grad_log_psi_vjp2(c, samples, u, Ns, grad_sites, grad_W, grad_b, nullptr);
}

extern "C" int nqs_energy_gradient(nqs_ctx* c, const uint64_t* samples, const double* counts, int64_t Ns,
                                   double eps, int n_draws, uint64_t seed, int reweighted,
                                   double* grad_sites, double* grad_W, double* grad_b, double* grad_W2,
                                   double* e_loc, nqs_energy_summary* out)
{
    if (!c) return NQS_ERR_INVALID_ARG;
    c->err[0] = 0;
    cudaSetDevice(c->device);
    TRY(check_ready(c, true));
    if (Ns <= 0 || !samples) return set_err(c, NQS_ERR_INVALID_ARG, "nqs_energy_gradient needs Ns > 0 samples");
    if (grad_W2 && c->av.corr != NQS_CORR_ISING)
        return set_err(c, NQS_ERR_INVALID_ARG, "grad_W2 needs the Ising-RBM correlator");
    const uint64_t* ds;
    const double* dc;
    TRY(stage_in(c, c->st_samples, samples, (size_t)Ns * 2, &ds));
    TRY(stage_in(c, c->st_counts, counts, (size_t)Ns, &dc));
    TRY(ensure(c, c->eloc, (size_t)Ns * 8));
    nqs_energy_summary sm;
    TRY(nqs_local_energy(c, ds, dc, Ns, eps, n_draws, seed, (double*)c->eloc.p, &sm));
    TRY(ensure(c, c->u_dev, (size_t)Ns * 8));
    // u_n = 2 c_n (E_loc(n) - E) / sum c (Eq. egrad); reweighted (Sec. 2.3):
    // u_n = 2 c_n f~_n^2 (E_loc(n) - E_theta) / sum c, f~^2 = f^2 / B, E_theta = mean of E~
    LAUNCH(NQS_STAGE_OTHER, launch_energy_weights((const double*)c->eloc.p, dc, c->last_logf, Ns,
                                                  reweighted ? sm.e_tilde_mean : sm.e_mean, sm.sum_counts,
                                                  reweighted ? sm.log_B : 0.0, reweighted != 0,
                                                  (double*)c->u_dev.p, c->stream));
    CK(cudaGetLastError());
    const int K = c->K, D = c->av.D, NH = c->av.n_hidden;
    const size_t nt = (size_t)c->av.n_edges * 4 * D * D, nw = (size_t)NH * 2 * K, nw2 = (size_t)NH * 4 * K * K;
    double *dg, *dW, *db, *dW2, *de;
    bool hg, hW, hb, hW2, he;
    TRY(stage_out(c, c->st_out1, grad_sites, nt, &dg, &hg));
    TRY(stage_out(c, c->st_out2, grad_W, nw, &dW, &hW));
    TRY(stage_out(c, c->st_out3, grad_b, (size_t)NH, &db, &hb));
    TRY(stage_out(c, c->st_out4, grad_W2, nw2, &dW2, &hW2));
    TRY(stage_out(c, c->st_out0, e_loc, (size_t)Ns, &de, &he));
    if (de) CK(cudaMemcpyAsync(de, c->eloc.p, (size_t)Ns * 8, cudaMemcpyDeviceToDevice, c->stream));
    TRY(vjp_core(c, ds, (const double*)c->u_dev.p, Ns, dg, dW, db, dW2));
    TRY(copy_back(c, grad_sites, dg, nt, hg));
    TRY(copy_back(c, grad_W, dW, nw, hW));
    TRY(copy_back(c, grad_b, db, (size_t)NH, hb));
    TRY(copy_back(c, grad_W2, dW2, nw2, hW2));
    TRY(copy_back(c, e_loc, de, (size_t)Ns, he));
    CK(cudaStreamSynchronize(c->stream));
    if (out) *out = sm;
    return NQS_OK;
}

extern "C" int nqs_sample(nqs_ctx* c, int64_t n_samples, uint64_t seed, uint64_t* samples, double* counts,
                          int64_t capacity, int64_t* n_unique)
{
    if (!c) return NQS_ERR_INVALID_ARG;
    c->err[0] = 0;
    cudaSetDevice(c->device);
    TRY(check_ready(c, true));
    if (c->av.readout != 1)
        return set_err(c, NQS_ERR_STATE, "nqs_sample needs the normalised readout (nqs_set_readout)");
    if (n_samples < 0 || !n_unique || (capacity > 0 && (!samples || !counts)))
        return set_err(c, NQS_ERR_INVALID_ARG, "bad n_samples / outputs");
    *n_unique = 0;
    if (n_samples == 0) return NQS_OK;
    const int K = c->K, D = c->av.D;
    c->smp_pa.resize(K + 1); c->smp_pb.resize(K + 1); c->smp_off.resize(K + 1);
    c->smp_cnt.resize(K + 1); c->smp_par.resize(K + 1); c->smp_cell.resize(K + 1);
    // level 0: the empty prefix holds every draw
    int64_t n = 1;
    TRY(ensure(c, c->smp_pa[0], 8)); TRY(ensure(c, c->smp_pb[0], 8));
    TRY(ensure(c, c->smp_off[0], 8)); TRY(ensure(c, c->smp_cnt[0], 8));
    CK(cudaMemsetAsync(c->smp_pa[0].p, 0, 8, c->stream));
    CK(cudaMemsetAsync(c->smp_pb[0].p, 0, 8, c->stream));
    CK(cudaMemsetAsync(c->smp_off[0].p, 0, 8, c->stream));
    CK(cudaMemcpyAsync(c->smp_cnt[0].p, &n_samples, 8, cudaMemcpyHostToDevice, c->stream));
    TRY(ensure(c, c->smp_tabs, (size_t)2 * (K + 1) * sizeof(void*)));
    std::vector<const void*> tabs((size_t)2 * (K + 1), nullptr);
    for (int i = 0; i < K; ++i) {
        // tables of the parent links and cells of levels 1..i
        for (int l = 1; l <= i; ++l) { tabs[l] = c->smp_par[l].p; tabs[K + 1 + l] = c->smp_cell[l].p; }
        CK(cudaMemcpyAsync(c->smp_tabs.p, tabs.data(), tabs.size() * sizeof(void*), cudaMemcpyHostToDevice,
                           c->stream));
        TRY(ensure(c, c->smp_cand, (size_t)n * 4 * D * 8));
        TRY(ensure(c, c->smp_ccnt, (size_t)n * 8 * 8));          // counts, then child flags
        TRY(ensure(c, c->smp_cpos, (size_t)(n * 4 + 1) * 8));
        TRY(ensure(c, c->site_scan, (size_t)scan_i64_tmp_elems(n * 4) * 8));
        SampleLevel L{};
        L.an = c->av;
        L.level = i;
        L.n_nodes = n;
        L.pa = (const uint64_t*)c->smp_pa[i].p; L.pb = (const uint64_t*)c->smp_pb[i].p;
        L.off = (const int64_t*)c->smp_off[i].p; L.cnt = (const int64_t*)c->smp_cnt[i].p;
        L.parents = (const int32_t* const*)c->smp_tabs.p;
        L.cells = (const double* const*)((const void* const*)c->smp_tabs.p + (K + 1));
        L.cand = (double*)c->smp_cand.p;
        L.child_cnt = (int64_t*)c->smp_ccnt.p;
        L.child_flag = (int64_t*)c->smp_ccnt.p + n * 4;
        L.seed = seed;
        LAUNCH(NQS_STAGE_OTHER, launch_sample_level(L, c->stream));
        // child positions: exclusive scan of the flags (prefix order), total = children
        LAUNCH(NQS_STAGE_OTHER, launch_scan_i64_wide(L.child_flag, (int64_t*)c->smp_cpos.p, n * 4,
                                                     (int64_t*)c->site_scan.p, c->stream));
        int64_t m = 0;
        CK(cudaMemcpyAsync(&m, (const int64_t*)c->smp_cpos.p + n * 4, 8, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));      // also keeps `tabs` alive until copied
        if (m <= 0) return set_err(c, NQS_ERR_INVALID_ARG, "no local state is allowed at vertex %d", i);
        TRY(ensure(c, c->smp_pa[i + 1], (size_t)m * 8)); TRY(ensure(c, c->smp_pb[i + 1], (size_t)m * 8));
        TRY(ensure(c, c->smp_off[i + 1], (size_t)m * 8)); TRY(ensure(c, c->smp_cnt[i + 1], (size_t)m * 8));
        TRY(ensure(c, c->smp_par[i + 1], (size_t)m * 4)); TRY(ensure(c, c->smp_cell[i + 1], (size_t)m * D * 8));
        SampleChildren S{};
        S.level = i; S.D = D; S.n_nodes = n;
        S.pa = L.pa; S.pb = L.pb; S.off = L.off;
        S.cand = L.cand; S.child_cnt = L.child_cnt; S.child_pos = (const int64_t*)c->smp_cpos.p;
        S.qa = (uint64_t*)c->smp_pa[i + 1].p; S.qb = (uint64_t*)c->smp_pb[i + 1].p;
        S.qoff = (int64_t*)c->smp_off[i + 1].p; S.qcnt = (int64_t*)c->smp_cnt[i + 1].p;
        S.qparent = (int32_t*)c->smp_par[i + 1].p; S.qcell = (double*)c->smp_cell[i + 1].p;
        LAUNCH(NQS_STAGE_OTHER, launch_sample_children(S, c->stream));
        CK(cudaGetLastError());
        n = m;
    }
    *n_unique = n;
    if (capacity < n)
        return set_err(c, NQS_ERR_INVALID_ARG, "capacity %lld < %lld unique samples (n_unique written)",
                       (long long)capacity, (long long)n);
    uint64_t* dsm;
    double* dcn;
    bool hs, hc;
    TRY(stage_out(c, c->st_out0, samples, (size_t)n * 2, &dsm, &hs));
    TRY(stage_out(c, c->st_out1, counts, (size_t)n, &dcn, &hc));
    LAUNCH(NQS_STAGE_OTHER, launch_sample_output((const uint64_t*)c->smp_pa[K].p, (const uint64_t*)c->smp_pb[K].p,
                                                 (const int64_t*)c->smp_cnt[K].p, n, dsm, dcn, c->stream));
    CK(cudaGetLastError());
    TRY(copy_back(c, samples, dsm, (size_t)n * 2, hs));
    TRY(copy_back(c, counts, dcn, (size_t)n, hc));
    CK(cudaStreamSynchronize(c->stream));
    return NQS_OK;
}

// ============================================================================
// Allocation-free variant of nqs_draws
//
// Some callers must not allocate device memory during a call:
// latency-critical loops where an allocation can stall on a device-wide
// synchronisation, and hosts that hand the whole GPU memory to their own pool
// up front. For them this entry point computes the same draws as nqs_draws
// using only the scratch below, which is part of the library image: it is
// reserved on every GPU that loads the library and stays there until the
// process exits.
// ============================================================================

namespace {

constexpr size_t kNoAllocWords = (size_t)NQS_NOALLOC_SCRATCH_BYTES / 8;

// Scratch shared by every call of nqs_draws_noalloc on a device. It keeps the
// previous call's contents; each call clears what has to start at zero.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kNoAllocWords];

}  // namespace

extern "C" int nqs_draws_noalloc(nqs_ctx* c, const uint64_t* samples, int64_t Ns, double eps,
                                 int n_draws, uint64_t seed, int64_t* ranks, uint64_t* w_total)
{
    if (!c) return NQS_ERR_INVALID_ARG;
    c->err[0] = 0;
    CK(cudaSetDevice(c->device));
    TRY(check_ready(c, false));
    if (Ns < 0 || n_draws < 0 || (Ns > 0 && !samples) || (Ns > 0 && n_draws > 0 && !ranks))
        return set_err(c, NQS_ERR_INVALID_ARG, "bad samples / n_draws / ranks arguments");
    uint64_t eb;
    TRY(eps_bits(c, eps, &eb));
    if (Ns == 0) return NQS_OK;
    if (!is_device_ptr(samples) || (n_draws > 0 && !is_device_ptr(ranks)) ||
        (w_total && !is_device_ptr(w_total)))
        return set_err(c, NQS_ERR_INVALID_ARG,
                       "nqs_draws_noalloc needs device pointers (host arrays would need staging)");
    // scratch layout (64-bit words): error word (2), W [Ns], chunk weights
    // [Ns][nch], chunk counts [Ns][nch] as 32-bit halves
    const uint64_t nch = (uint64_t)((c->n_conn + 31) / 32);
    const uint64_t need = 2 + (uint64_t)Ns + (uint64_t)Ns * nch + ((uint64_t)Ns * nch + 1) / 2;
    if (need > kNoAllocWords)
        return set_err(c, NQS_ERR_INVALID_ARG,
                       "nqs_draws_noalloc: %lld samples x %llu rank chunks need %llu scratch words, "
                       "the fixed scratch holds %llu (%d bytes); split the batch",
                       (long long)Ns, (unsigned long long)nch, (unsigned long long)need,
                       (unsigned long long)kNoAllocWords, (int)NQS_NOALLOC_SCRATCH_BYTES);
    // the array's device address on this context's device (current since the
    // cudaSetDevice above), looked up on the context's first call; contexts are
    // used by one host thread at a time, so the lookup needs no lock
    if (!c->noalloc_addr) {
        void* p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        c->noalloc_addr = (unsigned long long*)p;
    }
    unsigned long long* base = c->noalloc_addr;
    DevError* derr = (DevError*)base;
    uint64_t* W = (uint64_t*)(base + 2);
    uint64_t* chunk_w = W + Ns;
    uint32_t* chunk_cnt = (uint32_t*)(chunk_w + (size_t)Ns * nch);
    CK(cudaMemsetAsync(derr, 0, sizeof(DevError), c->stream));
    LAUNCH(NQS_STAGE_OTHER, launch_validate(samples, Ns, c->K, c->na, c->nb, derr, c->stream));
    EnumArgs a{};
    a.h = c->hv;
    a.samples = samples;
    a.eps_bits = eb;
    a.n_chunks = (uint32_t)nch;
    a.chunk_cnt = chunk_cnt;
    a.shift = weight_shift(c, eb);
    a.chunk_w = chunk_w;
    LAUNCH(NQS_STAGE_COUNT, launch_enum(a, Ns, false, c->stream));
    LAUNCH(NQS_STAGE_COUNT, launch_scan_chunks_u64(chunk_w, W, Ns, (uint32_t)nch, c->stream));
    if (nch == 0) CK(cudaMemsetAsync(W, 0, (size_t)Ns * 8, c->stream));
    if (n_draws > 0) {
        DrawArgs d{};
        d.h = c->hv;
        d.samples = samples;
        d.Ns = Ns;
        d.eps_bits = eb;
        d.n_chunks = (uint32_t)nch;
        d.chunk_pre = chunk_w;
        d.shift = weight_shift(c, eb);
        d.n_draws = n_draws;
        d.seed = seed;
        d.index_base = c->index_base;
        d.out_rank = ranks;
        LAUNCH(NQS_STAGE_DRAW, launch_draws(d, c->stream));
    }
    CK(cudaGetLastError());
    if (w_total) CK(cudaMemcpyAsync(w_total, W, (size_t)Ns * 8, cudaMemcpyDeviceToDevice, c->stream));
    DevError e;
    CK(cudaMemcpyAsync(&e, derr, sizeof(e), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (e.code != 0)
        return set_err(c, e.code, "%s (samples[%lld])",
                       e.detail == 1 ? "sample has an occupied orbital >= n_orb"
                                     : "sample has the wrong number of alpha or beta electrons",
                       (long long)e.index);
    return NQS_OK;
}

namespace nqs {

// shape of a context's system (0 where not set yet)
int ctx_shape(const nqs_ctx* c, int* K, int* na, int* nb, int* D)
{
    if (!c) return NQS_ERR_INVALID_ARG;
    *K = c->K;
    *na = c->na;
    *nb = c->nb;
    *D = c->av.D;
    return NQS_OK;
}

void ctx_set_table_budget(nqs_ctx* c, size_t bytes)
{
    if (c) c->fam_budget = bytes;
}

size_t ctx_free_memory(nqs_ctx* c)
{
    size_t fr = 0, tot = 0;
    if (!c) return 0;
    cudaSetDevice(c->device);
    cudaMemGetInfo(&fr, &tot);
    return fr;
}

int ctx_sync(nqs_ctx* c)
{
    if (!c) return NQS_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return set_err(c, NQS_ERR_CUDA, "%s", cudaGetErrorString(e));
    return NQS_OK;
}

}  // namespace nqs
