/*
 * nqs.h -- C ABI of the GB300 semistochastic local-energy library.
 *
 * Computes, for sampled occupation-number vectors n, the local energy of
 * Sec. 2.1, Eq. (exactElocal):  E_loc(n) = sum_m H_nm psi(m) / psi(n),
 * with H from Eq. (Ham) evaluated by the Slater-Condon rules (Sec. 3) and the
 * semistochastic split of Sec. 2.4: E_loc = E^d(n, eps) + E^s(n, eps, N_eps),
 * E^d summing every off-diagonal m with |H_nm| >= eps (the diagonal is always
 * exact) and E^s averaging N_eps draws m' ~ P_n(m') proportional to |H_nm'|
 * over the remainder |H_nm'| < eps. psi = psi_TN * f is a tensor network
 * (Eq. MPS-RNN-1D with v = 0 for a chain; Eq. bdg-rnn-update without the
 * tensor term for a graph) times an RBM correlator (Eq. RBM, 2cosh form).
 *
 * Conventions
 *  - K <= 64 spatial orbitals; spin orbital s = 2p + spin (alpha 0, beta 1),
 *    the interleaved order of Sec. 3, which fixes the fermionic phases:
 *    |n> = a+_{s1} a+_{s2} ... |0> with s1 < s2 < ...
 *  - A determinant is two uint64 words [alpha bits, beta bits]; bit p of a
 *    word is the occupation of spatial orbital p with that spin.
 *  - Local state sigma_p = n_{p,alpha} + 2 n_{p,beta}.
 *  - Connected determinants m of n are ranked 0..n_conn-1 in a canonical
 *    order: blocks [singles alpha, singles beta, doubles alpha-alpha,
 *    doubles beta-beta, doubles alpha-beta]; inside a block by the positions
 *    of the orbitals among the occupied / empty orbitals of that spin
 *    (ascending, pairs lexicographic; alpha-beta doubles ordered as
 *    ((i_a * nv_a + a_a) * no_b + j_b) * nv_b + b_b).
 *
 * Memory and ownership
 *  - The caller owns every buffer it passes. Array arguments may point to
 *    host or device memory; the library tells them apart with
 *    cudaPointerGetAttributes. Device arrays must be on the context's device.
 *    Host inputs are staged to the device on the context's stream; host
 *    outputs are copied back and the stream is synchronised before return.
 *  - nqs_set_* copy their arguments; the caller may free them afterwards.
 *  - Outputs are valid only when a call returns NQS_OK (their contents are
 *    unspecified otherwise).
 *  - A context is not thread safe; use one context per host thread.
 *
 * Errors: every call returns an nqs_status. NQS_ERR_INVALID_ARG names the
 * offending argument (and sample index) in nqs_last_error(). Nothing aborts;
 * device-side checks report through an error word that the host reads.
 */
#ifndef NQS_H
#define NQS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NQS_OK = 0,
    NQS_ERR_INVALID_ARG = 1,   /* bad size, pointer or determinant */
    NQS_ERR_STATE = 2,         /* call order violated (e.g. no Hamiltonian yet) */
    NQS_ERR_OOM = 3,           /* device allocation failed */
    NQS_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    NQS_ERR_TIMEOUT = 5,       /* a bounded device wait gave up */
    NQS_ERR_UNSUPPORTED = 6    /* valid request this build does not handle */
} nqs_status;

typedef enum {
    NQS_PREC_FP64 = 0,        /* the plain form: every amplitude psi(m) is its own
                                 FP64 product over the sites where m differs from n
                                 (cached left/right environments outside that span) */
    NQS_PREC_MIXED = 1,       /* contractions on the tensor cores (split FP16
                                 operands, FP32 accumulation, per-site power-of-two
                                 rescaling); H_nm, psi(n), the ratios and the E_loc
                                 sums in FP64. Chain ansatz: shared-prefix
                                 evaluation (partial products common to many m of
                                 one n are formed once and each psi(m) is one dot
                                 product). Graph ansatz: the vertices from each
                                 row's first changed site on are re-run for 128 rows
                                 of one sample at a time; needs D in {16, 32, 64},
                                 in-degree x 4 x D <= 512, at most 16 vertex states
                                 live at once, the linear readout, no tensor term
                                 and the 2cosh or cos correlator (otherwise
                                 NQS_ERR_UNSUPPORTED with the reason) */
    NQS_PREC_FP64_SHARED = 2  /* the shared-prefix evaluation with FP64
                                 contractions (chain ansatz only) */
} nqs_precision;

typedef struct nqs_ctx nqs_ctx;

typedef struct {
    int precision;        /* nqs_precision */
    int timing;           /* nonzero: time every stage with CUDA events on the
                             context's stream (see nqs_stage_times) */
    int64_t sample_index_base;  /* global position of samples[0] when one batch
                             is split across calls or devices: sample s of a
                             call draws with Philox counter (d, base + s), so
                             the draws do not depend on the split (default 0;
                             must be >= 0) */
    double energy_tolerance;    /* mixed form: bound (Ha) on the error of the
                             weighted energy sum c E_loc / sum c that
                             nqs_local_energy meets by re-evaluating samples in
                             FP64 (the shared-prefix form for chains, whose
                             tables then advance in double-FP32 arithmetic,
                             about 2^-44 per product; the plain form for
                             graphs). The
                             per-sample error of the mixed form relative to
                             e_abs = |H_nn| + sum |terms| is taken as a factor f
                             (1e-6 to start: what the parity tests hold the mixed
                             form to); samples are taken in decreasing order of
                             c_n e_abs_n until f * sum over the others of
                             c_n e_abs_n / sum c <= energy_tolerance. Each call
                             also re-evaluates audit_samples of the others and,
                             if one of them errs by more than f, raises f to
                             twice the largest observed error and extends the
                             re-evaluation (the summary reports both). The
                             re-evaluated E_loc are replaced by the FP64 values.
                             The factor is measured, not proven: the bound holds
                             for errors no larger than the audit saw.
                             0 (default): no re-evaluation. Ignored by the FP64
                             forms. Must be finite, >= 0 */
    int grad_chunk;       /* gradient calls: samples whose environments live on
                             the device at once (0, default: the whole batch);
                             bounds the gradient's memory at the cost of forming
                             the environments chunk by chunk. Must be >= 0 */
    int audit_samples;    /* samples of the energy-tolerance audit (0: the
                             default, 4; -1: none). Must be >= -1 */
    int tile_blocks_per_sm;   /* shared-prefix forms: blocks per multiprocessor of
                             each site-step tile launch (0: the default, 4; at most
                             32). A schedule parameter: results do not depend on it */
    int table_mb;         /* shared-prefix forms: cap (MiB) on the tables of one
                             sample batch (0: the default, 32 GiB); never more
                             than a third of the free device memory. Larger
                             batches mean fewer, fuller launches; results do not
                             depend on it */
    int reserved[6];      /* must be zero */
} nqs_options;

/* Correlator kinds of Sec. 2.3 (nqs_set_correlator). */
typedef enum {
    NQS_CORR_COSH = 0,    /* f = prod_k 2 cosh(theta_k) (Eq. RBM, the default) */
    NQS_CORR_COS = 1,     /* cos-RBM: f = prod_k cos(theta_k) */
    NQS_CORR_ISING = 2    /* Ising-RBM: f = prod_k cos(theta_k + 1/2 sum_{s,t} W2[k][s][t] n_s n_t) */
} nqs_correlator;

/* Stages of the local-energy path, as reported by nqs_stage_times. */
enum {
    NQS_STAGE_ENV = 0,        /* input checks, environments, psi(n), f(n), H_nn */
    NQS_STAGE_COUNT = 1,      /* enumeration pass 1: |H| >= eps counts, remainder weight sums */
    NQS_STAGE_WRITE = 2,      /* enumeration pass 2: deterministic lists (chunks holding entries) */
    NQS_STAGE_DRAW = 3,       /* Philox draws, inverse CDF, de-duplication */
    NQS_STAGE_AMP_DET = 4,    /* amplitudes and ratios of the deterministic rows */
    NQS_STAGE_AMP_DRAW = 5,   /* amplitudes and ratios of the drawn rows */
    NQS_STAGE_FINAL = 6,      /* E_loc sums and the weighted summary */
    NQS_STAGE_OTHER = 7,      /* nqs_connected / nqs_amplitude / gradient work */
    NQS_STAGE_TABLES = 8,     /* shared-prefix tables: one-change families, cluster
                                 marks, two-change clusters and their propagation,
                                 correlator factors */
    NQS_N_STAGES = 9
};

typedef struct {
    double e_mean;          /* sum_n c_n E_loc(n) / sum_n c_n */
    double sum_counts;      /* sum_n c_n */
    double log_B;           /* log B, B = sum c f^2 / sum c (Sec. 2.3, real f) */
    double e_tilde_mean;    /* sum_n c_n E~_loc(n) / sum c, E~ = f^2/B E_loc */
    int64_t n_conn;         /* connected determinants per sample */
    int64_t n_det;          /* sum over samples of |{m : |H_nm| >= eps}| */
    int64_t n_draw_unique;  /* sum over samples of distinct drawn m */
    int64_t n_amplitudes;   /* amplitudes evaluated = n_det + n_draw_unique */
    int64_t span_sites;     /* sum over evaluated amplitudes of the number of
                               sites (chain) or vertices (graph) between the first
                               and last changed one: the products a per-amplitude
                               evaluation performs */
    int64_t matvecs;        /* D x D matrix-vector products of the evaluation:
                               chains, plain form: span_sites; graphs (linear
                               readout): the in-edges with a vertex source of
                               every re-run vertex, summed over the amplitudes
                               (the tensor-core tiles also run rows and local
                               states a tile shares, not counted here);
                               shared-prefix form: one-change families plus
                               two-change clusters of the pass over the whole
                               batch */
    int64_t n_refined;      /* samples re-evaluated in FP64 (energy_tolerance),
                               the audited ones included */
    double e_error_bound;   /* with energy_tolerance > 0 in the mixed form: the
                               bound f * sum c_n e_abs_n / sum c over the samples
                               left in the mixed form (<= energy_tolerance); else 0 */
    int64_t n_audited;      /* samples of the audit (see nqs_options.energy_tolerance) */
    double audit_rel_error; /* largest |E_mixed - E_FP64| / max(|E|, e_abs) the audit saw */
    double error_factor;    /* the factor f the bound used (1e-6, or twice the audit's
                               largest error when that was larger) */
} nqs_energy_summary;

/* Create a context on CUDA device `device`; `cuda_stream` is a cudaStream_t
 * (NULL = the legacy default stream) on which all work of the context runs. */
int nqs_create(nqs_ctx** out, int device, void* cuda_stream);

/* Release every device buffer of the context. NULL is accepted. */
int nqs_destroy(nqs_ctx* ctx);

/* Message for the last failing call on this context ("" if none). */
const char* nqs_last_error(const nqs_ctx* ctx);

/* Select the precision of later calls (default NQS_PREC_FP64). */
int nqs_set_options(nqs_ctx* ctx, const nqs_options* opt);

/* Device time (ms) and number of kernel launches per stage, accumulated
 * since the previous call, then reset. `ms` (may be NULL) gets the times of
 * calls made with nqs_options.timing set; `launches` (may be NULL) counts every
 * kernel launch of this context. Both arrays hold n entries (n <=
 * NQS_N_STAGES). Synchronises the context's stream. */
int nqs_stage_times(nqs_ctx* ctx, double* ms, int64_t* launches, int n);

/* Hamiltonian of Eq. (Ham) in spatial orbitals.
 *  h1e [n_orb][n_orb]: one-electron integrals h_pq (symmetric).
 *  cholesky_or_eri: n_chol > 0: vectors L[n_chol][n_orb][n_orb], symmetric in
 *    (p,q), and (pq|rs) = sum_x L^x_pq L^x_rs is built on the device with a
 *    fused multiply-add chain over ascending x; n_chol == 0: the chemists'
 *    integrals (pq|rs) as [n_orb]^4, used as given (must be 8-fold symmetric
 *    for H_nm = H_mn to hold bitwise).
 *  1 <= n_orb <= 64, 0 <= n_alpha, n_beta <= n_orb. e_core adds to H_nn. */
int nqs_set_hamiltonian(nqs_ctx* ctx, const double* h1e, const double* cholesky_or_eri,
                        int n_chol, int n_orb, int n_alpha, int n_beta, double e_core);

/* Ansatz psi = psi_TN * f (Sec. 2.2-2.3).
 *  site_tensors [n_edges][4][D][D]: edge tensors M_e^sigma[a][b] with
 *    h_i = sum_{e=(j->i)} M_e^{sigma_i} h_j (column convention), h_{-1} = e_0,
 *    psi_TN = (h_{K-1})_0.
 *  pred_ptr [n_orb+1], pred_idx [n_edges]: the edges into vertex i are
 *    pred_idx[pred_ptr[i] .. pred_ptr[i+1]) (source vertex, -1 = the boundary
 *    vector; each source < i). Both NULL: a chain, n_edges = n_orb, edge i
 *    joins i-1 -> i.
 *  rbm_W [n_hidden][2*n_orb], rbm_b [n_hidden]: f = prod_k 2cosh(b_k +
 *    sum_s W[k][s] n_s) over the interleaved spin orbitals; n_hidden = 0 and
 *    NULL pointers: f = 1.
 *  1 <= D <= 256; a graph needs in-degree <= 8. Resets the readout to the
 *  linear one and the correlator kind to 2cosh. */
int nqs_set_ansatz(nqs_ctx* ctx, const double* site_tensors, int n_edges, int bond_dim,
                   const int* pred_ptr, const int* pred_idx, const double* rbm_W,
                   const double* rbm_b, int n_hidden);

/* The normalised MPS-RNN / BDG-RNN readout of Sec. 2.2 (Eq. MPS-RNN-1D with
 * the affine term; Eq. bdg-rnn-update without the tensor term) on the site
 * tensors of nqs_set_ansatz. Vertex i (spatial orbital i, the computation
 * order) forms the candidate cells h_i^s = sum_{e=(j->i)} M_e^s h_j + v_i^s
 * from the cells of the local states already chosen (h_{-1} = e_0), and
 *   P_i(s) = sum_a eta_i[a] (h_i^s[a])^2,  P~_i(s) = P_i(s) / sum_{s' allowed} P_i(s'),
 *   Phi(n) = prod_i sqrt(P~_i(s_i)) * prod_i sign(w_i . h_i^{s_i} + c_i)
 * (real parameters: the phase arg(.) of Sec. 2.2 is a sign; a zero argument
 * counts as +). With `constrained`, a local state is allowed at vertex i when,
 * after it, neither spin exceeds N_alpha / N_beta and the later vertices can
 * still hold the electrons left (Sec. 3); otherwise every state is allowed.
 * Phi is normalised over the (constrained) determinants, so psi = f Phi with
 * the correlator f as in Sec. 2.3.
 *  v [n_orb][4][D], eta [n_orb][D] (finite, >= 0), w [n_orb][D], c [n_orb].
 *  All four NULL: back to the linear readout.
 * Only the plain FP64 form evaluates this readout (the shared-prefix forms
 * return NQS_ERR_UNSUPPORTED); nqs_amplitude returns log|Phi f|; the
 * site-tensor gradient needs the linear readout (NQS_ERR_UNSUPPORTED). */
int nqs_set_readout(nqs_ctx* ctx, const double* v, const double* eta, const double* w,
                    const double* c, int constrained);

/* Correlator kind of Sec. 2.3 for the rbm_W, rbm_b of nqs_set_ansatz:
 * NQS_CORR_COSH (Eq. RBM), NQS_CORR_COS (cos-RBM) or NQS_CORR_ISING
 * (Ising-RBM, W2 [n_hidden][2 n_orb][2 n_orb] over the interleaved spin
 * orbitals, copied; NULL otherwise). The cos forms may make f and psi
 * negative; psi(n) = 0 for a sample is NQS_ERR_INVALID_ARG as before. The
 * shared-prefix forms (chains) support NQS_CORR_COSH only, the mixed form of
 * a graph ansatz NQS_CORR_COSH and NQS_CORR_COS (NQS_ERR_UNSUPPORTED). */
int nqs_set_correlator(nqs_ctx* ctx, int kind, const double* W2);

/* The tensor term of Eq. (bdg-rnn-update) with the Tucker factors of Sec. 2.2
 * (the BDG-TensorRNN), on a graph ansatz: a vertex i with d >= 2 in-edges and
 * rank r = ranks[i] > 0 adds to its cell (every readout)
 *   t_i^s[a] = sum_o Kout[a][o] sum_{q_1..q_d} U^s[o][q_1]..[q_d] prod_k z_k[q_k],
 *   z_k[q] = sum_b K_k[b][q] h_{j_k}[b]
 * (j_k the source of the k-th in-edge in pred_idx order, h_{-1} = e_0). The
 * paper sets r = ceil(D^(2/(d+1))). params packs, per such vertex in vertex
 * order, U [4][r^(d+1)] (index order o, q_1, .., q_d), Kout [D][r], then K_k
 * [D][r] for k = 1..d; n_params must equal that total (NQS_ERR_INVALID_ARG
 * otherwise, as for a chain or r outside 0..64). ranks NULL removes the term.
 * FP64 forms only; the site-tensor gradient returns NQS_ERR_UNSUPPORTED. */
int nqs_set_tensor_term(nqs_ctx* ctx, const int* ranks, const double* params, int64_t n_params);

/* Connected determinants with |H_mn| >= det_threshold, canonical order.
 *  samples [Ns][2]; offsets [Ns+1] receives the start of each sample's list.
 *  rank [capacity], dets [capacity][2], H [capacity], sign [capacity]
 *  receive, per entry, the canonical rank, the determinant m, <m|H|n> and the
 *  fermionic phase gamma (+1/-1) of the excitation operator.
 *  Any of rank/dets/H/sign may be NULL. With all four NULL only offsets is
 *  written (the sizes query). capacity < offsets[Ns] -> NQS_ERR_INVALID_ARG
 *  with offsets written. det_threshold 0 lists every connected m. */
int nqs_connected(nqs_ctx* ctx, const uint64_t* samples, int64_t Ns, double det_threshold,
                  int64_t* offsets, uint32_t* rank, uint64_t* dets, double* H, int8_t* sign,
                  int64_t capacity);

/* log|psi| and sign of psi for n determinants (full K-site product, FP64
 * whatever the precision option). sign is 0 where psi = 0. */
int nqs_amplitude(nqs_ctx* ctx, const uint64_t* dets, int64_t n, double* log_abs,
                  int8_t* sign);

/* The stochastic draws of Sec. 2.4 for each sample (exposed for testing).
 *  ranks [Ns][n_draws] (int64, -1 where the remainder has zero weight),
 *  w_total [Ns] (may be NULL). Draw d of sample s (s = index in `samples`)
 *  uses Philox4x64-10 with key (seed, 0) and counter (d, s, 0, 0); its first
 *  output x picks t = floor(x W / 2^64), and m' is the first remainder entry
 *  (canonical order) whose inclusive prefix of integer weights exceeds t.
 *  Weights: w = ceil(|H| 2^shift), shift = 62 - e - bitlen(n_conn), where
 *  det_threshold = f 2^e with f in [0.5, 1): every remainder |H| is below
 *  det_threshold, so every per-sample sum stays below 2^62. */
int nqs_draws(nqs_ctx* ctx, const uint64_t* samples, int64_t Ns, double det_threshold,
              int n_draws, uint64_t philox_seed, int64_t* ranks, uint64_t* w_total);

/* nqs_draws without any device allocation. The paper has no counterpart:
 * this is a service for callers that cannot allocate device memory while they
 * run -- latency-critical loops that must not wait on an allocator, or
 * applications that give all GPU memory to their own pool beforehand.
 *  Same arguments and results as nqs_draws (bit-identical ranks and W), but
 *  samples, ranks and w_total must be device pointers; host pointers are
 *  rejected with NQS_ERR_INVALID_ARG because staging them would allocate.
 *  Working memory is a fixed array of NQS_NOALLOC_SCRATCH_BYTES inside the
 *  library image, present on every GPU that loads the library until the
 *  process exits. A batch needs 8 * (2 + Ns + 1.5 Ns ceil(n_conn / 32))
 *  bytes of it; larger batches return NQS_ERR_INVALID_ARG (split them).
 *  The first call on each context looks up the array's device address on
 *  the context's device (with cudaGetSymbolAddress); make that first call
 *  before any stream capture on that device.
 *  All calls share the one array: calls that overlap on the GPU (other
 *  streams, other contexts on the same device) race and corrupt each other.
 *  Reads the device error word back and synchronises the context's stream
 *  before returning. */
#define NQS_NOALLOC_SCRATCH_BYTES (8 << 20)
int nqs_draws_noalloc(nqs_ctx* ctx, const uint64_t* samples, int64_t Ns, double det_threshold,
                      int n_draws, uint64_t philox_seed, int64_t* ranks, uint64_t* w_total);

/* Semistochastic local energy (Sec. 2.4):
 *  E_loc(n) = H_nn + sum_{|H_nm|>=eps} H_nm r_m
 *           + (1/N_eps) sum_d H_{m_d} (W / w_{m_d}) r_{m_d},  r_m = psi(m)/psi(n),
 *  draws as in nqs_draws. counts [Ns] weight the summary (may be NULL: all 1).
 *  e_loc [Ns] receives E_loc; `out` (host struct, may be NULL) the summary.
 *  n_draws = 0 keeps only the deterministic part (biased); an empty or
 *  zero-weight remainder gives E^s = 0. A sample with psi(n) = 0 yields
 *  NQS_ERR_INVALID_ARG. The shared-prefix forms return NQS_ERR_UNSUPPORTED
 *  for n_hidden > 512 and when one sample batch's tables would exceed 2^32
 *  rows of D elements (rows are addressed by 32-bit indices; the batch size
 *  follows the memory budget, so this needs a budget far above 2^32 rows). */
int nqs_local_energy(nqs_ctx* ctx, const uint64_t* samples, const double* counts, int64_t Ns,
                     double det_threshold, int n_draws, uint64_t philox_seed, double* e_loc,
                     nqs_energy_summary* out);

/* One system of a multi-system batch (nqs_local_energy_batch): the arguments
 * of nqs_local_energy for that system, and its status on return. With any of
 * grad_sites / grad_W / grad_b non-NULL the system runs nqs_energy_gradient
 * instead (the energy gradient of Eq. egrad, or of Sec. 2.3 with reweighted). */
typedef struct {
    const uint64_t* samples;     /* [n_samples][2], host or device */
    const double* counts;        /* [n_samples] or NULL */
    int64_t n_samples;
    double det_threshold;        /* eps */
    int n_draws;                 /* N_eps */
    uint64_t philox_seed;
    double* e_loc;               /* [n_samples] out */
    nqs_energy_summary* summary; /* host struct or NULL */
    int status;                  /* out: this system's nqs_status */
    int reweighted;              /* energy gradient form (see nqs_energy_gradient) */
    double* grad_sites;          /* [n_edges][4][D][D] out, or NULL */
    double* grad_W;              /* [n_hidden][2K] out, or NULL */
    double* grad_b;              /* [n_hidden] out, or NULL */
} nqs_batch_item;

/* Local energies of independent systems in one call (no counterpart in the
 * paper, which treats one molecule at a time; the path of each system is the
 * one of nqs_local_energy, Sec. 2.4). ctxs[i] holds system i's Hamiltonian,
 * ansatz and options (systems may differ in K, N_alpha, N_beta, D, precision);
 * the contexts must be distinct. Systems are taken in decreasing order of
 * estimated cost (n_samples * n_conn * K * D) from a shared queue by
 * `n_workers` host threads (<= 0: min(n_sys, 8)), each driving its system's
 * context stream, so the work of several systems overlaps on the GPU.
 * Each context's shared-prefix tables are capped at a 1/(3 n_sys) share of the
 * device memory free at the call (contexts keep their buffers between calls).
 * Returns NQS_OK when every system succeeded, else the status of the first
 * failing system (by index; nqs_last_error(ctxs[i]) has its message); every
 * item's `status` is set. Each context's stream is synchronised on return.
 * Systems overlap only if their contexts run on distinct non-default streams. */
int nqs_local_energy_batch(nqs_ctx* const* ctxs, int n_sys, nqs_batch_item* items, int n_workers);

/* Vector-Jacobian product of d log|psi(n)| / d theta (Eq. egrad):
 *  grad = sum_n u[n] d log|psi(n)| / d theta, theta = (site tensors, W, b).
 *  grad_sites [n_edges][4][D][D], grad_W [n_hidden][2K], grad_b [n_hidden];
 *  outputs are overwritten (not accumulated); NULL skips one. With
 *  u_n = 2 c_n (E_loc(n) - E_mean) / sum c this is the energy gradient.
 *  FP64. The site-tensor part is, per edge and local state, the sum over the
 *  samples of that local state of u_n / psi_TN(n) g_i(n) h_j(n)^T (adjoint
 *  times forward cell); nqs_options.grad_chunk bounds how many samples'
 *  environments are held at once. */
int nqs_grad_log_psi_vjp(nqs_ctx* ctx, const uint64_t* samples, const double* u, int64_t Ns,
                         double* grad_sites, double* grad_W, double* grad_b);

/* nqs_grad_log_psi_vjp with the Ising-RBM couplings as well:
 *  grad_W2 [n_hidden][2K][2K] (d theta_k / d W2[k][s][t] = n_s n_t / 2);
 *  non-NULL grad_W2 needs NQS_CORR_ISING. */
int nqs_grad_log_psi_vjp2(nqs_ctx* ctx, const uint64_t* samples, const double* u, int64_t Ns,
                          double* grad_sites, double* grad_W, double* grad_b, double* grad_W2);

/* Energy gradient in one call: nqs_local_energy (the context's precision and
 * options), then on the device the weights
 *   reweighted = 0 (Eq. egrad):  u_n = 2 c_n (E_loc(n) - E_mean) / sum c
 *   reweighted = 1 (Sec. 2.3):   u_n = 2 c_n f~_n^2 (E_loc(n) - E_theta) / sum c,
 *                                f~_n^2 = f_n^2 / B, E_theta = e_tilde_mean
 * (the latter for samples drawn from |Phi|^2 with the correlator f outside the
 * normalised part), then the FP64 VJP. Outputs as in nqs_grad_log_psi_vjp2
 * (any may be NULL); e_loc [Ns] (may be NULL) receives E_loc, `out` the
 * summary. Needs Ns > 0. */
int nqs_energy_gradient(nqs_ctx* ctx, const uint64_t* samples, const double* counts, int64_t Ns,
                        double det_threshold, int n_draws, uint64_t philox_seed, int reweighted,
                        double* grad_sites, double* grad_W, double* grad_b, double* grad_W2,
                        double* e_loc, nqs_energy_summary* out);

/* Autoregressive sampling from |Phi|^2 of the normalised readout (Sec. 2.1:
 * the ansatz's conditionals allow exact sampling; Sec. 3: breadth first over
 * the vertices, the constraint built into the conditionals). n_samples draws
 * grouped into unique determinants: a node of level i is a distinct prefix
 * holding `cnt` of the draws at offsets off .. off+cnt-1 (the nodes of a level
 * tile the draws in prefix order); draw j picks the local state of vertex i
 * as the first allowed s with u_j Z < sum_{allowed s' <= s} P_i(s') (Z the
 * sum over the allowed states; the last allowed state if rounding leaves
 * none), u_j = (x >> 11) 2^-53 with x the first output of Philox4x64-10 with
 * key (seed, 0) and counter (j, i, 1, 0); the children keep the offsets in the
 * order of s. The result depends on seed and n_samples only.
 *  samples [capacity][2], counts [capacity] (host or device) receive the
 *  unique determinants in prefix order (vertex 0 most significant, local
 *  state order 0..3) and their counts; *n_unique (host) their number.
 *  capacity < n_unique -> NQS_ERR_INVALID_ARG with *n_unique written.
 *  Needs nqs_set_readout (NQS_ERR_STATE otherwise). */
int nqs_sample(nqs_ctx* ctx, int64_t n_samples, uint64_t seed, uint64_t* samples, double* counts,
               int64_t capacity, int64_t* n_unique);

#ifdef __cplusplus
}
#endif
#endif
