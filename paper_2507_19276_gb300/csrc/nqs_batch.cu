// nqs_batch.cu -- local energies of independent systems in one call: a
// longest-first queue over systems, drained by host worker threads that each
// drive one system's context (and its CUDA stream) at a time.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <numeric>
#include <thread>
#include <vector>

#include "../../include/nqs.h"

namespace nqs {
// context queries of nqs_api.cu
int ctx_shape(const nqs_ctx* c, int* K, int* na, int* nb, int* D);
int ctx_sync(nqs_ctx* c);
void ctx_set_table_budget(nqs_ctx* c, size_t bytes);
size_t ctx_free_memory(nqs_ctx* c);
}  // namespace nqs

namespace {

// n_conn(K, N_a, N_b) = S_a + S_b + D_aa + D_bb + D_ab (single and double
// excitations that conserve N_alpha and N_beta)
double n_conn_of(int K, int na, int nb)
{
    const double sa = (double)na * (K - na), sb = (double)nb * (K - nb);
    auto c2 = [](double n) { return n * (n - 1) / 2; };
    return sa + sb + c2(na) * c2(K - na) + c2(nb) * c2(K - nb) + sa * sb;
}

}  // namespace

extern "C" int nqs_local_energy_batch(nqs_ctx* const* ctxs, int n_sys, nqs_batch_item* items,
                                      int n_workers)
{
    if (n_sys < 0 || (n_sys > 0 && (!ctxs || !items))) return NQS_ERR_INVALID_ARG;
    if (n_sys == 0) return NQS_OK;
    for (int i = 0; i < n_sys; ++i) {
        if (!ctxs[i]) return NQS_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) return NQS_ERR_INVALID_ARG;   // one context per system
    }
    // cost estimate from each context's shape
    std::vector<double> cost((size_t)n_sys, 0.0);
    for (int i = 0; i < n_sys; ++i) {
        int K = 0, na = 0, nb = 0, D = 0;
        if (nqs::ctx_shape(ctxs[i], &K, &na, &nb, &D) != NQS_OK) { K = 1; D = 1; }
        cost[(size_t)i] = (double)items[i].n_samples * n_conn_of(K, na, nb) * K * D;
        items[i].status = NQS_ERR_STATE;
    }
    // every context keeps its tables between calls: share a third of the free
    // memory among the systems of the batch
    const size_t share = nqs::ctx_free_memory(ctxs[0]) / 3 / (size_t)n_sys;
    for (int i = 0; i < n_sys; ++i) nqs::ctx_set_table_budget(ctxs[i], share);
    std::vector<int> order((size_t)n_sys);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[(size_t)a] > cost[(size_t)b]; });
    const int nw = std::max(1, std::min(n_sys, n_workers > 0 ? n_workers : 8));
    std::atomic<int> next{0};
    auto work = [&]() {
        for (;;) {
            const int q = next.fetch_add(1);
            if (q >= n_sys) break;
            const int i = order[(size_t)q];
            nqs_batch_item& it = items[i];
            if (it.grad_sites || it.grad_W || it.grad_b)
                it.status = nqs_energy_gradient(ctxs[i], it.samples, it.counts, it.n_samples, it.det_threshold,
                                                it.n_draws, it.philox_seed, it.reweighted, it.grad_sites,
                                                it.grad_W, it.grad_b, nullptr, it.e_loc, it.summary);
            else
                it.status = nqs_local_energy(ctxs[i], it.samples, it.counts, it.n_samples, it.det_threshold,
                                             it.n_draws, it.philox_seed, it.e_loc, it.summary);
            // leave nothing in flight on this system's stream
            if (it.status == NQS_OK) it.status = nqs::ctx_sync(ctxs[i]);
        }
    };
    std::vector<std::thread> pool;
    for (int w = 1; w < nw; ++w) pool.emplace_back(work);
    work();
    for (auto& t : pool) t.join();
    for (int i = 0; i < n_sys; ++i)
        if (items[i].status != NQS_OK) return items[i].status;
    return NQS_OK;
}
