// nqs_mixed.cuh -- interface of the tensor-core (mixed-precision) amplitude
// path for chain ansaetze.
#pragma once

#include "nqs_kernels.cuh"

namespace nqs {

struct MixedAnsatz {
    int K = 0, D = 0;
    void* params = nullptr;     // device buffer owned by the context
};

size_t mixed_param_bytes(int K, int D);
int mixed_upload(MixedAnsatz& m, const double* hA, int K, int D, void* dev_buf, cudaStream_t st);
int mixed_rows_per_block(const MixedAnsatz& m);
size_t mixed_workspace_bytes(const MixedAnsatz& m, const AmpArgs& a);
int mixed_amp(const MixedAnsatz& m, const AmpArgs& a, void* workspace, cudaStream_t st,
              int* launches);

}  // namespace nqs
