// gemm_tc.cu -- tensor-core ring GEMM (placeholder until the tcgen05 kernel
// lands): reports every shape as not eligible so the SIMT kernel runs.
#include "common.cuh"
#include "kernels.h"

namespace mpcl {

bool gemm_tc_eligible(int64_t, int64_t, int64_t, int) { return false; }
size_t gemm_tc_workspace(int64_t, int64_t, int64_t, int) { return 0; }
cudaError_t launch_gemm_tc(const GemmArgs&, void*, size_t, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace mpcl
