// transpose.cu -- out (cols x rows) = in (rows x cols)^T for ring elements.
//
// Training's backward layers (grad X = grad Z . W^T, grad W = X^T . grad Z) are
// the same per-party Beaver-triple products on transposed operands; a party
// transposes its local shares (no communication) before the opening and the
// GEMM.  32 x 32 element tiles staged in shared memory (padded against bank
// conflicts) keep both the reads and the writes coalesced.
#include "common.cuh"
#include "kernels.h"

namespace mpcl {

namespace {

constexpr int TILE = 32, ROWS = 8;

template <int W>
__global__ void __launch_bounds__(TILE * ROWS) transpose_kernel(int64_t rows, int64_t cols, const u64* in,
                                                                u64* out) {
    using T = typename Elem<W>::T;
    __shared__ T tile[TILE][TILE + 1];
    const int64_t c0 = (int64_t)blockIdx.x * TILE, r0 = (int64_t)blockIdx.y * TILE;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int j = 0; j < TILE; j += ROWS) {
        const int64_t r = r0 + ty + j, c = c0 + tx;
        if (r < rows && c < cols) tile[ty + j][tx] = ldg_elem<W>(in, r * cols + c);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < TILE; j += ROWS) {
        const int64_t c = c0 + ty + j, r = r0 + tx;   // out row c, out column r
        if (r < rows && c < cols) st_elem<W>(out, c * rows + r, tile[tx][ty + j]);
    }
}

}  // namespace

cudaError_t launch_transpose(int64_t rows, int64_t cols, int words, const u64* in, u64* out,
                             cudaStream_t st) {
    if (rows == 0 || cols == 0) return cudaSuccess;
    const int64_t gx = (cols + TILE - 1) / TILE, gy = (rows + TILE - 1) / TILE;
    if (gy > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((unsigned)gx, (unsigned)gy), block(TILE, ROWS);
    if (words == 1) transpose_kernel<1><<<grid, block, 0, st>>>(rows, cols, in, out);
    else transpose_kernel<2><<<grid, block, 0, st>>>(rows, cols, in, out);
    return cudaGetLastError();
}

}  // namespace mpcl
