// gemm_simt.cu -- exact ring GEMM on the integer pipes (CUDA cores).
//
// Computes Z = C + [E | X + c E] . [B ; F] mod 2^(64 W) (the 2K form of
// Eq. (compute-z) and Eq. (compute-ztag), §2.5).  Used for layers too small
// or too thin for the tensor-core kernel (gemm_tc.cu), e.g. K = 27 convs or
// single-row dense layers, where a 128-row MMA tile would be mostly padding.
//
// Tile: 64 x 64 outputs per 256-thread block, 16-deep K slices staged in
// shared memory; each thread owns a 4 x 4 strided sub-tile so that shared
// reads are conflict-free.  Out-of-range rows/columns/K are zero-filled.
#include "common.cuh"
#include "kernels.h"

namespace mpcl {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <int W>
__global__ void __launch_bounds__(NT) ring_gemm_simt_kernel(GemmArgs a) {
    using T = typename Elem<W>::T;
    __shared__ T Ls[BK][BM + 1];
    __shared__ T Rs[BK][BN];

    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
    const int64_t M = a.M, K = a.K, N = a.N, K2 = 2 * a.K;

    T c = 0;
    if (a.coef == COEF_ONE) c = 1;
    else if (a.coef == COEF_ALPHA) c = ld_elem<W>(a.alpha, 0);

    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0;

    for (int64_t k0 = 0; k0 < K2; k0 += BK) {
        // left operand tile: column kv of [E | X + cE]
#pragma unroll
        for (int r = 0; r < (BM * BK) / NT; ++r) {
            int idx = tid + r * NT;
            int mm = idx / BK, kk = idx % BK;
            int64_t m = m0 + mm, kv = k0 + kk;
            T v = 0;
            if (m < M && kv < K2) {
                if (kv < K) {
                    v = ldg_elem<W>(a.E, m * K + kv);
                } else {
                    int64_t kx = kv - K;
                    v = ldg_elem<W>(a.X, m * K + kx);
                    if (a.coef != COEF_ZERO) v += c * ldg_elem<W>(a.E, m * K + kx);
                }
            }
            Ls[kk][mm] = v;
        }
        // right operand tile: row kv of [B ; F]
#pragma unroll
        for (int r = 0; r < (BK * BN) / NT; ++r) {
            int idx = tid + r * NT;
            int kk = idx / BN, nn = idx % BN;
            int64_t n = n0 + nn, kv = k0 + kk;
            T v = 0;
            if (n < N && kv < K2) v = kv < K ? ldg_elem<W>(a.B, kv * N + n) : ldg_elem<W>(a.F, (kv - K) * N + n);
            Rs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = Ls[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Rs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t n = n0 + tx + 16 * j;
            if (n >= N) continue;
            st_elem<W>(a.Z, m * N + n, ldg_elem<W>(a.C, m * N + n) + acc[i][j]);
        }
    }
}

}  // namespace

cudaError_t launch_gemm_simt(const GemmArgs& a, cudaStream_t st) {
    if (a.M == 0 || a.N == 0) return cudaSuccess;
    dim3 grid((unsigned)((a.N + BN - 1) / BN), (unsigned)((a.M + BM - 1) / BM));
    if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
    if (a.words == 1) ring_gemm_simt_kernel<1><<<grid, NT, 0, st>>>(a);
    else ring_gemm_simt_kernel<2><<<grid, NT, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mpcl
