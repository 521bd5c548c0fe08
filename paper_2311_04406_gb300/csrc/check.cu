// check.cu -- check shares (a6).
//
// Compact check, Fig. Pi_CompactMatMul verification steps 3-5 reduced mod
// 2^(k+s):  cs = sum_r chi^_r (alpha Dc_r - mDc_r).  M values: one block.
//
// BatchRec tag check, Fig. Pi_BatchRec (§2.5) steps 2-3:
//   cs = sum_{p,q} chi_pq (mW_pq - alpha W_pq).  M x N values: a grid of
// blocks leaves per-block partial sums in the workspace, one block adds them.
// Wrapping sums mod 2^(64 W) are order independent, so the result is the same
// for any grid.
#include "common.cuh"
#include "kernels.h"
#include "sm100_ptx.cuh"

namespace mpcl {

namespace {

constexpr int NT = 512;

template <int W>
__device__ typename Elem<W>::T block_sum(typename Elem<W>::T v) {
    using T = typename Elem<W>::T;
    __shared__ T sh[NT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if constexpr (W == 1) {
            v += __shfl_xor_sync(0xffffffffu, v, o);
        } else {
            u64 lo = __shfl_xor_sync(0xffffffffu, (u64)v, o);
            u64 hi = __shfl_xor_sync(0xffffffffu, (u64)(v >> 64), o);
            v += (u128)lo | ((u128)hi << 64);
        }
    }
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T tot = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < NT / 32; ++i) tot += sh[i];
    return tot;  // valid in thread 0
}

template <int W>
__global__ void __launch_bounds__(NT) check_compact_kernel(int64_t M, const u64* alpha,
                                                           const u64* chi_hat, const u64* Dc,
                                                           const u64* mDc, u64* cs) {
    using T = typename Elem<W>::T;
    ptx::grid_dep_launch();
    ptx::grid_dep_wait();   // launched as a dependent of the kernel before it
    const T a = ld_elem<W>(alpha, 0);
    T acc = 0;
    for (int64_t r = threadIdx.x; r < M; r += NT)
        acc += ldg_elem<W>(chi_hat, r) * (a * ldg_elem<W>(Dc, r) - ldg_elem<W>(mDc, r));
    T tot = block_sum<W>(acc);
    if (threadIdx.x == 0) st_elem<W>(cs, 0, tot);
}

// Up to CHECK_GROUP_MAX compact checks in one launch: block b computes the
// check share of layer b (the same sum as check_compact_kernel).
struct CheckGroup {
    int count;
    int64_t M[CHECK_GROUP_MAX];
    const u64* alpha[CHECK_GROUP_MAX];
    const u64* chi_hat[CHECK_GROUP_MAX];
    const u64* Dc[CHECK_GROUP_MAX];
    const u64* mDc[CHECK_GROUP_MAX];
    u64* cs[CHECK_GROUP_MAX];
};

template <int W>
__global__ void __launch_bounds__(NT) check_compact_group_kernel(const __grid_constant__ CheckGroup g) {
    using T = typename Elem<W>::T;
    ptx::grid_dep_launch();
    ptx::grid_dep_wait();   // launched as a dependent of the kernel before it
    const int l = blockIdx.x;
    const T a = ld_elem<W>(g.alpha[l], 0);
    T acc = 0;
    for (int64_t r = threadIdx.x; r < g.M[l]; r += NT)
        acc += ldg_elem<W>(g.chi_hat[l], r) * (a * ldg_elem<W>(g.Dc[l], r) - ldg_elem<W>(g.mDc[l], r));
    T tot = block_sum<W>(acc);
    if (threadIdx.x == 0) st_elem<W>(g.cs[l], 0, tot);
}

template <int W>
__global__ void __launch_bounds__(NT) batchrec_partial_kernel(int64_t n, const u64* alpha,
                                                              const u64* chi, const u64* Wm,
                                                              const u64* mW, u64* part) {
    using T = typename Elem<W>::T;
    const T a = ld_elem<W>(alpha, 0);
    T acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) {
        T x = ldg_elem<W>(chi, i);
        acc += ldg_elem<W>(mW, i) * x - a * (ldg_elem<W>(Wm, i) * x);
    }
    T tot = block_sum<W>(acc);
    if (threadIdx.x == 0) st_elem<W>(part, blockIdx.x, tot);
}

// Combiners expanded from a public seed: the SplitMix64 sequence whose state
// starts at the seed (Steele, Lea & Flood 2014), chi_i = mix(seed + (i+1) g)
// mod 2^s.  Generated in registers, so the check reads only W and m(W).
__device__ __forceinline__ u64 splitmix64_at(u64 seed, int64_t i) {
    u64 z = seed + (u64)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <int W>
__global__ void __launch_bounds__(NT) batchrec_seeded_partial_kernel(int64_t n, int s, const u64* alpha,
                                                                     const u64* seedp, const u64* Wm,
                                                                     const u64* mW, u64* part) {
    using T = typename Elem<W>::T;
    const T a = ld_elem<W>(alpha, 0);
    const u64 seed = seedp[0];
    const u64 ms = s >= 64 ? ~0ull : ((1ull << s) - 1);
    T acc = 0;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) {
        const T x = (T)(splitmix64_at(seed, i) & ms);
        acc += ldg_elem<W>(mW, i) * x - a * (ldg_elem<W>(Wm, i) * x);
    }
    T tot = block_sum<W>(acc);
    if (threadIdx.x == 0) st_elem<W>(part, blockIdx.x, tot);
}

// Pi_BatchRec open phase step 1: [W]_i = [X]_i - [A]_i + [R]_i and the same
// combination of the tag shares (A, mA may be NULL)
template <int W>
__global__ void __launch_bounds__(NT) batchrec_mask_kernel(int64_t n, const u64* X, const u64* A,
                                                           const u64* R, const u64* mX, const u64* mA,
                                                           const u64* mR, u64* Wo, u64* mWo) {
    using T = typename Elem<W>::T;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) {
        T v = ldg_elem<W>(X, i) + ldg_elem<W>(R, i);
        T t = ldg_elem<W>(mX, i) + ldg_elem<W>(mR, i);
        if (A) v -= ldg_elem<W>(A, i);
        if (mA) t -= ldg_elem<W>(mA, i);
        st_elem<W>(Wo, i, v);
        st_elem<W>(mWo, i, t);
    }
}

template <int W>
__global__ void __launch_bounds__(NT) sum_kernel(int64_t n, const u64* part, u64* out) {
    using T = typename Elem<W>::T;
    T acc = 0;
    for (int64_t i = threadIdx.x; i < n; i += NT) acc += ld_elem<W>(part, i);
    T tot = block_sum<W>(acc);
    if (threadIdx.x == 0) st_elem<W>(out, 0, tot);
}

int64_t batchrec_blocks(int64_t n) {
    int64_t b = (n + NT * 8 - 1) / (NT * 8);
    if (b < 1) b = 1;
    if (b > 1216) b = 1216;
    return b;
}

}  // namespace

cudaError_t launch_check_compact(int64_t M, int words, const u64* alpha, const u64* chi_hat,
                                 const u64* Dc, const u64* mDc, u64* cs, cudaStream_t st) {
    const cudaError_t e = words == 1 ? launch_dependent(check_compact_kernel<1>, dim3(1), dim3(NT), 0, st, M, alpha,
                                                        chi_hat, Dc, mDc, cs)
                                     : launch_dependent(check_compact_kernel<2>, dim3(1), dim3(NT), 0, st, M, alpha,
                                                        chi_hat, Dc, mDc, cs);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_check_compact_grouped(int n, int words, const int64_t* M, const u64* const* alpha,
                                         const u64* const* chi_hat, const u64* const* Dc,
                                         const u64* const* mDc, u64* const* cs, cudaStream_t st) {
    for (int i0 = 0; i0 < n; i0 += CHECK_GROUP_MAX) {
        CheckGroup g{};
        g.count = n - i0 < CHECK_GROUP_MAX ? n - i0 : CHECK_GROUP_MAX;
        for (int j = 0; j < g.count; ++j) {
            g.M[j] = M[i0 + j];
            g.alpha[j] = alpha[i0 + j];
            g.chi_hat[j] = chi_hat[i0 + j];
            g.Dc[j] = Dc[i0 + j];
            g.mDc[j] = mDc[i0 + j];
            g.cs[j] = cs[i0 + j];
        }
        const cudaError_t e =
            words == 1 ? launch_dependent(check_compact_group_kernel<1>, dim3(g.count), dim3(NT), 0, st, g)
                       : launch_dependent(check_compact_group_kernel<2>, dim3(g.count), dim3(NT), 0, st, g);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t launch_check_batchrec_seeded(int64_t M, int64_t N, int words, int s, const u64* alpha,
                                         const u64* seed, const u64* Wm, const u64* mW, u64* cs,
                                         void* ws, size_t ws_bytes, cudaStream_t st) {
    const int64_t n = M * N;
    const int64_t blocks = batchrec_blocks(n);
    if (ws_bytes < (size_t)blocks * 8 * (size_t)words) return cudaErrorInvalidValue;
    u64* part = (u64*)ws;
    if (words == 1) {
        batchrec_seeded_partial_kernel<1><<<(unsigned)blocks, NT, 0, st>>>(n, s, alpha, seed, Wm, mW, part);
        sum_kernel<1><<<1, NT, 0, st>>>(blocks, part, cs);
    } else {
        batchrec_seeded_partial_kernel<2><<<(unsigned)blocks, NT, 0, st>>>(n, s, alpha, seed, Wm, mW, part);
        sum_kernel<2><<<1, NT, 0, st>>>(blocks, part, cs);
    }
    return cudaGetLastError();
}

cudaError_t launch_batchrec_mask(int64_t n, int words, const u64* X, const u64* A, const u64* R,
                                 const u64* mX, const u64* mA, const u64* mR, u64* Wo, u64* mWo,
                                 cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    int64_t blocks = (n + NT - 1) / NT;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (words == 1) batchrec_mask_kernel<1><<<(unsigned)blocks, NT, 0, st>>>(n, X, A, R, mX, mA, mR, Wo, mWo);
    else batchrec_mask_kernel<2><<<(unsigned)blocks, NT, 0, st>>>(n, X, A, R, mX, mA, mR, Wo, mWo);
    return cudaGetLastError();
}

size_t check_batchrec_workspace(int64_t M, int64_t N, int words) {
    return (size_t)batchrec_blocks(M * N) * 8 * (size_t)words;
}

cudaError_t launch_check_batchrec(int64_t M, int64_t N, int words, const u64* alpha,
                                  const u64* chi, const u64* Wm, const u64* mW, u64* cs,
                                  void* ws, size_t ws_bytes, cudaStream_t st) {
    const int64_t n = M * N;
    const int64_t blocks = batchrec_blocks(n);
    if (ws_bytes < check_batchrec_workspace(M, N, words)) return cudaErrorInvalidValue;
    u64* part = (u64*)ws;
    if (words == 1) {
        batchrec_partial_kernel<1><<<(unsigned)blocks, NT, 0, st>>>(n, alpha, chi, Wm, mW, part);
        sum_kernel<1><<<1, NT, 0, st>>>(blocks, part, cs);
    } else {
        batchrec_partial_kernel<2><<<(unsigned)blocks, NT, 0, st>>>(n, alpha, chi, Wm, mW, part);
        sum_kernel<2><<<1, NT, 0, st>>>(blocks, part, cs);
    }
    return cudaGetLastError();
}

}  // namespace mpcl
