// gemm_simt.cu -- exact ring GEMM on the integer pipes (CUDA cores).
//
// Computes Z = C + [E | X + c E] . [B ; F] mod 2^(64 W) (the 2K form of
// Eq. (compute-z) and Eq. (compute-ztag), §2.5) for layers the tensor-core
// kernel (gemm_tc.cu) does not take: Z_2^64 layers with odd N, layers too small
// to amortise a 128-row MMA tile, and skinny layers (M <= 8, e.g. dense layers
// at batch 1) whose cost is streaming [B ; F] from memory.
//
// Two kernels, both optionally split along K over grid.z:
//   * ring_gemm_simt_kernel<W, TM>: TM x 64 outputs per 256-thread block
//     (TM = 64, or 16 for layers whose 64-row tiles would leave most SMs
//     idle), 16-deep K slices staged in shared memory, each thread owns a
//     (TM / 16) x 4 strided sub-tile (conflict-free shared reads).
//   * ring_gemv_kernel (M <= 8): one thread per output column keeps M sums;
//     the M rows of the left operand are staged in shared memory per K chunk
//     and the right operand is read once, coalesced along N.  For narrow
//     layers (N <= 256) ring_gemv_narrow_kernel instead has a block's eight
//     warps take interleaved rows of its K range and add their sums up in
//     shared memory, so that a block contributes one partial per output.
// With a K split, Z is first set to C (a device-to-device copy) and every
// block adds its partial sums with exact wrapping atomics; without one, the
// block writes C + sum.  Out-of-range rows/columns/K are zero-filled.
#include "common.cuh"
#include "kernels.h"

namespace mpcl {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;
constexpr int BM_SMALL = 16;     // tile rows of the small-grid variant
constexpr int GV_M = 8;         // rows handled by the skinny kernel
constexpr int GV_KC = 128;      // K chunk staged in shared memory
constexpr int GV_NARROW = 256;  // widest layer (N) on the narrow GEMV (measured: faster up to N = 128-256,
                                // slower when streaming 4096-wide rows)

// element kv of row m of the left operand [E | X + cE] (one_half: X + cE)
template <int W>
__device__ __forceinline__ typename Elem<W>::T left(const GemmArgs& a, typename Elem<W>::T c,
                                                   int64_t m, int64_t kv) {
    using T = typename Elem<W>::T;
    if (a.one_half) kv += a.K;
    if (kv < a.K) return ldg_elem<W>(a.E, m * a.K + kv);
    const int64_t kx = kv - a.K;
    T v = ldg_elem<W>(a.X, m * a.K + kx);
    if (a.coef != COEF_ZERO) v += c * ldg_elem<W>(a.E, m * a.K + kx);
    return v;
}

template <int W>
__device__ __forceinline__ typename Elem<W>::T coef_value(const GemmArgs& a) {
    if (a.coef == COEF_ONE) return 1;
    if (a.coef == COEF_ALPHA) return ld_elem<W>(a.alpha, 0);
    return 0;
}

template <int W, int TM>
__global__ void __launch_bounds__(NT) ring_gemm_simt_kernel(GemmArgs a, int64_t kchunk, int atomic) {
    using T = typename Elem<W>::T;
    constexpr int RI = TM / 16;        // rows of a thread's sub-tile
    __shared__ T Ls[BK][TM + 1];
    __shared__ T Rs[BK][BN];

    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t m0 = (int64_t)blockIdx.y * TM, n0 = (int64_t)blockIdx.x * BN;
    const int64_t M = a.M, K = a.K, N = a.N, K2 = a.one_half ? a.K : 2 * a.K;
    const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
    const int64_t kend = kbeg + kchunk < K2 ? kbeg + kchunk : K2;
    const T c = coef_value<W>(a);
    const int64_t kr = a.one_half ? K : 0;   // row offset into [B ; F]

    T acc[RI][4];
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0;

    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
        for (int r = 0; r < (TM * BK) / NT; ++r) {
            int idx = tid + r * NT;
            int mm = idx / BK, kk = idx % BK;
            int64_t m = m0 + mm, kv = k0 + kk;
            Ls[kk][mm] = (m < M && kv < kend) ? left<W>(a, c, m, kv) : (T)0;
        }
#pragma unroll
        for (int r = 0; r < (BK * BN) / NT; ++r) {
            int idx = tid + r * NT;
            int kk = idx / BN, nn = idx % BN;
            int64_t n = n0 + nn, kv = k0 + kk;
            T v = 0;
            if (n < N && kv < kend) {
                const int64_t kq = kv + kr;
                v = kq < K ? ldg_elem<W>(a.B, kq * N + n) : ldg_elem<W>(a.F, (kq - K) * N + n);
            }
            Rs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            T av[RI], bv[4];
#pragma unroll
            for (int i = 0; i < RI; ++i) av[i] = Ls[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Rs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < RI; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += av[i] * bv[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < RI; ++i) {
        int64_t m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t n = n0 + tx + 16 * j;
            if (n >= N) continue;
            if (atomic) atomic_add_elem<W>(a.Z, m * N + n, acc[i][j]);
            else st_elem<W>(a.Z, m * N + n, (a.C ? ldg_elem<W>(a.C, m * N + n) : (T)0) + acc[i][j]);
        }
    }
}

// GEMV for wide layers: one thread per VEC output columns keeps M sums over
// every row of the block's K range (deep independent loads along K).  VEC = 2:
// two adjacent Z_2^64 columns per thread, read as one 16-byte vector (needs
// even N); VEC = 1 otherwise.  MM >= M rows are accumulated (1, 2, 4 or 8).
template <int W, int VEC, int MM>
__global__ void __launch_bounds__(NT) ring_gemv_kernel(GemmArgs a, int64_t kchunk, int atomic) {
    using T = typename Elem<W>::T;
    __shared__ T Ls[MM][GV_KC];
    const int64_t n = ((int64_t)blockIdx.x * NT + threadIdx.x) * VEC;
    const int64_t K = a.K, N = a.N, K2 = a.one_half ? a.K : 2 * a.K;
    const int64_t kr = a.one_half ? K : 0;   // row offset into [B ; F]
    const int M = (int)a.M;
    const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
    const int64_t kend = kbeg + kchunk < K2 ? kbeg + kchunk : K2;
    const T c = coef_value<W>(a);
    T acc[MM][VEC];
#pragma unroll
    for (int i = 0; i < MM; ++i)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[i][v] = 0;
    for (int64_t k0 = kbeg; k0 < kend; k0 += GV_KC) {
        const int kc = (int)(kend - k0 < GV_KC ? kend - k0 : GV_KC);
        for (int idx = threadIdx.x; idx < MM * GV_KC; idx += NT) {
            const int mm = idx / GV_KC, kk = idx % GV_KC;
            Ls[mm][kk] = (mm < M && kk < kc) ? left<W>(a, c, mm, k0 + kk) : (T)0;
        }
        __syncthreads();
        if (n < N) {
#pragma unroll 8
            for (int kk = 0; kk < kc; ++kk) {
                const int64_t kv = k0 + kk + kr;
                const u64* row = kv < K ? a.B + kv * N * W : a.F + (kv - K) * N * W;
                T r[VEC];
                if constexpr (VEC == 2) {
                    const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(row + n));
                    r[0] = v.x;
                    r[1] = v.y;
                } else {
                    r[0] = ldg_elem<W>(row, n);
                }
#pragma unroll
                for (int i = 0; i < MM; ++i)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[i][v] += Ls[i][kk] * r[v];
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
        const int64_t col = n + v;
        if (col >= N) break;
#pragma unroll
        for (int i = 0; i < MM; ++i) {
            if (i >= M) break;
            if (atomic) atomic_add_elem<W>(a.Z, (int64_t)i * N + col, acc[i][v]);
            else st_elem<W>(a.Z, (int64_t)i * N + col,
                            (a.C ? ldg_elem<W>(a.C, (int64_t)i * N + col) : (T)0) + acc[i][v]);
        }
    }
}

// GEMV for narrow layers (N <= GV_NARROW): a block covers 32 lanes x VEC
// output columns and its eight warps take rows w, w + 8, ... of each staged K
// chunk; the warps' sums are added in shared memory before the block writes
// (or atomically adds) one partial per output, so that many blocks can share
// the K range of few columns.  VEC and MM as above.
template <int W, int VEC, int MM>
__global__ void __launch_bounds__(NT) ring_gemv_narrow_kernel(GemmArgs a, int64_t kchunk, int atomic) {
    using T = typename Elem<W>::T;
    constexpr int NW = NT / 32;                 // warps per block
    constexpr int NCOL = 32 * VEC;              // columns per block
    __shared__ T Ls[MM][GV_KC];
    __shared__ T red[NW - 1][MM][NCOL];         // sums of warps 1 .. NW - 1
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t n = (int64_t)blockIdx.x * NCOL + lane * VEC;
    const int64_t K = a.K, N = a.N, K2 = a.one_half ? a.K : 2 * a.K;
    const int64_t kr = a.one_half ? K : 0;   // row offset into [B ; F]
    const int M = (int)a.M;
    const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
    const int64_t kend = kbeg + kchunk < K2 ? kbeg + kchunk : K2;
    const T c = coef_value<W>(a);
    T acc[MM][VEC];
#pragma unroll
    for (int i = 0; i < MM; ++i)
#pragma unroll
        for (int v = 0; v < VEC; ++v) acc[i][v] = 0;
    for (int64_t k0 = kbeg; k0 < kend; k0 += GV_KC) {
        const int kc = (int)(kend - k0 < GV_KC ? kend - k0 : GV_KC);
        for (int idx = threadIdx.x; idx < MM * GV_KC; idx += NT) {
            const int mm = idx / GV_KC, kk = idx % GV_KC;
            Ls[mm][kk] = (mm < M && kk < kc) ? left<W>(a, c, mm, k0 + kk) : (T)0;
        }
        __syncthreads();
        if (n < N) {
#pragma unroll 4
            for (int kk = warp; kk < kc; kk += NW) {
                const int64_t kv = k0 + kk + kr;
                const u64* row = kv < K ? a.B + kv * N * W : a.F + (kv - K) * N * W;
                T r[VEC];
                if constexpr (VEC == 2) {
                    const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(row + n));
                    r[0] = v.x;
                    r[1] = v.y;
                } else {
                    r[0] = ldg_elem<W>(row, n);
                }
#pragma unroll
                for (int i = 0; i < MM; ++i)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) acc[i][v] += Ls[i][kk] * r[v];
            }
        }
        __syncthreads();
    }
    if (warp > 0) {
#pragma unroll
        for (int i = 0; i < MM; ++i)
#pragma unroll
            for (int v = 0; v < VEC; ++v) red[warp - 1][i][lane * VEC + v] = acc[i][v];
    }
    __syncthreads();
    if (warp != 0) return;
#pragma unroll
    for (int w = 0; w < NW - 1; ++w)
#pragma unroll
        for (int i = 0; i < MM; ++i)
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[i][v] += red[w][i][lane * VEC + v];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
        const int64_t col = n + v;
        if (col >= N) break;
#pragma unroll
        for (int i = 0; i < MM; ++i) {
            if (i >= M) break;
            if (atomic) atomic_add_elem<W>(a.Z, (int64_t)i * N + col, acc[i][v]);
            else st_elem<W>(a.Z, (int64_t)i * N + col,
                            (a.C ? ldg_elem<W>(a.C, (int64_t)i * N + col) : (T)0) + acc[i][v]);
        }
    }
}

// K chunks (multiples of `step`, at least `min_chunk`) so that the grid covers
// about `waves` x 152 blocks
int64_t choose_kchunk(int64_t blocks_2d, int64_t K2, int64_t step, int64_t min_chunk, int64_t waves) {
    int64_t splits = waves * 152 / (blocks_2d > 0 ? blocks_2d : 1);
    const int64_t max_splits = (K2 + min_chunk - 1) / min_chunk;
    if (splits > max_splits) splits = max_splits;
    if (splits < 1) splits = 1;
    int64_t chunk = (K2 + splits - 1) / splits;
    chunk = ((chunk + step - 1) / step) * step;
    return chunk > 0 ? chunk : step;
}

}  // namespace

// Tile rows of the integer-pipe GEMM: the launch table's choice (64 or 16),
// else 16 when 64-row tiles would give fewer blocks than SMs.
int simt_tile_rows(int64_t M, int64_t N, int rows) {
    if (rows == 64 || rows == BM_SMALL) return rows;
    return ((M + BM - 1) / BM) * ((N + BN - 1) / BN) < 152 ? BM_SMALL : BM;
}

namespace {

template <int W>
cudaError_t run(const GemmArgs& a, cudaStream_t st) {
    const int64_t K2 = a.one_half ? a.K : 2 * a.K;
    const bool skinny = a.M <= GV_M;
    const int vec = (skinny && W == 1 && a.N % 2 == 0) ? 2 : 1;
    const int tm = simt_tile_rows(a.M, a.N, a.rows);
    const bool narrow = skinny && a.N <= GV_NARROW;
    const int64_t cols = narrow ? 32 * vec : NT * vec;   // columns per GEMV block
    const int64_t bx = skinny ? (a.N + cols - 1) / cols : (a.N + BN - 1) / BN;
    const int64_t by = skinny ? 1 : (a.M + tm - 1) / tm;
    if (by > 65535) return cudaErrorInvalidConfiguration;
    // K split so that the grid covers about `waves` x 152 blocks (launch table, else 4 / 2);
    // GEMV chunks give each of a block's eight warps at least 16 rows
    const int64_t waves = a.simt_waves > 0 ? a.simt_waves : (skinny ? 4 : 2);
    const int64_t kchunk = skinny ? choose_kchunk(bx * by, K2, 16, narrow ? 128 : 32, waves)
                                  : choose_kchunk(bx * by, K2, BK, 4 * BK, waves);
    const int64_t bz = K2 > 0 ? (K2 + kchunk - 1) / kchunk : 1;
    if (bz > 65535) return cudaErrorInvalidConfiguration;
    const int atomic = bz > 1 ? 1 : 0;
    if (atomic) {
        const size_t bytes = (size_t)a.M * a.N * 8 * W;
        cudaError_t e = a.C ? cudaMemcpyAsync(a.Z, a.C, bytes, cudaMemcpyDeviceToDevice, st)
                            : cudaMemsetAsync(a.Z, 0, bytes, st);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)bx, (unsigned)by, (unsigned)bz);
    if (skinny) {
        const int mm = a.M <= 1 ? 1 : a.M <= 2 ? 2 : a.M <= 4 ? 4 : 8;
#define MPCL_GEMV(V, R)                                                                  \
    (narrow ? ring_gemv_narrow_kernel<W, V, R><<<grid, NT, 0, st>>>(a, kchunk, atomic)   \
            : ring_gemv_kernel<W, V, R><<<grid, NT, 0, st>>>(a, kchunk, atomic))
        if (vec == 2) {
            if (mm == 1) MPCL_GEMV(2, 1); else if (mm == 2) MPCL_GEMV(2, 2);
            else if (mm == 4) MPCL_GEMV(2, 4); else MPCL_GEMV(2, 8);
        } else {
            if (mm == 1) MPCL_GEMV(1, 1); else if (mm == 2) MPCL_GEMV(1, 2);
            else if (mm == 4) MPCL_GEMV(1, 4); else MPCL_GEMV(1, 8);
        }
#undef MPCL_GEMV
    } else if (tm == BM_SMALL) {
        ring_gemm_simt_kernel<W, BM_SMALL><<<grid, NT, 0, st>>>(a, kchunk, atomic);
    } else {
        ring_gemm_simt_kernel<W, BM><<<grid, NT, 0, st>>>(a, kchunk, atomic);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_simt(const GemmArgs& a, cudaStream_t st) {
    if (a.M == 0 || a.N == 0) return cudaSuccess;
    return a.words == 1 ? run<1>(a, st) : run<2>(a, st);
}

}  // namespace mpcl
