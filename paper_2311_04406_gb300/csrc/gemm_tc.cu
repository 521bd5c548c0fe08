// gemm_tc.cu -- exact ring GEMM mod 2^64 on the fp16 tensor cores (tcgen05).
//
// Computes Z = C + L . R mod 2^64 with L = [E | X + cE] (M x 2K) and
// R = [B ; F] (2K x N): the 2K form of Eq. (compute-z) and Eq. (compute-ztag)
// (§2.5) shared by the share and the full tag.
//
// Exactness.  sm_103a has no int8 MMA, so every 64-bit word x is written as
// eight signed byte digits d_t in [-128, 127] with x = sum_t d_t 2^(8t) mod
// 2^64 (add 0x80 to every byte mod 2^64, subtract 128 from each byte; the carry
// out of the top byte vanishes mod 2^64).  Digits are exact in fp16, and
//     L.R mod 2^64 = sum_{i+j<=7} (L_i . R_j) 2^(8(i+j)),
// 36 digit products.  Products of digits are at most 2^14 in magnitude, so a
// diagonal accumulator sum_{i+j=t} L_i . R_j over 128 K values holds at most
// (t+1) * 128 * 2^14 <= 2^24 in magnitude: every partial sum is an integer
// exactly representable in fp32, so the fp32 tensor-core accumulation is exact.
// Every 128 K the accumulators are drained to integers and folded into wrapping
// 64-bit sums.
//
// Kernel layout (one CTA = 128 rows x 32 output columns x a K range):
//   * prologue_kernel writes L as 8 fp16 digit planes in exactly the shared
//     memory image the MMA reads (K-major, no swizzle, 8x16-byte core
//     matrices), one 32 KB block per (128-row tile, 16-deep K stage), so the
//     GEMM fetches each A stage with a single bulk TMA copy.
//   * the GEMM streams raw 64-bit R tiles (16 K x 32 N) with 2-D TMA; four
//     converter warps turn each into a stacked B operand of 256 rows: rows
//     32j..32j+31 hold digit plane j of the 32 columns.
//   * one thread issues, per 16-deep K step, 8 MMAs: D[:, 32i : 256] +=
//     L_i . [R_0 | ... | R_{7-i}], so that the product L_i . R_j lands in
//     TMEM column block i + j -- the diagonal it belongs to.  Two 256-column
//     accumulator sets alternate, so draining one overlaps MMAs into the other.
//   * four drain warps read the diagonals with tcgen05.ld, convert them to
//     integers and add d_t 2^(8t) into 32 wrapping 64-bit sums per row.
//   * scheduling is persistent: the (output tile, 128-deep K interval) work
//     units are split evenly over one CTA per SM, so a CTA may cover parts of
//     two tiles.  The prologue sets Z = C and every CTA adds each finished
//     tile segment into Z with red.global.add.u64 -- exact and independent of
//     the order of the additions, because addition mod 2^64 is associative and
//     commutative.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "kernels.h"
#include "sm100_ptx.cuh"

namespace mpcl {

__device__ unsigned int g_tc_timeout = 0;

namespace {

constexpr int BM = 128;                  // rows per tile (TMEM lanes)
constexpr int ND = 32;                   // output columns per tile
constexpr int NDIG = 8;                  // byte digits per 64-bit word
constexpr int NSTACK = NDIG * ND;        // rows of the stacked B operand
constexpr int KS = 16;                   // K per pipeline stage (one MMA K step)
constexpr int STAGES = 4;                // operand stages in shared memory
constexpr int RAW = 8;                   // raw R tiles in flight
constexpr int KD_STAGES = 8;             // stages per drain interval (128 K)
constexpr uint32_t A_PLANE_BYTES = BM * KS * 2;            // 4 KB
constexpr uint32_t A_STAGE_BYTES = NDIG * A_PLANE_BYTES;   // 32 KB
constexpr uint32_t B_STAGE_BYTES = NSTACK * KS * 2;        // 8 KB
constexpr uint32_t RAW_BYTES = KS * ND * 8;                // 4 KB
constexpr uint32_t CORE_LBO = 128;       // next core matrix along K
constexpr uint32_t CORE_SBO = 256;       // next group of 8 rows
constexpr uint32_t TMEM_COLS = 512;      // two accumulator sets of 8 x 32 columns
constexpr int NUM_WARPS = 11;
constexpr int NTHREADS = NUM_WARPS * 32;
constexpr int W_APROD = 0, W_CONV0 = 1, W_MMA = 5, W_BPROD = 10;   // warps 6-9 drain
constexpr int NCONV = 128;               // converter threads
constexpr int NDRAIN = 128;              // drain threads
constexpr long long WAIT_LIMIT = 4000000000LL;   // clock cycles (about 2 s)

constexpr uint32_t OFF_B = STAGES * A_STAGE_BYTES;
constexpr uint32_t OFF_RAW = OFF_B + STAGES * B_STAGE_BYTES;
constexpr uint32_t OFF_BAR = OFF_RAW + RAW * RAW_BYTES;
constexpr int NBARS = 2 * STAGES + 2 * RAW + 2 + 2 + 1;
constexpr uint32_t SMEM_BYTES = OFF_BAR + NBARS * 8 + 16;

constexpr unsigned long long DIGIT_BIAS = 0x8080808080808080ULL;
constexpr uint32_t F16_1152X2 = 0x64806480u;   // fp16 (1152, 1152)

// fp16x2 {digit of byte `b` of a, digit of byte `b` of c}: the byte placed
// under 0x64 reads as fp16 1024 + byte; subtracting 1152 gives byte - 128.
__device__ __forceinline__ uint32_t digit_pair(uint32_t a, uint32_t c, uint32_t b) {
    const uint32_t sel = b | (b << 4) | ((b + 4) << 8) | ((b + 4) << 12);
    uint32_t r = __byte_perm(a, c, sel);
    r = (r & 0x00FF00FFu) | 0x64006400u;
    uint32_t o;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(o) : "r"(r), "r"(F16_1152X2));
    return o;
}

__device__ __forceinline__ uint32_t lo32(u64 v) { return (uint32_t)v; }
__device__ __forceinline__ uint32_t hi32(u64 v) { return (uint32_t)(v >> 32); }

// ---------------------------------------------------------------------------
// prologue: L = [E | X + cE] as digit planes in the MMA's shared-memory image

struct PrologueParams {
    const u64 *E, *X, *alpha;
    int coef;
    int64_t M, K, N;
    int S_tot;     // 2K / KS
    uint8_t* Ap;
    const u64* C;  // Z = C, the base the GEMM adds its tile segments to
    u64* Z;
};

__global__ void __launch_bounds__(256) prologue_kernel(PrologueParams p) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    {
        const int64_t nv = p.M * p.N / 2;   // N is even
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        const ulonglong2* c2 = reinterpret_cast<const ulonglong2*>(p.C);
        ulonglong2* z2 = reinterpret_cast<ulonglong2*>(p.Z);
        for (int64_t i = id; i < nv; i += stride) z2[i] = __ldg(c2 + i);
    }
    const int64_t per_tile = (int64_t)p.S_tot * 256;
    const int64_t m_tiles = (p.M + BM - 1) / BM;
    if (id >= m_tiles * per_tile) return;
    const int r = id & 7, kg = (id >> 3) & 1, rg = (id >> 4) & 15;
    const int64_t kstage = (id >> 8) % p.S_tot;
    const int64_t mt = id / per_tile;
    const int64_t m = mt * BM + rg * 8 + r;
    const int64_t kv0 = kstage * KS + kg * 8;
    u64 x[8];
    if (m < p.M) {
        if (kv0 < p.K) {
            const ulonglong2* src = reinterpret_cast<const ulonglong2*>(p.E + m * p.K + kv0);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                ulonglong2 v = __ldg(src + e);
                x[2 * e] = v.x;
                x[2 * e + 1] = v.y;
            }
        } else {
            const int64_t kx = kv0 - p.K;
            const ulonglong2* sx = reinterpret_cast<const ulonglong2*>(p.X + m * p.K + kx);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                ulonglong2 v = __ldg(sx + e);
                x[2 * e] = v.x;
                x[2 * e + 1] = v.y;
            }
            if (p.coef != COEF_ZERO) {
                const u64 c = p.coef == COEF_ONE ? 1ull : p.alpha[0];
                const ulonglong2* se = reinterpret_cast<const ulonglong2*>(p.E + m * p.K + kx);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    ulonglong2 v = __ldg(se + e);
                    x[2 * e] += c * v.x;
                    x[2 * e + 1] += c * v.y;
                }
            }
        }
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = 0;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) x[e] += DIGIT_BIAS;
    uint8_t* dst = p.Ap + ((size_t)mt * p.S_tot + kstage) * A_STAGE_BYTES + rg * CORE_SBO +
                   kg * CORE_LBO + r * 16;
#pragma unroll
    for (int t = 0; t < NDIG; ++t) {
        const uint32_t b = t & 3;
        uint4 o;
        if (t < 4) {
            o.x = digit_pair(lo32(x[0]), lo32(x[1]), b);
            o.y = digit_pair(lo32(x[2]), lo32(x[3]), b);
            o.z = digit_pair(lo32(x[4]), lo32(x[5]), b);
            o.w = digit_pair(lo32(x[6]), lo32(x[7]), b);
        } else {
            o.x = digit_pair(hi32(x[0]), hi32(x[1]), b);
            o.y = digit_pair(hi32(x[2]), hi32(x[3]), b);
            o.z = digit_pair(hi32(x[4]), hi32(x[5]), b);
            o.w = digit_pair(hi32(x[6]), hi32(x[7]), b);
        }
        *reinterpret_cast<uint4*>(dst + t * A_PLANE_BYTES) = o;
    }
}

// ---------------------------------------------------------------------------
// the GEMM

struct TcParams {
    const uint8_t* Ap;
    u64* Z;
    int64_t M, K, N;
    int S_tot;       // 16-deep stages per tile (2K / 16)
    int I;           // 128-deep intervals per tile
    int64_t n_tiles;
    int64_t U;       // work units = tiles x I
};

// The work units [u0, u1) of this CTA; unit u is interval u % I of tile u / I.
struct Unit {
    int64_t tile;
    int ii;          // interval within the tile
    int nst;         // stages in this interval (8, or fewer at the end of K)
    bool flush;      // last unit of a segment: add the sums into Z
};

__device__ __forceinline__ Unit unit_of(const TcParams& p, int64_t u, int64_t u1) {
    Unit x;
    x.tile = u / p.I;
    x.ii = (int)(u % p.I);
    const int s_begin = x.ii * KD_STAGES;
    x.nst = min(KD_STAGES, p.S_tot - s_begin);
    x.flush = (u + 1 == u1) || (x.ii == p.I - 1);
    return x;
}

__device__ __forceinline__ void red_add_u64(u64* p, u64 v) {
    asm volatile("red.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void record_timeout(volatile int* abort_flag) {
    *abort_flag = 1;
    atomicExch(&g_tc_timeout, 1u);
}

__global__ void __launch_bounds__(NTHREADS, 1)
ring_gemm_tc_kernel(const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmF,
                    TcParams p) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;
    uint8_t* sB = smem + OFF_B;
    uint8_t* sRaw = smem + OFF_RAW;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + OFF_BAR);
    uint64_t* full = bars;
    uint64_t* empty = full + STAGES;
    uint64_t* rawFull = empty + STAGES;
    uint64_t* rawEmpty = rawFull + RAW;
    uint64_t* accFull = rawEmpty + RAW;
    uint64_t* accEmpty = accFull + 2;
    uint64_t* mmaDone = accEmpty + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mmaDone + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t u0 = (int64_t)blockIdx.x * p.U / gridDim.x;
    const int64_t u1 = (int64_t)(blockIdx.x + 1) * p.U / gridDim.x;
    const int nv = (int)(u1 - u0);   // intervals of this CTA

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            ptx::mbar_init(&full[s], 1 + NCONV);
            ptx::mbar_init(&empty[s], 1);
        }
        for (int r = 0; r < RAW; ++r) {
            ptx::mbar_init(&rawFull[r], 1);
            ptx::mbar_init(&rawEmpty[r], NCONV);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&accFull[b], 1);
            ptx::mbar_init(&accEmpty[b], NDRAIN);
        }
        ptx::mbar_init(mmaDone, 1);
        *abort_flag = 0;
        ptx::fence_barrier_init();
    }
    if (warp == W_APROD) {
        ptx::tmem_alloc(tmem_slot, TMEM_COLS);
        ptx::tmem_relinquish();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == W_APROD) {
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            for (int v = 0; v < nv && ok; ++v) {
                const Unit x = unit_of(p, u0 + v, u1);
                const int64_t m_tile = x.tile / p.n_tiles;
                const uint8_t* src = p.Ap + ((size_t)m_tile * p.S_tot + x.ii * KD_STAGES) * A_STAGE_BYTES;
                for (int j = 0; j < x.nst; ++j, ++it) {
                    const int s = it % STAGES;
                    if (!ptx::mbar_wait(&empty[s], ((it / STAGES) & 1) ^ 1, abort_flag, WAIT_LIMIT)) {
                        record_timeout(abort_flag);
                        ok = false;
                        break;
                    }
                    ptx::mbar_arrive_expect_tx(&full[s], A_STAGE_BYTES);
                    ptx::bulk_g2s(sA + s * A_STAGE_BYTES, src + (size_t)j * A_STAGE_BYTES, A_STAGE_BYTES,
                                  &full[s]);
                }
            }
            // copies still in flight (only possible after a timeout) must land
            // before the CTA's shared memory is released
            for (int j = max(0, it - STAGES); j < it; ++j)
                ptx::mbar_wait(&full[j % STAGES], (j / STAGES) & 1, abort_flag, WAIT_LIMIT);
        }
    } else if (warp == W_BPROD) {
        if (lane == 0) {
            ptx::prefetch_tmap(&tmB);
            ptx::prefetch_tmap(&tmF);
            int it = 0;
            bool ok = true;
            for (int v = 0; v < nv && ok; ++v) {
                const Unit x = unit_of(p, u0 + v, u1);
                const int n0 = (int)(x.tile % p.n_tiles) * ND;
                for (int j = 0; j < x.nst; ++j, ++it) {
                    const int r = it % RAW;
                    if (!ptx::mbar_wait(&rawEmpty[r], ((it / RAW) & 1) ^ 1, abort_flag, WAIT_LIMIT)) {
                        record_timeout(abort_flag);
                        ok = false;
                        break;
                    }
                    ptx::mbar_arrive_expect_tx(&rawFull[r], RAW_BYTES);
                    const int64_t kv0 = (int64_t)(x.ii * KD_STAGES + j) * KS;
                    if (kv0 < p.K)
                        ptx::tma_load_2d(sRaw + r * RAW_BYTES, &tmB, n0, (int)kv0, &rawFull[r]);
                    else
                        ptx::tma_load_2d(sRaw + r * RAW_BYTES, &tmF, n0, (int)(kv0 - p.K), &rawFull[r]);
                }
            }
            for (int j = max(0, it - RAW); j < it; ++j)
                ptx::mbar_wait(&rawFull[j % RAW], (j / RAW) & 1, abort_flag, WAIT_LIMIT);
        }
    } else if (warp >= W_CONV0 && warp < W_CONV0 + 4) {
        const int cw = warp - W_CONV0;
        const int n8 = lane & 7, half = (lane >> 3) & 1, kg = lane >> 4;
        const int ncol = cw * 8 + n8;               // column within the tile
        const int krow = kg * 8 + half * 4;         // first of 4 K rows
        int total = 0;
        for (int v = 0; v < nv; ++v) total += unit_of(p, u0 + v, u1).nst;
        for (int it = 0; it < total; ++it) {
            const int r = it % RAW;
            if (!ptx::mbar_wait(&rawFull[r], (it / RAW) & 1, abort_flag, WAIT_LIMIT)) {
                record_timeout(abort_flag);
                break;
            }
            const u64* raw = reinterpret_cast<const u64*>(sRaw + r * RAW_BYTES);
            u64 x[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) x[e] = raw[(krow + e) * ND + ncol] + DIGIT_BIAS;
            // the next TMA write into this slot is an async-proxy access: order
            // these generic-proxy reads before it (without this fence the TMA
            // overwrote tiles still being read, measured on GB300)
            ptx::fence_proxy_async_smem();
            ptx::mbar_arrive(&rawEmpty[r]);
            const int s = it % STAGES;
            if (!ptx::mbar_wait(&empty[s], ((it / STAGES) & 1) ^ 1, abort_flag, WAIT_LIMIT)) {
                record_timeout(abort_flag);
                break;
            }
            uint8_t* dst = sB + s * B_STAGE_BYTES + cw * CORE_SBO + kg * CORE_LBO + n8 * 16 + half * 8;
#pragma unroll
            for (int t = 0; t < NDIG; ++t) {
                const uint32_t b = t & 3;
                uint2 o;
                if (t < 4) {
                    o.x = digit_pair(lo32(x[0]), lo32(x[1]), b);
                    o.y = digit_pair(lo32(x[2]), lo32(x[3]), b);
                } else {
                    o.x = digit_pair(hi32(x[0]), hi32(x[1]), b);
                    o.y = digit_pair(hi32(x[2]), hi32(x[3]), b);
                }
                // stacked row t * 32 + ncol lies in 8-row group 4t + cw
                *reinterpret_cast<uint2*>(dst + t * 4 * CORE_SBO) = o;
            }
            ptx::fence_proxy_async_smem();
            ptx::mbar_arrive(&full[s]);
        }
    } else if (warp == W_MMA) {
        if (lane == 0) {
            const uint32_t aBase = ptx::smem_u32(sA), bBase = ptx::smem_u32(sB);
            bool ok = true;
            int it = 0;
            for (int v = 0; v < nv && ok; ++v) {
                const Unit x = unit_of(p, u0 + v, u1);
                const int set = v & 1;
                if (!ptx::mbar_wait(&accEmpty[set], ((v >> 1) & 1) ^ 1, abort_flag, WAIT_LIMIT)) {
                    record_timeout(abort_flag);
                    break;
                }
                ptx::tc_fence_after();
                for (int j = 0; j < x.nst; ++j, ++it) {
                    const int s = it % STAGES;
                    if (!ptx::mbar_wait(&full[s], (it / STAGES) & 1, abort_flag, WAIT_LIMIT)) {
                        record_timeout(abort_flag);
                        ok = false;
                        break;
                    }
                    ptx::tc_fence_after();
                    const uint64_t bdesc =
                        ptx::smem_desc_kmajor(bBase + s * B_STAGE_BYTES, CORE_LBO, CORE_SBO);
#pragma unroll
                    for (int i = 0; i < NDIG; ++i) {
                        const uint64_t adesc = ptx::smem_desc_kmajor(
                            aBase + s * A_STAGE_BYTES + i * A_PLANE_BYTES, CORE_LBO, CORE_SBO);
                        const uint32_t idesc = ptx::idesc_f16_f32(BM, (NDIG - i) * ND);
                        ptx::mma_f16(tmem + set * (NDIG * ND) + i * ND, adesc, bdesc, idesc,
                                     (j == 0 && i == 0) ? 0u : 1u);
                    }
                    ptx::mma_commit(&empty[s]);
                }
                ptx::mma_commit(&accFull[set]);
            }
            // all MMAs of this CTA complete before TMEM is released
            ptx::mma_commit(mmaDone);
            ptx::mbar_wait(mmaDone, 0, abort_flag, WAIT_LIMIT);
        }
    } else {
        // drain warps: TMEM lane quadrant = warp % 4
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        u64 sum[ND];
#pragma unroll
        for (int c = 0; c < ND; ++c) sum[c] = 0;
        for (int v = 0; v < nv; ++v) {
            const Unit x = unit_of(p, u0 + v, u1);
            const int set = v & 1;
            bool got = ptx::mbar_wait(&accFull[set], (v >> 1) & 1, abort_flag, WAIT_LIMIT);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) record_timeout(abort_flag);
                break;
            }
            ptx::tc_fence_after();
            const uint32_t base = tmem + ((uint32_t)(quad * 32) << 16) + set * (NDIG * ND);
#pragma unroll
            for (int t = 0; t < NDIG; ++t) {
                uint32_t f[32];
                ptx::tmem_ld32(base + t * ND, f);
                ptx::tmem_wait_ld();
                if (t == NDIG - 1) {
                    ptx::tc_fence_before();
                    ptx::mbar_arrive(&accEmpty[set]);
                }
#pragma unroll
                for (int c = 0; c < ND; ++c) {
                    const long long d = __float2int_rn(__uint_as_float(f[c]));
                    sum[c] += (u64)d << (8 * t);
                }
            }
            if (x.flush) {
                const int64_t m = (x.tile / p.n_tiles) * BM + row;
                const int64_t n0 = (x.tile % p.n_tiles) * ND;
                if (m < p.M) {
                    u64* zrow = p.Z + m * p.N + n0;
                    const int64_t rem = p.N - n0;
                    const int ncols = rem < ND ? (int)rem : ND;
#pragma unroll
                    for (int c = 0; c < ND; ++c)
                        if (c < ncols) red_add_u64(zrow + c, sum[c]);
                }
#pragma unroll
                for (int c = 0; c < ND; ++c) sum[c] = 0;
            }
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == W_APROD) ptx::tmem_dealloc(tmem, TMEM_COLS);
}

// ---------------------------------------------------------------------------
// host side

struct Plan {
    int64_t m_tiles, n_tiles;
    int S_tot, I;
    int64_t U;
    size_t ap_bytes;
};

Plan make_plan(int64_t M, int64_t K, int64_t N) {
    Plan pl{};
    pl.m_tiles = (M + BM - 1) / BM;
    pl.n_tiles = (N + ND - 1) / ND;
    pl.S_tot = (int)(2 * K / KS);
    pl.I = (pl.S_tot + KD_STAGES - 1) / KD_STAGES;
    pl.U = pl.m_tiles * pl.n_tiles * pl.I;
    pl.ap_bytes = (size_t)pl.m_tiles * pl.S_tot * A_STAGE_BYTES;
    return pl;
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 148;
    return n;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D map over a K x N row-major u64 matrix, box of 16 rows x 32 columns
bool make_map(CUtensorMap* map, const u64* base, int64_t rows, int64_t cols) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 8};
    cuuint32_t box[2] = {(cuuint32_t)ND, (cuuint32_t)KS};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<u64*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

bool gemm_tc_eligible(int64_t M, int64_t K, int64_t N, int words) {
    if (words != 1) return false;
    if (M < 1 || N < 2 || K < 32) return false;
    if (K % 32 != 0 || N % 2 != 0) return false;
    if (K > (int64_t(1) << 30) || N > (int64_t(1) << 30)) return false;
    if ((M + BM - 1) / BM > 65535) return false;
    return 2.0 * (double)M * (double)K * (double)N >= (double)(1 << 22);
}

size_t gemm_tc_workspace(int64_t M, int64_t K, int64_t N, int words) {
    if (!gemm_tc_eligible(M, K, N, words)) return 0;
    return align256(make_plan(M, K, N).ap_bytes);
}

cudaError_t launch_gemm_tc(const GemmArgs& a, void* ws, size_t ws_bytes, cudaStream_t st) {
    if (!gemm_tc_eligible(a.M, a.K, a.N, a.words)) return cudaErrorNotSupported;
    Plan pl = make_plan(a.M, a.K, a.N);
    if (ws_bytes < align256(pl.ap_bytes) || ws == nullptr) return cudaErrorInvalidValue;
    uint8_t* Ap = static_cast<uint8_t*>(ws);

    CUtensorMap tmB, tmF;
    if (!make_map(&tmB, a.B, a.K, a.N) || !make_map(&tmF, a.F, a.K, a.N)) return cudaErrorInvalidValue;

    PrologueParams pp{a.E, a.X, a.alpha, a.coef, a.M, a.K, a.N, pl.S_tot, Ap, a.C, a.Z};
    const int64_t pth = pl.m_tiles * pl.S_tot * 256;
    prologue_kernel<<<(unsigned)((pth + 255) / 256), 256, 0, st>>>(pp);

    cudaError_t e = cudaFuncSetAttribute(ring_gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    TcParams tp{Ap, a.Z, a.M, a.K, a.N, pl.S_tot, pl.I, pl.n_tiles, pl.U};
    const int64_t grid = pl.U < sm_count() ? pl.U : sm_count();
    ring_gemm_tc_kernel<<<(unsigned)grid, NTHREADS, SMEM_BYTES, st>>>(tmB, tmF, tp);
    return cudaGetLastError();
}

int gemm_tc_launches(int64_t M, int64_t K, int64_t N, int words) {
    if (!gemm_tc_eligible(M, K, N, words)) return 0;
    return 2;
}

// Reads and clears the device flag that a bounded wait sets when it gives up.
int tc_timeout_flag(bool* set) {
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_timeout, sizeof(v)) != cudaSuccess) return -1;
    *set = v != 0;
    if (v) {
        unsigned int z = 0;
        if (cudaMemcpyToSymbol(g_tc_timeout, &z, sizeof(z)) != cudaSuccess) return -1;
    }
    return 0;
}

}  // namespace mpcl
