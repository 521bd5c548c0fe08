// gemm_tc.cu -- exact ring GEMM mod 2^64 and mod 2^128 on the fp16 tensor
// cores (tcgen05).
//
// Computes Z = C + L . R mod 2^(64 W) with L = [E | X + cE] (M x 2K) and
// R = [B ; F] (2K x N): the 2K form of Eq. (compute-z) and Eq. (compute-ztag)
// (§2.5) shared by the share and the full tag.  W = 1 is Z_2^64, W = 2 is
// Z_2^128 (two 64-bit words per element, (lo, hi)).  Each K half is padded with
// zeros to Kp, a multiple of 16, so a 16-deep stage never straddles the halves.
//
// Exactness.  sm_103a has no int8 MMA, so every ring element x is written as
// D = 8 W signed byte digits d_t in [-128, 127] with x = sum_t d_t 2^(8t) mod
// 2^(64 W) (add 0x80 to every byte mod 2^(64 W), subtract 128 from each byte;
// the carry out of the top byte vanishes mod 2^(64 W)).  Digits are exact in
// fp16, and
//     L.R mod 2^(64 W) = sum_{i+j<D} (L_i . R_j) 2^(8(i+j)),
// D (D + 1) / 2 digit products (36 for Z_2^64, 136 for Z_2^128).  A product of
// two digits is at most 2^14 in magnitude, so the diagonal accumulator
// sum_{i+j=t} L_i . R_j over Kd K values holds at most D * Kd * 2^14 = 2^24
// for Kd = 128 (W = 1) or Kd = 64 (W = 2): every partial sum is an integer
// exactly representable in fp32, so the fp32 tensor-core accumulation is
// exact.  Every Kd the accumulators are drained to integers and folded into
// wrapping sums of 64 W bits.
//
// Kernel layout (one CTA per SM; output tiles of 128 rows x ND columns):
//   * prologue_kernel writes L as D fp16 digit planes in exactly the shared
//     memory image the MMA reads (K-major, no swizzle, 8x16-byte core
//     matrices), one block per (128-row tile, 16-deep K stage), so the GEMM
//     fetches each A stage with bulk TMA copies (two halves, each with its
//     own barriers).  It also sets Z = C on the tiles computed in pieces.  The
//     GEMM is launched as a programmatic dependent of the prologue.
//   * the GEMM streams raw R tiles (16 K x ND elements) with 2-D TMA; four
//     converter warps turn each into a stacked B operand of 256 rows: rows
//     ND j .. ND j + ND - 1 hold digit plane j of the ND columns.
//   * one elected lane of the MMA warp issues, per 16-deep K step, D MMAs:
//     acc[:, ND i : 256] += L_i . [R_0 | ... | R_{D-1-i}], so that the product
//     L_i . R_j lands in TMEM column block i + j -- the diagonal it belongs to.
//     Two 256-column accumulator sets alternate, so draining one overlaps
//     MMAs into the other.
//   * four drain warps read the diagonals with tcgen05.ld, convert them to
//     integers and add d_t 2^(8t) into wrapping sums, one per output column;
//     the MMA warp hands them each unit's tile and flags through shared memory.
//   * scheduling is persistent: the (output tile, Kd-deep K interval) work
//     units are dealt to the CTAs in waves of whole tiles, the remainder split
//     evenly (see the schedule below), so a CTA may cover parts of two tiles.
//     A tile computed whole is written as C + sum; the segments of a split
//     tile are added into Z with global atomics: exact and independent of the
//     order of the additions, because addition mod 2^(64 W) is associative
//     and commutative.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "sm100_ptx.cuh"

namespace mpcl {

__device__ unsigned int g_tc_timeout = 0;

namespace {

// ---------------------------------------------------------------------------
// configuration per ring width (pipeline depths: defaults measured best)

#ifndef MPCL_TC_STAGES_W1
#define MPCL_TC_STAGES_W1 4
#endif
#ifndef MPCL_TC_RAW
#define MPCL_TC_RAW 8
#endif

template <int W> struct Cfg;
template <> struct Cfg<1> {
    static constexpr int NDIG = 8;     // digits per element
    static constexpr int ND = 32;      // output columns per tile
    static constexpr int KD = 8;       // stages per drain interval (Kd = 128)
    static constexpr int STAGES = MPCL_TC_STAGES_W1;   // operand stages in shared memory
};
template <> struct Cfg<2> {
    static constexpr int NDIG = 16;
    static constexpr int ND = 16;
    static constexpr int KD = 4;       // Kd = 64
    static constexpr int STAGES = 2;
};

// Output tiles have R = 128 rows (one per TMEM lane) or R = 64 rows.  An
// M = 64 MMA takes as long as an M = 128 one with the same N (measured on
// GB300: 588 vs 611 clock cycles for the eight Z_2^64 MMAs of a stage), so a
// 64-row tile only pays for layers with M <= 64, where it halves the A-plane
// bytes that every stage moves through shared memory.  Its accumulator
// occupies lanes 0-15 of each 32-lane TMEM quadrant q, holding rows
// 16 q .. 16 q + 15 (measured).
constexpr int BM = 128;                  // rows of the default tile
constexpr int WIDE_COLS = 128;           // output columns of a wide tile (TMEM lanes)
constexpr int KS = 16;                   // K per stage (one MMA K step)
constexpr int NSTACK = 256;              // rows of the stacked B operand (NDIG * ND)
constexpr int RAW_ONE = MPCL_TC_RAW;     // raw R tiles in flight, one-layer launches
constexpr int RAW_GROUP = 4;             // grouped launches (their layer table also takes shared memory)
template <int R> constexpr uint32_t a_plane_bytes() { return (uint32_t)R * KS * 2; }   // 4 or 2 KB
constexpr uint32_t B_STAGE_BYTES = NSTACK * KS * 2;        // 8 KB
constexpr uint32_t RAW_BYTES = 4096;                       // 16 K x (ND * W) words
constexpr uint32_t CORE_LBO = 128;       // next core matrix along K
constexpr uint32_t CORE_SBO = 256;       // next group of 8 rows
constexpr uint32_t TMEM_COLS = 512;      // two accumulator sets of 256 columns
constexpr int NUM_WARPS = 11;
constexpr int NTHREADS = NUM_WARPS * 32;
constexpr int W_APROD = 0, W_CONV0 = 1, W_MMA = 5, W_BPROD = 10;   // warps 6-9 drain
constexpr int NCONV = 128;               // converter threads
constexpr int NDRAIN = 128;              // drain threads
constexpr long long WAIT_LIMIT = 4000000000LL;   // clock cycles (about 2 s)
constexpr int MAX_STAGES = 8;
constexpr int NINFO = 4;                 // unit descriptors in flight from the MMA warp to the drain

template <int W, int G = 1, int R = BM> struct Layout {
    static constexpr int RAW = G == 1 ? RAW_ONE : RAW_GROUP;   // raw tiles in flight
    static constexpr int NBARS = 4 * MAX_STAGES + 2 * RAW + 2 + 2 + 1 + NINFO;
    static constexpr uint32_t A_PLANE = a_plane_bytes<R>();
    static constexpr uint32_t A_STAGE = Cfg<W>::NDIG * A_PLANE;
    static constexpr uint32_t OFF_B = Cfg<W>::STAGES * A_STAGE;
    static constexpr uint32_t OFF_RAW = OFF_B + Cfg<W>::STAGES * B_STAGE_BYTES;
    // epilogue staging: per drain warp 32 rows x (ND + 1) sums (one element
    // of padding per row keeps the row-wise writes and column-wise reads free
    // of bank conflicts)
    static constexpr uint32_t OFF_STG = OFF_RAW + RAW * RAW_BYTES;
    static constexpr uint32_t STG_BYTES = 4 * 32 * (Cfg<W>::ND + 1) * 8 * W;
    static constexpr uint32_t OFF_BAR = OFF_STG + STG_BYTES;
    static constexpr uint32_t OFF_INFO = (OFF_BAR + NBARS * 8 + 16 + 15) / 16 * 16;   // int4 slots
    static constexpr uint32_t SMEM = OFF_INFO + NINFO * 16;
};
static_assert(Cfg<1>::NDIG * Cfg<1>::ND == NSTACK && Cfg<2>::NDIG * Cfg<2>::ND == NSTACK, "stack");
static_assert(Layout<1>::SMEM <= 227 * 1024 && Layout<2>::SMEM <= 227 * 1024, "smem");
static_assert(Cfg<1>::STAGES <= MAX_STAGES && Cfg<2>::STAGES <= MAX_STAGES, "barrier slots");
static_assert(Layout<1>::OFF_BAR % 16 == 0 && Layout<2>::OFF_BAR % 16 == 0, "barrier alignment");
static_assert(Layout<1>::OFF_INFO % 16 == 0 && Layout<2>::OFF_INFO % 16 == 0, "int4 slots need 16-byte alignment");

constexpr unsigned long long DIGIT_BIAS = 0x8080808080808080ULL;
constexpr uint32_t F16_1152X2 = 0x64806480u;   // fp16 (1152, 1152)

// ---------------------------------------------------------------------------
// drain arithmetic
//
// The value d of diagonal t (an integer, |d| <= 2^24, converted exactly from
// its fp32 accumulator) adds d 2^(8t) to its output's wrapping sum mod
// 2^(64 W).  Z_2^64 adds the sign-extended, shifted term.  Z_2^128 takes four
// consecutive diagonals t .. t + 3 (t = 0, 4, 8, 12) of one column together:
// g = d_t + 2^8 d_(t+1) + 2^16 d_(t+2) + 2^24 d_(t+3), |g| < 2^49, by a
// mad.wide.s32 chain, which then enters the sum's four 32-bit words through one
// explicit carry chain: at 2^0 (t = 0), 2^32 (t = 4), 2^64 (t = 8, low 64 bits
// of g) or 2^96 (t = 12, low 32 bits).

__device__ __forceinline__ long long mad_wide_s32(int a, int b, long long c) {
    long long d;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// sum + g 2^(32 q) mod 2^128 for a signed 64-bit g (q = 0, 1, 2) or, q = 3,
// the low 32 bits of g at 2^96
template <int Q>
__device__ __forceinline__ u128 add_at(u128 sum, long long g) {
    u64 lo = (u64)sum, hi = (u64)(sum >> 64);
    const uint32_t gl = (uint32_t)(u64)g, gh = (uint32_t)((u64)g >> 32);
    const uint32_t sg = (uint32_t)(g >> 63);   // sign word (0 or ~0)
    uint32_t w0, w1, w2, w3;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(w0), "=r"(w1) : "l"(lo));
    asm("mov.b64 {%0, %1}, %2;" : "=r"(w2), "=r"(w3) : "l"(hi));
    if constexpr (Q == 0) {
        asm("add.cc.u32 %0, %0, %4;\n\taddc.cc.u32 %1, %1, %5;\n\taddc.cc.u32 %2, %2, %6;\n\taddc.u32 %3, %3, %6;"
            : "+r"(w0), "+r"(w1), "+r"(w2), "+r"(w3) : "r"(gl), "r"(gh), "r"(sg));
    } else if constexpr (Q == 1) {
        asm("add.cc.u32 %0, %0, %3;\n\taddc.cc.u32 %1, %1, %4;\n\taddc.u32 %2, %2, %5;"
            : "+r"(w1), "+r"(w2), "+r"(w3) : "r"(gl), "r"(gh), "r"(sg));
    } else if constexpr (Q == 2) {
        asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, %3;" : "+r"(w2), "+r"(w3) : "r"(gl), "r"(gh));
    } else {
        w3 += gl;
    }
    asm("mov.b64 %0, {%1, %2};" : "=l"(lo) : "r"(w0), "r"(w1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(hi) : "r"(w2), "r"(w3));
    return (u128)lo | ((u128)hi << 64);
}

// The drain of one accumulator set (TMEM column block t of ND columns holds
// diagonal t) into the ND sums of the warp's lanes; `release` runs once every
// load of the set has completed, after which the MMAs may reuse it.
template <int W, int ND, typename Release>
__device__ __forceinline__ void drain_set(uint32_t base, typename Elem<W>::T (&sum)[ND], Release release) {
    constexpr int NDIG = 8 * W;
    if constexpr (W == 1) {
        static_assert(ND == 32, "one diagonal per 32-column load");
#pragma unroll
        for (int t0 = 0; t0 < NDIG; ++t0) {
            uint32_t f[32];
            ptx::tmem_ld32(base + t0 * ND, f);
            ptx::tmem_wait_ld();
            if (t0 + 1 == NDIG) release();
#pragma unroll
            for (int c = 0; c < ND; ++c) {
                const long long d = __float2int_rn(__uint_as_float(f[c]));
                sum[c] += (u64)d << (8 * t0);
            }
        }
    } else {
        // diagonals t0 .. t0 + 3 of 8 columns at a time (four 8-column loads,
        // one wait): g = d_t0 + 2^8 d_(t0+1) + 2^16 d_(t0+2) + 2^24 d_(t0+3)
        static_assert(ND == 16, "two halves of 8 columns");
#pragma unroll
        for (int t0 = 0; t0 < NDIG; t0 += 4) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t f[32];   // f[8 j + c]: diagonal t0 + j, column 8 h + c
#pragma unroll
                for (int j = 0; j < 4; ++j) ptx::tmem_ld8(base + (t0 + j) * ND + 8 * h, f + 8 * j);
                ptx::tmem_wait_ld();
                if (t0 + 4 == NDIG && h == 1) release();
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    int d[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) d[j] = __float2int_rn(__uint_as_float(f[8 * j + c]));
                    typename Elem<W>::T& sc = sum[8 * h + c];
                    if (t0 < 12) {
                        long long g = mad_wide_s32(d[1], 1 << 8, (long long)d[0]);
                        g = mad_wide_s32(d[2], 1 << 16, g);
                        g = mad_wide_s32(d[3], 1 << 24, g);
                        if (t0 == 0) sc = add_at<0>(sc, g);
                        else if (t0 == 4) sc = add_at<1>(sc, g);
                        else sc = add_at<2>(sc, g);
                    } else {
                        const uint32_t g = (uint32_t)d[0] + ((uint32_t)d[1] << 8) + ((uint32_t)d[2] << 16) +
                                           ((uint32_t)d[3] << 24);
                        sc = add_at<3>(sc, (long long)g);
                    }
                }
            }
        }
    }
}

// fp16x2 digits of bytes 0-3 of a and c: h[b] = {digit of byte b of a, digit
// of byte b of c}.  One permute gathers bytes 0-1 (2-3) of both words, one
// more per pair places them under 0x64: 6 ALU operations per 8 digits.
__device__ __forceinline__ void digit_quad(uint32_t a, uint32_t c, uint32_t (&h)[4]) {
    const uint32_t lo = __byte_perm(a, c, 0x5140), hi = __byte_perm(a, c, 0x7362);
    const uint32_t r[4] = {__byte_perm(lo, 0x64646464u, 0x5140), __byte_perm(lo, 0x64646464u, 0x5342),
                           __byte_perm(hi, 0x64646464u, 0x5140), __byte_perm(hi, 0x64646464u, 0x5342)};
#pragma unroll
    for (int b = 0; b < 4; ++b) asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(h[b]) : "r"(r[b]), "r"(F16_1152X2));
}

// A ring element with the digit bias added, as 2 W 32-bit words (little
// endian): word t / 4, byte t % 4 holds the biased digit t.
template <int W> struct Biased { uint32_t w[2 * W]; };

template <int W>
__device__ __forceinline__ Biased<W> biased(const u64* e) {
    Biased<W> b;
    if constexpr (W == 1) {
        const u64 y = e[0] + DIGIT_BIAS;
        b.w[0] = (uint32_t)y;
        b.w[1] = (uint32_t)(y >> 32);
    } else {
        // one carry chain over the four 32-bit words
        asm("add.cc.u32 %0, %4, 0x80808080;\n\taddc.cc.u32 %1, %5, 0x80808080;\n\t"
            "addc.cc.u32 %2, %6, 0x80808080;\n\taddc.u32 %3, %7, 0x80808080;"
            : "=r"(b.w[0]), "=r"(b.w[1]), "=r"(b.w[2]), "=r"(b.w[3])
            : "r"((uint32_t)e[0]), "r"((uint32_t)(e[0] >> 32)), "r"((uint32_t)e[1]), "r"((uint32_t)(e[1] >> 32)));
    }
    return b;
}


// The NDIG fp16 digit planes of 8 consecutive K values (biased words b[0..7]):
// 16 bytes per plane (8 digits), plane t at dst + t * stride.
template <int W>
__device__ __forceinline__ void store_planes8(const Biased<W> (&b)[8], uint8_t* dst, uint32_t stride) {
#pragma unroll
    for (int wi = 0; wi < 2 * W; ++wi) {
        uint32_t h[4][4];   // [value pair][byte]
#pragma unroll
        for (int pr = 0; pr < 4; ++pr) digit_quad(b[2 * pr].w[wi], b[2 * pr + 1].w[wi], h[pr]);
#pragma unroll
        for (int byte = 0; byte < 4; ++byte)
            *reinterpret_cast<uint4*>(dst + (4 * wi + byte) * stride) =
                make_uint4(h[0][byte], h[1][byte], h[2][byte], h[3][byte]);
    }
}

// ---------------------------------------------------------------------------
// schedule
//
// The work units of a layer -- (output tile, Kd-deep K interval) pairs,
// numbered tile by tile -- are dealt to the G CTAs of the launch in waves.
// Each full wave gives every CTA c = I consecutive units (I = intervals per
// tile), i.e. exactly one whole tile: the data-parallel schedule.  The units
// left after the full waves (fewer than G I) are split evenly over the CTAs
// (stream-K), which balances layers with fewer tiles than CTAs.  A launch of
// several layers deals every layer over all CTAs in turn (CTAs move on to the
// next layer without waiting), so the CTAs running at any moment share that
// layer's operands through L2; layer l's CTA index is rotated by the units of
// the layers before it, so that small layers land on different CTAs.  Tiles
// are numbered in groups of gm row tiles, column-major inside a group, so the
// G consecutive tiles of a wave form a compact block of the output.
struct Sched {
    int64_t c;       // units per CTA in each full wave (the layer's I)
    int64_t nfull;   // full waves
    int64_t S;       // units in the full waves (nfull G c)
    int64_t L;       // units of the last, partial wave
    int G;           // CTAs
};

constexpr int GM_DEFAULT = 8;   // row tiles per swizzle group unless the launch table says otherwise

__host__ __device__ __forceinline__ Sched sched_of(int64_t U, int64_t I, int G) {
    Sched s;
    s.G = G;
    s.c = I;
    s.nfull = U / ((int64_t)G * I);
    s.S = s.nfull * G * I;
    s.L = U - s.S;
    return s;
}

// units of (rotated) CTA b
__host__ __device__ __forceinline__ int64_t cta_units(const Sched& s, int64_t b) {
    return s.nfull * s.c + ((b + 1) * s.L) / s.G - (b * s.L) / s.G;
}

// end of the range (of one CTA) that holds unit u of a layer
__host__ __device__ __forceinline__ int64_t range_end_of(const Sched& s, int64_t u) {
    if (u < s.S) return (u / s.c + 1) * s.c;
    // owner: the largest b with floor(b L / G) <= u - S
    const int64_t t = u - s.S;
    const int64_t b = ((t + 1) * s.G - 1) / s.L;
    return s.S + ((b + 1) * s.L) / s.G;
}

// tile index -> (row tile, column tile), GM row tiles per group
__host__ __device__ __forceinline__ void tile_mn(int64_t t, int64_t m_tiles, int64_t n_tiles, int64_t GM,
                                                 int64_t* m, int64_t* n) {
    const int64_t grp = t / (GM * n_tiles);
    const int64_t r = t - grp * GM * n_tiles;
    const int64_t left = m_tiles - grp * GM;
    const int64_t gm = left < GM ? left : GM;
    *n = r / gm;
    *m = grp * GM + (r - *n * gm);
}


// ---------------------------------------------------------------------------
// prologue: L = [E | X + cE] as digit planes in the MMA's shared-memory
// image, and Z = C on the tiles whose sums arrive in several pieces

struct PrologueParams {
    const u64 *E, *X, *alpha;
    int coef;
    int one_half;
    int64_t M, K, N;
    int64_t Kp;    // K rounded up to a multiple of KS
    int S_tot;     // 2 Kp / KS
    uint8_t* Ap;
    const u64* C;
    u64* Z;
    int I;                    // intervals per tile
    int64_t m_tiles, n_tiles;
    int gm;                   // row tiles per swizzle group
};

// Up to G layers per launch: block b works for the layer g with
// b_off[g] <= b < b_off[g + 1] (one block per 128-row tile and 16-deep stage).
template <int G> struct PrologueGroup {
    int count;
    int64_t b_off[G + 1];
    PrologueParams p[G];
    int grid;                 // CTAs of the GEMM launch
};

// thread `id` of `nthreads` working for one layer: digit planes of L in
// R-row tiles; output tiles of R x ND (or, WIDE, ND x WIDE_COLS) for the Z = C
// preset
template <int W, int R, bool WIDE = false>
__device__ __forceinline__ void prologue_body(const PrologueParams& p, int grid, int64_t id,
                                              int64_t nthreads) {
    constexpr int NDIG = Cfg<W>::NDIG;
    constexpr uint32_t A_STAGE = Layout<W, 1, R>::A_STAGE;
    constexpr uint32_t A_PLANE = Layout<W, 1, R>::A_PLANE;
    {
        // Z = C (0 without an addend) on split tiles: their pieces are added
        // atomically.  A tile one CTA computes whole is written by that CTA.
        // 16-byte vectors: two elements of one row for W = 1 (N is even),
        // one element for W = 2.
        // Blocks take tiles in turn; a split tile's TR x TC block is copied by
        // the 256 threads, TC W / 2 vectors per row.  (A wide tile's first
        // index counts column tiles, its second row tiles.)
        constexpr int ND = Cfg<W>::ND;
        constexpr int TR = WIDE ? ND : R, TC = WIDE ? WIDE_COLS : ND;
        constexpr int VPR = TC * W / 2;                      // 16-byte vectors per tile row
        const int64_t blk = id >> 8, nblk = nthreads >> 8;
        const int tid = (int)(id & 255);
        const ulonglong2* c2 = reinterpret_cast<const ulonglong2*>(p.C);
        ulonglong2* z2 = reinterpret_cast<ulonglong2*>(p.Z);
        const int64_t T = p.m_tiles * p.n_tiles;
        const Sched sc = sched_of(T * p.I, p.I, grid);
        for (int64_t t = blk; t < T; t += nblk) {
            const int64_t u = t * p.I;
            if (u + p.I <= range_end_of(sc, u)) continue;   // whole: written by its CTA
            int64_t ta, tb;
            tile_mn(t, p.m_tiles, p.n_tiles, p.gm, &ta, &tb);
            const int64_t mt = WIDE ? tb : ta, nt = WIDE ? ta : tb;
            for (int q = tid; q < TR * VPR; q += 256) {
                const int r = q / VPR, j = q - r * VPR;
                const int64_t m = mt * TR + r;
                const int64_t n = nt * TC + (int64_t)j * 2 / W;
                if (m >= p.M || n >= p.N) continue;
                const int64_t i = (m * p.N + n) * W / 2;     // vector index
                z2[i] = c2 ? __ldg(c2 + i) : make_ulonglong2(0, 0);
            }
        }
    }
    // 2 R threads per (tile, stage): thread = (8-row group rg, K half kg, row r)
    const int64_t per_tile = (int64_t)p.S_tot * 2 * R;
    const int64_t m_tiles = (p.M + R - 1) / R;
    if (id >= m_tiles * per_tile) return;
    const int r = id & 7, kg = (id >> 3) & 1, rg = (int)((id >> 4) % (R / 8));
    const int64_t kstage = (id / (2 * R)) % p.S_tot;
    const int64_t mt = id / per_tile;
    const int64_t m = mt * R + rg * 8 + r;
    const int64_t kp0 = kstage * KS + kg * 8;      // index in [0, 2 Kp)
    const bool first_half = !p.one_half && kp0 < p.Kp;
    const int64_t kk = (first_half || p.one_half) ? kp0 : kp0 - p.Kp;   // K index of the 8 values
    u64 x[8 * W];
#pragma unroll
    for (int e = 0; e < 8 * W; ++e) x[e] = 0;
    if (m < p.M && kk < p.K) {
        const u64* base = (first_half ? p.E : p.X) + (m * p.K + kk) * W;
        const u64* ebase = p.E + (m * p.K + kk) * W;
        const bool whole = kk + 8 <= p.K && (((m * p.K + kk) * W) & 1) == 0;
        if (whole) {
            const ulonglong2* src = reinterpret_cast<const ulonglong2*>(base);
#pragma unroll
            for (int e = 0; e < 4 * W; ++e) {
                ulonglong2 v = __ldg(src + e);
                x[2 * e] = v.x;
                x[2 * e + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int e = 0; e < 8; ++e)
                if (kk + e < p.K) {
#pragma unroll
                    for (int h = 0; h < W; ++h) x[W * e + h] = __ldg(base + W * e + h);
                }
        }
        if (!first_half && p.coef != COEF_ZERO) {
            if constexpr (W == 1) {
                const u64 c = p.coef == COEF_ONE ? 1ull : p.alpha[0];
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if (kk + e < p.K) x[e] += c * __ldg(ebase + e);
            } else {
                const u128 c = p.coef == COEF_ONE ? (u128)1 : ((u128)p.alpha[0] | ((u128)p.alpha[1] << 64));
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    if (kk + e >= p.K) continue;
                    const u128 ev = (u128)__ldg(ebase + 2 * e) | ((u128)__ldg(ebase + 2 * e + 1) << 64);
                    const u128 xv = ((u128)x[2 * e] | ((u128)x[2 * e + 1] << 64)) + c * ev;
                    x[2 * e] = (u64)xv;
                    x[2 * e + 1] = (u64)(xv >> 64);
                }
            }
        }
    }
    Biased<W> b[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) b[e] = biased<W>(x + W * e);
    uint8_t* dst = p.Ap + ((size_t)mt * p.S_tot + kstage) * A_STAGE + rg * CORE_SBO + kg * CORE_LBO + r * 16;
    store_planes8<W>(b, dst, A_PLANE);
}

template <int W, int G, int R, bool WIDE = false>
__global__ void __launch_bounds__(256) prologue_kernel(const __grid_constant__ PrologueGroup<G> g) {
    // the GEMM may be scheduled now: it waits for this grid before reading
    ptx::grid_dep_launch();
    // launched as a dependent of the kernel before it on the stream
    ptx::grid_dep_wait();
    int gi = 0;
    if constexpr (G > 1) {
        // last layer whose first block is at or before this one
        int lo = 0, hi = g.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (g.b_off[mid] <= (int64_t)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        gi = lo;
    }
    const int64_t lb = (int64_t)blockIdx.x - g.b_off[gi];
    const int64_t nb = g.b_off[gi + 1] - g.b_off[gi];
    prologue_body<W, R, WIDE>(g.p[gi], g.grid, lb * 256 + threadIdx.x, nb * 256);
}

// ---------------------------------------------------------------------------
// the GEMM

struct TcParams {
    const uint8_t* Ap;
    u64* Z;
    const u64* C;    // addend (NULL: none), read by CTAs that write a whole tile
    int one_half;
    int64_t M, K, N;
    int64_t Kp;      // padded K half
    int S_tot;       // 16-deep stages per tile (2 Kp / 16)
    int I;           // Kd-deep intervals per tile
    int KD;          // stages per interval
    int ND;          // columns per tile
    int64_t m_tiles, n_tiles;
    int64_t U;       // work units = tiles x I
    int gm;          // row tiles per swizzle group
    int64_t rot;     // rotation of the CTA index for this layer
};

// Up to G layers per launch, each dealt over all CTAs in turn (see the
// schedule above).  The tensor maps live in the kernel's parameter space
// (__grid_constant__), as for a single layer.
template <int G> struct TcGroup {
    CUtensorMap tmB[G];
    CUtensorMap tmF[G];
    TcParams p[G];
    int count;
    int grid;        // CTAs of the launch
};

// Unit u (local to its layer) is interval u % I of tile u / I.
struct Unit {
    int64_t mt, nt;  // row tile, column tile
    int ii;          // interval within the tile
    int nst;         // stages in this interval (KD, or fewer at the end of K)
    bool flush;      // last unit of a segment: the sums go to Z
};

// Walks the units of one CTA in order.  Divisions happen only where one of
// the CTA's ranges of consecutive units starts; inside a range the position
// (layer, tile in swizzled order, interval) advances incrementally.
template <int G> struct Walker {
    const TcParams* P;                 // the launch's layers (a copy in shared memory)
    const int count, grid;
    const int cta;
    int gi = -1;
    int vl = 0, nvl = 0;               // units of this CTA in layer gi: taken, total (< 2^31)
    int left = 0, bp = 0;              // units left in the current range; rotated CTA index
    int64_t u = 0;                     // unit index within the layer
    int64_t nfull = 0, L = 0;          // layer gi's schedule: full waves, units of the last wave
    int ii = 0, m_in = 0, gm = 1;      // tile and swizzle counters (tile counts < 2^31)
    int mt = 0, nt = 0, grp = 0;
    // the current layer's parameters, read from the parameter space only when
    // the layer changes
    int cI = 1, cKD = 1, cS = 1, cGM = 1;
    int cNT = 1, cMT = 1;

    __device__ __forceinline__ Walker(const TcParams* P_, int count_, int grid_, int cta_)
        : P(P_), count(count_), grid(grid_), cta(cta_) {
        advance_layer();
    }

    // the next layer in which this CTA has units (or past the last layer)
    __device__ __forceinline__ void advance_layer() {
        while (++gi < count) {
            const TcParams& p = P[gi];
            const Sched sc = sched_of(p.U, p.I, grid);
            bp = (int)((cta + p.rot) % grid);
            nvl = (int)cta_units(sc, bp);
            vl = 0;
            left = 0;
            if (nvl > 0) {
                nfull = sc.nfull;
                L = sc.L;
                cI = p.I;
                cKD = p.KD;
                cS = p.S_tot;
                cGM = p.gm;
                cNT = (int)p.n_tiles;
                cMT = (int)p.m_tiles;
                return;
            }
        }
    }

    __device__ __forceinline__ Unit next() {
        if (vl == nvl) advance_layer();
        if (left == 0) {
            const int64_t G_ = grid;
            const int64_t full = nfull * cI;
            int64_t len;
            if (vl < full) {
                u = ((vl / cI) * G_ + bp) * cI;
                len = cI;
            } else {
                const int64_t a = (bp * L) / G_, e = ((bp + 1) * L) / G_;
                u = nfull * G_ * cI + a;
                len = e - a;
            }
            left = (int)len - 1;
            const int64_t GM = cGM;
            const int64_t tile = u / cI;
            ii = (int)(u - tile * cI);
            grp = (int)(tile / (GM * cNT));
            const int64_t r = tile - grp * GM * cNT;
            const int lft = cMT - grp * cGM;
            gm = lft < cGM ? lft : cGM;
            nt = (int)(r / gm);
            m_in = (int)(r - (int64_t)nt * gm);
            mt = grp * cGM + m_in;
        } else {
            ++u;
            --left;
            if (++ii == cI) {
                ii = 0;
                if (++m_in == gm) {
                    m_in = 0;
                    if (++nt == cNT) {
                        nt = 0;
                        ++grp;
                        const int lft = cMT - grp * cGM;
                        gm = lft < cGM ? lft : cGM;
                    }
                }
                mt = grp * cGM + m_in;
            }
        }
        ++vl;
        Unit x;
        x.mt = mt;
        x.nt = nt;
        x.ii = ii;
        x.nst = min(cKD, cS - x.ii * cKD);
        x.flush = (left == 0) || (x.ii == cI - 1);
        return x;
    }
};

// One layer per launch: the same dealing without the layer bookkeeping (the
// layer's parameters stay in registers; measured faster on small-K layers).
template <> struct Walker<1> {
    const int cta;
    static constexpr int gi = 0;
    Sched s;
    int64_t v = 0, left = 0, u = 0;
    int ii = 0, m_in = 0, gm = 1;
    int64_t mt = 0, nt = 0, grp = 0;
    int cI = 1, cKD = 1, cS = 1, cGM = 1;
    int64_t cNT = 1, cMT = 1;

    __device__ __forceinline__ Walker(const TcParams* P, int count, int grid, int cta_) : cta(cta_) {
        (void)count;
        const TcParams& p = P[0];
        s = sched_of(p.U, p.I, grid);
        cI = p.I;
        cKD = p.KD;
        cS = p.S_tot;
        cGM = p.gm;
        cNT = p.n_tiles;
        cMT = p.m_tiles;
    }

    __device__ __forceinline__ Unit next() {
        if (left == 0) {
            const int64_t full = s.nfull * s.c;
            int64_t len;
            if (v < full) {
                u = ((v / s.c) * s.G + cta) * s.c;
                len = s.c;
            } else {
                const int64_t a = (cta * s.L) / s.G, e = ((cta + 1) * s.L) / s.G;
                u = s.S + a;
                len = e - a;
            }
            left = len - 1;
            const int64_t GM = cGM;
            const int64_t tile = u / cI;
            ii = (int)(u - tile * cI);
            grp = tile / (GM * cNT);
            const int64_t r = tile - grp * GM * cNT;
            const int64_t lft = cMT - grp * GM;
            gm = (int)(lft < GM ? lft : GM);
            nt = r / gm;
            m_in = (int)(r - nt * gm);
            mt = grp * GM + m_in;
        } else {
            ++u;
            --left;
            if (++ii == cI) {
                ii = 0;
                if (++m_in == gm) {
                    m_in = 0;
                    if (++nt == cNT) {
                        nt = 0;
                        ++grp;
                        const int64_t lft = cMT - grp * cGM;
                        gm = (int)(lft < cGM ? lft : cGM);
                    }
                }
                mt = grp * cGM + m_in;
            }
        }
        ++v;
        Unit x;
        x.mt = mt;
        x.nt = nt;
        x.ii = ii;
        x.nst = min(cKD, cS - x.ii * cKD);
        x.flush = (left == 0) || (x.ii == cI - 1);
        return x;
    }
};

// units of CTA `cta` over all layers of the launch
__device__ __forceinline__ int64_t cta_total(const TcParams* P, int count, int grid, int64_t cta) {
    int64_t n = 0;
    for (int l = 0; l < count; ++l) n += cta_units(sched_of(P[l].U, P[l].I, grid), (cta + P[l].rot) % grid);
    return n;
}

__device__ __forceinline__ void record_timeout(volatile int* abort_flag) {
    *abort_flag = 1;
    atomicExch(&g_tc_timeout, 1u);
}

template <int W, int G, int R>
__global__ void __launch_bounds__(NTHREADS, 1) ring_gemm_tc_kernel(const __grid_constant__ TcGroup<G> g) {
    using Lay = Layout<W, G, R>;
    constexpr int NDIG = Cfg<W>::NDIG, ND = Cfg<W>::ND, STAGES = Cfg<W>::STAGES;
    constexpr uint32_t A_STAGE = Lay::A_STAGE;
    constexpr uint32_t A_PLANE = Lay::A_PLANE;
    constexpr uint32_t A_HALF = A_STAGE / 2;
    constexpr int RAW = Lay::RAW;
    using Sum = typename Elem<W>::T;

    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;
    uint8_t* sB = smem + Lay::OFF_B;
    uint8_t* sRaw = smem + Lay::OFF_RAW;
    uint8_t* sStg = smem + Lay::OFF_STG;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Lay::OFF_BAR);
    uint64_t* full = bars;
    uint64_t* empty = full + MAX_STAGES;
    // an A stage arrives and is released in two halves (planes 0 .. D/2 - 1 and
    // D/2 .. D - 1): full / emptyLo for the first half (with the B planes on
    // full), fullHi / empty for the second (empty also releases the B planes)
    uint64_t* fullHi = empty + MAX_STAGES;
    uint64_t* emptyLo = fullHi + MAX_STAGES;
    uint64_t* rawFull = emptyLo + MAX_STAGES;
    uint64_t* rawEmpty = rawFull + RAW;
    uint64_t* accFull = rawEmpty + RAW;
    uint64_t* accEmpty = accFull + 2;
    uint64_t* mmaDone = accEmpty + 2;
    uint64_t* infoFull = mmaDone + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(infoFull + NINFO);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    // the MMA warp hands each unit's (row tile, column tile, interval, flush |
    // layer << 1) to the drain warps through NINFO slots
    int4* info = reinterpret_cast<int4*>(smem + Lay::OFF_INFO);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t cta = blockIdx.x;
    // the layers' parameters, copied once into shared memory: the roles read
    // them at every unit, and shared-memory loads are cheap where dynamically
    // indexed parameter-space loads are not
    // (a one-layer launch reads its parameters straight from the parameter space)
    __shared__ TcParams sp[G > 1 ? G : 1];
    if constexpr (G > 1) {
        static_assert(sizeof(TcParams) % 8 == 0, "TcParams is copied as 64-bit words");
        const uint64_t* src = reinterpret_cast<const uint64_t*>(&g.p[0]);
        uint64_t* dst = reinterpret_cast<uint64_t*>(sp);
        const int nw = g.count * (int)(sizeof(TcParams) / 8);
        for (int i = threadIdx.x; i < nw; i += NTHREADS) dst[i] = src[i];
    }
    const int count = g.count, grid = g.grid;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            ptx::mbar_init(&full[s], 1 + NCONV / 32);
            ptx::mbar_init(&empty[s], 1);
            ptx::mbar_init(&fullHi[s], 1);
            ptx::mbar_init(&emptyLo[s], 1);
        }
        for (int r = 0; r < RAW; ++r) {
            ptx::mbar_init(&rawFull[r], 1);
            ptx::mbar_init(&rawEmpty[r], NCONV / 32);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&accFull[b], 1);
            ptx::mbar_init(&accEmpty[b], NDRAIN / 32);
        }
        ptx::mbar_init(mmaDone, 1);
        for (int i = 0; i < NINFO; ++i) ptx::mbar_init(&infoFull[i], 1);
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
    // Launched as a programmatic dependent of the prologue: the set-up above
    // (barriers, TMEM, the parameter copy) overlaps the prologue's tail; its
    // digit planes and the pre-set Z are read only after this wait.
    ptx::grid_dep_wait();
    const int64_t nv = G == 1 ? cta_units(sched_of(g.p[0].U, g.p[0].I, grid), cta)
                              : cta_total(sp, count, grid, cta);   // units of this CTA

    // The producer and MMA roles run as whole warps (waits included), with one
    // elected lane issuing the copies, MMAs and commits.
    if (warp == W_APROD) {
        int it = 0;
        bool ok = true;
        Walker<G> wk(G == 1 ? &g.p[0] : sp, count, grid, (int)cta);
        for (int64_t v = 0; v < nv && ok; ++v) {
            const Unit x = wk.next();
            const TcParams& p = G == 1 ? g.p[0] : sp[wk.gi];
            const int64_t m_tile = x.mt;
            const uint8_t* src = p.Ap + ((size_t)m_tile * p.S_tot + (size_t)x.ii * p.KD) * A_STAGE;
            for (int j = 0; j < x.nst; ++j, ++it) {
                const int s = it % STAGES;
                const uint32_t par = ((it / STAGES) & 1) ^ 1;
                // first half once the MMAs that read the slot's first half are done
                bool free_ = ptx::mbar_wait(&emptyLo[s], par, abort_flag, WAIT_LIMIT);
                if (!__all_sync(0xffffffffu, free_)) {
                    if (lane == 0) record_timeout(abort_flag);
                    ok = false;
                    break;
                }
                uint32_t leader = ptx::elect_one();
                ptx::mbar_arrive_expect_tx_if(leader, &full[s], A_HALF);
                ptx::bulk_g2s_if(leader, sA + s * A_STAGE, src + (size_t)j * A_STAGE, A_HALF, &full[s]);
                free_ = ptx::mbar_wait(&empty[s], par, abort_flag, WAIT_LIMIT);
                if (!__all_sync(0xffffffffu, free_)) {
                    if (lane == 0) record_timeout(abort_flag);
                    ok = false;
                    break;
                }
                leader = ptx::elect_one();
                ptx::mbar_arrive_expect_tx_if(leader, &fullHi[s], A_HALF);
                ptx::bulk_g2s_if(leader, sA + s * A_STAGE + A_HALF, src + (size_t)j * A_STAGE + A_HALF, A_HALF,
                                 &fullHi[s]);
            }
        }
        // copies still in flight (only possible after a timeout) must land
        // before the CTA's shared memory is released
        for (int j = max(0, it - STAGES); j < it; ++j) {
            ptx::mbar_wait(&full[j % STAGES], (j / STAGES) & 1, abort_flag, WAIT_LIMIT);
            ptx::mbar_wait(&fullHi[j % STAGES], (j / STAGES) & 1, abort_flag, WAIT_LIMIT);
        }
    } else if (warp == W_BPROD) {
        int it = 0;
        bool ok = true;
        Walker<G> wk(G == 1 ? &g.p[0] : sp, count, grid, (int)cta);
        int prefetched = -1;
        for (int64_t v = 0; v < nv && ok; ++v) {
            const Unit x = wk.next();
            const TcParams& p = G == 1 ? g.p[0] : sp[wk.gi];
            const CUtensorMap* tmB = &g.tmB[wk.gi];
            const CUtensorMap* tmF = &g.tmF[wk.gi];
            if (prefetched != wk.gi) {
                if (lane == 0) {
                    ptx::prefetch_tmap(tmB);
                    ptx::prefetch_tmap(tmF);
                }
                prefetched = wk.gi;
            }
            // x coordinate in 64-bit words (ND W words per tile)
            const int x0 = (int)x.nt * ND * W;
            for (int j = 0; j < x.nst; ++j, ++it) {
                const int r = it % RAW;
                const bool free_ = ptx::mbar_wait(&rawEmpty[r], ((it / RAW) & 1) ^ 1, abort_flag, WAIT_LIMIT);
                if (!__all_sync(0xffffffffu, free_)) {
                    if (lane == 0) record_timeout(abort_flag);
                    ok = false;
                    break;
                }
                const uint32_t leader = ptx::elect_one();
                ptx::mbar_arrive_expect_tx_if(leader, &rawFull[r], RAW_BYTES);
                // rows at or beyond K inside a padded half arrive zero-filled
                const int64_t kp0 = (int64_t)(x.ii * p.KD + j) * KS;
                const bool second = p.one_half || kp0 >= p.Kp;
                const CUtensorMap* tm = second ? tmF : tmB;
                const int y = (int)(p.one_half || kp0 < p.Kp ? kp0 : kp0 - p.Kp);
                ptx::tma_load_2d_if(leader, sRaw + r * RAW_BYTES, tm, x0, y, &rawFull[r]);
            }
        }
        for (int j = max(0, it - RAW); j < it; ++j)
            ptx::mbar_wait(&rawFull[j % RAW], (j / RAW) & 1, abort_flag, WAIT_LIMIT);
    } else if (warp >= W_CONV0 && warp < W_CONV0 + 4) {
        // Each converter thread turns 4 consecutive K values of one column into
        // digit planes (half a core-matrix row per plane): all 8 planes for
        // Z_2^64, 8 of the 16 planes for Z_2^128.  The barriers count one
        // arrival per converter warp.
        const int ct = threadIdx.x - W_CONV0 * 32;   // 0..127
        int ncol, krow, tlo, boff;
        if constexpr (W == 1) {
            // A raw tile row is 256 bytes, so every row starts at bank 0: the
            // four (kg, half) lane groups of a warp read four different
            // 8-column segments (the warp's segment rotated by 2 kg + half),
            // which keeps each raw read at two wavefronts; the plane writes
            // stay at two.
            const int cw = ct >> 5, n8 = lane & 7, half = (lane >> 3) & 1, kg = lane >> 4;
            ncol = ((cw + 2 * kg + half) & 3) * 8 + n8;
            krow = kg * 8 + half * 4;
            tlo = 0;
            boff = (ncol >> 3) * CORE_SBO + kg * CORE_LBO + (ncol & 7) * 16 + half * 8;
        } else {
            const int n = ct & 15, kq = (ct >> 4) & 3, dh = ct >> 6;
            ncol = n;
            krow = kq * 4;
            tlo = dh * 8;
            boff = (n >> 3) * CORE_SBO + (kq >> 1) * CORE_LBO + (n & 7) * 16 + (kq & 1) * 8;
        }
        constexpr int TPT = W == 1 ? NDIG : NDIG / 2;   // planes written per thread
        int total = 0;
        {
            Walker<G> wk(G == 1 ? &g.p[0] : sp, count, grid, (int)cta);
            for (int64_t v = 0; v < nv; ++v) total += wk.next().nst;
        }
        for (int it = 0; it < total; ++it) {
            const int r = it % RAW;
            // warp-uniform decisions: the warp arrives as one
            if (!__all_sync(0xffffffffu, ptx::mbar_wait(&rawFull[r], (it / RAW) & 1, abort_flag, WAIT_LIMIT))) {
                if (lane == 0) record_timeout(abort_flag);
                break;
            }
            const u64* raw = reinterpret_cast<const u64*>(sRaw + r * RAW_BYTES);
            u64 e[4 * W];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if constexpr (W == 1) {
                    e[q] = raw[(krow + q) * ND + ncol];
                } else {
                    // one 16-byte load per element: a warp reads two whole rows
                    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(raw + ((krow + q) * ND + ncol) * 2);
                    e[2 * q] = v.x;
                    e[2 * q + 1] = v.y;
                }
            }
            Biased<W> b[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) b[q] = biased<W>(e + q * W);
            const int s = it % STAGES;
            if (!__all_sync(0xffffffffu,
                            ptx::mbar_wait(&empty[s], ((it / STAGES) & 1) ^ 1, abort_flag, WAIT_LIMIT))) {
                if (lane == 0) record_timeout(abort_flag);
                break;
            }
            uint8_t* dst = sB + s * B_STAGE_BYTES + boff;
            // word wi of the 4 values gives planes 4 wi .. 4 wi + 3
#pragma unroll
            for (int wq = 0; wq < TPT / 4; ++wq) {
                const int wi = tlo / 4 + wq;
                uint32_t h01[4], h23[4];
                digit_quad(b[0].w[wi], b[1].w[wi], h01);
                digit_quad(b[2].w[wi], b[3].w[wi], h23);
#pragma unroll
                for (int byte = 0; byte < 4; ++byte) {
                    const int t = 4 * wi + byte;
                    // stacked row t * ND + ncol: 8-row group (t * ND) / 8 + ncol / 8
                    *reinterpret_cast<uint2*>(dst + t * (ND / 8) * CORE_SBO) = make_uint2(h01[byte], h23[byte]);
                }
            }
            // each thread orders its plane writes before the MMAs and its raw
            // reads before the next TMA write into the raw slot (both async
            // proxy; without ordering the reads the TMA overwrote tiles still
            // being read, measured on GB300); the warp then arrives once on each
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                ptx::mbar_arrive(&full[s]);
                ptx::mbar_arrive(&rawEmpty[r]);
            }
        }
    } else if (warp == W_MMA) {
        // The whole warp runs the loop (waits included) and one elected lane
        // issues the MMAs and commits.
        const uint32_t aBase = ptx::smem_u32(sA), bBase = ptx::smem_u32(sB);
        bool ok = true;
        int it = 0;
        Walker<G> wk(G == 1 ? &g.p[0] : sp, count, grid, (int)cta);
        for (int64_t v = 0; v < nv && ok; ++v) {
            const Unit x = wk.next();
            const int set = (int)(v & 1);
            const bool got = ptx::mbar_wait(&accEmpty[set], (int)((v >> 1) & 1) ^ 1, abort_flag, WAIT_LIMIT);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) record_timeout(abort_flag);
                break;
            }
            ptx::tc_fence_after();
            // slot v % NINFO last held unit v - NINFO, which the drain finished
            // before it released the accumulator set this wait was for
            if (lane == 0) {
                info[v % NINFO] = make_int4((int)x.mt, (int)x.nt, x.ii, (int)x.flush | (wk.gi << 1));
                ptx::mbar_arrive(&infoFull[v % NINFO]);
            }
            for (int j = 0; j < x.nst; ++j, ++it) {
                const int s = it % STAGES;
                const bool ready = ptx::mbar_wait(&full[s], (it / STAGES) & 1, abort_flag, WAIT_LIMIT);
                if (!__all_sync(0xffffffffu, ready)) {
                    if (lane == 0) record_timeout(abort_flag);
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                uint32_t leader = ptx::elect_one();
                const uint64_t bdesc = ptx::smem_desc_kmajor(bBase + s * B_STAGE_BYTES, CORE_LBO, CORE_SBO);
#pragma unroll
                for (int i = 0; i < NDIG / 2; ++i) {
                    const uint64_t adesc =
                        ptx::smem_desc_kmajor(aBase + s * A_STAGE + i * A_PLANE, CORE_LBO, CORE_SBO);
                    const uint32_t idesc = ptx::idesc_f16_f32(R, (NDIG - i) * ND);
                    ptx::mma_f16_if(leader, tmem + set * NSTACK + i * ND, adesc, bdesc, idesc,
                                    (j == 0 && i == 0) ? 0u : 1u);
                }
                ptx::mma_commit_if(leader, &emptyLo[s]);
                const bool hi = ptx::mbar_wait(&fullHi[s], (it / STAGES) & 1, abort_flag, WAIT_LIMIT);
                if (!__all_sync(0xffffffffu, hi)) {
                    if (lane == 0) record_timeout(abort_flag);
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                leader = ptx::elect_one();
#pragma unroll
                for (int i = NDIG / 2; i < NDIG; ++i) {
                    const uint64_t adesc =
                        ptx::smem_desc_kmajor(aBase + s * A_STAGE + i * A_PLANE, CORE_LBO, CORE_SBO);
                    const uint32_t idesc = ptx::idesc_f16_f32(R, (NDIG - i) * ND);
                    ptx::mma_f16_if(leader, tmem + set * NSTACK + i * ND, adesc, bdesc, idesc, 1u);
                }
                ptx::mma_commit_if(leader, &empty[s]);
            }
            if (ok) ptx::mma_commit_if(ptx::elect_one(), &accFull[set]);
        }
        // all MMAs of this CTA complete before TMEM is released
        ptx::mma_commit_if(ptx::elect_one(), mmaDone);
        ptx::mbar_wait(mmaDone, 0, abort_flag, WAIT_LIMIT);
    } else {
        // drain warps: TMEM lane quadrant = warp % 4
        const int quad = warp & 3;
        Sum sum[ND];
#pragma unroll
        for (int c = 0; c < ND; ++c) sum[c] = 0;
        int seg_ii = -1;   // first interval of the current segment
        for (int64_t v = 0; v < nv; ++v) {
            const bool have = ptx::mbar_wait(&infoFull[v % NINFO], (int)((v / NINFO) & 1), abort_flag, WAIT_LIMIT);
            if (!__all_sync(0xffffffffu, have)) {
                if (lane == 0) record_timeout(abort_flag);
                break;
            }
            const int4 u = info[v % NINFO];
            const int x_ii = u.z;
            const bool x_flush = (u.w & 1) != 0;
            const TcParams& p = G == 1 ? g.p[0] : sp[u.w >> 1];
            const int set = (int)(v & 1);
            bool got = ptx::mbar_wait(&accFull[set], (int)((v >> 1) & 1), abort_flag, WAIT_LIMIT);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) record_timeout(abort_flag);
                break;
            }
            ptx::tc_fence_after();
            const uint32_t base = tmem + ((uint32_t)(quad * 32) << 16) + set * NSTACK;
            drain_set<W, ND>(base, sum, [&] {
                // every lane's loads are complete (wait::ld); the warp
                // releases the accumulator set as one arrival
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&accEmpty[set]);
            });
            if (seg_ii < 0) seg_ii = x_ii;
            if (x_flush) {
                // a tile computed whole by this segment is written as C + sum;
                // pieces of a split tile are added to Z (set to C by the prologue)
                const bool whole = seg_ii == 0 && x_ii == p.I - 1;
                seg_ii = -1;
                // The warp's rows x ND sums go through shared memory so that
                // the global accesses run along rows: lane = column (W = 1), or
                // two rows of 16 columns per instruction (W = 2).  Lane l of
                // quadrant q holds row q RPW + l of the tile; with 64-row tiles
                // only lanes 0-15 hold rows (RPW = 16).
                constexpr int RPW = R / 4;      // tile rows per drain warp
                Sum* stg = reinterpret_cast<Sum*>(sStg) + quad * 32 * (ND + 1);
                __syncwarp();
#pragma unroll
                for (int c = 0; c < ND; ++c) stg[lane * (ND + 1) + c] = sum[c];
                __syncwarp();
                constexpr int RPI = 32 / ND;     // rows per instruction
                constexpr int NIT = RPW / RPI;
                constexpr int BATCH = NIT;        // addend loads in flight together
                const int rr = lane / ND, cc = lane % ND;
                const int64_t n = (int64_t)u.y * ND + cc;
                const int64_t mb = (int64_t)u.x * R + quad * RPW;
#pragma unroll
                for (int i0 = 0; i0 < NIT; i0 += BATCH) {
                    // a batch of addend loads first, then its stores or atomic adds
                    Sum cv[BATCH];
#pragma unroll
                    for (int i = 0; i < BATCH; ++i) {
                        const int64_t m = mb + (i0 + i) * RPI + rr;
                        cv[i] = (whole && p.C && m < p.M && n < p.N) ? ldg_elem<W>(p.C, m * p.N + n) : (Sum)0;
                    }
#pragma unroll
                    for (int i = 0; i < BATCH; ++i) {
                        const int r = (i0 + i) * RPI + rr;
                        const int64_t m = mb + r;
                        if (m < p.M && n < p.N) {
                            const Sum v = stg[r * (ND + 1) + cc];
                            const int64_t e = m * p.N + n;
                            if (whole) {
                                st_elem<W>(p.Z, e, cv[i] + v);
                            } else {
                                if constexpr (W == 1) red_add_u64(p.Z + e, v);
                                else atomic_add_u128(p.Z + 2 * e, v);
                            }
                        }
                    }
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
static_assert(Layout<1>::SMEM <= 227 * 1024 && Layout<2>::SMEM <= 227 * 1024, "smem with staging");
static_assert(Layout<1, 1, 64>::SMEM <= 227 * 1024 && Layout<2, 1, 64>::SMEM <= 227 * 1024, "smem, 64-row tiles");

// ---------------------------------------------------------------------------
// the wide tile: Z^T = R^T . L^T for layers with few rows
//
// An MMA costs the same for 64 or 128 rows (above), so a layer with M rows
// well below 128 wastes most of a row tile.  The wide tile exchanges the
// roles of the operands: the 128 TMEM lanes hold WIDE_COLS = 128 output
// COLUMNS, and the stacked operand holds ND of the layer's rows (ND = 32 for
// Z_2^64, 16 for Z_2^128).  Per 16-deep K step, MMA i multiplies digit plane i
// of R^T = [B ; F]^T (128 columns x 16 K, formed in shared memory by the
// converter warps from raw 16 x 128 tiles of [B ; F]) by the first
// (D - i) ND rows of the stack of L's digit planes (rows j ND + m hold digit j
// of row m; the prologue writes them with ND-row tiles, which is exactly this
// stacked layout, and the L producer copies one 8 KB stage at a time), into
// TMEM column block i.  The product R_i . L_j again lands in block i + j, so
// the MMA shapes, the exactness bound, the schedule and the drain's
// arithmetic are those of the row tiles; a drain thread now holds the ND rows
// of one output column, and its stores run along the rows (lane = column).
// Work unit: (column tile, row tile of ND rows, Kd interval); the walker's
// first index counts column tiles.

template <int W, int G = 1> struct WideLayout {
    static constexpr int STAGES = Cfg<W>::STAGES;            // operand stages: 4 (W = 1) or 2 (W = 2)
    static constexpr int RAW = W == 1 ? 3 : 2;               // raw [B ; F] tiles in flight
    static constexpr uint32_t A_PLANE = a_plane_bytes<WIDE_COLS>();      // 4 KB
    static constexpr uint32_t A_STAGE = Cfg<W>::NDIG * A_PLANE;
    static constexpr uint32_t RAW_TILE = KS * WIDE_COLS * 8 * W;        // 16 or 32 KB
    static constexpr int NBARS = 2 * MAX_STAGES + 2 * RAW + 2 + 2 + 1 + NINFO;
    static constexpr uint32_t OFF_B = STAGES * A_STAGE;
    static constexpr uint32_t OFF_RAW = OFF_B + STAGES * B_STAGE_BYTES;
    static constexpr uint32_t OFF_BAR = OFF_RAW + RAW * RAW_TILE;
    static constexpr uint32_t OFF_INFO = (OFF_BAR + NBARS * 8 + 16 + 15) / 16 * 16;
    static constexpr uint32_t SMEM = OFF_INFO + NINFO * 16;
};
static_assert(Cfg<1>::NDIG * Cfg<1>::ND * KS * 2 == B_STAGE_BYTES && Cfg<2>::NDIG * Cfg<2>::ND * KS * 2 == B_STAGE_BYTES,
              "a stage of the L stack is one B stage");
static_assert(WideLayout<1>::OFF_BAR % 16 == 0 && WideLayout<2>::OFF_BAR % 16 == 0, "barrier alignment");
static_assert(WideLayout<1>::OFF_INFO % 16 == 0 && WideLayout<2>::OFF_INFO % 16 == 0, "int4 slots");

template <int W, int G>
__global__ void __launch_bounds__(NTHREADS, 1) ring_gemm_tc_wide_kernel(const __grid_constant__ TcGroup<G> g) {
    using Lay = WideLayout<W, G>;
    constexpr int NDIG = Cfg<W>::NDIG, ND = Cfg<W>::ND, STAGES = Lay::STAGES, RAW = Lay::RAW;
    constexpr uint32_t A_STAGE = Lay::A_STAGE, A_PLANE = Lay::A_PLANE, RAW_TILE = Lay::RAW_TILE;
    using Sum = typename Elem<W>::T;

    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;                       // R^T digit planes (converter warps)
    uint8_t* sB = smem + Lay::OFF_B;          // L stack (copies of the prologue's planes)
    uint8_t* sRaw = smem + Lay::OFF_RAW;      // raw 16 x 128 tiles of [B ; F] (TMA)
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Lay::OFF_BAR);
    uint64_t* full = bars;                    // stage ready: the stack copy and the 4 converter warps
    uint64_t* empty = full + MAX_STAGES;      // stage free: its MMAs are done
    uint64_t* rawFull = empty + MAX_STAGES;
    uint64_t* rawEmpty = rawFull + RAW;
    uint64_t* accFull = rawEmpty + RAW;
    uint64_t* accEmpty = accFull + 2;
    uint64_t* mmaDone = accEmpty + 2;
    uint64_t* infoFull = mmaDone + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(infoFull + NINFO);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    int4* info = reinterpret_cast<int4*>(smem + Lay::OFF_INFO);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t cta = blockIdx.x;
    __shared__ TcParams sp[G > 1 ? G : 1];
    if constexpr (G > 1) {
        const uint64_t* src = reinterpret_cast<const uint64_t*>(&g.p[0]);
        uint64_t* dst = reinterpret_cast<uint64_t*>(sp);
        const int nw = g.count * (int)(sizeof(TcParams) / 8);
        for (int i = threadIdx.x; i < nw; i += NTHREADS) dst[i] = src[i];
    }
    const int count = g.count, grid = g.grid;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            ptx::mbar_init(&full[s], 1 + NCONV / 32);
            ptx::mbar_init(&empty[s], 1);
        }
        for (int r = 0; r < RAW; ++r) {
            ptx::mbar_init(&rawFull[r], 1);
            ptx::mbar_init(&rawEmpty[r], NCONV / 32);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&accFull[b], 1);
            ptx::mbar_init(&accEmpty[b], NDRAIN / 32);
        }
        ptx::mbar_init(mmaDone, 1);
        for (int i = 0; i < NINFO; ++i) ptx::mbar_init(&infoFull[i], 1);
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
    ptx::grid_dep_wait();   // the prologue's planes and pre-set Z are read below
    const int64_t nv = G == 1 ? cta_units(sched_of(g.p[0].U, g.p[0].I, grid), cta)
                              : cta_total(sp, count, grid, cta);

    if (warp == W_APROD) {
        // the L stack: one 8 KB stage per 16-deep K step
        int it = 0;
        bool ok = true;
        Walker<G> wk(G == 1 ? &g.p[0] : sp, count, grid, (int)cta);
        for (int64_t v = 0; v < nv && ok; ++v) {
            const Unit x = wk.next();
            const TcParams& p = G == 1 ? g.p[0] : sp[wk.gi];
            const uint8_t* src = p.Ap + ((size_t)x.nt * p.S_tot + (size_t)x.ii * p.KD) * B_STAGE_BYTES;
            for (int j = 0; j < x.nst; ++j, ++it) {
                const int s = it % STAGES;
                const bool free_ = ptx::mbar_wait(&empty[s], ((it / STAGES) & 1) ^ 1, abort_flag, WAIT_LIMIT);
                if (!__all_sync(0xffffffffu, free_)) {
                    if (lane == 0) record_timeout(abort_flag);
                    ok = false;
                    break;
                }
                const uint32_t leader = ptx::elect_one();
                ptx::mbar_arrive_expect_tx_if(leader, &full[s], B_STAGE_BYTES);
                ptx::bulk_g2s_if(leader, sB + s * B_STAGE_BYTES, src + (size_t)j * B_STAGE_BYTES, B_STAGE_BYTES,
                                 &full[s]);
            }
        }
        // copies still in flight (only after a timeout) land before the CTA exits
        for (int j = max(0, it - STAGES); j < it; ++j)
            ptx::mbar_wait(&full[j % STAGES], (j / STAGES) & 1, abort_flag, WAIT_LIMIT);
    } else if (warp == W_BPROD) {
        int it = 0;
        bool ok = true;
        Walker<G> wk(G == 1 ? &g.p[0] : sp, count, grid, (int)cta);
        int prefetched = -1;
        for (int64_t v = 0; v < nv && ok; ++v) {
            const Unit x = wk.next();
            const TcParams& p = G == 1 ? g.p[0] : sp[wk.gi];
            const CUtensorMap* tmB = &g.tmB[wk.gi];
            const CUtensorMap* tmF = &g.tmF[wk.gi];
            if (prefetched != wk.gi) {
                if (lane == 0) {
                    ptx::prefetch_tmap(tmB);
                    ptx::prefetch_tmap(tmF);
                }
                prefetched = wk.gi;
            }
            const int x0 = (int)x.mt * WIDE_COLS * W;   // first word of the column tile
            for (int j = 0; j < x.nst; ++j, ++it) {
                const int r = it % RAW;
                const bool free_ = ptx::mbar_wait(&rawEmpty[r], ((it / RAW) & 1) ^ 1, abort_flag, WAIT_LIMIT);
                if (!__all_sync(0xffffffffu, free_)) {
                    if (lane == 0) record_timeout(abort_flag);
                    ok = false;
                    break;
                }
                const uint32_t leader = ptx::elect_one();
                ptx::mbar_arrive_expect_tx_if(leader, &rawFull[r], RAW_TILE);
                const int64_t kp0 = (int64_t)(x.ii * p.KD + j) * KS;
                const bool second = p.one_half || kp0 >= p.Kp;
                const CUtensorMap* tm = second ? tmF : tmB;
                const int y = (int)(p.one_half || kp0 < p.Kp ? kp0 : kp0 - p.Kp);
                ptx::tma_load_2d_if(leader, sRaw + r * RAW_TILE, tm, x0, y, &rawFull[r]);
            }
        }
        for (int j = max(0, it - RAW); j < it; ++j)
            ptx::mbar_wait(&rawFull[j % RAW], (j / RAW) & 1, abort_flag, WAIT_LIMIT);
    } else if (warp >= W_CONV0 && warp < W_CONV0 + 4) {
        // converter thread n (0..127) forms row n of every R^T plane: the 16 K
        // values of output column n, digit by digit, in two 8-K halves
        const int n = threadIdx.x - W_CONV0 * 32;
        int total = 0;
        {
            Walker<G> wk(G == 1 ? &g.p[0] : sp, count, grid, (int)cta);
            for (int64_t v = 0; v < nv; ++v) total += wk.next().nst;
        }
        const uint32_t boff = (uint32_t)(n >> 3) * CORE_SBO + (uint32_t)(n & 7) * 16;
        for (int it = 0; it < total; ++it) {
            const int r = it % RAW;
            if (!__all_sync(0xffffffffu, ptx::mbar_wait(&rawFull[r], (it / RAW) & 1, abort_flag, WAIT_LIMIT))) {
                if (lane == 0) record_timeout(abort_flag);
                break;
            }
            // raw tile: 16 rows (K) of 128 W words; lanes read consecutive columns
            const u64* raw = reinterpret_cast<const u64*>(sRaw + r * RAW_TILE);
            u64 e[16 * W];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                if constexpr (W == 1) {
                    e[k] = raw[k * WIDE_COLS + n];
                } else {
                    const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(raw + (k * WIDE_COLS + n) * 2);
                    e[2 * k] = v.x;
                    e[2 * k + 1] = v.y;
                }
            }
            const int s = it % STAGES;
            if (!__all_sync(0xffffffffu,
                            ptx::mbar_wait(&empty[s], ((it / STAGES) & 1) ^ 1, abort_flag, WAIT_LIMIT))) {
                if (lane == 0) record_timeout(abort_flag);
                break;
            }
            uint8_t* dst = sA + s * A_STAGE + boff;
#pragma unroll
            for (int kh = 0; kh < 2; ++kh) {
                Biased<W> b[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) b[q] = biased<W>(e + (kh * 8 + q) * W);
                store_planes8<W>(b, dst + kh * CORE_LBO, A_PLANE);
            }
            // each thread orders its plane writes before the MMAs and its raw
            // reads before the next TMA write into the raw slot (async proxy);
            // the warp then arrives once on each
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                ptx::mbar_arrive(&full[s]);
                ptx::mbar_arrive(&rawEmpty[r]);
            }
        }
    } else if (warp == W_MMA) {
        const uint32_t aBase = ptx::smem_u32(sA), bBase = ptx::smem_u32(sB);
        bool ok = true;
        int it = 0;
        Walker<G> wk(G == 1 ? &g.p[0] : sp, count, grid, (int)cta);
        for (int64_t v = 0; v < nv && ok; ++v) {
            const Unit x = wk.next();
            const int set = (int)(v & 1);
            const bool got = ptx::mbar_wait(&accEmpty[set], (int)((v >> 1) & 1) ^ 1, abort_flag, WAIT_LIMIT);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) record_timeout(abort_flag);
                break;
            }
            ptx::tc_fence_after();
            if (lane == 0) {
                info[v % NINFO] = make_int4((int)x.mt, (int)x.nt, x.ii, (int)x.flush | (wk.gi << 1));
                ptx::mbar_arrive(&infoFull[v % NINFO]);
            }
            for (int j = 0; j < x.nst; ++j, ++it) {
                const int s = it % STAGES;
                const bool ready = ptx::mbar_wait(&full[s], (it / STAGES) & 1, abort_flag, WAIT_LIMIT);
                if (!__all_sync(0xffffffffu, ready)) {
                    if (lane == 0) record_timeout(abort_flag);
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t leader = ptx::elect_one();
                const uint64_t bdesc = ptx::smem_desc_kmajor(bBase + s * B_STAGE_BYTES, CORE_LBO, CORE_SBO);
#pragma unroll
                for (int i = 0; i < NDIG; ++i) {
                    const uint64_t adesc =
                        ptx::smem_desc_kmajor(aBase + s * A_STAGE + i * A_PLANE, CORE_LBO, CORE_SBO);
                    const uint32_t idesc = ptx::idesc_f16_f32(WIDE_COLS, (NDIG - i) * ND);
                    ptx::mma_f16_if(leader, tmem + set * NSTACK + i * ND, adesc, bdesc, idesc,
                                    (j == 0 && i == 0) ? 0u : 1u);
                }
                ptx::mma_commit_if(leader, &empty[s]);
            }
            if (ok) ptx::mma_commit_if(ptx::elect_one(), &accFull[set]);
        }
        ptx::mma_commit_if(ptx::elect_one(), mmaDone);
        ptx::mbar_wait(mmaDone, 0, abort_flag, WAIT_LIMIT);
    } else {
        // drain: lane l of quadrant q holds output column 32 q + l of the tile
        // and the sums of its ND rows
        const int quad = warp & 3;
        Sum sum[ND];
#pragma unroll
        for (int c = 0; c < ND; ++c) sum[c] = 0;
        int seg_ii = -1;
        for (int64_t v = 0; v < nv; ++v) {
            const bool have = ptx::mbar_wait(&infoFull[v % NINFO], (int)((v / NINFO) & 1), abort_flag, WAIT_LIMIT);
            if (!__all_sync(0xffffffffu, have)) {
                if (lane == 0) record_timeout(abort_flag);
                break;
            }
            const int4 u = info[v % NINFO];
            const int x_ii = u.z;
            const bool x_flush = (u.w & 1) != 0;
            const TcParams& p = G == 1 ? g.p[0] : sp[u.w >> 1];
            const int set = (int)(v & 1);
            const bool got = ptx::mbar_wait(&accFull[set], (int)((v >> 1) & 1), abort_flag, WAIT_LIMIT);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) record_timeout(abort_flag);
                break;
            }
            ptx::tc_fence_after();
            const uint32_t base = tmem + ((uint32_t)(quad * 32) << 16) + set * NSTACK;
            drain_set<W, ND>(base, sum, [&] {
                // every lane's loads are complete (wait::ld); the warp
                // releases the accumulator set as one arrival
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&accEmpty[set]);
            });
            if (seg_ii < 0) seg_ii = x_ii;
            if (x_flush) {
                // whole tiles store C + sum, pieces of split tiles are added
                // (Z was set to C by the prologue); for each row the warp's
                // lanes write 32 consecutive columns
                const bool whole = seg_ii == 0 && x_ii == p.I - 1;
                seg_ii = -1;
                const int64_t n = (int64_t)u.x * WIDE_COLS + quad * 32 + lane;
                const int64_t mb = (int64_t)u.y * ND;
                constexpr int BATCH = 8;
#pragma unroll
                for (int c0 = 0; c0 < ND; c0 += BATCH) {
                    Sum cv[BATCH];
#pragma unroll
                    for (int i = 0; i < BATCH; ++i) {
                        const int64_t m = mb + c0 + i;
                        cv[i] = (whole && p.C && m < p.M && n < p.N) ? ldg_elem<W>(p.C, m * p.N + n) : (Sum)0;
                    }
#pragma unroll
                    for (int i = 0; i < BATCH; ++i) {
                        const int64_t m = mb + c0 + i;
                        if (m < p.M && n < p.N) {
                            const int64_t e = m * p.N + n;
                            if (whole) {
                                st_elem<W>(p.Z, e, cv[i] + sum[c0 + i]);
                            } else {
                                if constexpr (W == 1) red_add_u64(p.Z + e, sum[c0 + i]);
                                else atomic_add_u128(p.Z + 2 * e, sum[c0 + i]);
                            }
                        }
                    }
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
// the tall tile: the left operand converted inside the GEMM
//
// Row tiles of 128 x ND as above, but L's digit planes never go through HBM:
// the c E term moves to the right operand, [E | X + cE] . [B ; F] =
// [E | X] . [B + cF ; F], so each 16-deep stage of L is one raw tile of E or X
// (128 rows x 16 K, loaded by 2-D TMA with the 128-byte swizzle so that the
// converters' row reads hit distinct banks) that the converter warps turn
// into the NDIG A planes.  The right operand R' = [B + cF ; F] is small for
// the layers this tile serves (M >> N); a prologue writes its digit planes in
// the stacked layout (per ND-column tile and stage: plane j holds rows
// j ND .. j ND + ND - 1), copied one 8 KB stage at a time.  The MMAs, the
// schedule and the drain's arithmetic are those of the 128-row tile; the
// drain stores each lane's row directly (16-byte vectors along the row).
// Stores of whole tiles are C + sum; split tiles add with atomics into Z,
// which the prologue pre-sets to C.

template <int W, int G = 1> struct TallLayout {
    static constexpr int STAGES = Cfg<W>::STAGES;
    static constexpr int RAW = W == 1 ? 3 : 2;               // raw L tiles in flight
    static constexpr uint32_t A_PLANE = a_plane_bytes<BM>();          // 4 KB
    static constexpr uint32_t A_STAGE = Cfg<W>::NDIG * A_PLANE;
    static constexpr uint32_t RAW_BOX = BM * 128;                     // 128 rows x 128 bytes
    static constexpr uint32_t RAW_TILE = RAW_BOX * W;                 // 16 K values: W boxes
    static constexpr int NBARS = 2 * MAX_STAGES + 2 * RAW + 2 + 2 + 1 + NINFO;
    static constexpr uint32_t OFF_B = STAGES * A_STAGE;
    static constexpr uint32_t OFF_RAW = OFF_B + STAGES * B_STAGE_BYTES;
    static constexpr uint32_t OFF_BAR = OFF_RAW + RAW * RAW_TILE;
    static constexpr uint32_t OFF_INFO = (OFF_BAR + NBARS * 8 + 16 + 15) / 16 * 16;
    static constexpr uint32_t SMEM = OFF_INFO + NINFO * 16;
};
static_assert(TallLayout<1>::OFF_RAW % 1024 == 0 && TallLayout<2>::OFF_RAW % 1024 == 0,
              "the 128-byte swizzle needs 1024-byte aligned raw tiles");
static_assert(TallLayout<1>::OFF_BAR % 16 == 0 && TallLayout<2>::OFF_BAR % 16 == 0, "barrier alignment");

// Prologue of the tall tile: digit planes of R' = [B + cF ; F] in the stacked
// layout, and Z = C on the tiles computed in pieces.  2 ND threads per
// (column tile, stage): thread (column nl, K half kh) converts 8 K values of
// one column (lanes read consecutive columns of a row of R').
struct PrologueRParams {
    const u64 *B, *F, *alpha;
    int coef;
    int64_t M, K, N;
    int64_t Kp;
    int S_tot;
    uint8_t* Rp;
    const u64* C;
    u64* Z;
    int I;
    int64_t m_tiles, n_tiles;
    int gm;
};

template <int G> struct PrologueRGroup {
    int count;
    int64_t b_off[G + 1];
    PrologueRParams p[G];
    int grid;
};

template <int W>
__device__ __forceinline__ void prologue_r_body(const PrologueRParams& p, int grid, int64_t id, int64_t nthreads) {
    constexpr int NDIG = Cfg<W>::NDIG, ND = Cfg<W>::ND;
    {
        // Z = C on split tiles (as the row-tile prologue does)
        constexpr int VPR = ND * W / 2;
        const int64_t blk = id >> 8, nblk = nthreads >> 8;
        const int tid = (int)(id & 255);
        const ulonglong2* c2 = reinterpret_cast<const ulonglong2*>(p.C);
        ulonglong2* z2 = reinterpret_cast<ulonglong2*>(p.Z);
        const int64_t T = p.m_tiles * p.n_tiles;
        const Sched sc = sched_of(T * p.I, p.I, grid);
        for (int64_t t = blk; t < T; t += nblk) {
            const int64_t u = t * p.I;
            if (u + p.I <= range_end_of(sc, u)) continue;
            int64_t mt, nt;
            tile_mn(t, p.m_tiles, p.n_tiles, p.gm, &mt, &nt);
            for (int q = tid; q < BM * VPR; q += 256) {
                const int r = q / VPR, j = q - r * VPR;
                const int64_t m = mt * BM + r;
                const int64_t n = nt * ND + (int64_t)j * 2 / W;
                if (m >= p.M || n >= p.N) continue;
                const int64_t i = (m * p.N + n) * W / 2;
                z2[i] = c2 ? __ldg(c2 + i) : make_ulonglong2(0, 0);
            }
        }
    }
    const int64_t per_tile = (int64_t)p.S_tot * 2 * ND;
    if (id >= p.n_tiles * per_tile) return;
    const int nl = (int)(id % ND), kh = (int)((id / ND) & 1);
    const int64_t kstage = (id / (2 * ND)) % p.S_tot;
    const int64_t nt = id / per_tile;
    const int64_t n = nt * ND + nl;
    const int64_t kp0 = kstage * KS + kh * 8;     // index in [0, 2 Kp)
    const bool first = kp0 < p.Kp;
    const int64_t kk = first ? kp0 : kp0 - p.Kp;
    using T = typename Elem<W>::T;
    T cv = 0;
    if (first && p.coef != COEF_ZERO) cv = p.coef == COEF_ONE ? (T)1 : ld_elem<W>(p.alpha, 0);
    u64 x[8 * W];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        T v = 0;
        if (n < p.N && kk + e < p.K) {
            const int64_t i = (kk + e) * p.N + n;
            v = ldg_elem<W>(first ? p.B : p.F, i);
            if (first && p.coef != COEF_ZERO) v += cv * ldg_elem<W>(p.F, i);
        }
        x[W * e] = (u64)v;
        if constexpr (W == 2) x[W * e + 1] = (u64)(v >> 64);
    }
    Biased<W> b[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) b[e] = biased<W>(x + W * e);
    uint8_t* dst = p.Rp + ((size_t)nt * p.S_tot + kstage) * B_STAGE_BYTES + (nl >> 3) * CORE_SBO + kh * CORE_LBO +
                   (nl & 7) * 16;
    store_planes8<W>(b, dst, ND * KS * 2);
}

template <int W, int G>
__global__ void __launch_bounds__(256) prologue_r_kernel(const __grid_constant__ PrologueRGroup<G> g) {
    ptx::grid_dep_launch();
    ptx::grid_dep_wait();
    int gi = 0;
    if constexpr (G > 1) {
        int lo = 0, hi = g.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (g.b_off[mid] <= (int64_t)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        gi = lo;
    }
    const int64_t lb = (int64_t)blockIdx.x - g.b_off[gi];
    const int64_t nb = g.b_off[gi + 1] - g.b_off[gi];
    prologue_r_body<W>(g.p[gi], g.grid, lb * 256 + threadIdx.x, nb * 256);
}

// byte offset of K value k (0..15) of row m in a raw tile of the tall kernel:
// W boxes of 128 rows x 128 bytes (8 W K values), 16-byte chunks swizzled by
// the row (TMA's 128-byte swizzle: chunk c of row m sits at chunk c ^ (m % 8))
template <int W>
__device__ __forceinline__ uint32_t raw_l_offset(int m, int k) {
    constexpr int PER_BOX = 8 * (W == 1 ? 2 : 1);          // K values per 128-byte box row
    const int box = k / PER_BOX, kb = k % PER_BOX;
    const int chunk = (kb * 8 * W) / 16, within = (kb * 8 * W) % 16;
    return (uint32_t)box * TallLayout<W>::RAW_BOX + (uint32_t)m * 128 + (uint32_t)((chunk ^ (m & 7)) * 16 + within);
}

template <int W, int G>
__global__ void __launch_bounds__(NTHREADS, 1) ring_gemm_tc_tall_kernel(const __grid_constant__ TcGroup<G> g) {
    using Lay = TallLayout<W, G>;
    constexpr int NDIG = Cfg<W>::NDIG, ND = Cfg<W>::ND, STAGES = Lay::STAGES, RAW = Lay::RAW;
    constexpr uint32_t A_STAGE = Lay::A_STAGE, A_PLANE = Lay::A_PLANE, RAW_TILE = Lay::RAW_TILE;
    using Sum = typename Elem<W>::T;

    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sA = smem;                       // L digit planes (converter warps)
    uint8_t* sB = smem + Lay::OFF_B;          // R' stack (copies of the prologue's planes)
    uint8_t* sRaw = smem + Lay::OFF_RAW;      // raw 128 x 16 tiles of E or X (TMA, swizzled)
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Lay::OFF_BAR);
    uint64_t* full = bars;
    uint64_t* empty = full + MAX_STAGES;
    uint64_t* rawFull = empty + MAX_STAGES;
    uint64_t* rawEmpty = rawFull + RAW;
    uint64_t* accFull = rawEmpty + RAW;
    uint64_t* accEmpty = accFull + 2;
    uint64_t* mmaDone = accEmpty + 2;
    uint64_t* infoFull = mmaDone + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(infoFull + NINFO);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    int4* info = reinterpret_cast<int4*>(smem + Lay::OFF_INFO);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t cta = blockIdx.x;
    __shared__ TcParams sp[G > 1 ? G : 1];
    if constexpr (G > 1) {
        const uint64_t* src = reinterpret_cast<const uint64_t*>(&g.p[0]);
        uint64_t* dst = reinterpret_cast<uint64_t*>(sp);
        const int nw = g.count * (int)(sizeof(TcParams) / 8);
        for (int i = threadIdx.x; i < nw; i += NTHREADS) dst[i] = src[i];
    }
    const int count = g.count, grid = g.grid;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            ptx::mbar_init(&full[s], 1 + NCONV / 32);
            ptx::mbar_init(&empty[s], 1);
        }
        for (int r = 0; r < RAW; ++r) {
            ptx::mbar_init(&rawFull[r], 1);
            ptx::mbar_init(&rawEmpty[r], NCONV / 32);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&accFull[b], 1);
            ptx::mbar_init(&accEmpty[b], NDRAIN / 32);
        }
        ptx::mbar_init(mmaDone, 1);
        for (int i = 0; i < NINFO; ++i) ptx::mbar_init(&infoFull[i], 1);
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
    ptx::grid_dep_wait();
    const int64_t nv = G == 1 ? cta_units(sched_of(g.p[0].U, g.p[0].I, grid), cta)
                              : cta_total(sp, count, grid, cta);

    if (warp == W_APROD) {
        // the R' stack: one 8 KB stage per 16-deep K step
        int it = 0;
        bool ok = true;
        Walker<G> wk(G == 1 ? &g.p[0] : sp, count, grid, (int)cta);
        for (int64_t v = 0; v < nv && ok; ++v) {
            const Unit x = wk.next();
            const TcParams& p = G == 1 ? g.p[0] : sp[wk.gi];
            const uint8_t* src = p.Ap + ((size_t)x.nt * p.S_tot + (size_t)x.ii * p.KD) * B_STAGE_BYTES;
            for (int j = 0; j < x.nst; ++j, ++it) {
                const int s = it % STAGES;
                const bool free_ = ptx::mbar_wait(&empty[s], ((it / STAGES) & 1) ^ 1, abort_flag, WAIT_LIMIT);
                if (!__all_sync(0xffffffffu, free_)) {
                    if (lane == 0) record_timeout(abort_flag);
                    ok = false;
                    break;
                }
                const uint32_t leader = ptx::elect_one();
                ptx::mbar_arrive_expect_tx_if(leader, &full[s], B_STAGE_BYTES);
                ptx::bulk_g2s_if(leader, sB + s * B_STAGE_BYTES, src + (size_t)j * B_STAGE_BYTES, B_STAGE_BYTES,
                                 &full[s]);
            }
        }
        for (int j = max(0, it - STAGES); j < it; ++j)
            ptx::mbar_wait(&full[j % STAGES], (j / STAGES) & 1, abort_flag, WAIT_LIMIT);
    } else if (warp == W_BPROD) {
        // raw tiles of L = [E | X]: map tmB over E, tmF over X
        int it = 0;
        bool ok = true;
        Walker<G> wk(G == 1 ? &g.p[0] : sp, count, grid, (int)cta);
        int prefetched = -1;
        for (int64_t v = 0; v < nv && ok; ++v) {
            const Unit x = wk.next();
            const TcParams& p = G == 1 ? g.p[0] : sp[wk.gi];
            const CUtensorMap* tmE = &g.tmB[wk.gi];
            const CUtensorMap* tmX = &g.tmF[wk.gi];
            if (prefetched != wk.gi) {
                if (lane == 0) {
                    ptx::prefetch_tmap(tmE);
                    ptx::prefetch_tmap(tmX);
                }
                prefetched = wk.gi;
            }
            const int y = (int)x.mt * BM;               // first row of the row tile
            for (int j = 0; j < x.nst; ++j, ++it) {
                const int r = it % RAW;
                const bool free_ = ptx::mbar_wait(&rawEmpty[r], ((it / RAW) & 1) ^ 1, abort_flag, WAIT_LIMIT);
                if (!__all_sync(0xffffffffu, free_)) {
                    if (lane == 0) record_timeout(abort_flag);
                    ok = false;
                    break;
                }
                const uint32_t leader = ptx::elect_one();
                ptx::mbar_arrive_expect_tx_if(leader, &rawFull[r], RAW_TILE);
                const int64_t kp0 = (int64_t)(x.ii * p.KD + j) * KS;
                const bool second = kp0 >= p.Kp;
                const CUtensorMap* tm = second ? tmX : tmE;
                const int x0 = (int)((second ? kp0 - p.Kp : kp0) * W);   // first word of the 16 K values
#pragma unroll
                for (int h = 0; h < W; ++h)
                    ptx::tma_load_2d_if(leader, sRaw + r * RAW_TILE + h * Lay::RAW_BOX, tm, x0 + 16 * h, y, &rawFull[r]);
            }
        }
        for (int j = max(0, it - RAW); j < it; ++j)
            ptx::mbar_wait(&rawFull[j % RAW], (j / RAW) & 1, abort_flag, WAIT_LIMIT);
    } else if (warp >= W_CONV0 && warp < W_CONV0 + 4) {
        // converter thread m (0..127) forms row m of every L plane
        const int m = threadIdx.x - W_CONV0 * 32;
        int total = 0;
        {
            Walker<G> wk(G == 1 ? &g.p[0] : sp, count, grid, (int)cta);
            for (int64_t v = 0; v < nv; ++v) total += wk.next().nst;
        }
        const uint32_t boff = (uint32_t)(m >> 3) * CORE_SBO + (uint32_t)(m & 7) * 16;
        for (int it = 0; it < total; ++it) {
            const int r = it % RAW;
            if (!__all_sync(0xffffffffu, ptx::mbar_wait(&rawFull[r], (it / RAW) & 1, abort_flag, WAIT_LIMIT))) {
                if (lane == 0) record_timeout(abort_flag);
                break;
            }
            const uint8_t* raw = sRaw + r * RAW_TILE;
            u64 e[16 * W];
#pragma unroll
            for (int k = 0; k < 16; k += (W == 1 ? 2 : 1)) {
                // one 16-byte chunk: two values (W = 1) or one (W = 2)
                const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(raw + raw_l_offset<W>(m, k));
                e[k * W] = v.x;
                e[k * W + 1] = v.y;
            }
            const int s = it % STAGES;
            if (!__all_sync(0xffffffffu,
                            ptx::mbar_wait(&empty[s], ((it / STAGES) & 1) ^ 1, abort_flag, WAIT_LIMIT))) {
                if (lane == 0) record_timeout(abort_flag);
                break;
            }
            uint8_t* dst = sA + s * A_STAGE + boff;
#pragma unroll
            for (int kh = 0; kh < 2; ++kh) {
                Biased<W> b[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) b[q] = biased<W>(e + (kh * 8 + q) * W);
                store_planes8<W>(b, dst + kh * CORE_LBO, A_PLANE);
            }
            // one fence orders the plane writes before the MMAs and the raw
            // reads before the next TMA write into the raw slot
            ptx::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                ptx::mbar_arrive(&full[s]);
                ptx::mbar_arrive(&rawEmpty[r]);
            }
        }
    } else if (warp == W_MMA) {
        const uint32_t aBase = ptx::smem_u32(sA), bBase = ptx::smem_u32(sB);
        bool ok = true;
        int it = 0;
        Walker<G> wk(G == 1 ? &g.p[0] : sp, count, grid, (int)cta);
        for (int64_t v = 0; v < nv && ok; ++v) {
            const Unit x = wk.next();
            const int set = (int)(v & 1);
            const bool got = ptx::mbar_wait(&accEmpty[set], (int)((v >> 1) & 1) ^ 1, abort_flag, WAIT_LIMIT);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) record_timeout(abort_flag);
                break;
            }
            ptx::tc_fence_after();
            if (lane == 0) {
                info[v % NINFO] = make_int4((int)x.mt, (int)x.nt, x.ii, (int)x.flush | (wk.gi << 1));
                ptx::mbar_arrive(&infoFull[v % NINFO]);
            }
            for (int j = 0; j < x.nst; ++j, ++it) {
                const int s = it % STAGES;
                const bool ready = ptx::mbar_wait(&full[s], (it / STAGES) & 1, abort_flag, WAIT_LIMIT);
                if (!__all_sync(0xffffffffu, ready)) {
                    if (lane == 0) record_timeout(abort_flag);
                    ok = false;
                    break;
                }
                ptx::tc_fence_after();
                const uint32_t leader = ptx::elect_one();
                const uint64_t bdesc = ptx::smem_desc_kmajor(bBase + s * B_STAGE_BYTES, CORE_LBO, CORE_SBO);
#pragma unroll
                for (int i = 0; i < NDIG; ++i) {
                    const uint64_t adesc =
                        ptx::smem_desc_kmajor(aBase + s * A_STAGE + i * A_PLANE, CORE_LBO, CORE_SBO);
                    const uint32_t idesc = ptx::idesc_f16_f32(BM, (NDIG - i) * ND);
                    ptx::mma_f16_if(leader, tmem + set * NSTACK + i * ND, adesc, bdesc, idesc,
                                    (j == 0 && i == 0) ? 0u : 1u);
                }
                ptx::mma_commit_if(leader, &empty[s]);
            }
            if (ok) ptx::mma_commit_if(ptx::elect_one(), &accFull[set]);
        }
        ptx::mma_commit_if(ptx::elect_one(), mmaDone);
        ptx::mbar_wait(mmaDone, 0, abort_flag, WAIT_LIMIT);
    } else {
        // drain: lane l of quadrant q holds row 32 q + l of the tile and its ND sums
        const int quad = warp & 3;
        Sum sum[ND];
#pragma unroll
        for (int c = 0; c < ND; ++c) sum[c] = 0;
        int seg_ii = -1;
        for (int64_t v = 0; v < nv; ++v) {
            const bool have = ptx::mbar_wait(&infoFull[v % NINFO], (int)((v / NINFO) & 1), abort_flag, WAIT_LIMIT);
            if (!__all_sync(0xffffffffu, have)) {
                if (lane == 0) record_timeout(abort_flag);
                break;
            }
            const int4 u = info[v % NINFO];
            const int x_ii = u.z;
            const bool x_flush = (u.w & 1) != 0;
            const TcParams& p = G == 1 ? g.p[0] : sp[u.w >> 1];
            const int set = (int)(v & 1);
            const bool got = ptx::mbar_wait(&accFull[set], (int)((v >> 1) & 1), abort_flag, WAIT_LIMIT);
            if (!__all_sync(0xffffffffu, got)) {
                if (lane == 0) record_timeout(abort_flag);
                break;
            }
            ptx::tc_fence_after();
            const uint32_t base = tmem + ((uint32_t)(quad * 32) << 16) + set * NSTACK;
            drain_set<W, ND>(base, sum, [&] {
                // every lane's loads are complete (wait::ld); the warp
                // releases the accumulator set as one arrival
                ptx::tc_fence_before();
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&accEmpty[set]);
            });
            if (seg_ii < 0) seg_ii = x_ii;
            if (x_flush) {
                const bool whole = seg_ii == 0 && x_ii == p.I - 1;
                seg_ii = -1;
                const int64_t m = (int64_t)u.x * BM + quad * 32 + lane;
                const int64_t n0 = (int64_t)u.y * ND;
                if (m < p.M) {
                    const int64_t e0 = m * p.N + n0;
                    if (whole && n0 + ND <= p.N) {
                        // the row's ND sums as 16-byte vectors (N is even for W = 1)
                        ulonglong2* z2 = reinterpret_cast<ulonglong2*>(p.Z + e0 * W);
                        const ulonglong2* c2 = reinterpret_cast<const ulonglong2*>(p.C + e0 * W);
                        constexpr int V = ND * W / 2;
#pragma unroll
                        for (int q = 0; q < V; ++q) {
                            const ulonglong2 cq = p.C ? __ldg(c2 + q) : make_ulonglong2(0, 0);
                            ulonglong2 o;
                            if constexpr (W == 1) {
                                o.x = cq.x + sum[2 * q];
                                o.y = cq.y + sum[2 * q + 1];
                            } else {
                                const Sum r = ((Sum)cq.x | ((Sum)cq.y << 64)) + sum[q];
                                o.x = (u64)r;
                                o.y = (u64)(r >> 64);
                            }
                            z2[q] = o;
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < ND; ++c) {
                            if (n0 + c >= p.N) break;
                            const int64_t e = e0 + c;
                            if (whole) {
                                st_elem<W>(p.Z, e, (p.C ? ldg_elem<W>(p.C, e) : (Sum)0) + sum[c]);
                            } else {
                                if constexpr (W == 1) red_add_u64(p.Z + e, sum[c]);
                                else atomic_add_u128(p.Z + 2 * e, sum[c]);
                            }
                        }
                    }
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
    int64_t m_tiles, n_tiles, Kp;
    int S_tot, I, KD, ND;
    int64_t U;
    size_t ap_bytes;
};

// The tile of a launch, from the launch table's `rows`: the wide tile when
// rows is the ring's ND (32 for Z_2^64, 16 for Z_2^128), else row tiles of
// 64 rows (rows == 64) or 128 (anything else).
bool wide_rows(int rows, int words) { return rows == (words == 1 ? Cfg<1>::ND : Cfg<2>::ND); }
// The tall tile: 128-row tiles whose left operand the GEMM converts itself.
constexpr int TALL_ROWS = TALL_TILE_ROWS;
static_assert(TALL_TILE_ROWS == -BM, "the tall tile has 128 rows");
bool tall_rows(int rows) { return rows == TALL_ROWS; }
int tile_rows(int rows) { return rows == 64 ? 64 : BM; }

// Row tiles: m_tiles x n_tiles output tiles of R x ND, digit planes of L in
// R-row tiles.  Wide tiles: m_tiles = column tiles (of WIDE_COLS columns),
// n_tiles = row tiles (of ND rows), digit planes of L in ND-row tiles.
Plan make_plan(int64_t M, int64_t K, int64_t N, int words, int one_half = 0, int rows = BM) {
    Plan pl{};
    if (tall_rows(rows)) {
        // row tiles of 128 x ND; the workspace holds the digit planes of
        // R' = [B + cF ; F] in ND-column tiles (8 KB per tile and stage)
        pl.KD = words == 1 ? Cfg<1>::KD : Cfg<2>::KD;
        pl.ND = words == 1 ? Cfg<1>::ND : Cfg<2>::ND;
        pl.m_tiles = (M + BM - 1) / BM;
        pl.n_tiles = (N + pl.ND - 1) / pl.ND;
        pl.Kp = ((K + KS - 1) / KS) * KS;
        pl.S_tot = (int)(2 * pl.Kp / KS);
        pl.I = (pl.S_tot + pl.KD - 1) / pl.KD;
        pl.U = pl.m_tiles * pl.n_tiles * pl.I;
        pl.ap_bytes = (size_t)pl.n_tiles * pl.S_tot * B_STAGE_BYTES;
        return pl;
    }
    const bool wide = wide_rows(rows, words);
    pl.KD = words == 1 ? Cfg<1>::KD : Cfg<2>::KD;
    pl.ND = words == 1 ? Cfg<1>::ND : Cfg<2>::ND;
    const int R = wide ? pl.ND : tile_rows(rows);   // rows of L per digit-plane tile
    const uint32_t a_stage = (words == 1 ? Cfg<1>::NDIG : Cfg<2>::NDIG) * (uint32_t)R * KS * 2;
    const int64_t l_tiles = (M + R - 1) / R;
    pl.m_tiles = wide ? (N + WIDE_COLS - 1) / WIDE_COLS : l_tiles;
    pl.n_tiles = wide ? l_tiles : (N + pl.ND - 1) / pl.ND;
    pl.Kp = ((K + KS - 1) / KS) * KS;
    pl.S_tot = (int)((one_half ? 1 : 2) * pl.Kp / KS);
    pl.I = (pl.S_tot + pl.KD - 1) / pl.KD;
    pl.U = pl.m_tiles * pl.n_tiles * pl.I;
    pl.ap_bytes = (size_t)l_tiles * pl.S_tot * a_stage;
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

// 2-D map over a K x N row-major matrix of `words`-word elements, viewed as
// K rows of N * words 64-bit words; box of 16 rows x (nd * words) words
bool make_map(CUtensorMap* map, const u64* base, int64_t rows, int64_t cols, int words, int nd) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)(cols * words), (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(cols * words) * 8};
    cuuint32_t box[2] = {(cuuint32_t)(nd * words), (cuuint32_t)KS};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<u64*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// 2-D map over an M x K row-major matrix of `words`-word elements for the tall
// tile's raw L tiles: box of 128 rows x 16 words (128 bytes), 128-byte swizzle
// (the K row stride, K words x 8 bytes, must be a multiple of 16 bytes)
bool make_map_l(CUtensorMap* map, const u64* base, int64_t rows, int64_t cols, int words) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)(cols * words), (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(cols * words) * 8};
    cuuint32_t box[2] = {16u, (cuuint32_t)BM};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<u64*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

constexpr int GMAX = 64;   // layers per grouped launch (kernel parameters stay below 32 KB)
static_assert(sizeof(TcGroup<GMAX>) + 64 <= 32764, "kernel parameter space");

// The dynamic shared-memory opt-in is set once per device and kernel (a host
// call that also keeps graph capture free of attribute changes after the
// first use).
// The GEMM kernel and its dynamic shared memory: row tiles of R rows, or the
// wide tile.
template <int W, int G, int R, bool WIDE> struct Gemm {
    static constexpr uint32_t SMEM = WIDE ? WideLayout<W, G>::SMEM : Layout<W, G, R>::SMEM;
    static constexpr int PR = WIDE ? Cfg<W>::ND : R;   // rows per digit-plane tile of L
    static void (*kernel())(TcGroup<G>) {
        if constexpr (WIDE) return ring_gemm_tc_wide_kernel<W, G>;
        else return ring_gemm_tc_kernel<W, G, R>;
    }
};

template <int W, int G, int R, bool WIDE = false>
cudaError_t ensure_smem_attr() {
    static bool smem_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
    if (dev >= 0 && dev < 64 && smem_set[dev]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(Gemm<W, G, R, WIDE>::kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Gemm<W, G, R, WIDE>::SMEM);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) smem_set[dev] = true;
    return cudaSuccess;
}

// Fills entry j of a group for layer `a` (digit planes at Ap; R-row tiles,
// or the wide tile).
template <int W, int G, int R, bool WIDE = false>
bool fill(TcGroup<G>& tg, PrologueGroup<G>& pg, int j, const GemmArgs& a, uint8_t* Ap, const Plan& pl) {
    constexpr int box = WIDE ? WIDE_COLS : Cfg<W>::ND;    // columns per raw tile of [B ; F]
    if (!make_map(&tg.tmF[j], a.F, a.K, a.N, W, box)) return false;
    if (a.one_half) tg.tmB[j] = tg.tmF[j];
    else if (!make_map(&tg.tmB[j], a.B, a.K, a.N, W, box)) return false;
    const int gm = a.gm > 0 ? a.gm : GM_DEFAULT;
    tg.p[j] = TcParams{Ap, a.Z, a.C, a.one_half, a.M, a.K, a.N, pl.Kp, pl.S_tot, pl.I, pl.KD, pl.ND,
                       pl.m_tiles, pl.n_tiles, pl.U, gm, 0};
    pg.p[j] = PrologueParams{a.E, a.X, a.alpha, a.coef, a.one_half, a.M, a.K, a.N, pl.Kp, pl.S_tot, Ap, a.C, a.Z,
                             pl.I, pl.m_tiles, pl.n_tiles, gm};
    // prologue blocks of 256 threads, 2 PR threads per (plane tile, stage)
    constexpr int PR = Gemm<W, G, R, WIDE>::PR;
    const int64_t l_tiles = WIDE ? pl.n_tiles : pl.m_tiles;
    pg.b_off[j + 1] = pg.b_off[j] + (l_tiles * pl.S_tot * 2 * PR + 255) / 256;
    return true;
}

template <int W, int G, int R, bool WIDE = false>
cudaError_t launch_group(TcGroup<G>& tg, PrologueGroup<G>& pg, cudaStream_t st) {
    // one CTA per SM (fewer when the launch has fewer units); each layer's
    // CTA index is rotated by the units of the layers before it
    int64_t total = 0;
    for (int j = 0; j < tg.count; ++j) total += tg.p[j].U;
    const int sms = sm_count();
    const int grid = (int)(total < sms ? (total > 0 ? total : 1) : sms);
    int64_t acc = 0;
    for (int j = 0; j < tg.count; ++j) {
        tg.p[j].rot = acc % grid;
        acc += tg.p[j].U;
    }
    tg.grid = pg.grid = grid;
    constexpr int PR = Gemm<W, G, R, WIDE>::PR;
    cudaError_t e = launch_dependent(prologue_kernel<W, G, PR, WIDE>, dim3((unsigned)pg.b_off[pg.count]), dim3(256),
                                     0, st, pg);
    if (e != cudaSuccess) return e;
    e = ensure_smem_attr<W, G, R, WIDE>();
    if (e != cudaSuccess) return e;
    // programmatic dependent launch: the GEMM's CTAs may start (and set up)
    // while the prologue finishes; they wait for it in the kernel
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = Gemm<W, G, R, WIDE>::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, Gemm<W, G, R, WIDE>::kernel(), tg);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int W, int R, bool WIDE = false>
cudaError_t launch(const GemmArgs& a, uint8_t* Ap, const Plan& pl, cudaStream_t st) {
    TcGroup<1> tg{};
    PrologueGroup<1> pg{};
    tg.count = pg.count = 1;
    pg.b_off[0] = 0;
    if (!fill<W, 1, R, WIDE>(tg, pg, 0, a, Ap, pl)) return cudaErrorInvalidValue;
    return launch_group<W, 1, R, WIDE>(tg, pg, st);
}

// One launch pair for the layers order[i0 .. i0 + cnt) (cnt <= G), R-row tiles
// or the wide tile.
template <int W, int G, int R, bool WIDE = false>
cudaError_t launch_chunk(const GemmArgs* a, uint8_t* const* Ap, const int* order, int cnt, cudaStream_t st) {
    static_assert(alignof(TcGroup<G>) >= 64, "tensor map alignment");
    auto* tg = new (std::nothrow) TcGroup<G>;
    auto* pg = new (std::nothrow) PrologueGroup<G>;
    cudaError_t e = (tg && pg) ? cudaSuccess : cudaErrorMemoryAllocation;
    if (e == cudaSuccess) {
        tg->count = pg->count = cnt;
        pg->b_off[0] = 0;
        for (int j = 0; j < cnt && e == cudaSuccess; ++j) {
            const GemmArgs& x = a[order[j]];
            const int rows = WIDE ? Cfg<W>::ND : R;
            if (!fill<W, G, R, WIDE>(*tg, *pg, j, x, Ap[order[j]], make_plan(x.M, x.K, x.N, W, x.one_half, rows)))
                e = cudaErrorInvalidValue;
        }
        if (e == cudaSuccess) e = launch_group<W, G, R, WIDE>(*tg, *pg, st);
    }
    delete tg;
    delete pg;
    return e;
}

// The tall tile: entry j of a group (R' planes at Rp).
template <int W, int G>
bool fill_tall(TcGroup<G>& tg, PrologueRGroup<G>& pg, int j, const GemmArgs& a, uint8_t* Rp, const Plan& pl) {
    if (!make_map_l(&tg.tmB[j], a.E, a.M, a.K, W)) return false;
    if (!make_map_l(&tg.tmF[j], a.X, a.M, a.K, W)) return false;
    const int gm = a.gm > 0 ? a.gm : GM_DEFAULT;
    tg.p[j] = TcParams{Rp, a.Z, a.C, 0, a.M, a.K, a.N, pl.Kp, pl.S_tot, pl.I, pl.KD, pl.ND,
                       pl.m_tiles, pl.n_tiles, pl.U, gm, 0};
    pg.p[j] = PrologueRParams{a.B, a.F, a.alpha, a.coef, a.M, a.K, a.N, pl.Kp, pl.S_tot, Rp, a.C, a.Z,
                              pl.I, pl.m_tiles, pl.n_tiles, gm};
    // blocks of 256 threads, 2 ND threads per (column tile, stage) of R'; the
    // same blocks also preset Z = C on the split tiles (32 KB each), so a layer
    // with few column tiles still gets about four blocks per SM for that copy
    const int64_t conv = (pl.n_tiles * pl.S_tot * 2 * pl.ND + 255) / 256;
    const int64_t copy = std::min<int64_t>(pl.m_tiles * pl.n_tiles, 4 * (int64_t)sm_count());
    pg.b_off[j + 1] = pg.b_off[j] + std::max(conv, copy);
    return true;
}

template <int W, int G>
cudaError_t ensure_smem_attr_tall() {
    static bool smem_set[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return cudaErrorInvalidDevice;
    if (dev >= 0 && dev < 64 && smem_set[dev]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(ring_gemm_tc_tall_kernel<W, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TallLayout<W, G>::SMEM);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) smem_set[dev] = true;
    return cudaSuccess;
}

template <int W, int G>
cudaError_t launch_group_tall(TcGroup<G>& tg, PrologueRGroup<G>& pg, cudaStream_t st) {
    int64_t total = 0;
    for (int j = 0; j < tg.count; ++j) total += tg.p[j].U;
    const int sms = sm_count();
    const int grid = (int)(total < sms ? (total > 0 ? total : 1) : sms);
    int64_t acc = 0;
    for (int j = 0; j < tg.count; ++j) {
        tg.p[j].rot = acc % grid;
        acc += tg.p[j].U;
    }
    tg.grid = pg.grid = grid;
    cudaError_t e = launch_dependent(prologue_r_kernel<W, G>, dim3((unsigned)pg.b_off[pg.count]), dim3(256), 0, st, pg);
    if (e != cudaSuccess) return e;
    e = ensure_smem_attr_tall<W, G>();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = TallLayout<W, G>::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, ring_gemm_tc_tall_kernel<W, G>, tg);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int W, int G>
cudaError_t launch_chunk_tall(const GemmArgs* a, uint8_t* const* Ap, const int* order, int cnt, cudaStream_t st) {
    auto* tg = new (std::nothrow) TcGroup<G>;
    auto* pg = new (std::nothrow) PrologueRGroup<G>;
    cudaError_t e = (tg && pg) ? cudaSuccess : cudaErrorMemoryAllocation;
    if (e == cudaSuccess) {
        tg->count = pg->count = cnt;
        pg->b_off[0] = 0;
        for (int j = 0; j < cnt && e == cudaSuccess; ++j) {
            const GemmArgs& x = a[order[j]];
            if (!fill_tall<W, G>(*tg, *pg, j, x, Ap[order[j]], make_plan(x.M, x.K, x.N, W, 0, TALL_ROWS)))
                e = cudaErrorInvalidValue;
        }
        if (e == cudaSuccess) e = launch_group_tall<W, G>(*tg, *pg, st);
    }
    delete tg;
    delete pg;
    return e;
}

constexpr int GSMALL = 16;   // small groups use a kernel with a smaller parameter block

// dynamic shared memory plus the grouped kernels' static layer table stay
// within the 227 KB a CTA may use (a launch over the limit fails)
template <int W, int G, int R = BM, bool WIDE = false> constexpr bool fits_smem() {
    return Gemm<W, G, R, WIDE>::SMEM + (G > 1 ? G * sizeof(TcParams) : 0) <= 227 * 1024;
}
static_assert(fits_smem<1, 1>() && fits_smem<2, 1>() && fits_smem<1, GSMALL>() && fits_smem<2, GSMALL>() &&
                  fits_smem<1, GMAX>() && fits_smem<2, GMAX>() && fits_smem<1, 1, 64>() && fits_smem<2, 1, 64>() &&
                  fits_smem<1, GSMALL, 64>() && fits_smem<2, GSMALL, 64>() && fits_smem<1, GMAX, 64>() &&
                  fits_smem<2, GMAX, 64>() && fits_smem<1, 1, BM, true>() && fits_smem<2, 1, BM, true>() &&
                  fits_smem<1, GSMALL, BM, true>() && fits_smem<2, GSMALL, BM, true>() &&
                  fits_smem<1, GMAX, BM, true>() && fits_smem<2, GMAX, BM, true>(),
              "shared memory of a TC GEMM instantiation");
static_assert(TallLayout<1, GMAX>::SMEM + GMAX * sizeof(TcParams) <= 227 * 1024 &&
                  TallLayout<2, GMAX>::SMEM + GMAX * sizeof(TcParams) <= 227 * 1024,
              "shared memory of the tall GEMM");

// A layer with units for at least LONG_WAVES waves of the grid gains little
// from sharing a launch (its last, partial wave is under 2 % of it), and the
// one-layer kernel runs it 2-10 % faster than a grouped kernel (measured on
// GB300 with pairs of long layers): grouped calls launch such layers alone.
// (At 12 waves VGG16 b16's 15-wave layers ran 6 % slower alone than grouped.)
constexpr int LONG_WAVES = 64;
bool long_layer(int64_t M, int64_t K, int64_t N, int words, int one_half, int sms, int rows = BM) {
    return make_plan(M, K, N, words, one_half, rows).U >= (int64_t)LONG_WAVES * sms;
}

// The layers idx[0 .. n) (all with R-row tiles) in launches of up to GMAX
// layers; layer i's digit planes at Ap[i].  Every layer is eligible and has
// the ring width W.
template <int W, int R, bool WIDE = false, bool TALL = false>
cudaError_t launch_many_rows(const GemmArgs* a, std::vector<int> order, uint8_t* const* Ap, cudaStream_t st) {
    constexpr int rows = TALL ? TALL_ROWS : WIDE ? Cfg<W>::ND : R;
    // layers with more K intervals first, so that whole tiles of the long
    // layers line up with the CTAs' ranges (the order changes no result)
    std::vector<std::pair<int, int>> by_iv;   // (intervals per tile, layer)
    for (int i : order) by_iv.push_back({make_plan(a[i].M, a[i].K, a[i].N, W, a[i].one_half, rows).I, i});
    std::stable_sort(by_iv.begin(), by_iv.end(),
                     [](const std::pair<int, int>& x, const std::pair<int, int>& y) { return x.first > y.first; });
    for (size_t j = 0; j < by_iv.size(); ++j) order[j] = by_iv[j].second;
    cudaError_t e = cudaSuccess;
    const int sms = sm_count();
    std::vector<int> rest;
    for (int i : order) {
        if (long_layer(a[i].M, a[i].K, a[i].N, W, a[i].one_half, sms, rows)) {
            if (e == cudaSuccess)
                e = TALL ? launch_chunk_tall<W, 1>(a, Ap, &i, 1, st) : launch_chunk<W, 1, R, WIDE>(a, Ap, &i, 1, st);
        } else {
            rest.push_back(i);
        }
    }
    const int n = (int)rest.size();
    for (int i0 = 0; i0 < n && e == cudaSuccess; i0 += GMAX) {
        const int cnt = n - i0 < GMAX ? n - i0 : GMAX;
        // a lone layer takes the one-layer kernel (parameters at constant offsets)
        if constexpr (TALL)
            e = cnt == 1        ? launch_chunk_tall<W, 1>(a, Ap, rest.data() + i0, cnt, st)
                : cnt <= GSMALL ? launch_chunk_tall<W, GSMALL>(a, Ap, rest.data() + i0, cnt, st)
                                : launch_chunk_tall<W, GMAX>(a, Ap, rest.data() + i0, cnt, st);
        else
            e = cnt == 1        ? launch_chunk<W, 1, R, WIDE>(a, Ap, rest.data() + i0, cnt, st)
                : cnt <= GSMALL ? launch_chunk<W, GSMALL, R, WIDE>(a, Ap, rest.data() + i0, cnt, st)
                                : launch_chunk<W, GMAX, R, WIDE>(a, Ap, rest.data() + i0, cnt, st);
    }
    return e;
}

// Layers [0, n): those with 128-row tiles, those with 64-row tiles and those
// with the wide tile in launches of their own (one kernel instantiation per
// tile).
template <int W>
cudaError_t launch_many(const GemmArgs* a, int n, uint8_t* const* Ap, cudaStream_t st) {
    std::vector<int> big, small, wide, tall;
    for (int i = 0; i < n; ++i)
        (tall_rows(a[i].rows) && !a[i].one_half ? tall
         : wide_rows(a[i].rows, W)               ? wide
         : tile_rows(a[i].rows) == 64            ? small
                                                 : big)
            .push_back(i);
    cudaError_t e = cudaSuccess;
    if (!big.empty()) e = launch_many_rows<W, BM>(a, big, Ap, st);
    if (e == cudaSuccess && !small.empty()) e = launch_many_rows<W, 64>(a, small, Ap, st);
    if (e == cudaSuccess && !wide.empty()) e = launch_many_rows<W, BM, true>(a, wide, Ap, st);
    if (e == cudaSuccess && !tall.empty()) e = launch_many_rows<W, BM, false, true>(a, tall, Ap, st);
    return e;
}

}  // namespace

bool gemm_tc_feasible(int64_t M, int64_t K, int64_t N, int words, int rows) {
    if (words != 1 && words != 2) return false;
    if (M <= 8 || N < 1 || K < 1) return false;        // skinny layers stream better on the SIMT GEMV
    if (words == 1 && N % 2 != 0) return false;       // TMA row stride: 16-byte multiple
    if (K > (int64_t(1) << 30) || N > (int64_t(1) << 28)) return false;
    // the tall tile loads rows of L by 2-D TMA: their stride (K words) must be a multiple of 16 bytes
    if (tall_rows(rows) && (K * words) % 2 != 0) return false;
    const int R = wide_rows(rows, words) ? (words == 1 ? Cfg<1>::ND : Cfg<2>::ND) : tile_rows(rows);
    if ((M + R - 1) / R > 65535) return false;
    return true;
}

bool gemm_tc_eligible(int64_t M, int64_t K, int64_t N, int words) {
    if (!gemm_tc_feasible(M, K, N, words)) return false;
    // smaller products run faster on the integer-pipe kernel
    const double macs = 2.0 * (double)M * (double)K * (double)N;
    return macs >= (words == 1 ? (double)(1 << 22) : (double)(1 << 20));
}

// the digit planes of every tile fit (the largest of the three tilings)
size_t gemm_tc_workspace(int64_t M, int64_t K, int64_t N, int words, int one_half) {
    if (!gemm_tc_feasible(M, K, N, words)) return 0;
    const int wide = words == 1 ? Cfg<1>::ND : Cfg<2>::ND;
    size_t b = make_plan(M, K, N, words, one_half, BM).ap_bytes;
    for (int rows : {64, wide, TALL_ROWS})
        if (gemm_tc_feasible(M, K, N, words, rows)) b = std::max(b, make_plan(M, K, N, words, one_half, rows).ap_bytes);
    return align256(b);
}

cudaError_t launch_gemm_tc(const GemmArgs& a, void* ws, size_t ws_bytes, cudaStream_t st) {
    if (tall_rows(a.rows) && !a.one_half && gemm_tc_feasible(a.M, a.K, a.N, a.words, TALL_ROWS)) {
        Plan pl = make_plan(a.M, a.K, a.N, a.words, 0, TALL_ROWS);
        if (ws_bytes < align256(pl.ap_bytes) || ws == nullptr) return cudaErrorInvalidValue;
        uint8_t* Rp = static_cast<uint8_t*>(ws);
        const int order = 0;
        return a.words == 1 ? launch_chunk_tall<1, 1>(&a, &Rp, &order, 1, st)
                            : launch_chunk_tall<2, 1>(&a, &Rp, &order, 1, st);
    }
    const bool wide = wide_rows(a.rows, a.words);
    const int rows = wide ? a.rows : tile_rows(a.rows);
    if (!gemm_tc_feasible(a.M, a.K, a.N, a.words, rows)) return cudaErrorNotSupported;
    Plan pl = make_plan(a.M, a.K, a.N, a.words, a.one_half, rows);
    if (ws_bytes < align256(pl.ap_bytes) || ws == nullptr) return cudaErrorInvalidValue;
    uint8_t* Ap = static_cast<uint8_t*>(ws);
    if (wide) return a.words == 1 ? launch<1, BM, true>(a, Ap, pl, st) : launch<2, BM, true>(a, Ap, pl, st);
    if (rows == 64) return a.words == 1 ? launch<1, 64>(a, Ap, pl, st) : launch<2, 64>(a, Ap, pl, st);
    return a.words == 1 ? launch<1, BM>(a, Ap, pl, st) : launch<2, BM>(a, Ap, pl, st);
}

int gemm_tc_launches(int64_t M, int64_t K, int64_t N, int words) {
    return gemm_tc_feasible(M, K, N, words) ? 2 : 0;
}

cudaError_t launch_gemm_tc_grouped(const GemmArgs* a, int n, uint8_t* const* Ap, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int w = a[0].words;
    for (int i = 0; i < n; ++i)
        if (a[i].words != w || !gemm_tc_feasible(a[i].M, a[i].K, a[i].N, w, a[i].rows) || !Ap[i] ||
            reinterpret_cast<uintptr_t>(Ap[i]) % 256 != 0)
            return cudaErrorInvalidValue;
    return w == 1 ? launch_many<1>(a, n, Ap, st) : launch_many<2>(a, n, Ap, st);
}

int gemm_tc_grouped_launches(const int64_t* M, const int64_t* K, const int64_t* N, int n, int words) {
    const int sms = sm_count();
    int alone = 0, rest[4] = {0, 0, 0, 0};
    for (int i = 0; i < n; ++i) {
        const int rows = gemm_choice(M[i], K[i], N[i], words).rows;
        const int kind = tall_rows(rows) ? 3 : wide_rows(rows, words) ? 2 : tile_rows(rows) == 64 ? 1 : 0;
        if (long_layer(M[i], K[i], N[i], words, 0, sms, kind >= 2 ? rows : tile_rows(rows))) ++alone;
        else ++rest[kind];
    }
    int pairs = alone;
    for (int k = 0; k < 4; ++k) pairs += (rest[k] + GMAX - 1) / GMAX;
    return 2 * pairs;
}

// ---------------------------------------------------------------------------
// self-test of the bounded wait: one thread waits on a barrier that nothing
// arrives at; the wait must give up after `limit` cycles and record the
// timeout exactly as the GEMM's roles do.

namespace {
__device__ int g_selftest_gave_up = 0;

__global__ void wait_selftest_kernel(long long limit) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        abort_flag = 0;
        ptx::fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool ok = ptx::mbar_wait(&bar, 0, &abort_flag, limit);
        if (!ok) {
            record_timeout(&abort_flag);
            g_selftest_gave_up = 1;
        }
    }
}
}  // namespace

int wait_selftest(long long limit, cudaStream_t st) {
    int zero = 0, v = 0;
    if (cudaMemcpyToSymbolAsync(g_selftest_gave_up, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st) !=
        cudaSuccess)
        return -1;
    wait_selftest_kernel<<<1, 32, 0, st>>>(limit);
    if (cudaGetLastError() != cudaSuccess) return -1;
    if (cudaMemcpyFromSymbolAsync(&v, g_selftest_gave_up, sizeof(v), 0, cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return -1;
    if (cudaStreamSynchronize(st) != cudaSuccess) return -1;
    return v;
}

namespace {
__device__ unsigned int g_tc_timeout_taken = 0;

// takes the flag atomically: a wait that gives up while the flag is being
// read is reported by the next query instead of being lost
__global__ void take_timeout_kernel() { g_tc_timeout_taken = atomicExch(&g_tc_timeout, 0u); }

// A non-blocking stream per device for the status query, so that reading the
// flag neither waits for nor orders itself with the caller's streams (a
// plain cudaMemcpyFromSymbol would run on the legacy default stream and wait
// for all work queued on blocking streams).
cudaStream_t status_stream() {
    static cudaStream_t streams[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
        streams[dev] = nullptr;
    return streams[dev];
}
}  // namespace

// Reads and clears the device flag that a bounded wait sets when it gives up.
// Kernels still running may set it after the read; the next query sees that.
int tc_timeout_flag(bool* set) {
    cudaStream_t s = status_stream();
    if (!s) return -1;
    take_timeout_kernel<<<1, 1, 0, s>>>();
    if (cudaGetLastError() != cudaSuccess) return -1;
    unsigned int v = 0;
    if (cudaMemcpyFromSymbolAsync(&v, g_tc_timeout_taken, sizeof(v), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return -1;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    *set = v != 0;
    return 0;
}

}  // namespace mpcl
