// kernels.h -- internal launcher interface between the C ABI (api.cu) and the
// kernel files.  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace mpcl {

using u64 = unsigned long long;

// The fused ring GEMM behind both a1 and a2.  With the 2K rewrite
//   Z = C + [E | X + c E] . [B ; F]
// a1 (share) uses (X, B, C) = (A_i, B_i, C_i), c = 1 for party 0 else 0, and
// a2 (full tag) uses (X, B, C) = (mA_i, mB_i, mC_i), c = alpha_i:
//   C + E.B + (X + cE).F = C + E.B + X.F + c (E.F).
enum CoefMode { COEF_ZERO = 0, COEF_ONE = 1, COEF_ALPHA = 2 };

struct GemmArgs {
    int64_t M, K, N;
    int words;
    const u64* E;      // M x K
    const u64* F;      // K x N
    const u64* X;      // M x K
    const u64* B;      // K x N (unused when one_half)
    const u64* C;      // M x N, or NULL for a zero addend
    u64* Z;            // M x N
    int coef;          // CoefMode
    const u64* alpha;  // one element (COEF_ALPHA)
    int one_half;      // 1: Z = C + (X + cE) . F over K only (the public product E.F)
    int gm;            // tensor cores: row tiles per swizzle group (0: default)
    int simt_waves;    // integer pipes: K-split target in waves of 152 blocks (0: default)
    int rows;          // tensor cores: tile rows, 128 or 64 (0: 128), the wide tile (32 for
                       // W = 1, 16 for W = 2) or the tall tile (-128); integer pipes: 64 or
                       // 16 (0: by grid size)
};

// The launch choice of one GEMM shape: path 1 = tensor cores (rows = tile
// height 128 or 64, gm = swizzle width), path 0 = integer pipes (waves =
// K-split target).  From the autotune table when the shape was tuned
// (tuned = 1), else the built-in heuristic.
struct Choice {
    int path;
    int gm;
    int waves;
    int tuned;
    int rows;
};
Choice gemm_choice(int64_t M, int64_t K, int64_t N, int words);
int wide_tile_rows(int words);   // the launch-table value of the wide tensor-core tile
// the launch-table value of the tall tensor-core tile (128-row tiles whose
// left operand the GEMM converts itself)
constexpr int TALL_TILE_ROWS = -128;

cudaError_t launch_gemm_simt(const GemmArgs& a, cudaStream_t st);

// tensor-core ring GEMM (fp16 digit products, exact); returns
// cudaErrorNotSupported when the shape is not handled by it.
cudaError_t launch_gemm_tc(const GemmArgs& a, void* ws, size_t ws_bytes, cudaStream_t st);
// several eligible layers of one ring width in grouped persistent launches
// (up to 64 layers per prologue + GEMM pair); layer i's digit planes at Ap[i]
// (gemm_tc_workspace bytes, 256-byte aligned)
cudaError_t launch_gemm_tc_grouped(const GemmArgs* a, int n, uint8_t* const* Ap, cudaStream_t st);
int gemm_tc_grouped_launches(const int64_t* M, const int64_t* K, const int64_t* N, int n, int words);
// 1 when a bounded wait on a barrier nothing arrives at gave up (as it must),
// 0 if it did not, -1 on a CUDA error; synchronous
int wait_selftest(long long limit, cudaStream_t st);
size_t gemm_tc_workspace(int64_t M, int64_t K, int64_t N, int words, int one_half = 0);
bool gemm_tc_eligible(int64_t M, int64_t K, int64_t N, int words);   // heuristic preference
// the kernel can run the shape with `rows`-row tiles (128 or 64)
bool gemm_tc_feasible(int64_t M, int64_t K, int64_t N, int words, int rows = 128);
int gemm_tc_launches(int64_t M, int64_t K, int64_t N, int words);
int tc_timeout_flag(bool* set);   // synchronous; 0 on success

// CompactTag path (a3, a4, a5)
struct CompactArgs {
    int64_t M, K, N;
    int words;
    int with_eu;       // 1: the compact tag includes alpha E.(F chi) (untruncated layer)
    const u64* alpha;
    const u64* E;
    const u64* F;
    const u64* mA;
    const u64* mB;
    const u64* mC;
    const u64* mR;
    const u64* Dt;
    const u64* chi;
    u64* mZ;   // M x N, or NULL (the OptMAC tag is not written)
    u64* mDc;  // M
    u64* Dc;   // M
};
size_t compact_workspace(int64_t M, int64_t K, int64_t N, int words);
int compact_launches(int64_t M, int64_t K, int64_t N);
cudaError_t launch_compact(const CompactArgs& a, void* ws, size_t ws_bytes, cudaStream_t st);
// the tags of many layers (one ring width) in three launches per 64 layers;
// layer i's workspace (compact_workspace bytes) at ws[i]
cudaError_t launch_compact_grouped(const CompactArgs* a, int n, char* const* ws, cudaStream_t st);
int compact_grouped_launches(const int64_t* M, const int64_t* K, const int64_t* N, int n);

// truncated layer: OptMAC&Trunc elementwise step
cudaError_t launch_optmac_trunc(int64_t MN, int words, int k, int f, int party0, const u64* alpha,
                                const u64* Rf, const u64* mRf, const u64* Dt, const u64* P, u64* Zf,
                                u64* mZf, cudaStream_t st);

// out = sum_j coef[j] in[j] (elementwise, count <= LINCOMB_MAX); out may be one
// of the inputs (each element is read before it is written, by one thread)
constexpr int LINCOMB_MAX = 16;
cudaError_t launch_lincomb(int64_t n, int words, int count, const int64_t* coef, const u64* const* in, u64* out,
                           cudaStream_t st);
// `groups` combinations with the same coefficients (count <= LINCOMB_GROUP_TERMS
// terms each), LINCOMB_GROUP_MAX groups per launch; group g reads
// in[g * count + j] and writes out[g] (n[g] elements)
constexpr int LINCOMB_GROUP_MAX = 64;
constexpr int LINCOMB_GROUP_TERMS = 4;
cudaError_t launch_lincomb_grouped(int groups, const int64_t* n, int words, int count, const int64_t* coef,
                                   const u64* const* in, u64* const* out, cudaStream_t st);

// im2col of NCHW ring-element images for an f x f convolution (stride, zero padding)
cudaError_t launch_im2col(int64_t B, int64_t C, int64_t H, int64_t W, int f, int pad, int stride, int words,
                          const u64* in, u64* out, cudaStream_t st);

// local transpose of a ring matrix (training's backward layers)
cudaError_t launch_transpose(int64_t rows, int64_t cols, int words, const u64* in, u64* out,
                             cudaStream_t st);

// checks (a6)
cudaError_t launch_check_compact(int64_t M, int words, const u64* alpha, const u64* chi_hat,
                                 const u64* Dc, const u64* mDc, u64* cs, cudaStream_t st);
// n compact checks, CHECK_GROUP_MAX per launch (one block per check)
constexpr int CHECK_GROUP_MAX = 64;
cudaError_t launch_check_compact_grouped(int n, int words, const int64_t* M, const u64* const* alpha,
                                         const u64* const* chi_hat, const u64* const* Dc,
                                         const u64* const* mDc, u64* const* cs, cudaStream_t st);
size_t check_batchrec_workspace(int64_t M, int64_t N, int words);
cudaError_t launch_check_batchrec_seeded(int64_t M, int64_t N, int words, int s, const u64* alpha,
                                         const u64* seed, const u64* W, const u64* mW, u64* cs,
                                         void* ws, size_t ws_bytes, cudaStream_t st);
cudaError_t launch_batchrec_mask(int64_t n, int words, const u64* X, const u64* A, const u64* R,
                                 const u64* mX, const u64* mA, const u64* mR, u64* W, u64* mW,
                                 cudaStream_t st);
cudaError_t launch_check_batchrec(int64_t M, int64_t N, int words, const u64* alpha,
                                  const u64* chi, const u64* W, const u64* mW, u64* cs,
                                  void* ws, size_t ws_bytes, cudaStream_t st);

}  // namespace mpcl
