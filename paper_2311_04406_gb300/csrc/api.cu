// api.cu -- the C ABI declared in include/mpclinear.h.
//
// Every entry point validates its arguments on the host (shapes, ring,
// pointers, alignment, workspace) and returns a negative status without
// launching anything when they are invalid, so no kernel ever runs on bad
// input.  Valid calls enqueue kernels on the caller's stream and return.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "mpclinear.h"
#include "kernels.h"

using mpcl::u64;

namespace {

constexpr int64_t kMaxDim = int64_t(1) << 31;     // per dimension
constexpr int64_t kMaxElems = int64_t(1) << 36;   // per matrix

bool ring_ok(const mpc_ring& r) {
    return (r.words == 1 || r.words == 2) && r.k >= 1 && r.s >= 1 && r.k + r.s == 64 * r.words;
}

int check_layer(const mpc_layer* L) {
    if (!L) return MPC_E_NULL;
    if (!ring_ok(L->ring)) return MPC_E_RING;
    if (L->M < 0 || L->K < 0 || L->N < 0) return MPC_E_SHAPE;
    if (L->M > kMaxDim || L->K > kMaxDim || L->N > kMaxDim) return MPC_E_SHAPE;
    if (L->M * L->K > kMaxElems || L->K * L->N > kMaxElems || L->M * L->N > kMaxElems)
        return MPC_E_SHAPE;
    if (L->nparties < 1 || L->party < 0 || L->party >= L->nparties) return MPC_E_PARTY;
    return MPC_OK;
}

// a pointer to `elems` ring elements: NULL allowed only when elems == 0
int check_ptr(const void* p, int64_t elems) {
    if (elems == 0) return MPC_OK;
    if (!p) return MPC_E_NULL;
    if (reinterpret_cast<uintptr_t>(p) % 16 != 0) return MPC_E_ALIGN;
    return MPC_OK;
}

#define CHK(x)                         \
    do {                               \
        int _s = (x);                  \
        if (_s != MPC_OK) return _s;   \
    } while (0)

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return MPC_OK;
    return MPC_E_CUDA;
}

// Workspace of a GEMM: the tensor-core digit planes whenever that kernel can
// run the shape, so that any launch-table choice fits the same workspace.
size_t gemm_ws(const mpc_layer* L, int one_half = 0) {
    return mpcl::gemm_tc_workspace(L->M, L->K, L->N, L->ring.words, one_half);
}

int run_gemm(mpcl::GemmArgs g, void* ws, size_t ws_bytes, cudaStream_t st) {
    if (g.M == 0 || g.N == 0) return MPC_OK;
    const mpcl::Choice c = mpcl::gemm_choice(g.M, g.K, g.N, g.words);
    if (c.path == 1) {
        if (!ws || ws_bytes < mpcl::gemm_tc_workspace(g.M, g.K, g.N, g.words, g.one_half))
            return MPC_E_WORKSPACE;
        if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return MPC_E_ALIGN;
        g.gm = c.gm;
        g.rows = c.rows;
        return cuda_status(mpcl::launch_gemm_tc(g, ws, ws_bytes, st));
    }
    g.simt_waves = c.waves;
    g.rows = c.rows;
    return cuda_status(mpcl::launch_gemm_simt(g, st));
}

}  // namespace

extern "C" {

int mpc_version(void) { return 200; }

int mpc_gemm_path(const mpc_layer* L) {
    int st = check_layer(L);
    if (st != MPC_OK) return st;
    return mpcl::gemm_choice(L->M, L->K, L->N, L->ring.words).path;
}

int mpc_launch_count(const mpc_layer* L, int which) {
    int st = check_layer(L);
    if (st != MPC_OK) return st;
    const int64_t M = L->M, K = L->K, N = L->N;
    const int w = L->ring.words;
    switch (which) {
        case MPC_WS_SHARE:
        case MPC_WS_SHARE_TRUNC:
        case MPC_WS_PUBLIC_PRODUCT:
        case MPC_WS_TAG_FULL:
            if (M == 0 || N == 0) return 0;
            return mpcl::gemm_choice(M, K, N, w).path == 1 ? mpcl::gemm_tc_launches(M, K, N, w) : 1;
        case MPC_WS_TAG_COMPACT: return mpcl::compact_launches(M, K, N);
        case MPC_WS_CHECK_COMPACT: return 1;
        case MPC_WS_CHECK_BATCHREC: return 2;
        case MPC_WS_OPTMAC_TRUNC: return (M > 0 && N > 0) ? 1 : 0;
        default: return MPC_E_MODE;
    }
}

int mpc_selftest_wait(long long limit_cycles, void* stream) {
    if (limit_cycles < 1000 || limit_cycles > 10000000000LL) return MPC_E_SHAPE;
    const int r = mpcl::wait_selftest(limit_cycles, (cudaStream_t)stream);
    if (r < 0) return MPC_E_CUDA;
    return r == 1 ? MPC_E_TIMEOUT : MPC_OK;
}

int mpc_device_status(void) {
    bool set = false;
    if (mpcl::tc_timeout_flag(&set) != 0) return MPC_E_CUDA;
    return set ? MPC_E_TIMEOUT : MPC_OK;
}

const char* mpc_status_str(int s) {
    switch (s) {
        case MPC_OK: return "ok";
        case MPC_E_NULL: return "a required pointer is NULL";
        case MPC_E_SHAPE: return "invalid shape (negative or too large M, K, N)";
        case MPC_E_RING: return "unsupported ring: need (k, s, words) with k + s = 64 * words, words 1 or 2";
        case MPC_E_ALIGN: return "a pointer is not 16-byte aligned";
        case MPC_E_WORKSPACE: return "workspace missing or smaller than mpc_workspace_size()";
        case MPC_E_CUDA: return "CUDA launch or runtime error";
        case MPC_E_MODE: return "unknown tag or check mode";
        case MPC_E_PARTY: return "party index outside [0, nparties)";
        case MPC_E_TIMEOUT: return "a device-side wait gave up";
        case MPC_E_SCRATCH_LIMIT:
            return "layer needs more scratch than the static MPC_NOALLOC_SCRATCH_BYTES buffer holds";
        case MPC_E_IO: return "an autotune table file could not be read or written";
        default: return "unknown status";
    }
}

size_t mpc_workspace_size(const mpc_layer* L, int which) {
    if (check_layer(L) != MPC_OK) return 0;
    const int w = L->ring.words;
    switch (which) {
        case MPC_WS_SHARE:
        case MPC_WS_SHARE_TRUNC:
        case MPC_WS_TAG_FULL: return gemm_ws(L);
        case MPC_WS_PUBLIC_PRODUCT: return gemm_ws(L, 1);
        case MPC_WS_OPTMAC_TRUNC: return 0;
        case MPC_WS_TAG_COMPACT: return mpcl::compact_workspace(L->M, L->K, L->N, w);
        case MPC_WS_CHECK_COMPACT: return 0;
        case MPC_WS_CHECK_BATCHREC: return mpcl::check_batchrec_workspace(L->M, L->N, w);
        default: return 0;
    }
}

int mpc_linear_share(const mpc_layer* L, const uint64_t* E, const uint64_t* F,
                     const uint64_t* A_i, const uint64_t* B_i, const uint64_t* C_i,
                     uint64_t* Z_i, void* ws, size_t ws_bytes, void* stream) {
    CHK(check_layer(L));
    const int64_t M = L->M, K = L->K, N = L->N;
    CHK(check_ptr(E, M * K));
    CHK(check_ptr(A_i, M * K));
    CHK(check_ptr(F, K * N));
    CHK(check_ptr(B_i, K * N));
    CHK(check_ptr(C_i, M * N));
    CHK(check_ptr(Z_i, M * N));
    mpcl::GemmArgs g{M, K, N, L->ring.words,
                     (const u64*)E, (const u64*)F, (const u64*)A_i, (const u64*)B_i,
                     (const u64*)C_i, (u64*)Z_i,
                     L->party == 0 ? mpcl::COEF_ONE : mpcl::COEF_ZERO, nullptr, 0};
    return run_gemm(g, ws, ws_bytes, (cudaStream_t)stream);
}

int mpc_lincomb(const mpc_ring* ring, int64_t n, int count, const int64_t* coef, const uint64_t* const* in,
                uint64_t* out, void* stream) {
    if (!ring || !coef || !in) return MPC_E_NULL;
    if (!ring_ok(*ring)) return MPC_E_RING;
    if (n < 0 || n > kMaxElems || count < 1 || count > mpcl::LINCOMB_MAX) return MPC_E_SHAPE;
    for (int j = 0; j < count; ++j) CHK(check_ptr(in[j], n));
    CHK(check_ptr(out, n));
    return cuda_status(mpcl::launch_lincomb(n, ring->words, count, coef, (const u64* const*)in, (u64*)out,
                                            (cudaStream_t)stream));
}

int mpc_lincomb_grouped(const mpc_ring* ring, int groups, const int64_t* n, int count, const int64_t* coef,
                        const uint64_t* const* in, uint64_t* const* out, void* stream) {
    if (groups < 0 || count < 1 || count > mpcl::LINCOMB_GROUP_TERMS) return MPC_E_SHAPE;
    if (groups == 0) return MPC_OK;
    if (!ring || !coef || !in || !out || !n) return MPC_E_NULL;
    if (!ring_ok(*ring)) return MPC_E_RING;
    for (int g = 0; g < groups; ++g) {
        if (n[g] < 0 || n[g] > kMaxElems) return MPC_E_SHAPE;
        for (int j = 0; j < count; ++j) CHK(check_ptr(in[(size_t)g * count + j], n[g]));
        CHK(check_ptr(out[g], n[g]));
    }
    return cuda_status(mpcl::launch_lincomb_grouped(groups, n, ring->words, count, coef, (const u64* const*)in,
                                                    (u64* const*)out, (cudaStream_t)stream));
}

int mpc_im2col(const mpc_ring* ring, int64_t batch, int64_t channels, int64_t height, int64_t width, int f,
               int pad, int stride, const uint64_t* in, uint64_t* out, void* stream) {
    if (!ring) return MPC_E_NULL;
    if (!ring_ok(*ring)) return MPC_E_RING;
    if (batch < 0 || channels < 0 || height < 0 || width < 0 || f < 1 || pad < 0 || stride < 1 ||
        f > 64 || pad >= f || height > kMaxDim || width > kMaxDim || channels > kMaxDim || batch > kMaxDim)
        return MPC_E_SHAPE;
    if (height + 2 * pad < f || width + 2 * pad < f) return MPC_E_SHAPE;
    const int64_t Ho = (height - f + 2 * pad) / stride + 1, Wo = (width - f + 2 * pad) / stride + 1;
    const int64_t nin = batch * channels * height * width;
    const int64_t rows = batch * Ho * Wo, cols = channels * f * f;
    if (nin > kMaxElems || rows > kMaxDim || cols > kMaxDim || rows * cols > kMaxElems) return MPC_E_SHAPE;
    CHK(check_ptr(in, nin));
    CHK(check_ptr(out, rows * cols));
    return cuda_status(mpcl::launch_im2col(batch, channels, height, width, f, pad, stride, ring->words,
                                           (const u64*)in, (u64*)out, (cudaStream_t)stream));
}

int mpc_transpose(const mpc_ring* ring, int64_t rows, int64_t cols, const uint64_t* in, uint64_t* out,
                  void* stream) {
    if (!ring) return MPC_E_NULL;
    if (!ring_ok(*ring)) return MPC_E_RING;
    if (rows < 0 || cols < 0 || rows > kMaxDim || cols > kMaxDim || rows * cols > kMaxElems)
        return MPC_E_SHAPE;
    CHK(check_ptr(in, rows * cols));
    CHK(check_ptr(out, rows * cols));
    return cuda_status(mpcl::launch_transpose(rows, cols, ring->words, (const u64*)in, (u64*)out,
                                              (cudaStream_t)stream));
}

int mpc_batchrec_mask(const mpc_ring* ring, int64_t rows, int64_t cols, const uint64_t* X_i,
                      const uint64_t* A_i, const uint64_t* R_i, const uint64_t* mX_i,
                      const uint64_t* mA_i, const uint64_t* mR_i, uint64_t* W_i, uint64_t* mW_i,
                      void* stream) {
    if (!ring) return MPC_E_NULL;
    if (!ring_ok(*ring)) return MPC_E_RING;
    if (rows < 0 || cols < 0 || rows > kMaxDim || cols > kMaxDim || rows * cols > kMaxElems)
        return MPC_E_SHAPE;
    const int64_t n = rows * cols;
    CHK(check_ptr(X_i, n));
    CHK(check_ptr(R_i, n));
    CHK(check_ptr(mX_i, n));
    CHK(check_ptr(mR_i, n));
    CHK(check_ptr(W_i, n));
    CHK(check_ptr(mW_i, n));
    if (A_i) CHK(check_ptr(A_i, n));
    if (mA_i) CHK(check_ptr(mA_i, n));
    return cuda_status(mpcl::launch_batchrec_mask(n, ring->words, (const u64*)X_i, (const u64*)A_i,
                                                  (const u64*)R_i, (const u64*)mX_i, (const u64*)mA_i,
                                                  (const u64*)mR_i, (u64*)W_i, (u64*)mW_i,
                                                  (cudaStream_t)stream));
}

int mpc_linear_share_trunc(const mpc_layer* L, const uint64_t* E, const uint64_t* F,
                           const uint64_t* A_i, const uint64_t* B_i, const uint64_t* C_i,
                           uint64_t* Z_i, void* ws, size_t ws_bytes, void* stream) {
    CHK(check_layer(L));
    const int64_t M = L->M, K = L->K, N = L->N;
    CHK(check_ptr(E, M * K));
    CHK(check_ptr(A_i, M * K));
    CHK(check_ptr(F, K * N));
    CHK(check_ptr(B_i, K * N));
    CHK(check_ptr(C_i, M * N));
    CHK(check_ptr(Z_i, M * N));
    mpcl::GemmArgs g{M, K, N, L->ring.words,
                     (const u64*)E, (const u64*)F, (const u64*)A_i, (const u64*)B_i,
                     (const u64*)C_i, (u64*)Z_i, mpcl::COEF_ZERO, nullptr, 0};
    return run_gemm(g, ws, ws_bytes, (cudaStream_t)stream);
}

int mpc_public_product(const mpc_layer* L, const uint64_t* E, const uint64_t* F, uint64_t* P,
                       void* ws, size_t ws_bytes, void* stream) {
    CHK(check_layer(L));
    const int64_t M = L->M, K = L->K, N = L->N;
    CHK(check_ptr(E, M * K));
    CHK(check_ptr(F, K * N));
    CHK(check_ptr(P, M * N));
    // P = (X + 0 E) . F with X = E over the K of one half; no addend
    mpcl::GemmArgs g{M, K, N, L->ring.words, (const u64*)E, (const u64*)F, (const u64*)E, nullptr,
                     nullptr, (u64*)P, mpcl::COEF_ZERO, nullptr, 1};
    return run_gemm(g, ws, ws_bytes, (cudaStream_t)stream);
}

int mpc_optmac_trunc(const mpc_layer* L, int f, const uint64_t* alpha_i, const uint64_t* Rf_i,
                     const uint64_t* mRf_i, const uint64_t* Dtilde, const uint64_t* P,
                     uint64_t* Zf_i, uint64_t* mZf_i, void* stream) {
    CHK(check_layer(L));
    if (f < 0 || f > L->ring.k) return MPC_E_SHAPE;
    const int64_t MN = L->M * L->N;
    CHK(check_ptr(alpha_i, 1));
    CHK(check_ptr(Rf_i, MN));
    CHK(check_ptr(mRf_i, MN));
    CHK(check_ptr(Dtilde, MN));
    CHK(check_ptr(P, MN));
    CHK(check_ptr(Zf_i, MN));
    CHK(check_ptr(mZf_i, MN));
    return cuda_status(mpcl::launch_optmac_trunc(MN, L->ring.words, L->ring.k, f, L->party == 0 ? 1 : 0,
                                                 (const u64*)alpha_i, (const u64*)Rf_i, (const u64*)mRf_i,
                                                 (const u64*)Dtilde, (const u64*)P, (u64*)Zf_i,
                                                 (u64*)mZf_i, (cudaStream_t)stream));
}

int mpc_linear_tag(const mpc_layer* L, int mode, const uint64_t* alpha_i,
                   const uint64_t* E, const uint64_t* F,
                   const uint64_t* mA_i, const uint64_t* mB_i, const uint64_t* mC_i,
                   const uint64_t* mR_i, const uint64_t* Dtilde, const uint64_t* chi,
                   uint64_t* mZ_i, uint64_t* mDc_i, uint64_t* Dc,
                   void* ws, size_t ws_bytes, void* stream) {
    CHK(check_layer(L));
    if (mode != MPC_TAG_FULL && mode != MPC_TAG_COMPACT && mode != MPC_TAG_COMPACT_TRUNC) return MPC_E_MODE;
    const int64_t M = L->M, K = L->K, N = L->N;
    const int w = L->ring.words;
    CHK(check_ptr(alpha_i, 1));
    CHK(check_ptr(E, M * K));
    CHK(check_ptr(mA_i, M * K));
    CHK(check_ptr(F, K * N));
    CHK(check_ptr(mB_i, K * N));
    CHK(check_ptr(mC_i, M * N));
    if (mode != MPC_TAG_COMPACT_TRUNC || mZ_i != nullptr) CHK(check_ptr(mZ_i, M * N));
    cudaStream_t st = (cudaStream_t)stream;
    if (mode == MPC_TAG_FULL) {
        mpcl::GemmArgs g{M, K, N, w, (const u64*)E, (const u64*)F, (const u64*)mA_i,
                         (const u64*)mB_i, (const u64*)mC_i, (u64*)mZ_i, mpcl::COEF_ALPHA,
                         (const u64*)alpha_i, 0};
        return run_gemm(g, ws, ws_bytes, st);
    }
    CHK(check_ptr(mR_i, M * N));
    CHK(check_ptr(Dtilde, M * N));
    CHK(check_ptr(chi, N));
    CHK(check_ptr(mDc_i, M));
    CHK(check_ptr(Dc, M));
    const size_t need = mpcl::compact_workspace(M, K, N, w);
    if (M > 0 && need > 0) {
        if (!ws || ws_bytes < need) return MPC_E_WORKSPACE;
        if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return MPC_E_ALIGN;
    }
    mpcl::CompactArgs c{M, K, N, w, mode == MPC_TAG_COMPACT ? 1 : 0, (const u64*)alpha_i,
                        (const u64*)E, (const u64*)F,
                        (const u64*)mA_i, (const u64*)mB_i, (const u64*)mC_i, (const u64*)mR_i,
                        (const u64*)Dtilde, (const u64*)chi, (u64*)mZ_i, (u64*)mDc_i, (u64*)Dc};
    return cuda_status(mpcl::launch_compact(c, ws, ws_bytes, st));
}

int mpc_tag_check(const mpc_layer* L, int mode, const uint64_t* alpha_i,
                  const uint64_t* chi_hat, const uint64_t* opened, const uint64_t* tag_i,
                  uint64_t* cs_i, void* ws, size_t ws_bytes, void* stream) {
    CHK(check_layer(L));
    const int64_t M = L->M, N = L->N;
    const int w = L->ring.words;
    cudaStream_t st = (cudaStream_t)stream;
    CHK(check_ptr(alpha_i, 1));
    CHK(check_ptr(cs_i, 1));
    if (mode == MPC_CHECK_COMPACT) {
        CHK(check_ptr(chi_hat, M));
        CHK(check_ptr(opened, M));
        CHK(check_ptr(tag_i, M));
        return cuda_status(mpcl::launch_check_compact(M, w, (const u64*)alpha_i,
                                                      (const u64*)chi_hat, (const u64*)opened,
                                                      (const u64*)tag_i, (u64*)cs_i, st));
    }
    if (mode == MPC_CHECK_BATCHREC_SEEDED) {
        if (L->ring.s > 64) return MPC_E_RING;
        CHK(check_ptr(chi_hat, 1));
        CHK(check_ptr(opened, M * N));
        CHK(check_ptr(tag_i, M * N));
        const size_t need = mpcl::check_batchrec_workspace(M, N, w);
        if (!ws || ws_bytes < need) return MPC_E_WORKSPACE;
        if (reinterpret_cast<uintptr_t>(ws) % 16 != 0) return MPC_E_ALIGN;
        return cuda_status(mpcl::launch_check_batchrec_seeded(
            M, N, w, L->ring.s, (const u64*)alpha_i, (const u64*)chi_hat, (const u64*)opened,
            (const u64*)tag_i, (u64*)cs_i, ws, ws_bytes, st));
    }
    if (mode != MPC_CHECK_BATCHREC) return MPC_E_MODE;
    CHK(check_ptr(chi_hat, M * N));
    CHK(check_ptr(opened, M * N));
    CHK(check_ptr(tag_i, M * N));
    const size_t need = mpcl::check_batchrec_workspace(M, N, w);
    if (!ws || ws_bytes < need) return MPC_E_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(ws) % 16 != 0) return MPC_E_ALIGN;
    return cuda_status(mpcl::launch_check_batchrec(M, N, w, (const u64*)alpha_i,
                                                   (const u64*)chi_hat, (const u64*)opened,
                                                   (const u64*)tag_i, (u64*)cs_i, ws, ws_bytes, st));
}

}  // extern "C"

// ---------------------------------------------------------------------------
// grouped calls

namespace {

bool same_ring(const mpc_ring& a, const mpc_ring& b) {
    return a.k == b.k && a.s == b.s && a.words == b.words;
}

int check_group(const mpc_layer* layers, int count, const void* ptrs) {
    if (count < 0) return MPC_E_SHAPE;
    if (count == 0) return MPC_OK;
    if (!layers || !ptrs) return MPC_E_NULL;
    for (int i = 0; i < count; ++i) {
        CHK(check_layer(&layers[i]));
        if (!same_ring(layers[i].ring, layers[0].ring)) return MPC_E_RING;
    }
    return MPC_OK;
}

bool on_tc(const mpc_layer& L) {
    return L.M > 0 && L.N > 0 && mpcl::gemm_choice(L.M, L.K, L.N, L.ring.words).path == 1;
}

// workspace of a grouped GEMM: the digit planes of every layer the
// tensor-core kernel can run (whatever the launch table picks)
size_t group_gemm_ws(const mpc_layer* layers, int count) {
    size_t t = 0;
    for (int i = 0; i < count; ++i)
        if (layers[i].M > 0 && layers[i].N > 0)
            t += (mpcl::gemm_tc_workspace(layers[i].M, layers[i].K, layers[i].N, layers[i].ring.words) + 255) &
                 ~size_t(255);
    return t;
}

size_t group_compact_ws(const mpc_layer* layers, int count) {
    size_t t = 0;
    for (int i = 0; i < count; ++i)
        t += (mpcl::compact_workspace(layers[i].M, layers[i].K, layers[i].N, layers[i].ring.words) + 255) &
             ~size_t(255);
    return t;
}

// the tensor-core layers as one grouped launch, the others one by one
// Side streams for the integer-pipe layers of a grouped call.  Those layers are
// independent of one another and of the tensor-core layers, and each uses a
// fraction of the GPU (a split-K GEMV of a batch-1 layer streams its weights
// with a few hundred blocks), so they run concurrently: a fork event recorded
// on the caller's stream before any of the call's launches, which every side
// stream waits for (nothing starts before the call's inputs are ready), the
// layers dealt round-robin to the side streams, and one join event per side
// stream that the caller's stream waits for.  Under stream capture the same
// calls make parallel branches of the graph.  Per device, created on first use
// and kept until the process exits; the mutex keeps two host threads from
// interleaving their fork and join records.  If the streams cannot be created
// the layers run one after another on the caller's stream.
constexpr int SIDE_STREAMS = 4;
constexpr int SIDE_DEVICES = 64;

struct SidePool {
    std::mutex mu;
    bool tried = false, ok = false;
    cudaStream_t s[SIDE_STREAMS] = {};
    cudaEvent_t fork = nullptr, join[SIDE_STREAMS] = {};
};

SidePool* side_pool() {
    static SidePool pools[SIDE_DEVICES];
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= SIDE_DEVICES) return nullptr;
    SidePool* p = &pools[dev];
    std::lock_guard<std::mutex> lk(p->mu);
    if (!p->tried) {
        p->tried = true;
        bool ok = cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) == cudaSuccess;
        for (int i = 0; ok && i < SIDE_STREAMS; ++i)
            ok = cudaStreamCreateWithFlags(&p->s[i], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&p->join[i], cudaEventDisableTiming) == cudaSuccess;
        p->ok = ok;
    }
    return p->ok ? p : nullptr;
}

int run_gemm_group(const mpc_layer* layers, int count, const mpcl::GemmArgs* g, void* ws, size_t ws_bytes,
                   cudaStream_t st) {
    const size_t need = group_gemm_ws(layers, count);
    if (need > 0) {
        if (!ws || ws_bytes < need) return MPC_E_WORKSPACE;
        if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return MPC_E_ALIGN;
    }
    std::vector<mpcl::GemmArgs> tc, simt;
    std::vector<uint8_t*> ap;
    uint8_t* cur = static_cast<uint8_t*>(ws);
    for (int i = 0; i < count; ++i) {
        if (g[i].M == 0 || g[i].N == 0) continue;
        const mpcl::Choice c = mpcl::gemm_choice(g[i].M, g[i].K, g[i].N, g[i].words);
        mpcl::GemmArgs x = g[i];
        if (c.path == 1) {
            x.gm = c.gm;
            x.rows = c.rows;
            tc.push_back(x);
            ap.push_back(cur);
        } else {
            x.simt_waves = c.waves;
            x.rows = c.rows;
            simt.push_back(x);
        }
        cur += (mpcl::gemm_tc_workspace(g[i].M, g[i].K, g[i].N, g[i].words) + 255) & ~size_t(255);
    }
    SidePool* side = (!simt.empty() && simt.size() + (tc.empty() ? 0 : 1) >= 2) ? side_pool() : nullptr;
    if (!side) {
        if (!tc.empty()) CHK(cuda_status(mpcl::launch_gemm_tc_grouped(tc.data(), (int)tc.size(), ap.data(), st)));
        for (const auto& x : simt) CHK(cuda_status(mpcl::launch_gemm_simt(x, st)));
        return MPC_OK;
    }
    std::lock_guard<std::mutex> lk(side->mu);
    const int ns = (int)std::min<size_t>(simt.size(), SIDE_STREAMS);
    CHK(cuda_status(cudaEventRecord(side->fork, st)));
    for (int i = 0; i < ns; ++i) CHK(cuda_status(cudaStreamWaitEvent(side->s[i], side->fork, 0)));
    // from here on every side stream is joined back whatever a launch returns,
    // so that the caller's stream never runs ahead of work queued on a side
    // stream; the first error is reported
    int status = MPC_OK;
    for (size_t j = 0; j < simt.size() && status == MPC_OK; ++j)
        status = cuda_status(mpcl::launch_gemm_simt(simt[j], side->s[j % ns]));
    if (status == MPC_OK && !tc.empty())
        status = cuda_status(mpcl::launch_gemm_tc_grouped(tc.data(), (int)tc.size(), ap.data(), st));
    for (int i = 0; i < ns; ++i) {
        const int a = cuda_status(cudaEventRecord(side->join[i], side->s[i]));
        const int b = a == MPC_OK ? cuda_status(cudaStreamWaitEvent(st, side->join[i], 0)) : a;
        if (status == MPC_OK) status = b;
    }
    return status;
}

}  // namespace

extern "C" {

int mpc_linear_share_grouped(const mpc_layer* layers, int count, const mpc_share_ptrs* ptrs, void* ws,
                             size_t ws_bytes, void* stream) {
    CHK(check_group(layers, count, ptrs));
    if (count == 0) return MPC_OK;
    std::vector<mpcl::GemmArgs> g((size_t)count);
    for (int i = 0; i < count; ++i) {
        const mpc_layer* L = &layers[i];
        const mpc_share_ptrs& p = ptrs[i];
        const int64_t M = L->M, K = L->K, N = L->N;
        CHK(check_ptr(p.E, M * K));
        CHK(check_ptr(p.A_i, M * K));
        CHK(check_ptr(p.F, K * N));
        CHK(check_ptr(p.B_i, K * N));
        CHK(check_ptr(p.C_i, M * N));
        CHK(check_ptr(p.Z_i, M * N));
        g[i] = mpcl::GemmArgs{M, K, N, L->ring.words, (const u64*)p.E, (const u64*)p.F, (const u64*)p.A_i,
                              (const u64*)p.B_i, (const u64*)p.C_i, (u64*)p.Z_i,
                              L->party == 0 ? mpcl::COEF_ONE : mpcl::COEF_ZERO, nullptr, 0};
    }
    return run_gemm_group(layers, count, g.data(), ws, ws_bytes, (cudaStream_t)stream);
}

int mpc_linear_tag_grouped(const mpc_layer* layers, int count, int mode, const mpc_tag_ptrs* ptrs, void* ws,
                           size_t ws_bytes, void* stream) {
    if (mode != MPC_TAG_FULL && mode != MPC_TAG_COMPACT && mode != MPC_TAG_COMPACT_TRUNC) return MPC_E_MODE;
    CHK(check_group(layers, count, ptrs));
    if (count == 0) return MPC_OK;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<mpcl::GemmArgs> g;
    std::vector<mpcl::CompactArgs> c;
    for (int i = 0; i < count; ++i) {
        const mpc_layer* L = &layers[i];
        const mpc_tag_ptrs& p = ptrs[i];
        const int64_t M = L->M, K = L->K, N = L->N;
        const int w = L->ring.words;
        CHK(check_ptr(p.alpha_i, 1));
        CHK(check_ptr(p.E, M * K));
        CHK(check_ptr(p.mA_i, M * K));
        CHK(check_ptr(p.F, K * N));
        CHK(check_ptr(p.mB_i, K * N));
        CHK(check_ptr(p.mC_i, M * N));
        if (mode != MPC_TAG_COMPACT_TRUNC || p.mZ_i != nullptr) CHK(check_ptr(p.mZ_i, M * N));
        if (mode == MPC_TAG_FULL) {
            g.push_back(mpcl::GemmArgs{M, K, N, w, (const u64*)p.E, (const u64*)p.F, (const u64*)p.mA_i,
                                       (const u64*)p.mB_i, (const u64*)p.mC_i, (u64*)p.mZ_i, mpcl::COEF_ALPHA,
                                       (const u64*)p.alpha_i, 0});
            continue;
        }
        CHK(check_ptr(p.mR_i, M * N));
        CHK(check_ptr(p.Dtilde, M * N));
        CHK(check_ptr(p.chi, N));
        CHK(check_ptr(p.mDc_i, M));
        CHK(check_ptr(p.Dc, M));
        c.push_back(mpcl::CompactArgs{M, K, N, w, mode == MPC_TAG_COMPACT ? 1 : 0, (const u64*)p.alpha_i,
                                      (const u64*)p.E, (const u64*)p.F, (const u64*)p.mA_i, (const u64*)p.mB_i,
                                      (const u64*)p.mC_i, (const u64*)p.mR_i, (const u64*)p.Dtilde,
                                      (const u64*)p.chi, (u64*)p.mZ_i, (u64*)p.mDc_i, (u64*)p.Dc});
    }
    if (mode == MPC_TAG_FULL) return run_gemm_group(layers, count, g.data(), ws, ws_bytes, st);
    const size_t need = group_compact_ws(layers, count);
    if (need > 0) {
        if (!ws || ws_bytes < need) return MPC_E_WORKSPACE;
        if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return MPC_E_ALIGN;
    }
    std::vector<char*> slices((size_t)count);
    char* cur = static_cast<char*>(ws);
    for (int i = 0; i < count; ++i) {
        slices[i] = cur;
        cur += (mpcl::compact_workspace(c[i].M, c[i].K, c[i].N, c[i].words) + 255) & ~size_t(255);
    }
    return cuda_status(mpcl::launch_compact_grouped(c.data(), count, slices.data(), st));
}

size_t mpc_workspace_size_grouped(const mpc_layer* layers, int count, int which) {
    if (count <= 0 || !layers) return 0;
    for (int i = 0; i < count; ++i) {
        if (check_layer(&layers[i]) != MPC_OK || !same_ring(layers[i].ring, layers[0].ring)) return 0;
    }
    switch (which) {
        case MPC_WS_SHARE:
        case MPC_WS_TAG_FULL: return group_gemm_ws(layers, count);
        case MPC_WS_TAG_COMPACT: return group_compact_ws(layers, count);
        default: return 0;
    }
}

int mpc_launch_count_grouped(const mpc_layer* layers, int count, int which) {
    if (count < 0) return MPC_E_SHAPE;
    if (count == 0) return 0;
    if (!layers) return MPC_E_NULL;
    int n = 0;
    std::vector<int64_t> tM, tK, tN;   // the tensor-core layers
    for (int i = 0; i < count; ++i) {
        CHK(check_layer(&layers[i]));
        if (!same_ring(layers[i].ring, layers[0].ring)) return MPC_E_RING;
        const mpc_layer& L = layers[i];
        if (which == MPC_WS_SHARE || which == MPC_WS_TAG_FULL) {
            if (on_tc(L)) {
                tM.push_back(L.M);
                tK.push_back(L.K);
                tN.push_back(L.N);
            } else if (L.M > 0 && L.N > 0) {
                n += 1;
            }
        } else if (which == MPC_WS_TAG_COMPACT) {
            // counted below for the whole group
        } else {
            return MPC_E_MODE;
        }
    }
    if (which == MPC_WS_TAG_COMPACT) {
        std::vector<int64_t> M((size_t)count), K((size_t)count), N((size_t)count);
        for (int i = 0; i < count; ++i) {
            M[i] = layers[i].M;
            K[i] = layers[i].K;
            N[i] = layers[i].N;
        }
        return mpcl::compact_grouped_launches(M.data(), K.data(), N.data(), count);
    }
    return n + mpcl::gemm_tc_grouped_launches(tM.data(), tK.data(), tN.data(), (int)tM.size(), layers[0].ring.words);
}

int mpc_tag_check_grouped(const mpc_layer* layers, int count, const mpc_check_ptrs* ptrs, void* stream) {
    if (count < 0) return MPC_E_SHAPE;
    if (count == 0) return MPC_OK;
    if (!layers || !ptrs) return MPC_E_NULL;
    std::vector<int64_t> M((size_t)count);
    std::vector<const u64*> al(count), ch(count), dc(count), md(count);
    std::vector<u64*> cs(count);
    for (int i = 0; i < count; ++i) {
        const mpc_layer* L = &layers[i];
        CHK(check_layer(L));
        if (!same_ring(L->ring, layers[0].ring)) return MPC_E_RING;
        const mpc_check_ptrs& p = ptrs[i];
        CHK(check_ptr(p.alpha_i, 1));
        CHK(check_ptr(p.cs_i, 1));
        CHK(check_ptr(p.chi_hat, L->M));
        CHK(check_ptr(p.Dc, L->M));
        CHK(check_ptr(p.mDc_i, L->M));
        M[i] = L->M;
        al[i] = (const u64*)p.alpha_i;
        ch[i] = (const u64*)p.chi_hat;
        dc[i] = (const u64*)p.Dc;
        md[i] = (const u64*)p.mDc_i;
        cs[i] = (u64*)p.cs_i;
    }
    return cuda_status(mpcl::launch_check_compact_grouped(count, layers[0].ring.words, M.data(), al.data(), ch.data(),
                                                          dc.data(), md.data(), cs.data(), (cudaStream_t)stream));
}

}  // extern "C"
