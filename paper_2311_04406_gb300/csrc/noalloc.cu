// noalloc.cu -- mpc_linear_tag_compact_noalloc: the CompactTag tag of
// mpc_linear_tag(MPC_TAG_COMPACT) for callers that cannot allocate device
// memory.  The paper has no counterpart; this is a deployment convenience.
//
// Who needs it: a host runtime that reaches this library through a plain C
// FFI and has no CUDA allocator of its own, or a serving process whose device
// memory is wholly owned by another framework's pool, so that it can neither
// call cudaMalloc nor hand over a workspace.  Instead of a caller workspace,
// the kernels' scratch (the per-chunk partial dot products and the compressed
// K-vectors) lives in one file-scope device array of MPC_NOALLOC_SCRATCH_BYTES.
//
// Rules of use:
//   * The array exists once per device that loads the library and is held
//     until the process exits.
//   * Host code cannot use the array's name as a device address.  The first
//     call on each device looks the address up with cudaGetSymbolAddress
//     (with that device current) and caches it; make that first call before
//     any stream capture.
//   * Every call shares the array and it keeps the last call's contents.  No
//     part of it needs to start at zero: each call writes every scratch word
//     it later reads.  Calls whose kernels overlap on the GPU (e.g. issued on
//     two streams without ordering) race on the array: order them on one
//     stream or with events.
//   * A layer whose scratch need, mpc_workspace_size(layer,
//     MPC_WS_TAG_COMPACT), exceeds MPC_NOALLOC_SCRATCH_BYTES is rejected with
//     MPC_E_SCRATCH_LIMIT before anything is launched.
//   * Nothing here calls cudaMalloc, cudaFree or any allocating routine.
#include <cstdint>
#include <mutex>

#include "mpclinear.h"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = MPC_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// device address of g_scratch on the current device (looked up once)
int scratch_address(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MPC_E_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return MPC_E_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return MPC_OK;
}

bool aligned_or_empty(const void* p, int64_t elems) {
    if (elems == 0) return true;
    return p != nullptr && reinterpret_cast<uintptr_t>(p) % 16 == 0;
}

}  // namespace

extern "C" int mpc_linear_tag_compact_noalloc(
    const mpc_layer* L, const uint64_t* alpha_i, const uint64_t* E, const uint64_t* F,
    const uint64_t* mA_i, const uint64_t* mB_i, const uint64_t* mC_i, const uint64_t* mR_i,
    const uint64_t* Dtilde, const uint64_t* chi, uint64_t* mZ_i, uint64_t* mDc_i, uint64_t* Dc,
    void* stream) {
    if (!L) return MPC_E_NULL;
    const mpc_ring& r = L->ring;
    if (!((r.words == 1 || r.words == 2) && r.k >= 1 && r.s >= 1 && r.k + r.s == 64 * r.words))
        return MPC_E_RING;
    const int64_t M = L->M, K = L->K, N = L->N;
    const int64_t lim = int64_t(1) << 31, elim = int64_t(1) << 36;
    if (M < 0 || K < 0 || N < 0 || M > lim || K > lim || N > lim) return MPC_E_SHAPE;
    if (M * K > elim || K * N > elim || M * N > elim) return MPC_E_SHAPE;
    if (L->nparties < 1 || L->party < 0 || L->party >= L->nparties) return MPC_E_PARTY;
    const struct { const void* p; int64_t n; } ptrs[] = {
        {alpha_i, 1}, {E, M * K}, {mA_i, M * K}, {F, K * N}, {mB_i, K * N}, {mC_i, M * N},
        {mR_i, M * N}, {Dtilde, M * N}, {chi, N}, {mZ_i, M * N}, {mDc_i, M}, {Dc, M}};
    for (const auto& q : ptrs) {
        if (q.n != 0 && q.p == nullptr) return MPC_E_NULL;
        if (!aligned_or_empty(q.p, q.n)) return MPC_E_ALIGN;
    }
    if (mpcl::compact_workspace(M, K, N, r.words) > kScratchBytes) return MPC_E_SCRATCH_LIMIT;
    if (M == 0) return MPC_OK;
    void* scratch = nullptr;
    int st = scratch_address(&scratch);
    if (st != MPC_OK) return st;
    mpcl::CompactArgs c{M, K, N, r.words, 1, (const mpcl::u64*)alpha_i, (const mpcl::u64*)E,
                        (const mpcl::u64*)F, (const mpcl::u64*)mA_i, (const mpcl::u64*)mB_i,
                        (const mpcl::u64*)mC_i, (const mpcl::u64*)mR_i, (const mpcl::u64*)Dtilde,
                        (const mpcl::u64*)chi, (mpcl::u64*)mZ_i, (mpcl::u64*)mDc_i, (mpcl::u64*)Dc};
    return mpcl::launch_compact(c, scratch, kScratchBytes, (cudaStream_t)stream) == cudaSuccess
               ? MPC_OK : MPC_E_CUDA;
}
