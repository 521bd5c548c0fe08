// tune.cu -- the per-shape launch table (autotuner) of the ring GEMM.
//
// Every GEMM path computes the same exact sums, so the choice of path and
// tiling changes only the time a layer takes.  For each layer shape
// (ring width, M, K, N) the table holds a Choice: the tensor-core kernel with
// a tile height (128 or 64 rows) and a row-tile swizzle width, or the
// integer-pipe kernels with a tile height (64 or 16 rows; 0 = by grid size)
// and a K-split target.  Shapes not in the table use
// the built-in heuristic (gemm_tc_eligible; 64-row tiles for M <= 64).
// mpc_autotune times the candidates of each distinct shape on the caller's
// stream and stores the fastest; the table can be saved to and loaded from a
// text file:
//     mpclinear-autotune 2
//     <words> <M> <K> <N> <path> <rows> <swizzle> <waves>   (one line per shape)
// (version 1 files, without <rows>, load as 128-row tiles).  The table is
// process-wide and guarded by a mutex.
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "kernels.h"
#include "mpclinear.h"

namespace mpcl {

// the wide tensor-core tile: this many rows by 128 columns (32 for Z_2^64, 16 for Z_2^128)
int wide_tile_rows(int words) { return words == 1 ? 32 : 16; }

namespace {

using Key = std::tuple<int, int64_t, int64_t, int64_t>;

std::mutex g_mu;
std::map<Key, Choice>& table() {
    static std::map<Key, Choice> t;
    return t;
}

bool choice_ok(const Choice& c, int64_t M, int64_t K, int64_t N, int words) {
    if (c.path == 1)
        return (c.rows == 64 || c.rows == 128 || c.rows == wide_tile_rows(words) || c.rows == TALL_TILE_ROWS) &&
               gemm_tc_feasible(M, K, N, words, c.rows) && c.gm >= 1 && c.gm <= 64;
    return c.path == 0 && c.waves >= 0 && c.waves <= 64 && (c.rows == 0 || c.rows == 16 || c.rows == 64);
}

// Built-in tile: the wide tile (128 columns on the TMEM lanes, the layer's rows
// in the stacked operand) for layers of at most two of its row tiles, 64-row
// tiles up to 64 rows, 128-row tiles above (an M = 64 MMA costs as much as an
// M = 128 one).
int default_rows(int64_t M, int64_t K, int64_t N, int words) {
    if (M <= 2 * wide_tile_rows(words)) return wide_tile_rows(words);
    // Z_2^128 layers of 33-64 rows: an M = 64 MMA costs as much as an M = 128
    // one, and the wide tile is faster once it has a work unit per SM (measured:
    // 64 x 2304 x 256 46 -> 39 us, 64 x 4608 x 512 129 -> 94 us, 48 x 2304 x 256
    // 45 -> 37 us; but 64 x 576 x 128, 72 wide units, 23 -> 27 us)
    if (words == 2 && M <= 64) {
        const int64_t rb = (M + 15) / 16, ct = (N + 127) / 128, iv = (2 * K + 63) / 64;
        if (rb * ct * iv >= 152) return wide_tile_rows(words);
    }
    if (M <= 64) return 64;
    // tall and narrow layers: the left operand's digit planes would cost an HBM
    // round trip comparable to the GEMM itself, so the GEMM converts them in
    // place.  Measured share calls, 128-row tile -> tall tile: Z_2^64
    // 32768 x 576 x 64 284 -> 184 us and 4096 x 1152 x 128 115 -> 100 us, equal
    // at 1024 x 576 x 64 (its small R' prologue runs on few blocks); Z_2^128
    // 32768 x 576 x 64 821 -> 616 us, 1024 x 576 x 64 51 -> 47 us,
    // 8192 x 1152 x 128 632 -> 585 us, but 2048 x 1152 x 128 196 -> 201 us and
    // wider layers mostly slower
    const int64_t tall_from = N <= 64 ? (words == 1 ? 2048 : 1024) : 4096;
    if (N <= 128 && M >= tall_from && gemm_tc_feasible(M, K, N, words, TALL_TILE_ROWS))
        return TALL_TILE_ROWS;
    return 128;
}

}  // namespace

Choice gemm_choice(int64_t M, int64_t K, int64_t N, int words) {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = table().find(Key{words, M, K, N});
        if (it != table().end()) return it->second;
    }
    Choice c;
    c.path = gemm_tc_eligible(M, K, N, words) ? 1 : 0;
    c.gm = 0;
    c.waves = 0;
    c.tuned = 0;
    c.rows = c.path == 1 ? default_rows(M, K, N, words) : 0;
    return c;
}

}  // namespace mpcl

namespace {

int check_shape(const mpc_layer* L) {
    if (!L) return MPC_E_NULL;
    const mpc_ring& r = L->ring;
    if (!((r.words == 1 || r.words == 2) && r.k >= 1 && r.s >= 1 && r.k + r.s == 64 * r.words)) return MPC_E_RING;
    if (L->M < 0 || L->K < 0 || L->N < 0) return MPC_E_SHAPE;
    return MPC_OK;
}

// one timed candidate: the best of `reps` runs after a warm-up run, in ms
float time_candidate(const mpcl::GemmArgs& a, const mpcl::Choice& c, void* ws, size_t ws_bytes, cudaStream_t st,
                     cudaEvent_t e0, cudaEvent_t e1, int reps, bool* ok) {
    mpcl::GemmArgs g = a;
    g.gm = c.gm;
    g.simt_waves = c.waves;
    g.rows = c.rows;
    auto run = [&]() -> cudaError_t {
        return c.path == 1 ? mpcl::launch_gemm_tc(g, ws, ws_bytes, st) : mpcl::launch_gemm_simt(g, st);
    };
    *ok = false;
    if (run() != cudaSuccess) return 0.f;
    float best = -1.f;
    for (int r = 0; r < reps; ++r) {
        if (cudaEventRecord(e0, st) != cudaSuccess) return 0.f;
        if (run() != cudaSuccess) return 0.f;
        if (cudaEventRecord(e1, st) != cudaSuccess) return 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess) return 0.f;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return 0.f;
        if (best < 0.f || ms < best) best = ms;
    }
    *ok = true;
    return best;
}

}  // namespace

extern "C" {

int mpc_autotune(const mpc_layer* layers, int count, void* stream) {
    if (count < 0) return MPC_E_SHAPE;
    if (count == 0) return 0;
    if (!layers) return MPC_E_NULL;
    for (int i = 0; i < count; ++i) {
        int s = check_shape(&layers[i]);
        if (s != MPC_OK) return s;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return MPC_E_CUDA;
    int tuned = 0, status = MPC_OK;
    std::map<std::tuple<int, int64_t, int64_t, int64_t>, bool> seen;
    for (int i = 0; i < count && status == MPC_OK; ++i) {
        const mpc_layer& L = layers[i];
        const int64_t M = L.M, K = L.K, N = L.N;
        const int w = L.ring.words;
        if (M == 0 || N == 0) continue;
        auto key = std::make_tuple(w, M, K, N);
        if (seen.count(key)) continue;
        seen[key] = true;
        std::vector<mpcl::Choice> cands;
        const bool tc = mpcl::gemm_tc_feasible(M, K, N, w);
        const double macs = 2.0 * (double)M * (double)K * (double)N;
        // tiles: 64 rows only where the layer has at most 64 rows (it would
        // double the MMA work of taller layers), the wide tile up to 128 rows
        if (tc)
            for (int rows : {128, 64, mpcl::wide_tile_rows(w), mpcl::TALL_TILE_ROWS}) {
                if (rows == 64 && M > 64) continue;
                if (rows == mpcl::TALL_TILE_ROWS && M < 128) continue;
                if (rows == mpcl::wide_tile_rows(w) && M > 128) continue;
                if (!mpcl::gemm_tc_feasible(M, K, N, w, rows)) continue;
                for (int gm : {1, 4, 8, 16}) cands.push_back(mpcl::Choice{1, gm, 0, 1, rows});
            }
        // the integer pipes are far slower on large products: not timed there;
        // their tile height (64 or 16 rows) matters only above M = 8
        if (!tc || macs < 2147483648.0)
            for (int rows : {64, 16}) {
                if (rows == 16 && M <= 8) continue;
                for (int wv : {1, 2, 4, 8}) cands.push_back(mpcl::Choice{0, 0, wv, 1, M <= 8 ? 0 : rows});
            }
        // operands (contents do not matter for the time: every path is exact)
        const size_t e = 8 * (size_t)w;
        const size_t b_mk = e * (size_t)(M * K), b_kn = e * (size_t)(K * N), b_mn = e * (size_t)(M * N);
        const size_t ws_bytes = tc ? mpcl::gemm_tc_workspace(M, K, N, w) : 0;
        void *E = nullptr, *X = nullptr, *B = nullptr, *F = nullptr, *C = nullptr, *Z = nullptr, *ws = nullptr;
        bool alloc = cudaMalloc(&E, b_mk > 0 ? b_mk : 16) == cudaSuccess &&
                     cudaMalloc(&X, b_mk > 0 ? b_mk : 16) == cudaSuccess &&
                     cudaMalloc(&B, b_kn > 0 ? b_kn : 16) == cudaSuccess &&
                     cudaMalloc(&F, b_kn > 0 ? b_kn : 16) == cudaSuccess &&
                     cudaMalloc(&C, b_mn) == cudaSuccess && cudaMalloc(&Z, b_mn) == cudaSuccess &&
                     (ws_bytes == 0 || cudaMalloc(&ws, ws_bytes) == cudaSuccess);
        if (alloc) {
            cudaMemsetAsync(E, 0, b_mk, st);
            cudaMemsetAsync(X, 0, b_mk, st);
            cudaMemsetAsync(B, 0, b_kn, st);
            cudaMemsetAsync(F, 0, b_kn, st);
            cudaMemsetAsync(C, 0, b_mn, st);
            mpcl::GemmArgs a{M, K, N, w, (const mpcl::u64*)E, (const mpcl::u64*)F, (const mpcl::u64*)X,
                             (const mpcl::u64*)B, (const mpcl::u64*)C, (mpcl::u64*)Z, mpcl::COEF_ZERO, nullptr, 0};
            float best = -1.f;
            mpcl::Choice pick{};
            for (const auto& c : cands) {
                bool ok = false;
                const float ms = time_candidate(a, c, ws, ws_bytes, st, e0, e1, 3, &ok);
                if (!ok) {
                    status = MPC_E_CUDA;
                    break;
                }
                if (best < 0.f || ms < best) {
                    best = ms;
                    pick = c;
                }
            }
            if (status == MPC_OK && best >= 0.f) {
                std::lock_guard<std::mutex> lk(mpcl::g_mu);
                mpcl::table()[key] = pick;
                ++tuned;
            }
        } else {
            status = MPC_E_CUDA;
        }
        cudaStreamSynchronize(st);
        for (void* p : {E, X, B, F, C, Z, ws})
            if (p) cudaFree(p);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return status == MPC_OK ? tuned : status;
}

int mpc_autotune_set(const mpc_layer* layer, int path, int tile_rows, int swizzle, int waves) {
    int s = check_shape(layer);
    if (s != MPC_OK) return s;
    mpcl::Choice c{path, swizzle, waves, 1, tile_rows};
    if (!mpcl::choice_ok(c, layer->M, layer->K, layer->N, layer->ring.words)) return MPC_E_MODE;
    std::lock_guard<std::mutex> lk(mpcl::g_mu);
    mpcl::table()[std::make_tuple(layer->ring.words, layer->M, layer->K, layer->N)] = c;
    return MPC_OK;
}

int mpc_autotune_choice(const mpc_layer* layer, int* path, int* tile_rows, int* swizzle, int* waves) {
    int s = check_shape(layer);
    if (s != MPC_OK) return s;
    const mpcl::Choice c = mpcl::gemm_choice(layer->M, layer->K, layer->N, layer->ring.words);
    if (path) *path = c.path;
    if (tile_rows) *tile_rows = c.rows;
    if (swizzle) *swizzle = c.gm;
    if (waves) *waves = c.waves;
    return c.tuned ? 1 : 0;
}

int mpc_autotune_clear(void) {
    std::lock_guard<std::mutex> lk(mpcl::g_mu);
    const int n = (int)mpcl::table().size();
    mpcl::table().clear();
    return n;
}

int mpc_autotune_save(const char* path) {
    if (!path) return MPC_E_NULL;
    FILE* f = std::fopen(path, "w");
    if (!f) return MPC_E_IO;
    std::lock_guard<std::mutex> lk(mpcl::g_mu);
    std::fprintf(f, "mpclinear-autotune 2\n");
    for (const auto& kv : mpcl::table()) {
        const auto& k = kv.first;
        const auto& c = kv.second;
        std::fprintf(f, "%d %lld %lld %lld %d %d %d %d\n", std::get<0>(k), (long long)std::get<1>(k),
                     (long long)std::get<2>(k), (long long)std::get<3>(k), c.path, c.rows, c.gm, c.waves);
    }
    const int n = (int)mpcl::table().size();
    return std::fclose(f) == 0 ? n : MPC_E_IO;
}

int mpc_autotune_load(const char* path) {
    if (!path) return MPC_E_NULL;
    FILE* f = std::fopen(path, "r");
    if (!f) return MPC_E_IO;
    int version = 0;
    if (std::fscanf(f, "mpclinear-autotune %d", &version) != 1 || (version != 1 && version != 2)) {
        std::fclose(f);
        return MPC_E_IO;
    }
    std::vector<std::pair<std::tuple<int, int64_t, int64_t, int64_t>, mpcl::Choice>> rows;
    int w, path_, tr = 128, gm, waves;
    long long M, K, N;
    auto next = [&]() {
        if (version == 1) return std::fscanf(f, "%d %lld %lld %lld %d %d %d", &w, &M, &K, &N, &path_, &gm, &waves) == 7;
        return std::fscanf(f, "%d %lld %lld %lld %d %d %d %d", &w, &M, &K, &N, &path_, &tr, &gm, &waves) == 8;
    };
    while (next()) {
        mpcl::Choice c{path_, gm, waves, 1, version == 1 ? (path_ == 1 ? 128 : 0) : tr};
        if ((w != 1 && w != 2) || M < 0 || K < 0 || N < 0 || !mpcl::choice_ok(c, M, K, N, w)) {
            std::fclose(f);
            return MPC_E_IO;
        }
        rows.push_back({std::make_tuple(w, (int64_t)M, (int64_t)K, (int64_t)N), c});
    }
    const bool at_end = std::feof(f) != 0;
    std::fclose(f);
    if (!at_end) return MPC_E_IO;
    std::lock_guard<std::mutex> lk(mpcl::g_mu);
    for (const auto& r : rows) mpcl::table()[r.first] = r.second;
    return (int)rows.size();
}

}  // extern "C"
