// compact.cu -- the CompactTag tag of one party (§3.1-§3.3), HBM-bound.
//
//   a3  mZ   = mR - alpha * D~                       (Fig. Pi_OptMAC step 3)
//   a4  mR.chi, D~.chi, mC.chi (M) ; mB.chi, F.chi (K) (Fig. Pi_Compress)
//   a5  mZc  = mC.chi + E.(mB.chi) + mA.(F.chi) + alpha * E.(F.chi)
//       mDc  = mR.chi - mZc,  Dc = D~.chi            (Eq. (compute-zcomptag))
//
// In Z_2^64 the two terms in E are one product: E.(mB.chi) + alpha * E.(F.chi)
// = E.(mB.chi + alpha * F.chi) mod 2^64 (the ring is commutative and the sums
// distribute).  The rows pass stores w = mB.chi + alpha * F.chi in place of
// mB.chi (chunk by chunk: the sum over chunks is linear), so the vec pass
// multiplies each element of E and mA once: mZc = mC.chi + E.w + mA.(F.chi).
// In Z_2^128 the vec pass keeps the three products (w = mB.chi): measured on
// GB300, 160 us against 188 us for the 32768 x 576 x 64 layer's call, where the
// Z_2^64 layers gain 2-5 % from the fold.
//
// Up to three launches on the caller's stream:
//   1. rows_kernel   one pass over the five N-wide matrices.  A warp owns a
//                    (row, column-chunk) task: it streams mR, D~, mC (writing
//                    mZ on the fly) or mB, F, and leaves per-chunk partial
//                    dot products with chi in the workspace.  Each input word
//                    is read from HBM exactly once.
//   2. finalize_kernel  sums the K-side partials into the vectors w (or mB.chi), F.chi
//                    (only when a row is split into several chunks; with one
//                    chunk the partials are those vectors and vec reads them).
//   3. vec_kernel    one warp per output row: the two M x K GEMVs over E and
//                    mA against those vectors, then mZc, mDc and Dc.
// Every sum is a wrapping sum mod 2^(64 W), so the split into chunks does not
// change any result bit.
#include <new>

#include "common.cuh"
#include "kernels.h"
#include "sm100_ptx.cuh"

namespace mpcl {

namespace {

constexpr int WARPS = 8;
constexpr int NT = WARPS * 32;

template <int W>
__device__ __forceinline__ typename Elem<W>::T warp_sum(typename Elem<W>::T v) {
    if constexpr (W == 1) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            u64 lo = (u64)v, hi = (u64)(v >> 64);
            lo = __shfl_xor_sync(0xffffffffu, lo, o);
            hi = __shfl_xor_sync(0xffffffffu, hi, o);
            v += (u128)lo | ((u128)hi << 64);
        }
        return v;
    }
}

struct Split {
    int64_t S;    // chunks per row
    int64_t cw;   // columns per chunk (even)
};

Split choose_split(int64_t M, int64_t K, int64_t N) {
    Split sp{1, N < 2 ? 2 : ((N + 1) / 2) * 2};
    const int64_t rows = M + K;
    const int64_t want_warps = 152 * 32;
    if (rows > 0 && rows < want_warps && N > 1024) {
        int64_t S = (want_warps + rows - 1) / rows;
        int64_t Smax = (N + 511) / 512;
        if (S > Smax) S = Smax;
        if (S < 1) S = 1;
        int64_t cw = (N + S - 1) / S;
        cw = ((cw + 63) / 64) * 64;
        sp.S = (N + cw - 1) / cw;
        sp.cw = cw;
    }
    return sp;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct WsLayout {
    size_t pmr, pd, pmc, qmb, qf, vmb, vf, total;
};

WsLayout ws_layout(int64_t M, int64_t K, int64_t N, int words) {
    Split sp = choose_split(M, K, N);
    size_t e = 8 * (size_t)words;
    WsLayout L{};
    size_t off = 0;
    L.pmr = off; off += align256(e * M * sp.S);
    L.pd = off;  off += align256(e * M * sp.S);
    L.pmc = off; off += align256(e * M * sp.S);
    L.qmb = off; off += align256(e * K * sp.S);
    L.qf = off;  off += align256(e * K * sp.S);
    L.vmb = off; off += align256(e * K);
    L.vf = off;  off += align256(e * K);
    L.total = off;
    return L;
}

struct RowsParams {
    int64_t M, K, N, S, cw;
    const u64 *alpha, *mR, *Dt, *mC, *mB, *F, *chi;
    u64* mZ;   // NULL: the OptMAC tag is not written
    u64 *pmr, *pd, *pmc, *qmb, *qf;
    int with_eu;   // the E.(F.chi) term is present (Z_2^64: folded into the K-side partial of mB.chi)
};

// VEC = 2: two Z_2^64 elements per 16-byte access (needs even N).  Warp
// task g of one layer.
template <int W, int VEC>
__device__ __forceinline__ void rows_body(const RowsParams& p, int64_t g, int lane) {
    using T = typename Elem<W>::T;
    const int64_t tasksA = p.M * p.S, tasksB = p.K * p.S;
    if (g >= tasksA + tasksB) return;
    const bool isA = g < tasksA;
    const int64_t t = isA ? g : g - tasksA;
    const int64_t row = t / p.S, s = t % p.S;
    const int64_t c0 = s * p.cw;
    int64_t c1 = c0 + p.cw;
    if (c1 > p.N) c1 = p.N;
    const T alpha = ld_elem<W>(p.alpha, 0);
    T s1 = 0, s2 = 0, s3 = 0;
    if (isA) {
        const int64_t base = row * p.N;
        if constexpr (VEC == 2) {
            for (int64_t c = c0 + 2 * lane; c < c1; c += 64) {
                ulonglong2 x = __ldg(reinterpret_cast<const ulonglong2*>(p.chi + c));
                ulonglong2 r = ld_stream2(p.mR + base + c);
                ulonglong2 d = ld_stream2(p.Dt + base + c);
                ulonglong2 m = ld_stream2(p.mC + base + c);
                s1 += r.x * x.x + r.y * x.y;
                s2 += d.x * x.x + d.y * x.y;
                s3 += m.x * x.x + m.y * x.y;
                if (p.mZ) {
                    ulonglong2 z;
                    z.x = r.x - alpha * d.x;
                    z.y = r.y - alpha * d.y;
                    st_stream2(p.mZ + base + c, z);
                }
            }
        } else {
            for (int64_t c = c0 + lane; c < c1; c += 32) {
                T x = ldg_elem<W>(p.chi, c);
                T r = ldg_elem<W>(p.mR, base + c);
                T d = ldg_elem<W>(p.Dt, base + c);
                T m = ldg_elem<W>(p.mC, base + c);
                s1 += r * x;
                s2 += d * x;
                s3 += m * x;
                if (p.mZ) st_elem<W>(p.mZ, base + c, r - alpha * d);
            }
        }
        s1 = warp_sum<W>(s1);
        s2 = warp_sum<W>(s2);
        s3 = warp_sum<W>(s3);
        if (lane == 0) {
            st_elem<W>(p.pmr, t, s1);
            st_elem<W>(p.pd, t, s2);
            st_elem<W>(p.pmc, t, s3);
        }
    } else {
        const int64_t base = row * p.N;
        if constexpr (VEC == 2) {
            for (int64_t c = c0 + 2 * lane; c < c1; c += 64) {
                ulonglong2 x = __ldg(reinterpret_cast<const ulonglong2*>(p.chi + c));
                ulonglong2 b = ld_stream2(p.mB + base + c);
                ulonglong2 f = ld_stream2(p.F + base + c);
                s1 += b.x * x.x + b.y * x.y;
                s2 += f.x * x.x + f.y * x.y;
            }
        } else {
            for (int64_t c = c0 + lane; c < c1; c += 32) {
                T x = ldg_elem<W>(p.chi, c);
                s1 += ldg_elem<W>(p.mB, base + c) * x;
                s2 += ldg_elem<W>(p.F, base + c) * x;
            }
        }
        s1 = warp_sum<W>(s1);
        s2 = warp_sum<W>(s2);
        if (W == 1 && p.with_eu) s1 += alpha * s2;   // the chunk's part of w = mB.chi + alpha * F.chi
        if (lane == 0) {
            st_elem<W>(p.qmb, t, s1);
            st_elem<W>(p.qf, t, s2);
        }
    }
}

template <int W, int VEC>
__global__ void __launch_bounds__(NT) rows_kernel(RowsParams p) {
    ptx::grid_dep_launch();   // finalize and vec wait for this grid before reading
    ptx::grid_dep_wait();     // launched as a dependent of the kernel before it
    rows_body<W, VEC>(p, (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5), threadIdx.x & 31);
}

template <int W>
__device__ __forceinline__ void finalize_body(int64_t K, int64_t S, const u64* qmb, const u64* qf, u64* vmb,
                                              u64* vf, int64_t id, int64_t nthreads) {
    using T = typename Elem<W>::T;
    for (int64_t k = id; k < K; k += nthreads) {
        T a = 0, b = 0;
        for (int64_t s = 0; s < S; ++s) {
            a += ld_elem<W>(qmb, k * S + s);
            b += ld_elem<W>(qf, k * S + s);
        }
        st_elem<W>(vmb, k, a);
        st_elem<W>(vf, k, b);
    }
}

template <int W>
__global__ void finalize_kernel(int64_t K, int64_t S, const u64* qmb, const u64* qf,
                                u64* vmb, u64* vf) {
    ptx::grid_dep_launch();
    ptx::grid_dep_wait();   // the rows pass's partials
    finalize_body<W>(K, S, qmb, qf, vmb, vf, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                     (int64_t)gridDim.x * blockDim.x);
}

struct VecParams {
    int64_t M, K, S;
    int with_eu;
    const u64 *alpha, *E, *mA, *vmb, *vf, *pmr, *pd, *pmc;   // vmb: w (Z_2^64) or mB.chi (Z_2^128)
    u64 *mDc, *Dc;
};

// `wpr` warps share one row (1, 2, 4 or 8), each taking every wpr-th chunk of
// 32 (or 64, vectorised) K values; their partial sums meet in shared memory.
template <int W, int VEC>
__device__ __forceinline__ void vec_body(const VecParams& p, int wpr, int64_t blk) {
    using T = typename Elem<W>::T;
    constexpr int NP = W == 1 ? 2 : 3;   // partial sums per row
    __shared__ T part[NP][WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rows_per_block = WARPS / wpr;
    const int64_t r = blk * rows_per_block + warp / wpr;
    const int sub = warp % wpr;
    T e_w = 0, ma_u = 0, e_u = 0;   // E.w, mA.(F.chi) and (Z_2^128) E.(F.chi) of row r
    if (r < p.M) {
        const int64_t base = r * p.K;
        if constexpr (VEC == 2) {
#pragma unroll 4
            for (int64_t k = 2 * (sub * 32 + lane); k < p.K; k += 64 * wpr) {
                ulonglong2 e = __ldg(reinterpret_cast<const ulonglong2*>(p.E + base + k));
                ulonglong2 ma = __ldg(reinterpret_cast<const ulonglong2*>(p.mA + base + k));
                ulonglong2 w = *reinterpret_cast<const ulonglong2*>(p.vmb + k);
                ulonglong2 u = *reinterpret_cast<const ulonglong2*>(p.vf + k);
                e_w += e.x * w.x + e.y * w.y;
                ma_u += ma.x * u.x + ma.y * u.y;
            }
        } else {
#pragma unroll 4
            for (int64_t k = sub * 32 + lane; k < p.K; k += 32 * wpr) {
                T e = ldg_elem<W>(p.E, base + k);
                T ma = ldg_elem<W>(p.mA, base + k);
                T w = ld_elem<W>(p.vmb, k);
                T u = ld_elem<W>(p.vf, k);
                e_w += e * w;
                ma_u += ma * u;
                if constexpr (W == 2) e_u += e * u;
            }
        }
        e_w = warp_sum<W>(e_w);
        ma_u = warp_sum<W>(ma_u);
        if constexpr (W == 2) e_u = warp_sum<W>(e_u);
    }
    if (lane == 0) {
        part[0][warp] = e_w;
        part[1][warp] = ma_u;
        if constexpr (W == 2) part[2][warp] = e_u;
    }
    __syncthreads();
    if (r < p.M && sub == 0 && lane == 0) {
        for (int j = 1; j < wpr; ++j) {
            e_w += part[0][warp + j];
            ma_u += part[1][warp + j];
            if constexpr (W == 2) e_u += part[2][warp + j];
        }
        T mrc = 0, dc = 0, mcc = 0;
        for (int64_t s = 0; s < p.S; ++s) {
            mrc += ld_elem<W>(p.pmr, r * p.S + s);
            dc += ld_elem<W>(p.pd, r * p.S + s);
            mcc += ld_elem<W>(p.pmc, r * p.S + s);
        }
        T mzc = mcc + e_w + ma_u;
        if (W == 2 && p.with_eu) mzc += ld_elem<W>(p.alpha, 0) * e_u;
        st_elem<W>(p.mDc, r, mrc - mzc);
        st_elem<W>(p.Dc, r, dc);
    }
}

template <int W, int VEC>
__global__ void __launch_bounds__(NT) vec_kernel(VecParams p, int wpr) {
    ptx::grid_dep_wait();   // the rows partials and the finalized vectors
    vec_body<W, VEC>(p, wpr, blockIdx.x);
}

// K < 64: one thread per row, the two compressed K-vectors staged in shared
// memory (a warp per row would leave most lanes idle)
constexpr int SMALL_K = 64;

template <int W>
__device__ __forceinline__ void vec_small_body(const VecParams& p, int64_t blk) {
    using T = typename Elem<W>::T;
    __shared__ T smb[SMALL_K], sf[SMALL_K];
    for (int k = threadIdx.x; k < p.K; k += NT) {
        smb[k] = ld_elem<W>(p.vmb, k);
        sf[k] = ld_elem<W>(p.vf, k);
    }
    __syncthreads();
    const int64_t r = blk * NT + threadIdx.x;
    if (r >= p.M) return;
    T e_w = 0, ma_u = 0, e_u = 0;
    const int64_t base = r * p.K;
    for (int k = 0; k < (int)p.K; ++k) {
        const T e = ldg_elem<W>(p.E, base + k);
        const T ma = ldg_elem<W>(p.mA, base + k);
        e_w += e * smb[k];
        ma_u += ma * sf[k];
        if constexpr (W == 2) e_u += e * sf[k];
    }
    T mrc = 0, dc = 0, mcc = 0;
    for (int64_t s = 0; s < p.S; ++s) {
        mrc += ld_elem<W>(p.pmr, r * p.S + s);
        dc += ld_elem<W>(p.pd, r * p.S + s);
        mcc += ld_elem<W>(p.pmc, r * p.S + s);
    }
    T mzc = mcc + e_w + ma_u;
    if (W == 2 && p.with_eu) mzc += ld_elem<W>(p.alpha, 0) * e_u;
    st_elem<W>(p.mDc, r, mrc - mzc);
    st_elem<W>(p.Dc, r, dc);
}

template <int W>
__global__ void __launch_bounds__(NT) vec_small_kernel(VecParams p) {
    ptx::grid_dep_wait();
    vec_small_body<W>(p, blockIdx.x);
}

int vec_warps_per_row(int64_t K) {
    return K >= 2048 ? 8 : K >= 1024 ? 4 : K >= 256 ? 2 : 1;
}

template <int W>
cudaError_t run(const CompactArgs& a, char* ws, cudaStream_t st) {
    Split sp = choose_split(a.M, a.K, a.N);
    WsLayout L = ws_layout(a.M, a.K, a.N, W);
    RowsParams rp{a.M, a.K, a.N, sp.S, sp.cw, a.alpha, a.mR, a.Dt, a.mC, a.mB, a.F, a.chi, a.mZ,
                  (u64*)(ws + L.pmr), (u64*)(ws + L.pd), (u64*)(ws + L.pmc),
                  (u64*)(ws + L.qmb), (u64*)(ws + L.qf), a.with_eu};
    const int64_t tasks = (a.M + a.K) * sp.S;
    if (tasks > 0) {
        const unsigned blocks = (unsigned)((tasks + WARPS - 1) / WARPS);
        const cudaError_t e = W == 1 && (a.N % 2) == 0
                                  ? launch_dependent(rows_kernel<W, 2>, dim3(blocks), dim3(NT), 0, st, rp)
                                  : launch_dependent(rows_kernel<W, 1>, dim3(blocks), dim3(NT), 0, st, rp);
        if (e != cudaSuccess) return e;
    }
    // with one chunk per row the K-side partials already are the vectors
    // mB.chi and F.chi: the vec pass reads them in place, no finalize pass
    const bool fin = a.K > 0 && sp.S > 1;
    if (fin) {
        unsigned fb = (unsigned)((a.K + 255) / 256);
        if (fb > 1024) fb = 1024;
        const cudaError_t e = launch_dependent(finalize_kernel<W>, dim3(fb), dim3(256), 0, st, a.K, sp.S,
                                               (const u64*)rp.qmb, (const u64*)rp.qf, (u64*)(ws + L.vmb),
                                               (u64*)(ws + L.vf));
        if (e != cudaSuccess) return e;
    }
    VecParams vp{a.M, a.K, sp.S, a.with_eu, a.alpha, a.E, a.mA, fin ? (const u64*)(ws + L.vmb) : rp.qmb,
                 fin ? (const u64*)(ws + L.vf) : rp.qf, rp.pmr, rp.pd, rp.pmc, a.mDc, a.Dc};
    if (a.K < SMALL_K) {
        const cudaError_t e =
            launch_dependent(vec_small_kernel<W>, dim3((unsigned)((a.M + NT - 1) / NT)), dim3(NT), 0, st, vp);
        if (e != cudaSuccess) return e;
    } else {
        const int wpr = vec_warps_per_row(a.K);
        const int64_t rpb = WARPS / wpr;
        const unsigned vb = (unsigned)((a.M + rpb - 1) / rpb);
        const cudaError_t e = W == 1 && (a.K % 2) == 0
                                  ? launch_dependent(vec_kernel<W, 2>, dim3(vb), dim3(NT), 0, st, vp, wpr)
                                  : launch_dependent(vec_kernel<W, 1>, dim3(vb), dim3(NT), 0, st, vp, wpr);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// grouped: the tags of up to CG layers in three launches (rows, finalize,
// vec).  Per-layer parameters travel in the kernels' parameter space; a block
// finds its layer by a binary search over the layers' first blocks.

constexpr int CG = 64;

struct CompactLayer {
    RowsParams rp;
    VecParams vp;
    int rows_vec2;   // rows pass on 16-byte pairs
    int vec_small;   // K < SMALL_K: one thread per row
    int vec_vec2;    // vec pass on 16-byte pairs
    int wpr;         // warps per row in the vec pass
    u64 *vmb, *vf;
};

struct CompactGroup {
    int count;
    int64_t rb[CG + 1], fb[CG + 1], vb[CG + 1];   // first block of each layer, per kernel
    CompactLayer L[CG];
};
static_assert(sizeof(CompactGroup) + 64 <= 32764, "kernel parameter space");

// the last layer whose first block is at or before block b (layers with no
// blocks in this kernel share their successor's offset and are skipped)
__device__ __forceinline__ int layer_of(const int64_t* off, int count, int64_t b) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int W>
__global__ void __launch_bounds__(NT) rows_group_kernel(const __grid_constant__ CompactGroup g) {
    ptx::grid_dep_launch();
    ptx::grid_dep_wait();
    const int li = layer_of(g.rb, g.count, blockIdx.x);
    const CompactLayer& L = g.L[li];
    const int64_t task = ((int64_t)blockIdx.x - g.rb[li]) * WARPS + (threadIdx.x >> 5);
    if (W == 1 && L.rows_vec2) rows_body<W, 2>(L.rp, task, threadIdx.x & 31);
    else rows_body<W, 1>(L.rp, task, threadIdx.x & 31);
}

template <int W>
__global__ void __launch_bounds__(256) finalize_group_kernel(const __grid_constant__ CompactGroup g) {
    ptx::grid_dep_launch();
    ptx::grid_dep_wait();
    const int li = layer_of(g.fb, g.count, blockIdx.x);
    const CompactLayer& L = g.L[li];
    const int64_t nb = g.fb[li + 1] - g.fb[li];
    finalize_body<W>(L.rp.K, L.rp.S, L.rp.qmb, L.rp.qf, L.vmb, L.vf,
                     ((int64_t)blockIdx.x - g.fb[li]) * 256 + threadIdx.x, nb * 256);
}

template <int W>
__global__ void __launch_bounds__(NT) vec_group_kernel(const __grid_constant__ CompactGroup g) {
    ptx::grid_dep_wait();
    const int li = layer_of(g.vb, g.count, blockIdx.x);
    const CompactLayer& L = g.L[li];
    const int64_t blk = (int64_t)blockIdx.x - g.vb[li];
    if (L.vec_small) vec_small_body<W>(L.vp, blk);
    else if (W == 1 && L.vec_vec2) vec_body<W, 2>(L.vp, L.wpr, blk);
    else vec_body<W, 1>(L.vp, L.wpr, blk);
}

// blocks of each kernel for one layer
struct CompactBlocks {
    int64_t rows, fin, vec;
};

CompactBlocks compact_blocks(int64_t M, int64_t K, int64_t N) {
    CompactBlocks b{0, 0, 0};
    if (M == 0) return b;
    const Split sp = choose_split(M, K, N);
    b.rows = ((M + K) * sp.S + WARPS - 1) / WARPS;
    if (K > 0 && sp.S > 1) {   // with one chunk per row there is nothing to finalize
        b.fin = (K + 255) / 256;
        if (b.fin > 1024) b.fin = 1024;
    }
    if (K < SMALL_K) {
        b.vec = (M + NT - 1) / NT;
    } else {
        const int64_t rpb = WARPS / vec_warps_per_row(K);
        b.vec = (M + rpb - 1) / rpb;
    }
    return b;
}

template <int W>
cudaError_t run_group(const CompactArgs* a, int n, char* const* ws, cudaStream_t st) {
    auto* g = new (std::nothrow) CompactGroup;
    if (!g) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaSuccess;
    int i = 0;
    while (i < n && e == cudaSuccess) {
        int cnt = 0;
        g->rb[0] = g->fb[0] = g->vb[0] = 0;
        for (; i < n && cnt < CG; ++i) {
            const CompactArgs& x = a[i];
            if (x.M == 0) continue;
            const Split sp = choose_split(x.M, x.K, x.N);
            const WsLayout wl = ws_layout(x.M, x.K, x.N, W);
            char* w = ws[i];
            CompactLayer& L = g->L[cnt];
            L.rp = RowsParams{x.M, x.K, x.N, sp.S, sp.cw, x.alpha, x.mR, x.Dt, x.mC, x.mB, x.F, x.chi, x.mZ,
                              (u64*)(w + wl.pmr), (u64*)(w + wl.pd), (u64*)(w + wl.pmc),
                              (u64*)(w + wl.qmb), (u64*)(w + wl.qf), x.with_eu};
            L.vmb = (u64*)(w + wl.vmb);
            L.vf = (u64*)(w + wl.vf);
            // one chunk per row: the vec pass reads the partials in place (no finalize blocks)
            const bool fin = x.K > 0 && sp.S > 1;
            L.vp = VecParams{x.M, x.K, sp.S, x.with_eu, x.alpha, x.E, x.mA, fin ? L.vmb : L.rp.qmb,
                             fin ? L.vf : L.rp.qf, L.rp.pmr, L.rp.pd,
                             L.rp.pmc, x.mDc, x.Dc};
            L.rows_vec2 = (x.N % 2) == 0;
            L.vec_small = x.K < SMALL_K;
            L.vec_vec2 = (x.K % 2) == 0;
            L.wpr = vec_warps_per_row(x.K);
            const CompactBlocks b = compact_blocks(x.M, x.K, x.N);
            g->rb[cnt + 1] = g->rb[cnt] + b.rows;
            g->fb[cnt + 1] = g->fb[cnt] + b.fin;
            g->vb[cnt + 1] = g->vb[cnt] + b.vec;
            ++cnt;
        }
        if (cnt == 0) break;
        g->count = cnt;
        if (g->rb[cnt] > 0)
            e = launch_dependent(rows_group_kernel<W>, dim3((unsigned)g->rb[cnt]), dim3(NT), 0, st, *g);
        if (g->fb[cnt] > 0)
            e = launch_dependent(finalize_group_kernel<W>, dim3((unsigned)g->fb[cnt]), dim3(256), 0, st, *g);
        if (e == cudaSuccess && g->vb[cnt] > 0)
            e = launch_dependent(vec_group_kernel<W>, dim3((unsigned)g->vb[cnt]), dim3(NT), 0, st, *g);
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    delete g;
    return e;
}

}  // namespace

int compact_launches(int64_t M, int64_t K, int64_t N) {
    if (M == 0) return 0;
    Split sp = choose_split(M, K, N);
    return ((M + K) * sp.S > 0 ? 1 : 0) + (K > 0 && sp.S > 1 ? 1 : 0) + 1;
}

size_t compact_workspace(int64_t M, int64_t K, int64_t N, int words) {
    return ws_layout(M, K, N, words).total;
}

int compact_grouped_launches(const int64_t* M, const int64_t* K, const int64_t* N, int n) {
    int launches = 0, cnt = 0;
    int64_t r = 0, f = 0, v = 0;
    for (int i = 0; i <= n; ++i) {
        if (i == n || cnt == CG) {
            launches += (r > 0) + (f > 0) + (v > 0);
            r = f = v = 0;
            cnt = 0;
            if (i == n) break;
        }
        if (M[i] == 0) continue;
        const CompactBlocks b = compact_blocks(M[i], K[i], N[i]);
        r += b.rows;
        f += b.fin;
        v += b.vec;
        ++cnt;
    }
    return launches;
}

cudaError_t launch_compact_grouped(const CompactArgs* a, int n, char* const* ws, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int w = a[0].words;
    for (int i = 0; i < n; ++i)
        if (a[i].words != w) return cudaErrorInvalidValue;
    return w == 1 ? run_group<1>(a, n, ws, st) : run_group<2>(a, n, ws, st);
}

cudaError_t launch_compact(const CompactArgs& a, void* ws, size_t ws_bytes, cudaStream_t st) {
    if (a.M == 0) return cudaSuccess;
    if (ws_bytes < compact_workspace(a.M, a.K, a.N, a.words)) return cudaErrorInvalidValue;
    return a.words == 1 ? run<1>(a, (char*)ws, st) : run<2>(a, (char*)ws, st);
}

}  // namespace mpcl
