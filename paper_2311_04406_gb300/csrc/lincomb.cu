// lincomb.cu -- out = sum_j c_j in_j mod 2^(64 W), elementwise, for small
// signed integer coefficients c_j: the local part of an opening when parties
// are simulated on one device (E = sum_i (X_i - A_i), D~ = sum_i (R_i - Z_i),
// §2.5 and Fig. Pi_OptMAC), and any other linear combination of sharings
// (linearity of authenticated shares under public constants, §2.4).
#include "common.cuh"
#include "kernels.h"

namespace mpcl {

namespace {

constexpr int NT = 256;

struct LincombArgs {
    int64_t n;
    int count;
    int64_t coef[LINCOMB_MAX];
    const u64* in[LINCOMB_MAX];
    u64* out;
};

template <int W>
__global__ void __launch_bounds__(NT) lincomb_kernel(const __grid_constant__ LincombArgs a) {
    using T = typename Elem<W>::T;
    if constexpr (W == 1) {
        // two elements per 16-byte access when n is even (else one at a time)
        const bool pairs = (a.n & 1) == 0;
        const int64_t nv = pairs ? a.n / 2 : a.n;
        for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < nv; i += (int64_t)gridDim.x * NT) {
            if (pairs) {
                u64 x = 0, y = 0;
                for (int j = 0; j < a.count; ++j) {
                    const ulonglong2 v = ld_stream2(a.in[j] + 2 * i);
                    x += (u64)a.coef[j] * v.x;
                    y += (u64)a.coef[j] * v.y;
                }
                st_stream2(a.out + 2 * i, make_ulonglong2(x, y));
            } else {
                u64 x = 0;
                for (int j = 0; j < a.count; ++j) x += (u64)a.coef[j] * ldg_elem<1>(a.in[j], i);
                st_elem<1>(a.out, i, x);
            }
        }
    } else {
        for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * NT) {
            T x = 0;
            for (int j = 0; j < a.count; ++j) x += (T)(__int128)a.coef[j] * ldg_elem<W>(a.in[j], i);
            st_elem<W>(a.out, i, x);
        }
    }
}

// Up to LINCOMB_GROUP_MAX combinations with the same coefficients in one
// launch: group g has n[g] elements; blocks are dealt to the groups by their
// element counts (block b works for the group whose block range holds b).
struct LincombGroup {
    int groups;
    int count;
    int64_t coef[LINCOMB_MAX];
    int64_t n[LINCOMB_GROUP_MAX];
    int64_t b_off[LINCOMB_GROUP_MAX + 1];
    const u64* in[LINCOMB_GROUP_MAX][LINCOMB_GROUP_TERMS];
    u64* out[LINCOMB_GROUP_MAX];
};

constexpr int GROUP_ELEMS = NT * 4;   // elements per block of a grouped launch

template <int W>
__global__ void __launch_bounds__(NT) lincomb_group_kernel(const __grid_constant__ LincombGroup a) {
    using T = typename Elem<W>::T;
    int lo = 0, hi = a.groups - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.b_off[mid] <= (int64_t)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const int g = lo;
    const int64_t base = ((int64_t)blockIdx.x - a.b_off[g]) * GROUP_ELEMS;
    const int64_t end = base + GROUP_ELEMS < a.n[g] ? base + GROUP_ELEMS : a.n[g];
    for (int64_t i = base + threadIdx.x; i < end; i += NT) {
        T x = 0;
        for (int j = 0; j < a.count; ++j) x += (T)(__int128)a.coef[j] * ldg_elem<W>(a.in[g][j], i);
        st_elem<W>(a.out[g], i, x);
    }
}

}  // namespace

cudaError_t launch_lincomb_grouped(int groups, const int64_t* n, int words, int count, const int64_t* coef,
                                   const u64* const* in, u64* const* out, cudaStream_t st) {
    if (count < 1 || count > LINCOMB_GROUP_TERMS) return cudaErrorInvalidValue;
    int g = 0;   // next group to place (empty groups are skipped)
    while (g < groups) {
        LincombGroup a{};
        a.count = count;
        for (int j = 0; j < count; ++j) a.coef[j] = coef[j];
        a.b_off[0] = 0;
        int k = 0;
        for (; g < groups && k < LINCOMB_GROUP_MAX; ++g) {
            if (n[g] == 0) continue;
            a.n[k] = n[g];
            for (int j = 0; j < count; ++j) a.in[k][j] = in[(size_t)g * count + j];
            a.out[k] = out[g];
            a.b_off[k + 1] = a.b_off[k] + (n[g] + GROUP_ELEMS - 1) / GROUP_ELEMS;
            ++k;
        }
        if (k == 0) continue;
        a.groups = k;
        const int64_t blocks = a.b_off[k];
        if (blocks > 0x7fffffff) return cudaErrorInvalidValue;
        if (words == 1) lincomb_group_kernel<1><<<(unsigned)blocks, NT, 0, st>>>(a);
        else lincomb_group_kernel<2><<<(unsigned)blocks, NT, 0, st>>>(a);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_lincomb(int64_t n, int words, int count, const int64_t* coef, const u64* const* in, u64* out,
                           cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    if (count < 1 || count > LINCOMB_MAX) return cudaErrorInvalidValue;
    LincombArgs a{};
    a.n = n;
    a.count = count;
    for (int j = 0; j < count; ++j) {
        a.coef[j] = coef[j];
        a.in[j] = in[j];
    }
    a.out = out;
    const int64_t per = words == 1 ? 2 : 1;
    int64_t blocks = (n / per + NT - 1) / NT;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    if (words == 1) lincomb_kernel<1><<<(unsigned)blocks, NT, 0, st>>>(a);
    else lincomb_kernel<2><<<(unsigned)blocks, NT, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mpcl
