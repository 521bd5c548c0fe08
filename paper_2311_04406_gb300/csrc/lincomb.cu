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

}  // namespace

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
