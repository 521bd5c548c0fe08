// trunc.cu -- the OptMAC&Trunc step of the truncated layer (Fig. Pi_OptMAC&Trunc
// steps 3-4 and Fig. Pi_CompactMatMul step 4, §3.4), elementwise and
// HBM-bound:
//   delta = (D~ mod 2^k) / 2^f,  rho = (E.U mod 2^k) / 2^f,  tau = rho - delta
//   [Z^f]_i    = [R^f]_i    + tau            (party 0 only: a public constant)
//   [m(Z^f)]_i = [m(R^f)]_i + [alpha]_i tau  (every party)
// "/ 2^f" is the floor division of the k-bit value; all sums wrap mod 2^(k+s).
#include "common.cuh"
#include "kernels.h"

namespace mpcl {

namespace {

constexpr int NT = 256;

template <int W>
__global__ void __launch_bounds__(NT) optmac_trunc_kernel(int64_t MN, int k, int f, int party0,
                                                          const u64* alpha, const u64* Rf,
                                                          const u64* mRf, const u64* Dt, const u64* P,
                                                          u64* Zf, u64* mZf) {
    using T = typename Elem<W>::T;
    const T mk = k >= 64 * W ? ~(T)0 : (((T)1 << k) - 1);
    const T a = ld_elem<W>(alpha, 0);
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < MN; i += (int64_t)gridDim.x * NT) {
        const T delta = (ldg_elem<W>(Dt, i) & mk) >> f;
        const T rho = (ldg_elem<W>(P, i) & mk) >> f;
        const T tau = rho - delta;
        st_elem<W>(Zf, i, ldg_elem<W>(Rf, i) + (party0 ? tau : (T)0));
        st_elem<W>(mZf, i, ldg_elem<W>(mRf, i) + a * tau);
    }
}

}  // namespace

cudaError_t launch_optmac_trunc(int64_t MN, int words, int k, int f, int party0, const u64* alpha,
                                const u64* Rf, const u64* mRf, const u64* Dt, const u64* P, u64* Zf,
                                u64* mZf, cudaStream_t st) {
    if (MN == 0) return cudaSuccess;
    int64_t blocks = (MN + NT - 1) / NT;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (words == 1)
        optmac_trunc_kernel<1><<<(unsigned)blocks, NT, 0, st>>>(MN, k, f, party0, alpha, Rf, mRf, Dt, P, Zf, mZf);
    else
        optmac_trunc_kernel<2><<<(unsigned)blocks, NT, 0, st>>>(MN, k, f, party0, alpha, Rf, mRf, Dt, P, Zf, mZf);
    return cudaGetLastError();
}

}  // namespace mpcl
