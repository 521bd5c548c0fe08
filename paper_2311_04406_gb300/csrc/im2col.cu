// im2col.cu -- the im2col view of a convolution (§2.6): a convolution of an
// f x f filter over a batch of C x H x W ring-element images (NCHW) becomes
// the ring GEMM  out (B H' W' x C f f) . W (C f f x O).  Row (b, oy, ox),
// column (c, ky, kx) of `out` is in[b][c][oy s + ky - p][ox s + kx - p], or 0
// where that falls in the zero padding.  Zero is a sharing of 0 and its tag
// (§2.4), so each party applies this to its own shares and tags locally.
#include "common.cuh"
#include "kernels.h"

namespace mpcl {

namespace {

constexpr int NT = 256;

struct Im2colArgs {
    int64_t B, C, H, W;
    int f, pad, stride;
    int64_t Ho, Wo;
    const u64* in;
    u64* out;
};

// one thread per output element; consecutive threads take consecutive
// columns (c, ky, kx) of one row, so the writes are coalesced
template <int WW>
__global__ void __launch_bounds__(NT) im2col_kernel(const Im2colArgs a) {
    using T = typename Elem<WW>::T;
    const int64_t Kc = a.C * a.f * a.f;
    const int64_t total = a.B * a.Ho * a.Wo * Kc;
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < total; i += (int64_t)gridDim.x * NT) {
        const int64_t row = i / Kc, col = i - row * Kc;
        const int64_t b = row / (a.Ho * a.Wo);
        const int64_t rem = row - b * a.Ho * a.Wo;
        const int64_t oy = rem / a.Wo, ox = rem - oy * a.Wo;
        const int64_t c = col / (a.f * a.f);
        const int kk = (int)(col - c * a.f * a.f);
        const int ky = kk / a.f, kx = kk - ky * a.f;
        const int64_t y = oy * a.stride + ky - a.pad, x = ox * a.stride + kx - a.pad;
        T v = 0;
        if (y >= 0 && y < a.H && x >= 0 && x < a.W) v = ldg_elem<WW>(a.in, ((b * a.C + c) * a.H + y) * a.W + x);
        st_elem<WW>(a.out, i, v);
    }
}

}  // namespace

cudaError_t launch_im2col(int64_t B, int64_t C, int64_t H, int64_t W, int f, int pad, int stride, int words,
                          const u64* in, u64* out, cudaStream_t st) {
    const int64_t Ho = (H - f + 2 * pad) / stride + 1, Wo = (W - f + 2 * pad) / stride + 1;
    const int64_t total = B * Ho * Wo * C * f * f;
    if (total <= 0) return cudaSuccess;
    Im2colArgs a{B, C, H, W, f, pad, stride, Ho, Wo, in, out};
    int64_t blocks = (total + NT - 1) / NT;
    if (blocks > 152 * 32) blocks = 152 * 32;
    if (words == 1) im2col_kernel<1><<<(unsigned)blocks, NT, 0, st>>>(a);
    else im2col_kernel<2><<<(unsigned)blocks, NT, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace mpcl
