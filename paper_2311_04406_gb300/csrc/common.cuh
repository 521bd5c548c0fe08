// common.cuh -- ring element types and small device helpers shared by the
// kernels of the library.  Elements of Z_2^64 are one uint64 word; elements of
// Z_2^128 are two words (lo, hi) loaded as one 16-byte vector.  All arithmetic
// wraps mod 2^(64 W), which is the share ring Z_{2^{k+s}} for k + s = 64 W.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mpcl {

// Launches `kernel` as a programmatic dependent of the kernel before it on
// `st`: it may be scheduled while that kernel finishes, and it must execute
// ptx::grid_dep_wait() before it reads anything that kernel (or any earlier
// one) wrote.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                    cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

using u64 = unsigned long long;
using u128 = unsigned __int128;

template <int W> struct Elem;
template <> struct Elem<1> { using T = u64; };
template <> struct Elem<2> { using T = u128; };

template <int W>
__device__ __forceinline__ typename Elem<W>::T ld_elem(const u64* p, int64_t i) {
    if constexpr (W == 1) {
        return p[i];
    } else {
        ulonglong2 v = *reinterpret_cast<const ulonglong2*>(p + 2 * i);
        return (u128)v.x | ((u128)v.y << 64);
    }
}

template <int W>
__device__ __forceinline__ typename Elem<W>::T ldg_elem(const u64* p, int64_t i) {
    if constexpr (W == 1) {
        return __ldg(p + i);
    } else {
        ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2*>(p + 2 * i));
        return (u128)v.x | ((u128)v.y << 64);
    }
}

template <int W>
__device__ __forceinline__ void st_elem(u64* p, int64_t i, typename Elem<W>::T v) {
    if constexpr (W == 1) {
        p[i] = v;
    } else {
        ulonglong2 o;
        o.x = (u64)v;
        o.y = (u64)(v >> 64);
        *reinterpret_cast<ulonglong2*>(p + 2 * i) = o;
    }
}

// streaming (evict-first) 16-byte load / store for data read or written once
__device__ __forceinline__ ulonglong2 ld_stream2(const u64* p) {
    ulonglong2 v;
    asm volatile("ld.global.cs.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_stream2(u64* p, ulonglong2 v) {
    asm volatile("st.global.cs.v2.u64 [%0], {%1, %2};" :: "l"(p), "l"(v.x), "l"(v.y) : "memory");
}

// Exact wrapping atomic additions into Z (any order gives the same result,
// since addition mod 2^(64 W) is associative and commutative).
__device__ __forceinline__ void red_add_u64(u64* p, u64 v) {
    asm volatile("red.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// 128-bit: the low word's atomic returns its old value, which gives the exact
// carry of this addition into the high word
__device__ __forceinline__ void atomic_add_u128(u64* p, u128 v) {
    const u64 lo = (u64)v;
    u64 hi = (u64)(v >> 64);
    u64 old;
    asm volatile("atom.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(lo) : "memory");
    hi += (old + lo < old) ? 1ull : 0ull;
    asm volatile("red.global.add.u64 [%0], %1;" ::"l"(p + 1), "l"(hi) : "memory");
}
template <int W>
__device__ __forceinline__ void atomic_add_elem(u64* p, int64_t i, typename Elem<W>::T v) {
    if constexpr (W == 1) red_add_u64(p + i, v);
    else atomic_add_u128(p + 2 * i, v);
}

}  // namespace mpcl
