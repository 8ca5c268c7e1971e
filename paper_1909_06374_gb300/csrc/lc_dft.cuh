// lc_dft.cuh -- in-register DFTs of R <= 16 points for the FFT passes.
#pragma once
#include "lc_common.cuh"

namespace lc {

__host__ __device__ constexpr int ilog2c(int r) { return r <= 1 ? 0 : 1 + ilog2c(r >> 1); }
__host__ __device__ constexpr int bitrev_c(int v, int bits)
{
    return bits == 0 ? 0 : (((v & 1) << (bits - 1)) | bitrev_c(v >> 1, bits - 1));
}

// cos(2 pi t / 16)
__device__ __forceinline__ double cos16(int t)
{
    switch (t & 15) {
    case 0: return 1.0;
    case 1: return 0.92387953251128675613;
    case 2: return 0.70710678118654752440;
    case 3: return 0.38268343236508977173;
    case 4: return 0.0;
    case 5: return -0.38268343236508977173;
    case 6: return -0.70710678118654752440;
    case 7: return -0.92387953251128675613;
    case 8: return -1.0;
    case 9: return -0.92387953251128675613;
    case 10: return -0.70710678118654752440;
    case 11: return -0.38268343236508977173;
    case 12: return 0.0;
    case 13: return 0.38268343236508977173;
    case 14: return 0.70710678118654752440;
    default: return 0.92387953251128675613;
    }
}

// b * e^{-+ 2 pi i t/16} (+ for the inverse transform); t is a compile-time
// constant at every call site, so the branches fold away.
template <typename T, bool INV>
__device__ __forceinline__ cplx<T> rot16(cplx<T> b, int t)
{
    cplx<T> r;
    if (t == 0) return b;
    if (t == 4) {
        if (INV) { r.x = -b.y; r.y = b.x; } else { r.x = b.y; r.y = -b.x; }
        return r;
    }
    if (t == 8) { r.x = -b.x; r.y = -b.y; return r; }
    const T c = (T)cos16(t);
    const T s = INV ? (T)cos16(t + 12) : -(T)cos16(t + 12);  // sin(2 pi t/16) = cos(2 pi (t - 4)/16)
    r.x = b.x * c - b.y * s;
    r.y = b.x * s + b.y * c;
    return r;
}

// Bit-reversal permutation with indices fixed at compile time (keeps the
// array in registers).
template <int I, int R, typename V>
struct BitrevSwaps {
    static __device__ __forceinline__ void run(V (&u)[R])
    {
        constexpr int J = bitrev_c(I, ilog2c(R));
        if constexpr (J > I) { V t = u[I]; u[I] = u[J]; u[J] = t; }
        BitrevSwaps<I + 1, R, V>::run(u);
    }
};
template <int R, typename V>
struct BitrevSwaps<R, R, V> {
    static __device__ __forceinline__ void run(V (&)[R]) {}
};

// out[q] = sum_r u[r] e^{-+ 2 pi i r q / R}: radix-2 decimation in time on the
// bit-reversed input.
template <typename T, int R, bool INV>
__device__ __forceinline__ void dft_regs(cplx<T> (&u)[R])
{
    constexpr int LR = ilog2c(R);
    BitrevSwaps<0, R, cplx<T>>::run(u);
#pragma unroll
    for (int s = 1; s <= LR; ++s) {
        const int m = 1 << s, h = m >> 1;
#pragma unroll
        for (int g = 0; g < R; g += m) {
#pragma unroll
            for (int j = 0; j < h; ++j) {
                const cplx<T> a = u[g + j];
                const cplx<T> b = rot16<T, INV>(u[g + j + h], j * (16 / m));
                u[g + j] = cadd(a, b);
                u[g + j + h] = csub(a, b);
            }
        }
    }
}

}  // namespace lc
