// lc_resident.cu -- fused, on-chip amplitude-adjustment iterations (Sec. 3.2.2)
// for curves whose working set fits in one CTA's shared memory.
//
// One CTA (N <= 2^14) or a cluster of C = N/2^14 CTAs (N = 2^15, 2^16) owns
// one curve (FP32) for all the iterations of a launch: the state x stays in shared memory, the target
// amplitudes A and the sorted draws s are read from L2 each iteration, and x
// goes back to HBM once at the end.  Per iteration:
//   1. complex Stockham FFT of z[m] = x[2m] + i x[2m+1] (M = N/2 points) in
//      shared memory, radix-16 register butterflies, XOR-swizzled addresses;
//   2. unpack to X_0..X_M, keep the phases, impose A, pack for the inverse
//      (the pairs (k, M-k) are both local);
//   3. inverse complex FFT -> x_adj;
//   4. stable LSD radix sort of the order keys of x_adj (4 passes of 8 bits;
//      warp-level match + per-warp digit counts, block-wide scan), the last
//      pass writing x[position] = s[rank] directly.
// Shared memory: two complex buffers (2 x 2N bytes... 4N bytes each), two u16
// index buffers (2N bytes each) and the per-warp digit counts (8 KB):
// 12 N + 8 KB <= 204 KB at N = 2^14.
#include <cooperative_groups.h>

#include "lc_dft.cuh"
#include "lc_internal.h"

namespace lc {

namespace {

constexpr int kResThreads = 512;
constexpr int kResWarps = kResThreads / 32;
constexpr uint32_t kResMinLog2 = 10;
constexpr uint32_t kResMaxLog2 = 14;      // one CTA
constexpr uint32_t kResClusterMaxLog2 = 16;  // clusters of 2 or 4 CTAs (16-bit positions)

__device__ __forceinline__ int swz(int e) { return e ^ ((e >> 4) & 15); }

// e^{-2 pi i k/N} for k in [0, N) from the class table rt (k < N/2).
__device__ __forceinline__ float2 twN(const float2* __restrict__ rt, int k, int M)
{
    if (k < M) return __ldg(rt + k);
    const float2 w = __ldg(rt + (k - M));
    return make_float2(-w.x, -w.y);
}

// One radix-R Stockham pass of the length-Mc complex transform in shared memory.
// W_Mc^t = e^{-2 pi i (N/Mc) t / N}.
template <int R, bool INV>
__device__ __forceinline__ void smem_pass(const float2* __restrict__ in, float2* __restrict__ out, int log2Mc,
                                          int log2p, const float2* __restrict__ rt, int M, int log2ratio)
{
    constexpr int LR = ilog2c(R);
    const int nb = 1 << (log2Mc - LR);
    const int p = 1 << log2p;
    for (int i = threadIdx.x; i < nb; i += kResThreads) {
        const int k = i & (p - 1);
        float2 u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = in[swz(i + r * nb)];
        if (p > 1) {
            const int step = k << (log2Mc - LR - log2p);
#pragma unroll
            for (int r = 1; r < R; ++r) {
                float2 w = twN(rt, (r * step) << log2ratio, M);
                if (INV) w.y = -w.y;
                u[r] = make_float2(u[r].x * w.x - u[r].y * w.y, u[r].x * w.y + u[r].y * w.x);
            }
        }
        dft_regs<float, R, INV>(u);
        const int j = ((i - k) << LR) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) out[swz(j + r * p)] = u[r];
    }
}

// Complex FFT of length Mc = 2^log2Mc held in shared memory (swizzled), ping-
// ponging between a and b; returns the buffer holding the result.
template <bool INV>
__device__ float2* smem_fft(float2* a, float2* b, int log2Mc, const float2* __restrict__ rt, int M, int log2ratio)
{
    int log2p = 0;
    float2* in = a;
    float2* out = b;
    const int rem = log2Mc & 3;
    if (rem) {
        if (rem == 1) smem_pass<2, INV>(in, out, log2Mc, 0, rt, M, log2ratio);
        else if (rem == 2) smem_pass<4, INV>(in, out, log2Mc, 0, rt, M, log2ratio);
        else smem_pass<8, INV>(in, out, log2Mc, 0, rt, M, log2ratio);
        __syncthreads();
        log2p = rem;
        float2* t = in; in = out; out = t;
    }
    for (; log2p < log2Mc; log2p += 4) {
        smem_pass<16, INV>(in, out, log2Mc, log2p, rt, M, log2ratio);
        __syncthreads();
        float2* t = in; in = out; out = t;
    }
    return in;
}

__device__ __forceinline__ float2 keep_phase_f(float2 X, float A)
{
    const float m2 = X.x * X.x + X.y * X.y;
    if (m2 == 0.0f) return make_float2(A, 0.0f);
    const float s = A * rsqrtf(m2);
    return make_float2(X.x * s, X.y * s);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// Spectral step on the local packed spectrum Z (length M): unpack, keep the
// phases with amplitudes A, pack for the inverse transform into Zo.
__device__ void spectral_local(const float2* __restrict__ Z, float2* __restrict__ Zo, const float* __restrict__ A,
                               const float2* __restrict__ rt, int M)
{
    const int half = M >> 1;
    for (int k = threadIdx.x; k < half; k += kResThreads) {
        if (k == 0) {
            const float2 z0 = Z[swz(0)];
            const float XM = z0.x - z0.y;
            const float Y0 = __ldg(A);
            const float YM = XM < 0.0f ? -__ldg(A + M) : __ldg(A + M);
            Zo[swz(0)] = make_float2(Y0 + YM, Y0 - YM);
            const float2 zh = Z[swz(half)];
            const float2 Yh = keep_phase_f(make_float2(zh.x, -zh.y), __ldg(A + half));
            Zo[swz(half)] = make_float2(2.0f * Yh.x, -2.0f * Yh.y);
        } else {
            const float2 za = Z[swz(k)], zb = Z[swz(M - k)];
            const float2 W = __ldg(rt + k);
            const float2 E = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y));
            const float2 O = make_float2(0.5f * (za.y + zb.y), -0.5f * (za.x - zb.x));
            const float2 WO = cmulf(W, O);
            const float2 Xk = make_float2(E.x + WO.x, E.y + WO.y);
            const float2 Xm = make_float2(E.x - WO.x, -(E.y - WO.y));
            const float2 Yk = keep_phase_f(Xk, __ldg(A + k));
            const float2 Ym = keep_phase_f(Xm, __ldg(A + M - k));
            const float2 Ep = make_float2(Yk.x + Ym.x, Yk.y - Ym.y);
            const float2 Dd = make_float2(Yk.x - Ym.x, Yk.y + Ym.y);
            const float2 Op = cmulf(Dd, make_float2(W.x, -W.y));
            Zo[swz(k)] = make_float2(Ep.x - Op.y, Ep.y + Op.x);
            Zo[swz(M - k)] = make_float2(Ep.x + Op.y, -Ep.y + Op.x);
        }
    }
}

// float index f of a swizzled complex buffer
__device__ __forceinline__ int fsw(int f) { return (swz(f >> 1) << 1) | (f & 1); }

// Exclusive scan of v over threads 0..255 (called by all threads; others pass 0).
__device__ __forceinline__ uint32_t scan256(uint32_t v, uint32_t* wsum)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31 && w < 8) wsum[w] = incl;
    __syncthreads();
    uint32_t off = 0;
    for (int q = 0; q < w && q < 8; ++q) off += wsum[q];
    return off + incl - v;
}

struct ResArgs {
    const int* cls_curves;
    const CurveDev* curves;
    const uint32_t* eff_iters;
    const int* d_iter;
    const float* A;
    const float* s;
    float* x;
    const float2* tw;
    uint32_t n_it;
    uint32_t log2n;
};

// One LSD radix pass over the L = N keys of the CTA.
// FIRST: keys are the order keys of the x_adj floats in xa (swizzled view);
// LAST: instead of the sorted pairs, writes xn[index] = s[rank].
template <bool FIRST, bool LAST>
__device__ __forceinline__ void radix_pass(const float* __restrict__ xa, const uint32_t* __restrict__ kin,
                                           uint32_t* __restrict__ kout, const uint16_t* __restrict__ iin,
                                           uint16_t* __restrict__ iout, float* __restrict__ xn,
                                           const float* __restrict__ s, int shift, int log2L, uint16_t* wh,
                                           uint32_t* dbase, uint32_t* wsum)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int EW = 1 << (log2L - 4);  // elements per warp
    const int slots = EW >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t rk[16];  // within-(warp, digit) ranks, two 16-bit values per register
#pragma unroll
    for (int e = 0; e < 32; ++e) {
        if (e < slots) {
            const int el = w * EW + e * 32 + lane;
            const uint32_t key = FIRST ? order_key(xa[fsw(el)]) : kin[el];
            const uint32_t d = (key >> shift) & 255u;
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const uint32_t below = __popc(peers & lt);
            const uint32_t base = wh[w * 256 + d];
            __syncwarp();
            if (below == 0) wh[w * 256 + d] = (uint16_t)(base + __popc(peers));
            __syncwarp();
            const uint32_t r = base + below;
            if (e & 1) rk[e >> 1] |= r << 16;
            else rk[e >> 1] = r;
        }
    }
    __syncthreads();
    uint32_t tot = 0;
    if (threadIdx.x < 256) {
        const int d = threadIdx.x;
#pragma unroll
        for (int q = 0; q < kResWarps; ++q) {
            const uint32_t v = wh[q * 256 + d];
            wh[q * 256 + d] = (uint16_t)tot;
            tot += v;
        }
    }
    const uint32_t db = scan256(threadIdx.x < 256 ? tot : 0u, wsum);
    if (threadIdx.x < 256) dbase[threadIdx.x] = db;
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 32; ++e) {
        if (e < slots) {
            const int el = w * EW + e * 32 + lane;
            const uint32_t key = FIRST ? order_key(xa[fsw(el)]) : kin[el];
            const uint32_t d = (key >> shift) & 255u;
            const uint32_t r = (e & 1) ? (rk[e >> 1] >> 16) : (rk[e >> 1] & 0xffffu);
            const uint32_t dest = dbase[d] + wh[w * 256 + d] + r;
            const uint32_t idx = FIRST ? (uint32_t)el : (uint32_t)iin[el];
            if (LAST) {
                xn[fsw((int)idx)] = __ldg(s + dest);
            } else {
                kout[dest] = key;
                iout[dest] = (uint16_t)idx;
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kResWarps * 256; q += kResThreads) wh[q] = 0;
    __syncthreads();
}

__global__ void __launch_bounds__(kResThreads, 1) k_resident_cta(const ResArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int log2L = (int)a.log2n;
    const int L = 1 << log2L;
    const int M = L >> 1;
    float2* buf0 = (float2*)smem;
    float2* buf1 = (float2*)(smem + (size_t)4 * L);
    uint16_t* ia = (uint16_t*)(smem + (size_t)8 * L);
    uint16_t* ib = (uint16_t*)(smem + (size_t)10 * L);
    uint16_t* wh = (uint16_t*)(smem + (size_t)12 * L);
    __shared__ uint32_t dbase[256];
    __shared__ uint32_t wsum[8];

    const int c = a.cls_curves[blockIdx.x];
    const CurveDev& cv = a.curves[c];
    const int it0 = *a.d_iter;
    int n_act = (int)a.eff_iters[c] - it0;
    if (n_act > (int)a.n_it) n_act = (int)a.n_it;
    if (n_act <= 0) return;
    const float* A = a.A + cv.offh;
    const float* s = a.s + cv.off;
    float* xg = a.x + cv.off;

    for (int q = threadIdx.x; q < kResWarps * 256; q += kResThreads) wh[q] = 0;
    // state -> buf0 (complex view, swizzled)
    const float2* xg2 = (const float2*)xg;
    for (int m = threadIdx.x; m < M; m += kResThreads) buf0[swz(m)] = xg2[m];
    __syncthreads();

    float2* z = buf0;
    float2* o = buf1;
    for (int it = 0; it < n_act; ++it) {
        float2* Z = smem_fft<false>(z, o, log2L - 1, a.tw, M, 1);
        float2* Zs = (Z == buf0) ? buf1 : buf0;
        spectral_local(Z, Zs, A, a.tw, M);
        __syncthreads();
        float2* X = smem_fft<true>(Zs, Z, log2L - 1, a.tw, M, 1);
        float2* other = (X == buf0) ? buf1 : buf0;
        uint32_t* kX = (uint32_t*)X;
        uint32_t* kO = (uint32_t*)other;
        // pass 0: x_adj (in X) -> keys in other; 1: other -> X; 2: X -> other; 3: other -> x in X
        radix_pass<true, false>((const float*)X, nullptr, kO, nullptr, ia, nullptr, s, 0, log2L, wh, dbase, wsum);
        radix_pass<false, false>(nullptr, kO, kX, ia, ib, nullptr, s, 8, log2L, wh, dbase, wsum);
        radix_pass<false, false>(nullptr, kX, kO, ib, ia, nullptr, s, 16, log2L, wh, dbase, wsum);
        radix_pass<false, true>(nullptr, kO, nullptr, ia, nullptr, (float*)X, s, 24, log2L, wh, dbase, wsum);
        z = X;
        o = other;
    }
    float2* xo2 = (float2*)xg;
    for (int m = threadIdx.x; m < M; m += kResThreads) xo2[m] = z[swz(m)];
}


// ---------------------------------------------------------------- clusters
// A curve of N = C * L samples on a cluster of C CTAs; CTA c holds samples
// [cL, (c+1)L).  The length-M (= N/2) complex transform is split as
// M = C x Mc: a cross-CTA radix-C step (decimation in frequency forward,
// in time inverse) reading the partners' blocks through distributed shared
// memory, and local length-Mc transforms; CTA c then holds Z[C k + c].  The
// spectral step reads Z[M - K] from the partner CTA (C - c) mod C.  The radix
// sort is cluster-wide: per pass every CTA ranks its keys locally, the
// per-CTA digit totals are exchanged, and each key is stored at its global
// destination in the owning CTA's shared memory; the last pass stores
// x[position] = s[rank] straight into the next state.
namespace cg = cooperative_groups;

template <int C>
__device__ __forceinline__ float2 ld_cta(cg::cluster_group& cl, float2* local, int q, int me, int at)
{
    if (q == me) return local[at];
    return cl.map_shared_rank(local, q)[at];
}

template <int C>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(kResThreads, 1) k_resident_cluster(const ResArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int me = (int)cl.block_rank();
    constexpr int LOGC = ilog2c(C);
    const int log2n = (int)a.log2n;
    const int log2L = log2n - LOGC;
    const int L = 1 << log2L;
    const int Mc = L >> 1;
    const int M = C * Mc;
    float2* buf0 = (float2*)smem;
    float2* buf1 = (float2*)(smem + (size_t)4 * L);
    uint16_t* ia = (uint16_t*)(smem + (size_t)8 * L);
    uint16_t* ib = (uint16_t*)(smem + (size_t)10 * L);
    uint16_t* wh = (uint16_t*)(smem + (size_t)12 * L);
    __shared__ uint32_t dbase[256];
    __shared__ uint32_t wsum[8];
    __shared__ uint32_t ctot[256];

    const int c = a.cls_curves[blockIdx.x / C];
    const CurveDev& cv = a.curves[c];
    const int it0 = *a.d_iter;
    int n_act = (int)a.eff_iters[c] - it0;
    if (n_act > (int)a.n_it) n_act = (int)a.n_it;
    if (n_act <= 0) return;  // uniform over the cluster (same curve)
    const float* A = a.A + cv.offh;
    const float* s = a.s + cv.off;
    float* xg = a.x + cv.off + (size_t)me * L;
    const float2* rt = a.tw;

    // W_C^{q me} for the cross-CTA steps
    float2 wc[C];
#pragma unroll
    for (int q = 0; q < C; ++q) wc[q] = twN(rt, ((q * me) % C) * (M * 2 / C), M);

    for (int q = threadIdx.x; q < kResWarps * 256; q += kResThreads) wh[q] = 0;
    const float2* xg2 = (const float2*)xg;
    for (int m = threadIdx.x; m < Mc; m += kResThreads) buf0[swz(m)] = xg2[m];
    float2* z = buf0;
    cl.sync();

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int EW = 1 << (log2L - 4);
    const int slots = EW >> 5;
    const uint32_t lt = (1u << lane) - 1u;

    for (int it = 0; it < n_act; ++it) {
        float2* y = (z == buf0) ? buf1 : buf0;
        // forward cross-CTA radix-C step: y[m] = W_M^{m me} sum_q z_q[m] W_C^{q me}
        for (int m = threadIdx.x; m < Mc; m += kResThreads) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < C; ++q) {
                const float2 v = ld_cta<C>(cl, z, q, me, swz(m));
                const float2 t = cmulf(v, wc[q]);
                acc.x += t.x; acc.y += t.y;
            }
            y[swz(m)] = cmulf(acc, twN(rt, 2 * m * me, M));
        }
        cl.sync();  // partners done reading z before it is overwritten
        float2* P = smem_fft<false>(y, z, log2L - 1, rt, M, LOGC + 1);
        float2* Q = (P == buf0) ? buf1 : buf0;
        cl.sync();  // every Z block complete
        const int pr = (C - me) % C;
        for (int k = threadIdx.x; k < Mc; k += kResThreads) {
            const int K = C * k + me;
            float2 out;
            if (K == 0) {
                const float2 z0 = P[swz(0)];
                const float XM = z0.x - z0.y;
                const float Y0 = __ldg(A);
                const float YM = XM < 0.0f ? -__ldg(A + M) : __ldg(A + M);
                out = make_float2(Y0 + YM, Y0 - YM);
            } else if (2 * K == M) {
                const float2 zh = P[swz(k)];
                const float2 Yh = keep_phase_f(make_float2(zh.x, -zh.y), __ldg(A + K));
                out = make_float2(2.0f * Yh.x, -2.0f * Yh.y);
            } else {
                const int kp = me == 0 ? Mc - k : Mc - 1 - k;
                const float2 za = P[swz(k)];
                const float2 zb = ld_cta<C>(cl, P, pr, me, swz(kp));
                const float2 W = twN(rt, K, M);
                const float2 E = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y));
                const float2 O = make_float2(0.5f * (za.y + zb.y), -0.5f * (za.x - zb.x));
                const float2 WO = cmulf(W, O);
                const float2 XK = make_float2(E.x + WO.x, E.y + WO.y);
                const float2 XMK = make_float2(E.x - WO.x, -(E.y - WO.y));
                const float2 YK = keep_phase_f(XK, __ldg(A + K));
                const float2 YMK = keep_phase_f(XMK, __ldg(A + M - K));
                const float2 Ep = make_float2(YK.x + YMK.x, YK.y - YMK.y);
                const float2 Dd = make_float2(YK.x - YMK.x, YK.y + YMK.y);
                const float2 Op = cmulf(Dd, make_float2(W.x, -W.y));
                out = make_float2(Ep.x - Op.y, Ep.y + Op.x);
            }
            Q[swz(k)] = out;
        }
        cl.sync();  // partners done reading P
        float2* U = smem_fft<true>(Q, P, log2L - 1, rt, M, LOGC + 1);
        float2* V = (U == buf0) ? buf1 : buf0;
        cl.sync();  // every u block complete
        // inverse cross-CTA step: x_adj block me = sum_r e^{+2 pi i r me/C} e^{+2 pi i r n/M} u_r[n]
        for (int n = threadIdx.x; n < Mc; n += kResThreads) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int r = 0; r < C; ++r) {
                const float2 v = ld_cta<C>(cl, U, r, me, swz(n));
                const float2 tw = twN(rt, 2 * r * n, M);
                const float2 t = cmulf(cmulf(v, make_float2(tw.x, -tw.y)), make_float2(wc[r].x, -wc[r].y));
                acc.x += t.x; acc.y += t.y;
            }
            V[swz(n)] = acc;
        }
        cl.sync();  // partners done reading U (it becomes a key buffer)

        // cluster-wide stable LSD radix sort of the order keys of x_adj
        uint32_t* kU = (uint32_t*)U;
        uint32_t* kV = (uint32_t*)V;
#pragma unroll 1
        for (int pass = 0; pass < 4; ++pass) {
            const bool first = pass == 0, last = pass == 3;
            const int shift = 8 * pass;
            const uint32_t* kin = (pass == 1 || pass == 3) ? kU : kV;   // pass 0 reads floats from V
            uint32_t* kout = (pass == 0 || pass == 2) ? kU : kV;
            const uint16_t* iin = (pass == 2) ? ib : ia;
            uint16_t* iout = (pass == 1) ? ib : ia;
            const float* xa = (const float*)V;
            uint32_t rk[16];
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                if (e < slots) {
                    const int el = w * EW + e * 32 + lane;
                    const uint32_t key = first ? order_key(xa[fsw(el)]) : kin[el];
                    const uint32_t d = (key >> shift) & 255u;
                    const uint32_t peers = __match_any_sync(0xffffffffu, d);
                    const uint32_t below = __popc(peers & lt);
                    const uint32_t base = wh[w * 256 + d];
                    __syncwarp();
                    if (below == 0) wh[w * 256 + d] = (uint16_t)(base + __popc(peers));
                    __syncwarp();
                    const uint32_t r = base + below;
                    if (e & 1) rk[e >> 1] |= r << 16;
                    else rk[e >> 1] = r;
                }
            }
            __syncthreads();
            if (threadIdx.x < 256) {
                const int d = threadIdx.x;
                uint32_t tot = 0;
#pragma unroll
                for (int q = 0; q < kResWarps; ++q) {
                    const uint32_t v = wh[q * 256 + d];
                    wh[q * 256 + d] = (uint16_t)tot;
                    tot += v;
                }
                ctot[d] = tot;
            }
            cl.sync();  // every CTA's digit totals published
            uint32_t all = 0, lower = 0;
            if (threadIdx.x < 256) {
#pragma unroll
                for (int q = 0; q < C; ++q) {
                    const uint32_t v = (q == me) ? ctot[threadIdx.x] : cl.map_shared_rank(ctot, q)[threadIdx.x];
                    all += v;
                    if (q < me) lower += v;
                }
            }
            const uint32_t db = scan256(threadIdx.x < 256 ? all : 0u, wsum);
            if (threadIdx.x < 256) dbase[threadIdx.x] = db + lower;
            __syncthreads();
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                if (e < slots) {
                    const int el = w * EW + e * 32 + lane;
                    const uint32_t key = first ? order_key(xa[fsw(el)]) : kin[el];
                    const uint32_t d = (key >> shift) & 255u;
                    const uint32_t r = (e & 1) ? (rk[e >> 1] >> 16) : (rk[e >> 1] & 0xffffu);
                    const uint32_t dest = dbase[d] + wh[w * 256 + d] + r;  // rank within the curve
                    const uint32_t idx = first ? (uint32_t)(me * L + el) : (uint32_t)iin[el];
                    if (last) {
                        const float v = __ldg(s + dest);
                        const int tq = (int)(idx >> log2L);
                        const int pos = (int)(idx & (uint32_t)(L - 1));
                        float* xs = (float*)V;  // next state
                        if (tq == me) xs[fsw(pos)] = v;
                        else cl.map_shared_rank(xs, tq)[fsw(pos)] = v;
                    } else {
                        const int tq = (int)(dest >> log2L);
                        const int pos = (int)(dest & (uint32_t)(L - 1));
                        if (tq == me) { kout[pos] = key; iout[pos] = (uint16_t)idx; }
                        else {
                            cl.map_shared_rank(kout, tq)[pos] = key;
                            cl.map_shared_rank(iout, tq)[pos] = (uint16_t)idx;
                        }
                    }
                }
            }
            __syncthreads();
            for (int q = threadIdx.x; q < kResWarps * 256; q += kResThreads) wh[q] = 0;
            cl.sync();  // every remote store of this pass has landed
        }
        z = V;
    }
    float2* xo2 = (float2*)xg;
    for (int m = threadIdx.x; m < Mc; m += kResThreads) xo2[m] = z[swz(m)];
    cl.sync();
}

}  // namespace

bool resident_supported(const Plan& p, uint32_t log2n)
{
    return p.use_resident && p.prec == LC_FP32 && log2n >= kResMinLog2 && log2n <= kResClusterMaxLog2;
}

void launch_resident(const Plan& p, const ClassInfo& k, uint32_t n_it, cudaStream_t st, uint64_t* launches)
{
    ResArgs a;
    a.cls_curves = k.d_curves;
    a.curves = p.d_curves;
    a.eff_iters = p.d_eff_iters;
    a.d_iter = p.d_iter;
    a.A = (const float*)p.d_A;
    a.s = (const float*)p.d_s;
    a.x = (float*)p.d_x;
    a.tw = (const float2*)k.d_tw;
    a.n_it = n_it;
    a.log2n = k.log2n;
    const int C = k.log2n <= kResMaxLog2 ? 1 : 1 << (k.log2n - kResMaxLog2);
    const size_t L = ((size_t)1 << k.log2n) / C;
    const size_t smem = 12 * L + (size_t)kResWarps * 256 * 2;
    const int smax = (int)(12 * ((size_t)1 << kResMaxLog2) + (size_t)kResWarps * 256 * 2);
    if (C == 1) {
        cudaFuncSetAttribute(k_resident_cta, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
        k_resident_cta<<<k.ncurves, kResThreads, smem, st>>>(a);
    } else if (C == 2) {
        cudaFuncSetAttribute(k_resident_cluster<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
        k_resident_cluster<2><<<k.ncurves * 2, kResThreads, smem, st>>>(a);
    } else {
        cudaFuncSetAttribute(k_resident_cluster<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
        k_resident_cluster<4><<<k.ncurves * 4, kResThreads, smem, st>>>(a);
    }
    if (launches) ++*launches;
}

}  // namespace lc
