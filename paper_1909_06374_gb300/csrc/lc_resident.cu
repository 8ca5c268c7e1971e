// lc_resident.cu -- fused, on-chip amplitude-adjustment iterations (Sec. 3.2.2).
//
// One CTA (N <= 2^14) or a cluster of C = N / 2^14 CTAs (N = 2^15, 2^16) owns
// one FP32 curve for all the iterations of a launch.  Per iteration:
//   1. complex Stockham FFT of z[m] = x[2m] + i x[2m+1] (M = N/2 points) in
//      shared memory: radix-16 register butterflies, XOR-swizzled addresses,
//      twiddles from two small shared tables (W^t = W^{128 a} W^b);
//   2. unpack to X_0..X_M, keep the phases, impose A, pack for the inverse;
//   3. inverse complex FFT -> x_adj;
//   4. stable LSD radix sort of the order keys of x_adj (4 passes of 8 bits;
//      ballot-based warp multisplit, per-warp digit counts, block-wide scan);
//   5. x[position] = s[rank].
// A and s stream from L2.  Single CTA: the state never leaves shared memory
// until the end of the launch.  Cluster: the length-M transform is split
// M = C x Mc (a cross-CTA radix-C step and local length-Mc transforms, CTA c
// holding Z[C k + c]); the cross-CTA data goes through L2 -- on this GPU L2
// moves ~10 TB/s between the SMs of a cluster against ~1-2.5 TB/s for
// distributed shared memory -- in a per-curve exchange area, ordered by
// cluster barriers (release/acquire).  Each CTA sorts its 2^14 keys locally
// and merges ranks against the partners' published sorted keys; the rank
// gather writes the next state straight into the curve's state array.
#include <cooperative_groups.h>

#include "lc_dft.cuh"
#include "lc_internal.h"

namespace lc {

namespace {

namespace cg = cooperative_groups;

constexpr int kResThreads = 512;
constexpr int kResWarps = kResThreads / 32;
constexpr uint32_t kResMinLog2 = 10;
constexpr uint32_t kResMaxLog2 = 14;          // one CTA
constexpr uint32_t kResAutoMaxLog2 = 12;      // the auto mode's crossover (autotune.py sweep)
constexpr uint32_t kResClusterMaxLog2 = 16;   // clusters of 2 or 4 CTAs
constexpr int kTwLo = 128;                    // low twiddle table (W^b, b < 128)
constexpr int kTwHiMax = 64;                  // high table (W^{128 a}), Mc <= 8192
constexpr size_t kWhBytes = (size_t)kResWarps * 256 * 4;
constexpr size_t kTwBytes = (size_t)(kTwLo + kTwHiMax) * 8;

__device__ __forceinline__ int swz(int e) { return e ^ ((e >> 4) & 15); }
// float index f of a swizzled complex buffer
__device__ __forceinline__ int fsw(int f) { return (swz(f >> 1) << 1) | (f & 1); }

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// e^{-2 pi i k/N} for k in [0, N) from the class table rt (k < N/2).
__device__ __forceinline__ float2 twN(const float2* __restrict__ rt, int k, int M)
{
    if (k < M) return __ldg(rt + k);
    const float2 w = __ldg(rt + (k - M));
    return make_float2(-w.x, -w.y);
}

// Shared twiddle tables of the local length-Mc transform: lo[b] = W_Mc^b,
// hi[a] = W_Mc^{128 a}; W_Mc^t = e^{-2 pi i (t 2^log2ratio)/N}.
__device__ __forceinline__ void build_tw(float2* lo, float2* hi, const float2* __restrict__ rt, int log2Mc,
                                         int log2ratio, int M)
{
    const int Mc = 1 << log2Mc;
    const int nhi = Mc > kTwLo ? Mc / kTwLo : 1;
    for (int t = threadIdx.x; t < kTwLo + nhi; t += kResThreads) {
        if (t < kTwLo) lo[t] = t < Mc ? twN(rt, t << log2ratio, M) : make_float2(1.f, 0.f);
        else hi[t - kTwLo] = twN(rt, ((t - kTwLo) * kTwLo) << log2ratio, M);
    }
}

__device__ __forceinline__ float2 tw_smem(const float2* lo, const float2* hi, int t)
{
    return cmulf(hi[t >> 7], lo[t & (kTwLo - 1)]);
}

// One radix-R Stockham pass of the length-Mc complex transform in shared memory.
template <int R, bool INV>
__device__ __forceinline__ void smem_pass(const float2* __restrict__ in, float2* __restrict__ out, int log2Mc,
                                          int log2p, const float2* lo, const float2* hi)
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
                float2 w = tw_smem(lo, hi, r * step);
                if (INV) w.y = -w.y;
                u[r] = cmulf(u[r], w);
            }
        }
        dft_regs<float, R, INV>(u);
        const int j = ((i - k) << LR) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) out[swz(j + r * p)] = u[r];
    }
}

// Complex FFT of length 2^log2Mc held in shared memory (swizzled), ping-
// ponging between a and b; returns the buffer holding the result.
template <bool INV>
__device__ float2* smem_fft(float2* a, float2* b, int log2Mc, const float2* lo, const float2* hi)
{
    int log2p = 0;
    float2* in = a;
    float2* out = b;
    const int rem = log2Mc & 3;
    if (rem) {
        if (rem == 1) smem_pass<2, INV>(in, out, log2Mc, 0, lo, hi);
        else if (rem == 2) smem_pass<4, INV>(in, out, log2Mc, 0, lo, hi);
        else smem_pass<8, INV>(in, out, log2Mc, 0, lo, hi);
        __syncthreads();
        log2p = rem;
        float2* t = in; in = out; out = t;
    }
    for (; log2p < log2Mc; log2p += 4) {
        smem_pass<16, INV>(in, out, log2Mc, log2p, lo, hi);
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

// Z'_K from Z_K, Z_{M-K}: X_K = E + W O, X_{M-K} = conj(E - W O) with
// E = (Z_K + conj Z_{M-K})/2, O = (Z_K - conj Z_{M-K})/(2i); Y = A X/|X|;
// Z'_K = E' + i O', E' = Y_K + conj Y_{M-K}, O' = (Y_K - conj Y_{M-K}) conj W.
// Called with the pair swapped and W -> -conj(W) it gives Z'_{M-K}.
__device__ __forceinline__ float2 spectral_pair(float2 za, float2 zb, float2 W, float AK, float AMK)
{
    const float2 E = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y));
    const float2 O = make_float2(0.5f * (za.y + zb.y), -0.5f * (za.x - zb.x));
    const float2 WO = cmulf(W, O);
    const float2 XK = make_float2(E.x + WO.x, E.y + WO.y);
    const float2 XMK = make_float2(E.x - WO.x, -(E.y - WO.y));
    const float2 YK = keep_phase_f(XK, AK);
    const float2 YMK = keep_phase_f(XMK, AMK);
    const float2 Ep = make_float2(YK.x + YMK.x, YK.y - YMK.y);
    const float2 Dd = make_float2(YK.x - YMK.x, YK.y + YMK.y);
    const float2 Op = cmulf(Dd, make_float2(W.x, -W.y));
    return make_float2(Ep.x - Op.y, Ep.y + Op.x);
}

// Spectral step with every pair (k, M-k) local (single CTA).
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
            const float AK = __ldg(A + k), AMK = __ldg(A + M - k);
            Zo[swz(k)] = spectral_pair(za, zb, W, AK, AMK);
            Zo[swz(M - k)] = spectral_pair(zb, za, make_float2(-W.x, W.y), AMK, AK);
        }
    }
}

// Lanes of the warp holding the same 8-bit digit: eight ballots, one per bit
// (the match instruction runs on a low-throughput pipe on this GPU).
__device__ __forceinline__ uint32_t digit_peers(uint32_t d)
{
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const uint32_t bal = __ballot_sync(0xffffffffu, (d >> b) & 1u);
        peers &= ((d >> b) & 1u) ? bal : ~bal;
    }
    return peers;
}

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
    uint32_t* eff_iters;  // lowered when the convergence test stops a curve
    const int* d_iter;
    const float* A;
    const float* s;
    float* x;
    const float2* tw;
    float* rx;           // cluster exchange area: 3 N floats per curve of the class
    uint32_t n_it;
    uint32_t log2n;
    ConvDev conv;        // convergence test (Sec. 3.2.2, Eq. 4); conv.delta null: off
};

// Sum of one float per thread of the CTA in FP64, in a fixed order (warp
// tree, then warps in order); every thread gets the result.  red: kResWarps
// doubles of shared memory.
__device__ __forceinline__ double cta_sum(float v, double* red)
{
    double d = (double)v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kResWarps; ++w) t += red[w];
    return t;
}

// One stable LSD radix pass over the L = 2^LOG2L keys of the CTA (warp w
// owns elements [w L/16, (w+1) L/16), lane-striped).  FIRST: keys are the
// order keys of the x_adj floats in xa (swizzled); positions are implicit.
// GATHER: instead of the sorted pairs, writes xn[position] = s[rank].
// Ranking runs in two phases: the digits and ballot masks of all the warp's
// slots (independent, so their ballot chains overlap), then the short chain
// of per-warp digit counters in shared memory.
template <int LOG2L, bool FIRST, bool GATHER>
__device__ __forceinline__ void radix_pass(const float* __restrict__ xa, const uint32_t* __restrict__ kin,
                                           uint32_t* __restrict__ kout, const uint16_t* __restrict__ iin,
                                           uint16_t* __restrict__ iout, float* __restrict__ xn,
                                           const float* __restrict__ s, int shift, uint32_t* wh,
                                           uint32_t* dbase, uint32_t* wsum)
{
    constexpr int EW = 1 << (LOG2L - 4);  // elements per warp
    constexpr int SLOTS = EW >> 5;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    constexpr int G = SLOTS < 8 ? SLOTS : 8;  // slots ranked per group (register budget)
    uint32_t rk[(SLOTS + 1) / 2];  // within-(warp, digit) ranks, two 16-bit values per register
#pragma unroll
    for (int g0 = 0; g0 < SLOTS; g0 += G) {
        uint32_t info[G];  // digit | below << 8 | count << 16
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int el = w * EW + (g0 + q) * 32 + lane;
            const uint32_t key = FIRST ? order_key(xa[fsw(el)]) : kin[el];
            const uint32_t d = (key >> shift) & 255u;
            // every third slot on the match pipe, the others on ballots: the two
            // run on different pipes, which cut the pass time by ~10% here
            const uint32_t peers = ((g0 + q) % 3 == 2) ? __match_any_sync(0xffffffffu, d) : digit_peers(d);
            info[q] = d | ((uint32_t)__popc(peers & lt) << 8) | ((uint32_t)__popc(peers) << 16);
        }
#pragma unroll
        for (int q = 0; q < G; ++q) {
            const int e = g0 + q;
            const uint32_t d = info[q] & 255u, below = (info[q] >> 8) & 255u;
            const uint32_t base = wh[w * 256 + d];
            __syncwarp();
            if (below == 0) wh[w * 256 + d] = base + (info[q] >> 16);
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
            wh[q * 256 + d] = tot;
            tot += v;
        }
    }
    const uint32_t db = scan256(threadIdx.x < 256 ? tot : 0u, wsum);
    if (threadIdx.x < 256) dbase[threadIdx.x] = db;
    __syncthreads();
#pragma unroll
    for (int e = 0; e < SLOTS; ++e) {
        const int el = w * EW + e * 32 + lane;
        const uint32_t key = FIRST ? order_key(xa[fsw(el)]) : kin[el];
        const uint32_t d = (key >> shift) & 255u;
        const uint32_t r = (e & 1) ? (rk[e >> 1] >> 16) : (rk[e >> 1] & 0xffffu);
        const uint32_t dest = dbase[d] + wh[w * 256 + d] + r;
        const uint32_t idx = FIRST ? (uint32_t)el : (uint32_t)iin[el];
        if (GATHER) {
            xn[fsw((int)idx)] = __ldg(s + dest);
        } else {
            kout[dest] = key;
            iout[dest] = (uint16_t)idx;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kResWarps * 256; q += kResThreads) wh[q] = 0;
    __syncthreads();
}

// ------------------------------------------------------------- one CTA
template <int LOG2L, bool CONV>
__global__ void __launch_bounds__(kResThreads, 1) k_resident_cta(const ResArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int log2L = LOG2L;
    const int L = 1 << log2L;
    const int M = L >> 1;
    float2* buf0 = (float2*)smem;
    float2* buf1 = (float2*)(smem + (size_t)4 * L);
    uint16_t* ia = (uint16_t*)(smem + (size_t)8 * L);
    uint16_t* ib = (uint16_t*)(smem + (size_t)10 * L);
    uint32_t* wh = (uint32_t*)(smem + (size_t)12 * L);
    float2* twlo = (float2*)(smem + (size_t)12 * L + kWhBytes);
    float2* twhi = twlo + kTwLo;
    __shared__ uint32_t dbase[256];
    __shared__ uint32_t wsum[8];
    __shared__ double red[kResWarps];

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
    build_tw(twlo, twhi, a.tw, log2L - 1, 1, M);
    const float2* xg2 = (const float2*)xg;
    for (int m = threadIdx.x; m < M; m += kResThreads) buf0[swz(m)] = xg2[m];
    __syncthreads();

    float2* z = buf0;
    float2* o = buf1;
    for (int it = 0; it < n_act; ++it) {
        float2* Z = smem_fft<false>(z, o, log2L - 1, twlo, twhi);
        float2* Zs = (Z == buf0) ? buf1 : buf0;
        spectral_local(Z, Zs, A, a.tw, M);
        __syncthreads();
        float2* X = smem_fft<true>(Zs, Z, log2L - 1, twlo, twhi);
        float2* other = (X == buf0) ? buf1 : buf0;
        uint32_t* kX = (uint32_t*)X;
        uint32_t* kO = (uint32_t*)other;
        // pass 0: x_adj (in X) -> keys in other; 1: other -> X; 2: X -> other; 3: other -> x in X
        radix_pass<LOG2L, true, false>((const float*)X, nullptr, kO, nullptr, ia, nullptr, s, 0, wh, dbase, wsum);
        radix_pass<LOG2L, false, false>(nullptr, kO, kX, ia, ib, nullptr, s, 8, wh, dbase, wsum);
        radix_pass<LOG2L, false, false>(nullptr, kX, kO, ib, ia, nullptr, s, 16, wh, dbase, wsum);
        radix_pass<LOG2L, false, true>(nullptr, kO, nullptr, ia, nullptr, (float*)X, s, 24, wh, dbase, wsum);
        z = X;
        o = other;
        if (CONV) {
            // Eq. 4 against the previous iterate, which the state in global
            // memory holds in this mode (it is rewritten every iteration)
            __syncthreads();
            const float* Xf = (const float*)X;
            float lsum = 0.0f;
            constexpr int PER = (1 << LOG2L) / kResThreads;  // 2 .. 32 samples per thread
            constexpr int G = PER < 8 ? PER : 8;              // loads issued before stores
#pragma unroll
            for (int g0 = 0; g0 < PER; g0 += G) {
                float xn[G], xo[G];
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    const int m = threadIdx.x + (g0 + j) * kResThreads;
                    xo[j] = xg[m];
                    xn[j] = Xf[fsw(m)];
                }
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    lsum += ln_ratio_sq(xn[j], xo[j]);
                    xg[threadIdx.x + (g0 + j) * kResThreads] = xn[j];
                }
            }
            const double delta = conv_delta(cta_sum(lsum, red), (double)L);
            const bool stop = delta < a.conv.thr[c];
            if (threadIdx.x == 0) {
                conv_record(a.conv, c, it0 + it, delta);
                if (stop) a.eff_iters[c] = (uint32_t)(it0 + it + 1);
            }
            if (stop) break;
        }
    }
    float2* xo2 = (float2*)xg;
    for (int m = threadIdx.x; m < M; m += kResThreads) xo2[m] = z[swz(m)];
}

// ------------------------------------------------------------- clusters
// First index i >= from with !(sorted[i] < key) (STRICT) or !(sorted[i] <= key),
// i.e. the number of keys of sorted[0, n) below / not above `key`, given that
// the first `from` keys already are: galloping probe, then binary search.
template <bool STRICT>
__device__ __forceinline__ int advance_count(const uint32_t* sorted, int n, int from, uint32_t key)
{
    int lo = from, step = 1;
    while (lo + step <= n) {
        const uint32_t v = sorted[lo + step - 1];
        if (!(STRICT ? (v < key) : (v <= key))) break;
        lo += step;
        step <<= 1;
    }
    int hi = lo + step - 1 < n ? lo + step - 1 : n;  // answer in [lo, hi]
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const uint32_t v = sorted[mid];
        if (STRICT ? (v < key) : (v <= key)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <int C, bool CONV>
__global__ void __cluster_dims__(C, 1, 1) __launch_bounds__(kResThreads, 1) k_resident_cluster(const ResArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    cg::cluster_group cl = cg::this_cluster();
    const int me = (int)cl.block_rank();
    constexpr int LOGC = ilog2c(C);
    constexpr int log2L = (int)kResMaxLog2;  // every CTA holds 2^14 samples
    const int L = 1 << log2L;
    const int Mc = L >> 1;
    const int M = C * Mc;
    const int N = 2 * M;
    float2* buf0 = (float2*)smem;
    float2* buf1 = (float2*)(smem + (size_t)4 * L);
    uint16_t* ia = (uint16_t*)(smem + (size_t)8 * L);
    uint16_t* ib = (uint16_t*)(smem + (size_t)10 * L);
    uint32_t* wh = (uint32_t*)(smem + (size_t)12 * L);
    float2* twlo = (float2*)(smem + (size_t)12 * L + kWhBytes);
    float2* twhi = twlo + kTwLo;
    __shared__ uint32_t dbase[256];
    __shared__ uint32_t wsum[8];
    __shared__ double red[kResWarps];

    const int ci = blockIdx.x / C;
    const int c = a.cls_curves[ci];
    const CurveDev& cv = a.curves[c];
    const int it0 = *a.d_iter;
    int n_act = (int)a.eff_iters[c] - it0;
    if (n_act > (int)a.n_it) n_act = (int)a.n_it;
    if (n_act <= 0) return;  // the same for every CTA of the cluster
    const float* A = a.A + cv.offh;
    const float* s = a.s + cv.off;
    float* xs = a.x + cv.off;                             // state, all N samples
    float2* gsp = (float2*)(a.rx + (size_t)ci * 3 * N);  // packed spectra (M complex)
    float2* gu = gsp + M;                                 // inverse-step inputs (M complex)
    uint32_t* gk = (uint32_t*)(gu + M);                  // sorted keys (N)
    const float2* rt = a.tw;

    float2 wc[C];  // W_C^{q me}
#pragma unroll
    for (int q = 0; q < C; ++q) wc[q] = twN(rt, ((q * me) % C) * (N / C), M);
    for (int q = threadIdx.x; q < kResWarps * 256; q += kResThreads) wh[q] = 0;
    build_tw(twlo, twhi, rt, log2L - 1, LOGC + 1, M);
    __syncthreads();

    const float2* xs2 = (const float2*)xs;
    const int pr = (C - me) % C;
    for (int it = 0; it < n_act; ++it) {
        // forward cross-CTA radix-C step from the state in L2:
        // y[m] = W_M^{m me} sum_q z[q Mc + m] W_C^{q me}
        for (int m = threadIdx.x; m < Mc; m += kResThreads) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < C; ++q) {
                const float2 t = cmulf(__ldcg(xs2 + q * Mc + m), wc[q]);
                acc.x += t.x; acc.y += t.y;
            }
            buf0[swz(m)] = cmulf(acc, twN(rt, 2 * m * me, M));
        }
        __syncthreads();
        float2* P = smem_fft<false>(buf0, buf1, log2L - 1, twlo, twhi);  // Z[C k + me]
        float2* Q = (P == buf0) ? buf1 : buf0;
        for (int k = threadIdx.x; k < Mc; k += kResThreads) __stcg(gsp + me * Mc + k, P[swz(k)]);
        cl.sync();  // every Z block published
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
                const float2 zb = pr == me ? P[swz(kp)] : __ldcg(gsp + pr * Mc + kp);
                out = spectral_pair(P[swz(k)], zb, twN(rt, K, M), __ldg(A + K), __ldg(A + M - K));
            }
            Q[swz(k)] = out;
        }
        __syncthreads();
        float2* U = smem_fft<true>(Q, P, log2L - 1, twlo, twhi);
        float2* V = (U == buf0) ? buf1 : buf0;
        for (int n = threadIdx.x; n < Mc; n += kResThreads) __stcg(gu + me * Mc + n, U[swz(n)]);
        cl.sync();  // every u block published
        // inverse cross-CTA step: x_adj block me = sum_r e^{+2 pi i r me/C} e^{+2 pi i r n/M} u_r[n]
        for (int n = threadIdx.x; n < Mc; n += kResThreads) {
            float2 acc = make_float2(0.f, 0.f);
#pragma unroll
            for (int r = 0; r < C; ++r) {
                const float2 v = r == me ? U[swz(n)] : __ldcg(gu + r * Mc + n);
                const float2 tw = twN(rt, 2 * r * n, M);
                const float2 t = cmulf(cmulf(v, make_float2(tw.x, -tw.y)), make_float2(wc[r].x, -wc[r].y));
                acc.x += t.x; acc.y += t.y;
            }
            V[swz(n)] = acc;
        }
        __syncthreads();
        // local stable sort of the block's keys (positions are local)
        uint32_t* kU = (uint32_t*)U;
        uint32_t* kV = (uint32_t*)V;
        radix_pass<kResMaxLog2, true, false>((const float*)V, nullptr, kU, nullptr, ia, nullptr, s, 0, wh, dbase, wsum);
        radix_pass<kResMaxLog2, false, false>(nullptr, kU, kV, ia, ib, nullptr, s, 8, wh, dbase, wsum);
        radix_pass<kResMaxLog2, false, false>(nullptr, kV, kU, ib, ia, nullptr, s, 16, wh, dbase, wsum);
        radix_pass<kResMaxLog2, false, false>(nullptr, kU, kV, ia, ib, nullptr, s, 24, wh, dbase, wsum);
        // sorted keys in kV, positions in ib; publish the keys
        for (int p = threadIdx.x; p < L; p += kResThreads) __stcg(gk + me * L + p, kV[p]);
        cl.sync();  // every sorted block published
        // global rank = local rank + keys of lower CTAs not above it + keys of
        // higher CTAs below it (ties: lower position first, i.e. lower CTA first)
        uint32_t gr[16];  // global ranks (< 2^16), two per register
        const int per = L / kResThreads;  // consecutive sorted positions per thread
#pragma unroll
        for (int e = 0; e < 32; e += 2)
            if (e < per) gr[e >> 1] = (uint32_t)(threadIdx.x * per + e) | ((uint32_t)(threadIdx.x * per + e + 1) << 16);
        uint32_t* part = kU;  // free: holds a partner's sorted keys
        for (int q = 0; q < C; ++q) {
            if (q == me) continue;
            for (int p = threadIdx.x; p < L; p += kResThreads) part[p] = __ldcg(gk + q * L + p);
            __syncthreads();
            int cnt = 0;
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                if (e < per) {
                    const uint32_t key = kV[threadIdx.x * per + e];
                    cnt = q < me ? advance_count<false>(part, L, cnt, key) : advance_count<true>(part, L, cnt, key);
                    gr[e >> 1] += (uint32_t)cnt << ((e & 1) * 16);
                }
            }
            __syncthreads();
        }
        // rank-order replacement straight into the state in L2 (with the
        // convergence test, the old value there enters Eq. 4 first)
        constexpr bool conv = CONV;
        float lsum = 0.0f;
        if (!conv) {
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                if (e < per) {
                    const int p = threadIdx.x * per + e;
                    __stcg(xs + me * L + ib[p], __ldg(s + ((gr[e >> 1] >> ((e & 1) * 16)) & 0xffffu)));
                }
            }
        } else {
            // groups of 8: the old values' loads are issued before the stores
#pragma unroll
            for (int e0 = 0; e0 < 32; e0 += 8) {
                if (e0 < per) {
                    float xn[8], xo[8];
#pragma unroll
                    for (int e = e0; e < e0 + 8; ++e) {
                        const int p = threadIdx.x * per + e;
                        xn[e - e0] = __ldg(s + ((gr[e >> 1] >> ((e & 1) * 16)) & 0xffffu));
                        xo[e - e0] = __ldcg(xs + me * L + ib[p]);
                    }
#pragma unroll
                    for (int e = e0; e < e0 + 8; ++e) {
                        const int p = threadIdx.x * per + e;
                        lsum += ln_ratio_sq(xn[e - e0], xo[e - e0]);
                        __stcg(xs + me * L + ib[p], xn[e - e0]);
                    }
                }
            }
        }
        if (conv) {
            const double part = cta_sum(lsum, red);
            if (threadIdx.x == 0) __stcg(a.conv.part + (size_t)ci * C + me, part);
        }
        cl.sync();  // the next state (and every CTA's partial sum) is complete
        if (conv) {
            // every CTA sums the C partials in the same order, so all take the
            // same decision; a partial is rewritten only after the next
            // iteration's first cluster barrier, when all have read it
            double sum = 0.0;
#pragma unroll
            for (int q = 0; q < C; ++q) sum += __ldcg(a.conv.part + (size_t)ci * C + q);
            const double delta = conv_delta(sum, (double)N);
            const bool stop = delta < a.conv.thr[c];
            if (me == 0 && threadIdx.x == 0) {
                conv_record(a.conv, c, it0 + it, delta);
                if (stop) a.eff_iters[c] = (uint32_t)(it0 + it + 1);
            }
            if (stop) break;
        }
    }
}

template <int LOG2L>
void launch_cta(const ResArgs& a, int ncurves, size_t smem, cudaStream_t st)
{
    if (a.conv.delta) k_resident_cta<LOG2L, true><<<ncurves, kResThreads, smem, st>>>(a);
    else k_resident_cta<LOG2L, false><<<ncurves, kResThreads, smem, st>>>(a);
}

template <int C>
void launch_cluster(const ResArgs& a, int ncurves, size_t smem, cudaStream_t st)
{
    if (a.conv.delta) k_resident_cluster<C, true><<<ncurves * C, kResThreads, smem, st>>>(a);
    else k_resident_cluster<C, false><<<ncurves * C, kResThreads, smem, st>>>(a);
}

// Shared memory of the fused kernels at their longest one-CTA length (the
// cluster kernels hold the same per CTA).
constexpr size_t kResSmemMax = 12 * ((size_t)1 << kResMaxLog2) + kWhBytes + kTwBytes;

template <typename F>
cudaError_t res_attr(F* f)
{
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kResSmemMax);
}

}  // namespace

// Every fused-kernel instantiation may use up to kResSmemMax bytes of dynamic
// shared memory; set once per device (see prepare_kernels).
cudaError_t resident_kernel_attributes()
{
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = res_attr(k_resident_cta<10, false>);
    if (e == cudaSuccess) e = res_attr(k_resident_cta<10, true>);
    if (e == cudaSuccess) e = res_attr(k_resident_cta<11, false>);
    if (e == cudaSuccess) e = res_attr(k_resident_cta<11, true>);
    if (e == cudaSuccess) e = res_attr(k_resident_cta<12, false>);
    if (e == cudaSuccess) e = res_attr(k_resident_cta<12, true>);
    if (e == cudaSuccess) e = res_attr(k_resident_cta<13, false>);
    if (e == cudaSuccess) e = res_attr(k_resident_cta<13, true>);
    if (e == cudaSuccess) e = res_attr(k_resident_cta<14, false>);
    if (e == cudaSuccess) e = res_attr(k_resident_cta<14, true>);
    if (e == cudaSuccess) e = res_attr(k_resident_cluster<2, false>);
    if (e == cudaSuccess) e = res_attr(k_resident_cluster<2, true>);
    if (e == cudaSuccess) e = res_attr(k_resident_cluster<4, false>);
    if (e == cudaSuccess) e = res_attr(k_resident_cluster<4, true>);
    return e;
}

// Path table of the auto mode: the one-CTA fused kernel from 2^10 to 2^12,
// the multi-kernel path above (autotune.py on GB300, 2^26 samples x 20
// iterations, sample*iter/s fused vs multi-kernel: 2^12 3.79e10 vs 2.51e10,
// 2^13 4.22e10 vs 4.48e10, 2^14 3.99e10 vs 4.87e10, 2^15 2.20e10 for the
// 2-CTA cluster kernel vs 4.92e10).  With the LSD argsort the crossover was
// 2^14.  LC_RESIDENT_MAX_LOG2 (up to 14 for the one-CTA kernel) moves it;
// LC_PATH=resident also runs the cluster kernels at 2^15 and 2^16.
bool resident_supported(const Plan& p, uint32_t log2n)
{
    if (p.prec != LC_FP32 || log2n < kResMinLog2) return false;
    if (p.path_mode == 2) return false;
    if (p.path_mode == 1) return log2n <= kResClusterMaxLog2;
    return log2n <= (uint32_t)(p.res_max_log2 >= 0 ? p.res_max_log2 : (int)kResAutoMaxLog2);
}

size_t resident_exchange_floats(uint32_t log2n)
{
    return log2n > kResMaxLog2 && log2n <= kResClusterMaxLog2 ? (size_t)3 << log2n : 0;
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
    a.rx = k.d_rx;
    a.n_it = n_it;
    a.log2n = k.log2n;
    a.conv = conv_of(p);
    const int C = k.log2n <= kResMaxLog2 ? 1 : 1 << (k.log2n - kResMaxLog2);
    const size_t L = ((size_t)1 << k.log2n) / C;
    const size_t smem = 12 * L + kWhBytes + kTwBytes;
    if (C == 1) {
        switch (k.log2n) {
        case 10: launch_cta<10>(a, k.ncurves, smem, st); break;
        case 11: launch_cta<11>(a, k.ncurves, smem, st); break;
        case 12: launch_cta<12>(a, k.ncurves, smem, st); break;
        case 13: launch_cta<13>(a, k.ncurves, smem, st); break;
        default: launch_cta<14>(a, k.ncurves, smem, st); break;
        }
    } else if (C == 2) {
        launch_cluster<2>(a, k.ncurves, smem, st);
    } else {
        launch_cluster<4>(a, k.ncurves, smem, st);
    }
    if (launches) ++*launches;
}

}  // namespace lc
