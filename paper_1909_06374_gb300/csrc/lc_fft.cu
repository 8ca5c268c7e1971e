// lc_fft.cu -- batched Stockham FFT passes and the fused spectral step of one
// amplitude-adjustment iteration (Sec. 2.1 third step; Sec. 3.2.2).
//
// A real series of N = 2M samples is transformed as the complex series
// z[n] = x[2n] + i x[2n+1] of length M (the float array reinterpreted), so the
// forward transform reads the state in place and the inverse transform writes
// the real series directly.  The spectral kernel unpacks the half-length
// spectrum into X_0..X_M, imposes the target amplitudes keeping the phases,
// and packs the result for the inverse transform, all in one pass over the
// conjugate pairs (k, M-k).
#include "lc_dft.cuh"
#include "lc_internal.h"

namespace lc {

// W_M^t = e^{-2 pi i t/M} from the class table rt[k] = e^{-2 pi i k/N} (N = 2M).
template <typename T>
__device__ __forceinline__ cplx<T> twiddle_M(const cplx<T>* __restrict__ rt, uint64_t t, uint64_t M)
{
    if (2 * t < M) return rt[2 * t];
    cplx<T> w = rt[2 * t - M];
    w.x = -w.x; w.y = -w.y;
    return w;
}

// W_M^e (e < M <= 2^26) from three shared-memory tables of 512 entries,
// W^e = W^{e2 2^18} W^{e1 2^9} W^{e0} (e = e2 2^18 + e1 2^9 + e0; the top
// level only when M > 2^18), each entry read from the class table once per
// block.  Replaces scattered reads of the class table, whose per-block
// footprint is several times the block's data.
constexpr int kTwLevel = 512;
template <typename T>
struct SmemTw {
    const cplx<T>* t0;
    const cplx<T>* t1;
    const cplx<T>* t2;
    const cplx<T>* tR;  // W_R^e, e < R: every twiddle of a radix-R pass's sub-passes
    bool three;
    __device__ __forceinline__ cplx<T> operator()(uint32_t e) const
    {
        cplx<T> w = cmul(t1[(e >> 9) & (kTwLevel - 1)], t0[e & (kTwLevel - 1)]);
        if (three) w = cmul(t2[e >> 18], w);
        return w;
    }
};

__host__ __device__ constexpr int smem_tw_entries(int log2M, int LR)
{
    return kTwLevel + (log2M >= 18 ? kTwLevel : (1 << (log2M - 9))) + (log2M > 18 ? (1 << (log2M - 18)) : 0) +
           (1 << LR);
}

// Fills the tables at `mem` (smem_tw_entries(log2M, LR) entries: 512, then
// the 2^(log2M-9) or 512 of the second level, then those of the third, then
// W_R^e = W_M^{e M/R} for e < R = 2^LR, each read from the class table) for a
// radix-R pass of a length-M transform; ends with a block barrier.
template <typename T>
__device__ __forceinline__ SmemTw<T> build_smem_tw(cplx<T>* mem, const cplx<T>* __restrict__ rt, int log2M, int LR)
{
    const uint64_t M = 1ull << log2M;
    SmemTw<T> tw;
    tw.t0 = mem;
    tw.three = log2M > 18;
    const int n1 = log2M >= 18 ? kTwLevel : (1 << (log2M - 9));
    const int n2 = log2M > 18 ? (1 << (log2M - 18)) : 0;
    const int lv = kTwLevel + n1 + n2;
    tw.t1 = mem + kTwLevel;
    tw.t2 = mem + kTwLevel + n1;
    tw.tR = mem + lv;
    for (int x = threadIdx.x; x < lv + (1 << LR); x += blockDim.x) {
        uint64_t e;
        if (x < kTwLevel) e = (uint64_t)x;
        else if (x < kTwLevel + n1) e = (uint64_t)(x - kTwLevel) << 9;
        else if (x < lv) e = (uint64_t)(x - kTwLevel - n1) << 18;
        else e = (uint64_t)(x - lv) << (log2M - LR);
        mem[x] = twiddle_M<T>(rt, e, M);
    }
    __syncthreads();
    return tw;
}

// Table e^{-2 pi i k/N}, k < N/2, computed in FP64 and rounded once to T.
template <typename T>
__global__ void k_twiddles(cplx<T>* __restrict__ rt, uint32_t log2n)
{
    const uint64_t M = 1ull << (log2n - 1);
    for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < M;
         k += (uint64_t)gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-(double)k / (double)M, &s, &c);
        cplx<T> w; w.x = (T)c; w.y = (T)s;
        rt[k] = w;
    }
}

struct PassArgs {
    const int* cls_curves;
    const CurveDev* curves;
    const uint32_t* eff_iters;
    const int* d_iter;   // null: every curve active
    const void* tw;
    const void* in;
    void* out;
    int ncurves;
    uint32_t log2M;
    uint32_t log2p;
    // inverse last pass of a sample-sorted class: every (M/2^(smp_shift))-th
    // output's real part, at complex index d with d mod 2^smp_shift =
    // 2^(smp_shift-1), also goes to smp[ci smp_words + d >> smp_shift] (null:
    // no sample)
    float* smp;
    uint32_t smp_words;
    uint32_t smp_shift;
};

// One radix-R Stockham pass (decimation in time, natural-order output) over
// every curve of a class: with span p, butterfly i (k = i mod p) reads
// u_r = z[i + r M/R], applies W_{Rp}^{rk}, takes an R-point DFT and writes
// y[(i-k)R + k + r p].
template <typename T, int R, bool INV>
__global__ void __launch_bounds__(256) k_fft_pass(const PassArgs a)
{
    using V = cplx<T>;
    constexpr int LR = ilog2c(R);
    const uint32_t log2nb = a.log2M - LR;
    const uint64_t nb = 1ull << log2nb;
    const uint64_t total = (uint64_t)a.ncurves << log2nb;
    const uint64_t p = 1ull << a.log2p;
    const uint64_t M = 1ull << a.log2M;
    const int it = a.d_iter ? *a.d_iter : 0;
    const V* __restrict__ rt = (const V*)a.tw;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const int ci = (int)(t >> log2nb);
        const uint64_t i = t & (nb - 1);
        const int c = a.cls_curves[ci];
        if (a.d_iter && (uint32_t)it >= a.eff_iters[c]) continue;
        const uint64_t base = a.curves[c].off >> 1;
        const V* __restrict__ src = (const V*)a.in + base;
        V* __restrict__ dst = (V*)a.out + base;
        V u[R];
#pragma unroll
        for (int r = 0; r < R; ++r) u[r] = src[i + (uint64_t)r * nb];
        const uint64_t k = i & (p - 1);
        if (p > 1) {
            const uint64_t step = k << (a.log2M - LR - a.log2p);
#pragma unroll
            for (int r = 1; r < R; ++r) {
                V w = twiddle_M<T>(rt, (uint64_t)r * step, M);
                if (INV) w.y = -w.y;
                u[r] = cmul(u[r], w);
            }
        }
        dft_regs<T, R, INV>(u);
        const uint64_t j = ((i - k) << LR) + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[j + (uint64_t)r * p] = u[r];
    }
}

// One Stockham pass of radix R = 2^LR computed in shared memory over a tile
// of C adjacent columns i0..i0+C-1 of one curve (C = tile_cols: R C = 4096
// elements for FP32 and R <= 256, so that every radix-16 sub-pass gives each of the
// 256 threads one butterfly): the tile loads u_r[i] = z[i + r M/R]
// (coalesced runs of C columns), applies W_{Rp}^{r k}, takes the R-point DFT
// of every column by radix-16 Stockham sub-passes in one shared-memory buffer
// (rows padded to C+1 elements; each sub-pass reads its butterflies into
// registers, then overwrites the buffer), and stores y[(i-k)R + k + q p]
// (coalesced along i, or along q when p = 1).
// (FP64 keeps C = 16: with its radices a span 1 < p < C would occur.)
__host__ __device__ constexpr int tile_cols(int LR, int elem_bytes)
{
    return (LR >= 8 || elem_bytes > 8) ? 16 : (4096 >> LR);
}

template <typename T, int Q, bool INV, int LR, int C>
__device__ __forceinline__ void tile_subpass(cplx<T>* __restrict__ buf, int log2p2, const SmemTw<T>& tw, int log2M)
{
    using V = cplx<T>;
    constexpr int LQ = ilog2c(Q);
    constexpr int LC = ilog2c(C);
    constexpr int S = C + 1;                     // row stride
    constexpr int R = 1 << LR;
    constexpr int nbq = R >> LQ;                 // butterflies per column
    constexpr int NB = nbq * C;                  // butterflies of the tile
    constexpr int BPT = (NB + 255) / 256;        // per thread
    const int p2 = 1 << log2p2;
    V u[BPT][Q];
#pragma unroll
    for (int bi = 0; bi < BPT; ++bi) {
        const int b = threadIdx.x + bi * 256;
        if (NB % 256 == 0 || b < NB) {
            const int j = b & (C - 1), i2 = b >> LC;
#pragma unroll
            for (int q = 0; q < Q; ++q) u[bi][q] = buf[(i2 + q * nbq) * S + j];
        }
    }
    __syncthreads();
#pragma unroll
    for (int bi = 0; bi < BPT; ++bi) {
        const int b = threadIdx.x + bi * 256;
        if (NB % 256 == 0 || b < NB) {
            const int j = b & (C - 1), i2 = b >> LC;
            const int k2 = i2 & (p2 - 1);
            if (p2 > 1) {
                // W_{Q p2}^{q k2} = W_R^{q k2 R/(Q p2)}, q k2 < Q p2 <= R
                const int sh = LR - LQ - log2p2;
#pragma unroll
                for (int q = 1; q < Q; ++q) {
                    V w = tw.tR[(q * k2) << sh];
                    if (INV) w.y = -w.y;
                    u[bi][q] = cmul(u[bi][q], w);
                }
            }
            dft_regs<T, Q, INV>(u[bi]);
            const int jo = ((i2 - k2) << LQ) + k2;
#pragma unroll
            for (int q = 0; q < Q; ++q) buf[(jo + q * p2) * S + j] = u[bi][q];
        }
    }
}

// All radix-2^LR sub-passes of one tile of C columns, in place in `buf`: a
// radix-2/4/8 sub-pass for LR mod 4, then radix-16 ones.  Ends with a block
// barrier.
template <typename T, bool INV, int LR, int C>
__device__ __forceinline__ void tile_dft(cplx<T>* __restrict__ buf, const SmemTw<T>& tw, int log2M)
{
    constexpr int rem = LR & 3;
    int log2p2 = 0;
    if (rem) {
        tile_subpass<T, (1 << (rem ? rem : 1)), INV, LR, C>(buf, 0, tw, log2M);
        __syncthreads();
        log2p2 = rem;
    }
    for (; log2p2 < LR; log2p2 += 4) {
        tile_subpass<T, 16, INV, LR, C>(buf, log2p2, tw, log2M);
        __syncthreads();
    }
}

template <typename T, int LR, bool INV, bool MULTI>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && LR < 9) ? 4 : 2)
    k_fft_tile(const __grid_constant__ LaunchSet<PassArgs> set)
{
    uint32_t blk;
    const PassArgs& a = set.pick<MULTI>(blk);
    using V = cplx<T>;
    constexpr int R = 1 << LR;
    constexpr int C = tile_cols(LR, (int)sizeof(V));
    constexpr int LC = ilog2c(C);
    constexpr int S = C + 1;
    extern __shared__ __align__(16) unsigned char tile_smem[];
    V* b0 = (V*)tile_smem;
    V* twm = b0 + R * S;
    const uint32_t log2nb = a.log2M - LR;
    const int tpc = 1 << (log2nb - LC);      // tiles per curve (nb >= C)
    const int ci = (int)blk / tpc;
    const int ti = (int)blk % tpc;
    const int c = a.cls_curves[ci];
    if (a.d_iter && (uint32_t)(*a.d_iter) >= a.eff_iters[c]) return;
    const uint64_t base = a.curves[c].off >> 1;
    const V* __restrict__ src = (const V*)a.in + base;
    V* __restrict__ dst = (V*)a.out + base;
    const V* __restrict__ rt = (const V*)a.tw;
    // indices within a curve stay below M <= 2^26: 32-bit arithmetic
    const uint32_t nb = 1u << log2nb;
    const uint32_t p = 1u << a.log2p;
    const uint32_t i0 = (uint32_t)ti * C;
    constexpr int PER = R * C / 256;  // elements per thread
    V v[PER];
#pragma unroll
    for (int e = 0; e < PER; ++e) {  // every load in flight before any use
        const int idx = threadIdx.x + e * 256;
        v[e] = src[i0 + (uint32_t)(idx & (C - 1)) + (uint32_t)(idx >> LC) * nb];
    }
    const SmemTw<T> tw = build_smem_tw<T>(twm, rt, (int)a.log2M, LR);
#pragma unroll
    for (int e = 0; e < PER; ++e) {
        const int idx = threadIdx.x + e * 256;
        const int r = idx >> LC, j = idx & (C - 1);
        V x = v[e];
        if (p > 1) {
            const uint32_t k = (i0 + (uint32_t)j) & (p - 1);
            V w = tw(((uint32_t)r * k) << (a.log2M - LR - a.log2p));
            if (INV) w.y = -w.y;
            x = cmul(x, w);
        }
        b0[r * S + j] = x;
    }
    __syncthreads();
    tile_dft<T, INV, LR, C>(b0, tw, (int)a.log2M);
    const V* in = b0;
    const uint32_t smask = (1u << a.smp_shift) - 1u, shalf = (smask + 1u) >> 1;
    float* const smp = INV && a.smp ? a.smp + (size_t)ci * a.smp_words : nullptr;
    if (p >= (uint32_t)C) {
        for (int idx = threadIdx.x; idx < R * C; idx += 256) {
            const int q = idx >> LC, j = idx & (C - 1);
            const uint32_t i = i0 + (uint32_t)j, k = i & (p - 1);
            const uint32_t d = ((i - k) << LR) + k + (uint32_t)q * p;
            const V y = in[q * S + j];
            dst[d] = y;
            if (smp && (d & smask) == shalf) smp[d >> a.smp_shift] = (float)y.x;
        }
    } else {  // p == 1 (the host guarantees p == 1 or p >= C): column i owns y[i R .. i R + R)
        for (int idx = threadIdx.x; idx < R * C; idx += 256) {
            const int j = idx >> LR, q = idx & (R - 1);
            const uint32_t d = ((i0 + (uint32_t)j) << LR) + (uint32_t)q;
            const V y = in[q * S + j];
            dst[d] = y;
            if (smp && (d & smask) == shalf) smp[d >> a.smp_shift] = (float)y.x;
        }
    }
}

// Phase kept, amplitude replaced: A X/|X|, and A (phase 0) when X = 0.
__device__ __forceinline__ float2 keep_phase(float2 X, float A)
{
    const float m2 = X.x * X.x + X.y * X.y;
    if (m2 == 0.0f) return make_float2(A, 0.0f);
    const float s = A * rsqrtf(m2);
    return make_float2(X.x * s, X.y * s);
}
__device__ __forceinline__ double2 keep_phase(double2 X, double A)
{
    const double m2 = X.x * X.x + X.y * X.y;
    if (m2 == 0.0) return make_double2(A, 0.0);
    const double s = A / sqrt(m2);
    return make_double2(X.x * s, X.y * s);
}

// Pack Y_k, Y_{M-k} (a Hermitian half spectrum) for the length-M inverse
// transform: Z'_k = E' + i O' with E' = Y_k + conj(Y_{M-k}),
// O' = (Y_k - conj(Y_{M-k})) e^{+2 pi i k/N}; Z'_{M-k} = conj(E') + i conj(O').
template <typename V>
__device__ __forceinline__ void pack_pair(V Yk, V Ym, V W, V& Zk, V& Zm)
{
    const V Ep = cadd(Yk, cconj(Ym));
    const V Op = cmul(csub(Yk, cconj(Ym)), cconj(W));
    Zk.x = Ep.x - Op.y; Zk.y = Ep.y + Op.x;
    Zm.x = Ep.x + Op.y; Zm.y = -Ep.y + Op.x;
}

struct SpecArgs {
    const int* cls_curves;
    const CurveDev* curves;
    const uint32_t* eff_iters;
    const int* d_iter;
    const void* tw;
    const void* Z;       // forward output (iteration) -- unused for TK
    void* Zp;            // packed spectrum for the inverse transform
    const void* A;
    const double2* spec; // TK: FP64 spectrum
    const double* sigma;
    int ncurves;
    uint32_t log2M;
};

// Iteration spectral step (E13): X from the packed forward transform
// (X_k = E_k + W^k O_k with E_k = (Z_k + conj Z_{M-k})/2,
// O_k = (Z_k - conj Z_{M-k})/(2i)), Y = keep_phase(X, A) with
// Y_0 = A_0 and Y_M = A_M sign(X_M), then packed for the inverse.
template <typename T>
__global__ void __launch_bounds__(256) k_spectral_iter(const SpecArgs a)
{
    using V = cplx<T>;
    const uint32_t log2h = a.log2M - 1;
    const uint64_t half = 1ull << log2h;
    const uint64_t M = 1ull << a.log2M;
    const uint64_t total = (uint64_t)a.ncurves << log2h;
    const int it = *a.d_iter;
    const V* __restrict__ rt = (const V*)a.tw;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const int ci = (int)(t >> log2h);
        const uint64_t k = t & (half - 1);
        const int c = a.cls_curves[ci];
        if ((uint32_t)it >= a.eff_iters[c]) continue;
        const CurveDev& cv = a.curves[c];
        const V* __restrict__ Z = (const V*)a.Z + (cv.off >> 1);
        V* __restrict__ Zo = (V*)a.Zp + (cv.off >> 1);
        const T* __restrict__ A = (const T*)a.A + cv.offh;
        if (k == 0) {
            const V z0 = Z[0];
            const T XM = z0.x - z0.y;
            const T Y0 = A[0];
            const T YM = XM < (T)0 ? -A[M] : A[M];
            V o; o.x = Y0 + YM; o.y = Y0 - YM;
            Zo[0] = o;
            // self-paired bin k = M/2: X = conj(Z), packed value 2 conj(Y)
            const V Yh = keep_phase(cconj(Z[half]), A[half]);
            V oh; oh.x = (T)2 * Yh.x; oh.y = -(T)2 * Yh.y;
            Zo[half] = oh;
        } else {
            const V za = Z[k], zb = Z[M - k];
            const V W = rt[k];
            V E; E.x = (T)0.5 * (za.x + zb.x); E.y = (T)0.5 * (za.y - zb.y);
            V O; O.x = (T)0.5 * (za.y + zb.y); O.y = (T)-0.5 * (za.x - zb.x);
            const V WO = cmul(W, O);
            const V Xk = cadd(E, WO);
            const V Xm = cconj(csub(E, WO));
            const V Yk = keep_phase(Xk, A[k]);
            const V Ym = keep_phase(Xm, A[M - k]);
            V Zk, Zm;
            pack_pair(Yk, Ym, W, Zk, Zm);
            Zo[k] = Zk;
            Zo[M - k] = Zm;
        }
    }
}

// TK95 output: Y_j = X_j / sigma (FP64, rounded to T) packed for the inverse
// transform, so that the transform yields the normalised TK95 series.
template <typename T>
__global__ void __launch_bounds__(256) k_spectral_tk(const SpecArgs a)
{
    using V = cplx<T>;
    const uint32_t log2h = a.log2M - 1;
    const uint64_t half = 1ull << log2h;
    const uint64_t M = 1ull << a.log2M;
    const uint64_t total = (uint64_t)a.ncurves << log2h;
    const V* __restrict__ rt = (const V*)a.tw;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const int ci = (int)(t >> log2h);
        const uint64_t k = t & (half - 1);
        const int c = a.cls_curves[ci];
        const CurveDev& cv = a.curves[c];
        const double2* __restrict__ X = a.spec + cv.offh;
        const double inv = 1.0 / a.sigma[c];
        V* __restrict__ Zo = (V*)a.Zp + (cv.off >> 1);
        if (k == 0) {
            const T Y0 = (T)(X[0].x * inv), YM = (T)(X[M].x * inv);
            V o; o.x = Y0 + YM; o.y = Y0 - YM;
            Zo[0] = o;
            V oh; oh.x = (T)2 * (T)(X[half].x * inv); oh.y = -(T)2 * (T)(X[half].y * inv);
            Zo[half] = oh;
        } else {
            V Yk; Yk.x = (T)(X[k].x * inv); Yk.y = (T)(X[k].y * inv);
            V Ym; Ym.x = (T)(X[M - k].x * inv); Ym.y = (T)(X[M - k].y * inv);
            V Zk, Zm;
            pack_pair(Yk, Ym, rt[k], Zk, Zm);
            Zo[k] = Zk;
            Zo[M - k] = Zm;
        }
    }
}

// One conjugate pair (t, M - t) of the spectral step on values held by the
// caller: za = Z_t, zb = Z_{M-t} in, Z'_t, Z'_{M-t} out.  The arithmetic runs
// on the representative k = min(t, M - t), as in k_spectral_iter.
// W = e^{-2 pi i k/N} (rt[k]), Ak = A[k], Am = A[M - k] for k = min(t, M - t),
// loaded by the caller.
template <typename T>
__device__ __forceinline__ void spectral_pair_vals(cplx<T>& za, cplx<T>& zb, uint32_t t, uint32_t M,
                                                   const cplx<T> W, const T Ak, const T Am)
{
    using V = cplx<T>;
    const bool low = 2 * t < M;
    const V zk = low ? za : zb, zm = low ? zb : za;
    V E; E.x = (T)0.5 * (zk.x + zm.x); E.y = (T)0.5 * (zk.y - zm.y);
    V O; O.x = (T)0.5 * (zk.y + zm.y); O.y = (T)-0.5 * (zk.x - zm.x);
    const V WO = cmul(W, O);
    const V Yk = keep_phase(cadd(E, WO), Ak);
    const V Ym = keep_phase(cconj(csub(E, WO)), Am);
    V Zk, Zm;
    pack_pair(Yk, Ym, W, Zk, Zm);
    za = low ? Zk : Zm;
    zb = low ? Zm : Zk;
}

template <typename T>
__device__ __forceinline__ void spectral_pair_tk(cplx<T>& za, cplx<T>& zb, uint32_t t, uint32_t M,
                                                 const cplx<T>* __restrict__ rt, const T* __restrict__ A)
{
    const uint32_t k = 2 * t < M ? t : M - t;
    spectral_pair_vals<T>(za, zb, t, M, rt[k], A[k], A[M - k]);
}

// The middle of one iteration on the tile path, in one kernel: the forward
// transform's last pass (radix R = 2^LR, span p = M/R), the spectral step, and
// the inverse transform's first pass (radix R, span 1; the inverse runs its
// passes in the reverse radix order).  Both passes touch column i through the
// elements i + q p (q < R), and the conjugate partner M - t of t = i + q p is
// in column p - i at row R-1-q; in column 0 itself at row R-q; and, for
// i = p/2, in the same column at row R-1-q.  A block takes H = C/2 columns
// and their H partner columns -- column pairs (0, p/2), then (g, p - g) -- so
// all three steps stay in shared memory, saving two passes over the spectrum
// and the spectral kernel.  Output: y[i R + q] for the block's columns i.
template <typename T, int LR, bool MULTI>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && LR < 9) ? 4 : 2)
    k_fft_spectral(const __grid_constant__ LaunchSet<PassArgs> set, const void* __restrict__ A_all)
{
    uint32_t blk;
    const PassArgs& a = set.pick<MULTI>(blk);
    using V = cplx<T>;
    constexpr int R = 1 << LR;
    constexpr int C = tile_cols(LR, (int)sizeof(V));
    constexpr int LC = ilog2c(C);
    constexpr int S = C + 1;
    constexpr int H = C / 2;
    constexpr int LH = LC - 1;
    extern __shared__ __align__(16) unsigned char tile_smem[];
    V* b0 = (V*)tile_smem;
    V* twm = b0 + R * S;
    const uint32_t log2p = a.log2M - LR;
    const uint32_t p = 1u << log2p;  // indices within a curve: 32-bit (M <= 2^26)
    const int tpc = (int)(p >> LC);
    const int ci = (int)blk / tpc;
    const int ti = (int)blk % tpc;
    const int c = a.cls_curves[ci];
    if (a.d_iter && (uint32_t)(*a.d_iter) >= a.eff_iters[c]) return;
    const CurveDev& cv = a.curves[c];
    const uint64_t base = cv.off >> 1;
    const V* __restrict__ src = (const V*)a.in + base;
    V* __restrict__ dst = (V*)a.out + base;
    const T* __restrict__ A = (const T*)A_all + cv.offh;
    const V* __restrict__ rt = (const V*)a.tw;
    const uint32_t M = 1u << a.log2M;
    // slot j < H: column g = H ti + j; slot j + H: its partner (p/2 for g = 0)
    auto column = [&](int j) -> uint32_t {
        const uint32_t g = (uint32_t)ti * H + (uint32_t)(j & (H - 1));
        if (j < H) return g;
        return g == 0 ? p / 2 : p - g;
    };
    constexpr int PER = R * C / 256;  // elements per thread
    V v[PER];
#pragma unroll
    for (int e = 0; e < PER; ++e) {  // every load in flight before any use
        const int idx = threadIdx.x + e * 256;
        v[e] = src[column(idx & (C - 1)) + (uint32_t)(idx >> LC) * p];
    }
    const SmemTw<T> tw = build_smem_tw<T>(twm, rt, (int)a.log2M, LR);
#pragma unroll
    for (int e = 0; e < PER; ++e) {
        const int idx = threadIdx.x + e * 256;
        const int r = idx >> LC, j = idx & (C - 1);
        // forward last pass: W_{R p}^{r k} = W_M^{r i} (k = i < p)
        b0[r * S + j] = cmul(v[e], tw((uint32_t)r * column(j)));
    }
    __syncthreads();
    tile_dft<T, false, LR, C>(b0, tw, (int)a.log2M);
    V* in = b0;
    // spectral step on the conjugate pairs, in place: in[q][j] = Z_{column(j) + q p}.
    // FP32: the twiddles and amplitudes of all of the thread's pairs are loaded
    // first, so that their latencies overlap (one wait instead of one per pair).
    constexpr bool kPre = sizeof(T) == 4;
    constexpr int NP = kPre ? (R * H + 255) / 256 : 1;
    V Wp[NP];
    T Akp[NP], Amp[NP];
    if (kPre) {
#pragma unroll
        for (int m = 0; m < NP; ++m) {
            const int idx = threadIdx.x + m * 256;
            if ((R * H) % 256 == 0 || idx < R * H) {
                const uint32_t t = column(idx & (H - 1)) + (uint32_t)(idx >> LH) * p;
                const uint32_t k = 2 * t < M ? t : M - t;
                Wp[m] = rt[k];
                Akp[m] = A[k];
                Amp[m] = A[M - k];
            }
        }
    }
#pragma unroll
    for (int m = 0; m < (kPre ? NP : 1); ++m)
    for (int idx = threadIdx.x + m * 256; idx < R * H; idx += (kPre ? R * H : 256)) {
        const int q = idx >> LH, j = idx & (H - 1);
        const uint32_t col = column(j);
        const uint32_t t = col + (uint32_t)q * p;
        if (col == 0) {
            if (q == 0) {  // DC and Nyquist: Y_0 = A_0, Y_M = A_M sign(X_M), packed together
                const V z0 = in[0];
                const T XM = z0.x - z0.y;
                const T Y0 = A[0];
                const T YM = XM < (T)0 ? -A[M] : A[M];
                V o; o.x = Y0 + YM; o.y = Y0 - YM;
                in[0] = o;
            } else if (q == R / 2) {  // k = M/2 pairs with itself: X = conj(Z), packed 2 conj(Y)
                const V Yh = keep_phase(cconj(in[q * S]), A[M >> 1]);
                V oh; oh.x = (T)2 * Yh.x; oh.y = -(T)2 * Yh.y;
                in[q * S] = oh;
            } else if (q < R / 2) {
                if (kPre) spectral_pair_vals<T>(in[q * S], in[(R - q) * S], t, M, Wp[m], Akp[m], Amp[m]);
                else spectral_pair_tk<T>(in[q * S], in[(R - q) * S], t, M, rt, A);
            }
        } else {
            if (kPre) spectral_pair_vals<T>(in[q * S + j], in[(R - 1 - q) * S + j + H], t, M, Wp[m], Akp[m], Amp[m]);
            else spectral_pair_tk<T>(in[q * S + j], in[(R - 1 - q) * S + j + H], t, M, rt, A);
        }
        if (ti == 0 && j == 0 && q < R / 2) {  // column p/2 pairs with itself
            spectral_pair_tk<T>(in[q * S + H], in[(R - 1 - q) * S + H], p / 2 + (uint32_t)q * p, M, rt, A);
        }
    }
    __syncthreads();
    // inverse first pass (span 1: no input twiddle)
    tile_dft<T, true, LR, C>(b0, tw, (int)a.log2M);
    for (int idx = threadIdx.x; idx < R * C; idx += 256) {
        const int j = idx >> LR, q = idx & (R - 1);
        dst[(column(j) << LR) + q] = in[q * S + j];
    }
}

// ------------------------------------------------------------ launchers
static int grid_for(uint64_t work, int block)
{
    uint64_t g = (work + block - 1) / block;
    const uint64_t cap = 152ull * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

std::vector<int> fft_radices(uint32_t log2m)
{
    std::vector<int> r;
    int rem = (int)(log2m % 4);
    if (rem) r.push_back(1 << rem);
    for (uint32_t q = 0; q < log2m / 4; ++q) r.push_back(16);
    return r;
}

template <typename T>
void launch_twiddles(const ClassInfo& k, cudaStream_t st)
{
    const uint64_t M = 1ull << (k.log2n - 1);
    k_twiddles<T><<<grid_for(M, 256), 256, 0, st>>>((cplx<T>*)k.d_tw, k.log2n);
}

template <typename T, bool INV>
static void launch_pass(int R, const PassArgs& a, uint64_t work, cudaStream_t st)
{
    const int g = grid_for(work, 256);
    switch (R) {
    case 2: k_fft_pass<T, 2, INV><<<g, 256, 0, st>>>(a); break;
    case 4: k_fft_pass<T, 4, INV><<<g, 256, 0, st>>>(a); break;
    case 8: k_fft_pass<T, 8, INV><<<g, 256, 0, st>>>(a); break;
    default: k_fft_pass<T, 16, INV><<<g, 256, 0, st>>>(a); break;
    }
}

// Tile passes for a length-2^log2M transform (log2M >= 12): as few passes as
// possible with at most 9 (float) or 8 (double) bits each -- a tile of
// 2^bits x 17 elements in shared memory with room for two or more resident
// blocks per SM -- bits spread evenly, so every pass has between 5 and 9 bits.
std::vector<int> tile_radices(uint32_t log2m, bool fp64)
{
    const int maxb = fp64 ? 8 : 9;
    const int P = ((int)log2m + maxb - 1) / maxb;
    std::vector<int> r;
    for (int q = 0; q < P; ++q) r.push_back((int)log2m / P + (q < (int)log2m % P ? 1 : 0));
    return r;
}

// Blocks of one tile pass (or of the fused spectral kernel) over a class:
// curves x (M/R columns) / C columns per block.
template <typename T>
static int tile_blocks(int ncurves, uint32_t log2M, int LR)
{
    return ncurves << (log2M - LR - ilog2c(tile_cols(LR, (int)sizeof(cplx<T>))));
}

// The tile kernels need nb = M/R >= C columns per curve, and a span p that
// is 1 or at least C (their two output layouts); the fused spectral kernel
// needs M/R >= C for the last forward radix.  Checked for the forward and
// the (reversed) inverse radix order of a length-2^log2M tile-path transform.
bool tile_schedule_ok(uint32_t log2M, bool fp64)
{
    const std::vector<int> lr = tile_radices(log2M, fp64);
    const int eb = fp64 ? 16 : 8;
    for (int dir = 0; dir < 2; ++dir) {
        uint32_t log2p = 0;
        for (size_t q = 0; q < lr.size(); ++q) {
            const int L = dir == 0 ? lr[q] : lr[lr.size() - 1 - q];
            const uint32_t C = (uint32_t)tile_cols(L, eb);
            if ((1u << (log2M - L)) < C) return false;
            if (log2p > 0 && (1u << log2p) < C) return false;
            log2p += (uint32_t)L;
        }
    }
    const int Ls = lr.back();
    return (1u << (log2M - Ls)) >= (uint32_t)tile_cols(Ls, eb);
}

// Dynamic shared memory of one tile-kernel launch (k_fft_tile, k_fft_spectral)
// of radix 2^LR on a length-2^log2M transform: the tile (R rows of C + 1
// elements) and the twiddle tables.  Grows with log2M.
template <typename T>
static size_t tile_smem_bytes(int LR, int log2M)
{
    return (((size_t)1 << LR) * (tile_cols(LR, (int)sizeof(cplx<T>)) + 1) + smem_tw_entries(log2M, LR)) *
           sizeof(cplx<T>);
}

// The longest transform of the tile path: M = 2^26 (N = 2^27).
constexpr int kTileMaxLog2M = 26;

template <typename T, int LR, bool MULTI>
static cudaError_t tile_attrs_m(int smem)
{
    cudaError_t e = cudaFuncSetAttribute(k_fft_tile<T, LR, false, MULTI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_tile<T, LR, true, MULTI>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_fft_spectral<T, LR, MULTI>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return e;
}

template <typename T, int LR>
static cudaError_t tile_attrs()
{
    const int smem = (int)tile_smem_bytes<T>(LR, kTileMaxLog2M);
    cudaError_t e = tile_attrs_m<T, LR, false>(smem);
    if (e == cudaSuccess) e = tile_attrs_m<T, LR, true>(smem);
    return e;
}

// Raises the dynamic shared-memory limit of every tile-kernel instantiation
// to what its longest transform needs, once per device (see
// prepare_kernels).  One limit per function for all lengths: a graph that
// holds launches of one instantiation for several lengths, or a kernel node
// replayed on its own, never asks for more than the function allows.
cudaError_t fft_kernel_attributes()
{
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = tile_attrs<float, 5>();
    if (e == cudaSuccess) e = tile_attrs<float, 6>();
    if (e == cudaSuccess) e = tile_attrs<float, 7>();
    if (e == cudaSuccess) e = tile_attrs<float, 8>();
    if (e == cudaSuccess) e = tile_attrs<float, 9>();
    if (e == cudaSuccess) e = tile_attrs<double, 5>();
    if (e == cudaSuccess) e = tile_attrs<double, 6>();
    if (e == cudaSuccess) e = tile_attrs<double, 7>();
    if (e == cudaSuccess) e = tile_attrs<double, 8>();
    return e;
}

// One tile pass of radix 2^LR over the launch set's classes; dynamic shared
// memory for the longest of them.
template <typename T, int LR, bool INV>
static void launch_tile_lr(const LaunchSet<PassArgs>& s, uint32_t blocks, size_t smem, bool multi, cudaStream_t st)
{
    if (multi) k_fft_tile<T, LR, INV, true><<<blocks, 256, smem, st>>>(s);
    else k_fft_tile<T, LR, INV, false><<<blocks, 256, smem, st>>>(s);
}

template <typename T, bool INV>
static void launch_tile_set(int LR, const LaunchSet<PassArgs>& s, uint32_t blocks, bool multi, cudaStream_t st)
{
    size_t smem = 0;
    for (int i = 0; i < s.n; ++i) smem = std::max(smem, tile_smem_bytes<T>(LR, (int)s.c[i].log2M));
    switch (LR) {
    case 5: launch_tile_lr<T, 5, INV>(s, blocks, smem, multi, st); break;
    case 6: launch_tile_lr<T, 6, INV>(s, blocks, smem, multi, st); break;
    case 7: launch_tile_lr<T, 7, INV>(s, blocks, smem, multi, st); break;
    case 8: launch_tile_lr<T, 8, INV>(s, blocks, smem, multi, st); break;
    default:
        if (sizeof(T) == 4 && LR == 9) launch_tile_lr<float, 9, INV>(s, blocks, smem, multi, st);
        else set_error("internal: unsupported tile radix");
        break;
    }
}

template <typename T, bool INV>
static void launch_tile(int LR, const PassArgs& a, int blocks, cudaStream_t st)
{
    LaunchSet<PassArgs> s{};
    s.c[0] = a;
    s.n = 1;
    launch_tile_set<T, INV>(LR, s, (uint32_t)blocks, false, st);
}

// The fused spectral kernel of radix 2^LR over the launch set's classes.
template <typename T>
static void launch_spectral_set(int LR, const LaunchSet<PassArgs>& s, uint32_t blocks, bool multi, const void* A,
                                cudaStream_t st)
{
    size_t smem = 0;
    for (int i = 0; i < s.n; ++i) smem = std::max(smem, tile_smem_bytes<T>(LR, (int)s.c[i].log2M));
    switch (LR) {
#define LC_FUSED_CASE(L)                                                               \
    case L:                                                                            \
        if (multi) k_fft_spectral<T, L, true><<<blocks, 256, smem, st>>>(s, A);         \
        else k_fft_spectral<T, L, false><<<blocks, 256, smem, st>>>(s, A);              \
        break;
        LC_FUSED_CASE(5)
        LC_FUSED_CASE(6)
        LC_FUSED_CASE(7)
        LC_FUSED_CASE(8)
#undef LC_FUSED_CASE
    default:
        if (sizeof(T) == 4 && LR == 9) {
            if (multi) k_fft_spectral<float, 9, true><<<blocks, 256, smem, st>>>(s, A);
            else k_fft_spectral<float, 9, false><<<blocks, 256, smem, st>>>(s, A);
        } else {
            set_error("internal: unsupported fused radix");
        }
        break;
    }
}

template <typename T>
void* launch_fft(const Plan& p, const ClassInfo& k, bool inverse, void* in, void* other, void* final_out,
                 bool gated, cudaStream_t st, uint64_t* launches, void* scratch)
{
    if (k.log2n - 1 >= 12) {
        PassArgs a{};
        a.cls_curves = k.d_curves;
        a.curves = p.d_curves;
        a.eff_iters = p.d_eff_iters;
        a.d_iter = gated ? p.d_iter : nullptr;
        a.tw = k.d_tw;
        a.ncurves = k.ncurves;
        a.log2M = k.log2n - 1;
        const std::vector<int> lr = tile_radices(a.log2M, sizeof(T) == 8);
        uint32_t log2p = 0;
        void* cur = in;
        void* nxt = other;
        for (size_t q = 0; q < lr.size(); ++q) {
            a.in = cur;
            a.out = (q + 1 == lr.size() && final_out) ? final_out : nxt;
            a.log2p = log2p;
            const int blocks = tile_blocks<T>(k.ncurves, a.log2M, lr[q]);
            if (inverse) launch_tile<T, true>(lr[q], a, blocks, st);
            else launch_tile<T, false>(lr[q], a, blocks, st);
            if (launches) ++*launches;
            log2p += (uint32_t)lr[q];
            void* written = a.out;
            nxt = (q == 0 && scratch) ? scratch : cur;
            cur = written;
        }
        return cur;
    }
    PassArgs a{};
    a.cls_curves = k.d_curves;
    a.curves = p.d_curves;
    a.eff_iters = p.d_eff_iters;
    a.d_iter = gated ? p.d_iter : nullptr;
    a.tw = k.d_tw;
    a.ncurves = k.ncurves;
    a.log2M = k.log2n - 1;
    uint32_t log2p = 0;
    void* cur = in;
    void* nxt = other;
    const size_t P = k.radices.size();
    for (size_t q = 0; q < P; ++q) {
        const int R = k.radices[q];
        a.in = cur;
        a.out = (q + 1 == P && final_out) ? final_out : nxt;
        a.log2p = log2p;
        const uint64_t work = (uint64_t)k.ncurves << (a.log2M - ilog2c(R));
        if (inverse) launch_pass<T, true>(R, a, work, st);
        else launch_pass<T, false>(R, a, work, st);
        if (launches) ++*launches;
        log2p += (uint32_t)ilog2c(R);
        void* written = a.out;
        nxt = (q == 0 && scratch) ? scratch : cur;
        cur = written;
    }
    return cur;
}

template <typename T>
void launch_spectral_iter(const Plan& p, const ClassInfo& k, const void* Z, void* Zp, cudaStream_t st)
{
    SpecArgs a{};
    a.cls_curves = k.d_curves; a.curves = p.d_curves; a.eff_iters = p.d_eff_iters; a.d_iter = p.d_iter;
    a.tw = k.d_tw; a.Z = Z; a.Zp = Zp; a.A = p.d_A; a.ncurves = k.ncurves; a.log2M = k.log2n - 1;
    const uint64_t work = (uint64_t)k.ncurves << (k.log2n - 2);
    k_spectral_iter<T><<<grid_for(work, 256), 256, 0, st>>>(a);
}

template <typename T>
void launch_spectral_tk(const Plan& p, const ClassInfo& k, void* Zp, cudaStream_t st)
{
    SpecArgs a{};
    a.cls_curves = k.d_curves; a.curves = p.d_curves; a.tw = k.d_tw; a.Zp = Zp; a.spec = p.d_spec;
    a.sigma = p.d_sigma; a.ncurves = k.ncurves; a.log2M = k.log2n - 1;
    const uint64_t work = (uint64_t)k.ncurves << (k.log2n - 2);
    k_spectral_tk<T><<<grid_for(work, 256), 256, 0, st>>>(a);
}

// Forward transform, spectral step and inverse transform of one iteration
// on the tile path (log2 M >= 12) for several classes at once: the forward
// passes but the last, the fused k_fft_spectral, then the inverse passes in
// reverse radix order.  Stage by stage, each kernel form (tile pass or fused
// kernel, radix) is launched once for every class that takes it at that
// stage; forward pass f of every class runs in stage f, and the inverse
// passes are aligned on the last one (which also writes the sample-sorted
// classes' sample of x_adj).  Buffers: `in` is read by the first pass only;
// the passes alternate between b and c (c may be `in` itself).  outs[i]
// receives the buffer with class i's x_adj.
template <typename T>
void launch_fft_iteration(const Plan& p, const std::vector<const ClassInfo*>& ks, void* in, void* b, void* c,
                          cudaStream_t st, uint64_t* launches, std::vector<void*>& outs)
{
    struct ClassState {
        const ClassInfo* k;
        PassArgs a;
        std::vector<int> lr;
        int P;
        void* cur;
        void* nxt;
        uint32_t log2p;
    };
    const size_t nk = ks.size();
    std::vector<ClassState> cs(nk);
    int maxf = 0;
    for (size_t i = 0; i < nk; ++i) {
        ClassState& x = cs[i];
        x.k = ks[i];
        x.a = PassArgs{};
        x.a.cls_curves = x.k->d_curves;
        x.a.curves = p.d_curves;
        x.a.eff_iters = p.d_eff_iters;
        x.a.d_iter = p.d_iter;
        x.a.tw = x.k->d_tw;
        x.a.ncurves = x.k->ncurves;
        x.a.log2M = x.k->log2n - 1;
        x.lr = tile_radices(x.a.log2M, sizeof(T) == 8);
        x.P = (int)x.lr.size();
        x.cur = in;
        x.nxt = b;
        x.log2p = 0;
        maxf = std::max(maxf, x.P - 1);
    }
    auto step = [&](ClassState& x) {
        void* w = x.nxt;
        x.nxt = (w == b) ? c : b;
        x.cur = w;
    };
    // (class, radix) pairs of one stage, launched grouped by radix
    std::vector<std::pair<int, int>> sel;
    auto stage = [&](int kind) {  // 0: forward tile pass, 1: fused spectral kernel, 2: inverse tile pass
        for (int LR = 5; LR <= 9; ++LR) {
            std::vector<PassArgs> args;
            std::vector<uint32_t> blocks;
            for (const auto& e : sel) {
                if (e.second != LR) continue;
                const ClassState& x = cs[e.first];
                args.push_back(x.a);
                blocks.push_back((uint32_t)tile_blocks<T>(x.k->ncurves, x.a.log2M, LR));
            }
            if (args.empty()) continue;
            const int n = for_launch_sets(args, blocks, [&](const LaunchSet<PassArgs>& s, uint32_t g, bool multi) {
                if (kind == 0) launch_tile_set<T, false>(LR, s, g, multi, st);
                else if (kind == 1) launch_spectral_set<T>(LR, s, g, multi, p.d_A, st);
                else launch_tile_set<T, true>(LR, s, g, multi, st);
            });
            if (launches) *launches += (uint64_t)n;
        }
    };
    for (int f = 0; f < maxf; ++f) {
        sel.clear();
        for (size_t i = 0; i < nk; ++i) {
            ClassState& x = cs[i];
            if (f >= x.P - 1) continue;
            x.a.in = x.cur; x.a.out = x.nxt; x.a.log2p = x.log2p;
            sel.emplace_back((int)i, x.lr[f]);
        }
        stage(0);
        for (const auto& e : sel) {
            ClassState& x = cs[e.first];
            x.log2p += (uint32_t)x.lr[f];
            step(x);
        }
    }
    sel.clear();
    for (size_t i = 0; i < nk; ++i) {
        ClassState& x = cs[i];
        x.a.in = x.cur; x.a.out = x.nxt; x.a.log2p = x.log2p;
        sel.emplace_back((int)i, x.lr[x.P - 1]);
    }
    stage(1);
    for (size_t i = 0; i < nk; ++i) {
        ClassState& x = cs[i];
        step(x);
        x.log2p = (uint32_t)x.lr[x.P - 1];
    }
    for (int r = maxf - 1; r >= 0; --r) {
        sel.clear();
        for (size_t i = 0; i < nk; ++i) {
            ClassState& x = cs[i];
            if (r > x.P - 2) continue;
            x.a.in = x.cur; x.a.out = x.nxt; x.a.log2p = x.log2p;
            if (r == 0 && x.k->bucket && sizeof(T) == 4) {  // the sample sort's sample of x_adj
                x.a.smp = bucket_sample_area(*x.k);
                x.a.smp_words = (uint32_t)bucket_curve_words(x.k->log2n);
                x.a.smp_shift = bucket_sample_shift(x.k->log2n);
            }
            sel.emplace_back((int)i, x.lr[r]);
        }
        stage(2);
        for (const auto& e : sel) {
            ClassState& x = cs[e.first];
            x.log2p += (uint32_t)x.lr[r];
            step(x);
        }
    }
    outs.assign(nk, nullptr);
    for (size_t i = 0; i < nk; ++i) outs[i] = cs[i].cur;
}

template <typename T>
void* launch_fft_iteration(const Plan& p, const ClassInfo& k, void* in, void* b, void* c, cudaStream_t st,
                           uint64_t* launches)
{
    std::vector<void*> outs;
    launch_fft_iteration<T>(p, std::vector<const ClassInfo*>{&k}, in, b, c, st, launches, outs);
    return outs[0];
}

template void launch_twiddles<float>(const ClassInfo&, cudaStream_t);
template void launch_twiddles<double>(const ClassInfo&, cudaStream_t);
template void* launch_fft<float>(const Plan&, const ClassInfo&, bool, void*, void*, void*, bool, cudaStream_t, uint64_t*,
                                 void*);
template void* launch_fft<double>(const Plan&, const ClassInfo&, bool, void*, void*, void*, bool, cudaStream_t, uint64_t*,
                                  void*);
template void* launch_fft_iteration<float>(const Plan&, const ClassInfo&, void*, void*, void*, cudaStream_t,
                                           uint64_t*);
template void* launch_fft_iteration<double>(const Plan&, const ClassInfo&, void*, void*, void*, cudaStream_t,
                                            uint64_t*);
template void launch_fft_iteration<float>(const Plan&, const std::vector<const ClassInfo*>&, void*, void*, void*,
                                          cudaStream_t, uint64_t*, std::vector<void*>&);
template void launch_fft_iteration<double>(const Plan&, const std::vector<const ClassInfo*>&, void*, void*, void*,
                                           cudaStream_t, uint64_t*, std::vector<void*>&);
template void launch_spectral_iter<float>(const Plan&, const ClassInfo&, const void*, void*, cudaStream_t);
template void launch_spectral_iter<double>(const Plan&, const ClassInfo&, const void*, void*, cudaStream_t);
template void launch_spectral_tk<float>(const Plan&, const ClassInfo&, void*, cudaStream_t);
template void launch_spectral_tk<double>(const Plan&, const ClassInfo&, void*, cudaStream_t);

}  // namespace lc
