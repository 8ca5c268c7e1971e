// lc_post.cu -- estimators of App. A on batches of generated series: the
// periodogram (Eq. A2, and the fractional rms normalisation of Eq. A4) and the
// structure function (Eq. A6), used for the ensemble checks of Sec. 3.2.5.
//
// Both read a series laid out like a plan's state (curve c at sum_{c'<c} N),
// e.g. the output of lc_generate.  The periodogram reuses the plan's
// half-length complex FFT (the series packed as z_m = x_{2m} + i x_{2m+1}) and
// unpacks |X_j|^2; the structure function is a direct sum over the pairs at
// each lag.
#include <algorithm>

#include "lc_internal.h"

namespace lc {

// |X_j|^2 of a real series from its packed half-length transform Z:
// X_0 = Re Z_0 + Im Z_0, X_M = Re Z_0 - Im Z_0, X_{M/2} = conj Z_{M/2}, and for
// 0 < k < M/2: X_k = E + W^k O, X_{M-k} = conj(E - W^k O) with
// E = (Z_k + conj Z_{M-k})/2, O = (Z_k - conj Z_{M-k})/(2i).
// P_j = |X_j|^2 2/N^2 (Eq. A2) or |X_j|^2 2 dt N / X_0^2 (Eq. A4, X_0 = N mu).
template <typename T>
__global__ void __launch_bounds__(256) k_periodogram(const int* __restrict__ cls_curves,
                                                     const CurveDev* __restrict__ curves, int ncurves,
                                                     uint32_t log2M, const void* __restrict__ tw,
                                                     const void* __restrict__ Zin, int rms,
                                                     double* __restrict__ P)
{
    using V = cplx<T>;
    const uint32_t log2h = log2M - 1;
    const uint64_t half = 1ull << log2h;
    const uint64_t M = 1ull << log2M;
    const double nd = (double)(2 * M);
    const uint64_t total = (uint64_t)ncurves << log2h;
    const V* __restrict__ rt = (const V*)tw;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const int ci = (int)(t >> log2h);
        const uint64_t k = t & (half - 1);
        const CurveDev& cv = curves[cls_curves[ci]];
        const V* __restrict__ Z = (const V*)Zin + (cv.off >> 1);
        double* __restrict__ out = P + cv.offh;
        const V z0 = Z[0];
        const double X0 = (double)(z0.x + z0.y);
        const double scale = rms ? 2.0 * cv.dt * nd / (X0 * X0) : 2.0 / (nd * nd);
        if (k == 0) {
            const double XM = (double)(z0.x - z0.y);
            const V zh = Z[half];
            out[0] = X0 * X0 * scale;
            out[M] = XM * XM * scale;
            out[half] = ((double)zh.x * zh.x + (double)zh.y * zh.y) * scale;
        } else {
            const V za = Z[k], zb = Z[M - k];
            const V W = rt[k];
            V E; E.x = (T)0.5 * (za.x + zb.x); E.y = (T)0.5 * (za.y - zb.y);
            V O; O.x = (T)0.5 * (za.y + zb.y); O.y = (T)-0.5 * (za.x - zb.x);
            const V WO = cmul(W, O);
            const V Xk = cadd(E, WO);
            const V Xm = csub(E, WO);  // conj(X_{M-k}); the modulus is the same
            out[k] = ((double)Xk.x * Xk.x + (double)Xk.y * Xk.y) * scale;
            out[M - k] = ((double)Xm.x * Xm.x + (double)Xm.y * Xm.y) * scale;
        }
    }
}

// SF(tau)^2 of Eq. A6 for one (curve, lag) per block: the mean over the
// N - tau pairs of (x_i - x_{i+tau})^2.  Each thread adds runs of 64 strided
// squares in T, then in FP64; the block sums in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256) k_structure_function(const CurveDev* __restrict__ curves, int nlags,
                                                            const uint32_t* __restrict__ lags,
                                                            const T* __restrict__ x, double* __restrict__ out)
{
    const int c = blockIdx.x / nlags;
    const int l = blockIdx.x % nlags;
    const CurveDev& cv = curves[c];
    const uint64_t tau = lags[l];
    const uint64_t npairs = (1ull << cv.log2n) - tau;
    const T* __restrict__ xc = x + cv.off;
    double acc = 0.0;
    T run = 0;
    int cnt = 0;
    for (uint64_t i = threadIdx.x; i < npairs; i += blockDim.x) {
        const T d = xc[i] - xc[i + tau];
        run += d * d;
        if (++cnt == 64) {
            acc += (double)run;
            run = 0;
            cnt = 0;
        }
    }
    acc += (double)run;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double wpart[8];
    if ((threadIdx.x & 31) == 0) wpart[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wpart[w];
        out[(size_t)c * nlags + l] = s / (double)npairs;
    }
}

template <typename T>
static void run_periodogram(Plan& p, const void* x, int rms, double* out, cudaStream_t st)
{
    for (auto& k : p.classes) {
        // x is only read: the passes ping-pong between d_f and d_keysB
        void* Z = launch_fft<T>(p, k, false, const_cast<void*>(x), p.d_f, nullptr, false, st, nullptr, p.d_keysB);
        const uint64_t work = (uint64_t)k.ncurves << (k.log2n - 2);
        const int blocks = (int)std::min<uint64_t>((work + 255) / 256, 152ull * 16);
        k_periodogram<T><<<blocks, 256, 0, st>>>(k.d_curves, p.d_curves, k.ncurves, k.log2n - 1, k.d_tw, Z, rms,
                                                 out);
    }
}

}  // namespace lc

using namespace lc;

extern "C" {

lc_status lc_periodogram(lc_plan plan, const void* x, int rms, double* out_p, void* stream)
{
    if (!plan || !x || !out_p) { set_error("null plan, x or out_p"); return LC_ERR_INVALID; }
    DeviceGuard g(plan->device);
    StreamJoin j(*plan, stream);
    if (plan->prec == LC_FP32) run_periodogram<float>(*plan, x, rms, out_p, plan->stream);
    else run_periodogram<double>(*plan, x, rms, out_p, plan->stream);
    LC_CK(cudaGetLastError());
    return LC_OK;
}

lc_status lc_structure_function(lc_plan plan, const void* x, const uint32_t* lags, size_t nlags, double* out_sf2,
                                void* stream)
{
    if (!plan || !x || !lags || !out_sf2) { set_error("null plan, x, lags or out_sf2"); return LC_ERR_INVALID; }
    if (nlags < 1 || nlags > kMaxLags) { set_error("nlags must be in [1, 4096]"); return LC_ERR_INVALID; }
    uint32_t nmin = 0xffffffffu;
    for (auto& k : plan->classes) nmin = std::min(nmin, 1u << k.log2n);
    for (size_t l = 0; l < nlags; ++l) {
        if (lags[l] < 1 || lags[l] >= nmin) {
            set_error("lag " + std::to_string(l) + " outside [1, N) of the shortest curve");
            return LC_ERR_INVALID;
        }
    }
    const uint64_t blocks = (uint64_t)plan->ncurves * nlags;
    if (blocks > 0x7fffffffull) { set_error("ncurves * nlags too large"); return LC_ERR_INVALID; }
    DeviceGuard g(plan->device);
    StreamJoin j(*plan, stream);
    // pageable source: the copy is staged before the call returns
    LC_CK(cudaMemcpyAsync(plan->d_lags, lags, nlags * sizeof(uint32_t), cudaMemcpyHostToDevice, plan->stream));
    if (plan->prec == LC_FP32)
        k_structure_function<float><<<(unsigned)blocks, 256, 0, plan->stream>>>(plan->d_curves, (int)nlags,
                                                                             plan->d_lags, (const float*)x, out_sf2);
    else
        k_structure_function<double><<<(unsigned)blocks, 256, 0, plan->stream>>>(
            plan->d_curves, (int)nlags, plan->d_lags, (const double*)x, out_sf2);
    LC_CK(cudaGetLastError());
    return LC_OK;
}

}  // extern "C"
