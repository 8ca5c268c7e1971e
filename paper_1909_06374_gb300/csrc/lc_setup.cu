// lc_setup.cu -- setup stage of the generator (Sec. 2.1, first two steps):
// TK95 spectrum of the Eq. 3 PSD, its FP64 variance, the target amplitudes,
// and the ERDF draws by inverse CDF.
#include "lc_internal.h"

namespace lc {

constexpr int kSpecBlock = 256;
constexpr int kSpecPerThread = 4;
constexpr int kSpecTile = kSpecBlock * kSpecPerThread;  // bins per block

// TK95 (Sec. 2.1; Sec. 3.2.5): f_j = j/(N dt) (App. A), P_j from Eq. 3 with
// A = 1, X_0 = 0, X_j = sqrt(P_j/2)(g_re + i g_im) for 0 < j < N/2 and the
// real Nyquist bin sqrt(P_{N/2}) g_re; g from Box-Muller on the two uniforms
// of Philox block j (stream 0).  Also the block's share of
// sigma^2 = X_{N/2}^2 + 2 sum_{0<j<N/2} |X_j|^2 (Parseval for the
// unnormalised inverse transform), reduced in a fixed order, and the same sum
// with |X_j|^2 replaced by P_j (the variance the PSD implies, for PSD target
// amplitudes).  coeffs = fixed amplitude: X_j = sqrt(P_j) e^{2 pi i U2},
// X_{N/2} = +-sqrt(P_{N/2}) with the sign of cos(2 pi U2).
__global__ void __launch_bounds__(kSpecBlock)
k_tk_spectrum(const CurveDev* __restrict__ curves, const int* __restrict__ cls_curves,
              int blocks_per_curve, double2* __restrict__ spec, double* __restrict__ partial,
              double* __restrict__ partial_p)
{
    const int ci = blockIdx.x / blocks_per_curve;
    const int jb = blockIdx.x % blocks_per_curve;
    const CurveDev cv = curves[cls_curves[ci]];
    const uint64_t nh = 1ull << (cv.log2n - 1);
    // y_j = f_j / f_br = j c; Eq. 3 as 1 / (e^{a_lo ln y} + e^{a_hi ln y}) (one
    // logarithm for both terms); the amplitude sqrt(P/2) sqrt(-2 ln U1) as one
    // square root: these are the FP64 operations this FP64-rate-bound kernel
    // spends its time on
    const double c = 1.0 / ((double)(1ull << cv.log2n) * cv.dt * cv.f_br);
    const bool fixed = cv.coeffs == 1;
    double acc = 0.0, acc_p = 0.0;
#pragma unroll
    for (int q = 0; q < kSpecPerThread; ++q) {
        const uint64_t j = (uint64_t)jb * kSpecTile + (uint64_t)q * kSpecBlock + threadIdx.x;
        if (j > nh) continue;
        double2 X = make_double2(0.0, 0.0);
        if (j > 0) {
            const uint4 w = philox(j, cv.curve_id, 0u, cv.seed);
            const double U1 = unit_open(w.x, w.y), U2 = unit_open(w.z, w.w);
            const double lu = fixed ? 0.0 : log(U1);  // rad^2 = -2 lu
            double sn, cs;
            sincospi(2.0 * U2, &sn, &cs);
            const double ly = log((double)j * c);
            const double P = 1.0 / (exp(cv.a_lo * ly) + exp(cv.a_hi * ly));
            if (j < nh) {
                const double a = fixed ? sqrt(P) : sqrt(-P * lu);
                X = make_double2(a * cs, a * sn);
                acc += 2.0 * (X.x * X.x + X.y * X.y);
                acc_p += 2.0 * P;
            } else {
                X = make_double2(fixed ? (cs < 0.0 ? -sqrt(P) : sqrt(P)) : sqrt(-2.0 * P * lu) * cs, 0.0);
                acc += X.x * X.x;
                acc_p += P;
            }
        }
        spec[cv.offh + j] = X;
    }
    __shared__ double red[kSpecBlock], red_p[kSpecBlock];
    red[threadIdx.x] = acc;
    red_p[threadIdx.x] = acc_p;
    __syncthreads();
    for (int s = kSpecBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red[threadIdx.x] += red[threadIdx.x + s];
            red_p[threadIdx.x] += red_p[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = red[0];
        partial_p[blockIdx.x] = red_p[0];
    }
}

// sigma (realised) and sigma_P (PSD) of each curve of a class: the partial
// sums added in block order.
__global__ void k_sigma(const int* __restrict__ cls_curves, int ncurves, int blocks_per_curve,
                        const double* __restrict__ partial, const double* __restrict__ partial_p,
                        double* __restrict__ sigma, double* __restrict__ sigma_p)
{
    const int ci = blockIdx.x * blockDim.x + threadIdx.x;
    if (ci >= ncurves) return;
    double s = 0.0, sp = 0.0;
    for (int b = 0; b < blocks_per_curve; ++b) {
        s += partial[(size_t)ci * blocks_per_curve + b];
        sp += partial_p[(size_t)ci * blocks_per_curve + b];
    }
    sigma[cls_curves[ci]] = sqrt(s);
    sigma_p[cls_curves[ci]] = sqrt(sp);
}

// Target amplitudes of the normalised TK95 series: A_j = |X_j| / sigma, A_0 = 0;
// with PSD targets A_j = sqrt(P_j) / sigma_P.
// One block covers kAmpTile bins of one curve (blockIdx.x = curve of the
// class x chunks per curve + chunk), so no thread divides by N/2 + 1.
constexpr int kAmpTile = 1024;
template <typename T>
__global__ void __launch_bounds__(256) k_amplitudes(const CurveDev* __restrict__ curves,
                                                    const int* __restrict__ cls_curves, int chunks, uint32_t log2n,
                                                    const double2* __restrict__ spec,
                                                    const double* __restrict__ sigma,
                                                    const double* __restrict__ sigma_p, T* __restrict__ A)
{
    const uint64_t nh1 = (1ull << (log2n - 1)) + 1;
    const int c = cls_curves[blockIdx.x / chunks];
    const CurveDev& cv = curves[c];
    const uint64_t j0 = (uint64_t)(blockIdx.x % chunks) * kAmpTile;
    const bool psd = cv.targets == 1;
    const double inv = 1.0 / (psd ? sigma_p[c] : sigma[c]);
    const double cy = 1.0 / ((double)(1ull << log2n) * cv.dt * cv.f_br);
    for (uint64_t j = j0 + threadIdx.x; j < j0 + kAmpTile && j < nh1; j += blockDim.x) {
        double a = 0.0;
        if (j > 0 && psd) {
            const double ly = log((double)j * cy);
            a = sqrt(1.0 / (exp(cv.a_lo * ly) + exp(cv.a_hi * ly))) * inv;
        } else if (j > 0) {
            const double2 X = spec[cv.offh + j];
            a = sqrt(X.x * X.x + X.y * X.y) * inv;
        }
        A[cv.offh + j] = (T)a;
    }
}

__global__ void k_erdf_constants(const CurveDev* __restrict__ curves, int ncurves, ErdfConst* __restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < ncurves) out[c] = erdf_constants(curves[c]);
}

// ERDF draws (Sec. 2.1 second step; inverse CDF instead of slice sampling):
// draw k uses Philox block k/2 of stream 1, words (w0,w1) for even k and
// (w2,w3) for odd k; lambda is computed in FP64 and rounded to T.
template <typename T>
__global__ void k_erdf_draws(const CurveDev* __restrict__ curves, const int* __restrict__ cls_curves,
                             int ncurves, uint32_t log2n, const ErdfConst* __restrict__ ek,
                             T* __restrict__ x)
{
    const uint64_t half = 1ull << (log2n - 1);
    const uint64_t total = (uint64_t)ncurves * half;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const int ci = (int)(t >> (log2n - 1));
        const uint64_t q = t & (half - 1);
        const int c = cls_curves[ci];
        const CurveDev& cv = curves[c];
        if (cv.kind != 0) continue;  // tabulated shapes: k_erdf_draws_tab
        const ErdfConst k = ek[c];
        const uint4 w = philox(q, cv.curve_id, 1u, cv.seed);
        const double l0 = erdf_draw(k, unit_open(w.x, w.y));
        const double l1 = erdf_draw(k, unit_open(w.z, w.w));
        x[cv.off + 2 * q] = (T)l0;
        x[cv.off + 2 * q + 1] = (T)l1;
    }
}

// CDF tables of the tabulated ERDF shapes, one block per curve: the
// intervals in parallel, then their sum in order by one thread.
__global__ void __launch_bounds__(256) k_erdf_table(const CurveDev* __restrict__ curves,
                                                    const int* __restrict__ tab_curves, double* __restrict__ tab)
{
    __shared__ double I[kErdfTable];
    const CurveDev& cv = curves[tab_curves[blockIdx.x]];
    for (int k = threadIdx.x; k < kErdfTable; k += blockDim.x) I[k] = erdf_table_interval(cv, k);
    __syncthreads();
    if (threadIdx.x == 0) {
        double* F = tab + cv.tab;
        double acc = 0.0;
        F[0] = 0.0;
        for (int k = 0; k < kErdfTable; ++k) {
            acc = __dadd_rn(acc, I[k]);
            F[k + 1] = acc;
        }
    }
}

// Draws of the tabulated shapes: a block stages its curve's table in shared
// memory and inverts `pairs` Philox blocks (same stream and word use as
// k_erdf_draws).
template <typename T>
__global__ void __launch_bounds__(256) k_erdf_draws_tab(const CurveDev* __restrict__ curves,
                                                        const int* __restrict__ tab_cls_curves, int chunks,
                                                        uint64_t pairs, const ErdfConst* __restrict__ ek,
                                                        const double* __restrict__ tab, T* __restrict__ x)
{
    __shared__ double F[kErdfTable + 1];
    const int c = tab_cls_curves[blockIdx.x / chunks];
    const uint64_t q0 = (uint64_t)(blockIdx.x % chunks) * pairs;
    const CurveDev& cv = curves[c];
    for (int i = threadIdx.x; i <= kErdfTable; i += blockDim.x) F[i] = tab[cv.tab + i];
    __syncthreads();
    const ErdfConst k = ek[c];
    const double h = erdf_table_step(cv);
    for (uint64_t q = q0 + threadIdx.x; q < q0 + pairs; q += blockDim.x) {
        const uint4 w = philox(q, cv.curve_id, 1u, cv.seed);
        const double l0 = erdf_draw_tab(F, cv.umin, h, k.lo, k.hi, unit_open(w.x, w.y));
        const double l1 = erdf_draw_tab(F, cv.umin, h, k.lo, k.hi, unit_open(w.z, w.w));
        x[cv.off + 2 * q] = (T)l0;
        x[cv.off + 2 * q + 1] = (T)l1;
    }
}

// ------------------------------------------------------------ launchers
static int grid_for(uint64_t work, int block)
{
    uint64_t g = (work + block - 1) / block;
    const uint64_t cap = 152ull * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

int spec_blocks_per_curve(uint32_t log2n)
{
    const uint64_t nh1 = (1ull << (log2n - 1)) + 1;
    return (int)((nh1 + kSpecTile - 1) / kSpecTile);
}

void launch_tk_spectrum(const Plan& p, const ClassInfo& k, cudaStream_t st)
{
    const int bpc = spec_blocks_per_curve(k.log2n);
    double* part = p.d_partial + k.partial_off;
    double* part_p = p.d_partial + p.partial_total + k.partial_off;
    k_tk_spectrum<<<k.ncurves * bpc, kSpecBlock, 0, st>>>(p.d_curves, k.d_curves, bpc, p.d_spec, part, part_p);
    k_sigma<<<(k.ncurves + 127) / 128, 128, 0, st>>>(k.d_curves, k.ncurves, bpc, part, part_p, p.d_sigma,
                                                     p.d_sigma + p.ncurves);
}

template <typename T>
void launch_amplitudes(const Plan& p, const ClassInfo& k, cudaStream_t st)
{
    const uint64_t nh1 = (1ull << (k.log2n - 1)) + 1;
    const int chunks = (int)((nh1 + kAmpTile - 1) / kAmpTile);
    k_amplitudes<T><<<k.ncurves * chunks, 256, 0, st>>>(p.d_curves, k.d_curves, chunks, k.log2n, p.d_spec,
                                                        p.d_sigma, p.d_sigma + p.ncurves, (T*)p.d_A);
}

void launch_erdf_constants(const Plan& p, cudaStream_t st)
{
    k_erdf_constants<<<(int)((p.ncurves + 127) / 128), 128, 0, st>>>(p.d_curves, (int)p.ncurves, p.d_erdf);
}

void launch_erdf_tables(const Plan& p, cudaStream_t st)
{
    if (p.ntab) k_erdf_table<<<(int)p.ntab, 256, 0, st>>>(p.d_curves, p.d_tab_curves, p.d_tab);
}

template <typename T>
void launch_erdf_draws(const Plan& p, const ClassInfo& k, cudaStream_t st)
{
    if (k.ntab < k.ncurves) {
        const uint64_t work = (uint64_t)k.ncurves << (k.log2n - 1);
        k_erdf_draws<T><<<grid_for(work, 256), 256, 0, st>>>(p.d_curves, k.d_curves, k.ncurves, k.log2n,
                                                             p.d_erdf, (T*)p.d_x);
    }
    if (k.ntab) {
        // up to 8192 Philox blocks (16384 draws) per block of threads
        const uint64_t half = 1ull << (k.log2n - 1);
        const uint64_t pairs = half < 8192 ? half : 8192;
        const int chunks = (int)(half / pairs);
        k_erdf_draws_tab<T><<<k.ntab * chunks, 256, 0, st>>>(p.d_curves, k.d_tab_curves, chunks, pairs, p.d_erdf,
                                                             p.d_tab, (T*)p.d_x);
    }
}

template void launch_amplitudes<float>(const Plan&, const ClassInfo&, cudaStream_t);
template void launch_amplitudes<double>(const Plan&, const ClassInfo&, cudaStream_t);
template void launch_erdf_draws<float>(const Plan&, const ClassInfo&, cudaStream_t);
template void launch_erdf_draws<double>(const Plan&, const ClassInfo&, cudaStream_t);

}  // namespace lc
