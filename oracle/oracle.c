/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the AGN light-curve generator of
 * Sartori et al. (arXiv:1909.06374), Sec. 2.1: a Timmer & Koenig (TK95)
 * Gaussian realisation of the target PSD, a random draw of N values from the
 * Eddington-ratio distribution function (ERDF), and the iterative amplitude
 * adjusted Fourier transform of Schreiber & Schmitz / Emmanoulopoulos
 * (S96/E13; Sec. 3.2.2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this code.  It shares nothing with the
 * CUDA path (no headers, tables, constants or helpers); the two sides meet only
 * through the job parameters passed in by the caller.
 *
 * Every floating-point step is IEEE double with contraction disabled
 * (-ffp-contract=off), so the few operations that must be bit-identical with
 * the GPU (the ERDF draws) are fixed sequences of correctly rounded operations
 * and explicit fma() calls.
 *
 * Readings of points where the paper is silent (each is also listed in the
 * design notes of the repository):
 *   - TK95 coefficients are complex Gaussians (Re, Im independent), so the
 *     periodogram scatters around the PSD as Sec. 3.2.5 states.
 *   - The replacement amplitudes are those of the realised, normalised TK95
 *     spectrum (E13 step iii); the DC amplitude is 0.
 *   - Phases are kept as the ratio X/|X|; a zero bin takes phase 0; the Nyquist
 *     bin keeps the sign of its real part (sign(0) = +1).
 *   - Forward DFT uses exp(-2 pi i jk/N), inverse exp(+2 pi i jk/N), 0-based
 *     (App. A, Eq. A1 has the opposite sign and 1-based k; only |DFT|^2 is used
 *     there).
 *   - The ERDF is drawn by inverse CDF of a sharp broken power law in
 *     u = log10(lambda) (the paper uses slice sampling, Sec. 3.1).
 *   - The rank-order replacement is a stable ascending sort (ties: lower index
 *     first).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#if defined(__FAST_MATH__)
#error "the oracle must be built without -ffast-math"
#endif

#define OR_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11 "Parallel random        */
/* numbers: as easy as 1, 2, 3"): ten rounds of two 32x32->64 multiplies,    */
/* xor with the other words and the key; the key is bumped by the Weyl       */
/* constants (golden ratio and sqrt(3)-1 in 32-bit fixed point) per round.   */
/* ------------------------------------------------------------------------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

OR_API void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                             uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Two 32-bit words -> a double strictly inside (0,1): the top 52 bits of the
 * 64-bit word w1:w0 give u, and U = (2u + 1) * 2^-53, exactly representable. */
OR_API double or_u01(uint32_t w0, uint32_t w1)
{
    uint64_t x = ((uint64_t)w1 << 32) | (uint64_t)w0;
    uint64_t u = x >> 12;
    return (double)(2 * u + 1) * 0x1p-53;
}

/* One counter block for stream `tag` of curve `curve_id` at block index `idx`. */
static void philox_block(uint64_t seed, uint64_t curve_id, uint32_t tag,
                         uint64_t idx, uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), (uint32_t)curve_id, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Bit-reproducible exp / log used by the ERDF inverse CDF.                 */
/* exp: Cody & Waite argument reduction x = k ln2 + r, |r| <= ln2/2, and    */
/* the degree-13 Taylor polynomial of e^r in Horner form with fma.          */
/* log: x = 2^e m with m in [sqrt(1/2), sqrt(2)), s = (m-1)/(m+1) and        */
/* ln m = 2 atanh(s) = 2 (s + s^3/3 + ... + s^21/21).                       */
/* ------------------------------------------------------------------------ */
/* ln 2 split into a 32-significant-bit head and the rounded remainder. */
static const double OR_LN2_HI = 0.69314718036912381649017333984375;
static const double OR_LN2_LO = 1.9082149292705877000220e-10;
static const double OR_INV_LN2 = 1.4426950408889634073599246810018921;
static const double OR_SQRT_HALF = 0.70710678118654752440084436210484904;
static const double OR_LN10 = 2.3025850929940456840179914546843642;

OR_API double or_spec_exp(double x)
{
    if (x != x) return x;
    if (x > 709.0) return HUGE_VAL;
    if (x < -708.0) return 0.0;
    double k = rint(x * OR_INV_LN2);
    double r = fma(-k, OR_LN2_HI, x);
    r = fma(-k, OR_LN2_LO, r);
    /* Taylor coefficients 1/i!, i = 13 .. 0; each i! is an exact double. */
    double p = 1.0 / 6227020800.0;
    p = fma(p, r, 1.0 / 479001600.0);
    p = fma(p, r, 1.0 / 39916800.0);
    p = fma(p, r, 1.0 / 3628800.0);
    p = fma(p, r, 1.0 / 362880.0);
    p = fma(p, r, 1.0 / 40320.0);
    p = fma(p, r, 1.0 / 5040.0);
    p = fma(p, r, 1.0 / 720.0);
    p = fma(p, r, 1.0 / 120.0);
    p = fma(p, r, 1.0 / 24.0);
    p = fma(p, r, 1.0 / 6.0);
    p = fma(p, r, 0.5);
    p = fma(p, r, 1.0);
    p = fma(p, r, 1.0);
    return ldexp(p, (int)k);
}

OR_API double or_spec_log(double x)
{
    if (x != x || x < 0.0) return NAN;
    if (x == 0.0) return -HUGE_VAL;
    if (isinf(x)) return x;
    int e;
    double m = frexp(x, &e);               /* m in [0.5, 1) */
    if (m < OR_SQRT_HALF) { m = m * 2.0; e = e - 1; }
    /* s = f/d with f = m-1 (exact) and d = m+1 rounded; dl is the rounding
     * error of d and s_lo the first-order correction of the quotient. */
    double f = m - 1.0;
    double d = m + 1.0;
    double dl = m - (d - 1.0);
    double s = f / d;
    double r = fma(-s, d, f);
    r = fma(-s, dl, r);
    double s_lo = r / d;
    double z = s * s;
    /* q = 1/3 + z/5 + ... + z^9/21 (odd reciprocals 3 .. 21) */
    double q = 1.0 / 21.0;
    q = fma(q, z, 1.0 / 19.0);
    q = fma(q, z, 1.0 / 17.0);
    q = fma(q, z, 1.0 / 15.0);
    q = fma(q, z, 1.0 / 13.0);
    q = fma(q, z, 1.0 / 11.0);
    q = fma(q, z, 1.0 / 9.0);
    q = fma(q, z, 1.0 / 7.0);
    q = fma(q, z, 1.0 / 5.0);
    q = fma(q, z, 1.0 / 3.0);
    double two_s = 2.0 * s;                 /* exact */
    double sz = two_s * z;
    double de = (double)e;
    /* ln x = e ln2_hi + 2s + (e ln2_lo + 2 s_lo + 2 s z q), small terms first */
    double small = fma(de, OR_LN2_LO, 2.0 * s_lo);
    small = fma(sz, q, small);
    double t = two_s + small;
    return fma(de, OR_LN2_HI, t);
}

/* log(1+y): w = 1+y rounded, then log(1+y) = log(w) + log(1 + c/w) with the
 * exactly representable rounding error c = y - (w-1); log(1 + c/w) ~ c/w. */
OR_API double or_spec_log1p(double y)
{
    double w = 1.0 + y;
    if (w == 1.0) return y;
    double d = w - 1.0;
    double c = y - d;
    double t = c / w;
    return or_spec_log(w) + t;
}

/* ------------------------------------------------------------------------ */
/* ERDF: broken power law in u = log10(lambda) (Sec. 2.1.1, Eq. 1, sharp-   */
/* break form): dN/du ~ 10^{a1 (u-ub)} below the break ub, 10^{a2 (u-ub)}   */
/* above, on [umin, umax].  With linear_space the slopes describe dN/dlambda */
/* (Sec. 2.1.1, last paragraph), which shifts both by +1 in log space.       */
/* Inverse CDF, written with c = a ln10:                                    */
/*   M1 = (1 - e^{c1 (umin-ub)})/c1,  M2 = (e^{c2 (umax-ub)} - 1)/c2         */
/*   v = U (M1 + M2);  v < M1: u = ub + ln(e^{c1(umin-ub)} + c1 v)/c1        */
/*                     else  : u = ub + ln(1 + c2 (v - M1))/c2               */
/* (a slope of exactly 0 uses the uniform-density limits), lambda = e^{ln10 u},*/
/* clamped to [10^umin, 10^umax].                                            */
/* erdf[] = {log_lmin, log_lmax, log_lbreak, slope_low, slope_high}.         */
/* ------------------------------------------------------------------------ */
/* Intervals of the tabulated ERDF CDF (kinds 1 and 2 below). */
#define OR_ERDF_TABLE 4096

OR_API double or_erdf_icdf(const double erdf[5], int linear_space, double U)
{
    double umin = erdf[0], umax = erdf[1], ub = erdf[2];
    double a1 = erdf[3], a2 = erdf[4];
    if (linear_space) { a1 = a1 + 1.0; a2 = a2 + 1.0; }
    double c1 = a1 * OR_LN10, c2 = a2 * OR_LN10;
    double e1 = 0.0, M1, M2;
    if (a1 != 0.0) {
        e1 = or_spec_exp(c1 * (umin - ub));
        M1 = (1.0 - e1) / c1;
    } else {
        M1 = ub - umin;
    }
    if (a2 != 0.0) {
        double e2 = or_spec_exp(c2 * (umax - ub));
        M2 = (e2 - 1.0) / c2;
    } else {
        M2 = umax - ub;
    }
    double v = U * (M1 + M2);
    double u;
    if (v < M1) {
        if (a1 != 0.0) {
            double t = or_spec_log(e1 + c1 * v);
            u = ub + t / c1;
        } else {
            u = umin + v;
        }
    } else {
        if (a2 != 0.0) {
            double t = or_spec_log1p(c2 * (v - M1));
            u = ub + t / c2;
        } else {
            u = ub + (v - M1);
        }
    }
    double lam = or_spec_exp(OR_LN10 * u);
    double lo = or_spec_exp(OR_LN10 * umin), hi = or_spec_exp(OR_LN10 * umax);
    if (lam < lo) lam = lo;
    if (lam > hi) lam = hi;
    return lam;
}

/* ------------------------------------------------------------------------ */
/* ERDF shapes without a closed-form inverse CDF (Sec. 2.1.1):              */
/*   kind 1, the smooth broken power law of Eq. 1:                          */
/*     dN/du ~ [10^{-a1 (u-ub)} + 10^{-a2 (u-ub)}]^-1                       */
/*     (Eq. 1's delta_1 = -a1, delta_2 = -a2, log lambda* = ub), which tends  */
/*     to the sharp form's branches 10^{a1 (u-ub)} / 10^{a2 (u-ub)} away from */
/*     the break;                                                           */
/*   kind 2, the log-normal of Eq. 2: dN/du ~ exp(-(u-ub)^2 / (2 sigma^2))  */
/*     (log lambda* = ub, sigma-tilde = sigma, in dex);                     */
/*   kind 0, the sharp form, is also accepted here (used to check the        */
/*     tabulated inversion against the closed form).                        */
/* linear_space multiplies the density by 10^{u-ub} (dN/dlambda form).      */
/* erdf[] = {log_lmin, log_lmax, log_lbreak, slope_low, slope_high, sigma}.  */
/* ------------------------------------------------------------------------ */
OR_API double or_erdf_density(const double erdf[6], int kind, int linear_space, double u)
{
    double ub = erdf[2], d = u - ub;
    double a1 = erdf[3], a2 = erdf[4];
    if (linear_space) { a1 = a1 + 1.0; a2 = a2 + 1.0; }
    if (kind == 0) return d < 0.0 ? or_spec_exp(a1 * OR_LN10 * d) : or_spec_exp(a2 * OR_LN10 * d);
    if (kind == 1) {
        double c1 = a1 * OR_LN10, c2 = a2 * OR_LN10;
        return 1.0 / (or_spec_exp(-c1 * d) + or_spec_exp(-c2 * d));
    }
    double t = d / erdf[5];
    double e = -0.5 * t * t;
    if (linear_space) e = e + OR_LN10 * d;
    return or_spec_exp(e);
}

/* Unnormalised CDF on the uniform grid u_k = umin + k h, h = (umax-umin)/T, */
/* T = OR_ERDF_TABLE: F_0 = 0, F_{k+1} = F_k + Simpson's rule on [u_k,      */
/* u_{k+1}] = F_k + (f(u_k) + 4 f(u_k + h/2) + f(u_{k+1})) h/6, summed in    */
/* order.  F has T+1 entries.                                               */
OR_API void or_erdf_table(const double erdf[6], int kind, int linear_space, double* F)
{
    double umin = erdf[0], h = (erdf[1] - erdf[0]) / (double)OR_ERDF_TABLE;
    double h6 = h / 6.0;
    F[0] = 0.0;
    for (int k = 0; k < OR_ERDF_TABLE; ++k) {
        double u0 = umin + (double)k * h;
        double u1 = umin + (double)(k + 1) * h;
        double um = u0 + 0.5 * h;
        double sum = or_erdf_density(erdf, kind, linear_space, u0)
                     + 4.0 * or_erdf_density(erdf, kind, linear_space, um);
        sum = sum + or_erdf_density(erdf, kind, linear_space, u1);
        F[k + 1] = F[k] + sum * h6;
    }
}

/* Inverse of the tabulated CDF: v = U F_T; the interval k with             */
/* F_k <= v < F_{k+1} by bisection; u linear in v inside it (the density     */
/* taken constant over one interval); lambda = e^{ln10 u} clamped to the     */
/* range as in the closed form.                                             */
OR_API double or_erdf_icdf_tab(const double erdf[6], const double* F, double U)
{
    double umin = erdf[0], umax = erdf[1];
    double h = (umax - umin) / (double)OR_ERDF_TABLE;
    double v = U * F[OR_ERDF_TABLE];
    int lo = 0, hi = OR_ERDF_TABLE;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (F[mid] <= v) lo = mid; else hi = mid;
    }
    double den = F[lo + 1] - F[lo];
    double t = den > 0.0 ? (v - F[lo]) / den : 0.0;
    double u = (umin + (double)lo * h) + t * h;
    double lam = or_spec_exp(OR_LN10 * u);
    double lmin = or_spec_exp(OR_LN10 * umin), lmax = or_spec_exp(OR_LN10 * umax);
    if (lam < lmin) lam = lmin;
    if (lam > lmax) lam = lmax;
    return lam;
}

/* N draws from the ERDF in draw order (Sec. 2.1, second step).  Draw k uses
 * Philox block k/2 of stream 1, words (w0,w1) for even k and (w2,w3) for odd k.
 * kind 0 inverts the sharp form in closed form, kinds 1 and 2 through the
 * table above.  prec = 0 rounds each draw to float (round to nearest),
 * prec = 1 keeps it. */
OR_API void or_erdf_draws(const double erdf[6], int linear_space, int kind, uint64_t seed,
                          uint64_t curve_id, int prec, size_t n, double* out)
{
    uint32_t w[4];
    double* F = NULL;
    if (kind != 0) {
        F = (double*)malloc(sizeof(double) * (OR_ERDF_TABLE + 1));
        or_erdf_table(erdf, kind, linear_space, F);
    }
    for (size_t k = 0; k < n; ++k) {
        if ((k & 1) == 0) philox_block(seed, curve_id, 1u, (uint64_t)(k >> 1), w);
        double U = (k & 1) ? or_u01(w[2], w[3]) : or_u01(w[0], w[1]);
        double lam = kind == 0 ? or_erdf_icdf(erdf, linear_space, U) : or_erdf_icdf_tab(erdf, F, U);
        out[k] = prec == 0 ? (double)(float)lam : lam;
    }
    free(F);
}

/* ------------------------------------------------------------------------ */
/* PSD (Sec. 2.1.2, Eq. 3) with A = 1: [(f/f_br)^a_low + (f/f_br)^a_high]^-1 */
/* ------------------------------------------------------------------------ */
OR_API double or_psd(double f, double f_br, double a_low, double a_high)
{
    double y = f / f_br;
    return 1.0 / (pow(y, a_low) + pow(y, a_high));
}

/* TK95 spectrum (Sec. 2.1; Sec. 3.2.5): Fourier frequencies f_j = j/(N dt)
 * (App. A), X_0 = 0, X_j = sqrt(P_j/2) (g_re + i g_im) for 0 < j < N/2 and the
 * real Nyquist bin X_{N/2} = sqrt(P_{N/2}) g_re.  The Gaussians come from Box-
 * Muller on the two uniforms of Philox block j of stream 0.
 * coeffs = 1 is the fixed-amplitude variant: X_j = sqrt(P_j) e^{2 pi i U2}
 * (same mean power, no scatter of |X_j|) and X_{N/2} = +-sqrt(P_{N/2}) with
 * the sign of cos(2 pi U2).
 * X has 2*(N/2+1) doubles (re, im interleaved). */
OR_API void or_tk_spectrum(uint32_t log2n, double dt, const double psd[3], int coeffs,
                           uint64_t seed, uint64_t curve_id, double* X)
{
    size_t n = (size_t)1 << log2n, nh = n / 2;
    const double two_pi = 6.283185307179586476925286766559;
    X[0] = 0.0; X[1] = 0.0;
    for (size_t j = 1; j <= nh; ++j) {
        uint32_t w[4];
        philox_block(seed, curve_id, 0u, (uint64_t)j, w);
        double U1 = or_u01(w[0], w[1]), U2 = or_u01(w[2], w[3]);
        double rad = coeffs == 1 ? 1.0 : sqrt(-2.0 * log(U1));
        double g_re = rad * cos(two_pi * U2), g_im = rad * sin(two_pi * U2);
        double f = (double)j / ((double)n * dt);
        double P = or_psd(f, psd[0], psd[1], psd[2]);
        if (j < nh) {
            double a = coeffs == 1 ? sqrt(P) : sqrt(P / 2.0);
            X[2 * j] = a * g_re;
            X[2 * j + 1] = a * g_im;
        } else {
            X[2 * j] = coeffs == 1 ? (g_re < 0.0 ? -sqrt(P) : sqrt(P)) : sqrt(P) * g_re;
            X[2 * j + 1] = 0.0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Discrete Fourier transforms (App. A, Eq. A1, 0-based, sign as an argument). */
/* ------------------------------------------------------------------------ */
typedef struct { double re, im; } cplx;

/* Direct O(n^2) definition; the angle uses (j k mod n) so it stays exact. */
OR_API void or_dft(size_t n, const double* in, double* out, int sign)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (size_t j = 0; j < n; ++j) {
        double sr = 0.0, si = 0.0;
        for (size_t k = 0; k < n; ++k) {
            size_t t = (j * k) % n;
            double ang = (double)sign * two_pi * (double)t / (double)n;
            double c = cos(ang), s = sin(ang);
            double xr = in[2 * k], xi = in[2 * k + 1];
            sr += xr * c - xi * s;
            si += xr * s + xi * c;
        }
        out[2 * j] = sr;
        out[2 * j + 1] = si;
    }
}

/* Recursive radix-2 decimation in time: DFT of the even- and odd-indexed
 * halves, combined with twiddles exp(sign 2 pi i k/n) from cos/sin in FP64. */
static void fft_rec(size_t n, const cplx* in, size_t stride, cplx* out, int sign)
{
    if (n == 1) { out[0] = in[0]; return; }
    size_t h = n / 2;
    fft_rec(h, in, 2 * stride, out, sign);
    fft_rec(h, in + stride, 2 * stride, out + h, sign);
    const double two_pi = 6.283185307179586476925286766559;
    for (size_t k = 0; k < h; ++k) {
        double ang = (double)sign * two_pi * (double)k / (double)n;
        double c = cos(ang), s = sin(ang);
        cplx e = out[k], o = out[k + h];
        cplx t = {o.re * c - o.im * s, o.re * s + o.im * c};
        out[k].re = e.re + t.re;     out[k].im = e.im + t.im;
        out[k + h].re = e.re - t.re; out[k + h].im = e.im - t.im;
    }
}

/* Complex transform of length n (a power of two): direct sum for n <= 64,
 * recursive radix-2 otherwise. */
OR_API void or_fft(size_t n, const double* in, double* out, int sign)
{
    if (n <= 64) { or_dft(n, in, out, sign); return; }
    fft_rec(n, (const cplx*)in, 1, (cplx*)out, sign);
}

/* Real-to-complex forward DFT: X_j = sum_k x_k exp(-2 pi i jk/n), j = 0..n/2,
 * computed as the complex transform of (x, 0). X has 2*(n/2+1) doubles. */
OR_API void or_r2c(size_t n, const double* x, double* X)
{
    double* buf = (double*)malloc(sizeof(double) * 4 * n);
    double* spec = buf + 2 * n;
    for (size_t k = 0; k < n; ++k) { buf[2 * k] = x[k]; buf[2 * k + 1] = 0.0; }
    or_fft(n, buf, spec, -1);
    memcpy(X, spec, sizeof(double) * 2 * (n / 2 + 1));
    free(buf);
}

/* Complex-to-real inverse DFT without normalisation:
 * x_k = sum_{j=0}^{n-1} Y_j exp(+2 pi i jk/n), with Y_{n-j} = conj(Y_j)
 * (a real series), so only Y_0 .. Y_{n/2} are given; the imaginary parts of
 * Y_0 and Y_{n/2} are ignored. */
OR_API void or_c2r(size_t n, const double* Y, double* x)
{
    size_t nh = n / 2;
    double* buf = (double*)malloc(sizeof(double) * 4 * n);
    double* res = buf + 2 * n;
    for (size_t j = 0; j <= nh; ++j) { buf[2 * j] = Y[2 * j]; buf[2 * j + 1] = Y[2 * j + 1]; }
    buf[1] = 0.0;
    buf[2 * nh + 1] = 0.0;
    for (size_t j = 1; j < nh; ++j) {
        buf[2 * (n - j)] = Y[2 * j];
        buf[2 * (n - j) + 1] = -Y[2 * j + 1];
    }
    or_fft(n, buf, res, +1);
    for (size_t k = 0; k < n; ++k) x[k] = res[2 * k];
    free(buf);
}

/* ------------------------------------------------------------------------ */
/* TK95 series and target amplitudes (Sec. 2.1 first step; normalised E13   */
/* series): x = C2R(X), mu = mean, sigma^2 = population variance,           */
/* x_TK = (x - mu)/sigma, A_j = |X_j|/sigma with A_0 = 0.                    */
/* targets = 1 takes the amplitudes from the PSD itself instead of the       */
/* realisation: A_j = sqrt(P_j)/sigma_P with sigma_P^2 = P_{N/2} +           */
/* 2 sum_{0<j<N/2} P_j, the series variance that the PSD implies.           */
/* ------------------------------------------------------------------------ */
OR_API void or_tk_series(uint32_t log2n, double dt, const double psd[3], int coeffs, int targets,
                         uint64_t seed, uint64_t curve_id, double* x_tk, double* A, double* sigma_out)
{
    size_t n = (size_t)1 << log2n, nh = n / 2;
    double* X = (double*)malloc(sizeof(double) * 2 * (nh + 1));
    or_tk_spectrum(log2n, dt, psd, coeffs, seed, curve_id, X);
    or_c2r(n, X, x_tk);
    double mu = 0.0;
    for (size_t k = 0; k < n; ++k) mu += x_tk[k];
    mu /= (double)n;
    double var = 0.0;
    for (size_t k = 0; k < n; ++k) { double d = x_tk[k] - mu; var += d * d; }
    var /= (double)n;
    double sigma = sqrt(var);
    for (size_t k = 0; k < n; ++k) x_tk[k] = (x_tk[k] - mu) / sigma;
    A[0] = 0.0;
    if (targets == 1) {
        double sp = 0.0;
        for (size_t j = 1; j <= nh; ++j) {
            double P = or_psd((double)j / ((double)n * dt), psd[0], psd[1], psd[2]);
            sp += j < nh ? 2.0 * P : P;
        }
        double sigma_p = sqrt(sp);
        for (size_t j = 1; j <= nh; ++j)
            A[j] = sqrt(or_psd((double)j / ((double)n * dt), psd[0], psd[1], psd[2])) / sigma_p;
    } else {
        for (size_t j = 1; j <= nh; ++j) A[j] = hypot(X[2 * j], X[2 * j + 1]) / sigma;
    }
    if (sigma_out) *sigma_out = sigma;
    free(X);
}

/* ------------------------------------------------------------------------ */
/* Stable ascending argsort (ties: lower index first).                      */
/* ------------------------------------------------------------------------ */
typedef struct { double v; size_t i; } keyed;

static int keyed_cmp(const void* pa, const void* pb)
{
    const keyed* a = (const keyed*)pa;
    const keyed* b = (const keyed*)pb;
    if (a->v < b->v) return -1;
    if (a->v > b->v) return 1;
    return a->i < b->i ? -1 : (a->i > b->i ? 1 : 0);
}

OR_API void or_argsort(size_t n, const double* v, int64_t* perm)
{
    keyed* kv = (keyed*)malloc(sizeof(keyed) * n);
    for (size_t k = 0; k < n; ++k) { kv[k].v = v[k]; kv[k].i = k; }
    qsort(kv, n, sizeof(keyed), keyed_cmp);
    for (size_t r = 0; r < n; ++r) perm[r] = (int64_t)kv[r].i;
    free(kv);
}

static int dbl_cmp(const void* pa, const void* pb)
{
    double a = *(const double*)pa, b = *(const double*)pb;
    return a < b ? -1 : (a > b ? 1 : 0);
}

OR_API void or_sort(size_t n, double* v) { qsort(v, n, sizeof(double), dbl_cmp); }

/* ------------------------------------------------------------------------ */
/* One E13 iteration (Sec. 2.1 third step; Sec. 3.2.2): X = DFT(x); keep the  */
/* phases and impose the target amplitudes A; x_adj = IDFT(Y); the value of   */
/* rank r in x_adj becomes s[r] (the sorted draws).                         */
/*   Y_0 = A_0, Y_j = A_j X_j/|X_j| (|X_j| = 0 -> A_j), Y_{n/2} = A_{n/2}    */
/*   sign(Re X_{n/2}) with sign(0) = +1.                                    */
/* x is updated in place; x_adj (n doubles) receives the pre-ranking series   */
/* and perm (n) the argsort of it when they are non-NULL.                   */
/* ------------------------------------------------------------------------ */
/* One iteration on n = 2^log2n samples; X (n/2+1 complex), xa (n) and perm
 * (n) are work arrays that hold this iteration's spectrum, pre-ranking series
 * and argsort afterwards. */
static void iterate_once(size_t n, const double* A, const double* s, double* x,
                         double* X, double* xa, int64_t* perm)
{
    size_t nh = n / 2;
    or_r2c(n, x, X);
    X[0] = A[0]; X[1] = 0.0;
    for (size_t j = 1; j < nh; ++j) {
        double re = X[2 * j], im = X[2 * j + 1];
        double mag = hypot(re, im);
        if (mag == 0.0) { X[2 * j] = A[j]; X[2 * j + 1] = 0.0; }
        else { X[2 * j] = A[j] * (re / mag); X[2 * j + 1] = A[j] * (im / mag); }
    }
    X[2 * nh] = X[2 * nh] < 0.0 ? -A[nh] : A[nh];
    X[2 * nh + 1] = 0.0;
    or_c2r(n, X, xa);
    or_argsort(n, xa, perm);
    for (size_t r = 0; r < n; ++r) x[perm[r]] = s[r];
}

OR_API void or_iterate(uint32_t log2n, const double* A, const double* s, double* x,
                       uint32_t iters, double* x_adj_out, int64_t* perm_out)
{
    size_t n = (size_t)1 << log2n, nh = n / 2;
    double* X = (double*)malloc(sizeof(double) * 2 * (nh + 1));
    double* xa = (double*)malloc(sizeof(double) * n);
    int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * n);
    for (uint32_t it = 0; it < iters; ++it) iterate_once(n, A, s, x, X, xa, perm);
    if (x_adj_out && iters > 0) memcpy(x_adj_out, xa, sizeof(double) * n);
    if (perm_out && iters > 0) memcpy(perm_out, perm, sizeof(int64_t) * n);
    free(X); free(xa); free(perm);
}

/* ------------------------------------------------------------------------ */
/* Convergence distance of Sec. 3.2.2, Eq. 4, between consecutive iterates:  */
/*   delta = rms_n [ log10( x_new(t_n) / x_old(t_n) ) ],  n = 1..N           */
/* read as the root mean square about zero with the base-10 logarithm (the  */
/* paper's "log" of Eddington ratios).  Both series must be positive.        */
/* ------------------------------------------------------------------------ */
OR_API double or_delta(size_t n, const double* x_old, const double* x_new)
{
    double acc = 0.0;
    for (size_t k = 0; k < n; ++k) {
        double t = log10(x_new[k] / x_old[k]);
        acc += t * t;
    }
    return sqrt(acc / (double)n);
}

/* Iterations with the convergence test of Sec. 3.2.2: after iteration i     */
/* (1-based) delta[i-1] = delta_i = Eq. 4 between x_{i-1} and x_i; the loop   */
/* ends after the first i with delta_i < thr (strictly; thr <= 0 never ends  */
/* it early) or after `iters`.  Returns the number of iterations run; x holds */
/* the last iterate.                                                         */
OR_API uint32_t or_iterate_conv(uint32_t log2n, const double* A, const double* s, double* x,
                                uint32_t iters, double thr, double* delta)
{
    size_t n = (size_t)1 << log2n, nh = n / 2;
    double* X = (double*)malloc(sizeof(double) * 2 * (nh + 1));
    double* xa = (double*)malloc(sizeof(double) * n);
    double* xp = (double*)malloc(sizeof(double) * n);
    int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * n);
    uint32_t it = 0;
    while (it < iters) {
        memcpy(xp, x, sizeof(double) * n);
        iterate_once(n, A, s, x, X, xa, perm);
        double d = or_delta(n, xp, x);
        delta[it] = d;
        ++it;
        if (d < thr) break;
    }
    free(X); free(xa); free(xp); free(perm);
    return it;
}

/* ------------------------------------------------------------------------ */
/* Whole generator for one curve.  params[] = {dt, f_br, a_low, a_high,      */
/* log_lmin, log_lmax, log_lbreak, slope_low, slope_high, sigma};           */
/* modes[] = {linear_space, ERDF kind (0 sharp, 1 smooth Eq. 1, 2 log-normal */
/* Eq. 2), TK coefficients (0 Gaussian, 1 fixed amplitude), targets (0 the   */
/* realised amplitudes, 1 those of the PSD)}.                               */
/* out_x (n) receives the final series; out_tk (n, nullable) the normalised   */
/* TK95 series; out_A (n/2+1, nullable) the amplitudes; out_s (n, nullable)  */
/* the sorted draws.  prec 0 = draws rounded to float, 1 = double.          */
/* ------------------------------------------------------------------------ */
OR_API void or_generate(uint32_t log2n, const double params[10], const int modes[4],
                        uint32_t iters, uint64_t seed, uint64_t curve_id, int prec,
                        double* out_x, double* out_tk, double* out_A, double* out_s)
{
    size_t n = (size_t)1 << log2n, nh = n / 2;
    double psd[3] = {params[1], params[2], params[3]};
    double erdf[6] = {params[4], params[5], params[6], params[7], params[8], params[9]};
    double* xtk = (double*)malloc(sizeof(double) * n);
    double* A = (double*)malloc(sizeof(double) * (nh + 1));
    double* s = (double*)malloc(sizeof(double) * n);
    or_tk_series(log2n, params[0], psd, modes[2], modes[3], seed, curve_id, xtk, A, NULL);
    or_erdf_draws(erdf, modes[0], modes[1], seed, curve_id, prec, n, out_x);
    memcpy(s, out_x, sizeof(double) * n);
    or_sort(n, s);
    or_iterate(log2n, A, s, out_x, iters, NULL, NULL);
    if (out_tk) memcpy(out_tk, xtk, sizeof(double) * n);
    if (out_A) memcpy(out_A, A, sizeof(double) * (nh + 1));
    if (out_s) memcpy(out_s, s, sizeof(double) * n);
    free(xtk); free(A); free(s);
}

/* ------------------------------------------------------------------------ */
/* Periodogram (App. A, Eq. A2): P_j = (2/N^2) |DFT_j|^2 for j = 0..N/2 (the   */
/* sign of the exponent in Eq. A1 does not change |DFT_j|).  rms = 1 gives the */
/* fractional rms normalisation of Eq. A4: P_j = 2 dt |DFT_j|^2 / (mu^2 N),    */
/* mu the mean of the series.  P has N/2+1 entries.                          */
/* ------------------------------------------------------------------------ */
OR_API void or_periodogram(size_t n, const double* x, double dt, int rms, double* P)
{
    size_t nh = n / 2;
    double* X = (double*)malloc(sizeof(double) * 2 * (nh + 1));
    or_r2c(n, x, X);
    double mu = 0.0;
    for (size_t k = 0; k < n; ++k) mu += x[k];
    mu /= (double)n;
    double nd = (double)n;
    for (size_t j = 0; j <= nh; ++j) {
        double p2 = X[2 * j] * X[2 * j] + X[2 * j + 1] * X[2 * j + 1];
        P[j] = rms ? 2.0 * dt * p2 / (mu * mu * nd) : 2.0 * p2 / (nd * nd);
    }
    free(X);
}

/* Structure function (App. A, Eq. A6) at integer lags tau (in samples):     */
/* SF(tau)^2 = (1/P) sum over the P = N - tau pairs (x_i, x_{i+tau}) of       */
/* (x_i - x_{i+tau})^2.  Lags must satisfy 1 <= tau < N.                     */
OR_API void or_structure_function(size_t n, const double* x, size_t nlags, const uint32_t* lags,
                                  double* sf2)
{
    for (size_t l = 0; l < nlags; ++l) {
        size_t tau = lags[l];
        double acc = 0.0;
        for (size_t i = 0; i + tau < n; ++i) {
            double d = x[i] - x[i + tau];
            acc += d * d;
        }
        sf2[l] = acc / (double)(n - tau);
    }
}

/* ------------------------------------------------------------------------ */
/* A batch of independent curves on `nthreads` host threads (curves are      */
/* independent, so this is only a loop split across threads).               */
/* log2n[c], params[10c..10c+9], modes[4c..4c+3], iters[c], seed[c],       */
/* curve_id[c]; out_x is the concatenation of the curves in order.          */
/* ------------------------------------------------------------------------ */
typedef struct {
    size_t ncurves;
    const uint32_t* log2n; const double* params; const int* modes; const uint32_t* iters;
    const uint64_t* seed; const uint64_t* curve_id; int prec;
    double* out_x; const size_t* offsets;
    size_t next; pthread_mutex_t lock;
} batch_ctx;

static void* batch_worker(void* arg)
{
    batch_ctx* b = (batch_ctx*)arg;
    for (;;) {
        pthread_mutex_lock(&b->lock);
        size_t c = b->next++;
        pthread_mutex_unlock(&b->lock);
        if (c >= b->ncurves) break;
        or_generate(b->log2n[c], b->params + 10 * c, b->modes + 4 * c, b->iters[c], b->seed[c],
                    b->curve_id[c], b->prec, b->out_x + b->offsets[c], NULL, NULL, NULL);
    }
    return NULL;
}

OR_API int or_generate_batch(size_t ncurves, const uint32_t* log2n, const double* params,
                             const int* modes, const uint32_t* iters,
                             const uint64_t* seed, const uint64_t* curve_id, int prec,
                             int nthreads, double* out_x)
{
    size_t* offsets = (size_t*)malloc(sizeof(size_t) * (ncurves + 1));
    offsets[0] = 0;
    for (size_t c = 0; c < ncurves; ++c) offsets[c + 1] = offsets[c] + ((size_t)1 << log2n[c]);
    batch_ctx b = {ncurves, log2n, params, modes, iters, seed, curve_id, prec,
                   out_x, offsets, 0, PTHREAD_MUTEX_INITIALIZER};
    if (nthreads < 1) nthreads = 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    int started = 0;
    for (int t = 0; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, batch_worker, &b) == 0) ++started;
    if (started == 0) batch_worker(&b);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    free(th);
    free(offsets);
    return started > 0 ? started : 1;
}

/* Vector helpers for the self-tests (a loop over the scalar functions). */
OR_API void or_spec_exp_v(size_t n, const double* in, double* out)
{ for (size_t i = 0; i < n; ++i) out[i] = or_spec_exp(in[i]); }
OR_API void or_spec_log_v(size_t n, const double* in, double* out)
{ for (size_t i = 0; i < n; ++i) out[i] = or_spec_log(in[i]); }
OR_API void or_spec_log1p_v(size_t n, const double* in, double* out)
{ for (size_t i = 0; i < n; ++i) out[i] = or_spec_log1p(in[i]); }
OR_API void or_erdf_icdf_v(const double erdf[5], int linear_space, size_t n,
                           const double* U, double* out)
{ for (size_t i = 0; i < n; ++i) out[i] = or_erdf_icdf(erdf, linear_space, U[i]); }
OR_API void or_philox_v(size_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{ for (size_t i = 0; i < n; ++i) or_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i); }
