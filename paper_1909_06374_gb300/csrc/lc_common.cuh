// lc_common.cuh -- device-side building blocks of the GB300 light-curve generator
// (Sartori et al. 2019, Sec. 2.1): per-curve descriptors, the Philox4x32-10
// counter-based generator, bit-reproducible exp/log for the ERDF inverse CDF,
// and complex helpers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lc {

// ------------------------------------------------------------------ layout
// One light curve in a ragged batch.  Sample k of curve c lives at off + k of
// the flat state/draw buffers; its N/2+1 amplitudes at offh + j.
struct CurveDev {
    uint64_t off;
    uint64_t offh;
    uint32_t log2n;
    uint32_t iters;
    double dt, f_br, a_lo, a_hi;          // Eq. 3
    double umin, umax, ub, sl_lo, sl_hi;  // ERDF in log10(lambda)
    int32_t lin;
    int32_t cls;
    uint64_t seed, curve_id;
    int32_t kind;                         // lc_erdf_kind
    int32_t coeffs;                       // lc_tk_coeffs
    int32_t targets;                      // lc_targets
    int32_t pad;
    double sigma;                         // log-normal width (dex)
    uint64_t tab;                         // tabulated shapes: offset of the CDF table (doubles)
};

// Per-curve constants of the ERDF inverse CDF (computed once per curve on the
// device with the same operation sequence that every draw then reuses).
struct ErdfConst {
    double c1, c2, e1, M1, Msum, lo, hi, umin, ub;
    int32_t a1nz, a2nz;
};

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cplx = typename cplx_of<T>::type;

template <typename T> struct key_of;
template <> struct key_of<float> { using type = uint32_t; };
template <> struct key_of<double> { using type = unsigned long long; };

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { V r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { V r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b)
{
    V r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename V> __device__ __forceinline__ V cconj(V a) { a.y = -a.y; return a; }
template <typename V, typename S> __device__ __forceinline__ V cscale(V a, S s) { a.x *= s; a.y *= s; return a; }

// ------------------------------------------------------------ order keys
// Monotone map of an IEEE value to an unsigned key (ascending order of the
// value is ascending order of the key); -0 is folded onto +0 first.
__device__ __forceinline__ uint32_t order_key(float v)
{
    v = v + 0.0f;
    uint32_t b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ unsigned long long order_key(double v)
{
    v = v + 0.0;
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ float key_value(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
__device__ __forceinline__ double key_value(unsigned long long k)
{
    return __longlong_as_double((long long)((k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k));
}

// ------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror & Shaw (SC'11): ten rounds of the Philox-4x32 bijection
// with multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key increments
// 0x9E3779B9 / 0xBB67AE85.  Counter (idx lo, idx hi, curve_id lo, stream tag),
// key (seed lo, seed hi).  Stream tags: 0 = TK95 Gaussians, 1 = ERDF uniforms.
__device__ __forceinline__ uint4 philox(uint64_t idx, uint64_t curve_id, uint32_t tag, uint64_t seed)
{
    uint32_t c0 = (uint32_t)idx, c1 = (uint32_t)(idx >> 32), c2 = (uint32_t)curve_id, c3 = tag;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo_a = 0xD2511F53u * c0, hi_a = __umulhi(0xD2511F53u, c0);
        const uint32_t lo_b = 0xCD9E8D57u * c2, hi_b = __umulhi(0xCD9E8D57u, c2);
        c0 = hi_b ^ c1 ^ k0;
        c1 = lo_b;
        c2 = hi_a ^ c3 ^ k1;
        c3 = lo_a;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// (w0, w1) -> U in (0,1): the top 52 bits u of w1:w0, U = (2u+1) 2^-53 (exact).
__device__ __forceinline__ double unit_open(uint32_t w0, uint32_t w1)
{
    const unsigned long long x = ((unsigned long long)w1 << 32) | w0;
    const unsigned long long u = x >> 12;
    return __dmul_rn((double)(2ull * u + 1ull), 0x1p-53);
}

// --------------------------------------------------- reproducible exp / log
// Every step is a correctly rounded IEEE operation (explicit _rn intrinsics,
// so the compiler cannot contract or reorder), hence the same bits on any
// IEEE machine that runs the same sequence.
//   exp: Cody-Waite reduction x = k ln2 + r with ln2 split into a 32-bit head
//        and a tail, then e^r by its degree-13 Taylor polynomial (Horner, fma).
//   log: x = 2^e m, m in [sqrt(1/2), sqrt(2)); ln m = 2 atanh(s),
//        s = (m-1)/(m+1) with the quotient's rounding error carried along.
#define LC_LN2_HI 0x1.62e42fee00000p-1
#define LC_LN2_LO 0x1.a39ef35793c76p-33
#define LC_INV_LN2 0x1.71547652b82fep+0
#define LC_SQRT_HALF 0x1.6a09e667f3bcdp-1
#define LC_LN10 0x1.26bb1bbb55516p+1

__device__ __forceinline__ double pow2_scale(double p, int k)
{
    // p * 2^k for -1022 <= k <= 1023 as one multiply by an exact power of two.
    const double two_k = __longlong_as_double((long long)(k + 1023) << 52);
    return __dmul_rn(p, two_k);
}

__device__ inline double spec_exp(double x)
{
    if (x != x) return x;
    if (x > 709.0) return __longlong_as_double(0x7ff0000000000000ll);
    if (x < -708.0) return 0.0;
    const double k = rint(__dmul_rn(x, LC_INV_LN2));
    double r = __fma_rn(-k, LC_LN2_HI, x);
    r = __fma_rn(-k, LC_LN2_LO, r);
    double p = 0x1.6124613a86d09p-33;        // 1/13!
    p = __fma_rn(p, r, 0x1.1eed8eff8d898p-29); // 1/12!
    p = __fma_rn(p, r, 0x1.ae64567f544e4p-26); // 1/11!
    p = __fma_rn(p, r, 0x1.27e4fb7789f5cp-22); // 1/10!
    p = __fma_rn(p, r, 0x1.71de3a556c734p-19); // 1/9!
    p = __fma_rn(p, r, 0x1.a01a01a01a01ap-16); // 1/8!
    p = __fma_rn(p, r, 0x1.a01a01a01a01ap-13); // 1/7!
    p = __fma_rn(p, r, 0x1.6c16c16c16c17p-10); // 1/6!
    p = __fma_rn(p, r, 0x1.1111111111111p-7);  // 1/5!
    p = __fma_rn(p, r, 0x1.5555555555555p-5);  // 1/4!
    p = __fma_rn(p, r, 0x1.5555555555555p-3);  // 1/3!
    p = __fma_rn(p, r, 0.5);
    p = __fma_rn(p, r, 1.0);
    p = __fma_rn(p, r, 1.0);
    return pow2_scale(p, (int)k);
}

__device__ inline double spec_log(double x)
{
    if (x != x || x < 0.0) return __longlong_as_double(0x7ff8000000000000ll);
    if (x == 0.0) return __longlong_as_double((long long)0xfff0000000000000ull);
    if (x == __longlong_as_double(0x7ff0000000000000ll)) return x;
    long long b = __double_as_longlong(x);
    int ex = (int)((b >> 52) & 0x7ff);
    int e;
    if (ex == 0) {  // subnormal input: scale into the normal range first
        b = __double_as_longlong(__dmul_rn(x, 0x1p54));
        ex = (int)((b >> 52) & 0x7ff);
        e = ex - 1022 - 54;
    } else {
        e = ex - 1022;
    }
    double m = __longlong_as_double((b & (long long)0x800fffffffffffffull) | (1022ll << 52));  // [0.5, 1)
    if (m < LC_SQRT_HALF) { m = __dmul_rn(m, 2.0); e = e - 1; }
    const double f = __dsub_rn(m, 1.0);
    const double d = __dadd_rn(m, 1.0);
    const double dl = __dsub_rn(m, __dsub_rn(d, 1.0));
    const double s = __ddiv_rn(f, d);
    double r = __fma_rn(-s, d, f);
    r = __fma_rn(-s, dl, r);
    const double s_lo = __ddiv_rn(r, d);
    const double z = __dmul_rn(s, s);
    double q = 0x1.8618618618618p-5;          // 1/21
    q = __fma_rn(q, z, 0x1.af286bca1af28p-5); // 1/19
    q = __fma_rn(q, z, 0x1.e1e1e1e1e1e1ep-5); // 1/17
    q = __fma_rn(q, z, 0x1.1111111111111p-4); // 1/15
    q = __fma_rn(q, z, 0x1.3b13b13b13b14p-4); // 1/13
    q = __fma_rn(q, z, 0x1.745d1745d1746p-4); // 1/11
    q = __fma_rn(q, z, 0x1.c71c71c71c71cp-4); // 1/9
    q = __fma_rn(q, z, 0x1.2492492492492p-3); // 1/7
    q = __fma_rn(q, z, 0x1.999999999999ap-3); // 1/5
    q = __fma_rn(q, z, 0x1.5555555555555p-2); // 1/3
    const double two_s = __dmul_rn(2.0, s);
    const double sz = __dmul_rn(two_s, z);
    const double de = (double)e;
    double small = __fma_rn(de, LC_LN2_LO, __dmul_rn(2.0, s_lo));
    small = __fma_rn(sz, q, small);
    const double t = __dadd_rn(two_s, small);
    return __fma_rn(de, LC_LN2_HI, t);
}

// log(1+y) = log(w) + c/w with w = 1+y rounded and c = y - (w-1) exact.
__device__ inline double spec_log1p(double y)
{
    const double w = __dadd_rn(1.0, y);
    if (w == 1.0) return y;
    const double d = __dsub_rn(w, 1.0);
    const double c = __dsub_rn(y, d);
    const double t = __ddiv_rn(c, w);
    return __dadd_rn(spec_log(w), t);
}

// ------------------------------------------------------------ ERDF (Sec. 2.1.1)
// Sharp broken power law in u = log10(lambda), slopes a1 below / a2 above the
// break ub on [umin, umax]; with c = a ln10 the unnormalised CDF pieces are
// M1 = (1 - e^{c1 (umin-ub)})/c1 and M2 = (e^{c2 (umax-ub)} - 1)/c2.
__device__ inline ErdfConst erdf_constants(const CurveDev& cv)
{
    ErdfConst k;
    double a1 = cv.sl_lo, a2 = cv.sl_hi;
    if (cv.lin) { a1 = __dadd_rn(a1, 1.0); a2 = __dadd_rn(a2, 1.0); }
    k.c1 = __dmul_rn(a1, LC_LN10);
    k.c2 = __dmul_rn(a2, LC_LN10);
    k.a1nz = a1 != 0.0;
    k.a2nz = a2 != 0.0;
    k.e1 = 0.0;
    double M1, M2;
    if (k.a1nz) {
        k.e1 = spec_exp(__dmul_rn(k.c1, __dsub_rn(cv.umin, cv.ub)));
        M1 = __ddiv_rn(__dsub_rn(1.0, k.e1), k.c1);
    } else {
        M1 = __dsub_rn(cv.ub, cv.umin);
    }
    if (k.a2nz) {
        const double e2 = spec_exp(__dmul_rn(k.c2, __dsub_rn(cv.umax, cv.ub)));
        M2 = __ddiv_rn(__dsub_rn(e2, 1.0), k.c2);
    } else {
        M2 = __dsub_rn(cv.umax, cv.ub);
    }
    k.M1 = M1;
    k.Msum = __dadd_rn(M1, M2);
    k.lo = spec_exp(__dmul_rn(LC_LN10, cv.umin));
    k.hi = spec_exp(__dmul_rn(LC_LN10, cv.umax));
    k.umin = cv.umin;
    k.ub = cv.ub;
    return k;
}

// Inverse CDF: v = U (M1+M2); below the break u = ub + ln(e1 + c1 v)/c1,
// above u = ub + ln(1 + c2 (v - M1))/c2 (spec_log1p's steps); lambda =
// e^{ln10 u} clamped.  The two branches only prepare the argument of one
// shared spec_log call (and the quotient log1p adds), so a warp whose lanes
// fall on both sides of the break runs the logarithm once; every lane still
// performs exactly the operations, in the order, of its own branch.
__device__ __forceinline__ double erdf_draw(const ErdfConst& k, double U)
{
    const double v = __dmul_rn(U, k.Msum);
    double u = 0.0, arg = 1.0, add = 0.0, cdiv = 1.0, t = 0.0;
    bool need_log = false, add_q = false, have_t = false;
    if (v < k.M1) {
        if (k.a1nz) {
            arg = __dadd_rn(k.e1, __dmul_rn(k.c1, v));
            cdiv = k.c1;
            need_log = true;
        } else {
            u = __dadd_rn(k.umin, v);
        }
    } else {
        if (k.a2nz) {
            const double y = __dmul_rn(k.c2, __dsub_rn(v, k.M1));
            const double w = __dadd_rn(1.0, y);
            cdiv = k.c2;
            if (w == 1.0) {  // spec_log1p(y) = y
                t = y;
                have_t = true;
            } else {
                const double d = __dsub_rn(w, 1.0);
                add = __ddiv_rn(__dsub_rn(y, d), w);
                arg = w;
                need_log = add_q = true;
            }
        } else {
            u = __dadd_rn(k.ub, __dsub_rn(v, k.M1));
        }
    }
    if (need_log) {
        const double L = spec_log(arg);
        t = add_q ? __dadd_rn(L, add) : L;
        have_t = true;
    }
    if (have_t) u = __dadd_rn(k.ub, __ddiv_rn(t, cdiv));
    double lam = spec_exp(__dmul_rn(LC_LN10, u));
    if (lam < k.lo) lam = k.lo;
    if (lam > k.hi) lam = k.hi;
    return lam;
}

// ---------------------------------------- tabulated ERDF shapes (Eq. 1, Eq. 2)
// The smooth broken power law of Eq. 1 and the log-normal of Eq. 2 have no
// closed-form inverse CDF.  Their unnormalised CDF is tabulated on
// kErdfTable uniform intervals of u = log10(lambda) (Simpson's rule per
// interval, accumulated in order by one thread), inverted by bisection and
// linear interpolation inside the interval.  Every step is a correctly
// rounded operation with the order fixed, so the table and the draws have the
// same bits in any IEEE reimplementation of the same sequence.
constexpr int kErdfTable = 4096;

// Density in u, up to a constant: with d = u - ub,
//   kind 1: [e^{-c1 d} + e^{-c2 d}]^-1, c = slope ln10 (+ ln10 with lin);
//   kind 2: e^{-(d/sigma)^2/2} (times e^{ln10 d} with lin).
__device__ inline double erdf_density(const CurveDev& cv, double u)
{
    const double d = __dsub_rn(u, cv.ub);
    if (cv.kind == 1) {
        double a1 = cv.sl_lo, a2 = cv.sl_hi;
        if (cv.lin) { a1 = __dadd_rn(a1, 1.0); a2 = __dadd_rn(a2, 1.0); }
        const double c1 = __dmul_rn(a1, LC_LN10), c2 = __dmul_rn(a2, LC_LN10);
        return __ddiv_rn(1.0, __dadd_rn(spec_exp(__dmul_rn(-c1, d)), spec_exp(__dmul_rn(-c2, d))));
    }
    const double t = __ddiv_rn(d, cv.sigma);
    double e = __dmul_rn(__dmul_rn(-0.5, t), t);
    if (cv.lin) e = __dadd_rn(e, __dmul_rn(LC_LN10, d));
    return spec_exp(e);
}

__device__ __forceinline__ double erdf_table_step(const CurveDev& cv)
{
    return __ddiv_rn(__dsub_rn(cv.umax, cv.umin), (double)kErdfTable);
}

// Simpson's rule on interval k: (f(u_k) + 4 f(u_k + h/2) + f(u_{k+1})) h/6,
// u_k = umin + k h.
__device__ inline double erdf_table_interval(const CurveDev& cv, int k)
{
    const double h = erdf_table_step(cv);
    const double h6 = __ddiv_rn(h, 6.0);
    const double u0 = __dadd_rn(cv.umin, __dmul_rn((double)k, h));
    const double u1 = __dadd_rn(cv.umin, __dmul_rn((double)(k + 1), h));
    const double um = __dadd_rn(u0, __dmul_rn(0.5, h));
    double sum = __dadd_rn(erdf_density(cv, u0), __dmul_rn(4.0, erdf_density(cv, um)));
    sum = __dadd_rn(sum, erdf_density(cv, u1));
    return __dmul_rn(sum, h6);
}

// Inverse of the tabulated CDF F[0..kErdfTable] (F in any memory space):
// v = U F_T, interval k with F_k <= v < F_{k+1}, u linear in v inside it,
// lambda = e^{ln10 u} clamped to [lo, hi].
__device__ __forceinline__ double erdf_draw_tab(const double* F, double umin, double h, double lo, double hi,
                                                double U)
{
    const double v = __dmul_rn(U, F[kErdfTable]);
    int a = 0, b = kErdfTable;
    while (b - a > 1) {
        const int mid = (a + b) >> 1;
        if (F[mid] <= v) a = mid; else b = mid;
    }
    const double den = __dsub_rn(F[a + 1], F[a]);
    const double t = den > 0.0 ? __ddiv_rn(__dsub_rn(v, F[a]), den) : 0.0;
    const double u = __dadd_rn(__dadd_rn(umin, __dmul_rn((double)a, h)), __dmul_rn(t, h));
    double lam = spec_exp(__dmul_rn(LC_LN10, u));
    if (lam < lo) lam = lo;
    if (lam > hi) lam = hi;
    return lam;
}

// ----------------------------------------------------------- convergence
// Convergence test of Sec. 3.2.2 (Eq. 4): delta_i = rms_n log10(x_i/x_{i-1}).
struct ConvDev {
    const double* thr;   // [ncurves] stop thresholds (delta_i < thr stops the curve)
    double* delta;       // [ncurves][hist] delta of 0-based iteration i (NaN: not run)
    double* part;        // per-block partial sums of squared natural-log ratios
    uint32_t hist;       // iterations recorded per curve
};

// (ln(xn/xp))^2 for positive xn, xp.  Near 1 the ratio is taken as
// log1p((xn - xp)/xp): the difference is exact there (the two are within a
// factor two), so a small change keeps its relative accuracy.  Far from 1 the
// quotient is used, or the difference of logs when it would leave the normal
// range.
__device__ __forceinline__ float ln_ratio_sq(float xn, float xp)
{
    const float d = xn - xp;
    float t;
    if (fabsf(d) <= 0.5f * xp) {
        t = log1pf(__fdiv_rn(d, xp));
    } else {
        const float r = __fdiv_rn(xn, xp);
        t = (r >= 1.17549435e-38f && r <= 3.40282347e+38f) ? logf(r) : logf(xn) - logf(xp);
    }
    return t * t;
}
__device__ __forceinline__ double ln_ratio_sq(double xn, double xp)
{
    const double d = xn - xp;
    double t;
    if (fabs(d) <= 0.5 * xp) {
        t = log1p(__ddiv_rn(d, xp));
    } else {
        const double r = __ddiv_rn(xn, xp);
        t = (r >= 2.2250738585072014e-308 && r <= 1.7976931348623157e+308) ? log(r) : log(xn) - log(xp);
    }
    return t * t;
}

// delta from the sum of (ln ratio)^2 over the n samples of a curve
// (log10 = ln / ln 10).
__device__ __forceinline__ double conv_delta(double sum_ln2, double n)
{
    return sqrt(sum_ln2 / n) * 0.43429448190325182765;
}

// Records delta of iteration i for curve c (caller: one thread) and returns
// whether the curve stops after it.
__device__ __forceinline__ bool conv_record(const ConvDev& cv, int c, int i, double delta)
{
    if ((uint32_t)i < cv.hist) cv.delta[(size_t)c * cv.hist + i] = delta;
    return delta < cv.thr[c];
}

}  // namespace lc
