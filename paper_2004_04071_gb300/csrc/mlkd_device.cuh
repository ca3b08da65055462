// mlkd_device.cuh -- device primitives of the correlated-pair path.
//
//   * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with the ten round
//     keys precomputed on the host and read from the kernel's parameter bank.
//   * uniform -> N(0,1) by Box-Muller and -> Exp(1) by -log u (the paper's
//     draw sets of Alg. 1 and Alg. 2: nu_{k+1}, E_{k+1}, chi_k per fine event).
//   * homogeneous KD coefficients a, d of eqs. advection/diffusion (Sec. 2)
//     and the dimensionless aggregation weights of Sec. 3.2.
//   * inverse CDF of the density 1 + cos(2 pi x) on [0, 1).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mlkd {

constexpr uint32_t kPhiloxMulA = 0xD2511F53u;
constexpr uint32_t kPhiloxMulB = 0xCD9E8D57u;

struct PhiloxKeys {
    uint32_t k0[10];   // key word 0 for rounds 0..9 (key + r * Weyl constant)
    uint32_t k1[10];
};

// One Philox4x32-10 block.  Each round multiplies counter words 0 and 2 by the
// two published multipliers (32x32 -> 64 bits), permutes and xors the high
// halves with the other words and the round key.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxKeys &rk)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32x32 -> 64-bit product per multiplier gives both halves
        const unsigned long long pa = (unsigned long long)kPhiloxMulA * c.x;
        const unsigned long long pb = (unsigned long long)kPhiloxMulB * c.z;
        c = make_uint4((uint32_t)(pb >> 32) ^ c.y ^ rk.k0[r], (uint32_t)pb,
                       (uint32_t)(pa >> 32) ^ c.w ^ rk.k1[r], (uint32_t)pa);
    }
    return c;
}

// ---------------------------------------------------------------------------
// Arithmetic of one precision.
// ---------------------------------------------------------------------------
template <typename Real> struct Arith;

template <> struct Arith<float> {
    static __device__ __forceinline__ float log_(float x) { return logf(x); }
    static __device__ __forceinline__ float exp_(float x) { return expf(x); }
    static __device__ __forceinline__ float min_(float a, float b) { return fminf(a, b); }
    static __device__ __forceinline__ float max_(float a, float b) { return fmaxf(a, b); }
    static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
    // a / b to about 2 ulp (|b| below 2^126), for quotients whose error the
    // FP32 per-pair bound absorbs
    static __device__ __forceinline__ float div_(float a, float b) { return __fdividef(a, b); }
    // sqrt of x >= 0 from y = x * rsqrt(x) and one Newton correction
    // y + (x - y^2) rsqrt(x)/2 (Heron's step), without a branch; 0 for x <= 0.
    // The raw product alone is biased by up to about 2^-22 relative, which
    // shows in the fine-minus-coarse means; the corrected root does not.
    static __device__ __forceinline__ float sqrt_pos_(float x)
    {
        const float r = rsqrtf(fmaxf(x, 1e-37f));
        const float y = x * r;
        const float z = fmaf(fmaf(-y, y, x), 0.5f * r, y);
        return x > 0.0f ? z : 0.0f;
    }
    // the raw product, for uses whose bias cancels
    static __device__ __forceinline__ float sqrt_pos_fast_(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
    static __device__ __forceinline__ float cbrt_(float x) { return cbrtf(x); }
    static __device__ __forceinline__ void sincospi_(float x, float *s, float *c) { sincospif(x, s, c); }
    static __device__ __forceinline__ float sinpi_(float x) { return sinpif(x); }
    static __device__ __forceinline__ float floor_(float x) { return floorf(x); }

    // (f(s)/s^3, g(s)/s^3, h(s)/s^2) for 0 <= s < 1, where
    //   f(s) = 2(e^{-s}-1) + s(e^{-s}+1) = sum_{n>=3} (-1)^n (2-n)     s^n/n!
    //   g(s) = 1 - 2 s e^{-s} - e^{-2s}   = sum_{n>=3} (-1)^n (2n-2^n) s^n/n!
    //   h(s) = e^{-s} + s - 1             = sum_{n>=2} (-1)^n          s^n/n!
    // as Chebyshev interpolants on [0, 1] (degrees 6, 9, 6; FP32 Horner error
    // at most 2.2, 2.7 and 1.2 x 2^-24 relative), written by
    // gen_series_fp32.py beside this file.
    static __device__ __forceinline__ float f_series(float s)
    {
        float p = 1.301975954e-05f;
        p = fmaf(p, s, -1.407892123e-04f); p = fmaf(p, s, 9.867830668e-04f);
        p = fmaf(p, s, -5.553742871e-03f); p = fmaf(p, s, 2.499970049e-02f);
        p = fmaf(p, s, -8.333331347e-02f); p = fmaf(p, s, 1.666666716e-01f);
        return p;
    }
    static __device__ __forceinline__ float g_series(float s)
    {
        float p = -4.008331416e-06f;
        p = fmaf(p, s, 4.246406752e-05f);  p = fmaf(p, s, -2.675861761e-04f);
        p = fmaf(p, s, 1.355129993e-03f);  p = fmaf(p, s, -5.949722603e-03f);
        p = fmaf(p, s, 2.261834778e-02f);  p = fmaf(p, s, -7.222211361e-02f);
        p = fmaf(p, s, 1.833333224e-01f);  p = fmaf(p, s, -3.333333433e-01f);
        p = fmaf(p, s, 3.333333433e-01f);
        return p;
    }
    static __device__ __forceinline__ float h_series(float s)
    {
        float p = 1.692812657e-05f;
        p = fmaf(p, s, -1.883247605e-04f); p = fmaf(p, s, 1.382241608e-03f);
        p = fmaf(p, s, -8.331050165e-03f); p = fmaf(p, s, 4.166629165e-02f);
        p = fmaf(p, s, -1.666666418e-01f); p = fmaf(p, s, 5.000000000e-01f);
        return p;
    }
    // z - sin z = z^3 S(z^2) with S = sum_{n>=1} (-1)^{n+1} z^{2n-2}/(2n+1)!,
    // used for |z| <= pi/4.
    static __device__ __forceinline__ float zms_series(float z2)
    {
        float p = -1.60590438e-10f;
        p = fmaf(p, z2, 2.50521084e-08f);  p = fmaf(p, z2, -2.75573192e-06f);
        p = fmaf(p, z2, 0.000198412698f);  p = fmaf(p, z2, -0.00833333333f);
        p = fmaf(p, z2, 0.166666667f);
        return p;
    }
    static constexpr int kHalleySteps = 2;
};

template <> struct Arith<double> {
    static __device__ __forceinline__ double log_(double x) { return log(x); }
    static __device__ __forceinline__ double exp_(double x) { return exp(x); }
    static __device__ __forceinline__ double min_(double a, double b) { return fmin(a, b); }
    static __device__ __forceinline__ double max_(double a, double b) { return fmax(a, b); }
    static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
    static __device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
    static __device__ __forceinline__ double div_(double a, double b) { return a / b; }
    static __device__ __forceinline__ double sqrt_pos_(double x) { return x > 0.0 ? sqrt(x) : 0.0; }
    static __device__ __forceinline__ double cbrt_(double x) { return cbrt(x); }
    static __device__ __forceinline__ void sincospi_(double x, double *s, double *c) { sincospi(x, s, c); }
    static __device__ __forceinline__ double sinpi_(double x) { return sinpi(x); }
    static __device__ __forceinline__ double floor_(double x) { return floor(x); }

    // Same series as the float version, truncated below 2^-53 of the leading
    // term at s = 1.
    static __device__ __forceinline__ double f_series(double s)
    {
        double p = -7.398571721961897e-18;
        p = fma(p, s, 1.3975079919261362e-16);  p = fma(p, s, -2.499073114973796e-15);
        p = fma(p, s, 4.2171858815182813e-14);  p = fma(p, s, -6.6912682653423392e-13);
        p = fma(p, s, 9.941312851365761e-12);   p = fma(p, s, -1.376489471727567e-10);
        p = fma(p, s, 1.7664948220503776e-09);  p = fma(p, s, -2.08767569878681e-08);
        p = fma(p, s, 2.2546897546897547e-07);  p = fma(p, s, -2.2045855379188711e-06);
        p = fma(p, s, 1.9290123456790123e-05);  p = fma(p, s, -0.00014880952380952382);
        p = fma(p, s, 0.00099206349206349201);  p = fma(p, s, -0.0055555555555555558);
        p = fma(p, s, 0.025000000000000001);    p = fma(p, s, -0.083333333333333329);
        p = fma(p, s, 0.16666666666666666);
        return p;
    }
    static __device__ __forceinline__ double g_series(double s)
    {
        double p = 2.1632343257724527e-18;
        p = fma(p, s, -2.7040392002191521e-17); p = fma(p, s, 3.2448385302886073e-16);
        p = fma(p, s, -3.7315456265699741e-15); p = fma(p, s, 4.1046610433448451e-14);
        p = fma(p, s, -4.3098159994772441e-13); p = fma(p, s, 4.3096680280428047e-12);
        p = fma(p, s, -4.0939191001221986e-11); p = fma(p, s, 3.6840773569492835e-10);
        p = fma(p, s, -3.1307488318070328e-09); p = fma(p, s, 2.5035284625231715e-08);
        p = fma(p, s, -1.8761551499646739e-07); p = fma(p, s, 1.3113815197148531e-06);
        p = fma(p, s, -8.5010154454598902e-06); p = fma(p, s, 5.0755571588904921e-05);
        p = fma(p, s, -0.00027667548500881836); p = fma(p, s, 0.0013613315696649031);
        p = fma(p, s, -0.0059523809523809521);  p = fma(p, s, 0.022619047619047618);
        p = fma(p, s, -0.072222222222222215);   p = fma(p, s, 0.18333333333333332);
        p = fma(p, s, -0.33333333333333331);    p = fma(p, s, 0.33333333333333331);
        return p;
    }
    static __device__ __forceinline__ double h_series(double s)
    {
        double p = -8.2206352466243295e-18;
        p = fma(p, s, 1.5619206968586225e-16);  p = fma(p, s, -2.8114572543455206e-15);
        p = fma(p, s, 4.7794773323873853e-14);  p = fma(p, s, -7.6471637318198164e-13);
        p = fma(p, s, 1.1470745597729725e-11);  p = fma(p, s, -1.6059043836821613e-10);
        p = fma(p, s, 2.08767569878681e-09);    p = fma(p, s, -2.505210838544172e-08);
        p = fma(p, s, 2.7557319223985888e-07);  p = fma(p, s, -2.7557319223985893e-06);
        p = fma(p, s, 2.4801587301587302e-05);  p = fma(p, s, -0.00019841269841269841);
        p = fma(p, s, 0.0013888888888888889);   p = fma(p, s, -0.0083333333333333332);
        p = fma(p, s, 0.041666666666666664);    p = fma(p, s, -0.16666666666666666);
        p = fma(p, s, 0.5);
        return p;
    }
    static __device__ __forceinline__ double zms_series(double z2)
    {
        double p = 8.2206352466243295e-18;
        p = fma(p, z2, -2.8114572543455206e-15); p = fma(p, z2, 7.6471637318198164e-13);
        p = fma(p, z2, -1.6059043836821613e-10); p = fma(p, z2, 2.505210838544172e-08);
        p = fma(p, z2, -2.7557319223985893e-06); p = fma(p, z2, 0.00019841269841269841);
        p = fma(p, z2, -0.0083333333333333332);  p = fma(p, z2, 0.16666666666666666);
        return p;
    }
    static constexpr int kHalleySteps = 3;
};

// ---------------------------------------------------------------------------
// Draws of one fine event: nu_{k+1}, E_{k+1}, chi_k.
//   float : one Philox block; u = ((w >> 8) + 1) 2^-24 in (0, 1].
//   double: two Philox blocks (tag 0 and 1 in counter word 2);
//           u = (((w_a << 21) ^ (w_b >> 11)) + 1) 2^-53 in (0, 1].
// The init block (k = 0) gives nu_0 (cosine half of Box-Muller), E_0 and the
// uniform of the initial position.
// ---------------------------------------------------------------------------
template <typename Real> struct Draw { Real nu, E, chi, u4; };

__device__ __forceinline__ float unit24(uint32_t w)
{
    return __uint2float_rn((w >> 8) + 1u) * 0x1p-24f;
}

__device__ __forceinline__ double unit53(uint32_t wa, uint32_t wb)
{
    const unsigned long long m = ((unsigned long long)wa << 21) ^ (unsigned long long)(wb >> 11);
    return __ull2double_rn(m + 1ull) * 0x1p-53;
}

template <typename Real>
__device__ __forceinline__ Draw<Real> draw(uint32_t k, uint32_t pair_lo, uint32_t word2,
                                           uint32_t request, const PhiloxKeys &rk);

// FP64 arithmetic on the 24-bit stream of the FP32 modes: one Philox block
// per fine event, u = ((w >> 8) + 1) 2^-24 (exact in FP64).
__device__ __forceinline__ Draw<double> draw_u24_fp64(uint32_t k, uint32_t pair_lo, uint32_t word2,
                                                      uint32_t request, const PhiloxKeys &rk)
{
    const uint4 w = philox4x32_10(make_uint4(k, pair_lo, word2, request), rk);
    const double u1 = (double)((w.x >> 8) + 1u) * 0x1p-24;
    const double u2 = (double)((w.y >> 8) + 1u) * 0x1p-24;
    const double u3 = (double)((w.z >> 8) + 1u) * 0x1p-24;
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    Draw<double> d;
    d.nu = r * c;
    d.chi = r * s;
    d.E = -log(u3);
    d.u4 = (double)((w.w >> 8) + 1u) * 0x1p-24;
    return d;
}

// Draw of mode RECIPE: 0 the precision's own stream, 1 the 24-bit stream in FP64.
template <typename Real, int RECIPE>
__device__ __forceinline__ Draw<Real> draw_r(uint32_t k, uint32_t pair_lo, uint32_t word2,
                                             uint32_t request, const PhiloxKeys &rk)
{
    if constexpr (RECIPE == 1) return draw_u24_fp64(k, pair_lo, word2, request, rk);
    else return draw<Real>(k, pair_lo, word2, request, rk);
}

// log u for the 24-bit uniform u = n 2^-24, n = (w >> 8) + 1 in [1, 2^24].
// n = m 2^e with the mantissa m in [sqrt(1/2), sqrt(2)), read from the bits
// of float(n) (exact for n <= 2^24): subtracting the bits of the float just
// above sqrt(1/2) (0x3F3504F4) leaves e in the exponent field, and removing
// e from the exponent leaves m.  Then the series
// log m = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + s^7/7 + s^9/9),
// s = (m - 1)/(m + 1), |s| <= 0.1716 (truncation below 1e-9).
__device__ __forceinline__ float log_unit24(uint32_t w)
{
    const uint32_t n = (w >> 8) + 1u;
    const uint32_t b = __float_as_uint(__uint2float_rn(n));
    const int e = (int)(b - 0x3F3504F4u) >> 23;
    const float m = __uint_as_float(b - ((uint32_t)e << 23));
    const float s = __fdividef(m - 1.0f, m + 1.0f);
    const float s2 = s * s;
    float p = fmaf(s2, 0.111111111f, 0.142857143f);
    p = fmaf(p, s2, 0.2f);
    p = fmaf(p, s2, 0.333333333f);
    const float lm = fmaf(2.0f * s * s2, p, 2.0f * s);
    // log u = (e - 24) ln 2 + log m, with ln 2 split into two floats
    const float k = (float)(e - 24);
    return fmaf(k, 0.693145752f, fmaf(k, 1.42860677e-06f, lm));
}

// sin and cos of 2 pi u, u = n 2^-24: 4u = k + f with k the nearest quarter
// turn (exact integer arithmetic), z = (pi/2) f in [-pi/4, pi/4], Taylor
// polynomials through z^9 (sin) and z^10 (cos), then the quarter-turn
// rotation.
__device__ __forceinline__ void sincos_2pi_unit24(uint32_t w, float *sn, float *cs)
{
    const uint32_t n = (w >> 8) + 1u;
    const uint32_t k = (n + (1u << 21)) >> 22;
    const int r = (int)n - (int)(k << 22);
    const float z = (float)r * 3.74507033e-07f;               // (pi/2) / 2^22
    const float z2 = z * z;
    float sp = fmaf(z2, 2.75573192e-06f, -1.98412698e-04f);
    sp = fmaf(sp, z2, 8.33333333e-03f);
    sp = fmaf(sp, z2, -1.66666667e-01f);
    const float sz = fmaf(sp * z2, z, z);
    float cp = fmaf(z2, -2.75573192e-07f, 2.48015873e-05f);
    cp = fmaf(cp, z2, -1.38888889e-03f);
    cp = fmaf(cp, z2, 4.16666667e-02f);
    cp = fmaf(cp, z2, -0.5f);
    const float cz = fmaf(cp, z2, 1.0f);
    const uint32_t q = k & 3u;
    const float a = (q & 1u) ? cz : sz;                       // |sin| part
    const float b = (q & 1u) ? sz : cz;                       // |cos| part
    *sn = (q & 2u) ? -a : a;
    *cs = ((q + 1u) & 2u) ? -b : b;
}

template <>
__device__ __forceinline__ Draw<float> draw<float>(uint32_t k, uint32_t pair_lo, uint32_t word2,
                                                   uint32_t request, const PhiloxKeys &rk)
{
    const uint4 w = philox4x32_10(make_uint4(k, pair_lo, word2, request), rk);
    const float r = Arith<float>::sqrt_pos_(-2.0f * log_unit24(w.x));
    float s, c;
    sincos_2pi_unit24(w.y, &s, &c);
    Draw<float> d;
    d.nu = r * c;
    d.chi = r * s;
    d.E = -log_unit24(w.z);
    d.u4 = unit24(w.w);
    return d;
}

template <>
__device__ __forceinline__ Draw<double> draw<double>(uint32_t k, uint32_t pair_lo, uint32_t word2,
                                                     uint32_t request, const PhiloxKeys &rk)
{
    const uint4 a = philox4x32_10(make_uint4(k, pair_lo, word2, request), rk);
    const uint4 b = philox4x32_10(make_uint4(k, pair_lo, word2 ^ (1u << 16), request), rk);
    const double u1 = unit53(a.x, a.y), u2 = unit53(a.z, a.w), u3 = unit53(b.x, b.y);
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    Draw<double> d;
    d.nu = r * c;
    d.chi = r * s;
    d.E = -log(u3);
    d.u4 = unit53(b.z, b.w);
    return d;
}

// ---------------------------------------------------------------------------
// floor(n / M) for 0 <= n < 2^31 and 2 <= M <= 2^30 by a multiply-high and a
// shift (division by an invariant integer, Granlund and Montgomery, PLDI
// 1994, Thm. 4.2).  With l = ceil(log2 M) and m = ceil(2^(31+l) / M):
// 2^(31+l) <= m M <= 2^(31+l) + M - 1 < 2^(31+l) + 2^l, hence
// floor(n/M) = floor(m n / 2^(31+l)) = umulhi(n, m) >> (l - 1), and m < 2^32
// (m = 2^31 when M is a power of two).  The coarse-grid index of a fine step
// takes two instructions for every M.
// ---------------------------------------------------------------------------
struct DivM {
    uint32_t mul;
    int post;
    __host__ __device__ void init(int M)
    {
        int l = 1;
        while ((1 << l) < M) ++l;
        const unsigned long long t = 1ull << (31 + l);
        mul = (uint32_t)((t + (unsigned long long)(M - 1)) / (unsigned long long)M);
        post = l - 1;
    }
    __device__ __forceinline__ int operator()(int n) const
    {
        return (int)(__umulhi((uint32_t)n, mul) >> post);
    }
};

// ---------------------------------------------------------------------------
// Homogeneous background in the working precision.
// ---------------------------------------------------------------------------
template <typename Real> struct Background {
    Real R, invR, mu, sigma;
    Real two_c2;   // 2 sigma^2 / R^2
    Real dt;       // fine step
    Real Rdt;      // R dt
    Real inv_Rdt;  // 1/(R dt): flight in fine steps per unit of E

    // KD increment of the diffusive phase of length theta with final velocity
    // offset dv = v' - mu (eqs. advection, diffusion):
    //   a = mu theta + dv (1 - e^{-s})/R,
    //   d = sqrt(2 sigma^2/R^2 f(s) + dv^2/R^2 g(s)),  s = R theta.
    // Also returns hs = h(s) = e^{-s} + s - 1 and om = 1 - e^{-s} for the
    // aggregation weights.
    // For s < 1 everything comes from the series (1 - e^{-s} = s - h(s));
    // otherwise from e^{-s}, where the closed forms do not cancel.
    __device__ __forceinline__ void kd_coeffs(Real theta, Real dv, Real &a, Real &d, Real &hs,
                                              Real &om) const
    {
        typedef Arith<Real> A;
        const Real s = R * theta;
        Real f, g;
        if (s < Real(1)) {
            const Real s2 = s * s;
            hs = s2 * A::h_series(s);
            om = s - hs;
            f = s2 * s * A::f_series(s);
            g = s2 * s * A::g_series(s);
        } else {
            const Real e = A::exp_(-s);
            om = Real(1) - e;
            hs = s - om;
            f = Real(2) * (e - Real(1)) + s * (e + Real(1));
            g = Real(1) - Real(2) * s * e - e * e;
        }
        a = mu * theta + dv * om * invR;
        const Real dvR = dv * invR;
        const Real d2 = two_c2 * f + dvR * dvR * g;
        d = A::sqrt_pos_(d2);
    }

    // Dimensionless beta weight (Sec. 3.2, eq. weights-beta) of a diffusive
    // phase with h(s) = hs, s = R theta:
    //   theta' = theta - zeta with zeta = (1 - e^{-s})/R, so s' = R theta' = h(s),
    //   and beta = (sigma/R) sqrt(2 h(s')).  Returns (beta R / sigma)^2.
    __device__ __forceinline__ Real beta_hat_sq(Real hs) const
    {
        typedef Arith<Real> A;
        const Real sp = hs;
        const Real hp = (sp < Real(1)) ? sp * sp * A::h_series(sp) : A::exp_(-sp) + sp - Real(1);
        return Real(2) * hp;
    }
};

// ---------------------------------------------------------------------------
// Initial position with density 1 + cos(2 pi x) on [0, 1): solve
// G(y) = y - sin(2 pi y)/(2 pi) = u - 1/2 for y in [-1/2, 1/2], x = y + 1/2
// wrapped into [0, 1).  Start from the small-|y| inverse
// y0 = cbrt(6 g/(2 pi)^2) (error below 0.08 everywhere) and take Halley
// steps, y <- y - 2 r G' / (2 G'^2 - r G''), r = G(y) - g, with
// G' = 2 sin^2(pi y) and G'' = 4 pi sin(pi y) cos(pi y) from one sincospi.
// Convergence is cubic: two steps reach FP32 rounding, three FP64 rounding.
// ---------------------------------------------------------------------------
template <typename Real> __device__ __forceinline__ Real cosine_inverse(Real u)
{
    typedef Arith<Real> A;
    const Real two_pi = Real(6.283185307179586476925286766559);
    const Real four_pi = Real(12.566370614359172953850573533118);
    const Real inv_pi = Real(0.31830988618379067153776752674503);
    const Real inv_two_pi = Real(0.15915494309189533576888376337251);
    const Real six_over_two_pi_sq = Real(0.15198177546350666);   // 6 / (2 pi)^2
    const Real g = u - Real(0.5);
    Real y = A::cbrt_(g * six_over_two_pi_sq);
    y = A::min_(A::max_(y, Real(-0.5)), Real(0.5));
#pragma unroll
    for (int it = 0; it < A::kHalleySteps; ++it) {
        Real sp, cp;
        A::sincospi_(y, &sp, &cp);
        Real Gy;
        if (y < Real(-0.125) || y > Real(0.125)) {
            Gy = y - sp * cp * inv_pi;                         // sin(2 pi y)/(2 pi) = s c / pi
        } else {
            const Real z = two_pi * y;                         // no cancellation near 0
            const Real z2 = z * z;
            Gy = z2 * z * A::zms_series(z2) * inv_two_pi;
        }
        const Real r = Gy - g;
        const Real g1 = Real(2) * sp * sp;
        const Real g2 = four_pi * sp * cp;
        const Real den = Real(2) * g1 * g1 - r * g2;
        if (den > Real(0)) y = y - Real(2) * r * g1 / den;
        y = A::min_(A::max_(y, Real(-0.5)), Real(0.5));
    }
    Real x = y + Real(0.5);
    if (x >= Real(1)) x -= Real(1);
    return x;
}

}  // namespace mlkd
