// mlkd_pair.cuh -- one correlated fine/coarse pair as a register-resident
// state machine, shared by the per-level kernel and the batched kernel.
//
//   pair_start : Alg. 1 / Alg. 2 initialisation (nu_0, E_0 shared by both
//                paths, x_0).
//   pair_event : one fine KD event (Alg. 1 KineticDiffusionStep) and, when
//                the new fine collision lies at or after the end of the
//                current coarse step, the coarse KD step built from the
//                aggregated random numbers (Sec. 3.1 mapping, Sec. 3.2
//                aggregation, Alg. 2).
//   pair_drift : the final kinetic move of both paths to T.
// Time is an integer count of fine steps plus a flight in fine-step units,
// so the coarse collision equals the fine collision kappa_k exactly.
#pragma once

#include <type_traits>

#include "mlkd_internal.h"

namespace mlkd {

// Observer of the coarse steps (validation only): pair_event calls
// tr->coarse(nu~, E~, chi~) at each coarse KD step when a tracer is given.
// NoTrace compiles to nothing.
struct NoTrace {};

template <typename Real> struct PairState {
    Real xf, vf, qf;            // fine path: position, velocity, flight (fine units)
    Real xc, vc, qc;            // coarse path
    Real num, den, chi_first;   // streamed eq. chi-update of the open coarse window
    int i_f, ic, Ec;            // fine-step index of each path's phase start; coarse step end
    uint32_t k, evc;            // fine events (= Philox block of the next draw - 1), coarse events
    uint32_t pair_lo, word2;    // Philox counter words of this pair
    bool fresh;                 // the open window has no term yet
};

template <typename Real> struct LevelCtx {
    Background<Real> bg;
    int n;                      // fine steps to T on this level
    int M;                      // refinement factor
    DivM divM;                  // floor(n / M)
    int init;                   // 0: x0 = 0; 1: cosine density
    uint32_t word2;             // level << 24
    uint32_t request;
};

// End of the coarse step that contains fine-step position base + steps + f
// (0 <= f < 1), with base on the coarse grid: base + M (steps / M + 1).
template <typename Real>
__device__ __forceinline__ int next_coarse_end(const LevelCtx<Real> &L, int base, int steps)
{
    return base + L.M * (L.divM(steps) + 1);
}

// CPL: 0 = level 0 (single path), 1 = coupled pair, 2 = decided at run time.
template <typename Real, int CPL>
__device__ __forceinline__ bool pair_is_coupled(bool runtime) { return CPL == 2 ? runtime : CPL == 1; }

// Alg. 1 / Alg. 2 initialisation values of pair p: x_0, v_0 and the first
// flight in fine-step units (nu_0, E_0 and the initial-position uniform of
// Philox block 0), shared by both paths.
template <typename Real, int RECIPE = 0>
__device__ __forceinline__ void pair_start_values(Real &x0, Real &v0, Real &q0, unsigned long long p,
                                                  const LevelCtx<Real> &L, const PhiloxKeys &keys)
{
    const Draw<Real> d0 = draw_r<Real, RECIPE>(0u, (uint32_t)p, L.word2 ^ (uint32_t)(p >> 32),
                                               L.request, keys);
    x0 = L.init ? cosine_inverse<Real>(d0.u4) : Real(0);
    v0 = L.bg.mu + L.bg.sigma * d0.nu;
    q0 = d0.E * L.bg.inv_Rdt;
}

// The state of pair p at t = 0 from its initialisation values.  Returns true
// if the pair has no collision before T (already finished).
template <typename Real, int CPL>
__device__ __forceinline__ bool pair_init(PairState<Real> &st, unsigned long long p, Real x0, Real v0,
                                          Real q0, const LevelCtx<Real> &L, bool coupled_rt)
{
    const bool coupled = pair_is_coupled<Real, CPL>(coupled_rt);
    st.pair_lo = (uint32_t)p;
    st.word2 = L.word2 ^ (uint32_t)(p >> 32);
    st.xf = x0;
    st.vf = v0;
    st.qf = q0;
    st.i_f = 0;
    st.k = 0;
    st.evc = 0;
    if (coupled) {
        st.xc = x0;
        st.vc = v0;
        st.qc = q0;
        st.ic = 0;
        st.num = Real(0);
        st.den = Real(0);
        st.fresh = true;
        if (q0 < (Real)L.n) st.Ec = next_coarse_end(L, 0, (int)q0);
    }
    return !(q0 < (Real)L.n);
}

// Returns true if the pair has no collision before T (already finished).
template <typename Real, int CPL, int RECIPE = 0>
__device__ __forceinline__ bool pair_start(PairState<Real> &st, unsigned long long p,
                                           const LevelCtx<Real> &L, const PhiloxKeys &keys,
                                           bool coupled_rt)
{
    Real x0, v0, q0;
    pair_start_values<Real, RECIPE>(x0, v0, q0, p, L, keys);
    return pair_init<Real, CPL>(st, p, x0, v0, q0, L, coupled_rt);
}

// One fine event; returns true when the pair has reached T.
template <typename Real, int CPL, int RECIPE = 0, typename Trace = NoTrace>
__device__ __forceinline__ bool pair_event(PairState<Real> &st, const LevelCtx<Real> &L,
                                           const PhiloxKeys &keys, bool coupled_rt,
                                           Trace *tr = nullptr)
{
    typedef Arith<Real> A;
    const bool coupled = pair_is_coupled<Real, CPL>(coupled_rt);
    const Background<Real> &bg = L.bg;
    const Draw<Real> d = draw_r<Real, RECIPE>(st.k + 1u, st.pair_lo, st.word2, L.request, keys);
    const int sq = (int)st.qf;                                  // floor: qf >= 0
    const Real theta = bg.dt * ((Real)(sq + 1) - st.qf);        // eq. diffusive-time
    const Real dv = bg.sigma * d.nu;                            // v_{k+1} - mu
    const Real v1 = bg.mu + dv;
    Real a, dd, hs, om;
    bg.kd_coeffs(theta, dv, a, dd, hs, om);
    st.xf = st.xf + st.vf * (st.qf * bg.dt) + (a + dd * d.chi); // eq. position-update
    st.i_f += sq + 1;                                           // eq. time-update
    st.vf = v1;
    st.qf = d.E * bg.inv_Rdt;                                   // eq. intinv (homogeneous)
    ++st.k;

    if (coupled) {
        // Sec. 3.2 aggregation, streamed: this phase's chi with beta, and the
        // new phase's nu with alpha if it collides inside the coarse step.
        const Real bh2 = bg.beta_hat_sq(hs);
        if (st.fresh) {
            st.chi_first = d.chi;
            st.fresh = false;
        }
        st.num += A::sqrt_pos_(bh2) * d.chi;
        st.den += bh2;
        if (st.qf < (Real)(st.Ec - st.i_f)) {
            const Real ah = st.qf * bg.Rdt + om;                  // R tau' = R tau + R zeta
            st.num += ah * d.nu;
            st.den += ah * ah;
        } else {
            // coarse KD step with nu~ = nu_kappa (eq. nu-update), chi~ (eq.
            // chi-update), then the coarse flight tau~ = fine collision - E_c
            // (homogeneous eq. epsilon-update), carried in fine units.
            const Real thc = bg.dt * ((Real)(st.Ec - st.ic) - st.qc);
            Real ac, dc, hsc, omc;
            bg.kd_coeffs(thc, dv, ac, dc, hsc, omc);
            const Real chit = st.den > Real(0) ? st.num * A::rsqrt_(st.den) : st.chi_first;
            st.xc = st.xc + st.vc * (st.qc * bg.dt) + (ac + dc * chit);
            st.qc = st.qf - (Real)(st.Ec - st.i_f);
            if constexpr (!std::is_same<Trace, NoTrace>::value)
                tr->coarse(d.nu, st.qc * bg.Rdt, chit);      // nu~, E~ = R tau~, chi~
            st.ic = st.Ec;
            st.vc = v1;
            ++st.evc;
            if (st.qc < (Real)(L.n - st.ic)) st.Ec = next_coarse_end(L, st.ic, (int)st.qc);
            st.num = Real(0);
            st.den = Real(0);
            st.fresh = true;
        }
    }
    return !(st.qf < (Real)(L.n - st.i_f));
}

// Alg. 1 / Alg. 2 epilogue: move both paths kinetically to T.
template <typename Real, int CPL>
__device__ __forceinline__ void pair_drift(PairState<Real> &st, const LevelCtx<Real> &L, bool coupled_rt)
{
    const bool coupled = pair_is_coupled<Real, CPL>(coupled_rt);
    if (st.i_f < L.n) st.xf = st.xf + st.vf * ((Real)(L.n - st.i_f) * L.bg.dt);
    if (coupled && st.ic < L.n) st.xc = st.xc + st.vc * ((Real)(L.n - st.ic) * L.bg.dt);
}

// ---------------------------------------------------------------------------
// Per-lane sums: Y, Y^2, F(x_f), F(x_f)^2, F(x_c), F(x_c)^2.
//   FP64 mode      : all six in FP64.
//   FP32_DY64 mode : Y and Y^2 formed and summed in FP64 from the FP32 state;
//                    the four F moments as compensated FP32 pairs.
//   FP32_COMP mode : all six as compensated FP32 (sum, error) pairs.
// Compensation is an error-free TwoSum per addition.
// ---------------------------------------------------------------------------
constexpr unsigned kFullMask = 0xffffffffu;

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

struct CompF {
    float s, c;
    __device__ void zero() { s = 0.0f; c = 0.0f; }
    __device__ void add(float x) {
        float t, e;
        two_sum(s, x, t, e);
        s = t;
        c += e;
    }
    __device__ void shfl_merge(int off) {
        const float so = __shfl_down_sync(kFullMask, s, off);
        const float co = __shfl_down_sync(kFullMask, c, off);
        float t, e;
        two_sum(s, so, t, e);
        s = t;
        c = c + co + e;
    }
    __device__ double value() const { return (double)s + (double)c; }
};

template <int MODE> struct PairSums;

template <> struct PairSums<kModeFP64> {
    double v[6];
    __device__ void zero() {
#pragma unroll
        for (int j = 0; j < 6; ++j) v[j] = 0.0;
    }
    __device__ void warp_reduce() {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int j = 0; j < 6; ++j) v[j] += __shfl_down_sync(kFullMask, v[j], off);
    }
    __device__ double value(int j) const { return v[j]; }
};

template <> struct PairSums<kModeFP32DY64> {
    double sy, sy2;
    CompF q[4];
    __device__ void zero() {
        sy = 0.0;
        sy2 = 0.0;
#pragma unroll
        for (int j = 0; j < 4; ++j) q[j].zero();
    }
    __device__ void warp_reduce() {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            sy += __shfl_down_sync(kFullMask, sy, off);
            sy2 += __shfl_down_sync(kFullMask, sy2, off);
#pragma unroll
            for (int j = 0; j < 4; ++j) q[j].shfl_merge(off);
        }
    }
    __device__ double value(int j) const { return j == 0 ? sy : j == 1 ? sy2 : q[j - 2].value(); }
};

template <> struct PairSums<kModeFP64U24> : PairSums<kModeFP64> {};

template <> struct PairSums<kModeFP32Comp> {
    CompF q[6];
    __device__ void zero() {
#pragma unroll
        for (int j = 0; j < 6; ++j) q[j].zero();
    }
    __device__ void warp_reduce() {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int j = 0; j < 6; ++j) q[j].shfl_merge(off);
    }
    __device__ double value(int j) const { return q[j].value(); }
};

// QoI of one finished pair (eq. mlmc-compact): F(x) = x^2 in free space or
// (x mod 1)^2 on the periodic unit interval; Y = F(x_f) - F(x_c), with
// x_f^2 - x_c^2 formed as (x_f - x_c)(x_f + x_c).
__device__ __forceinline__ void add_pair(PairSums<kModeFP64> &ps, double xf, double xc, bool coupled,
                                         bool per)
{
    const double mf = per ? xf - floor(xf) : xf;
    const double mc = per ? xc - floor(xc) : xc;
    const double Ff = mf * mf, Fc = coupled ? mc * mc : 0.0;
    const double y = !coupled ? Ff : per ? Ff - Fc : (xf - xc) * (xf + xc);
    ps.v[0] += y;
    ps.v[1] += y * y;
    ps.v[2] += Ff;
    ps.v[3] += Ff * Ff;
    ps.v[4] += Fc;
    ps.v[5] += Fc * Fc;
}

__device__ __forceinline__ void add_pair(PairSums<kModeFP32DY64> &ps, float xf, float xc, bool coupled,
                                         bool per)
{
    const float mf = per ? xf - floorf(xf) : xf;     // exact in FP32
    const float mc = per ? xc - floorf(xc) : xc;
    const double a = (double)mf, b = (double)mc;
    const double y = !coupled ? a * a : per ? a * a - b * b : (a - b) * (a + b);
    ps.sy += y;
    ps.sy2 += y * y;
    const float Ff = mf * mf, Fc = coupled ? mc * mc : 0.0f;
    ps.q[0].add(Ff);
    ps.q[1].add(Ff * Ff);
    ps.q[2].add(Fc);
    ps.q[3].add(Fc * Fc);
}

__device__ __forceinline__ void add_pair(PairSums<kModeFP32Comp> &ps, float xf, float xc, bool coupled,
                                         bool per)
{
    const float mf = per ? xf - floorf(xf) : xf;
    const float mc = per ? xc - floorf(xc) : xc;
    const float Ff = mf * mf, Fc = coupled ? mc * mc : 0.0f;
    const float y = !coupled ? Ff : per ? Ff - Fc : (xf - xc) * (xf + xc);
    ps.q[0].add(y);
    ps.q[1].add(y * y);
    ps.q[2].add(Ff);
    ps.q[3].add(Ff * Ff);
    ps.q[4].add(Fc);
    ps.q[5].add(Fc * Fc);
}

// Linear QoI F(x) = x (the position at T, the paper's test case): Y = x_f -
// x_c.  fk selects F: 0 x^2, 1 (x mod 1)^2, 2 x.
__device__ __forceinline__ void add_pair_linear(PairSums<kModeFP64> &ps, double xf, double xc, bool coupled)
{
    const double Fc = coupled ? xc : 0.0;
    const double y = xf - Fc;
    ps.v[0] += y;
    ps.v[1] += y * y;
    ps.v[2] += xf;
    ps.v[3] += xf * xf;
    ps.v[4] += Fc;
    ps.v[5] += Fc * Fc;
}

__device__ __forceinline__ void add_pair_linear(PairSums<kModeFP32DY64> &ps, float xf, float xc, bool coupled)
{
    const float Fc = coupled ? xc : 0.0f;
    const double y = (double)xf - (double)Fc;
    ps.sy += y;
    ps.sy2 += y * y;
    ps.q[0].add(xf);
    ps.q[1].add(xf * xf);
    ps.q[2].add(Fc);
    ps.q[3].add(Fc * Fc);
}

__device__ __forceinline__ void add_pair_linear(PairSums<kModeFP32Comp> &ps, float xf, float xc, bool coupled)
{
    const float Fc = coupled ? xc : 0.0f;
    const float y = xf - Fc;
    ps.q[0].add(y);
    ps.q[1].add(y * y);
    ps.q[2].add(xf);
    ps.q[3].add(xf * xf);
    ps.q[4].add(Fc);
    ps.q[5].add(Fc * Fc);
}

template <typename Sums, typename Real>
__device__ __forceinline__ void add_pair_fk(Sums &ps, Real xf, Real xc, bool coupled, int fk)
{
    if (fk == 2)
        add_pair_linear(ps, xf, xc, coupled);
    else
        add_pair(ps, xf, xc, coupled, fk == 1);
}

// Histogram bin: floor((x - lo)/h) inside [lo, hi), else -1; periodic
// positions are first wrapped into [0, 1).  FP64 state divides in FP64; FP32
// state decides its bins in FP32.
struct Bins {
    double lo, hi, h;
    float lo_f, hi_f, inv_h_f;
    int nbins;
    bool periodic;
    __device__ int operator()(double x) const {
        if (periodic) x = x - floor(x);
        if (!(x >= lo && x < hi)) return -1;
        const int b = (int)floor((x - lo) / h);
        return b < nbins ? b : nbins - 1;
    }
    __device__ int operator()(float x) const {
        if (periodic) x = x - floorf(x);
        if (!(x >= lo_f && x < hi_f)) return -1;
        const int b = (int)floorf((x - lo_f) * inv_h_f);
        return b < nbins ? b : nbins - 1;
    }
};

}  // namespace mlkd
