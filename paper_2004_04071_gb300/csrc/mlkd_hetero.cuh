// mlkd_hetero.cuh -- correlated pairs in the heterogeneous backgrounds B1/B2
// of Sec. 5: mu = 0, sigma = 1 and the piecewise-linear collision rate
//
//   R(x) = b (1 + a_left max(1 - x, 0) + a_right max(x - 1, 0)),
//
// B1: a_left = a_right = a (symmetric about x = 1), B2: a_left = 0.
//
//   * eq. intinv is solved per linear piece of R along the kinetic path, in
//     fine-step units (rho = R dt is the rate per step): on a piece
//     rho0 u + s u^2/2 = E, u = 2E/(rho0 + sqrt(rho0^2 + 2 s E));
//   * eq. epsilon-update subtracts the optical depth the fine kinetic phase
//     kappa has collected up to the coarse time t_c (its upper limit
//     t_c - t_kappa can be negative, Fig. 2(d)); the coarse flight then
//     solves eq. intinv from the coarse position;
//   * the coarse collision is no longer the fine one: Alg. 2 in its general
//     form moves the fine path (at least one KD step per window) until its
//     collision's step ends after the coarse collision's step, and the fine
//     path may step past T to feed the coarse path; its output is its state
//     at its first collision at or after T.  The pair ends once both
//     collisions lie at or after T.
//   * The corrected coefficients a^hetero, d^hetero are not printed in the
//     paper (Sec. 2 defers them to another work): the homogeneous
//     eqs. advection/diffusion are used with R at the collision point (the
//     start of the diffusive phase), and so are zeta_m and beta_m of
//     Sec. 3.2 with the rate R_m of their phase.  This is a stand-in.
#pragma once

#include "mlkd_pair.cuh"

namespace mlkd {

template <typename Real> struct HetBg {
    Real b, a_left, a_right;
    Real dt;               // fine step

    __device__ __forceinline__ Real R(Real x) const
    {
        const Real l = Real(1) - x > Real(0) ? Real(1) - x : Real(0);
        const Real r = x - Real(1) > Real(0) ? x - Real(1) : Real(0);
        return b * (Real(1) + a_left * l + a_right * r);
    }
    // dR/dx on the side of x that a path with velocity v is on (at x = 1:
    // the side it enters)
    __device__ __forceinline__ Real slope(Real x, Real v) const
    {
        const bool right = x > Real(1) || (x == Real(1) && v > Real(0));
        return right ? b * a_right : -b * a_left;
    }
    // steps u > 0 to x = 1 along x0 + v dt u, or a negative value if never
    __device__ __forceinline__ Real kink(Real x0, Real v) const
    {
        if (v == Real(0) || x0 == Real(1)) return Real(-1);
        return Arith<Real>::div_(Real(1) - x0, v * dt);
    }
    // optical depth over u >= 0 steps from x0 (eq. intinv's integral)
    __device__ Real depth_fwd(Real x0, Real v, Real u) const
    {
        const Real rho0 = R(x0) * dt;
        const Real s1 = slope(x0, v) * v * dt * dt;
        const Real s2 = slope(Real(1), v) * v * dt * dt;
        const Real uk = s1 == s2 ? Real(-1) : kink(x0, v);
        if (!(uk > Real(0)) || u <= uk) return rho0 * u + Real(0.5) * s1 * u * u;
        const Real I1 = rho0 * uk + Real(0.5) * s1 * uk * uk;
        const Real w = u - uk;
        return I1 + b * dt * w + Real(0.5) * s2 * w * w;
    }
    // the same for any sign of u (the segment behind x0 counts negative)
    __device__ Real depth(Real x0, Real v, Real u) const
    {
        if (u < Real(0)) return -depth_fwd(x0 + v * dt * u, v, -u);
        return depth_fwd(x0, v, u);
    }
    __device__ __forceinline__ static Real piece_root(Real rho, Real s, Real E)
    {
        if (s == Real(0)) return Arith<Real>::div_(E, rho);
        Real disc = rho * rho + Real(2) * s * E;
        if (disc < Real(0)) disc = Real(0);
        return Arith<Real>::div_(Real(2) * E, rho + Arith<Real>::sqrt_pos_(disc));
    }
    // eq. intinv: steps u with depth E from x0 at velocity v
    __device__ Real flight(Real x0, Real v, Real E) const
    {
        const Real rho0 = R(x0) * dt;
        const Real s1 = slope(x0, v) * v * dt * dt;
        const Real s2 = slope(Real(1), v) * v * dt * dt;
        const Real uk = s1 == s2 ? Real(-1) : kink(x0, v);
        if (uk > Real(0)) {
            const Real I1 = rho0 * uk + Real(0.5) * s1 * uk * uk;
            if (E > I1) return uk + piece_root(b * dt, s2, E - I1);
        }
        return piece_root(rho0, s1, E);
    }
};

template <typename Real> struct HetPairState {
    // fine path: position and velocity at the phase start, flight (steps) and its E
    Real xf, vf, qf, Ef;
    // coarse path
    Real xc, vc, qc;
    // open window of eq. chi-update
    Real num, den, chi_first;
    // fine output: the state at the first fine collision at or after T
    Real xo, vo;
    int i_f, ic, io;
    uint32_t k, evc;              // fine KD steps taken, coarse KD steps
    uint32_t pair_lo, word2;
    bool fresh, have_out;
};

template <typename Real> struct HetLevel {
    HetBg<Real> bg;
    int n, M;
    DivM divM;                    // floor(n / M)
    Real x0;
    uint32_t word2, request;
};

// Homogeneous KD coefficients (eqs. advection/diffusion, mu = 0, sigma = 1)
// at rate R: a, d and the aggregation quantities hs = h(R theta),
// om = 1 - e^{-R theta}.
template <typename Real>
__device__ __forceinline__ void het_kd(Real R, Real theta, Real v1, Real &a, Real &d, Real &hs, Real &om)
{
    Background<Real> bg;
    bg.R = R;
    bg.invR = Arith<Real>::div_(Real(1), R);
    bg.mu = Real(0);
    bg.sigma = Real(1);
    bg.two_c2 = Real(2) * bg.invR * bg.invR;
    bg.kd_coeffs(theta, v1, a, d, hs, om);
}

template <typename Real>
__device__ __forceinline__ int het_coarse_end(const HetLevel<Real> &L, int ic, Real qc)
{
    const int c = ic + (int)Arith<Real>::min_(qc, (Real)(4 * L.n + 4));
    const int k = L.divM(c);
    return L.M * (k + 1);
}

template <typename Real>
__device__ __forceinline__ bool het_fine_done(const HetPairState<Real> &st, const HetLevel<Real> &L)
{
    return !(st.qf < (Real)(L.n - st.i_f));
}

template <typename Real>
__device__ __forceinline__ bool het_coarse_done(const HetPairState<Real> &st, const HetLevel<Real> &L)
{
    return !(st.qc < (Real)(L.n - st.ic));
}

template <typename Real>
__device__ __forceinline__ void het_keep_output(HetPairState<Real> &st, const HetLevel<Real> &L)
{
    if (!st.have_out && het_fine_done(st, L)) {
        st.have_out = true;
        st.xo = st.xf;
        st.vo = st.vf;
        st.io = st.i_f;
    }
}

// Alg. 1 / Alg. 2 initialisation values of pair p: v_0 = nu_0 (mu = 0,
// sigma = 1), E_0 and its flight from x_0 (eq. intinv), shared by both paths.
template <typename Real, int RECIPE>
__device__ __forceinline__ void het_start_values(Real &v0, Real &e0, Real &q0, unsigned long long p,
                                                 const HetLevel<Real> &L, const PhiloxKeys &keys)
{
    const Draw<Real> d0 = draw_r<Real, RECIPE>(0u, (uint32_t)p, L.word2 ^ (uint32_t)(p >> 32),
                                               L.request, keys);
    v0 = d0.nu;
    e0 = d0.E;
    q0 = L.bg.flight(L.x0, v0, e0);
}

// The state of pair p at t = 0 from its initialisation values; returns true
// if there is nothing to do (no collision of either path before T).
template <typename Real>
__device__ __forceinline__ bool het_pair_init(HetPairState<Real> &st, unsigned long long p, Real v0,
                                              Real e0, Real q0, const HetLevel<Real> &L, bool coupled)
{
    st.pair_lo = (uint32_t)p;
    st.word2 = L.word2 ^ (uint32_t)(p >> 32);
    st.xf = L.x0;
    st.vf = v0;
    st.Ef = e0;
    st.qf = q0;
    st.i_f = 0;
    st.k = 0;
    st.evc = 0;
    st.have_out = false;
    st.xc = st.xf;
    st.vc = st.vf;
    st.qc = st.qf;
    st.ic = 0;
    st.num = Real(0);
    st.den = Real(0);
    st.fresh = true;
    het_keep_output(st, L);
    return het_fine_done(st, L) && (!coupled || het_coarse_done(st, L));
}

// Alg. 1 / Alg. 2 initialisation; returns true if there is nothing to do.
template <typename Real, int RECIPE>
__device__ __forceinline__ bool het_pair_start(HetPairState<Real> &st, unsigned long long p,
                                               const HetLevel<Real> &L, const PhiloxKeys &keys,
                                               bool coupled)
{
    Real v0, e0, q0;
    het_start_values<Real, RECIPE>(v0, e0, q0, p, L, keys);
    return het_pair_init(st, p, v0, e0, q0, L, coupled);
}

// One fine KD step, the window terms and, when the window closes, the
// coarse KD step.  Returns true when the pair is done.
template <typename Real, int RECIPE>
__device__ __forceinline__ bool het_pair_event(HetPairState<Real> &st, const HetLevel<Real> &L,
                                               const PhiloxKeys &keys, bool coupled)
{
    typedef Arith<Real> A;
    const HetBg<Real> &bg = L.bg;
    const Draw<Real> d = draw_r<Real, RECIPE>(st.k + 1u, st.pair_lo, st.word2, L.request, keys);
    // the coarse step end of the coarse collision (the window's bound), from
    // the state before this event
    const int coarse_end = coupled ? het_coarse_end(L, st.ic, st.qc) : 0;
    // fine KD step (Alg. 1) with the stand-in coefficients at the collision point
    const int sq = (int)A::min_(st.qf, (Real)(4 * L.n + 4));
    const Real theta = bg.dt * ((Real)(sq + 1) - st.qf);
    const Real xcol = st.xf + st.vf * (st.qf * bg.dt);
    const Real Rloc = bg.R(xcol);
    const Real v1 = d.nu;
    Real a, dd, hs, om;
    het_kd<Real>(Rloc, theta, v1, a, dd, hs, om);
    st.xf = xcol + (a + dd * d.chi);
    st.i_f = min(st.i_f + sq + 1, 4 * L.n + 4);                   // capped past T (reading H3)
    st.vf = v1;
    st.Ef = d.E;
    st.qf = bg.flight(st.xf, st.vf, d.E);
    ++st.k;
    het_keep_output(st, L);
    if (!coupled) return het_fine_done(st, L);

    // Sec. 3.2 aggregation: beta of this phase (rate Rloc), then alpha of
    // the new phase if the window goes on
    const Real invR = Arith<Real>::div_(Real(1), Rloc);
    const Real hp = hs < Real(1) ? hs * hs * A::h_series(hs) : A::exp_(-hs) + hs - Real(1);
    const Real beta = A::sqrt_pos_(Real(2) * hp) * invR;          // eq. weights-beta, sigma = 1
    if (st.fresh) {
        st.chi_first = d.chi;
        st.fresh = false;
    }
    st.num += beta * d.chi;
    st.den += beta * beta;
    const Real zeta = om * invR;                                  // zeta of this phase
    const int fc = st.i_f + (int)A::min_(st.qf, (Real)(4 * L.n + 4));
    const bool closes = fc + 1 > coarse_end;                      // the until-test of Alg. 2
    if (!closes) {
        if (het_coarse_done(st, L) && het_fine_done(st, L)) return true;
        const Real alpha = st.qf * bg.dt + zeta;                  // sigma (tau + zeta)
        st.num += alpha * d.nu;
        st.den += alpha * alpha;
        return false;
    }
    if (!het_coarse_done(st, L)) {
        // eq. nu-update, eq. epsilon-update, eq. chi-update
        const Real nu_t = d.nu;
        const Real E_t = st.Ef - bg.depth(st.xf, st.vf, (Real)(coarse_end - st.i_f));
        const Real chi_t = st.den > Real(0) ? st.num * A::rsqrt_(st.den) : st.chi_first;
        // coarse KD step at step width M
        const Real thc = bg.dt * ((Real)(coarse_end - st.ic) - st.qc);
        const Real xcc = st.xc + st.vc * (st.qc * bg.dt);
        Real ac, dc, hsc, omc;
        het_kd<Real>(bg.R(xcc), thc, nu_t, ac, dc, hsc, omc);
        st.xc = xcc + (ac + dc * chi_t);
        st.ic = min(coarse_end, 4 * L.n + 4);
        st.vc = nu_t;
        st.qc = bg.flight(st.xc, st.vc, E_t);
        ++st.evc;
    }
    st.num = Real(0);
    st.den = Real(0);
    st.fresh = true;
    return het_coarse_done(st, L) && het_fine_done(st, L);
}

// Final kinetic moves to T: the fine path from its kept output state.
template <typename Real>
__device__ __forceinline__ void het_pair_drift(HetPairState<Real> &st, const HetLevel<Real> &L, bool coupled)
{
    Real x = st.have_out ? st.xo : st.xf;
    const Real v = st.have_out ? st.vo : st.vf;
    const int i = st.have_out ? st.io : st.i_f;
    if (i < L.n) x = x + v * ((Real)(L.n - i) * L.bg.dt);
    st.xf = x;
    if (coupled && st.ic < L.n) st.xc = st.xc + st.vc * ((Real)(L.n - st.ic) * L.bg.dt);
}

}  // namespace mlkd
