// mlkd_warp_pair.cuh -- one correlated pair advanced by a whole warp, 32 fine
// events per step (the event-parallel form for pairs with long serial chains).
//
// A pair of a deep level in the diffusive regime makes up to 12 288 KD events,
// one after another; run by one lane, its chain sets the length of a round.
// Everything expensive in an event depends only on the event's own draws and
// on the previous event's flight: the Philox block, the variate transforms,
// theta, the KD coefficients of eqs. advection/diffusion and the aggregation
// weights of Sec. 3.2.  The sequential parts are integer or additive:
//
//   * the fine time index is a prefix sum of the step counts floor(q) + 1
//     (eq. time-update in step units);
//   * an event is taken while the previous collision lies before T, so the
//     events of a step that happen form a prefix of the warp;
//   * the coarse window test (Sec. 3.1) is local: the collision after event j
//     lies at or past the end of the current coarse step exactly when its
//     coarse step index K = floor(floor(c)/M) differs from that of the
//     collision before it (the coarse step end is always M (K + 1) of the
//     last triggering collision);
//   * the window sums of eq. chi-update are a segmented scan whose segments
//     end at those triggers; the position updates are sums.
//
// So lane j takes event k + 1 + j of the pair: every lane draws and computes
// its event, the warp scans the step counts, finds the triggers and the
// window sums, the triggering lanes take their coarse KD steps (each from the
// coarse state its previous trigger left), and the position increments are
// summed.  Lanes past the pair's last event compute and discard.  The result
// equals the one-lane result up to the order of the FP sums of the positions
// and window terms; every decision (event counts, windows, coarse steps) is
// the same, because it is made in the same arithmetic from the same values.
#pragma once

#include "mlkd_pair.cuh"

namespace mlkd {

template <typename Real>
__device__ __forceinline__ Real warp_sum(Real v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFullMask, v, off);
    return v;
}

// Advances the pair in st (the same value in every lane) by up to 32 fine
// events; returns true (in every lane) when the pair has reached T.
template <typename Real, int RECIPE>
__device__ __forceinline__ bool warp_pair_step(PairState<Real> &st, const LevelCtx<Real> &L,
                                               const PhiloxKeys &keys, bool coupled, int lane)
{
    typedef Arith<Real> A;
    const Background<Real> &bg = L.bg;
    const Draw<Real> d = draw_r<Real, RECIPE>(st.k + 1u + (uint32_t)lane, st.pair_lo, st.word2,
                                              L.request, keys);
    const Real qn = d.E * bg.inv_Rdt;                          // flight after this event
    const Real dv = bg.sigma * d.nu;                           // v_{k+1} - mu
    const Real v1 = bg.mu + dv;
    Real qp = __shfl_up_sync(kFullMask, qn, 1);                // flight before this event
    Real vp = __shfl_up_sync(kFullMask, v1, 1);
    if (lane == 0) {
        qp = st.qf;
        vp = st.vf;
    }
    // step count floor(q) + 1, its prefix sum saturated at n + 1 (only
    // events with an index below n are ever taken)
    const int n = L.n;
    const Real qpc = A::min_(qp, (Real)n);
    const int sq = (int)qpc;
    // In the diffusive regime every flight is shorter than a fine step
    // (R dt >> 1): each event then advances one step, the prefix sum is the
    // lane index, and a coarse window holds at most M events.  The scans
    // below take that shortcut when it holds for the whole step; their
    // results are the same values either way.
    const bool one_step = __all_sync(kFullMask, qp < Real(1) && qn < Real(1));
    int ia = sq + 1;                                           // inclusive prefix -> index after
    if (one_step) {
        ia = lane + 1;
    } else {
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int up = __shfl_up_sync(kFullMask, ia, off);
            if (lane >= off) ia = min(ia + up, n + 1);
        }
    }
    ia = min(st.i_f + ia, n + 1);
    const int ib = ia - (sq + 1);                              // index before this event
    const bool valid = qp < (Real)(n - ib);                    // previous collision before T
    const unsigned vmask = __ballot_sync(kFullMask, valid);
    const int nvalid = __popc(vmask);                          // a prefix of the lanes
    const int last = nvalid - 1;

    const Real theta = bg.dt * ((Real)(sq + 1) - qp);          // eq. diffusive-time
    Real a, dd, hs, om;
    bg.kd_coeffs(theta, dv, a, dd, hs, om);
    const Real dx = valid ? vp * (qp * bg.dt) + (a + dd * d.chi) : Real(0);   // eq. position-update
    st.xf = st.xf + warp_sum(dx);

    bool done;
    {
        const Real ql = __shfl_sync(kFullMask, qn, last);
        const Real vl = __shfl_sync(kFullMask, v1, last);
        const int il = __shfl_sync(kFullMask, ia, last);
        done = !(ql < (Real)(n - il));
        if (coupled) {
            // ---- coarse window: triggers, window sums, coarse steps ----
            const int qnc = (int)A::min_(qn, (Real)n);
            // floor of the collision after, clamped at n: any collision at or
            // after T lies past the coarse step of the one before it (n is a
            // multiple of M), so the clamp changes no trigger
            const int cfl = ia + min(qnc, n - min(ia, n));
            const int Kn = L.divM(cfl);
            int Kp = __shfl_up_sync(kFullMask, Kn, 1);
            if (lane == 0) Kp = L.divM(st.Ec) - 1;             // coarse step of the carried collision
            const bool trig = valid && Kn != Kp;
            const unsigned tmask = __ballot_sync(kFullMask, trig);
            const Real bh2 = valid ? bg.beta_hat_sq(hs) : Real(0);
            Real cn = valid ? A::sqrt_pos_(bh2) * d.chi : Real(0);
            Real cd = bh2;
            if (valid && !trig) {
                const Real ah = qn * bg.Rdt + om;              // R tau' = R tau + R zeta
                cn += ah * d.nu;
                cd += ah * ah;
            }
            // segmented inclusive scan; a window starts after each trigger.
            // With one step per event a window spans at most M lanes, and
            // the scan is complete after the offsets below M.
            bool head = lane == 0 || ((tmask >> (lane - 1)) & 1u);
            if (lane == 0) {
                cn += st.num;
                cd += st.den;
            }
            const int span = one_step && L.M < 32 ? L.M : 32;
            for (int off = 1; off < span; off <<= 1) {
                const Real nu_ = __shfl_up_sync(kFullMask, cn, off);
                const Real du_ = __shfl_up_sync(kFullMask, cd, off);
                const int hu = __shfl_up_sync(kFullMask, (int)head, off);
                if (lane >= off && !head) {
                    cn += nu_;
                    cd += du_;
                    head = head || hu;
                }
            }
            // the trigger before this lane (or the carried coarse state)
            const unsigned below = tmask & ((1u << lane) - 1u);
            const int p = below ? 31 - __clz(below) : -1;
            const int src = p >= 0 ? p : 0;
            const int ecp = L.M * (Kp + 1);                    // coarse step end in force
            // post-trigger coarse state of each lane (used from its trigger lanes)
            const Real qc_post = qn - (Real)(ecp - ia);
            const int ic_from = __shfl_sync(kFullMask, ecp, src);      // ic after trigger p
            const Real qc_from = __shfl_sync(kFullMask, qc_post, src);
            const Real vc_from = __shfl_sync(kFullMask, v1, src);
            const int ic_pre = p >= 0 ? ic_from : st.ic;
            const Real qc_pre = p >= 0 ? qc_from : st.qc;
            const Real vc_pre = p >= 0 ? vc_from : st.vc;
            const Real chi_head = __shfl_sync(kFullMask, d.chi, p + 1 < 32 ? p + 1 : 31);
            const Real chi_first = (p < 0 && !st.fresh) ? st.chi_first : chi_head;
            Real dxc = Real(0);
            if (trig) {
                const Real thc = bg.dt * ((Real)(ecp - ic_pre) - qc_pre);
                Real ac, dc, hsc, omc;
                bg.kd_coeffs(thc, dv, ac, dc, hsc, omc);
                const Real chit = cd > Real(0) ? cn * A::rsqrt_(cd) : chi_first;
                dxc = vc_pre * (qc_pre * bg.dt) + (ac + dc * chit);
            }
            st.xc = st.xc + warp_sum(dxc);
            st.evc += (uint32_t)__popc(tmask);
            // carry out: the coarse state after the last trigger, the open window
            if (tmask) {
                const int t = 31 - __clz(tmask);
                const int ic_t = __shfl_sync(kFullMask, ecp, t);
                const Real qc_t = __shfl_sync(kFullMask, qc_post, t);
                st.ic = ic_t;
                st.qc = qc_t;
                st.vc = __shfl_sync(kFullMask, v1, t);
                if (qc_t < (Real)(n - ic_t)) st.Ec = next_coarse_end(L, ic_t, (int)qc_t);
            }
            const bool trig_last = (tmask >> last) & 1u;
            const Real num_l = __shfl_sync(kFullMask, cn, last);
            const Real den_l = __shfl_sync(kFullMask, cd, last);
            const Real cf_l = __shfl_sync(kFullMask, chi_first, last);
            if (trig_last) {
                st.num = Real(0);
                st.den = Real(0);
                st.fresh = true;
            } else {
                st.num = num_l;
                st.den = den_l;
                st.chi_first = cf_l;
                st.fresh = false;
            }
        }
        st.k += (uint32_t)nvalid;
        st.i_f = il;
        st.qf = ql;
        st.vf = vl;
    }
    return done;
}

}  // namespace mlkd
