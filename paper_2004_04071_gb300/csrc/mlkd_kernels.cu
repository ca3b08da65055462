// mlkd_kernels.cu -- the correlated-pair kernel and its reductions.
//
// One lane simulates one pair at a time: the fine path of Alg. 1 at dt_l and,
// on levels l >= 1, the coarse path at dt_{l-1} = M dt_l built on the fly from
// the fine path's random numbers (Alg. 2 with the mapping of Sec. 3.1 and the
// aggregation of Sec. 3.2).  All pair state lives in registers; the only
// memory traffic is one row of block partial sums, and the histogram flush.
//
// Work distribution: each warp owns a contiguous chunk of pairs; a lane whose
// pair has finished takes the next pair of the chunk (ballot + popc), so lanes
// stay busy although pairs need different numbers of KD events.  The
// assignment depends only on the event counts, so results are reproducible.
#include <cfloat>

#include "mlkd_internal.h"

namespace mlkd {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Per-lane sums of one launch: Y, Y^2, F(x_f), F(x_f)^2, F(x_c), F(x_c)^2.
//   FP64 mode      : all six in FP64.
//   FP32_DY64 mode : Y and Y^2 formed and summed in FP64 from the FP32 state;
//                    the four F moments as compensated FP32 pairs.
//   FP32_COMP mode : all six as compensated FP32 (sum, error) pairs.
// Compensation is an error-free TwoSum per addition.
// ---------------------------------------------------------------------------
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
        const float so = __shfl_down_sync(kFull, s, off);
        const float co = __shfl_down_sync(kFull, c, off);
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
            for (int j = 0; j < 6; ++j) v[j] += __shfl_down_sync(kFull, v[j], off);
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
            sy += __shfl_down_sync(kFull, sy, off);
            sy2 += __shfl_down_sync(kFull, sy2, off);
#pragma unroll
            for (int j = 0; j < 4; ++j) q[j].shfl_merge(off);
        }
    }
    __device__ double value(int j) const { return j == 0 ? sy : j == 1 ? sy2 : q[j - 2].value(); }
};

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

// Histogram bin of x: floor((x - lo)/h) inside [lo, hi), else -1; periodic
// positions are first wrapped into [0, 1).  FP64 state uses the division in
// FP64; FP32 state decides its bins in FP32.
__device__ __forceinline__ int bin_of(double x, const PairLaunch &P)
{
    if (P.periodic) x = x - floor(x);
    if (!(x >= P.lo && x < P.hi)) return -1;
    const int b = (int)floor((x - P.lo) / P.h);
    return b < P.nbins ? b : P.nbins - 1;
}

struct BinsF {
    float lo, hi, inv_h;
    int nbins;
    bool periodic;
    __device__ int operator()(float x) const {
        if (periodic) x = x - floorf(x);
        if (!(x >= lo && x < hi)) return -1;
        const int b = (int)floorf((x - lo) * inv_h);
        return b < nbins ? b : nbins - 1;
    }
};

__device__ __forceinline__ int bin_any(double x, const PairLaunch &P, const BinsF &) { return bin_of(x, P); }
__device__ __forceinline__ int bin_any(float x, const PairLaunch &, const BinsF &bf) { return bf(x); }

}  // namespace

template <typename Real> __device__ __forceinline__ const BgParams<Real> &level_params(const PairLaunch &P);
template <> __device__ __forceinline__ const BgParams<float> &level_params<float>(const PairLaunch &P) { return P.bf; }
template <> __device__ __forceinline__ const BgParams<double> &level_params<double>(const PairLaunch &P) { return P.bd; }

// Blocks per SM the register allocation must allow: FP32 state fits 64
// registers (8 blocks of 128 threads); the FP64 form is bound by the FP64 pipe.
template <typename Real> struct MinBlocks { static constexpr int value = 8; };
template <> struct MinBlocks<double> { static constexpr int value = 1; };

template <typename Real, int MODE, bool COUPLED>
__global__ void __launch_bounds__(kThreads, MinBlocks<Real>::value)
pair_kernel(const __grid_constant__ PairLaunch P)
{
    typedef Arith<Real> A;
    extern __shared__ unsigned int s_hist[];          // [3][nbins]
    __shared__ double s_red[kWarpsPerBlock][kPartialWords];

    const int nbins = P.nbins;
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x) s_hist[i] = 0u;
    if (nbins > 0) __syncthreads();

    const BgParams<Real> &bp = level_params<Real>(P);
    Background<Real> bg;
    bg.R = bp.R;
    bg.invR = bp.invR;
    bg.mu = bp.mu;
    bg.sigma = bp.sigma;
    bg.two_c2 = bp.two_c2;
    bg.dt = bp.dt;
    bg.Rdt = bp.Rdt;
    bg.inv_Rdt = bp.inv_Rdt;

    const int n = P.n;
    const int M = P.M;
    const int lane = threadIdx.x & 31;
    const unsigned long long warp_id =
        (unsigned long long)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const unsigned long long end_all = P.first_pair + P.n_pairs;
    unsigned long long w_begin = P.first_pair + warp_id * P.pairs_per_warp;
    if (w_begin > end_all) w_begin = end_all;
    unsigned long long w_end = w_begin + P.pairs_per_warp;
    if (w_end > end_all) w_end = end_all;
    unsigned long long next = w_begin;                 // warp-uniform

    // pair state (registers)
    bool active = false;
    unsigned long long pair = 0;
    uint32_t pair_lo = 0, word2 = 0;
    Real xf = 0, vf = 0, qf = 0, xc = 0, vc = 0, qc = 0, num = 0, den = 0, chi_first = 0;
    int i_f = 0, ic = 0, Ec = 0;
    uint32_t k = 0, evc = 0;
    bool fresh = true;

    PairSums<MODE> mom;
    mom.zero();
    BinsF binsf;
    binsf.lo = P.bf.lo;
    binsf.hi = P.bf.hi;
    binsf.inv_h = P.bf.inv_h;
    binsf.nbins = P.nbins;
    binsf.periodic = P.periodic != 0;
    unsigned long long ev_f_sum = 0, ev_c_sum = 0;

    // Alg. 1 final drift, QoI, sums and histogram of the finished pair.
    auto finish_pair = [&]() {
        if (i_f < n) xf = xf + vf * ((Real)(n - i_f) * bg.dt);
        if (COUPLED && ic < n) xc = xc + vc * ((Real)(n - ic) * bg.dt);
        add_pair(mom, xf, xc, COUPLED, P.periodic != 0);
        ev_f_sum += k;
        ev_c_sum += evc;
        if (nbins > 0) {
            const int bf = bin_any(xf, P, binsf);
            if (bf >= 0) atomicAdd(&s_hist[bf], 1u);
            if (COUPLED) {
                const int bc = bin_any(xc, P, binsf);
                if (bc >= 0) atomicAdd(&s_hist[nbins + bc], 1u);
                if (bc >= 0 && bc == bf) atomicAdd(&s_hist[2 * nbins + bf], 1u);
            }
        }
        if (P.dbg_xf) {
            const unsigned long long j = pair - P.first_pair;
            P.dbg_xf[j] = (double)xf;
            if (P.dbg_xc) P.dbg_xc[j] = COUPLED ? (double)xc : 0.0;
            if (P.dbg_kf) P.dbg_kf[j] = (int32_t)k;
            if (P.dbg_kc) P.dbg_kc[j] = (int32_t)evc;
        }
        active = false;
    };

    // Alg. 1 / Alg. 2 initialisation: nu_0, E_0 (shared by both paths), x_0.
    auto start_pair = [&](unsigned long long p) {
        pair = p;
        pair_lo = (uint32_t)p;
        word2 = P.word2 ^ (uint32_t)(p >> 32);
        const Draw<Real> d0 = draw<Real>(0u, pair_lo, word2, P.request, P.keys);
        const Real x0 = P.init ? cosine_inverse<Real>(d0.u4) : Real(0);
        xf = x0;
        vf = bg.mu + bg.sigma * d0.nu;
        qf = d0.E * bg.inv_Rdt;
        i_f = 0;
        k = 0;
        if (COUPLED) {
            xc = x0;
            vc = vf;
            qc = qf;
            ic = 0;
            evc = 0;
            num = Real(0);
            den = Real(0);
            fresh = true;
            if (qf < (Real)n) Ec = M * ((int)qf / M + 1);
        }
        active = true;
        if (!(qf < (Real)n)) finish_pair();            // no collision before T
    };

    for (;;) {
        // refill idle lanes from the warp's chunk
        const unsigned idle = __ballot_sync(kFull, !active);
        if (idle != 0u && next < w_end) {
            const unsigned rank = __popc(idle & ((1u << lane) - 1u));
            const unsigned long long cand = next + rank;
            if (!active && cand < w_end) start_pair(cand);
            next += __popc(idle);
            if (next > w_end) next = w_end;
        }
        if (!__any_sync(kFull, active)) {
            if (next >= w_end) break;
            continue;
        }
        if (!active) continue;

        // ---- one fine KD event (Alg. 1 KineticDiffusionStep) ----
        const Draw<Real> d = draw<Real>(k + 1u, pair_lo, word2, P.request, P.keys);
        const int sq = (int)qf;                                   // floor: qf >= 0
        const Real theta = bg.dt * ((Real)(sq + 1) - qf);         // eq. diffusive-time
        const Real dv = bg.sigma * d.nu;                          // v_{k+1} - mu
        const Real v1 = bg.mu + dv;
        Real a, dd, hs, om;
        bg.kd_coeffs(theta, dv, a, dd, hs, om);
        xf = xf + vf * (qf * bg.dt) + (a + dd * d.chi);           // eq. position-update
        i_f += sq + 1;                                            // eq. time-update
        vf = v1;
        qf = d.E * bg.inv_Rdt;                                    // eq. intinv (homogeneous)
        ++k;

        if (COUPLED) {
            // Sec. 3.2 aggregation, streamed: this phase's chi with beta, and the
            // new phase's nu with alpha if it collides inside the coarse step.
            const Real bh2 = bg.beta_hat_sq(hs);
            if (fresh) { chi_first = d.chi; fresh = false; }
            num += A::sqrt_(bh2) * d.chi;
            den += bh2;
            if (qf < (Real)(Ec - i_f)) {
                const Real ah = qf * bg.Rdt + om;                 // R tau' = R tau + R zeta
                num += ah * d.nu;
                den += ah * ah;
            } else {
                // coarse KD step with nu~ = nu_{kappa}, chi~ (eq. chi-update) and,
                // after it, the coarse flight tau~ = fine collision - E_c
                // (homogeneous eq. epsilon-update), carried in fine units.
                const Real thc = bg.dt * ((Real)(Ec - ic) - qc);
                Real ac, dc, hsc, omc;
                bg.kd_coeffs(thc, dv, ac, dc, hsc, omc);
                const Real chit = den > Real(0) ? num * A::rsqrt_(den) : chi_first;
                xc = xc + vc * (qc * bg.dt) + (ac + dc * chit);
                qc = qf - (Real)(Ec - i_f);
                ic = Ec;
                vc = v1;
                ++evc;
                if (qc < (Real)(n - ic)) Ec = M * ((ic + (int)qc) / M + 1);
                num = Real(0);
                den = Real(0);
                fresh = true;
            }
        }
        if (!(qf < (Real)(n - i_f))) finish_pair();
    }

    // ---- block reduction of the sums (fixed order) ----
    mom.warp_reduce();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ev_f_sum += __shfl_down_sync(kFull, ev_f_sum, off);
        ev_c_sum += __shfl_down_sync(kFull, ev_c_sum, off);
    }
    const int warp = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < 6; ++j) s_red[warp][j] = mom.value(j);
        s_red[warp][6] = (double)ev_f_sum;
        s_red[warp][7] = (double)ev_c_sum;
    }
    __syncthreads();
    if (threadIdx.x < kPartialWords) {
        double acc = 0.0;
#pragma unroll
        for (int w = 0; w < kWarpsPerBlock; ++w) acc += s_red[w][threadIdx.x];
        P.partials[(size_t)blockIdx.x * kPartialWords + threadIdx.x] = acc;
    }
    if (nbins > 0 && P.hist) {
        for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x) {
            const unsigned int c = s_hist[i];
            if (c) atomicAdd(&P.hist[i], (unsigned long long)c);
        }
    }
}

// ---------------------------------------------------------------------------
// Fixed-order sum of the block partials.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
finalize_kernel(const double *__restrict__ partials, int nblocks, long long n_pairs,
                DevLevelStats *out, DevLevelStats *acc)
{
    __shared__ double sh[kPartialWords][256];
    const int t = threadIdx.x;
    double v[kPartialWords];
#pragma unroll
    for (int j = 0; j < kPartialWords; ++j) v[j] = 0.0;
    for (int b = t; b < nblocks; b += 256)
#pragma unroll
        for (int j = 0; j < kPartialWords; ++j) v[j] += partials[(size_t)b * kPartialWords + j];
#pragma unroll
    for (int j = 0; j < kPartialWords; ++j) sh[j][t] = v[j];
    __syncthreads();
    for (int stride = 128; stride > 0; stride >>= 1) {
        if (t < stride)
#pragma unroll
            for (int j = 0; j < kPartialWords; ++j) sh[j][t] += sh[j][t + stride];
        __syncthreads();
    }
    if (t == 0) {
        DevLevelStats s;
        s.n = n_pairs;
        s.sy = sh[0][0];
        s.sy2 = sh[1][0];
        s.sqf = sh[2][0];
        s.sqf2 = sh[3][0];
        s.sqc = sh[4][0];
        s.sqc2 = sh[5][0];
        s.events_f = (unsigned long long)llrint(sh[6][0]);
        s.events_c = (unsigned long long)llrint(sh[7][0]);
        if (out) *out = s;
        if (acc) {
            acc->n += s.n;
            acc->sy += s.sy;
            acc->sy2 += s.sy2;
            acc->sqf += s.sqf;
            acc->sqf2 += s.sqf2;
            acc->sqc += s.sqc;
            acc->sqc2 += s.sqc2;
            acc->events_f += s.events_f;
            acc->events_c += s.events_c;
        }
    }
}

__global__ void hist_accumulate_kernel(const unsigned long long *h, unsigned long long *acc,
                                       int count)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        acc[i] += h[i];
}

// ---------------------------------------------------------------------------
// Sample-count controller in FP64 (eqs. mse, Nopt1, Noptj): one block.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
controller_kernel(const DevLevelStats *acc, const unsigned long long *hist_acc, int n_levels,
                  int nbins, double h, int density_qoi, double tol, DevControl *out)
{
    __shared__ double s_var[16];
    __shared__ double s_max[256];
    const int t = threadIdx.x;
    for (int l = 0; l < n_levels; ++l) {
        const double n = (double)acc[l].n;
        double v = 0.0;
        if (density_qoi && nbins > 0) {
            double m = 0.0;
            for (int b = t; b < nbins; b += 256) {
                const unsigned long long *H = hist_acc + (size_t)l * 3 * nbins;
                const double sy = (double)H[b] - (double)H[nbins + b];
                const double sy2 = (double)H[b] + (double)H[nbins + b] - 2.0 * (double)H[2 * nbins + b];
                const double vb = n >= 2.0 ? (sy2 - sy * sy / n) / (n - 1.0) : 0.0;
                m = fmax(m, vb);
            }
            s_max[t] = m;
            __syncthreads();
            for (int stride = 128; stride > 0; stride >>= 1) {
                if (t < stride) s_max[t] = fmax(s_max[t], s_max[t + stride]);
                __syncthreads();
            }
            v = s_max[0] / (h * h);
            __syncthreads();
        } else if (n >= 2.0) {
            v = (acc[l].sy2 - acc[l].sy * acc[l].sy / n) / (n - 1.0);
        }
        if (t == 0) s_var[l] = v > 0.0 ? v : 0.0;
    }
    __syncthreads();
    if (t == 0) {
        double est = 0.0, var = 0.0, total = 0.0;
        for (int l = 0; l < n_levels; ++l) {
            const double n = (double)acc[l].n;
            const double c = n > 0.0 ? (double)(acc[l].events_f + acc[l].events_c) / n : 0.0;
            out->var_level[l] = s_var[l];
            out->cost_level[l] = c;
            if (n > 0.0) {
                est += acc[l].sy / n;
                var += s_var[l] / n;
            }
            total += sqrt(s_var[l] * c);
        }
        for (int l = 0; l < n_levels; ++l) {
            const double v = s_var[l], c = out->cost_level[l];
            long long target = 0;
            if (v > 0.0 && c > 0.0 && tol > 0.0)
                target = (long long)ceil(2.0 / (tol * tol) * sqrt(v / c) * total);
            out->target[l] = target;
        }
        out->estimate = est;
        out->variance = var;
    }
}

// ---------------------------------------------------------------------------
// Host-side launch helpers.
// ---------------------------------------------------------------------------
namespace {

typedef void (*PairKernelFn)(const PairLaunch);

PairKernelFn pick(int mode, bool coupled)
{
    switch (mode) {
    case kModeFP64:
        return coupled ? pair_kernel<double, kModeFP64, true> : pair_kernel<double, kModeFP64, false>;
    case kModeFP32DY64:
        return coupled ? pair_kernel<float, kModeFP32DY64, true>
                       : pair_kernel<float, kModeFP32DY64, false>;
    default:
        return coupled ? pair_kernel<float, kModeFP32Comp, true>
                       : pair_kernel<float, kModeFP32Comp, false>;
    }
}

}  // namespace

cudaError_t pair_kernel_info(int mode, bool coupled, int nbins, KernelInfo *out)
{
    int blocks = 0;
    const size_t smem = (size_t)3 * nbins * sizeof(unsigned int);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &blocks, (const void *)pick(mode, coupled), kThreads, smem);
    out->blocks_per_sm = blocks;
    return e;
}

cudaError_t launch_pair_kernel(int mode, bool coupled, const PairLaunch &p, int grid,
                               cudaStream_t stream)
{
    const size_t smem = (size_t)3 * p.nbins * sizeof(unsigned int);
    pick(mode, coupled)<<<grid, kThreads, smem, stream>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double *partials, int nblocks, long long n_pairs,
                            DevLevelStats *out, DevLevelStats *acc, cudaStream_t stream)
{
    finalize_kernel<<<1, 256, 0, stream>>>(partials, nblocks, n_pairs, out, acc);
    return cudaGetLastError();
}

cudaError_t launch_controller(const DevLevelStats *acc, const unsigned long long *hist_acc,
                              int n_levels, int nbins, double h, int density_qoi, double tol,
                              DevControl *out, cudaStream_t stream)
{
    controller_kernel<<<1, 256, 0, stream>>>(acc, hist_acc, n_levels, nbins, h, density_qoi, tol,
                                             out);
    return cudaGetLastError();
}

cudaError_t launch_hist_accumulate(const unsigned long long *hist, unsigned long long *acc,
                                   int count, cudaStream_t stream)
{
    if (count <= 0) return cudaSuccess;
    hist_accumulate_kernel<<<(count + 255) / 256, 256, 0, stream>>>(hist, acc, count);
    return cudaGetLastError();
}

}  // namespace mlkd
