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

#include "mlkd_hetero.cuh"
#include "mlkd_internal.h"
#include "mlkd_pair.cuh"

namespace mlkd {

template <typename Real> __device__ __forceinline__ const BgParams<Real> &level_params(const PairLaunch &P);
template <> __device__ __forceinline__ const BgParams<float> &level_params<float>(const PairLaunch &P) { return P.bf; }
template <> __device__ __forceinline__ const BgParams<double> &level_params<double>(const PairLaunch &P) { return P.bd; }

// Blocks per SM the register allocation must allow: FP32 state of the
// homogeneous background fits 64 registers (8 blocks of 128 threads); the
// heterogeneous pair state does not, and at 64 registers its kernel kept the
// FP64 pipe 21-83 % busy (ncu) without a line of FP64 arithmetic, so it gets
// 128 (4 blocks); the FP64 form is bound by the FP64 pipe.
template <typename Real, int PHYS> struct MinBlocks { static constexpr int value = PHYS == 1 ? 4 : 8; };
template <int PHYS> struct MinBlocks<double, PHYS> { static constexpr int value = 1; };

// Pair state of the two physics: the homogeneous background (PHYS 0) and the
// heterogeneous backgrounds B1/B2 of Sec. 5 (PHYS 1).
template <typename Real, int PHYS> struct PhysState { typedef PairState<Real> type; };
template <typename Real> struct PhysState<Real, 1> { typedef HetPairState<Real> type; };

template <typename Real, int MODE, bool COUPLED, int PHYS>
__global__ void __launch_bounds__(kThreads, (MinBlocks<Real, PHYS>::value))
pair_kernel(const __grid_constant__ PairLaunch P)
{
    constexpr int CPL = COUPLED ? 1 : 0;
    constexpr int RECIPE = ModeRecipe<MODE>::value;
    extern __shared__ unsigned int s_hist[];          // [3][nbins]
    __shared__ double s_red[kWarpsPerBlock][kPartialWords];

    const int nbins = P.nbins;
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x) s_hist[i] = 0u;
    if (nbins > 0) __syncthreads();

    const BgParams<Real> &bp = level_params<Real>(P);
    LevelCtx<Real> L;
    L.bg.R = bp.R;
    L.bg.invR = bp.invR;
    L.bg.mu = bp.mu;
    L.bg.sigma = bp.sigma;
    L.bg.two_c2 = bp.two_c2;
    L.bg.dt = bp.dt;
    L.bg.Rdt = bp.Rdt;
    L.bg.inv_Rdt = bp.inv_Rdt;
    L.n = P.n;
    L.M = P.M;
    L.divM.init(P.M);
    L.init = P.init == 1 ? 1 : 0;          // a point start is set after pair_start
    L.word2 = P.word2;
    L.request = P.request;
    HetLevel<Real> H;
    if constexpr (PHYS == 1) {
        H.bg.b = (Real)P.bg_b;
        H.bg.a_left = (Real)P.bg_a_left;
        H.bg.a_right = (Real)P.bg_a_right;
        H.bg.dt = bp.dt;
        H.n = P.n;
        H.M = P.M;
        H.divM = L.divM;
        H.x0 = (Real)P.x0;
        H.word2 = P.word2;
        H.request = P.request;
    }

    Bins bins;
    bins.lo = P.lo;
    bins.hi = P.hi;
    bins.h = P.h;
    bins.lo_f = P.bf.lo;
    bins.hi_f = P.bf.hi;
    bins.inv_h_f = P.bf.inv_h;
    bins.nbins = nbins;
    bins.periodic = P.periodic != 0;

    const int lane = threadIdx.x & 31;
    const unsigned long long warp_id =
        (unsigned long long)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    const unsigned long long end_all = P.first_pair + P.n_pairs;
    unsigned long long w_begin = P.first_pair + warp_id * P.pairs_per_warp;
    if (w_begin > end_all) w_begin = end_all;
    unsigned long long w_end = w_begin + P.pairs_per_warp;
    if (w_end > end_all) w_end = end_all;
    unsigned long long next = w_begin;                 // warp-uniform

    bool active = false;        // the lane's pair has events left
    bool done = false;          // the lane holds a finished pair not yet summed
    unsigned long long pair = 0;
    typename PhysState<Real, PHYS>::type st;
    st.fresh = true;
    PairSums<MODE> mom;
    mom.zero();
    unsigned long long ev_f_sum = 0, ev_c_sum = 0;

    // QoI, sums and histogram of the finished pair.
    auto finish_pair = [&]() {
        if constexpr (PHYS == 1)
            het_pair_drift<Real>(st, H, COUPLED);
        else
            pair_drift<Real, CPL>(st, L, COUPLED);
        add_pair_fk(mom, st.xf, st.xc, COUPLED, P.fkind);
        ev_f_sum += st.k;
        ev_c_sum += st.evc;
        if (nbins > 0) {
            int bf = bins(st.xf);
            if (!MLKD_DCHECK(bf < nbins)) bf = -1;
            if (bf >= 0) atomicAdd(&s_hist[bf], 1u);
            if (COUPLED) {
                int bc = bins(st.xc);
                if (!MLKD_DCHECK(bc < nbins)) bc = -1;
                if (bc >= 0) atomicAdd(&s_hist[nbins + bc], 1u);
                if (bc >= 0 && bc == bf) atomicAdd(&s_hist[2 * nbins + bf], 1u);
            }
        }
        if (P.dbg_xf && MLKD_DCHECK(pair - P.first_pair < P.n_pairs)) {
            const unsigned long long j = pair - P.first_pair;
            P.dbg_xf[j] = (double)st.xf;
            if (P.dbg_xc) P.dbg_xc[j] = COUPLED ? (double)st.xc : 0.0;
            if (P.dbg_kf) P.dbg_kf[j] = (int32_t)st.k;
            if (P.dbg_kc) P.dbg_kc[j] = (int32_t)st.evc;
        }
        done = false;
    };

    for (;;) {
        // Lanes whose pair reached T stay idle until kRefillMin of them (or
        // the whole warp) can be summed and restarted from the warp's chunk
        // in one pass.
        const unsigned idle = __ballot_sync(kFullMask, !active);
        if (idle != 0u && (__popc(idle) >= kRefillMin || idle == kFullMask)) {
            if (done) finish_pair();
            if (next < w_end) {
                const unsigned rank = __popc(idle & ((1u << lane) - 1u));
                const unsigned long long cand = next + rank;
                if (!active && cand < w_end) {
                    pair = cand;
                    bool none;
                    if constexpr (PHYS == 1) {
                        none = het_pair_start<Real, RECIPE>(st, cand, H, P.keys, COUPLED);
                    } else {
                        none = pair_start<Real, CPL, RECIPE>(st, cand, L, P.keys, COUPLED);
                        if (P.init == 2) {
                            st.xf = (Real)P.x0;
                            st.xc = st.xf;
                        }
                    }
                    if (none)
                        done = true;
                    else
                        active = true;
                }
                next += __popc(idle);
                if (next > w_end) next = w_end;
            }
        }
        if (!__any_sync(kFullMask, active)) {
            if (next >= w_end && !__any_sync(kFullMask, done)) break;
            continue;
        }
        if (active) {
            bool fin;
            if constexpr (PHYS == 1)
                fin = het_pair_event<Real, RECIPE>(st, H, P.keys, COUPLED);
            else
                fin = pair_event<Real, CPL, RECIPE>(st, L, P.keys, COUPLED);
            if (fin) {
                active = false;
                done = true;
            }
        }
    }

    // ---- block reduction of the sums (fixed order) ----
    mom.warp_reduce();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ev_f_sum += __shfl_down_sync(kFullMask, ev_f_sum, off);
        ev_c_sum += __shfl_down_sync(kFullMask, ev_c_sum, off);
    }
    const int warp = threadIdx.x >> 5;
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < 6; ++j) s_red[warp][j] = mom.value(j);
        s_red[warp][6] = (double)ev_f_sum;
        s_red[warp][7] = (double)ev_c_sum;
    }
    __syncthreads();
    if (threadIdx.x < kPartialWords && MLKD_DCHECK(blockIdx.x < (unsigned)P.partial_rows)) {
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

// ---------------------------------------------------------------------------
// Coarse random numbers of each pair (validation of Sec. 5.1): one thread
// per pair runs the same pair_start/pair_event as the pair kernel and
// records the first per_pair coarse steps' (nu~, E~, chi~).
// ---------------------------------------------------------------------------
struct CoarseTrace {
    double *nu, *E, *chi;
    int cap, n;
    template <typename Real> __device__ void coarse(Real a, Real b, Real c)
    {
        if (n < cap) {
            nu[n] = (double)a;
            E[n] = (double)b;
            chi[n] = (double)c;
        }
        ++n;
    }
};

template <typename Real, int MODE>
__global__ void __launch_bounds__(kThreads)
coarse_draws_kernel(const __grid_constant__ PairLaunch P, int per_pair, double *nu, double *E,
                    double *chi, int32_t *count)
{
    const unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.n_pairs) return;
    const BgParams<Real> &bp = level_params<Real>(P);
    LevelCtx<Real> L;
    L.bg.R = bp.R;
    L.bg.invR = bp.invR;
    L.bg.mu = bp.mu;
    L.bg.sigma = bp.sigma;
    L.bg.two_c2 = bp.two_c2;
    L.bg.dt = bp.dt;
    L.bg.Rdt = bp.Rdt;
    L.bg.inv_Rdt = bp.inv_Rdt;
    L.n = P.n;
    L.M = P.M;
    L.divM.init(P.M);
    L.init = P.init;
    L.word2 = P.word2;
    L.request = P.request;
    const size_t base = (size_t)j * (size_t)per_pair;
    CoarseTrace tr{nu + base, E + base, chi + base, per_pair, 0};
    PairState<Real> st;
    st.fresh = true;
    bool done = pair_start<Real, 1, ModeRecipe<MODE>::value>(st, P.first_pair + j, L, P.keys, true);
    // a pair has at most n fine events
    for (int it = 0; !done && it <= P.n; ++it)
        done = pair_event<Real, 1, ModeRecipe<MODE>::value, CoarseTrace>(st, L, P.keys, true, &tr);
    count[j] = tr.n;
}

cudaError_t launch_coarse_draws(int mode, const PairLaunch &p, int per_pair, double *nu, double *E,
                                double *chi, int32_t *count, cudaStream_t stream)
{
    if (p.n_pairs == 0) return cudaSuccess;
    const unsigned long long blocks = (p.n_pairs + kThreads - 1) / kThreads;
    switch (mode) {
    case kModeFP64:
        coarse_draws_kernel<double, kModeFP64><<<(unsigned)blocks, kThreads, 0, stream>>>(p, per_pair, nu, E, chi, count);
        break;
    case kModeFP64U24:
        coarse_draws_kernel<double, kModeFP64U24><<<(unsigned)blocks, kThreads, 0, stream>>>(p, per_pair, nu, E, chi, count);
        break;
    default:
        coarse_draws_kernel<float, kModeFP32Comp><<<(unsigned)blocks, kThreads, 0, stream>>>(p, per_pair, nu, E, chi, count);
        break;
    }
    return cudaGetLastError();
}

// KD coefficients of eqs. advection/diffusion and the aggregation quantities
// exactly as the pair kernels compute them in precision Real, for given
// (theta, v' - mu); the level constants are prepared as for a launch (FP64 on
// the host, rounded once to Real).
template <typename Real>
__global__ void debug_kd_kernel(double R, double mu, double sigma, const double *theta,
                                const double *dv, unsigned long long n, double *a, double *d,
                                double *hs, double *om, double *bh2)
{
    Background<Real> bg;
    bg.R = (Real)R;
    bg.invR = (Real)(1.0 / R);
    bg.mu = (Real)mu;
    bg.sigma = (Real)sigma;
    bg.two_c2 = (Real)(2.0 * sigma * sigma / (R * R));
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        Real ai, di, hsi, omi;
        bg.kd_coeffs((Real)theta[i], (Real)dv[i], ai, di, hsi, omi);
        a[i] = (double)ai;
        d[i] = (double)di;
        hs[i] = (double)hsi;
        om[i] = (double)omi;
        bh2[i] = (double)bg.beta_hat_sq(hsi);
    }
}

cudaError_t launch_debug_kd(int fp64, double R, double mu, double sigma, const double *theta,
                            const double *dv, unsigned long long n, double *a, double *d, double *hs,
                            double *om, double *bh2, cudaStream_t stream)
{
    if (n == 0) return cudaSuccess;
    const unsigned long long blocks = (n + 255) / 256;
    const unsigned g = (unsigned)(blocks < 65536 ? blocks : 65536);
    if (fp64)
        debug_kd_kernel<double><<<g, 256, 0, stream>>>(R, mu, sigma, theta, dv, n, a, d, hs, om, bh2);
    else
        debug_kd_kernel<float><<<g, 256, 0, stream>>>(R, mu, sigma, theta, dv, n, a, d, hs, om, bh2);
    return cudaGetLastError();
}

__global__ void debug_transforms_kernel(const uint32_t *words, unsigned long long n, float *log_u,
                                        float *sn, float *cs)
{
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t w = words[i];
        if (log_u) log_u[i] = log_unit24(w);
        float a, b;
        sincos_2pi_unit24(w, &a, &b);
        if (sn) sn[i] = a;
        if (cs) cs[i] = b;
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
            if (v > 0.0 && c > 0.0 && tol > 0.0) {
                const double tg = ceil(2.0 / (tol * tol) * sqrt(v / c) * total);
                target = tg < 1e15 ? (long long)tg : 1000000000000000LL;
            }
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

template <int PHYS>
PairKernelFn pick_phys(int mode, bool coupled)
{
    switch (mode) {
    case kModeFP64:
        return coupled ? pair_kernel<double, kModeFP64, true, PHYS> : pair_kernel<double, kModeFP64, false, PHYS>;
    case kModeFP32DY64:
        return coupled ? pair_kernel<float, kModeFP32DY64, true, PHYS>
                       : pair_kernel<float, kModeFP32DY64, false, PHYS>;
    case kModeFP64U24:
        return coupled ? pair_kernel<double, kModeFP64U24, true, PHYS>
                       : pair_kernel<double, kModeFP64U24, false, PHYS>;
    default:
        return coupled ? pair_kernel<float, kModeFP32Comp, true, PHYS>
                       : pair_kernel<float, kModeFP32Comp, false, PHYS>;
    }
}

PairKernelFn pick(int mode, bool coupled, int background)
{
    return background ? pick_phys<1>(mode, coupled) : pick_phys<0>(mode, coupled);
}

}  // namespace

cudaError_t pair_kernel_info(int mode, bool coupled, int nbins, KernelInfo *out, int background)
{
    int blocks = 0;
    const size_t smem = (size_t)3 * nbins * sizeof(unsigned int);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &blocks, (const void *)pick(mode, coupled, background), kThreads, smem);
    out->blocks_per_sm = blocks;
    return e;
}

cudaError_t launch_pair_kernel(int mode, bool coupled, const PairLaunch &p, int grid,
                               cudaStream_t stream)
{
    const size_t smem = (size_t)3 * p.nbins * sizeof(unsigned int);
    pick(mode, coupled, p.background)<<<grid, kThreads, smem, stream>>>(p);
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

cudaError_t launch_debug_transforms(const uint32_t *words, unsigned long long n, float *log_u,
                                    float *sn, float *cs, cudaStream_t stream)
{
    if (n == 0) return cudaSuccess;
    const unsigned long long blocks = (n + 255) / 256;
    debug_transforms_kernel<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, stream>>>(words, n, log_u, sn, cs);
    return cudaGetLastError();
}

cudaError_t launch_hist_accumulate(const unsigned long long *hist, unsigned long long *acc,
                                   int count, cudaStream_t stream)
{
    if (count <= 0) return cudaSuccess;
    hist_accumulate_kernel<<<(count + 255) / 256, 256, 0, stream>>>(hist, acc, count);
    return cudaGetLastError();
}

#ifdef MLKD_CHECKS
__global__ void check_selftest_kernel(int n)
{
    // a check that fails on purpose: the index stays clamped, nothing is written
    int i = n;
    if (!MLKD_DCHECK(i < 0)) i = 0;
    (void)i;
}
#endif

cudaError_t launch_check_selftest(cudaStream_t stream)
{
#ifdef MLKD_CHECKS
    check_selftest_kernel<<<1, 32, 0, stream>>>(1);
    return cudaGetLastError();
#else
    (void)stream;
    return cudaErrorNotSupported;
#endif
}

cudaError_t check_word_kernels(unsigned *line)
{
    *line = 0u;
#ifdef MLKD_CHECKS
    cudaError_t e = cudaMemcpyFromSymbol(line, g_mlkd_check_line, sizeof(unsigned));
    if (e != cudaSuccess) return e;
    if (*line) {
        const unsigned zero = 0u;
        e = cudaMemcpyToSymbol(g_mlkd_check_line, &zero, sizeof(unsigned));
    }
    return e;
#else
    return cudaSuccess;
#endif
}

}  // namespace mlkd
