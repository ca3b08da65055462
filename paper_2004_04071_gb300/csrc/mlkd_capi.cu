// mlkd_capi.cu -- the C ABI of include/mlkd.h: problem validation, the
// context over a caller-owned device arena, and the host side of the
// per-level run and of the adaptive MLMC estimate (Sec. 4.1).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <cuda.h>

#include "mlkd_host.h"

using namespace mlkd;

namespace mlkd {

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

Layout arena_layout()
{
    Layout L;
    L.n_guard = 0;
    size_t off = 0;
    // a region of `bytes` at the current offset, then (debug build) its canary
    auto place = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes);
        if (kGuardBytes) {
            L.guard[L.n_guard++] = off;
            off += kGuardBytes;
        }
        return at;
    };
    // one scratch slot (block partials, level sums, histogram) per level, so
    // that the levels of a round can run at the same time
    L.partials = place((size_t)MLKD_MAX_LEVELS * kMaxBlocks * kPartialWords * sizeof(double));
    L.tmp_stats = place(MLKD_MAX_LEVELS * sizeof(DevLevelStats));
    L.acc_stats = place(MLKD_MAX_LEVELS * sizeof(DevLevelStats));
    L.tmp_hist = place((size_t)MLKD_MAX_LEVELS * 3 * MLKD_MAX_BINS * sizeof(unsigned long long));
    L.acc_hist = place((size_t)MLKD_MAX_LEVELS * 3 * MLKD_MAX_BINS * sizeof(unsigned long long));
    L.control = place(sizeof(DevControl));
    L.total = off;
    return L;
}

mlkd_status guards_write(char *arena, const size_t *guard, int n, cudaStream_t s)
{
    for (int i = 0; i < n && kGuardBytes; ++i)
        MLKD_CUDA(cudaMemsetAsync(arena + guard[i], kGuardByte, kGuardBytes, s));
    return MLKD_OK;
}

mlkd_status guards_check(const char *arena, const size_t *guard, int n)
{
    if (!kGuardBytes) return MLKD_OK;
    unsigned char buf[kGuardBytes > 0 ? kGuardBytes : 1];
    for (int i = 0; i < n; ++i) {
        MLKD_CUDA(cudaMemcpy(buf, arena + guard[i], kGuardBytes, cudaMemcpyDeviceToHost));
        for (size_t j = 0; j < kGuardBytes; ++j)
            if (buf[j] != kGuardByte) return MLKD_EINTERNAL;
    }
    return MLKD_OK;
}

bool validate(const mlkd_problem *p, Derived *d)
{
    if (!p) return false;
    const bool het = p->background != MLKD_BG_HOMOGENEOUS;
    if (p->background < MLKD_BG_HOMOGENEOUS || p->background > MLKD_BG_B2) return false;
    if (het) {
        if (!(p->bg_b > 0.0) || !std::isfinite(p->bg_b) || !(p->bg_a >= 0.0) || !std::isfinite(p->bg_a))
            return false;
        if (p->mu != 0.0) return false;
    } else if (!(p->eps > 0.0) || !std::isfinite(p->eps)) {
        return false;
    }
    if (!(p->T > 0.0) || !(p->dt0 > 0.0) || !std::isfinite(p->T) || !std::isfinite(p->dt0)) return false;
    if (!std::isfinite(p->mu)) return false;
    if (p->M < 2 || p->M > 64) return false;
    if (p->L < 0 || p->L >= MLKD_MAX_LEVELS) return false;
    if (p->qoi < MLKD_QOI_X2 || p->qoi > MLKD_QOI_X) return false;
    if (p->init != MLKD_INIT_ORIGIN && p->init != MLKD_INIT_COSINE && p->init != MLKD_INIT_POINT) return false;
    if (p->init == MLKD_INIT_POINT && !std::isfinite(p->x0)) return false;
    if (p->qoi == MLKD_QOI_X && (p->init == MLKD_INIT_COSINE)) return false;
    // the heterogeneous backgrounds start from a point (the paper's x0 = 1)
    if (het && p->init == MLKD_INIT_COSINE) return false;
    if (p->precision < MLKD_PREC_FP64 || p->precision > MLKD_PREC_FP64_U24) return false;
    if (p->nbins < 0 || p->nbins > MLKD_MAX_BINS) return false;
    if (p->qoi == MLKD_QOI_DENSITY && p->nbins == 0) return false;
    const double r = p->T / p->dt0;
    const double n0 = std::nearbyint(r);
    if (n0 < 1.0 || std::fabs(r - n0) > 1e-12 * std::max(1.0, r)) return false;
    // finest level: n0 * M^L fine steps; FP32 state needs exact step indices
    double nmax = n0;
    for (int l = 0; l < p->L; ++l) nmax *= p->M;
    const bool fp64_state = p->precision == MLKD_PREC_FP64 || p->precision == MLKD_PREC_FP64_U24;
    const double cap = fp64_state && !het ? 1073741824.0 : 16777216.0;
    if (nmax > cap) return false;
    if (het) {
        d->R = p->bg_b;
        d->sigma = 1.0;
    } else {
        const double R = 1.0 / (p->eps * p->eps);
        if (!std::isfinite(R) || R <= 0.0) return false;
        d->R = R;
        d->sigma = 1.0 / p->eps;
    }
    d->mu = p->mu;
    d->n0 = (long long)n0;
    d->mode = p->precision;
    d->background = p->background;
    // x(T) and a point start run in the batched form for the heterogeneous
    // backgrounds (whose test case they are), and only per level otherwise
    d->per_level_only = !het && (p->qoi == MLKD_QOI_X || p->init == MLKD_INIT_POINT);
    d->periodic = p->qoi == MLKD_QOI_X2_PERIODIC || p->init == MLKD_INIT_COSINE;
    if (d->periodic) {
        d->lo = 0.0;
        d->hi = 1.0;
    } else {
        if (p->nbins > 0 && !(p->lo < p->hi && std::isfinite(p->lo) && std::isfinite(p->hi))) return false;
        d->lo = p->lo;
        d->hi = p->hi;
    }
    d->h = p->nbins > 0 ? (d->hi - d->lo) / p->nbins : 1.0;
    // estimator levels: all of 0..L, or a level set ending at L (Sec. 4.2)
    if (p->n_set == 0) {
        d->J = p->L + 1;
        for (int j = 0; j <= p->L; ++j) {
            d->lev[j] = j;
            d->Mj[j] = p->M;
        }
    } else {
        if (p->n_set < 1 || p->n_set > p->L + 1 || !p->level_set) return false;
        d->J = p->n_set;
        for (int j = 0; j < p->n_set; ++j) {
            const int l = p->level_set[j];
            if (l < 0 || l > p->L) return false;
            if (j > 0 && l <= p->level_set[j - 1]) return false;
            d->lev[j] = l;
            d->Mj[j] = p->M;
            if (j > 0) {
                double mj = 1.0;
                for (int g = p->level_set[j - 1]; g < l; ++g) mj *= p->M;
                if (mj > 1048576.0) return false;
                d->Mj[j] = (int)mj;
            }
        }
        if (p->level_set[p->n_set - 1] != p->L) return false;
    }
    return true;
}

long long ipow(long long b, int e)
{
    long long r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

}  // namespace mlkd

namespace mlkd {

// Fills the kernel parameters of pairs [first, first+count) of `level`.
void fill_launch(const mlkd_problem *p, const Derived &d, int j, uint64_t first, uint64_t count,
                 PairLaunch *P)
{
    std::memset(P, 0, sizeof(*P));
    const int level = d.lev[j];                  // fine level of estimator level j
    const long long Ml = ipow(p->M, level);
    P->R = d.R;
    P->mu = d.mu;
    P->sigma = d.sigma;
    P->dt = p->dt0 / (double)Ml;
    P->lo = d.lo;
    P->hi = d.hi;
    P->h = d.h;
    P->n = (int32_t)(d.n0 * Ml);
    P->M = d.Mj[j];
    P->periodic = d.periodic ? 1 : 0;
    P->fkind = p->qoi == MLKD_QOI_X ? 2 : d.periodic ? 1 : 0;
    P->init = p->init;
    P->x0 = p->init == MLKD_INIT_POINT ? p->x0 : 0.0;
    P->background = d.background;
    P->bg_b = p->bg_b;
    P->bg_a_left = d.background == MLKD_BG_B1 ? p->bg_a : 0.0;
    P->bg_a_right = p->bg_a;
    P->nbins = p->nbins;
    P->word2 = (uint32_t)level << 24;
    P->request = p->request;
    const uint32_t s0 = (uint32_t)p->seed, s1 = (uint32_t)(p->seed >> 32);
    for (int r = 0; r < 10; ++r) {
        P->keys.k0[r] = s0 + (uint32_t)r * kWeylA;
        P->keys.k1[r] = s1 + (uint32_t)r * kWeylB;
    }
    P->first_pair = first;
    P->n_pairs = count;
    BgParams<double> &b = P->bd;
    b.R = P->R;
    b.invR = 1.0 / P->R;
    b.mu = P->mu;
    b.sigma = P->sigma;
    b.two_c2 = 2.0 * P->sigma * P->sigma / (P->R * P->R);
    b.dt = P->dt;
    b.Rdt = P->R * P->dt;
    b.inv_Rdt = 1.0 / (P->R * P->dt);
    b.lo = P->lo;
    b.hi = P->hi;
    b.inv_h = 1.0 / P->h;
    BgParams<float> &f = P->bf;
    f.R = (float)b.R;
    f.invR = (float)b.invR;
    f.mu = (float)b.mu;
    f.sigma = (float)b.sigma;
    f.two_c2 = (float)b.two_c2;
    f.dt = (float)b.dt;
    f.Rdt = (float)b.Rdt;
    f.inv_Rdt = (float)b.inv_Rdt;
    f.lo = (float)b.lo;
    f.hi = (float)b.hi;
    f.inv_h = (float)b.inv_h;
}

}  // namespace mlkd

namespace {

// Grid of the pair kernel: enough warps for the pairs, at most one full wave
// of resident blocks; each warp gets an equal contiguous chunk.
mlkd_status choose_grid(mlkd_context *ctx, int mode, bool coupled, int nbins, uint64_t count,
                        int *grid, unsigned long long *ppw, int background)
{
    KernelInfo info;
    if (pair_kernel_info(mode, coupled, nbins, &info, background) != cudaSuccess) return MLKD_ECUDA;
    const int per_sm = std::max(1, info.blocks_per_sm);
    const long long wave = std::min<long long>((long long)ctx->sm_count * per_sm, kMaxBlocks);
    const unsigned long long warps_needed = (count + 31) / 32;
    const unsigned long long blocks_needed = (warps_needed + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const long long g = (long long)std::min<unsigned long long>(blocks_needed, (unsigned long long)wave);
    *grid = (int)std::max<long long>(1, g);
    const unsigned long long warps = (unsigned long long)(*grid) * kWarpsPerBlock;
    *ppw = (count + warps - 1) / warps;
    return MLKD_OK;
}

}  // namespace

static unsigned g_last_check_line = 0;   // source line of the last failed device check

mlkd_status mlkd::device_checks()
{
#ifdef MLKD_CHECKS
    unsigned a = 0u, b = 0u;
    MLKD_CUDA(check_word_kernels(&a));
    MLKD_CUDA(check_word_batch(&b));
    if (a || b) {
        g_last_check_line = a ? a : b;
        return MLKD_EINTERNAL;
    }
#endif
    return MLKD_OK;
}

// Adds the elapsed time of every recorded pair-kernel launch (waiting for
// each to end; the launches may be on several streams).
mlkd_status mlkd::harvest_timing(mlkd_context *ctx)
{
    for (int i = 0; i < ctx->pending; ++i) {
        float ms = 0.0f;
        MLKD_CUDA(cudaEventSynchronize(ctx->ev_stop[i]));
        MLKD_CUDA(cudaEventElapsedTime(&ms, ctx->ev_start[i], ctx->ev_stop[i]));
        ctx->kernel_ms += ms;
        ++ctx->launches;
    }
    ctx->pending = 0;
    return MLKD_OK;
}

namespace {

// Enqueues one level run: pair kernel + fixed-order finalize (+ accumulation).
mlkd_status enqueue_level(mlkd_context *ctx, const mlkd_problem *p, const Derived &d, int level,
                          uint64_t first, uint64_t count, cudaStream_t stream,
                          bool accumulate, double *dxf, double *dxc, int32_t *dkf, int32_t *dkc,
                          int slot = 0)
{
    // this launch's scratch slot: concurrent launches use different slots
    double *partials = ctx->partials + (size_t)slot * kMaxBlocks * kPartialWords;
    DevLevelStats *tmp_stats = ctx->tmp_stats + slot;
    unsigned long long *tmp_hist = ctx->tmp_hist + (size_t)slot * 3 * MLKD_MAX_BINS;
    PairLaunch P;
    fill_launch(p, d, level, first, count, &P);
    int grid = 1;
    unsigned long long ppw = 0;
    mlkd_status st = choose_grid(ctx, d.mode, level > 0, p->nbins, count, &grid, &ppw, d.background);
    if (st != MLKD_OK) return st;
    P.pairs_per_warp = ppw;
    P.partials = partials;
    P.partial_rows = kMaxBlocks;
    P.hist = p->nbins > 0 ? tmp_hist : nullptr;
    P.dbg_xf = dxf;
    P.dbg_xc = dxc;
    P.dbg_kf = dkf;
    P.dbg_kc = dkc;
    if (p->nbins > 0)
        MLKD_CUDA(cudaMemsetAsync(tmp_hist, 0, 3 * (size_t)p->nbins * sizeof(unsigned long long), stream));
    const bool timed = ctx->timing && ctx->events_made;
    if (timed && ctx->pending == kTimingRing) {
        mlkd_status st2 = harvest_timing(ctx);
        if (st2 != MLKD_OK) return st2;
    }
    if (timed) MLKD_CUDA(cudaEventRecord(ctx->ev_start[ctx->pending], stream));
    MLKD_CUDA(launch_pair_kernel(d.mode, level > 0, P, grid, stream));
    if (timed) MLKD_CUDA(cudaEventRecord(ctx->ev_stop[ctx->pending++], stream));
    MLKD_CUDA(launch_finalize(partials, grid, (long long)count, tmp_stats,
                              accumulate ? ctx->acc_stats + level : nullptr, stream));
    ++ctx->other_launches;
    if (accumulate && p->nbins > 0) {
        MLKD_CUDA(launch_hist_accumulate(tmp_hist, ctx->acc_hist + (size_t)level * 3 * p->nbins,
                                         3 * p->nbins, stream));
        ++ctx->other_launches;
    }
    return MLKD_OK;
}

void to_host_stats(const DevLevelStats &s, mlkd_level_stats *o)
{
    o->n = s.n;
    o->sy = s.sy;
    o->sy2 = s.sy2;
    o->sqf = s.sqf;
    o->sqf2 = s.sqf2;
    o->sqc = s.sqc;
    o->sqc2 = s.sqc2;
    o->events_f = s.events_f;
    o->events_c = s.events_c;
}

}  // namespace

extern "C" {

int mlkd_device_checks(uint32_t *last_line)
{
    if (last_line) *last_line = g_last_check_line;
#ifdef MLKD_CHECKS
    return 1;
#else
    return 0;
#endif
}

mlkd_status mlkd_debug_check_selftest(int device)
{
#ifdef MLKD_CHECKS
    MLKD_CUDA(cudaSetDevice(device));
    MLKD_CUDA(launch_check_selftest(0));
    MLKD_CUDA(cudaDeviceSynchronize());
    return device_checks();
#else
    (void)device;
    return MLKD_ENOTFOUND;
#endif
}

const char *mlkd_status_string(int status)
{
    switch (status) {
    case MLKD_OK: return "ok";
    case MLKD_EINVAL: return "invalid argument";
    case MLKD_ENOMEM: return "arena too small";
    case MLKD_ECUDA: return "CUDA error";
    case MLKD_ETIMEDOUT: return "timed out";
    case MLKD_EBUSY: return "busy";
    case MLKD_ENOTFOUND: return "not found";
    case MLKD_EINTERNAL: return "device consistency check failed";
    default: return "unknown status";
    }
}

int mlkd_abi_version(void) { return MLKD_ABI_VERSION; }

size_t mlkd_workspace_bytes(const mlkd_problem *problem)
{
    Derived d;
    if (!validate(problem, &d)) return 0;
    return arena_layout().total;
}

mlkd_status mlkd_context_create(int device, void *arena, size_t arena_bytes, mlkd_context **out)
{
    if (!out || !arena) return MLKD_EINVAL;
    if (((uintptr_t)arena) % kAlign != 0) return MLKD_EINVAL;
    const Layout L = arena_layout();
    if (arena_bytes < L.total) return MLKD_ENOMEM;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) return MLKD_ECUDA;
    if (device < 0 || device >= ndev) return MLKD_EINVAL;
    MLKD_CUDA(cudaSetDevice(device));
    int sms = 0;
    MLKD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    mlkd_context *c = new (std::nothrow) mlkd_context;
    if (!c) return MLKD_ENOMEM;
    c->device = device;
    c->sm_count = sms;
    c->timing = false;
    c->pending = 0;
    c->events_made = false;
    c->launches = 0;
    c->other_launches = 0;
    c->kernel_ms = 0.0;
    c->batch = nullptr;
    c->server = nullptr;
    c->streams_made = false;
    c->arena = (char *)arena;
    c->arena_bytes = arena_bytes;
    c->L = L;
    c->partials = (double *)(c->arena + L.partials);
    c->tmp_stats = (DevLevelStats *)(c->arena + L.tmp_stats);
    c->acc_stats = (DevLevelStats *)(c->arena + L.acc_stats);
    c->tmp_hist = (unsigned long long *)(c->arena + L.tmp_hist);
    c->acc_hist = (unsigned long long *)(c->arena + L.acc_hist);
    c->control = (DevControl *)(c->arena + L.control);
    if (kGuardBytes && (guards_write(c->arena, L.guard, L.n_guard, 0) != MLKD_OK ||
                        cudaDeviceSynchronize() != cudaSuccess)) {
        delete c;
        return MLKD_ECUDA;
    }
    *out = c;
    return MLKD_OK;
}

void mlkd_context_destroy(mlkd_context *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    mlkd::server_release(ctx);
    mlkd::batch_release(ctx);
    if (ctx->events_made || ctx->streams_made) cudaDeviceSynchronize();
    if (ctx->events_made) {
        for (int i = 0; i < kTimingRing; ++i) {
            cudaEventDestroy(ctx->ev_start[i]);
            cudaEventDestroy(ctx->ev_stop[i]);
        }
    }
    if (ctx->streams_made) {
        for (int l = 0; l < MLKD_MAX_LEVELS; ++l) {
            cudaStreamDestroy(ctx->level_stream[l]);
            cudaEventDestroy(ctx->level_done[l]);
        }
        cudaEventDestroy(ctx->round_start);
    }
    delete ctx;
}

mlkd_status mlkd_level_select(const double *V, const double *Vd, int L, int32_t *set_out, int32_t *n_out)
{
    if (!V || !Vd || !set_out || !n_out || L < 1 || L >= MLKD_MAX_LEVELS) return MLKD_EINVAL;
    // Alg. 3: the first level whose difference variance falls below its own
    // variance, and the level below it
    int l = 1;
    while (l <= L && Vd[l] > V[l]) ++l;
    int n = 0;
    if (l > L) {                      // no decay anywhere: single-level estimate on L
        set_out[n++] = L;
        *n_out = n;
        return MLKD_OK;
    }
    set_out[n++] = l - 1;
    set_out[n++] = l;
    double vmin = Vd[l];
    for (int k = l + 1; k <= L; ++k) {
        if (Vd[k] < vmin / 2.0) {
            set_out[n++] = k;
            vmin = Vd[k];
        }
    }
    if (set_out[n - 1] != L) set_out[n++] = L;   // the estimator's finest level
    *n_out = n;
    return MLKD_OK;
}

mlkd_status mlkd_level_select_opt(const double *V, const double *rho, const double *C, int L,
                                  int32_t *set_out, int32_t *n_out)
{
    if (!V || !rho || !C || !set_out || !n_out || L < 1 || L >= MLKD_MAX_LEVELS) return MLKD_EINVAL;
    for (int i = 0; i <= L; ++i)
        if (!(V[i] >= 0.0) || !(C[i] >= 0.0) || (i < L && !(rho[i] >= -1.0 && rho[i] <= 1.0)))
            return MLKD_EINVAL;
    auto r = [&](int i) { return i == L ? 1.0 : rho[i]; };
    // eq. V_approx, with a negative root argument read as 0
    auto vpair = [&](int b, int a) {
        const double arg = (r(b) * r(b) + r(a) * r(a) - 1.0) * V[b] * V[a];
        const double v = V[b] + V[a] - 2.0 * std::sqrt(arg > 0.0 ? arg : 0.0);
        return v > 0.0 ? v : 0.0;
    };
    // eq. integerLP is a shortest path through increasing levels ending at L:
    // best[k] is the least cost of a set whose last level is k
    double best[MLKD_MAX_LEVELS];
    int prev[MLKD_MAX_LEVELS];
    for (int k = 0; k <= L; ++k) {
        best[k] = std::sqrt(V[k] * C[k]);
        prev[k] = -1;
        for (int i = 0; i < k; ++i) {
            const double c = best[i] + std::sqrt(vpair(k, i) * (C[i] + C[k]));
            if (c < best[k]) {
                best[k] = c;
                prev[k] = i;
            }
        }
    }
    int rev[MLKD_MAX_LEVELS], n = 0;
    for (int k = L; k >= 0; k = prev[k]) rev[n++] = k;
    for (int j = 0; j < n; ++j) set_out[j] = rev[n - 1 - j];
    *n_out = n;
    return MLKD_OK;
}

mlkd_status mlkd_level_pilot(mlkd_context *ctx, const mlkd_problem *problem, uint64_t n, void *stream,
                             double *V, double *rho, double *C)
{
    NvtxRange nvtx_range("mlkd_level_pilot");
    Derived d;
    if (!ctx || !problem || !V || !rho || !C || n < 2 || !validate(problem, &d)) return MLKD_EINVAL;
    if (problem->qoi == MLKD_QOI_DENSITY || problem->L < 1) return MLKD_EINVAL;
    const int L = problem->L;
    for (int i = 0; i < L; ++i) {
        // pairs coupling L with i; the fine path of pair p is the same in
        // every coupling (its stream is keyed by level L)
        mlkd_problem q = *problem;
        const int32_t set[2] = {i, L};
        q.level_set = set;
        q.n_set = 2;
        q.n_fixed = nullptr;
        mlkd_level_stats st;
        const mlkd_status s = mlkd_run_level(ctx, &q, 1, 0, n, stream, &st, nullptr);
        if (s != MLKD_OK) return s;
        const double nn = (double)st.n;
        const double vf = (st.sqf2 - st.sqf * st.sqf / nn) / (nn - 1.0);
        const double vc = (st.sqc2 - st.sqc * st.sqc / nn) / (nn - 1.0);
        // sum F_f F_c from Y = F_f - F_c: (sum F_f^2 + sum F_c^2 - sum Y^2)/2
        const double cov = (0.5 * (st.sqf2 + st.sqc2 - st.sy2) - st.sqf * st.sqc / nn) / (nn - 1.0);
        V[i] = vc > 0.0 ? vc : 0.0;
        C[i] = (double)st.events_c / nn;
        double rr = vf > 0.0 && vc > 0.0 ? cov / std::sqrt(vf * vc) : 0.0;
        rho[i] = rr > 1.0 ? 1.0 : rr < -1.0 ? -1.0 : rr;
        if (i == L - 1) {
            V[L] = vf > 0.0 ? vf : 0.0;
            C[L] = (double)st.events_f / nn;
        }
    }
    return MLKD_OK;
}

mlkd_status mlkd_level_warmup(mlkd_context *ctx, const mlkd_problem *problem, uint64_t n_warmup,
                              void *stream, double *V, double *Vd, int32_t *tau_out)
{
    NvtxRange nvtx_range("mlkd_level_warmup");
    Derived d;
    if (!ctx || !problem || !V || !Vd || !tau_out || n_warmup < 2 || !validate(problem, &d))
        return MLKD_EINVAL;
    if (problem->qoi == MLKD_QOI_DENSITY || problem->L < 1 || problem->n_set > 0) return MLKD_EINVAL;
    const int L = problem->L;
    const double R = 1.0 / (problem->eps * problem->eps);
    // tau: the first level whose step is at most 1/R, the mean time between
    // collisions (where V_{l,l-1} peaks); the finest level if none is
    int tau = L;
    for (int l = 1; l <= L; ++l) {
        const double dtl = problem->dt0 / std::pow((double)problem->M, (double)l);
        if (R * dtl <= 1.0) {
            tau = l;
            break;
        }
    }
    mlkd_problem q = *problem;
    q.n_fixed = nullptr;
    for (int l = 0; l <= tau; ++l) {
        mlkd_level_stats st;
        const mlkd_status s = mlkd_run_level(ctx, &q, l, 0, n_warmup, stream, &st, nullptr);
        if (s != MLKD_OK) return s;
        const double nn = (double)st.n;
        const double vf = (st.sqf2 - st.sqf * st.sqf / nn) / (nn - 1.0);
        const double vy = (st.sy2 - st.sy * st.sy / nn) / (nn - 1.0);
        V[l] = vf > 0.0 ? vf : 0.0;
        Vd[l] = l > 0 && vy > 0.0 ? vy : 0.0;
    }
    // beyond tau: V_l as on tau, V_{l,l-1} decaying like dt_l^3
    const double M3 = (double)problem->M * problem->M * problem->M;
    for (int l = tau + 1; l <= L; ++l) {
        V[l] = V[tau];
        Vd[l] = Vd[tau] / std::pow(M3, (double)(l - tau));
    }
    *tau_out = tau;
    return MLKD_OK;
}

mlkd_status mlkd_debug_transforms(const uint32_t *words, uint64_t n, float *log_u, float *sin_2pi_u,
                                  float *cos_2pi_u, void *stream)
{
    if (!words && n > 0) return MLKD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    MLKD_CUDA(launch_debug_transforms(words, n, log_u, sin_2pi_u, cos_2pi_u, s));
    MLKD_CUDA(cudaStreamSynchronize(s));
    return MLKD_OK;
}

mlkd_status mlkd_debug_kd_coeffs(int precision, double R, double mu, double sigma,
                                 const double *theta, const double *dv, uint64_t n, double *a,
                                 double *d, double *hs, double *om, double *beta_hat_sq,
                                 void *stream)
{
    if (precision < MLKD_PREC_FP64 || precision > MLKD_PREC_FP64_U24) return MLKD_EINVAL;
    if (!(R > 0.0) || !std::isfinite(R) || !std::isfinite(mu) || !(sigma >= 0.0)) return MLKD_EINVAL;
    if (n > 0 && (!theta || !dv || !a || !d || !hs || !om || !beta_hat_sq)) return MLKD_EINVAL;
    const int fp64 = precision == MLKD_PREC_FP64 || precision == MLKD_PREC_FP64_U24;
    cudaStream_t s = (cudaStream_t)stream;
    MLKD_CUDA(launch_debug_kd(fp64, R, mu, sigma, theta, dv, n, a, d, hs, om, beta_hat_sq, s));
    MLKD_CUDA(cudaStreamSynchronize(s));
    return device_checks();
}

mlkd_status mlkd_context_set_timing(mlkd_context *ctx, int enable)
{
    if (!ctx) return MLKD_EINVAL;
    MLKD_CUDA(cudaSetDevice(ctx->device));
    if (enable && !ctx->events_made) {
        for (int i = 0; i < kTimingRing; ++i) {
            MLKD_CUDA(cudaEventCreate(&ctx->ev_start[i]));
            MLKD_CUDA(cudaEventCreate(&ctx->ev_stop[i]));
        }
        ctx->events_made = true;
    }
    ctx->timing = enable != 0;
    return MLKD_OK;
}

mlkd_status mlkd_context_get_timing(mlkd_context *ctx, mlkd_kernel_timing *out, int reset)
{
    if (!ctx || !out) return MLKD_EINVAL;
    if (ctx->pending) {
        MLKD_CUDA(cudaDeviceSynchronize());
        mlkd_status st = harvest_timing(ctx);
        if (st != MLKD_OK) return st;
    }
    out->launches = ctx->launches;
    out->pair_kernel_ms = ctx->kernel_ms;
    out->other_launches = ctx->other_launches;
    if (reset) {
        ctx->launches = 0;
        ctx->other_launches = 0;
        ctx->kernel_ms = 0.0;
    }
    return MLKD_OK;
}

mlkd_status mlkd_run_level(mlkd_context *ctx, const mlkd_problem *problem, int level,
                           uint64_t first_pair, uint64_t n_pairs, void *stream,
                           mlkd_level_stats *out, uint64_t *hist_out)
{
    NvtxRange nvtx_range("mlkd_run_level");
    Derived d;
    if (!ctx || !out || !validate(problem, &d)) return MLKD_EINVAL;
    if (level < 0 || level >= d.J) return MLKD_EINVAL;
    if (first_pair + n_pairs < first_pair) return MLKD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    MLKD_CUDA(cudaSetDevice(ctx->device));
    if (n_pairs == 0) {
        std::memset(out, 0, sizeof(*out));
        if (hist_out && problem->nbins > 0) std::memset(hist_out, 0, 3 * (size_t)problem->nbins * sizeof(uint64_t));
        return MLKD_OK;
    }
    mlkd_status st = enqueue_level(ctx, problem, d, level, first_pair, n_pairs, s, false,
                                   nullptr, nullptr, nullptr, nullptr);
    if (st != MLKD_OK) return st;
    DevLevelStats hs;
    MLKD_CUDA(cudaMemcpyAsync(&hs, ctx->tmp_stats, sizeof(hs), cudaMemcpyDeviceToHost, s));
    if (hist_out && problem->nbins > 0)
        MLKD_CUDA(cudaMemcpyAsync(hist_out, ctx->tmp_hist, 3 * (size_t)problem->nbins * sizeof(uint64_t),
                                  cudaMemcpyDeviceToHost, s));
    MLKD_CUDA(cudaStreamSynchronize(s));
    to_host_stats(hs, out);
    st = harvest_timing(ctx);
    if (st == MLKD_OK) st = device_checks();
    return st != MLKD_OK ? st : guards_check(ctx->arena, ctx->L.guard, ctx->L.n_guard);
}

mlkd_status mlkd_debug_pairs(mlkd_context *ctx, const mlkd_problem *problem, int level,
                             uint64_t first_pair, uint64_t n_pairs, void *stream, double *xf,
                             double *xc, int32_t *kf, int32_t *kc)
{
    NvtxRange nvtx_range("mlkd_debug_pairs");
    Derived d;
    if (!ctx || !validate(problem, &d)) return MLKD_EINVAL;
    if (level < 0 || level >= d.J) return MLKD_EINVAL;
    if (!xf && (xc || kf || kc)) return MLKD_EINVAL;   // xf gates the per-pair writes
    cudaStream_t s = (cudaStream_t)stream;
    MLKD_CUDA(cudaSetDevice(ctx->device));
    if (n_pairs == 0) return MLKD_OK;
    mlkd_status st = enqueue_level(ctx, problem, d, level, first_pair, n_pairs, s, false, xf, xc,
                                   kf, kc);
    if (st != MLKD_OK) return st;
    MLKD_CUDA(cudaStreamSynchronize(s));
    return harvest_timing(ctx);
}

mlkd_status mlkd_debug_coarse_draws(mlkd_context *ctx, const mlkd_problem *problem, int level,
                                    uint64_t first_pair, uint64_t n_pairs, int per_pair,
                                    void *stream, double *nu_t, double *E_t, double *chi_t,
                                    int32_t *count)
{
    NvtxRange nvtx_range("mlkd_debug_coarse_draws");
    Derived d;
    if (!ctx || !validate(problem, &d) || d.per_level_only || d.background != MLKD_BG_HOMOGENEOUS)
        return MLKD_EINVAL;
    if (level < 1 || level >= d.J || per_pair < 1) return MLKD_EINVAL;
    if (!nu_t || !E_t || !chi_t || !count) return MLKD_EINVAL;
    if (n_pairs > (1ull << 31) / (unsigned long long)per_pair) return MLKD_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    MLKD_CUDA(cudaSetDevice(ctx->device));
    if (n_pairs == 0) return MLKD_OK;
    PairLaunch P;
    fill_launch(problem, d, level, first_pair, n_pairs, &P);
    MLKD_CUDA(launch_coarse_draws(d.mode, P, per_pair, nu_t, E_t, chi_t, count, s));
    ctx->other_launches += 1;
    MLKD_CUDA(cudaStreamSynchronize(s));
    return MLKD_OK;
}

}  // extern "C"

// Streams and events of the concurrent per-level rounds, made once per context.
static mlkd_status ensure_level_streams(mlkd_context *ctx)
{
    if (ctx->streams_made) return MLKD_OK;
    MLKD_CUDA(cudaEventCreateWithFlags(&ctx->round_start, cudaEventDisableTiming));
    for (int l = 0; l < MLKD_MAX_LEVELS; ++l) {
        MLKD_CUDA(cudaStreamCreateWithFlags(&ctx->level_stream[l], cudaStreamNonBlocking));
        MLKD_CUDA(cudaEventCreateWithFlags(&ctx->level_done[l], cudaEventDisableTiming));
    }
    ctx->streams_made = true;
    return MLKD_OK;
}

// Adaptive MLMC (Sec. 4.1) with an optional starting state and a round limit.
static mlkd_status estimate_impl(mlkd_context *ctx, const mlkd_problem *problem,
                                 const mlkd_result *resume, const uint64_t *hist_in, int max_rounds,
                                 void *stream, mlkd_result *out, uint64_t *hist_out)
{
    NvtxRange nvtx_range("mlkd_estimate");
    Derived d;
    if (!ctx || !out || !validate(problem, &d)) return MLKD_EINVAL;
    if (max_rounds < 0) return MLKD_EINVAL;
    if (!problem->n_fixed && !(problem->tol > 0.0)) return MLKD_EINVAL;
    if (!problem->n_fixed && problem->n_warmup < 2) return MLKD_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    MLKD_CUDA(cudaSetDevice(ctx->device));
    const int nl = d.J;
    const int nb = problem->nbins;
    MLKD_CUDA(cudaMemsetAsync(ctx->acc_stats, 0, nl * sizeof(DevLevelStats), s));
    if (nb > 0)
        MLKD_CUDA(cudaMemsetAsync(ctx->acc_hist, 0, (size_t)nl * 3 * nb * sizeof(unsigned long long), s));
    long long have[MLKD_MAX_LEVELS] = {0};
    const int density = problem->qoi == MLKD_QOI_DENSITY ? 1 : 0;
    DevControl ctl;
    int rounds = 0;
    if (resume) {
        // restart from a saved state: the level sums and pair counts (pair p
        // always uses the same stream, so the run continues where it stopped)
        if (resume->n_levels != nl || (nb > 0 && !hist_in)) return MLKD_EINVAL;
        DevLevelStats init[MLKD_MAX_LEVELS];
        for (int l = 0; l < nl; ++l) {
            const mlkd_level_stats &r = resume->lv[l];
            if (r.n < 0) return MLKD_EINVAL;
            init[l].n = r.n;
            init[l].sy = r.sy;
            init[l].sy2 = r.sy2;
            init[l].sqf = r.sqf;
            init[l].sqf2 = r.sqf2;
            init[l].sqc = r.sqc;
            init[l].sqc2 = r.sqc2;
            init[l].events_f = r.events_f;
            init[l].events_c = r.events_c;
            have[l] = r.n;
        }
        MLKD_CUDA(cudaMemcpyAsync(ctx->acc_stats, init, nl * sizeof(DevLevelStats), cudaMemcpyHostToDevice, s));
        if (nb > 0)
            MLKD_CUDA(cudaMemcpyAsync(ctx->acc_hist, hist_in, (size_t)nl * 3 * nb * sizeof(unsigned long long),
                                      cudaMemcpyHostToDevice, s));
        MLKD_CUDA(cudaStreamSynchronize(s));
        rounds = resume->rounds;
    }

    // One round: every level l with want[l] > have[l] runs its new pairs.
    // The levels are independent (own pairs, own scratch slot, own sums), so
    // they run at the same time, each on its level stream, between an event
    // recorded on the caller's stream and the caller's stream waiting for
    // all of them.  A round of small deep levels then lasts about as long as
    // its longest chain instead of the sum of the levels.
    MLKD_CUDA(ensure_level_streams(ctx));
    auto round = [&](const long long *want) -> mlkd_status {
        MLKD_CUDA(cudaEventRecord(ctx->round_start, s));
        bool used[MLKD_MAX_LEVELS] = {false};
        mlkd_status st = MLKD_OK;
        for (int l = 0; l < nl && st == MLKD_OK; ++l) {
            if (want[l] <= have[l]) continue;
            cudaStream_t ls = ctx->level_stream[l];
            MLKD_CUDA(cudaStreamWaitEvent(ls, ctx->round_start, 0));
            used[l] = true;
            st = enqueue_level(ctx, problem, d, l, (uint64_t)have[l], (uint64_t)(want[l] - have[l]), ls,
                               true, nullptr, nullptr, nullptr, nullptr, l);
            if (st == MLKD_OK) have[l] = want[l];
        }
        for (int l = 0; l < nl; ++l) {
            if (!used[l]) continue;
            MLKD_CUDA(cudaEventRecord(ctx->level_done[l], ctx->level_stream[l]));
            MLKD_CUDA(cudaStreamWaitEvent(s, ctx->level_done[l], 0));
        }
        return st;
    };
    auto control = [&]() -> mlkd_status {
        MLKD_CUDA(launch_controller(ctx->acc_stats, ctx->acc_hist, nl, nb, d.h, density,
                                    problem->tol, ctx->control, s));
        ++ctx->other_launches;
        MLKD_CUDA(cudaMemcpyAsync(&ctl, ctx->control, sizeof(ctl), cudaMemcpyDeviceToHost, s));
        MLKD_CUDA(cudaStreamSynchronize(s));
        return harvest_timing(ctx);
    };

    mlkd_status st;
    long long want[MLKD_MAX_LEVELS];
    if (problem->n_fixed) {
        for (int l = 0; l < nl; ++l) {
            if (problem->n_fixed[l] < 0) return MLKD_EINVAL;
            want[l] = problem->n_fixed[l];
        }
        if ((st = round(want)) != MLKD_OK) return st;
        if ((st = control()) != MLKD_OK) return st;
    } else {
        if (!resume) {
            for (int l = 0; l < nl; ++l) want[l] = problem->n_warmup;
            if ((st = round(want)) != MLKD_OK) return st;
        }
        for (;;) {
            if ((st = control()) != MLKD_OK) return st;
            if (rounds >= max_rounds) break;           // stop; resumable from here
            bool grew = false;
            for (int l = 0; l < nl; ++l) {
                want[l] = ctl.target[l];
                grew = grew || ctl.target[l] > have[l];
            }
            if (!grew) break;
            if ((st = round(want)) != MLKD_OK) return st;
            ++rounds;
        }
    }
    DevLevelStats acc[MLKD_MAX_LEVELS];
    MLKD_CUDA(cudaMemcpyAsync(acc, ctx->acc_stats, nl * sizeof(DevLevelStats), cudaMemcpyDeviceToHost, s));
    unsigned long long hacc[3 * MLKD_MAX_BINS];
    double *dens = out->density;
    std::memset(out, 0, sizeof(*out));
    out->density = dens;
    if ((dens || hist_out) && nb > 0) {
        if (dens)
            for (int i = 0; i < nb; ++i) dens[i] = 0.0;
        MLKD_CUDA(cudaStreamSynchronize(s));
        for (int l = 0; l < nl; ++l) {
            MLKD_CUDA(cudaMemcpy(hacc, ctx->acc_hist + (size_t)l * 3 * nb, 3 * (size_t)nb * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost));
            if (hist_out)
                for (int b = 0; b < 3 * nb; ++b) hist_out[(size_t)l * 3 * nb + b] = hacc[b];
            if (dens && acc[l].n > 0)
                for (int b = 0; b < nb; ++b)
                    dens[b] += ((double)hacc[b] - (double)hacc[nb + b]) / (double)acc[l].n;
        }
        if (dens)
            for (int b = 0; b < nb; ++b) dens[b] /= d.h;
    }
    MLKD_CUDA(cudaStreamSynchronize(s));
    out->estimate = ctl.estimate;
    out->variance = ctl.variance;
    out->n_levels = nl;
    out->rounds = rounds;
    for (int l = 0; l < nl; ++l) {
        to_host_stats(acc[l], &out->lv[l]);
        out->var_level[l] = ctl.var_level[l];
        out->cost_level[l] = ctl.cost_level[l];
    }
    out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    mlkd_status hst = harvest_timing(ctx);
    if (hst == MLKD_OK) hst = device_checks();
    return hst != MLKD_OK ? hst : guards_check(ctx->arena, ctx->L.guard, ctx->L.n_guard);
}

extern "C" {

mlkd_status mlkd_estimate(mlkd_context *ctx, const mlkd_problem *problem, void *stream,
                          mlkd_result *out)
{
    return estimate_impl(ctx, problem, nullptr, nullptr, 64, stream, out, nullptr);
}

mlkd_status mlkd_estimate_resumable(mlkd_context *ctx, const mlkd_problem *problem,
                                    const mlkd_result *resume, const uint64_t *hist_in,
                                    int max_rounds, void *stream, mlkd_result *out,
                                    uint64_t *hist_out)
{
    return estimate_impl(ctx, problem, resume, hist_in, max_rounds, stream, out, hist_out);
}

mlkd_status mlkd_estimate_sequence(mlkd_context *ctx, const mlkd_problem *problem, int n_tol,
                                   const double *tols, void *stream, mlkd_result *results)
{
    NvtxRange nvtx_range("mlkd_estimate_sequence");
    Derived d;
    if (!ctx || !problem || !tols || !results || n_tol < 1 || !validate(problem, &d))
        return MLKD_EINVAL;
    if (problem->n_fixed) return MLKD_EINVAL;
    for (int r = 0; r < n_tol; ++r)
        if (!(tols[r] > 0.0)) return MLKD_EINVAL;
    // one estimator continued through the sequence: each stage resumes the
    // previous one's sums and histogram counts under the next tolerance
    const int nb = problem->nbins;
    std::vector<uint64_t> hist[2];
    if (nb > 0)
        for (auto &h : hist) h.assign((size_t)d.J * 3 * nb, 0);
    mlkd_problem q = *problem;
    for (int r = 0; r < n_tol; ++r) {
        q.tol = tols[r];
        const mlkd_result *prev = r > 0 ? &results[r - 1] : nullptr;
        const int max_rounds = (prev ? prev->rounds : 0) + 64;
        const uint64_t *hin = nb > 0 && r > 0 ? hist[(r - 1) & 1].data() : nullptr;
        uint64_t *hout = nb > 0 ? hist[r & 1].data() : nullptr;
        const mlkd_status st = estimate_impl(ctx, &q, prev, hin, max_rounds, stream, &results[r], hout);
        if (st != MLKD_OK) return st;
    }
    return MLKD_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free entry point: the same pair kernel and finalize, with their
// scratch in a file-scope device array instead of a caller arena.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocStatsOffset = (size_t)MLKD_NOALLOC_MAX_BLOCKS * kPartialWords * sizeof(double);
constexpr size_t kNoAllocHistOffset = kNoAllocStatsOffset + 256;
constexpr size_t kNoAllocBytes = kNoAllocHistOffset + 3 * (size_t)MLKD_NOALLOC_MAX_BINS * sizeof(unsigned long long);
static_assert(kNoAllocBytes == (size_t)MLKD_NOALLOC_SCRATCH_BYTES, "scratch size mismatch");
static_assert(sizeof(DevLevelStats) <= 256, "level stats exceed their scratch slot");

}  // namespace

// Shared by every call on a device; see the header for the race rule.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

constexpr int kNoAllocMaxDevices = 64;

// The array's device address belongs to the CUDA context that loaded the
// module: after a device reset (or a primary-context teardown) the module is
// loaded again at another address.  The cached address is therefore keyed on
// the unique id of the current context (cuCtxGetId, reached through the
// runtime's driver entry points, so the library does not link libcuda), and
// looked up again whenever that id changes.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

struct NoAllocSlot {
    unsigned long long ctx_id;
    void *ptr;
};

std::mutex g_noalloc_mutex;
NoAllocSlot g_noalloc_slot[kNoAllocMaxDevices] = {};
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// Unique id of the current context (0 if it cannot be read).
bool current_context_id(unsigned long long *id)
{
    if (!g_ctx_get_current || !g_ctx_get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
            return false;
        g_ctx_get_current = (CtxGetCurrentFn)f1;
        g_ctx_get_id = (CtxGetIdFn)f2;
    }
    CUcontext ctx = nullptr;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return g_ctx_get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the scratch array in the current context of `device`
// (the current device): looked up on the first call in each context.
mlkd_status noalloc_scratch(int device, unsigned char **out)
{
    if (device < 0 || device >= kNoAllocMaxDevices) return MLKD_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    unsigned long long id = 0;
    if (!current_context_id(&id)) return MLKD_ECUDA;
    NoAllocSlot &slot = g_noalloc_slot[device];
    if (!slot.ptr || slot.ctx_id != id) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return MLKD_ECUDA;
        slot.ptr = ptr;
        slot.ctx_id = id;
    }
    *out = (unsigned char *)slot.ptr;
    return MLKD_OK;
}

}  // namespace

extern "C" mlkd_status mlkd_run_level_noalloc(const mlkd_problem *problem, int level,
                                              uint64_t first_pair, uint64_t n_pairs, void *stream,
                                              mlkd_level_stats *out, uint64_t *hist_out)
{
    Derived d;
    if (!out || !validate(problem, &d)) return MLKD_EINVAL;
    if (level < 0 || level >= d.J) return MLKD_EINVAL;
    if (first_pair + n_pairs < first_pair) return MLKD_EINVAL;
    if (problem->nbins > MLKD_NOALLOC_MAX_BINS) return MLKD_ENOMEM;
    int device = 0;
    MLKD_CUDA(cudaGetDevice(&device));
    unsigned char *scratch = nullptr;
    mlkd_status st = noalloc_scratch(device, &scratch);
    if (st != MLKD_OK) return st;
    if (n_pairs == 0) {
        std::memset(out, 0, sizeof(*out));
        if (hist_out && problem->nbins > 0) std::memset(hist_out, 0, 3 * (size_t)problem->nbins * sizeof(uint64_t));
        return MLKD_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int sms = 0;
    MLKD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    KernelInfo info;
    MLKD_CUDA(pair_kernel_info(d.mode, level > 0, problem->nbins, &info, d.background));
    const long long wave = std::min<long long>((long long)sms * std::max(1, info.blocks_per_sm),
                                               MLKD_NOALLOC_MAX_BLOCKS);
    const unsigned long long warps_needed = (n_pairs + 31) / 32;
    const unsigned long long blocks_needed = (warps_needed + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const int grid = (int)std::max<long long>(
        1, (long long)std::min<unsigned long long>(blocks_needed, (unsigned long long)wave));
    const unsigned long long warps = (unsigned long long)grid * kWarpsPerBlock;

    PairLaunch P;
    fill_launch(problem, d, level, first_pair, n_pairs, &P);
    P.pairs_per_warp = (n_pairs + warps - 1) / warps;
    P.partials = (double *)scratch;
    P.partial_rows = MLKD_NOALLOC_MAX_BLOCKS;
    P.hist = problem->nbins > 0 ? (unsigned long long *)(scratch + kNoAllocHistOffset) : nullptr;
    DevLevelStats *dstats = (DevLevelStats *)(scratch + kNoAllocStatsOffset);
    if (problem->nbins > 0)   // counters keep the previous call's values
        MLKD_CUDA(cudaMemsetAsync(P.hist, 0, 3 * (size_t)problem->nbins * sizeof(unsigned long long), s));
    MLKD_CUDA(launch_pair_kernel(d.mode, level > 0, P, grid, s));
    MLKD_CUDA(launch_finalize(P.partials, grid, (long long)n_pairs, dstats, nullptr, s));
    DevLevelStats hs;
    MLKD_CUDA(cudaMemcpyAsync(&hs, dstats, sizeof(hs), cudaMemcpyDeviceToHost, s));
    if (hist_out && problem->nbins > 0)
        MLKD_CUDA(cudaMemcpyAsync(hist_out, P.hist, 3 * (size_t)problem->nbins * sizeof(uint64_t),
                                  cudaMemcpyDeviceToHost, s));
    MLKD_CUDA(cudaStreamSynchronize(s));
    to_host_stats(hs, out);
    return MLKD_OK;
}
