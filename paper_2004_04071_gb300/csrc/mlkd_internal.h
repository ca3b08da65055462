// mlkd_internal.h -- shared between the kernel and host translation units of
// the library (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mlkd_device.cuh"

namespace mlkd {

constexpr int kThreads = 128;          // threads per block of the pair kernel
constexpr int kWarpsPerBlock = kThreads / 32;
constexpr int kPartialWords = 8;       // sy, sy2, sqf, sqf2, sqc, sqc2, ev_f, ev_c

enum Mode { kModeFP64 = 0, kModeFP32DY64 = 1, kModeFP32Comp = 2, kModeFP64U24 = 3 };

// Device checks of the debug build (compiled with -DMLKD_CHECKS, the library
// libmlkd_checked.so).  MLKD_DCHECK(c) evaluates c; if it is false it records
// the source line in this translation unit's check word (the first failure
// wins) and yields false, so that the caller clamps its index into bounds and
// goes on: a failed check never touches memory out of bounds, traps or
// stops the kernel.  The host reads the words after each synchronising call
// and returns MLKD_EINTERNAL.  In normal builds MLKD_DCHECK(c) is the
// constant true and compiles to nothing.
#ifdef MLKD_CHECKS
static __device__ unsigned int g_mlkd_check_line;
__device__ __forceinline__ bool check_record(bool ok, int line)
{
    if (!ok) atomicCAS(&g_mlkd_check_line, 0u, (unsigned)line);
    return ok;
}
#define MLKD_DCHECK(...) (::mlkd::check_record((__VA_ARGS__), __LINE__))
#else
#define MLKD_DCHECK(...) true
#endif

// Reads and clears the check word of one translation unit (0: no failure;
// always 0 in normal builds).
cudaError_t check_word_kernels(unsigned *line);
cudaError_t check_word_batch(unsigned *line);
// Launches one kernel whose check fails on purpose (checked builds only).
cudaError_t launch_check_selftest(cudaStream_t stream);

// Random-number recipe of a mode: 1 = 24-bit uniforms in FP64 arithmetic.
template <int MODE> struct ModeRecipe { static constexpr int value = MODE == kModeFP64U24 ? 1 : 0; };

// Device copy of one level's sums; same layout as mlkd_level_stats.
struct DevLevelStats {
    long long n;
    double sy, sy2, sqf, sqf2, sqc, sqc2;
    unsigned long long events_f, events_c;
};

// Derived constants of one level in one precision, computed on the host so
// that the kernel reads them from the parameter bank with no arithmetic.
template <typename Real> struct BgParams {
    Real R, invR, mu, sigma;
    Real two_c2;      // 2 sigma^2 / R^2
    Real dt, Rdt, inv_Rdt;
    Real lo, hi, inv_h;
};

// Parameters of one pair-kernel launch (passed by value as __grid_constant__).
// Idle lanes a warp of the pair kernels gathers before it sums their finished
// pairs and starts new ones in one pass (the batched form can override it).
constexpr int kRefillMin = 8;

struct PairLaunch {
    double R, mu, sigma, dt;   // background and fine step of this level
    double lo, hi, h;          // histogram range [lo, hi) and bin width
    int32_t n;                 // fine steps to T
    int32_t M;                 // refinement factor
    int32_t periodic;          // F = (x mod 1)^2 and wrapped bins
    int32_t init;              // 0: x0 = 0; 1: cosine density
    int32_t nbins;             // 0: no histogram
    uint32_t word2;            // level << 24 (pair_hi xor'ed in per pair)
    uint32_t request;
    int32_t fkind;             // F: 0 x^2, 1 (x mod 1)^2, 2 x
    int32_t background;        // 0 homogeneous, 1 B1, 2 B2 (heterogeneous kernel)
    double x0;                 // start of every path (init 2)
    double bg_b, bg_a_left, bg_a_right;   // R(x) = b (1 + a_l max(1-x,0) + a_r max(x-1,0))
    PhiloxKeys keys;
    BgParams<double> bd;
    BgParams<float> bf;
    unsigned long long first_pair, n_pairs, pairs_per_warp;
    double *partials;                  // [gridDim.x][kPartialWords]
    int32_t partial_rows;              // rows the partials buffer holds (>= gridDim.x)
    unsigned long long *hist;          // [3][nbins] fine, coarse, both; or null
    double *dbg_xf, *dbg_xc;           // optional per-pair outputs
    int32_t *dbg_kf, *dbg_kc;
};

struct KernelInfo {
    int blocks_per_sm;
};

// Kernel-variant occupancy (blocks per SM with kThreads threads).
cudaError_t pair_kernel_info(int mode, bool coupled, int nbins, KernelInfo *out, int background = 0);

// Launches the pair kernel on `grid` blocks.
cudaError_t launch_pair_kernel(int mode, bool coupled, const PairLaunch &p, int grid,
                               cudaStream_t stream);

// Sums `nblocks` partial rows in a fixed order into *out (n = n_pairs).  If
// acc != null also adds them to *acc.
cudaError_t launch_finalize(const double *partials, int nblocks, long long n_pairs,
                            DevLevelStats *out, DevLevelStats *acc, cudaStream_t stream);

// Output of the on-device sample-count controller (eqs. Nopt1/Noptj).
struct DevControl {
    double estimate, variance;
    double var_level[16];
    double cost_level[16];
    long long target[16];
};

// From the accumulated level sums (and histograms, for a density QoI),
// computes V_l, C_l, N_l*, the estimate and its variance in FP64.
cudaError_t launch_controller(const DevLevelStats *acc, const unsigned long long *hist_acc,
                              int n_levels, int nbins, double h, int density_qoi, double tol,
                              DevControl *out, cudaStream_t stream);

// Coarse random numbers (nu~, E~, chi~) of the first per_pair coarse steps of
// each pair of a coupled level (validation); count[j] = coarse steps of pair j.
cudaError_t launch_coarse_draws(int mode, const PairLaunch &p, int per_pair, double *nu, double *E,
                                double *chi, int32_t *count, cudaStream_t stream);

// FP32 variate transforms of n words (validation).
cudaError_t launch_debug_kd(int fp64, double R, double mu, double sigma, const double *theta,
                            const double *dv, unsigned long long n, double *a, double *d, double *hs,
                            double *om, double *bh2, cudaStream_t stream);
cudaError_t launch_debug_transforms(const uint32_t *words, unsigned long long n, float *log_u,
                                    float *sn, float *cs, cudaStream_t stream);

// Adds hist [3*nbins] into acc [3*nbins] (integer).
cudaError_t launch_hist_accumulate(const unsigned long long *hist, unsigned long long *acc,
                                   int count, cudaStream_t stream);

}  // namespace mlkd
