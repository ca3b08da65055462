// mlkd_host.h -- host-side internals shared by the C ABI translation units:
// the context over the caller's arena, problem validation and the launch
// parameters of one level.
#pragma once

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "mlkd_internal.h"
#include "../../include/mlkd.h"

namespace mlkd {

// NVTX range over a host call (tracing; header-only NVTX, a no-op unless a
// profiler or tracer is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr int kMaxBlocks = 4096;                  // grid cap of the pair kernel
constexpr size_t kAlign = 256;
constexpr uint32_t kWeylA = 0x9E3779B9u;         // Philox key increments (SC'11)
constexpr uint32_t kWeylB = 0xBB67AE85u;
constexpr int kTimingRing = 64;

// Canary bytes after each arena region in the debug build (MLKD_CHECKS):
// written when the region is set up, compared after each synchronising call.
#ifdef MLKD_CHECKS
constexpr size_t kGuardBytes = 256;
#else
constexpr size_t kGuardBytes = 0;
#endif
constexpr unsigned char kGuardByte = 0xA5;
constexpr int kMaxGuards = 16;

// Arena layout of the base workspace (offsets in bytes).
struct Layout {
    size_t partials, tmp_stats, acc_stats, tmp_hist, acc_hist, control, total;
    size_t guard[kMaxGuards];    // canary offsets (debug build)
    int n_guard;
};

// Derived, validated description of a problem.
struct Derived {
    double R, sigma, mu;
    long long n0;          // T / dt0
    int mode;
    int background;        // mlkd_background
    bool per_level_only;   // a problem the batched and serving forms do not run (the
                           // heterogeneous backgrounds run batched, but not served)
    bool periodic;
    double lo, hi, h;
    int J;                 // estimator levels
    int lev[MLKD_MAX_LEVELS];   // fine level of estimator level j
    int Mj[MLKD_MAX_LEVELS];    // coarsening to the previous estimator level (j >= 1)
};

size_t align_up(size_t v);
Layout arena_layout();
bool validate(const mlkd_problem *p, Derived *d);
long long ipow(long long b, int e);
void fill_launch(const mlkd_problem *p, const Derived &d, int level, uint64_t first, uint64_t count,
                 PairLaunch *P);

struct BatchCache;   // instantiated batch graph (mlkd_batch.cu)
struct Server;       // serving form (mlkd_batch.cu)

}  // namespace mlkd

struct mlkd_context;

namespace mlkd {
void batch_release(mlkd_context *ctx);   // frees the batch graph cache (host side)
void server_release(mlkd_context *ctx);  // stops a running server
mlkd_status harvest_timing(mlkd_context *ctx);
// Debug build: fills / compares the canaries at these arena offsets
// (MLKD_EINTERNAL if a byte changed); no-ops in normal builds.
mlkd_status guards_write(char *arena, const size_t *guard, int n, cudaStream_t s);
mlkd_status guards_check(const char *arena, const size_t *guard, int n);
// Debug builds: MLKD_EINTERNAL if a device check failed since the last call
// (the caller has synchronised); MLKD_OK always in normal builds.
mlkd_status device_checks();
}

struct mlkd_context {
    int device;
    bool timing;
    int pending;
    cudaEvent_t ev_start[mlkd::kTimingRing], ev_stop[mlkd::kTimingRing];
    bool events_made;
    unsigned long long launches, other_launches;
    double kernel_ms;
    int sm_count;
    char *arena;
    size_t arena_bytes;
    mlkd::Layout L;
    double *partials;
    mlkd::DevLevelStats *tmp_stats, *acc_stats;
    unsigned long long *tmp_hist, *acc_hist;
    mlkd::DevControl *control;
    mlkd::BatchCache *batch;    // lazily created by the batched form
    mlkd::Server *server;       // running serving form, or null
    // the per-level estimate runs the levels of a round on these streams
    // (created on first use), forked from and joined to the caller's stream
    bool streams_made;
    cudaStream_t level_stream[MLKD_MAX_LEVELS];
    cudaEvent_t level_done[MLKD_MAX_LEVELS];
    cudaEvent_t round_start;
};

#define MLKD_CUDA(call)                                  \
    do {                                                 \
        if ((call) != cudaSuccess) return MLKD_ECUDA;    \
    } while (0)
