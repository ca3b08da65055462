// mlkd_batch.cu -- batched form: many independent MLMC estimates advanced by
// one persistent pair kernel whose warps claim chunks from device queues.
//
// Device state (in the context arena, after the base workspace):
//   ReqDesc[max_requests]   problem of each request slot (host-written)
//   ReqState[max_requests]  level sums, pairs scheduled, round bookkeeping
//   Chunk[slots][kSlotChunks]  (request, level, first pair, count); each
//                           request slot owns its range of chunk ids
//   rows[...][8]            one row of sums per chunk (fixed-order input of
//                           the finalize)
//   q/l/p id rings          queues of chunk ids: main, long chunks, small rounds
//   hist[max_requests][16][3][max_nbins]  fine/coarse/both bin counts
//   BatchCtl                queue counters, live and running requests, events,
//                           the error flag
//   slice state             stored chunk positions and lane states of sliced
//                           launches
//
// One iteration of the loop: the scheduler kernel (one warp per request
// slot) admits new requests and frees cancelled ones; the pair kernel runs
// one slice, and the warp that finishes a round's last chunk finalizes it,
// runs the FP64 controller of Sec. 4.1 and publishes the next round (finest
// level first) on the spot; the bookkeeping kernel sets the live count and,
// in the graph form, the while-node condition.
#include <condition_variable>
#include <cstdio>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mlkd_host.h"
#include "mlkd_hetero.cuh"
#include "mlkd_pair.cuh"
#include "mlkd_warp_pair.cuh"

namespace mlkd {

constexpr int kBL = MLKD_MAX_LEVELS;            // levels per request
constexpr int kMaxChunksPerJob = 2048;           // chunks per level and round, at most
constexpr int kChunkQuantum = 32;                // chunk sizes are multiples of one pair per lane
constexpr int kTargetIters = 1024;               // target warp iterations per chunk
constexpr double kPairStartIters = 2.0;          // start + summation of a pair, in event iterations
constexpr long long kMaxChunkPairs = 1LL << 22;  // pairs per chunk at most
constexpr long long kMaxChunkGrow = 8;           // chunk enlargement to fit a round, at most
constexpr long long kRoundChunks = (long long)kBL * kMaxChunksPerJob;  // chunks of one request per round
// chunk ids owned by one request slot: one round's chunks
constexpr long long kSlotChunks = kRoundChunks;
constexpr int kPublishSpins = 1 << 22;           // bounded wait for earlier reservations to publish
constexpr double kSmallRoundEvents = 2e8;        // predicted KD events of a round that goes first (about 2 ms)
constexpr int kWarpPairEvents = 1024;            // events per pair from which a pair runs on a whole warp
constexpr int kIdleSpins = 4096;                 // bounded wait for new work: sleeps of up to 64 us, about 0.25 s

struct ReqDesc {
    BgParams<double> bd[kBL];
    BgParams<float> bf[kBL];
    long long n_fixed[kBL];
    double tol, h;
    int32_t n_level[kBL];
    int32_t M_level[kBL];       // coarsening to the previous estimator level
    int32_t level_of[kBL];      // fine level of estimator level j (Philox counter word)
    int32_t L, M, init, nbins, periodic, density, n_warmup, use_fixed;
    uint32_t request;
    int32_t fkind;              // QoI F: 0 x^2, 1 (x mod 1)^2, 2 x
    int32_t background, pad_;   // mlkd_background
    double x0, bg_b, bg_a_left, bg_a_right;   // heterogeneous backgrounds
};

struct ReqState {
    DevLevelStats acc[kBL];
    long long have[kBL];
    long long job_cb[kBL];      // first chunk id of this round's job per level
    long long job_count[kBL];   // pairs of this round's job per level
    int32_t job_nch[kBL];       // chunks of this round's job per level (0: none)
    int32_t status;             // 0 free, 1 admitted, 2 running, 3 done
    int32_t pending;            // chunks of the open round not yet finished
    int32_t rounds;
    int32_t pad_;
    double estimate, variance;
    double var_level[kBL], cost_level[kBL];
    long long target[kBL];
    long long job_ch[kBL];      // pairs per chunk of this round's job per level
    int32_t job_queue[kBL];     // queue of the level's chunks: 0 main, 1 long chunks, 2 small rounds
    int32_t job_warp[kBL];      // 1: the level's pairs run one per warp
    long long plan_want[kBL];   // planning scratch: pairs wanted per level
    double plan_epp[kBL];       // planning scratch: events per pair per level
    int32_t counted;            // 1: counted in BatchCtl::running
    int32_t pad2_;
};

struct Chunk {
    int32_t req, level;
    unsigned long long first;
    int32_t count;
    int32_t warp_pair;           // 1: one pair per warp, 32 events per step
};

// Work queues are rings of chunk ids.  A producer reserves places at *_resv,
// writes the ids, publishes them by moving *_tail in reservation order, and
// then adds them to *_avail.  A consumer first takes one unit of *_avail (so
// that it never runs past the published ids), then its place from *_head;
// both are plain atomic adds, which stay fast with thousands of claimers.
struct BatchCtl {
    unsigned long long q_head, q_tail, q_resv;
    unsigned long long l_head, l_tail, l_resv;   // chunks longer than a target slice
    unsigned long long p_head, p_tail, p_resv;   // rounds of little predicted work, drained first
    int32_t q_avail, l_avail;   // published ids not yet claimed
    int32_t p_avail, pad_;
    int32_t live;
    int32_t iterations;         // loop iterations run (three kernel launches each)
    unsigned long long events;  // fine + coarse events merged into request sums so far
    unsigned long long events_done;  // fine + coarse events of finished chunks so far
    int32_t running;            // requests with a round in flight
    int32_t error;              // 1: a publication wait ran out; 2: a consistency check failed
};
// the server reads events .. error in one copy
static_assert(offsetof(BatchCtl, error) == offsetof(BatchCtl, events) + 20, "BatchCtl tail layout");

// Persisted state of one warp between slices: the chunk it is working on.
struct WarpHdr {
    int32_t valid;
    int32_t pad_;
    unsigned long long c;        // chunk id
    unsigned long long next;     // next unassigned pair of the chunk
};

struct BatchLaunch {
    const ReqDesc *req;
    ReqState *state;
    Chunk *chunks;               // [slots][kSlotChunks]
    double *rows;                // [slots][kSlotChunks][kPartialWords]
    unsigned long long *hist;
    BatchCtl *ctl;
    WarpHdr *hdr;                // [grid warps]
    int32_t *status_out;         // [slots]: status after the scheduler (host-readable copy)
    uint32_t *lane_words;        // [words][grid lanes]: pair states and sums per lane
    int32_t lane_word_count;     // words allocated per lane
    unsigned long long *q_ids;   // [ring]: queue of chunk ids
    unsigned long long *l_ids;   // [ring]: queue of long chunks' ids
    unsigned long long *p_ids;   // [ring]: queue of the chunks of small rounds
    unsigned long long ring_mask;
    int32_t max_nbins;
    int32_t slice_iters;
    int32_t n_slots;
    int32_t refill_min;          // idle lanes a warp gathers before it hands them started pairs
    int32_t publish_spins;       // bound of the publication wait
    int32_t warp_pair_events;    // levels with at least this many events per pair run one pair per warp (0: never)
    int32_t dbg_req;             // per-pair readout of request slot dbg_req, estimator level
    int32_t dbg_level;           // dbg_level (-1: none)
    int32_t pad_;
    unsigned long long dbg_n;    // entries of the readout arrays
    double *dbg_xf, *dbg_xc;
    int32_t *dbg_kf, *dbg_kc;
    PhiloxKeys keys;
};

constexpr int kMaxPPT = 8;
// Idle lanes a warp gathers before it hands them started pairs from its pool
// (measured on the periodic benchmark: 2 and 3 best, 1 and 4 within 1 %).
constexpr int kBatchRefillMin = 2;
constexpr size_t kMaxLanes = 256ull * 16 * kThreads;   // lane slots: up to 256 SMs x 16 blocks

// Lane words of T, stored word-major so that a warp's 32 lanes write 32
// consecutive words.
template <typename T> __device__ __forceinline__ void put_words(const T &v, uint32_t *base, size_t stride, int &w)
{
    static_assert(sizeof(T) % 4 == 0, "lane state must be whole words");
    uint32_t tmp[sizeof(T) / 4];
    memcpy(tmp, &v, sizeof(T));
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 4); ++i) base[(size_t)(w + i) * stride] = tmp[i];
    w += (int)(sizeof(T) / 4);
}

template <typename T> __device__ __forceinline__ void get_words(T &v, const uint32_t *base, size_t stride, int &w)
{
    uint32_t tmp[sizeof(T) / 4];
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 4); ++i) tmp[i] = base[(size_t)(w + i) * stride];
    memcpy(&v, tmp, sizeof(T));
    w += (int)(sizeof(T) / 4);
}

// Per-warp pools of the one-pair-per-lane loop.  New pairs are started 32 at
// a time in one pass with every lane busy (Philox block 0, the initial
// position, the first flight) and handed out as lanes fall idle; finished
// pairs are queued and summed 32 at a time.  A lane whose pair reaches T thus
// takes a new one at once, and the start and summation paths no longer run
// for only the few lanes that finished in the same iteration.
template <typename Real> struct StartPool {
    Real x0[32], v0[32], q0[32];
    Real e0[32];                     // E_0 (heterogeneous backgrounds)
    int32_t off[32];                 // pair index - the chunk's first pair index
};
template <typename Real> struct FinishPool {
    Real xf[64], xc[64];             // both paths at T
    uint32_t kf[64], kc[64];         // fine and coarse events
};
// A lane's share of its warp's pools in a stored slice.
template <typename Real> struct PoolWords {
    Real x0, v0, q0, e0;
    int32_t off;
    Real xf[2], xc[2];
    uint32_t kf[2], kc[2];
    uint32_t counts;                 // entries: started | handed out << 8 | finished << 16
    uint32_t pad_;
};

// Pair state of the two physics: the homogeneous background (PHYS 0) and the
// heterogeneous backgrounds B1/B2 of Sec. 5 (PHYS 1).
template <typename Real, int PHYS> struct BatchState { typedef PairState<Real> type; };
template <typename Real> struct BatchState<Real, 1> { typedef HetPairState<Real> type; };

template <typename Real, int MODE, int PPT, int PHYS = 0> constexpr int lane_words()
{
    return (int)((PPT * sizeof(typename BatchState<Real, PHYS>::type) + sizeof(PairSums<MODE>) +
                  2 * sizeof(unsigned long long) + sizeof(PoolWords<Real>)) / 4) + 1;
}

// Blocks per SM of the batched pair kernel by pair states per lane.  Five
// 128-thread blocks (96 registers) rather than six: the deep levels' chunks
// are chains of up to 12 288 serial events, and a warp that shares its
// scheduler with fewer warps finishes its chain sooner; measured on the
// periodic benchmark, five balances that against latency hiding best.
template <typename Real, int PPT> struct BatchMinBlocks { static constexpr int value = PPT == 1 ? 5 : PPT == 2 ? 4 : PPT == 4 ? 2 : 1; };
template <int PPT> struct BatchMinBlocks<double, PPT> { static constexpr int value = 1; };

template <typename Real> __device__ __forceinline__ const BgParams<Real> &req_params(const ReqDesc &D, int l);
template <> __device__ __forceinline__ const BgParams<float> &req_params<float>(const ReqDesc &D, int l) { return D.bf[l]; }
template <> __device__ __forceinline__ const BgParams<double> &req_params<double>(const ReqDesc &D, int l) { return D.bd[l]; }

// ---------------------------------------------------------------------------
// Persistent pair kernel.  Each warp works on one chunk at a time, taking
// chunks from the queue until it is empty; a slice advances each warp at most
// slice_iters event iterations (0: no limit), after which the warp stores its
// chunk position, its PPT pair states and its sums and the next slice resumes
// them.  Slicing changes no arithmetic and no order: results are the same for
// every slice length.
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// Rounds of one request, run by one warp: finalize (the round's chunk rows
// into the request's sums, in chunk order), the FP64 controller (eqs.
// Nopt1/Noptj) and the plan of the next round.  The warp that finishes a
// round's last chunk runs them inside the pair kernel, so a request's next
// round starts while other requests' work goes on; the scheduler kernel runs
// the same functions for admissions.  Every decision depends only on the
// request's own sums, so its results are the same alone and in any mix.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long vload64(const unsigned long long *p)
{
    return *(volatile const unsigned long long *)p;
}

// Target chunk size of a level: a multiple of 32 pairs sized for about
// kTargetIters warp iterations.
__device__ long long chunk_target(double events_per_pair)
{
    // a pair costs its events plus its start (draw, initial position) and
    // its summation, about two event iterations together
    const double per_pair = (events_per_pair > 1.0 ? events_per_pair : 1.0) + kPairStartIters;
    double ch = 32.0 * kTargetIters / per_pair;
    long long c = (long long)ch / kChunkQuantum * kChunkQuantum;
    if (c < kChunkQuantum) c = kChunkQuantum;
    if (c > kMaxChunkPairs) c = kMaxChunkPairs;
    return c;
}

// Appends chunk ids [id0, id0 + n) to a queue (whole warp): reserve, write,
// publish in reservation order.  The wait for earlier reservations is
// bounded; running out sets BatchCtl::error, which ends the loop, and leaves
// the ids unpublished (consumers never see places that an earlier, stalled
// reservation may not have written).
__device__ void push_ids(const BatchLaunch &B, unsigned long long *ring, unsigned long long *resv,
                         unsigned long long *tail, int32_t *avail, unsigned long long id0, int n, int lane)
{
    if (n <= 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(resv, (unsigned long long)n);
    base = __shfl_sync(kFullMask, base, 0);
    for (int i = lane; i < n; i += 32) ring[(base + i) & B.ring_mask] = id0 + (unsigned long long)i;
    __threadfence();
    __syncwarp();
    if (lane == 0) {
        int k = 0;
        bool published = true;
        while (atomicCAS(tail, base, base + (unsigned long long)n) != base) {
            if (++k >= B.publish_spins) {
                atomicExch(&B.ctl->error, 1);
                published = false;
                break;
            }
            __nanosleep(32);
        }
        if (published) atomicAdd(avail, n);
    }
    __syncwarp();
}

// Claims the next published id of a queue (one lane); false if there is none.
__device__ bool claim_id(const BatchLaunch &B, int32_t *avail, unsigned long long *head,
                         const unsigned long long *ring, unsigned long long *id)
{
    if (*(volatile int32_t *)avail <= 0) return false;
    if (atomicSub(avail, 1) <= 0) {
        atomicAdd(avail, 1);
        return false;
    }
    const unsigned long long h = atomicAdd(head, 1ull);
    __threadfence();
    *id = vload64(&ring[h & B.ring_mask]);
    return true;
}

__device__ __noinline__ void warp_finalize(const BatchLaunch &B, int r, int lane)
{
    ReqState &S = B.state[r];
    const int nl = B.req[r].L + 1;
    for (int l = 0; l < nl; ++l) {
        const int nch = S.job_nch[l];
        if (nch == 0) continue;
        double v[kPartialWords];
#pragma unroll
        for (int j = 0; j < kPartialWords; ++j) v[j] = 0.0;
        for (int i = lane; i < nch; i += 32) {
            const double *row = B.rows + (size_t)(S.job_cb[l] + i) * kPartialWords;
#pragma unroll
            for (int j = 0; j < kPartialWords; ++j) v[j] += row[j];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int j = 0; j < kPartialWords; ++j) v[j] += __shfl_down_sync(kFullMask, v[j], off);
        __syncwarp();
        if (lane == 0) {
            DevLevelStats &a = S.acc[l];
            a.n += S.job_count[l];
            a.sy += v[0];
            a.sy2 += v[1];
            a.sqf += v[2];
            a.sqf2 += v[3];
            a.sqc += v[4];
            a.sqc2 += v[5];
            const unsigned long long ef = (unsigned long long)llrint(v[6]);
            const unsigned long long ec = (unsigned long long)llrint(v[7]);
            a.events_f += ef;
            a.events_c += ec;
            atomicAdd(&B.ctl->events, ef + ec);
            S.job_nch[l] = 0;
            S.job_count[l] = 0;
        }
        __syncwarp();
    }
}

// Controller after a completed round.  Returns true if another round is
// needed (targets in S.target), false when the request is done.
__device__ __noinline__ bool warp_controller(const BatchLaunch &B, int r, int lane)
{
    ReqState &S = B.state[r];
    const ReqDesc &D = B.req[r];
    const int nl = D.L + 1;
    for (int l = 0; l < nl; ++l) {
        const double n = (double)S.acc[l].n;
        double v = 0.0;
        if (D.density && D.nbins > 0) {
            // sup over bins of the bin indicators' level variance
            const unsigned long long *H = B.hist + ((size_t)r * kBL + l) * 3 * B.max_nbins;
            double m = 0.0;
            for (int b = lane; b < D.nbins; b += 32) {
                const double sy = (double)H[b] - (double)H[D.nbins + b];
                const double sy2 = (double)H[b] + (double)H[D.nbins + b] - 2.0 * (double)H[2 * D.nbins + b];
                const double vb = n >= 2.0 ? (sy2 - sy * sy / n) / (n - 1.0) : 0.0;
                m = fmax(m, vb);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(kFullMask, m, off));
            v = m / (D.h * D.h);
        } else if (n >= 2.0) {
            v = (S.acc[l].sy2 - S.acc[l].sy * S.acc[l].sy / n) / (n - 1.0);
        }
        if (lane == 0) {
            S.var_level[l] = v > 0.0 ? v : 0.0;
            S.cost_level[l] = n > 0.0 ? (double)(S.acc[l].events_f + S.acc[l].events_c) / n : 0.0;
        }
    }
    __syncwarp();
    int more = 0;
    if (lane == 0) {
        double est = 0.0, var = 0.0, total = 0.0;
        for (int l = 0; l < nl; ++l) {
            const double n = (double)S.acc[l].n;
            if (n > 0.0) {
                est += S.acc[l].sy / n;
                var += S.var_level[l] / n;
            }
            total += sqrt(S.var_level[l] * S.cost_level[l]);
        }
        S.estimate = est;
        S.variance = var;
        bool grow = false;
        for (int l = 0; l < nl; ++l) {
            long long target = 0;
            const double vl = S.var_level[l], cl = S.cost_level[l];
            if (!D.use_fixed && vl > 0.0 && cl > 0.0 && D.tol > 0.0) {
                const double tg = ceil(2.0 / (D.tol * D.tol) * sqrt(vl / cl) * total);
                target = tg < 1e15 ? (long long)tg : 1000000000000000LL;
            }
            S.target[l] = target;
            if (target > S.have[l]) grow = true;
        }
        if (!grow || D.use_fixed || S.rounds >= 64) {
            S.status = 3;
            B.status_out[r] = 3;
            if (atomicExch(&S.counted, 0) == 1) atomicSub(&B.ctl->running, 1);
        } else {
            S.rounds += 1;
            more = 1;
        }
    }
    return __shfl_sync(kFullMask, more, 0) != 0;
}

// Plans the next round toward S.target, finest level first, and publishes
// its chunks in the request's own chunk-id range.  A round holds at most
// kMaxChunksPerJob chunks per level: a level that needs more target-size
// chunks gets chunks up to kMaxChunkGrow times larger, and beyond that its
// round is cut and the next round continues with the same targets, so that
// no chunk holds a warp much longer than a target slice however many pairs a
// request asks for.
__device__ __noinline__ void warp_plan(const BatchLaunch &B, int r, int lane)
{
    ReqState &S = B.state[r];
    const ReqDesc &D = B.req[r];
    const int nl = D.L + 1;
    const unsigned long long slot0 = (unsigned long long)r * kSlotChunks;
    if (lane == 0) {
        long long *want = S.plan_want, *tch = S.job_ch;
        double *epps = S.plan_epp;
        for (int l = 0; l < nl; ++l) {
            want[l] = S.target[l] - S.have[l];
            if (want[l] < 0) want[l] = 0;
            double epp = 1.0;
            if (S.acc[l].n > 0) {
                epp = (double)(S.acc[l].events_f + S.acc[l].events_c) / (double)S.acc[l].n;
            } else {
                const double nf = (double)D.n_level[l];
                const double coll = (double)D.bd[l].Rdt * nf + 1.0;
                epp = (coll < nf ? coll : nf) * (l > 0 ? 1.5 : 1.0);
            }
            epps[l] = epp;
            tch[l] = chunk_target(epp);
        }
        int total = 0;
        double work = 0.0;
        for (int l = nl - 1; l >= 0; --l) {
            S.job_nch[l] = 0;
            S.job_count[l] = 0;
            long long count = want[l];
            if (count <= 0) continue;
            // A level whose pairs are long serial chains runs one pair per
            // warp, 32 events per step; its chunks then hold about
            // kTargetIters warp steps of pairs, not a multiple of 32.  (The
            // heterogeneous backgrounds always run one pair per lane.)
            const bool wp = B.warp_pair_events > 0 && epps[l] >= (double)B.warp_pair_events &&
                            D.background == 0;
            if (wp) {
                double c = 32.0 * kTargetIters / (epps[l] + 32.0 * kPairStartIters);
                tch[l] = c < 1.0 ? 1 : (long long)c;
            }
            S.job_warp[l] = wp ? 1 : 0;
            long long ch = tch[l];
            long long nch = (count + ch - 1) / ch;
            if (nch > kMaxChunksPerJob) {
                long long g = (nch + kMaxChunksPerJob - 1) / kMaxChunksPerJob;
                if (g > kMaxChunkGrow) g = kMaxChunkGrow;
                ch *= g;
                nch = (count + ch - 1) / ch;
                if (nch > kMaxChunksPerJob) {
                    nch = kMaxChunksPerJob;
                    count = nch * ch;
                }
            }
            tch[l] = ch;
            S.job_cb[l] = (long long)(slot0 + (unsigned long long)total);
            S.job_nch[l] = (int32_t)nch;
            S.job_count[l] = count;
            // one pair per lane already exceeds a target slice: the long queue
            S.job_queue[l] = epps[l] > (double)kTargetIters ? 1 : 0;
            work += (double)count * epps[l];
            total += (int)nch;
        }
        // A round of little predicted work (a warm-up round, or a request
        // near its tolerance) goes ahead of all other work: under load,
        // cheap requests finish in about their own run time instead of
        // sharing the GPU with every heavy request in flight.
        if (work <= kSmallRoundEvents)
            for (int l = 0; l < nl; ++l) S.job_queue[l] = 2;
        S.pending = total;
        S.status = 2;
    }
    __syncwarp();
    // chunk descriptors, then the ids in the queues (published last)
    for (int l = nl - 1; l >= 0; --l) {
        const int nch = S.job_nch[l];
        const long long ch = S.job_ch[l];
        const long long have = S.have[l];
        for (int i = lane; i < nch; i += 32) {
            const long long first = have + (long long)i * ch;
            long long cnt = have + S.job_count[l] - first;
            if (cnt > ch) cnt = ch;
            Chunk c;
            c.req = r;
            c.level = l;
            c.first = (unsigned long long)first;
            c.count = (int32_t)cnt;
            c.warp_pair = S.job_warp[l];
            B.chunks[S.job_cb[l] + i] = c;
        }
    }
    __syncwarp();
    if (lane == 0)
        for (int l = 0; l < nl; ++l) S.have[l] += S.job_count[l];
    __threadfence();
    __syncwarp();
    for (int l = nl - 1; l >= 0; --l) {
        const int nch = S.job_nch[l];
        if (nch == 0) continue;
        if (S.job_queue[l] == 2)
            push_ids(B, B.p_ids, &B.ctl->p_resv, &B.ctl->p_tail, &B.ctl->p_avail,
                     (unsigned long long)S.job_cb[l], nch, lane);
        else if (S.job_queue[l] == 1)
            push_ids(B, B.l_ids, &B.ctl->l_resv, &B.ctl->l_tail, &B.ctl->l_avail,
                     (unsigned long long)S.job_cb[l], nch, lane);
        else
            push_ids(B, B.q_ids, &B.ctl->q_resv, &B.ctl->q_tail, &B.ctl->q_avail,
                     (unsigned long long)S.job_cb[l], nch, lane);
    }
}

// A round whose last chunk has finished: merge it, then continue a cut round,
// or run the controller and plan the next round (or finish the request).
__device__ __noinline__ void warp_round_complete(const BatchLaunch &B, int r, int lane)
{
    ReqState &S = B.state[r];
    const int nl = B.req[r].L + 1;
    warp_finalize(B, r, lane);
    int cont = 0;
    if (lane == 0)
        for (int l = 0; l < nl; ++l)
            if (S.have[l] < S.target[l]) cont = 1;
    cont = __shfl_sync(kFullMask, cont, 0);
    if (cont || warp_controller(B, r, lane)) warp_plan(B, r, lane);
}

// A lane's running sums of its current chunk.  They change only when a pair
// finishes, so they live in shared memory rather than in registers that the
// event loop needs; 72 bytes per lane keeps bank conflicts at two-way.
template <int MODE> struct LaneSums {
    PairSums<MODE> mom;
    unsigned long long ev_f, ev_c;
    uint32_t pad_[2];
};

// A warp's bookkeeping of its current chunk and pools (all warp-uniform).  It
// lives in shared memory and is read (volatile) where it is used, so that the
// registers of the event loop hold only pair states and level constants.
struct WarpCtx {
    unsigned long long c;            // chunk id
    unsigned long long first, end;   // the chunk's pair range
    unsigned long long next;         // next pair of the chunk to start
    double blo, bhi, bh;             // histogram range and bin width (FP64 state)
    float blo_f, bhi_f, binv_h_f;    // the same for FP32 state
    int32_t req, level, warp_pair, nbins, per, fkind;
    int32_t sp_n, sp_i, fp_n;        // start pool: started, handed out; finish pool: queued
};

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename Real, int MODE, int PPT, int PHYS = 0>
__global__ void __launch_bounds__(kThreads, (BatchMinBlocks<Real, PPT>::value))
batch_pair_kernel(const __grid_constant__ BatchLaunch B)
{
    static_assert(PHYS == 0 || PPT == 1, "the heterogeneous backgrounds run one pair per lane");
    constexpr int RECIPE = ModeRecipe<MODE>::value;
    extern __shared__ unsigned int s_hist_all[];        // [warps][3 * max_nbins]
    __shared__ LaneSums<MODE> s_sums[kThreads];
    __shared__ StartPool<Real> s_start[kWarpsPerBlock];
    __shared__ FinishPool<Real> s_finish[kWarpsPerBlock];
    __shared__ WarpCtx s_ctx[kWarpsPerBlock];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const size_t gw = (size_t)blockIdx.x * kWarpsPerBlock + warp;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    uint32_t *lw = B.lane_words + gw * 32 + lane;
    unsigned int *wh = s_hist_all + (size_t)warp * 3 * B.max_nbins;
    WarpHdr *hdr = B.hdr + gw;

    // the stored slice state of this instantiation fits the words per lane
    if (!MLKD_DCHECK(lane_words<Real, MODE, PPT, PHYS>() <= B.lane_word_count)) {
        if (threadIdx.x == 0) atomicExch(&B.ctl->error, 2);
        return;
    }
    int valid = hdr->valid;
    int iters = 0;
    int idle = 0;
    // event iterations of this launch before the warp stores its state; an
    // unbounded launch stops only if one warp ever reached 2^31 - 1 of them
    // (it would then store its state like a slice, and the next launch resumes)
    const int iter_limit = B.slice_iters > 0 ? B.slice_iters : 0x7fffffff;
    StartPool<Real> &SP = s_start[warp];
    FinishPool<Real> &FP = s_finish[warp];
    // warp-uniform bookkeeping, read from shared memory where it is needed
    volatile WarpCtx &X = s_ctx[warp];
    X.c = hdr->c;
    X.next = hdr->next;
    X.sp_n = 0;
    X.sp_i = 0;
    X.fp_n = 0;
    __syncwarp();

    LevelCtx<Real> L;
    HetLevel<Real> H;           // PHYS 1: the level in the heterogeneous background
    bool coupled = false;
    typename BatchState<Real, PHYS>::type st[PPT];
    bool active[PPT];           // the lane's pair has events left
    bool done[PPT];             // the lane holds a pair that reached T, not yet queued for summing
    PairSums<MODE> &mom = s_sums[threadIdx.x].mom;
    unsigned long long &ev_f_sum = s_sums[threadIdx.x].ev_f;
    unsigned long long &ev_c_sum = s_sums[threadIdx.x].ev_c;

    auto load_chunk = [&]() {
        const Chunk ch = B.chunks[X.c];
        const ReqDesc *D = &B.req[ch.req];
        const int level = ch.level;
        const int nbins = D->nbins;
        coupled = level > 0;
        __syncwarp();
        X.req = ch.req;
        X.level = level;
        X.first = ch.first;
        X.end = ch.first + (unsigned long long)ch.count;
        X.warp_pair = ch.warp_pair;
        X.nbins = nbins;
        X.per = D->periodic != 0;
        X.fkind = D->fkind;
        {
            const BgParams<Real> &bp = req_params<Real>(*D, level);
            L.bg.R = bp.R;
            L.bg.invR = bp.invR;
            L.bg.mu = bp.mu;
            L.bg.sigma = bp.sigma;
            L.bg.two_c2 = bp.two_c2;
            L.bg.dt = bp.dt;
            L.bg.Rdt = bp.Rdt;
            L.bg.inv_Rdt = bp.inv_Rdt;
            L.n = D->n_level[level];
            L.M = D->M_level[level];
            L.divM.init(L.M);
            L.init = D->init;
            L.word2 = (uint32_t)D->level_of[level] << 24;
            L.request = D->request;
            if constexpr (PHYS == 1) {
                H.bg.b = (Real)D->bg_b;
                H.bg.a_left = (Real)D->bg_a_left;
                H.bg.a_right = (Real)D->bg_a_right;
                H.bg.dt = bp.dt;
                H.n = L.n;
                H.M = L.M;
                H.divM = L.divM;
                H.x0 = (Real)D->x0;
                H.word2 = L.word2;
                H.request = L.request;
            }
            X.blo = D->bd[level].lo;
            X.bhi = D->bd[level].hi;
            X.bh = D->h;
            X.blo_f = D->bf[level].lo;
            X.bhi_f = D->bf[level].hi;
            X.binv_h_f = D->bf[level].inv_h;
        }
        for (int i = lane; i < 3 * nbins; i += 32) wh[i] = 0u;
        __syncwarp();
    };
    auto flush_hist = [&]() {
        __syncwarp();
        const int nbins = X.nbins;
        if (nbins > 0) {
            unsigned long long *gh = B.hist + ((size_t)X.req * kBL + X.level) * 3 * B.max_nbins;
            for (int i = lane; i < 3 * nbins; i += 32) {
                const unsigned int v = wh[i];
                if (v) atomicAdd(&gh[i], (unsigned long long)v);
            }
        }
        __syncwarp();
    };
    // the sums, event counts and histogram counts of one pair at T
    auto account = [&](Real xf, Real xc, uint32_t kf, uint32_t kc) {
        add_pair_fk(mom, xf, xc, coupled, X.fkind);
        ev_f_sum += kf;
        ev_c_sum += kc;
        const int nbins = X.nbins;
        if (nbins > 0 && MLKD_DCHECK(nbins <= B.max_nbins)) {
            Bins bins;
            bins.lo = X.blo;
            bins.hi = X.bhi;
            bins.h = X.bh;
            bins.lo_f = X.blo_f;
            bins.hi_f = X.bhi_f;
            bins.inv_h_f = X.binv_h_f;
            bins.nbins = nbins;
            bins.periodic = X.per != 0;
            const int bf = bins(xf);
            if (bf >= 0 && MLKD_DCHECK(bf < nbins)) atomicAdd(&wh[bf], 1u);
            if (coupled) {
                const int bc = bins(xc);
                if (!MLKD_DCHECK(bc < nbins)) return;
                if (bc >= 0) atomicAdd(&wh[nbins + bc], 1u);
                if (bc >= 0 && bc == bf) atomicAdd(&wh[2 * nbins + bf], 1u);
            }
        }
    };
    // validation readout: one pair's final state, by its pair index
    auto dbg_record = [&](unsigned long long p, Real xf, Real xc, uint32_t kf, uint32_t kc) {
        if (B.dbg_xf && X.req == B.dbg_req && X.level == B.dbg_level && p < B.dbg_n) {
            B.dbg_xf[p] = (double)xf;
            B.dbg_xc[p] = coupled ? (double)xc : 0.0;
            B.dbg_kf[p] = (int32_t)kf;
            B.dbg_kc[p] = (int32_t)kc;
        }
    };
    auto pair_index = [&](const auto &q) {
        return ((unsigned long long)(q.word2 ^ L.word2) << 32) | q.pair_lo;
    };
    // the physics' steps: final drift to T and one event
    auto drift = [&](int j) {
        if constexpr (PHYS == 1)
            het_pair_drift<Real>(st[j], H, coupled);
        else
            pair_drift<Real, 2>(st[j], L, coupled);
    };
    auto event = [&](int j) -> bool {
        if constexpr (PHYS == 1)
            return het_pair_event<Real, RECIPE>(st[j], H, B.keys, coupled);
        else
            return pair_event<Real, 2, RECIPE>(st[j], L, B.keys, coupled);
    };
    auto finish = [&](int j) {
        drift(j);
        const Real xc = coupled ? st[j].xc : Real(0);
        account(st[j].xf, xc, st[j].k, st[j].evc);
        dbg_record(pair_index(st[j]), st[j].xf, xc, st[j].k, st[j].evc);
        done[j] = false;
    };
    // Sum the first cnt entries of the finish pool (lane i takes entry i) and
    // move the rest to the front.  All lanes call it.
    auto fp_process = [&](int cnt) {
        __syncwarp();
        if (!MLKD_DCHECK(cnt >= 0 && cnt <= 32)) cnt = 0;
        if (lane < cnt) account(FP.xf[lane], FP.xc[lane], FP.kf[lane], FP.kc[lane]);
        int rest = X.fp_n - cnt;
        if (!MLKD_DCHECK(rest >= 0 && rest <= 32)) rest = 0;
        Real a = Real(0), b = Real(0);
        uint32_t ka = 0u, kb = 0u;
        if (lane < rest) {
            a = FP.xf[cnt + lane];
            b = FP.xc[cnt + lane];
            ka = FP.kf[cnt + lane];
            kb = FP.kc[cnt + lane];
        }
        __syncwarp();
        if (lane < rest) {
            FP.xf[lane] = a;
            FP.xc[lane] = b;
            FP.kf[lane] = ka;
            FP.kc[lane] = kb;
        }
        X.fp_n = rest;
        __syncwarp();
    };
    // Queue the pairs of the lanes with f set, in lane order; sum a full
    // pool of 32.  All lanes call it.
    auto fp_push = [&](bool f, Real xf, Real xc, uint32_t kf, uint32_t kc) {
        const unsigned m = __ballot_sync(kFullMask, f);
        const int n0 = X.fp_n;
        if (f) {
            int i = n0 + __popc(m & lanemask_lt());
            if (!MLKD_DCHECK(i < 64)) i = 63;
            FP.xf[i] = xf;
            FP.xc[i] = xc;
            FP.kf[i] = kf;
            FP.kc[i] = kc;
        }
        __syncwarp();
        X.fp_n = n0 + __popc(m);
        __syncwarp();
        if (n0 + __popc(m) >= 32) fp_process(32);
    };
    // Start the next min(32, end - next) pairs of the chunk, one per lane.  A
    // pair with no collision before T is finished at once (both paths drift
    // to T); the others go to the start pool in pair order.  All lanes call
    // it, with the start pool empty.
    auto refill = [&]() {
        __syncwarp();
        const unsigned long long nx = X.next, first = X.first;
        const unsigned long long rem = X.end - nx;
        const int nav = rem < 32ull ? (int)rem : 32;
        const unsigned long long pr = nx + (unsigned long long)lane;
        const bool have = lane < nav;
        Real x0 = Real(0), v0 = Real(0), q0 = Real(0), e0 = Real(0);
        if (have) {
            if constexpr (PHYS == 1) {
                x0 = H.x0;
                het_start_values<Real, RECIPE>(v0, e0, q0, pr, H, B.keys);
            } else {
                pair_start_values<Real, RECIPE>(x0, v0, q0, pr, L, B.keys);
            }
        }
        const bool dead = have && !(q0 < (Real)L.n);
        Real xT = Real(0);
        if (dead) {
            xT = x0 + v0 * ((Real)L.n * L.bg.dt);          // pair_drift from t = 0
            dbg_record(pr, xT, xT, 0u, 0u);
        }
        fp_push(dead, xT, coupled ? xT : Real(0), 0u, 0u);
        const bool live = have && !dead;
        const unsigned lm = __ballot_sync(kFullMask, live);
        if (live) {
            const int i = __popc(lm & lanemask_lt());
            SP.x0[i] = x0;
            SP.v0[i] = v0;
            SP.q0[i] = q0;
            SP.e0[i] = e0;
            SP.off[i] = (int32_t)(pr - first);
        }
        __syncwarp();
        X.sp_n = __popc(lm);
        X.sp_i = 0;
        X.next = nx + (unsigned long long)nav;
        __syncwarp();
    };
    auto put_pools = [&](int &w) {
        PoolWords<Real> pw;
        pw.x0 = SP.x0[lane];
        pw.v0 = SP.v0[lane];
        pw.q0 = SP.q0[lane];
        pw.e0 = SP.e0[lane];
        pw.off = SP.off[lane];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            pw.xf[h] = FP.xf[32 * h + lane];
            pw.xc[h] = FP.xc[32 * h + lane];
            pw.kf[h] = FP.kf[32 * h + lane];
            pw.kc[h] = FP.kc[32 * h + lane];
        }
        pw.counts = (uint32_t)X.sp_n | ((uint32_t)X.sp_i << 8) | ((uint32_t)X.fp_n << 16);
        pw.pad_ = 0u;
        put_words(pw, lw, stride, w);
    };
    auto get_pools = [&](int &w) {
        PoolWords<Real> pw;
        get_words(pw, lw, stride, w);
        SP.x0[lane] = pw.x0;
        SP.v0[lane] = pw.v0;
        SP.q0[lane] = pw.q0;
        SP.e0[lane] = pw.e0;
        SP.off[lane] = pw.off;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            FP.xf[32 * h + lane] = pw.xf[h];
            FP.xc[32 * h + lane] = pw.xc[h];
            FP.kf[32 * h + lane] = pw.kf[h];
            FP.kc[32 * h + lane] = pw.kc[h];
        }
        __syncwarp();
        X.sp_n = (int)(pw.counts & 0xffu);
        X.sp_i = (int)((pw.counts >> 8) & 0xffu);
        X.fp_n = (int)((pw.counts >> 16) & 0xffu);
        __syncwarp();
    };

    if (valid) {                                      // resume the stored chunk
        load_chunk();
        int w = 0;
#pragma unroll
        for (int j = 0; j < PPT; ++j) get_words(st[j], lw, stride, w);
        get_words(mom, lw, stride, w);
        get_words(ev_f_sum, lw, stride, w);
        get_words(ev_c_sum, lw, stride, w);
        uint32_t bits;
        get_words(bits, lw, stride, w);
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            active[j] = (bits >> j) & 1u;
            done[j] = (bits >> (kMaxPPT + j)) & 1u;
        }
        get_pools(w);
    }

    for (;;) {
        if (!valid) {
            if (iters >= iter_limit) break;
            // Claim order: chunks of small rounds, then chunks whose single
            // pairs outlast a target slice (deep levels, so that the longest
            // serial work starts earliest), then the rest.  With nothing published, a warp of an
            // unbounded launch waits (a bounded time) while some request
            // still has a round in flight: the warp finishing that round
            // publishes the next one.  In a sliced launch it leaves at once;
            // the next slice picks up what was published meanwhile.
            unsigned long long cn = 0;
            int got = 0;
            if (lane == 0) {
                got = claim_id(B, &B.ctl->p_avail, &B.ctl->p_head, B.p_ids, &cn);
                if (!got) got = claim_id(B, &B.ctl->l_avail, &B.ctl->l_head, B.l_ids, &cn);
                if (!got) got = claim_id(B, &B.ctl->q_avail, &B.ctl->q_head, B.q_ids, &cn);
            }
            got = __shfl_sync(kFullMask, got, 0);
            if (!got) {
                int stop = 0;
                ++idle;
                if (lane == 0)
                    stop = B.slice_iters > 0 || *(volatile int32_t *)&B.ctl->running == 0 ||
                           *(volatile int32_t *)&B.ctl->error != 0 || idle >= kIdleSpins;
                if (__shfl_sync(kFullMask, stop, 0)) break;
                // back off to sleeps of 64 us, so that waiting warps take
                // almost no issue slots from the warps still at work
                __nanosleep(1000u << (idle < 6 ? idle : 6));
                continue;
            }
            idle = 0;
            const unsigned long long c = __shfl_sync(kFullMask, cn, 0);
            {
                // Consistency checks of the claimed id and its descriptor
                // (cheap, once per chunk): a failure stops the loop with
                // error 2 instead of reading outside the batch region.
                bool bad = c >= (unsigned long long)B.n_slots * kSlotChunks;
                if (!bad) {
                    const Chunk q = B.chunks[c];
                    bad = q.req < 0 || q.req >= B.n_slots || q.level < 0 || q.level >= kBL ||
                          q.count <= 0 || q.level > B.req[q.req].L;
                }
                if (bad) {
                    if (lane == 0) atomicExch(&B.ctl->error, 2);
                    break;
                }
            }
            {
                // a chunk of a cancelled request is dropped unprocessed
                const Chunk peek = B.chunks[c];
                if (*(volatile int32_t *)&B.state[peek.req].status == 4) {
                    if (lane == 0) atomicSub(&B.state[peek.req].pending, 1);
                    continue;
                }
            }
            X.c = c;
            __syncwarp();
            load_chunk();
            X.next = X.first;
            X.sp_n = 0;
            X.sp_i = 0;
            X.fp_n = 0;
            __syncwarp();
            mom.zero();
            ev_f_sum = 0;
            ev_c_sum = 0;
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                active[j] = false;
                done[j] = false;
                st[j].fresh = true;
            }
            valid = 1;
        }
        bool chunk_done = false;
        if (PHYS == 0 && X.warp_pair) {
          if constexpr (PHYS == 0) {
            // One pair per warp: every lane holds the pair's state, lane j
            // takes its event k + 1 + j; the pair's QoI is summed by lane
            // (pair index mod 32).
            for (;;) {
                if (iters >= iter_limit) break;
                if (done[0]) {
                    if (lane == (int)(st[0].pair_lo & 31u)) finish(0);
                    done[0] = false;
                }
                if (!active[0]) {
                    const unsigned long long nx = X.next;
                    if (nx >= X.end) {
                        chunk_done = true;
                        break;
                    }
                    if (pair_start<Real, 2, ModeRecipe<MODE>::value>(st[0], nx, L, B.keys, coupled))
                        done[0] = true;
                    else
                        active[0] = true;
                    __syncwarp();
                    X.next = nx + 1;
                    __syncwarp();
                    continue;
                }
                if (warp_pair_step<Real, ModeRecipe<MODE>::value>(st[0], L, B.keys, coupled, lane)) {
                    active[0] = false;
                    done[0] = true;
                }
                ++iters;
            }
          }
        } else
        for (;;) {
            // the budget is checked before the pools are touched, so a
            // resumed slice runs exactly the sequence an unsliced run would
            if (iters >= iter_limit) break;
#pragma unroll
            for (int j = 0; j < PPT; ++j) {
                // pairs that reached T in the last iteration: to the finish pool
                if (__any_sync(kFullMask, done[j])) {
                    Real xf = Real(0), xc = Real(0);
                    if (done[j]) {
                        drift(j);
                        xf = st[j].xf;
                        xc = coupled ? st[j].xc : Real(0);
                        dbg_record(pair_index(st[j]), xf, xc, st[j].k, st[j].evc);
                    }
                    fp_push(done[j], xf, xc, st[j].k, st[j].evc);
                    done[j] = false;
                }
                // idle lanes take started pairs, in lane order, once refill_min
                // of them are idle (or all); the pool is refilled from the chunk
                unsigned im = __ballot_sync(kFullMask, !active[j]);
                if (im != 0u && (__popc(im) >= B.refill_min || im == kFullMask)) {
                    while (im != 0u) {
                        const int si = X.sp_i, sn = X.sp_n;
                        if (si == sn) {
                            if (X.next >= X.end) break;
                            refill();
                            continue;
                        }
                        const int avail = sn - si;
                        const int rank = __popc(im & lanemask_lt());
                        if (!active[j] && rank < avail) {
                            int e = si + rank;
                            if (!MLKD_DCHECK(e < 32)) e = 31;
                            const unsigned long long pe = X.first + (unsigned long long)SP.off[e];
                            if constexpr (PHYS == 1)
                                het_pair_init<Real>(st[j], pe, SP.v0[e], SP.e0[e], SP.q0[e], H, coupled);
                            else
                                pair_init<Real, 2>(st[j], pe, SP.x0[e], SP.v0[e], SP.q0[e], L, coupled);
                            active[j] = true;
                        }
                        const int took = __popc(im) < avail ? __popc(im) : avail;
                        __syncwarp();
                        X.sp_i = si + took;
                        __syncwarp();
                        im = __ballot_sync(kFullMask, !active[j]);
                    }
                }
            }
            bool any_local = false;
#pragma unroll
            for (int j = 0; j < PPT; ++j) any_local |= active[j];
            if (!__any_sync(kFullMask, any_local)) {
                // every lane idle with nothing to hand out: the chunk is done
                if (X.next >= X.end && X.sp_i == X.sp_n) {
                    const int nf = X.fp_n;
                    if (nf > 0) fp_process(nf);
                    chunk_done = true;
                    break;
                }
                continue;
            }
            // events until a pair reaches T (or the slice budget is spent)
            for (;;) {
                bool any_done = false;
#pragma unroll
                for (int j = 0; j < PPT; ++j)
                    if (active[j] && event(j)) {
                        active[j] = false;
                        done[j] = true;
                        any_done = true;
                    }
                ++iters;
                if (__any_sync(kFullMask, any_done) || iters >= iter_limit) break;
            }
        }
        if (!chunk_done) {
            // budget spent inside the chunk: store it for the next slice
            int w = 0;
#pragma unroll
            for (int j = 0; j < PPT; ++j) put_words(st[j], lw, stride, w);
            put_words(mom, lw, stride, w);
            put_words(ev_f_sum, lw, stride, w);
            put_words(ev_c_sum, lw, stride, w);
            uint32_t bits = 0;
#pragma unroll
            for (int j = 0; j < PPT; ++j)
                bits |= ((active[j] ? 1u : 0u) << j) | ((done[j] ? 1u : 0u) << (kMaxPPT + j));
            put_words(bits, lw, stride, w);
            put_pools(w);
            flush_hist();
            if (lane == 0) {
                hdr->valid = 1;
                hdr->c = X.c;
                hdr->next = X.next;
            }
            return;
        }
        // one row of sums for this chunk (fixed reduction order)
        mom.warp_reduce();
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            ev_f_sum += __shfl_down_sync(kFullMask, ev_f_sum, off);
            ev_c_sum += __shfl_down_sync(kFullMask, ev_c_sum, off);
        }
        if (lane == 0) {
            double *row = B.rows + (size_t)X.c * kPartialWords;
#pragma unroll
            for (int j = 0; j < 6; ++j) row[j] = mom.value(j);
            row[6] = (double)ev_f_sum;
            row[7] = (double)ev_c_sum;
            atomicAdd(&B.ctl->events_done, ev_f_sum + ev_c_sum);
        }
        flush_hist();
        // the row and the histogram counts are visible before the count
        // drops; the warp that takes it to zero completes the round
        __threadfence();
        const int req = X.req;
        int last = 0;
        if (lane == 0) last = atomicSub(&B.state[req].pending, 1) == 1;
        if (__shfl_sync(kFullMask, last, 0)) {
            __threadfence();
            if (*(volatile int32_t *)&B.state[req].status == 2) warp_round_complete(B, req, lane);
        }
        valid = 0;
    }
    if (lane == 0) hdr->valid = 0;
}

// ---------------------------------------------------------------------------
// Scheduler kernel: one warp per request slot.  Admits requests (their first
// round), frees cancelled ones once drained, and completes any round that no
// pair-kernel warp completed (normally the warp that finishes a round's last
// chunk completes it inside the pair kernel).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32) batch_sched_kernel(const BatchLaunch B)
{
    const int r = blockIdx.x;
    if (r >= B.n_slots) return;
    ReqState &S = B.state[r];
    const ReqDesc &D = B.req[r];
    const int lane = threadIdx.x;
    const int status = *(volatile int32_t *)&S.status;
    const int pending = *(volatile int32_t *)&S.pending;
    if (status == 0 || status == 3) {
        if (lane == 0) B.status_out[r] = status;
        return;
    }
    if (status == 4) {                    // cancelled: free once its chunks have drained
        if (lane == 0) {
            if (pending > 0) {
                atomicAdd(&B.ctl->live, 1);
                B.status_out[r] = 4;
            } else {
                S.status = 0;
                B.status_out[r] = 0;
                if (atomicExch(&S.counted, 0) == 1) atomicSub(&B.ctl->running, 1);
            }
        }
        return;
    }
    if (status == 2 && pending > 0) {
        if (lane == 0) {
            atomicAdd(&B.ctl->live, 1);
            B.status_out[r] = 2;
        }
        return;
    }
    if (status == 2) {
        warp_round_complete(B, r, lane);
    } else {
        // admitted: warm-up round (or the fixed counts)
        if (lane == 0) {
            for (int l = 0; l <= D.L; ++l) S.target[l] = D.use_fixed ? D.n_fixed[l] : (long long)D.n_warmup;
            S.counted = 1;
            atomicAdd(&B.ctl->running, 1);
        }
        __syncwarp();
        warp_plan(B, r, lane);
    }
    if (lane == 0) {
        const int st = *(volatile int32_t *)&S.status;
        B.status_out[r] = st;
        if (st == 2) atomicAdd(&B.ctl->live, 1);
    }
}

// Counts the loop iteration and publishes the loop condition (no request
// live, or a bounded wait ran out).
__global__ void batch_post_kernel(BatchCtl *ctl, int *live_out, cudaGraphConditionalHandle h, int use_graph)
{
    ctl->iterations += 1;
    const int live = ctl->error ? 0 : ctl->live;
    ctl->live = 0;
    if (live_out) *live_out = live;
    if (use_graph) cudaGraphSetConditional(h, live > 0 ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
struct BatchLayout {
    size_t desc, state, chunks, rows, qids, lids, pids, hist, ctl, live, hdr, lanes, status, total;
    size_t words;                // lane words per lane
    unsigned long long ring;
    size_t guard[kMaxGuards];    // canary offsets (debug build)
    int n_guard;
};

static bool batch_cfg_ok(const mlkd_batch_config *c)
{
    if (!c) return false;
    if (c->pairs_per_thread != 1 && c->pairs_per_thread != 2 && c->pairs_per_thread != 4 &&
        c->pairs_per_thread != 8) return false;
    if (c->substeps_per_launch < 0) return false;
    if (c->refill_min < 0 || c->refill_min > 32) return false;
    if (c->publish_wait_spins < 0) return false;
    if (c->warp_pair_min_events < -1) return false;
    if (c->test_stall_queues < 0 || c->test_stall_queues > (1 << 20)) return false;
    if (c->max_requests < 1 || c->max_requests > 4096) return false;
    if (c->max_nbins < 0 || c->max_nbins > 256) return false;
    return true;
}

static BatchLayout batch_layout(const mlkd_batch_config *c)
{
    BatchLayout B;
    // Each request slot owns kSlotChunks chunk ids (a request has at most one
    // round outstanding).  The id queues hold at most every slot's ids at
    // once; twice that keeps a claimed id's ring cell from being reused
    // before its claimer has read it.
    const unsigned long long ids = (unsigned long long)c->max_requests * kSlotChunks;
    unsigned long long ring = 1024;
    while (ring < 2 * ids) ring <<= 1;
    B.ring = ring;
    size_t off = arena_layout().total;
    B.n_guard = 0;
    // a region of `bytes` at the current offset, then (debug build) its canary
    auto place = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes);
        if (kGuardBytes) {
            B.guard[B.n_guard++] = off;
            off += kGuardBytes;
        }
        return at;
    };
    B.desc = place((size_t)c->max_requests * sizeof(ReqDesc));
    B.state = place((size_t)c->max_requests * sizeof(ReqState));
    B.chunks = place((size_t)ids * sizeof(Chunk));
    B.rows = place((size_t)ids * kPartialWords * sizeof(double));
    B.qids = place((size_t)ring * sizeof(unsigned long long));
    B.lids = place((size_t)ring * sizeof(unsigned long long));
    B.pids = place((size_t)ring * sizeof(unsigned long long));
    B.hist = place((size_t)c->max_requests * kBL * 3 * (size_t)(c->max_nbins > 0 ? c->max_nbins : 1) * sizeof(unsigned long long));
    B.ctl = place(sizeof(BatchCtl));
    B.live = place(sizeof(int));
    B.hdr = place((kMaxLanes / 32) * sizeof(WarpHdr));
    const size_t words = (size_t)std::max(std::max(lane_words<float, kModeFP32Comp, kMaxPPT>(),
                                                   lane_words<double, kModeFP64, 1>()),
                                          std::max(lane_words<float, kModeFP32Comp, 1, 1>(),
                                                   lane_words<double, kModeFP64, 1, 1>()));
    B.words = words;
    B.lanes = place(words * kMaxLanes * sizeof(uint32_t));
    B.status = place((size_t)c->max_requests * sizeof(int32_t));
    B.total = off;
    return B;
}

struct BatchCache {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    mlkd_batch_config cfg{};
    int mode = -1;
    uint64_t seed = 0;
    int n_slots = 0;
    cudaStream_t stream = nullptr;
};

void batch_release(mlkd_context *ctx)
{
    if (!ctx || !ctx->batch) return;
    if (ctx->batch->exec) cudaGraphExecDestroy(ctx->batch->exec);
    if (ctx->batch->graph) cudaGraphDestroy(ctx->batch->graph);
    delete ctx->batch;
    ctx->batch = nullptr;
}

typedef void (*BatchKernelFn)(const BatchLaunch);

// Kernel id: the precision mode, plus kPhysHet for the heterogeneous
// backgrounds (one pair per lane).
constexpr int kPhysHet = 16;

static BatchKernelFn pick_batch(int kid, int ppt)
{
    if (kid & kPhysHet) {
        switch (kid & ~kPhysHet) {
        case kModeFP64: return batch_pair_kernel<double, kModeFP64, 1, 1>;
        case kModeFP64U24: return batch_pair_kernel<double, kModeFP64U24, 1, 1>;
        case kModeFP32DY64: return batch_pair_kernel<float, kModeFP32DY64, 1, 1>;
        default: return batch_pair_kernel<float, kModeFP32Comp, 1, 1>;
        }
    }
    const int mode = kid;
    switch (mode) {
    case kModeFP64:
        return batch_pair_kernel<double, kModeFP64, 1>;
    case kModeFP64U24:
        return batch_pair_kernel<double, kModeFP64U24, 1>;
    case kModeFP32DY64:
        return ppt == 1 ? batch_pair_kernel<float, kModeFP32DY64, 1>
             : ppt == 2 ? batch_pair_kernel<float, kModeFP32DY64, 2>
             : ppt == 4 ? batch_pair_kernel<float, kModeFP32DY64, 4>
                        : batch_pair_kernel<float, kModeFP32DY64, 8>;
    default:
        return ppt == 1 ? batch_pair_kernel<float, kModeFP32Comp, 1>
             : ppt == 2 ? batch_pair_kernel<float, kModeFP32Comp, 2>
             : ppt == 4 ? batch_pair_kernel<float, kModeFP32Comp, 4>
                        : batch_pair_kernel<float, kModeFP32Comp, 8>;
    }
}

static void fill_desc(const mlkd_problem *p, const Derived &d, ReqDesc *D)
{
    std::memset(D, 0, sizeof(*D));
    for (int l = 0; l < d.J; ++l) {
        PairLaunch P;
        fill_launch(p, d, l, 0, 0, &P);
        D->bd[l] = P.bd;
        D->bf[l] = P.bf;
        D->n_level[l] = P.n;
        D->M_level[l] = P.M;
        D->level_of[l] = d.lev[l];
        D->n_fixed[l] = p->n_fixed ? p->n_fixed[l] : 0;
        if (l == 0) {
            D->fkind = P.fkind;
            D->background = P.background;
            D->x0 = P.x0;
            D->bg_b = P.bg_b;
            D->bg_a_left = P.bg_a_left;
            D->bg_a_right = P.bg_a_right;
        }
    }
    D->tol = p->tol;
    D->h = d.h;
    D->L = d.J - 1;                    // estimator levels 0..J-1
    D->M = p->M;
    D->init = p->init;
    D->nbins = p->nbins;
    D->periodic = d.periodic ? 1 : 0;
    D->density = p->qoi == MLKD_QOI_DENSITY ? 1 : 0;
    D->n_warmup = p->n_warmup;
    D->use_fixed = p->n_fixed ? 1 : 0;
    D->request = p->request;
}

static void fill_keys(uint64_t seed, PhiloxKeys *k)
{
    const uint32_t s0 = (uint32_t)seed, s1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        k->k0[r] = s0 + (uint32_t)r * kWeylA;
        k->k1[r] = s1 + (uint32_t)r * kWeylB;
    }
}

static void make_launch(mlkd_context *ctx, const BatchLayout &BL, const mlkd_batch_config *cfg,
                        int n_slots, uint64_t seed, BatchLaunch *B)
{
    std::memset(B, 0, sizeof(*B));
    B->req = (const ReqDesc *)(ctx->arena + BL.desc);
    B->state = (ReqState *)(ctx->arena + BL.state);
    B->chunks = (Chunk *)(ctx->arena + BL.chunks);
    B->rows = (double *)(ctx->arena + BL.rows);
    B->hist = (unsigned long long *)(ctx->arena + BL.hist);
    B->ctl = (BatchCtl *)(ctx->arena + BL.ctl);
    B->hdr = (WarpHdr *)(ctx->arena + BL.hdr);
    B->lane_words = (uint32_t *)(ctx->arena + BL.lanes);
    B->lane_word_count = (int32_t)BL.words;
    B->q_ids = (unsigned long long *)(ctx->arena + BL.qids);
    B->l_ids = (unsigned long long *)(ctx->arena + BL.lids);
    B->p_ids = (unsigned long long *)(ctx->arena + BL.pids);
    B->status_out = (int32_t *)(ctx->arena + BL.status);
    B->ring_mask = BL.ring - 1;
    B->max_nbins = cfg->max_nbins > 0 ? cfg->max_nbins : 1;
    B->slice_iters = cfg->substeps_per_launch;
    B->refill_min = cfg->refill_min > 0 ? cfg->refill_min : kBatchRefillMin;
    B->publish_spins = cfg->publish_wait_spins > 0 ? cfg->publish_wait_spins : kPublishSpins;
    B->dbg_req = -1;
    B->dbg_level = -1;
    B->warp_pair_events = cfg->warp_pair_min_events > 0 ? cfg->warp_pair_min_events
                        : cfg->warp_pair_min_events < 0 ? 0 : kWarpPairEvents;
    B->n_slots = n_slots;
    fill_keys(seed, &B->keys);
}

// Test hook (mlkd_batch_config::test_stall_queues): n places reserved at the
// head of every queue that nobody ever publishes, so that the first
// producer's bounded publication wait runs out.  Written after BatchCtl is
// cleared.
static mlkd_status stall_queues(char *ctl, int n, cudaStream_t s)
{
    if (n <= 0) return MLKD_OK;
    const unsigned long long v = (unsigned long long)n;
    MLKD_CUDA(cudaMemcpyAsync(ctl + offsetof(BatchCtl, q_resv), &v, sizeof(v), cudaMemcpyHostToDevice, s));
    MLKD_CUDA(cudaMemcpyAsync(ctl + offsetof(BatchCtl, l_resv), &v, sizeof(v), cudaMemcpyHostToDevice, s));
    MLKD_CUDA(cudaMemcpyAsync(ctl + offsetof(BatchCtl, p_resv), &v, sizeof(v), cudaMemcpyHostToDevice, s));
    MLKD_CUDA(cudaStreamSynchronize(s));
    return MLKD_OK;
}

// Enqueues the loop body once: scheduler, pair slice, bookkeeping.
static mlkd_status enqueue_body(mlkd_context *ctx, const BatchLaunch &B, int mode, int ppt, int grid,
                                cudaGraphConditionalHandle h, int use_graph, int *live_dev,
                                cudaStream_t s)
{
    batch_sched_kernel<<<B.n_slots, 32, 0, s>>>(B);
    MLKD_CUDA(cudaGetLastError());
    const size_t smem = (size_t)kWarpsPerBlock * 3 * B.max_nbins * sizeof(unsigned int);
    // host-loop form: the pair slice is timed like the per-level kernel
    const bool timed = !use_graph && ctx->timing && ctx->events_made && ctx->pending < kTimingRing;
    if (timed) MLKD_CUDA(cudaEventRecord(ctx->ev_start[ctx->pending], s));
    pick_batch(mode, ppt)<<<grid, kThreads, smem, s>>>(B);
    MLKD_CUDA(cudaGetLastError());
    if (timed) MLKD_CUDA(cudaEventRecord(ctx->ev_stop[ctx->pending++], s));
    batch_post_kernel<<<1, 1, 0, s>>>(B.ctl, live_dev, h, use_graph);
    MLKD_CUDA(cudaGetLastError());
    ctx->other_launches += 2;
    if (!timed) ctx->launches += 1;
    return MLKD_OK;
}

static mlkd_status batch_grid(mlkd_context *ctx, int mode, int ppt, int max_nbins, int *grid)
{
    int blocks = 0;
    const size_t smem = (size_t)kWarpsPerBlock * 3 * (max_nbins > 0 ? max_nbins : 1) * sizeof(unsigned int);
    MLKD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, (const void *)pick_batch(mode, ppt),
                                                           kThreads, smem));
    *grid = ctx->sm_count * std::max(1, blocks);
    if ((size_t)(*grid) * kThreads > kMaxLanes) *grid = (int)(kMaxLanes / kThreads);
    return MLKD_OK;
}

// Per-pair readout of one (request, estimator level) of a batched run.
struct BatchDebug {
    int req, level;
    unsigned long long n;
    double *xf, *xc;
    int32_t *kf, *kc;
};

static mlkd_status run_batch(mlkd_context *ctx, const mlkd_problem *problems, int n,
                             const mlkd_batch_config *cfg, cudaStream_t s, mlkd_result *results,
                             const BatchDebug *dbg = nullptr)
{
    NvtxRange nvtx_range("mlkd_estimate_batch");
    if (!ctx || !problems || n < 1 || !results || !batch_cfg_ok(cfg)) return MLKD_EINVAL;
    if (ctx->server) return MLKD_EBUSY;
    if (n > cfg->max_requests) return MLKD_EINVAL;
    const BatchLayout BL = batch_layout(cfg);
    if (ctx->arena_bytes < BL.total) return MLKD_ENOMEM;
    std::vector<ReqDesc> desc(n);
    int mode = -1;
    uint64_t seed = 0;
    const bool het = problems[0].background != MLKD_BG_HOMOGENEOUS;
    for (int i = 0; i < n; ++i) {
        Derived d;
        if (!validate(&problems[i], &d) || d.per_level_only) return MLKD_EINVAL;
        // one call holds either homogeneous or heterogeneous problems
        if ((problems[i].background != MLKD_BG_HOMOGENEOUS) != het) return MLKD_EINVAL;
        if (!problems[i].n_fixed && (!(problems[i].tol > 0.0) || problems[i].n_warmup < 2)) return MLKD_EINVAL;
        if (problems[i].nbins > cfg->max_nbins) return MLKD_EINVAL;
        if (i == 0) {
            mode = d.mode;
            seed = problems[i].seed;
        } else if (d.mode != mode || problems[i].seed != seed) {
            return MLKD_EINVAL;
        }
        fill_desc(&problems[i], d, &desc[i]);
    }
    const int ppt = (mode == kModeFP64 || mode == kModeFP64U24 || het) ? 1 : cfg->pairs_per_thread;
    const int kid = mode | (het ? kPhysHet : 0);
    const auto t0 = std::chrono::steady_clock::now();
    MLKD_CUDA(cudaSetDevice(ctx->device));

    // reset the request slots, queue, histograms and control words
    MLKD_CUDA(cudaMemcpyAsync(ctx->arena + BL.desc, desc.data(), n * sizeof(ReqDesc), cudaMemcpyHostToDevice, s));
    MLKD_CUDA(cudaMemsetAsync(ctx->arena + BL.state, 0, (size_t)n * sizeof(ReqState), s));
    std::vector<int32_t> admitted(n, 1);
    for (int i = 0; i < n; ++i)
        MLKD_CUDA(cudaMemcpyAsync(ctx->arena + BL.state + (size_t)i * sizeof(ReqState) + offsetof(ReqState, status),
                                  &admitted[i], sizeof(int32_t), cudaMemcpyHostToDevice, s));
    const size_t hist_bytes = (size_t)n * kBL * 3 * (size_t)(cfg->max_nbins > 0 ? cfg->max_nbins : 1) * sizeof(unsigned long long);
    MLKD_CUDA(cudaMemsetAsync(ctx->arena + BL.hist, 0, hist_bytes, s));
    MLKD_CUDA(cudaMemsetAsync(ctx->arena + BL.ctl, 0, sizeof(BatchCtl), s));
    MLKD_CUDA(cudaMemsetAsync(ctx->arena + BL.hdr, 0, (kMaxLanes / 32) * sizeof(WarpHdr), s));
    {
        const mlkd_status hs = stall_queues(ctx->arena + BL.ctl, cfg->test_stall_queues, s);
        if (hs != MLKD_OK) return hs;
        const mlkd_status gs = guards_write(ctx->arena, BL.guard, BL.n_guard, s);
        if (gs != MLKD_OK) return gs;
    }

    BatchLaunch B;
    make_launch(ctx, BL, cfg, n, seed, &B);
    if (dbg) {
        B.dbg_req = dbg->req;
        B.dbg_level = dbg->level;
        B.dbg_n = dbg->n;
        B.dbg_xf = dbg->xf;
        B.dbg_xc = dbg->xc;
        B.dbg_kf = dbg->kf;
        B.dbg_kc = dbg->kc;
        batch_release(ctx);          // a graph with the readout is not kept for later calls
    }
    int grid = 0;
    mlkd_status st = batch_grid(ctx, kid, ppt, cfg->max_nbins, &grid);
    if (st != MLKD_OK) return st;
    int *live_dev = (int *)(ctx->arena + BL.live);

    if (cfg->use_graph) {
        BatchCache *bc = ctx->batch;
        const bool reuse = bc && bc->exec && bc->mode == kid && bc->seed == seed && bc->n_slots == n &&
                           std::memcmp(&bc->cfg, cfg, sizeof(*cfg)) == 0 && bc->stream == s;
        if (!reuse) {
            batch_release(ctx);
            bc = new (std::nothrow) BatchCache;
            if (!bc) return MLKD_ENOMEM;
            ctx->batch = bc;
            cudaGraph_t g = nullptr;
            MLKD_CUDA(cudaGraphCreate(&g, 0));
            bc->graph = g;
            cudaGraphConditionalHandle h;
            MLKD_CUDA(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t node;
            MLKD_CUDA(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            cudaStream_t cs;
            MLKD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            cudaError_t e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                                          cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) {
                cudaStreamDestroy(cs);
                return MLKD_ECUDA;
            }
            st = enqueue_body(ctx, B, kid, ppt, grid, h, 1, nullptr, cs);
            cudaGraph_t captured = nullptr;
            e = cudaStreamEndCapture(cs, &captured);
            cudaStreamDestroy(cs);
            if (st != MLKD_OK) return st;
            if (e != cudaSuccess) return MLKD_ECUDA;
            ctx->other_launches -= 2;
            ctx->launches -= 1;   // the capture launched nothing
            MLKD_CUDA(cudaGraphInstantiate(&bc->exec, g, 0));
            bc->cfg = *cfg;
            bc->mode = kid;
            bc->seed = seed;
            bc->n_slots = n;
            bc->stream = s;
        }
        MLKD_CUDA(cudaGraphLaunch(bc->exec, s));
        if (dbg) {
            MLKD_CUDA(cudaStreamSynchronize(s));
            batch_release(ctx);
        }
    } else {
        for (int it = 0; it < 1000000; ++it) {
            st = enqueue_body(ctx, B, kid, ppt, grid, 0, 0, live_dev, s);
            if (st != MLKD_OK) return st;
            int live = 0;
            MLKD_CUDA(cudaMemcpyAsync(&live, live_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
            MLKD_CUDA(cudaStreamSynchronize(s));
            st = harvest_timing(ctx);
            if (st != MLKD_OK) return st;
            if (live == 0) break;
        }
    }

    // results
    BatchCtl hctl;
    MLKD_CUDA(cudaMemcpyAsync(&hctl, ctx->arena + BL.ctl, sizeof(hctl), cudaMemcpyDeviceToHost, s));
    std::vector<ReqState> hs(n);
    MLKD_CUDA(cudaMemcpyAsync(hs.data(), ctx->arena + BL.state, (size_t)n * sizeof(ReqState), cudaMemcpyDeviceToHost, s));
    std::vector<unsigned long long> hh;
    if (cfg->max_nbins > 0) {
        hh.resize(hist_bytes / sizeof(unsigned long long));
        MLKD_CUDA(cudaMemcpyAsync(hh.data(), ctx->arena + BL.hist, hist_bytes, cudaMemcpyDeviceToHost, s));
    }
    MLKD_CUDA(cudaStreamSynchronize(s));
    if (hctl.error) return hctl.error == 1 ? MLKD_ETIMEDOUT : MLKD_EINTERNAL;
    if (cfg->use_graph) {
        ctx->launches += (unsigned long long)hctl.iterations;
        ctx->other_launches += 2ull * (unsigned long long)hctl.iterations;
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    const int NB = cfg->max_nbins > 0 ? cfg->max_nbins : 1;
    for (int i = 0; i < n; ++i) {
        mlkd_result *o = &results[i];
        double *dens = o->density;
        std::memset(o, 0, sizeof(*o));
        o->density = dens;
        const ReqState &S = hs[i];
        Derived di;
        validate(&problems[i], &di);
        const int nl = di.J;
        o->estimate = S.estimate;
        o->variance = S.variance;
        o->n_levels = nl;
        o->rounds = S.rounds;
        for (int l = 0; l < nl; ++l) {
            const DevLevelStats &a = S.acc[l];
            o->lv[l].n = a.n;
            o->lv[l].sy = a.sy;
            o->lv[l].sy2 = a.sy2;
            o->lv[l].sqf = a.sqf;
            o->lv[l].sqf2 = a.sqf2;
            o->lv[l].sqc = a.sqc;
            o->lv[l].sqc2 = a.sqc2;
            o->lv[l].events_f = a.events_f;
            o->lv[l].events_c = a.events_c;
            o->var_level[l] = S.var_level[l];
            o->cost_level[l] = S.cost_level[l];
        }
        const int nb = problems[i].nbins;
        if (dens && nb > 0) {
            Derived d;
            validate(&problems[i], &d);
            for (int b = 0; b < nb; ++b) dens[b] = 0.0;
            for (int l = 0; l < nl; ++l) {
                const unsigned long long *H = hh.data() + ((size_t)i * kBL + l) * 3 * NB;
                if (S.acc[l].n > 0)
                    for (int b = 0; b < nb; ++b)
                        dens[b] += ((double)H[b] - (double)H[nb + b]) / (double)S.acc[l].n;
            }
            for (int b = 0; b < nb; ++b) dens[b] /= d.h;
        }
        o->seconds = secs;
    }
    mlkd_status cs = device_checks();
    if (cs == MLKD_OK) cs = guards_check(ctx->arena, BL.guard, BL.n_guard);
    if (cs == MLKD_OK) cs = guards_check(ctx->arena, ctx->L.guard, ctx->L.n_guard);
    return cs;
}

// ---------------------------------------------------------------------------
// Serving form.
// ---------------------------------------------------------------------------
struct ServerReq {
    mlkd_problem p;
    std::vector<int64_t> n_fixed;
    std::vector<int32_t> level_set;
    double t_submit = 0.0, t_done = 0.0;
    int slot = -1;
    int state = 0;              // 0 waiting, 1 admitted, 2 done, 3 cancel requested
    mlkd_result result;
    std::vector<double> density;
};

struct Server {
    mlkd_context *ctx = nullptr;
    mlkd_server_config cfg;
    BatchLayout BL;
    BatchLaunch B;
    int mode = 0, ppt = 1, grid = 1;
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    int error = MLKD_OK;
    uint64_t next_id = 1;
    std::deque<uint64_t> waiting;
    std::unordered_map<uint64_t, ServerReq> reqs;
    std::vector<uint64_t> slot_req;     // request id per slot, 0 = free
    std::vector<int32_t> slot_status;
    mlkd_server_stats stats{};
    std::chrono::steady_clock::time_point t0;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

static mlkd_status server_admit(Server *S, uint64_t id, int slot)
{
    ServerReq &q = S->reqs[id];
    Derived d;
    validate(&q.p, &d);
    ReqDesc desc;
    fill_desc(&q.p, d, &desc);
    char *base = S->ctx->arena;
    MLKD_CUDA(cudaMemcpyAsync(base + S->BL.desc + (size_t)slot * sizeof(ReqDesc), &desc, sizeof(desc),
                              cudaMemcpyHostToDevice, S->stream));
    MLKD_CUDA(cudaMemsetAsync(base + S->BL.state + (size_t)slot * sizeof(ReqState), 0, sizeof(ReqState), S->stream));
    const int32_t admitted = 1;
    MLKD_CUDA(cudaMemcpyAsync(base + S->BL.state + (size_t)slot * sizeof(ReqState) + offsetof(ReqState, status),
                              &admitted, sizeof(admitted), cudaMemcpyHostToDevice, S->stream));
    const size_t nb = (size_t)(S->cfg.batch.max_nbins > 0 ? S->cfg.batch.max_nbins : 1);
    MLKD_CUDA(cudaMemsetAsync(base + S->BL.hist + (size_t)slot * kBL * 3 * nb * sizeof(unsigned long long), 0,
                              kBL * 3 * nb * sizeof(unsigned long long), S->stream));
    q.slot = slot;
    q.state = 1;
    S->slot_req[slot] = id;
    return MLKD_OK;
}

static mlkd_status server_collect(Server *S, int slot)
{
    const uint64_t id = S->slot_req[slot];
    ServerReq &q = S->reqs[id];
    char *base = S->ctx->arena;
    ReqState st;
    const size_t nb = (size_t)(S->cfg.batch.max_nbins > 0 ? S->cfg.batch.max_nbins : 1);
    std::vector<unsigned long long> h(kBL * 3 * nb);
    MLKD_CUDA(cudaMemcpyAsync(&st, base + S->BL.state + (size_t)slot * sizeof(ReqState), sizeof(st),
                              cudaMemcpyDeviceToHost, S->stream));
    if (q.p.nbins > 0)
        MLKD_CUDA(cudaMemcpyAsync(h.data(), base + S->BL.hist + (size_t)slot * kBL * 3 * nb * sizeof(unsigned long long),
                                  h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, S->stream));
    const int32_t freed = 0;
    MLKD_CUDA(cudaMemcpyAsync(base + S->BL.state + (size_t)slot * sizeof(ReqState) + offsetof(ReqState, status),
                              &freed, sizeof(freed), cudaMemcpyHostToDevice, S->stream));
    MLKD_CUDA(cudaStreamSynchronize(S->stream));
    mlkd_result &o = q.result;
    std::memset(&o, 0, sizeof(o));
    Derived dq;
    validate(&q.p, &dq);
    const int nl = dq.J;
    o.estimate = st.estimate;
    o.variance = st.variance;
    o.n_levels = nl;
    o.rounds = st.rounds;
    for (int l = 0; l < nl; ++l) {
        const DevLevelStats &a = st.acc[l];
        o.lv[l].n = a.n;
        o.lv[l].sy = a.sy;
        o.lv[l].sy2 = a.sy2;
        o.lv[l].sqf = a.sqf;
        o.lv[l].sqf2 = a.sqf2;
        o.lv[l].sqc = a.sqc;
        o.lv[l].sqc2 = a.sqc2;
        o.lv[l].events_f = a.events_f;
        o.lv[l].events_c = a.events_c;
        o.var_level[l] = st.var_level[l];
        o.cost_level[l] = st.cost_level[l];
    }
    if (q.p.nbins > 0) {
        Derived d;
        validate(&q.p, &d);
        const int nbq = q.p.nbins;
        q.density.assign(nbq, 0.0);
        for (int l = 0; l < nl; ++l) {
            const unsigned long long *H = h.data() + (size_t)l * 3 * nb;
            if (st.acc[l].n > 0)
                for (int b = 0; b < nbq; ++b)
                    q.density[b] += ((double)H[b] - (double)H[nbq + b]) / (double)st.acc[l].n;
        }
        for (int b = 0; b < nbq; ++b) q.density[b] /= d.h;
    }
    q.t_done = S->now();
    o.seconds = q.t_done - q.t_submit;
    q.state = 2;
    q.slot = -1;
    S->slot_req[slot] = 0;
    return MLKD_OK;
}

static void server_loop(Server *S)
{
    cudaSetDevice(S->ctx->device);
    const int n = S->cfg.batch.max_requests;
    for (;;) {
        NvtxRange nvtx_range("mlkd_server_iteration");
        int active = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop) break;
            // cancellations of admitted requests: mark the device slot
            for (int slot = 0; slot < n; ++slot) {
                const uint64_t id = S->slot_req[slot];
                if (!id) continue;
                ServerReq &q = S->reqs[id];
                if (q.state == 3 && S->slot_status[slot] != 4) {
                    const int32_t cancel = 4;
                    if (cudaMemcpyAsync(S->ctx->arena + S->BL.state + (size_t)slot * sizeof(ReqState) +
                                            offsetof(ReqState, status),
                                        &cancel, sizeof(cancel), cudaMemcpyHostToDevice, S->stream) != cudaSuccess)
                        S->error = MLKD_ECUDA;
                    S->slot_status[slot] = 4;
                }
            }
            // admission: free slots take waiting requests in arrival order
            for (int slot = 0; slot < n && !S->waiting.empty(); ++slot) {
                if (S->slot_req[slot]) continue;
                const uint64_t id = S->waiting.front();
                S->waiting.pop_front();
                if (server_admit(S, id, slot) != MLKD_OK) S->error = MLKD_ECUDA;
                S->slot_status[slot] = 1;
                S->stats.admitted += 1;
            }
            for (int slot = 0; slot < n; ++slot) active += S->slot_req[slot] ? 1 : 0;
            if (active == 0) {
                S->cv_work.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
        }
        const double t_it = S->now();
        struct {
            unsigned long long events, events_done;
            int32_t running, error;
        } tail = {0, 0, 0, 0};
        if (cudaGraphLaunch(S->exec, S->stream) != cudaSuccess ||
            cudaMemcpyAsync(S->slot_status.data(), S->B.status_out, n * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, S->stream) != cudaSuccess ||
            cudaMemcpyAsync(&tail, &S->B.ctl->events, sizeof(tail), cudaMemcpyDeviceToHost,
                            S->stream) != cudaSuccess ||
            cudaStreamSynchronize(S->stream) != cudaSuccess) {
            std::lock_guard<std::mutex> lk(S->mu);
            S->error = MLKD_ECUDA;
            S->stop = true;
            S->cv_done.notify_all();
            break;
        }
        std::lock_guard<std::mutex> lk(S->mu);
        S->stats.iterations += 1;
        S->stats.busy_seconds += S->now() - t_it;
        S->stats.events = tail.events;
        S->stats.events_processed = tail.events_done;
        if (tail.error) {
            S->error = tail.error == 1 ? MLKD_ETIMEDOUT : MLKD_EINTERNAL;
            S->stop = true;
            S->cv_done.notify_all();
            break;
        }
        bool any_done = false;
        for (int slot = 0; slot < n; ++slot) {
            const uint64_t id = S->slot_req[slot];
            if (!id) continue;
            ServerReq &q = S->reqs[id];
            if (S->slot_status[slot] == 3 && q.state == 1) {
                if (server_collect(S, slot) != MLKD_OK) S->error = MLKD_ECUDA;
                S->stats.completed += 1;
                any_done = true;
            } else if (S->slot_status[slot] == 0 && q.state == 3) {
                S->slot_req[slot] = 0;           // cancelled and drained
                S->reqs.erase(id);
                S->stats.cancelled += 1;
            } else if (S->slot_status[slot] == 3 && q.state == 3) {
                // finished before the cancel reached it: free and drop
                const int32_t freed = 0;
                cudaMemcpyAsync(S->ctx->arena + S->BL.state + (size_t)slot * sizeof(ReqState) +
                                    offsetof(ReqState, status),
                                &freed, sizeof(freed), cudaMemcpyHostToDevice, S->stream);
                cudaStreamSynchronize(S->stream);
                S->slot_req[slot] = 0;
                S->reqs.erase(id);
                S->stats.cancelled += 1;
            }
        }
        if (any_done) S->cv_done.notify_all();
    }
    cudaStreamSynchronize(S->stream);
}

void server_release(mlkd_context *ctx)
{
    if (!ctx || !ctx->server) return;
    Server *S = ctx->server;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->cv_done.notify_all();
    }
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->graph) cudaGraphDestroy(S->graph);
    if (S->stream) cudaStreamDestroy(S->stream);
    ctx->server = nullptr;
    delete S;
}

static mlkd_status server_start(mlkd_context *ctx, const mlkd_server_config *cfg)
{
    if (!ctx || !cfg || !batch_cfg_ok(&cfg->batch)) return MLKD_EINVAL;
    if (cfg->precision < MLKD_PREC_FP64 || cfg->precision > MLKD_PREC_FP64_U24) return MLKD_EINVAL;
    if (cfg->max_pending < 1) return MLKD_EINVAL;
    if (ctx->server) return MLKD_EBUSY;
    const BatchLayout BL = batch_layout(&cfg->batch);
    if (ctx->arena_bytes < BL.total) return MLKD_ENOMEM;
    MLKD_CUDA(cudaSetDevice(ctx->device));
    Server *S = new (std::nothrow) Server;
    if (!S) return MLKD_ENOMEM;
    S->ctx = ctx;
    S->cfg = *cfg;
    S->BL = BL;
    S->mode = cfg->precision;
    S->ppt = (S->mode == kModeFP64 || S->mode == kModeFP64U24) ? 1 : cfg->batch.pairs_per_thread;
    S->slot_req.assign(cfg->batch.max_requests, 0);
    S->slot_status.assign(cfg->batch.max_requests, 0);
    S->t0 = std::chrono::steady_clock::now();
    auto fail = [&](mlkd_status st) {
        if (S->exec) cudaGraphExecDestroy(S->exec);
        if (S->graph) cudaGraphDestroy(S->graph);
        if (S->stream) cudaStreamDestroy(S->stream);
        delete S;
        return st;
    };
    if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(MLKD_ECUDA);
    const int n = cfg->batch.max_requests;
    if (cudaMemsetAsync(ctx->arena + BL.state, 0, (size_t)n * sizeof(ReqState), S->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->arena + BL.ctl, 0, sizeof(BatchCtl), S->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->arena + BL.hdr, 0, (kMaxLanes / 32) * sizeof(WarpHdr), S->stream) != cudaSuccess ||
        cudaMemsetAsync(ctx->arena + BL.status, 0, (size_t)n * sizeof(int32_t), S->stream) != cudaSuccess)
        return fail(MLKD_ECUDA);
    if (stall_queues(ctx->arena + BL.ctl, cfg->batch.test_stall_queues, S->stream) != MLKD_OK)
        return fail(MLKD_ECUDA);
    make_launch(ctx, BL, &cfg->batch, n, cfg->seed, &S->B);
    if (batch_grid(ctx, S->mode, S->ppt, cfg->batch.max_nbins, &S->grid) != MLKD_OK) return fail(MLKD_ECUDA);
    // one iteration as a graph: scheduler, pair slice, bookkeeping
    if (cudaStreamBeginCapture(S->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail(MLKD_ECUDA);
    int *live_dev = (int *)(ctx->arena + BL.live);
    batch_sched_kernel<<<n, 32, 0, S->stream>>>(S->B);
    const size_t smem = (size_t)kWarpsPerBlock * 3 * S->B.max_nbins * sizeof(unsigned int);
    pick_batch(S->mode, S->ppt)<<<S->grid, kThreads, smem, S->stream>>>(S->B);
    batch_post_kernel<<<1, 1, 0, S->stream>>>(S->B.ctl, live_dev, 0, 0);
    const cudaError_t le = cudaGetLastError();
    if (cudaStreamEndCapture(S->stream, &S->graph) != cudaSuccess || le != cudaSuccess) return fail(MLKD_ECUDA);
    if (cudaGraphInstantiate(&S->exec, S->graph, 0) != cudaSuccess) return fail(MLKD_ECUDA);
    if (cudaStreamSynchronize(S->stream) != cudaSuccess) return fail(MLKD_ECUDA);
    ctx->server = S;
    S->th = std::thread(server_loop, S);
    return MLKD_OK;
}

cudaError_t check_word_batch(unsigned *line)
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

using namespace mlkd;

extern "C" {

size_t mlkd_batch_workspace_bytes(const mlkd_batch_config *cfg)
{
    if (!batch_cfg_ok(cfg)) return 0;
    return batch_layout(cfg).total;
}

mlkd_status mlkd_estimate_batch(mlkd_context *ctx, const mlkd_problem *problems, int n,
                                const mlkd_batch_config *cfg, void *stream, mlkd_result *results)
{
    return run_batch(ctx, problems, n, cfg, (cudaStream_t)stream, results);
}

mlkd_status mlkd_debug_batch_pairs(mlkd_context *ctx, const mlkd_problem *problem,
                                   const mlkd_batch_config *cfg, int level, void *stream,
                                   mlkd_result *result, double *xf, double *xc, int32_t *kf,
                                   int32_t *kc)
{
    if (!problem || !problem->n_fixed || !xf || !xc || !kf || !kc || level < 0) return MLKD_EINVAL;
    Derived d;
    if (!validate(problem, &d) || level >= d.J) return MLKD_EINVAL;
    const long long nl = problem->n_fixed[level];
    if (nl < 0) return MLKD_EINVAL;
    BatchDebug dbg{0, level, (unsigned long long)nl, xf, xc, kf, kc};
    return run_batch(ctx, problem, 1, cfg, (cudaStream_t)stream, result, &dbg);
}

mlkd_status mlkd_autotune_batch(mlkd_context *ctx, const mlkd_problem *problems, int n,
                                const mlkd_batch_config *base, void *stream,
                                mlkd_batch_config *best, double *seconds)
{
    NvtxRange nvtx_range("mlkd_autotune_batch");
    if (!ctx || !base || !best || !batch_cfg_ok(base)) return MLKD_EINVAL;
    if (ctx->server) return MLKD_EBUSY;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<mlkd_result> res(n);
    const int ppts[4] = {1, 2, 4, 8};
    const int slices[4] = {16, 64, 256, 0};
    const int warps[3] = {0, -1, 4 * kWarpPairEvents};
    double best_t = 1e300;
    *best = *base;
    cudaEvent_t e0, e1;
    MLKD_CUDA(cudaSetDevice(ctx->device));
    MLKD_CUDA(cudaEventCreate(&e0));
    MLKD_CUDA(cudaEventCreate(&e1));
    mlkd_status st = MLKD_OK;
    for (int w = 0; w < 3 && st == MLKD_OK; ++w)
    for (int a = 0; a < 4 && st == MLKD_OK; ++a) {
        for (int b = 0; b < 4 && st == MLKD_OK; ++b) {
            mlkd_batch_config c = *base;
            c.pairs_per_thread = ppts[a];
            c.substeps_per_launch = slices[b];
            c.warp_pair_min_events = warps[w];
            c.use_graph = 1;
            for (int i = 0; i < n; ++i) res[i].density = nullptr;
            st = run_batch(ctx, problems, n, &c, s, res.data());       // warm (instantiates)
            if (st != MLKD_OK) break;
            if (cudaEventRecord(e0, s) != cudaSuccess) { st = MLKD_ECUDA; break; }
            st = run_batch(ctx, problems, n, &c, s, res.data());
            if (st != MLKD_OK) break;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                st = MLKD_ECUDA;
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (seconds) seconds[w * 16 + a * 4 + b] = ms * 1e-3;
            if (ms * 1e-3 < best_t) {
                best_t = ms * 1e-3;
                *best = c;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

}  // extern "C"

extern "C" {

mlkd_status mlkd_server_start(mlkd_context *ctx, const mlkd_server_config *cfg)
{
    return server_start(ctx, cfg);
}

mlkd_status mlkd_submit(mlkd_context *ctx, const mlkd_problem *problem, uint64_t *req_id)
{
    if (!ctx || !problem || !req_id) return MLKD_EINVAL;
    Server *S = ctx->server;
    if (!S) return MLKD_EINVAL;
    Derived d;
    if (!validate(problem, &d) || d.per_level_only) return MLKD_EINVAL;
    if (d.background != MLKD_BG_HOMOGENEOUS) return MLKD_EINVAL;    // the server runs the homogeneous kernel
    if (problem->precision != S->cfg.precision || problem->seed != S->cfg.seed) return MLKD_EINVAL;
    if (problem->nbins > S->cfg.batch.max_nbins) return MLKD_EINVAL;
    if (!problem->n_fixed && (!(problem->tol > 0.0) || problem->n_warmup < 2)) return MLKD_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->error != MLKD_OK) return (mlkd_status)S->error;
    if ((int)S->waiting.size() >= S->cfg.max_pending) {
        S->stats.rejected += 1;
        return MLKD_EBUSY;
    }
    const uint64_t id = S->next_id++;
    ServerReq &q = S->reqs[id];
    q.p = *problem;
    if (problem->n_fixed) {
        q.n_fixed.assign(problem->n_fixed, problem->n_fixed + d.J);
        q.p.n_fixed = q.n_fixed.data();
    }
    if (problem->n_set > 0) {
        q.level_set.assign(problem->level_set, problem->level_set + problem->n_set);
        q.p.level_set = q.level_set.data();
    }
    q.t_submit = S->now();
    S->waiting.push_back(id);
    S->stats.submitted += 1;
    *req_id = id;
    S->cv_work.notify_one();
    return MLKD_OK;
}

mlkd_status mlkd_poll(mlkd_context *ctx, uint64_t req_id, int timeout_ms, mlkd_result *out)
{
    if (!ctx || !out) return MLKD_EINVAL;
    Server *S = ctx->server;
    if (!S) return MLKD_ENOTFOUND;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end() || it->second.state == 3) return MLKD_ENOTFOUND;
    auto ready = [&]() {
        auto j = S->reqs.find(req_id);
        return j == S->reqs.end() || j->second.state == 2 || S->error != MLKD_OK || S->stop;
    };
    if (timeout_ms < 0) {
        S->cv_done.wait(lk, ready);
    } else if (timeout_ms > 0) {
        S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    }
    it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return MLKD_ENOTFOUND;
    if (it->second.state != 2) {
        if (S->error != MLKD_OK) return (mlkd_status)S->error;
        return MLKD_ETIMEDOUT;
    }
    double *dens = out->density;
    *out = it->second.result;
    out->density = dens;
    if (dens)
        for (size_t b = 0; b < it->second.density.size(); ++b) dens[b] = it->second.density[b];
    S->reqs.erase(it);
    return MLKD_OK;
}

mlkd_status mlkd_cancel(mlkd_context *ctx, uint64_t req_id)
{
    if (!ctx) return MLKD_EINVAL;
    Server *S = ctx->server;
    if (!S) return MLKD_ENOTFOUND;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return MLKD_ENOTFOUND;
    ServerReq &q = it->second;
    if (q.state == 0) {
        for (auto w = S->waiting.begin(); w != S->waiting.end(); ++w)
            if (*w == req_id) {
                S->waiting.erase(w);
                break;
            }
        S->reqs.erase(it);
        S->stats.cancelled += 1;
    } else if (q.state == 1) {
        q.state = 3;                 // the scheduler thread frees the slot once drained
    } else if (q.state == 2) {
        S->reqs.erase(it);           // finished: drop the result
        S->stats.cancelled += 1;
    }
    return MLKD_OK;
}

mlkd_status mlkd_server_stats_get(mlkd_context *ctx, mlkd_server_stats *out)
{
    if (!ctx || !out) return MLKD_EINVAL;
    Server *S = ctx->server;
    if (!S) return MLKD_ENOTFOUND;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    return MLKD_OK;
}

mlkd_status mlkd_server_stop(mlkd_context *ctx)
{
    if (!ctx) return MLKD_EINVAL;
    server_release(ctx);
    return MLKD_OK;
}

}  // extern "C"
