// Batched registration: many independent registrations (each its own target,
// source, variant and state) advance together, one device step for all of them
// per set of launches:
//   k_plan         one block: the list of tiles of the registrations that are
//                  not done, and each one's step head (load_head);
//   k_nn_batch     persistent warps take tickets of `chunk` queries over that
//                  list, from an atomic counter (uneven registrations share
//                  the GPU evenly) or dealt in a fixed stride (no atomics, the
//                  warps in flight on one window of the list), whichever the
//                  autotuner timed faster; each query is searched by a warp,
//                  or each ticket of kTileQ queries by a warp as one query
//                  tile (search_tile);
//   k_accum_batch  persistent blocks take tiles from a second counter; the
//                  block that completes a registration's pass reduces its tile
//                  records and runs its solver step on one warp, so the
//                  solvers of different registrations overlap with each other
//                  and with the remaining tiles.
// Per point and per tile the arithmetic and the reduction order are those of
// the single-registration step (step_common.cuh), so every registration gives
// the same bits alone and in a batch.
//
// The same engine carries the serving loop (fricp_server_*): its slots are
// filled and emptied between steps while the captured step graph keeps
// replaying.
#include <algorithm>
#include <deque>
#include <map>
#include <memory>
#include <mutex>

#include "host_common.cuh"
#include "step_common.cuh"

namespace fricp {

namespace {

// Device-side descriptor of one registration in flight.
struct Slot {
    PairState *st;
    Index ix;
    const float4 *src;
    int *prev;
    double *partial;
    double *resid;
    double *trace;
    int ntiles;
    int live;   // 1 while the slot holds a registration
};

struct BatchCtl {
    int n_tiles;         // tiles of the unfinished registrations in this step
    int active;          // unfinished registrations at the start of this step
    unsigned nn_next;    // next search ticket
    unsigned acc_next;   // next accumulate ticket
    int overflow;        // the tile list did not fit (never expected: the host sizes it)
    int pad[3];
};

constexpr int kPlanThreads = 1024;
// Order of the search tickets (BatchShape::order): from an atomic counter, in a
// fixed stride, or query tiles of kTileQ from the counter.
constexpr int kOrderCounter = 0, kOrderStride = 1, kOrderTiles = 2;
constexpr int kMaxSlots = 4096;
constexpr int kSlotsPerThread = kMaxSlots / kPlanThreads;

__global__ void __launch_bounds__(kPlanThreads) k_plan(const Slot *__restrict__ slots, int nslots,
                                                       StepHead *__restrict__ heads, int *__restrict__ done,
                                                       int *__restrict__ tile_slot, int *__restrict__ tile_local,
                                                       int max_tiles, BatchCtl *ctl) {
    __shared__ int s_off[kMaxSlots + 1];
    __shared__ int s_scan[kPlanThreads];
    __shared__ int s_active;
    const int t = threadIdx.x;
    if (t == 0) s_active = 0;
    __syncthreads();
    // contiguous run of slots per thread: [t * kSlotsPerThread, ...)
    int cnt[kSlotsPerThread];
    int run = 0, act = 0;
#pragma unroll
    for (int k = 0; k < kSlotsPerThread; ++k) {
        const int p = t * kSlotsPerThread + k;
        cnt[k] = 0;
        if (p < nslots) {
            const Slot sl = slots[p];
            int d = 1;
            if (sl.live) {
                d = sl.st->done;
                if (!d) {
                    cnt[k] = sl.ntiles;
                    load_head(sl.st, heads[p]);
                    ++act;
                }
            }
            done[p] = sl.live && d;
        }
        run += cnt[k];
    }
    if (act) atomicAdd(&s_active, act);
    // inclusive scan of the per-thread runs (Hillis-Steele)
    s_scan[t] = run;
    __syncthreads();
    for (int o = 1; o < kPlanThreads; o <<= 1) {
        const int v = t >= o ? s_scan[t - o] : 0;
        __syncthreads();
        s_scan[t] += v;
        __syncthreads();
    }
    int base = s_scan[t] - run;
#pragma unroll
    for (int k = 0; k < kSlotsPerThread; ++k) {
        s_off[t * kSlotsPerThread + k] = base;
        base += cnt[k];
    }
    if (t == kPlanThreads - 1) s_off[kMaxSlots] = s_scan[t];
    __syncthreads();
    int total = s_off[kMaxSlots];
    if (total > max_tiles) {   // the host sizes the list for every live slot; keep the bound anyway
        if (t == 0) ctl->overflow = 1;
        total = 0;
    }
    for (int g = t; g < total; g += kPlanThreads) {
        int lo = 0, hi = kMaxSlots;   // largest p with s_off[p] <= g (empty slots repeat offsets)
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_off[mid] <= g) lo = mid; else hi = mid;
        }
        tile_slot[g] = lo;
        tile_local[g] = g - s_off[lo];
    }
    if (t == 0) {
        ctl->n_tiles = total;
        ctl->active = s_active;
        ctl->nn_next = 0u;
        ctl->acc_next = 0u;
    }
}

// Copy of a head into shared memory by the threads of a warp (or block).
__device__ __forceinline__ void copy_head(const StepHead *src, StepHead *dst, int lane, int nthreads) {
    const int *s = reinterpret_cast<const int *>(src);
    int *d = reinterpret_cast<int *>(dst);
    constexpr int W = (int)(sizeof(StepHead) / sizeof(int));
    for (int k = lane; k < W; k += nthreads) d[k] = __ldcg(s + k);
}

__global__ void __launch_bounds__(kBlock, 4) k_nn_batch(const Slot *__restrict__ slots, const StepHead *heads,
                                                     const int *__restrict__ tile_slot,
                                                     const int *__restrict__ tile_local, BatchCtl *ctl, int chunk,
                                                     unsigned max_tickets, int order) {
    __shared__ int s_stk[kBlock / 32][kWarpStack];
    __shared__ __align__(16) float4 s_stage[kBlock / 32][kRing * 32];
    __shared__ StepHead s_head[kBlock / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int *stk = s_stk[w];
    StepHead &h = s_head[w];
    const bool tiles = order == kOrderTiles;
    const int static_order = order == kOrderStride;
    if (tiles) chunk = kTileQ;
    const int per_tile = kBlock / chunk;
    const unsigned total = min((unsigned)__ldcg(&ctl->n_tiles) * (unsigned)per_tile, max_tickets);
    int cur = -1;
    unsigned next = blockIdx.x * (kBlock / 32) + w;   // fixed stride: this warp's tickets
    const unsigned nwarps = gridDim.x * (kBlock / 32);
    for (;;) {
        unsigned tk = 0;
        if (static_order) {
            tk = next;
            next += nwarps;
        } else {
            if (lane == 0) tk = atomicAdd(&ctl->nn_next, 1u);
            tk = __shfl_sync(0xffffffffu, tk, 0);
        }
        if (tk >= total) break;
        const int tile = (int)(tk / per_tile), sub = (int)(tk % per_tile);
        const int p = __ldg(tile_slot + tile), lt = __ldg(tile_local + tile);
        if (p != cur) {
            __syncwarp();
            copy_head(heads + p, &h, lane, 32);
            __syncwarp();
            cur = p;
        }
        const Slot sl = slots[p];
        const int i0 = lt * kBlock + sub * chunk;
        const int i1 = min(i0 + chunk, h.M);
        const bool p2p = !fricp::variant_p2pl(h.variant);
        if (tiles) {   // the ticket's queries as one query tile
            bool ok;
            if (h.prec == PREC_FP32)
                ok = search_tile<PREC_FP32>(sl.ix, sl.src, sl.prev, h, i0, i1, p2p, stk, s_stage[w]);
            else if (h.prec == PREC_FP16)
                ok = search_tile<PREC_FP16>(sl.ix, sl.src, sl.prev, h, i0, i1, p2p, stk, s_stage[w]);
            else
                ok = search_tile<PREC_FP64>(sl.ix, sl.src, sl.prev, h, i0, i1, p2p, stk, s_stage[w]);
            if (!ok && lane == 0) sl.st->nn_overflow = 1;   // search-stack overflow: never expected
        } else if (p2p && h.welsch && h.phase != PH_INIT) {   // Welsch cap active: one query per warp (as k_nn)
            for (int i = i0; i < i1; ++i) {
                bool ok;
                if (h.prec == PREC_FP32)
                    ok = search_query<PREC_FP32>(sl.ix, sl.src, sl.prev, h, i, p2p, stk);
                else if (h.prec == PREC_FP16)
                    ok = search_query<PREC_FP16>(sl.ix, sl.src, sl.prev, h, i, p2p, stk);
                else
                    ok = search_query<PREC_FP64>(sl.ix, sl.src, sl.prev, h, i, p2p, stk);
                if (!ok && lane == 0) sl.st->nn_overflow = 1;   // search-stack overflow: never expected
            }
        } else {   // two queries per warp, one per half
            int *hstk = stk + ((lane & 16) ? kHalfStack : 0);
            for (int i2 = i0; i2 < i1; i2 += 2) {
                const int i = i2 + ((lane & 16) ? 1 : 0);
                const bool live = i < i1;
                bool ok;
                if (h.prec == PREC_FP32)
                    ok = search_pair<PREC_FP32>(sl.ix, sl.src, sl.prev, h, i, live, p2p, hstk);
                else if (h.prec == PREC_FP16)
                    ok = search_pair<PREC_FP16>(sl.ix, sl.src, sl.prev, h, i, live, p2p, hstk);
                else
                    ok = search_pair<PREC_FP64>(sl.ix, sl.src, sl.prev, h, i, live, p2p, hstk);
                if (!ok && lane == 0) sl.st->nn_overflow = 1;   // search-stack overflow: never expected
            }
        }
    }
}

__global__ void __launch_bounds__(kBlock, 3) k_accum_batch(const Slot *__restrict__ slots, const StepHead *heads,
                                                        const int *__restrict__ tile_slot,
                                                        const int *__restrict__ tile_local, BatchCtl *ctl) {
    __shared__ StepHead h;
    __shared__ double red[kSumsP2PL * kRedHalf];
    __shared__ double sS[kSumsP2PL];
    __shared__ int s_last, s_tile;
    const int n_tiles = __ldcg(&ctl->n_tiles);
    for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(&ctl->acc_next, 1u);
        __syncthreads();
        const int tk = s_tile;
        if (tk >= n_tiles) break;
        const int p = __ldg(tile_slot + tk), lt = __ldg(tile_local + tk);
        copy_head(heads + p, &h, threadIdx.x, kBlock);
        const Slot sl = slots[p];
        __syncthreads();
        if (fricp::variant_p2pl(h.variant)) {
            bool last;
            if (h.prec == PREC_FP32)
                last = accum_tile<1, PREC_FP32>(h, sl.st, sl.ix, sl.src, sl.prev, sl.resid, sl.partial, lt, sl.ntiles,
                                                red, &s_last);
            else if (h.prec == PREC_FP16)
                last = accum_tile<1, PREC_FP16>(h, sl.st, sl.ix, sl.src, sl.prev, sl.resid, sl.partial, lt, sl.ntiles,
                                                red, &s_last);
            else
                last = accum_tile<1, PREC_FP64>(h, sl.st, sl.ix, sl.src, sl.prev, sl.resid, sl.partial, lt, sl.ntiles,
                                                red, &s_last);
            if (last) finish_pass<kSumsP2PL>(h, sl.st, sl.partial, sl.ntiles, sl.resid, sl.trace, sS, red);
        } else {
            bool last;
            if (h.prec == PREC_FP32)
                last = accum_tile<0, PREC_FP32>(h, sl.st, sl.ix, sl.src, sl.prev, sl.resid, sl.partial, lt, sl.ntiles,
                                                red, &s_last);
            else if (h.prec == PREC_FP16)
                last = accum_tile<0, PREC_FP16>(h, sl.st, sl.ix, sl.src, sl.prev, sl.resid, sl.partial, lt, sl.ntiles,
                                                red, &s_last);
            else
                last = accum_tile<0, PREC_FP64>(h, sl.st, sl.ix, sl.src, sl.prev, sl.resid, sl.partial, lt, sl.ntiles,
                                                red, &s_last);
            if (last) finish_pass<kSumsP2P>(h, sl.st, sl.partial, sl.ntiles, sl.resid, sl.trace, sS, red);
        }
        __syncthreads();   // s_tile and h are rewritten next round
    }
}

__global__ void k_reset_nn_ticket(BatchCtl *ctl) { ctl->nn_next = 0u; }

using namespace fricp::host;

// Launch shape of the batched step (what the autotuner picks).
struct BatchShape {
    int chunk;        // queries per search ticket (divides kBlock)
    int nn_per_sm;    // search blocks per SM
    int acc_per_sm;   // accumulate blocks per SM
    int order;        // kOrderCounter, kOrderStride or kOrderTiles
};

int sm_count() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 152;
    }
    return sms;
}

int max_per_sm(const void *kernel) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kBlock, 0);
    return n > 0 ? n : 1;
}

// Autotuner memory: the best shape per size class (log2 of the points in flight,
// number of registrations in flight rounded to a power of two).
std::mutex g_tune_mu;
std::map<std::pair<int, int>, BatchShape> g_tuned;
BatchShape g_last_shape{1, 0, 0, 0};
BatchShape g_forced{0, 0, 0, 0};   // chunk > 0: the shape fricp_batch_set_shape fixed

std::pair<int, int> size_class(int64_t points, int nslots) {
    int a = 0, b = 0;
    while (((int64_t)1 << a) < points) ++a;
    while ((1 << b) < nslots) ++b;
    return {a, b};
}

}  // namespace

// The batched step engine: device-side slot table, tile lists and control
// block, and the captured step graph.
class BatchEngine {
  public:
    int max_slots = 0;
    int max_tiles = 0;
    Slot *d_slots = nullptr;
    StepHead *d_heads = nullptr;
    int *d_done = nullptr;
    int *d_tile_slot = nullptr;
    int *d_tile_local = nullptr;
    BatchCtl *d_ctl = nullptr;
    int *h_done = nullptr;        // pinned copy of d_done
    BatchCtl *h_ctl = nullptr;    // pinned copy of d_ctl
    BatchShape shape{1, 0, 0};
    host::Graph graph;
    int graph_steps = 0;
    BatchShape graph_shape{0, 0, 0, 0};   // the shape the graph was captured with
    int64_t graph_kernels = 0;   // kernel nodes per replay
    cudaStream_t s = nullptr;

    ~BatchEngine() { release(); }

    void release() {
        graph.reset();
        if (d_slots) cudaFree(d_slots);
        if (d_heads) cudaFree(d_heads);
        if (d_done) cudaFree(d_done);
        if (d_tile_slot) cudaFree(d_tile_slot);
        if (d_tile_local) cudaFree(d_tile_local);
        if (d_ctl) cudaFree(d_ctl);
        if (h_done) cudaFreeHost(h_done);
        if (h_ctl) cudaFreeHost(h_ctl);
        d_slots = nullptr;
        d_heads = nullptr;
        d_done = d_tile_slot = d_tile_local = nullptr;
        d_ctl = nullptr;
        h_done = nullptr;
        h_ctl = nullptr;
    }

    cudaError_t init(int slots, int tiles, cudaStream_t stream) {
        s = stream;
        max_slots = slots;
        max_tiles = tiles > 0 ? tiles : 1;
        cudaError_t e = cudaMalloc(&d_slots, sizeof(Slot) * slots);
        if (e == cudaSuccess) e = cudaMalloc(&d_heads, sizeof(StepHead) * slots);
        if (e == cudaSuccess) e = cudaMalloc(&d_done, sizeof(int) * slots);
        if (e == cudaSuccess) e = cudaMalloc(&d_tile_slot, sizeof(int) * max_tiles);
        if (e == cudaSuccess) e = cudaMalloc(&d_tile_local, sizeof(int) * max_tiles);
        if (e == cudaSuccess) e = cudaMalloc(&d_ctl, sizeof(BatchCtl));
        if (e == cudaSuccess) e = cudaMallocHost(&h_done, sizeof(int) * slots);
        if (e == cudaSuccess) e = cudaMallocHost(&h_ctl, sizeof(BatchCtl));
        if (e == cudaSuccess) e = cudaMemsetAsync(d_slots, 0, sizeof(Slot) * slots, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_ctl, 0, sizeof(BatchCtl), s);
        return e;
    }

    cudaError_t upload_slot(int p, const Slot &sl) {
        counters().h2d += sizeof(Slot);
        return cudaMemcpyAsync(d_slots + p, &sl, sizeof(Slot), cudaMemcpyHostToDevice, s);
    }

    int nn_blocks() const { return sm_count() * shape.nn_per_sm; }
    int acc_blocks() const { return sm_count() * shape.acc_per_sm; }

    void launch_plan(cudaStream_t st) {
        k_plan<<<1, kPlanThreads, 0, st>>>(d_slots, max_slots, d_heads, d_done, d_tile_slot, d_tile_local,
                                           max_tiles, d_ctl);
    }

    // One device step on `st`: plan, search, accumulate/solve (3 launches).
    void launch_step(cudaStream_t st) {
        launch_plan(st);
        k_nn_batch<<<nn_blocks(), kBlock, 0, st>>>(d_slots, d_heads, d_tile_slot, d_tile_local, d_ctl, shape.chunk,
                                                    0xffffffffu, shape.order);
        k_accum_batch<<<acc_blocks(), kBlock, 0, st>>>(d_slots, d_heads, d_tile_slot, d_tile_local, d_ctl);
        counters().launches += 3;
    }

    // Graph of `steps` device steps followed by a plan (so that ctl and the done
    // flags describe the state after the last step).
    cudaError_t capture(int steps) {
        if (graph.exec && graph_steps == steps && graph_shape.chunk == shape.chunk &&
            graph_shape.nn_per_sm == shape.nn_per_sm && graph_shape.acc_per_sm == shape.acc_per_sm &&
            graph_shape.order == shape.order)
            return cudaSuccess;
        graph.reset();
        const int64_t before = counters().launches;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        for (int k = 0; k < steps; ++k) launch_step(s);
        launch_plan(s);
        e = cudaStreamEndCapture(s, &graph.g);
        counters().launches = before;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&graph.exec, graph.g, 0);
        if (e == cudaSuccess) {
            graph_steps = steps;
            graph_shape = shape;
            graph_kernels = host::graph_kernel_nodes(graph.g);
        }
        return e;
    }

    cudaError_t run_graph() {
        counters().launches += graph_kernels;
        return cudaGraphLaunch(graph.exec, s);
    }

    // Copy the control block and done flags to the pinned mirrors (async on s).
    cudaError_t fetch_status() {
        cudaError_t e = cudaMemcpyAsync(h_ctl, d_ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_done, d_done, sizeof(int) * max_slots, cudaMemcpyDeviceToHost, s);
        counters().d2h += sizeof(BatchCtl) + sizeof(int) * max_slots;
        return e;
    }

    // Autotuner: time one full search pass over the live registrations at
    // their current transforms for each candidate shape and keep the fastest.
    // The search is exact, so repeating it leaves every correspondence as it
    // was; only the warm starts make the repeats cheaper, as in the steady
    // state. Small tickets balance the warps and keep the warps in flight on a
    // compact window of Morton-ordered queries (shared cache lines); large
    // tickets take fewer atomics; a fixed stride takes none.
    cudaError_t tune(int64_t points, int nslots) {
        const auto key = size_class(points, nslots);
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            if (g_forced.chunk > 0) {
                shape = g_forced;
                shape.nn_per_sm = std::min(std::max(shape.nn_per_sm, 1), max_per_sm((const void *)k_nn_batch));
                shape.acc_per_sm = max_per_sm((const void *)k_accum_batch);
                g_last_shape = shape;
                return cudaSuccess;
            }
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) {
                shape = it->second;
                g_last_shape = shape;
                return cudaSuccess;
            }
        }
        const int nn_max = max_per_sm((const void *)k_nn_batch);
        const int acc_max = max_per_sm((const void *)k_accum_batch);
        launch_plan(s);
        counters().launches += 1;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        // (chunk, order): query tiles, tickets of 1 or 4 queries from the counter,
        // single queries in a fixed stride (the shapes that have won on some
        // size class: tiles on every mix of many or large registrations, the
        // others on a few small ones)
        const int cands[][2] = {{kTileQ, kOrderTiles}, {4, kOrderCounter}, {1, kOrderCounter}, {1, kOrderStride}};
        int per_sm[2] = {nn_max, (nn_max + 1) / 2};
        BatchShape best{1, nn_max, acc_max, 0};
        float best_ms = 1e30f;
        cudaError_t e = cudaSuccess;
        // warm-up pass: sets the correspondences the timed repeats start from
        k_nn_batch<<<sm_count() * nn_max, kBlock, 0, s>>>(d_slots, d_heads, d_tile_slot, d_tile_local, d_ctl, 32,
                                                          0xffffffffu, 0);
        counters().launches += 1;
        for (const auto &cd : cands) {
            const int c = cd[0], so = cd[1];
            for (int pi = 0; pi < 2; ++pi) {
                const int ps = per_sm[pi];
                if (ps < 1 || ps > nn_max || (pi == 1 && ps == per_sm[0])) continue;
                k_reset_nn_ticket<<<1, 1, 0, s>>>(d_ctl);
                cudaEventRecord(e0, s);
                k_nn_batch<<<sm_count() * ps, kBlock, 0, s>>>(d_slots, d_heads, d_tile_slot, d_tile_local, d_ctl, c,
                                                              0xffffffffu, so);
                cudaEventRecord(e1, s);
                counters().launches += 2;
                e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) break;
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best_ms) {
                    best_ms = ms;
                    best = BatchShape{c, ps, acc_max, so};
                }
            }
            if (e != cudaSuccess) break;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (e != cudaSuccess) return e;
        shape = best;
        g_last_shape = shape;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[key] = shape;
        return cudaSuccess;
    }
};

}  // namespace fricp

using fricp::BatchEngine;
using fricp::counters;
using fricp::PairState;
using fricp::TargetDev;
using namespace fricp::host;

namespace {

// Device buffers of one registration, carved out of one allocation.
struct PairBuffers {
    char *base = nullptr;
    PairState *st = nullptr;
    float4 *src = nullptr;
    int *prev = nullptr;
    double *partial = nullptr;
    double *resid = nullptr;
    double *trace = nullptr;
    size_t bytes = 0;

    static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
    static size_t need(int64_t m, int trace_cap) {
        const int64_t ntiles = (m + fricp::kBlock - 1) / fricp::kBlock;
        return align256(sizeof(PairState)) + align256(sizeof(float4) * m) + align256(sizeof(int) * m) +
               align256(sizeof(double) * ntiles * fricp::kMaxSums) + align256(sizeof(double) * m) +
               align256(sizeof(double) * (trace_cap > 0 ? trace_cap : 1));
    }
    cudaError_t alloc(int64_t m, int trace_cap, cudaStream_t s) {
        bytes = need(m, trace_cap);
        cudaError_t e = cudaMallocAsync(&base, bytes, s);
        if (e != cudaSuccess) return e;
        const int64_t ntiles = (m + fricp::kBlock - 1) / fricp::kBlock;
        char *p = base;
        st = reinterpret_cast<PairState *>(p);
        p += align256(sizeof(PairState));
        src = reinterpret_cast<float4 *>(p);
        p += align256(sizeof(float4) * m);
        prev = reinterpret_cast<int *>(p);
        p += align256(sizeof(int) * m);
        partial = reinterpret_cast<double *>(p);
        p += align256(sizeof(double) * ntiles * fricp::kMaxSums);
        resid = reinterpret_cast<double *>(p);
        p += align256(sizeof(double) * m);
        trace = reinterpret_cast<double *>(p);
        return cudaSuccess;
    }
    void free(cudaStream_t s) {
        if (base) cudaFreeAsync(base, s);
        base = nullptr;
    }
};

// Stage, pack and set up one registration into freshly allocated buffers on
// stream s; the state, the cleared correspondences and the slot descriptor are
// written on stream `commit` (ordered after s) so that a running step graph on
// `commit` never sees a half-written slot.
fricp_status admit_pair(const fricp_target *target, const float *p_xyz, int64_t m, int on_device, const double *T0,
                        const fricp_params &prm, int trace_cap, cudaStream_t s, PairBuffers *buf, PairState *h,
                        double *scale, double c[3], fricp::Slot *slot) {
    const TargetDev &t = *fricp::target_dev(target);
    DevInput p;
    fricp_status st = stage_input(p_xyz, m, on_device, s, &p, "p_xyz");
    if (st != FRICP_OK) return st;
    if (buf->alloc(m, trace_cap, s) != cudaSuccess) return fail(FRICP_ENOMEM, "device allocation for a registration");
    float plo[3], phi[3];
    int bad = 0;
    cudaError_t e = fricp::prepare_source(p.ptr, m, s, buf->src, plo, phi, &bad);
    if (e != cudaSuccess) return cuda_fail(e, "preparing the source");
    if (bad) return fail(FRICP_EINVAL, "p_xyz has NaN or Inf");
    st = setup_pair(t, prm, m, plo, phi, T0, trace_cap, s, h, scale, c);
    if (st != FRICP_OK) return st;
    slot->st = buf->st;
    slot->ix = fricp::make_index(t);
    slot->src = buf->src;
    slot->prev = buf->prev;
    slot->partial = buf->partial;
    slot->resid = buf->resid;
    slot->trace = trace_cap > 0 ? buf->trace : nullptr;
    slot->ntiles = h->ntiles;
    slot->live = 1;
    return FRICP_OK;
}

fricp_status check_pair(const fricp_target *t, const float *p, int64_t m, const double *T0,
                        const fricp_params *prm) {
    if (!t || !p || !prm) return fail(FRICP_EINVAL, "NULL argument");
    if (m < 1 || m > (int64_t)1 << 30) return fail(FRICP_EINVAL, "m must be in 1..2^30");
    fricp_status st = check_params(prm);
    if (st != FRICP_OK) return st;
    if (fricp::variant_sym(prm->variant))
        return fail(FRICP_EUNSUPPORTED, "the symmetric objective needs source normals: fricp_register_symmetric");
    if (fricp::variant_p2pl(prm->variant) && !fricp::target_dev(t)->has_normals)
        return fail(FRICP_EUNSUPPORTED, "point-to-plane needs target normals");
    if (T0)
        for (int i = 0; i < 16; ++i)
            if (!std::isfinite(T0[i])) return fail(FRICP_EINVAL, "T0 has NaN or Inf");
    return FRICP_OK;
}

}  // namespace

extern "C" fricp_status fricp_batch_register(int32_t npairs, const fricp_target *const *targets,
                                             const float *const *p_xyz, const int64_t *m, int32_t on_device,
                                             const double *T0, const fricp_params *params, void *stream,
                                             fricp_result *out, double *trace, int32_t trace_capacity) {
    const auto wall0 = std::chrono::steady_clock::now();
    if (npairs < 1 || npairs > fricp::kMaxSlots) return fail(FRICP_EINVAL, "npairs must be in 1..4096");
    if (!targets || !p_xyz || !m || !params || !out) return fail(FRICP_EINVAL, "NULL argument");
    if (trace_capacity < 0 || (trace_capacity > 0 && !trace)) return fail(FRICP_EINVAL, "bad trace buffer");
    int64_t total_tiles = 0, total_points = 0;
    for (int i = 0; i < npairs; ++i) {
        fricp_status st = check_pair(targets[i], p_xyz[i], m[i], T0 ? T0 + 16 * i : nullptr, params + i);
        if (st != FRICP_OK) {
            fail(st, "pair " + std::to_string(i) + ": " + fricp_last_error());
            return st;
        }
        total_tiles += (m[i] + fricp::kBlock - 1) / fricp::kBlock;
        total_points += m[i];
    }
    if (total_tiles > ((int64_t)1 << 30) / fricp::kBlock) return fail(FRICP_EINVAL, "too many points in one batch");
    std::memset(out, 0, sizeof(fricp_result) * npairs);
    const fricp_params &ctl_prm = params[0];
    Ordered ord(stream);
    const cudaStream_t s = ord.work;
    BatchEngine eng;
    if (eng.init(npairs, (int)total_tiles, s) != cudaSuccess) return fail(FRICP_ENOMEM, "batch tables");
    std::vector<PairBuffers> bufs(npairs);
    std::vector<PairState> states(npairs);
    std::vector<double> scales(npairs), centers(3 * npairs);
    bool leak = false;
    struct Cleanup {
        std::vector<PairBuffers> &b;
        cudaStream_t s;
        bool &leak;
        ~Cleanup() {
            if (!leak)
                for (auto &x : b) x.free(s);
        }
    } cleanup{bufs, s, leak};
    for (int i = 0; i < npairs; ++i) {
        fricp::Slot sl;
        fricp_status st = admit_pair(targets[i], p_xyz[i], m[i], on_device, T0 ? T0 + 16 * i : nullptr, params[i],
                                     trace_capacity, s, &bufs[i], &states[i], &scales[i], &centers[3 * i], &sl);
        if (st != FRICP_OK) {
            fail(st, "pair " + std::to_string(i) + ": " + fricp_last_error());
            return st;
        }
        cudaError_t e = cudaMemcpyAsync(bufs[i].st, &states[i], sizeof(PairState), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(bufs[i].prev, 0xff, sizeof(int) * m[i], s);
        if (e == cudaSuccess) e = eng.upload_slot(i, sl);
        counters().h2d += sizeof(PairState);
        if (e != cudaSuccess) return cuda_fail(e, "uploading a registration");
    }
    cudaError_t e = eng.tune(total_points, npairs);
    if (e != cudaSuccess) return cuda_fail(e, "tuning the batched step");
    const int chunk = ctl_prm.use_graph ? ctl_prm.steps_per_sync : 1;
    e = eng.capture(chunk);
    if (e != cudaSuccess) return cuda_fail(e, "capturing the batched step");

    using clock = std::chrono::steady_clock;
    const auto deadline = clock::now() + std::chrono::duration_cast<clock::duration>(
                                             std::chrono::duration<double>(ctl_prm.timeout_s));
    cudaEvent_t poll;
    cudaEventCreateWithFlags(&poll, cudaEventDisableTiming);
    fricp_status rs = FRICP_OK;
    int64_t steps = 0;
    for (;;) {
        e = eng.run_graph();
        if (e == cudaSuccess) e = eng.fetch_status();
        if (e == cudaSuccess) e = cudaEventRecord(poll, s);
        if (e != cudaSuccess) {
            rs = cuda_fail(e, "running the batched step");
            break;
        }
        steps += chunk;
        rs = wait_event(poll, deadline);
        if (rs != FRICP_OK) {
            leak = true;   // steps may still be queued: keep their buffers alive
            break;
        }
        if (eng.h_ctl->overflow) {
            rs = fail(FRICP_EOVERFLOW, "batched tile list overflow");
            break;
        }
        if (eng.h_ctl->active == 0) break;
        if (steps >= ctl_prm.max_steps) {
            rs = fail(FRICP_ETIMEOUT, "step budget exhausted before convergence");
            break;
        }
    }
    cudaEventDestroy(poll);
    if (leak) {
        eng.d_slots = nullptr;   // the queued steps still read the tables
        eng.d_heads = nullptr;
        eng.d_done = eng.d_tile_slot = eng.d_tile_local = nullptr;
        eng.d_ctl = nullptr;
        return rs;
    }
    if (rs != FRICP_OK && rs != FRICP_ETIMEOUT) return rs;
    for (int i = 0; i < npairs; ++i) {
        e = cudaMemcpyAsync(&states[i], bufs[i].st, sizeof(PairState), cudaMemcpyDeviceToHost, s);
        counters().d2h += sizeof(PairState);
        if (e == cudaSuccess && trace_capacity > 0) {
            e = cudaMemcpyAsync(trace + (size_t)i * trace_capacity, bufs[i].trace, sizeof(double) * trace_capacity,
                                cudaMemcpyDeviceToHost, s);
            counters().d2h += (int64_t)sizeof(double) * trace_capacity;
        }
        if (e != cudaSuccess) return cuda_fail(e, "reading the results");
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "reading the results");
    const double wall = std::chrono::duration<double, std::milli>(clock::now() - wall0).count();
    for (int i = 0; i < npairs; ++i) {
        fill_result(states[i], params[i].variant, scales[i], &centers[3 * i], trace_capacity, out + i);
        out[i].wall_ms = wall;
    }
    return rs;
}

extern "C" fricp_status fricp_batch_set_shape(int32_t chunk, int32_t search_blocks_per_sm, int32_t static_order) {
    if (chunk != 0 && (chunk < 1 || chunk > fricp::kBlock || fricp::kBlock % chunk != 0 || search_blocks_per_sm < 1 ||
                       static_order < fricp::kOrderCounter || static_order > fricp::kOrderTiles))
        return fricp::host::fail(FRICP_EINVAL, "batch shape: chunk must divide 256, blocks per SM >= 1, order 0, 1 or 2");
    std::lock_guard<std::mutex> lk(fricp::g_tune_mu);
    fricp::g_forced = fricp::BatchShape{static_order == fricp::kOrderTiles ? fricp::kTileQ : chunk,
                                        search_blocks_per_sm, 0, static_order};
    return FRICP_OK;
}

extern "C" void fricp_batch_last_shape(int32_t *chunk, int32_t *search_blocks_per_sm,
                                       int32_t *accumulate_blocks_per_sm, int32_t *static_order) {
    std::lock_guard<std::mutex> lk(fricp::g_tune_mu);
    if (static_order) *static_order = fricp::g_last_shape.order;
    if (chunk) *chunk = fricp::g_last_shape.chunk;
    if (search_blocks_per_sm) *search_blocks_per_sm = fricp::g_last_shape.nn_per_sm;
    if (accumulate_blocks_per_sm) *accumulate_blocks_per_sm = fricp::g_last_shape.acc_per_sm;
}

// ---------------------------------------------------------------------------
// Serving loop: continuous batching over the batched step engine.
// ---------------------------------------------------------------------------

namespace {

struct Request {
    uint64_t ticket = 0;
    const fricp_target *target = nullptr;
    std::vector<float> host_pts;   // copy of a host source
    float *dev_pts = nullptr;      // library copy of a device source
    int64_t m = 0;
    bool has_T0 = false;
    double T0[16];
    fricp_params prm;
    size_t bytes = 0;              // device buffers while in flight
};

struct Running {
    Request req;
    PairBuffers buf;
    double scale = 1.0, c[3] = {0, 0, 0};
};

}  // namespace

struct fricp_server {
    BatchEngine eng;
    cudaStream_t s_step = nullptr, s_admit = nullptr, user = nullptr;
    cudaEvent_t ev_admit = nullptr, ev_user = nullptr, poll = nullptr;
    size_t budget = 0, used = 0;
    int max_slots = 0;
    int steps_per_graph = 16;
    int max_queue = 0;
    bool tuned = false;
    std::pair<int, int> tuned_class{-1, -1};   // size class the step graph's shape was tuned for
    double timeout_s = 600.0;
    std::deque<Request> queue;
    std::vector<std::unique_ptr<Running>> slots;
    std::map<uint64_t, fricp_result> finished;
    // targets of the requests in flight: requests using each, and the bytes
    // counted against the budget for it (once per distinct target)
    std::map<const fricp_target *, std::pair<int, size_t>> targets;
    uint64_t next_ticket = 1;
    std::mutex mu;
};

namespace {

// Device bytes of a target's index: points, normals, box tree, oriented bucket boxes and (once built)
// the FP16 storage.
size_t target_bytes(const fricp_target *t) {
    const TargetDev &d = *fricp::target_dev(t);
    size_t b = sizeof(float4) * (size_t)d.n * (d.has_normals ? 2 : 1) + sizeof(float4) * 8 * (size_t)d.L;
    if (d.pts16) b += sizeof(ushort4) * (size_t)d.n;
    return b;
}

// Bytes a request adds to the budget in use: its own buffers, and its target's
// index unless a request in flight already holds that target (FP16 storage is
// counted as if it will be built).
size_t admission_bytes(const fricp_server *sv, const Request &rq) {
    size_t b = rq.bytes;
    if (sv->targets.find(rq.target) == sv->targets.end()) {
        b += target_bytes(rq.target);
        if (rq.prm.precision == FRICP_PREC_FP16_STORAGE && fricp::target_dev(rq.target)->pts16 == nullptr)
            b += sizeof(ushort4) * (size_t)fricp::target_dev(rq.target)->n;
    }
    return b;
}

// Admission of the queue's head requests that fit (FIFO, a free slot and room
// in the budget): heavy work on s_admit, then the commit of each one on s_step
// (after everything already queued there).
fricp_status admit_queued(fricp_server *sv, int *admitted) {
    *admitted = 0;
    while (!sv->queue.empty()) {
        Request &rq = sv->queue.front();
        const size_t need = admission_bytes(sv, rq);
        if (sv->used + need > sv->budget) break;
        int slot = -1;
        for (int p = 0; p < sv->max_slots; ++p)
            if (!sv->slots[p]) {
                slot = p;
                break;
            }
        if (slot < 0) break;
        auto run = std::make_unique<Running>();
        run->req = std::move(rq);
        sv->queue.pop_front();
        Request &r = run->req;
        PairState h;
        fricp::Slot sl;
        const float *src = r.dev_pts ? r.dev_pts : r.host_pts.data();
        fricp_status st = admit_pair(r.target, src, r.m, r.dev_pts != nullptr, r.has_T0 ? r.T0 : nullptr, r.prm, 0,
                                     sv->s_admit, &run->buf, &h, &run->scale, run->c, &sl);
        if (st != FRICP_OK) {   // the request fails alone; the server carries on
            fricp_result res;
            std::memset(&res, 0, sizeof(res));
            res.status = st;
            sv->finished[r.ticket] = res;
            run->buf.free(sv->s_admit);
            if (r.dev_pts) cudaFreeAsync(r.dev_pts, sv->s_admit);
            continue;
        }
        cudaError_t e = cudaEventRecord(sv->ev_admit, sv->s_admit);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sv->s_step, sv->ev_admit, 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(run->buf.st, &h, sizeof(PairState), cudaMemcpyHostToDevice, sv->s_step);
        if (e == cudaSuccess) e = cudaMemsetAsync(run->buf.prev, 0xff, sizeof(int) * r.m, sv->s_step);
        if (e == cudaSuccess) e = sv->eng.upload_slot(slot, sl);
        counters().h2d += sizeof(PairState);
        if (e != cudaSuccess) return cuda_fail(e, "admitting a request");
        if (r.dev_pts) {
            cudaFreeAsync(r.dev_pts, sv->s_step);
            r.dev_pts = nullptr;
        }
        r.host_pts.clear();
        r.host_pts.shrink_to_fit();
        auto &tr = sv->targets[r.target];
        if (tr.first++ == 0) tr.second = need - r.bytes;
        sv->used += need;
        sv->slots[slot] = std::move(run);
        ++*admitted;
    }
    return FRICP_OK;
}

// Results of the slots the last plan reported done: read, convert, free.
fricp_status harvest(fricp_server *sv) {
    std::vector<int> ready;
    for (int p = 0; p < sv->max_slots; ++p)
        if (sv->slots[p] && sv->eng.h_done[p]) ready.push_back(p);
    if (ready.empty()) return FRICP_OK;
    std::vector<PairState> states(ready.size());
    cudaError_t e = cudaSuccess;
    for (size_t k = 0; k < ready.size() && e == cudaSuccess; ++k) {
        e = cudaMemcpyAsync(&states[k], sv->slots[ready[k]]->buf.st, sizeof(PairState), cudaMemcpyDeviceToHost,
                            sv->s_step);
        counters().d2h += sizeof(PairState);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(sv->s_step);
    if (e != cudaSuccess) return cuda_fail(e, "reading finished requests");
    fricp::Slot empty;
    std::memset(&empty, 0, sizeof(empty));
    for (size_t k = 0; k < ready.size(); ++k) {
        const int p = ready[k];
        Running &run = *sv->slots[p];
        fricp_result res;
        std::memset(&res, 0, sizeof(res));
        fill_result(states[k], run.req.prm.variant, run.scale, run.c, 0, &res);
        sv->finished[run.req.ticket] = res;
        e = sv->eng.upload_slot(p, empty);   // stream-ordered before the buffers are freed and reused
        if (e != cudaSuccess) return cuda_fail(e, "releasing a slot");
        run.buf.free(sv->s_step);
        sv->used -= run.req.bytes;
        auto it = sv->targets.find(run.req.target);
        if (it != sv->targets.end() && --it->second.first == 0) {
            sv->used -= it->second.second;
            sv->targets.erase(it);
        }
        sv->slots[p].reset();
    }
    return FRICP_OK;
}

int count_in_flight(const fricp_server *sv) {
    int n = 0;
    for (const auto &r : sv->slots) n += r != nullptr;
    return n;
}

}  // namespace

extern "C" fricp_status fricp_server_create(size_t hbm_budget, int32_t max_slots, int32_t steps_per_sync,
                                            int32_t max_queue, void *stream, fricp_server **out) {
    if (!out) return fail(FRICP_EINVAL, "NULL argument");
    *out = nullptr;
    if (max_slots < 1 || max_slots > fricp::kMaxSlots) return fail(FRICP_EINVAL, "max_slots must be in 1..4096");
    if (steps_per_sync < 1 || steps_per_sync > 4096) return fail(FRICP_EINVAL, "steps_per_sync in 1..4096");
    if (max_queue < 1) return fail(FRICP_EINVAL, "max_queue must be >= 1");
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return cuda_fail(e, "querying device memory");
    if (hbm_budget == 0) hbm_budget = free_b / 2;
    if (hbm_budget > free_b) return fail(FRICP_EINVAL, "hbm_budget exceeds free device memory");
    auto sv = std::make_unique<fricp_server>();
    sv->budget = hbm_budget;
    sv->max_slots = max_slots;
    sv->steps_per_graph = steps_per_sync;
    sv->max_queue = max_queue;
    sv->user = (cudaStream_t)stream;
    sv->slots.resize(max_slots);
    e = cudaStreamCreateWithFlags(&sv->s_step, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->s_admit, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sv->ev_admit, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sv->ev_user, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sv->poll, cudaEventDisableTiming);
    // the tile list holds every tile the budget can keep in flight, plus one per slot
    const int64_t max_points = (int64_t)(hbm_budget / (sizeof(float4) + sizeof(int) + sizeof(double))) + 1;
    const int64_t tiles = max_points / fricp::kBlock + max_slots + 1;
    if (e == cudaSuccess) e = sv->eng.init(max_slots, (int)std::min<int64_t>(tiles, 1 << 30), sv->s_step);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sv->s_step);
    if (e != cudaSuccess) {
        fricp_server *raw = sv.release();
        fricp_server_destroy(raw);
        return cuda_fail(e, "creating the server");
    }
    *out = sv.release();
    return FRICP_OK;
}

extern "C" fricp_status fricp_server_submit(fricp_server *sv, const fricp_target *target, const float *p_xyz,
                                            int64_t m, int32_t on_device, const double *T0,
                                            const fricp_params *params, uint64_t *ticket) {
    if (!sv || !ticket) return fail(FRICP_EINVAL, "NULL argument");
    fricp_status st = check_pair(target, p_xyz, m, T0, params);
    if (st != FRICP_OK) return st;
    std::lock_guard<std::mutex> lk(sv->mu);
    if ((int)sv->queue.size() >= sv->max_queue) return fail(FRICP_EBUSY, "request queue is full");
    Request r;
    r.target = target;
    r.m = m;
    r.prm = *params;
    r.has_T0 = T0 != nullptr;
    if (T0) std::memcpy(r.T0, T0, sizeof(r.T0));
    r.bytes = PairBuffers::need(m, 0);
    if (r.bytes + target_bytes(target) > sv->budget)
        return fail(FRICP_EINVAL, "request and its target need more device memory than the server budget");
    if (on_device) {
        cudaError_t e = cudaEventRecord(sv->ev_user, sv->user);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sv->s_admit, sv->ev_user, 0);
        if (e == cudaSuccess) e = cudaMallocAsync(&r.dev_pts, sizeof(float) * 3 * m, sv->s_admit);
        if (e != cudaSuccess) return fail(FRICP_ENOMEM, "device copy of a request");
        e = cudaMemcpyAsync(r.dev_pts, p_xyz, sizeof(float) * 3 * m, cudaMemcpyDeviceToDevice, sv->s_admit);
        if (e == cudaSuccess) e = cudaEventRecord(sv->ev_user, sv->s_admit);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sv->user, sv->ev_user, 0);   // caller may reuse p_xyz after it
        if (e != cudaSuccess) return cuda_fail(e, "copying a request");
    } else {
        if (!host_finite(p_xyz, 3 * m)) return fail(FRICP_EINVAL, "p_xyz has NaN or Inf");
        r.host_pts.assign(p_xyz, p_xyz + 3 * m);
    }
    r.ticket = sv->next_ticket++;
    *ticket = r.ticket;
    sv->queue.push_back(std::move(r));
    return FRICP_OK;
}

extern "C" fricp_status fricp_server_step(fricp_server *sv, int32_t nsteps, int32_t *in_flight, int32_t *queued) {
    if (!sv) return fail(FRICP_EINVAL, "NULL argument");
    if (nsteps < 0) return fail(FRICP_EINVAL, "nsteps must be >= 0");
    std::lock_guard<std::mutex> lk(sv->mu);
    int admitted = 0;
    fricp_status st = FRICP_OK;
    if (!sv->tuned) {
        st = admit_queued(sv, &admitted);
        if (st != FRICP_OK) return st;
    }
    {
        // the launch shape follows the work in flight: re-tuned (once per size
        // class, remembered) whenever the class changes, the graph re-captured
        // when the shape does
        int64_t pts = 0;
        for (const auto &r : sv->slots)
            if (r) pts += r->req.m;
        const int n = count_in_flight(sv);
        if (n > 0) {
            const auto cls = fricp::size_class(pts, n);
            if (!sv->tuned || cls != sv->tuned_class) {
                cudaError_t e = sv->eng.tune(pts, n);
                if (e == cudaSuccess) e = sv->eng.capture(sv->steps_per_graph);
                if (e != cudaSuccess) return cuda_fail(e, "tuning the served step");
                sv->tuned = true;
                sv->tuned_class = cls;
            }
        }
    }
    const int graphs = sv->tuned && count_in_flight(sv) > 0 ? (nsteps + sv->steps_per_graph - 1) / sv->steps_per_graph : 0;
    for (int k = 0; k < graphs; ++k) {
        const cudaError_t e = sv->eng.run_graph();
        if (e != cudaSuccess) return cuda_fail(e, "running the served step");
    }
    // admission overlaps the steps just launched
    st = admit_queued(sv, &admitted);
    if (st != FRICP_OK) return st;
    cudaError_t e = sv->eng.fetch_status();
    if (e == cudaSuccess) e = cudaEventRecord(sv->poll, sv->s_step);
    if (e != cudaSuccess) return cuda_fail(e, "polling the served step");
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                              std::chrono::duration<double>(sv->timeout_s));
    st = wait_event(sv->poll, deadline);
    if (st != FRICP_OK) return st;
    if (sv->eng.h_ctl->overflow) return fail(FRICP_EOVERFLOW, "served tile list overflow");
    if (graphs > 0) {   // the done flags describe the state after the launched steps
        st = harvest(sv);
        if (st != FRICP_OK) return st;
    }
    if (in_flight) *in_flight = count_in_flight(sv);
    if (queued) *queued = (int32_t)sv->queue.size();
    return FRICP_OK;
}

extern "C" fricp_status fricp_server_poll(fricp_server *sv, uint64_t ticket, fricp_result *out, int32_t *done) {
    if (!sv || !out || !done) return fail(FRICP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->finished.find(ticket);
    if (it == sv->finished.end()) {
        *done = 0;
        if (ticket == 0 || ticket >= sv->next_ticket) return fail(FRICP_EINVAL, "unknown ticket");
        return FRICP_OK;
    }
    *out = it->second;
    *done = 1;
    sv->finished.erase(it);
    return FRICP_OK;
}

extern "C" fricp_status fricp_server_destroy(fricp_server *sv) {
    if (!sv) return FRICP_OK;
    if (sv->s_step) cudaStreamSynchronize(sv->s_step);
    if (sv->s_admit) cudaStreamSynchronize(sv->s_admit);
    for (auto &r : sv->slots)
        if (r) r->buf.free(sv->s_step);
    for (auto &r : sv->queue)
        if (r.dev_pts) cudaFreeAsync(r.dev_pts, sv->s_step);
    if (sv->s_step) cudaStreamSynchronize(sv->s_step);
    sv->eng.release();
    if (sv->ev_admit) cudaEventDestroy(sv->ev_admit);
    if (sv->ev_user) cudaEventDestroy(sv->ev_user);
    if (sv->poll) cudaEventDestroy(sv->poll);
    if (sv->s_step) cudaStreamDestroy(sv->s_step);
    if (sv->s_admit) cudaStreamDestroy(sv->s_admit);
    delete sv;
    return FRICP_OK;
}
