// bsw_api.cu - C ABI and host runtime of the BSW library (see include/bsw.h).
//
// Host side of the batched extension: argument checks, a device-memory arena
// held within the context's budget, staging of host inputs, CUDA-graph replay
// for device-pointer calls, and the serving loop (bsw_stream_submit/poll):
// a server thread that admits queued batches into a few execution lanes (one
// stream set and buffer set each), merges small batches into one launch and
// overlaps lanes on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <system_error>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bsw.h"
#include "bsw_device.cuh"
#include "bsw_launch.h"

extern "C" int bsw_sa_build(const uint8_t *codes, int64_t n, int32_t *sa);

using namespace bsw;

namespace {

constexpr uint32_t kKnownFlags = BSW_DEVICE_PTRS | BSW_FORCE_I8 | BSW_FORCE_I16 | BSW_FORCE_I32 |
                                 BSW_PLAIN_KERNEL | BSW_NO_GRAPH | BSW_COPY_INPUTS | BSW_PACKED_PAIRS |
                                 BSW_TIME_KERNELS | BSW_PLAIN_GLOBAL;
constexpr int64_t kTuneSample = 1 << 21;   // default autotune sample (pairs)
constexpr int kServeLanes = 3;
constexpr int64_t kMergePairs = 1 << 20;   // the serving loop merges queued batches up to this many pairs
constexpr int64_t kMergeCells = 4000000000ll;   // ... and up to this many estimated DP cells
constexpr int kGraphCache = 8;

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Budget {
    int64_t cap = 0;
    std::atomic<int64_t> used{0};
};

// ---------------------------------------------------------- fault injection
//
// bsw_fault_inject: listed host call sites fail after `skip` passing hits,
// `count` times.  The fast path of an unarmed site is one relaxed load.
struct Faults {
    std::mutex mu;
    std::atomic<uint32_t> sites{0};
    int32_t skip = 0, count = 0;
};

Faults &faults()
{
    static Faults f;
    return f;
}

bool fault_hit(uint32_t site)
{
    Faults &f = faults();
    if (!(f.sites.load(std::memory_order_relaxed) & site)) return false;
    std::lock_guard<std::mutex> lk(f.mu);
    if (!(f.sites.load() & site)) return false;
    if (f.skip > 0) {
        --f.skip;
        return false;
    }
    if (f.count > 0 && --f.count > 0) return true;
    f.sites = 0;   // the last failure, or nothing left to fail
    return true;
}

// "name[,name...][:skip[:count]]" with names alloc, h2d, launch, thread, host.
bool parse_faults(const char *spec, uint32_t *sites, int32_t *skip, int32_t *count)
{
    *sites = 0;
    *skip = 0;
    *count = 1;
    if (!spec || !*spec) {
        *count = 0;
        return true;
    }
    const char *p = spec;
    for (;;) {
        const char *q = p;
        while (*q && *q != ',' && *q != ':') ++q;
        const size_t len = (size_t)(q - p);
        static const struct { const char *name; uint32_t bit; } kSites[] = {
            {"alloc", BSW_FAULT_ALLOC}, {"h2d", BSW_FAULT_H2D}, {"launch", BSW_FAULT_LAUNCH},
            {"thread", BSW_FAULT_THREAD}, {"host", BSW_FAULT_HOST}};
        uint32_t bit = 0;
        for (const auto &k : kSites)
            if (std::strlen(k.name) == len && std::strncmp(k.name, p, len) == 0) bit = k.bit;
        if (!bit) return false;
        *sites |= bit;
        p = q;
        if (*p != ',') break;
        ++p;
    }
    int32_t *num[2] = {skip, count};
    for (int k = 0; k < 2 && *p == ':'; ++k) {
        ++p;
        if (*p < '0' || *p > '9') return false;
        long v = 0;
        while (*p >= '0' && *p <= '9') {
            v = v * 10 + (*p++ - '0');
            if (v > INT32_MAX) return false;
        }
        *num[k] = (int32_t)v;
    }
    return *p == '\0';
}

void set_faults(uint32_t sites, int32_t skip, int32_t count)
{
    Faults &f = faults();
    std::lock_guard<std::mutex> lk(f.mu);
    f.skip = skip;
    f.count = count;
    f.sites = count > 0 ? sites : 0u;
}

// BSW_FAULT_INJECT in the environment when the library loads.
struct FaultsFromEnv {
    FaultsFromEnv()
    {
        uint32_t s;
        int32_t k, c;
        if (parse_faults(std::getenv("BSW_FAULT_INJECT"), &s, &k, &c)) set_faults(s, k, c);
    }
} g_faults_from_env;

// A host-to-device copy that the h2d site can make fail.
cudaError_t h2d(void *dst, const void *src, size_t bytes, cudaStream_t st)
{
    if (fault_hit(BSW_FAULT_H2D)) return cudaErrorInvalidValue;
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
}

// One growable device allocation, charged to the context's budget.
struct DevBuf {
    uint8_t *p = nullptr;
    size_t cap = 0;

    int reserve(size_t bytes, Budget &B, bool *moved = nullptr)
    {
        if (bytes <= cap) return BSW_OK;
        size_t want = align_up(std::max(bytes, cap + cap / 4), 1 << 20);
        if (B.used.load() - (int64_t)cap + (int64_t)want > B.cap) want = align_up(bytes, 256);
        if (B.used.load() - (int64_t)cap + (int64_t)want > B.cap) return BSW_EBUDGET;
        release(B);
        if (fault_hit(BSW_FAULT_ALLOC) || cudaMalloc(&p, want) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            if (moved) *moved = true;   // the old buffer is gone too
            return BSW_ENOMEM;
        }
        cap = want;
        B.used += (int64_t)want;
        if (moved) *moved = true;
        return BSW_OK;
    }
    void release(Budget &B)
    {
        if (p) {
            cudaFree(p);
            B.used -= (int64_t)cap;
        }
        p = nullptr;
        cap = 0;
    }
};

// Byte offsets of the work buffers inside one allocation.
struct WorkLayout {
    size_t key, order, rec, rerun, hist, cursor, cls_start, cls_count, cls_next, cells, status, slots, total;
    int64_t slot_bytes;
};

WorkLayout work_layout(int64_t n, int64_t slot_bytes, int nwarps)
{
    WorkLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
    L.key = take(4 * (size_t)n);
    L.order = take(4 * (size_t)n);
    L.rec = take(sizeof(PairRec) * (size_t)n);
    L.rerun = take(4 * (size_t)n);
    L.hist = take(4 * kNumBins);
    L.cursor = take(4 * kNumBins);
    L.cls_start = take(4 * (kNumClass + 1));
    L.cls_count = take(4 * (kNumClass + 1));
    L.cls_next = take(4 * kNumCounters);
    L.cells = take(8);
    L.status = take(4);
    L.slots = take((size_t)slot_bytes * (size_t)nwarps);
    L.total = o;
    L.slot_bytes = slot_bytes;
    return L;
}

Work make_work(uint8_t *base, const WorkLayout &L)
{
    Work W;
    W.key = (int32_t *)(base + L.key);
    W.order = (int32_t *)(base + L.order);
    W.rec = (PairRec *)(base + L.rec);
    W.rerun = (int32_t *)(base + L.rerun);
    W.hist = (uint32_t *)(base + L.hist);
    W.cursor = (uint32_t *)(base + L.cursor);
    W.cls_start = (int32_t *)(base + L.cls_start);
    W.cls_count = (int32_t *)(base + L.cls_count);
    W.cls_next = (uint32_t *)(base + L.cls_next);
    W.cells = (unsigned long long *)(base + L.cells);
    W.status = (uint32_t *)(base + L.status);
    W.slots = base + L.slots;
    W.slot_bytes_per_warp = L.slot_bytes;
    return W;
}

int64_t slot_bytes_for(int maxn) { return (int64_t)align_up((size_t)(maxn + 1 + 32 * 8) * 8, 256); }

// One execution lane: a stream set, work buffers and staging buffers.
struct Lane {
    Streams S{};
    cudaEvent_t done = nullptr;
    cudaEvent_t t_start = nullptr, t_end = nullptr;   // serving lanes: a launch's device interval
    DevBuf work, io, seq;       // seq: sequences of a staged host batch
    WorkLayout wl{};
    bool work_dirty = true;     // histogram must be zeroed before the next launch
    uint8_t *pinned = nullptr;  // host staging (serving lanes)
    size_t pinned_cap = 0;

    int create()
    {
        if (cudaStreamCreateWithFlags(&S.main, cudaStreamNonBlocking) != cudaSuccess) return BSW_ECUDA;
        for (int k = 0; k < 3; ++k) {
            if (cudaStreamCreateWithFlags(&S.side[k], cudaStreamNonBlocking) != cudaSuccess) return BSW_ECUDA;
            if (cudaEventCreateWithFlags(&S.join[k], cudaEventDisableTiming) != cudaSuccess) return BSW_ECUDA;
        }
        if (cudaEventCreateWithFlags(&S.fork, cudaEventDisableTiming) != cudaSuccess) return BSW_ECUDA;
        if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) return BSW_ECUDA;
        if (cudaEventCreate(&t_start) != cudaSuccess || cudaEventCreate(&t_end) != cudaSuccess) return BSW_ECUDA;
        return BSW_OK;
    }
    void destroy(Budget &B)
    {
        if (S.main) cudaStreamSynchronize(S.main);
        for (int k = 0; k < 3; ++k) {
            if (S.side[k]) { cudaStreamSynchronize(S.side[k]); cudaStreamDestroy(S.side[k]); }
            if (S.join[k]) cudaEventDestroy(S.join[k]);
        }
        if (S.fork) cudaEventDestroy(S.fork);
        if (done) cudaEventDestroy(done);
        if (t_start) cudaEventDestroy(t_start);
        if (t_end) cudaEventDestroy(t_end);
        t_start = t_end = nullptr;
        if (S.main) cudaStreamDestroy(S.main);
        work.release(B);
        io.release(B);
        seq.release(B);
        if (pinned) cudaFreeHost(pinned);
        pinned = nullptr;
    }
    // Work buffers for n pairs and queries up to maxn; sets *moved on reallocation.
    int ensure_work(int64_t n, int maxn, int sms, Budget &B, bool *moved)
    {
        const int64_t sb = slot_bytes_for(maxn);
        const bool fits = wl.total && n <= (int64_t)(wl.order - wl.key) / 4 && sb <= wl.slot_bytes;
        if (fits && work.p) return BSW_OK;
        const int64_t n_cap = std::max<int64_t>(n, (int64_t)((wl.order - wl.key) / 4));
        const int64_t sb_cap = std::max<int64_t>(sb, wl.slot_bytes);
        WorkLayout L = work_layout(n_cap, sb_cap, warp_slots_needed(sms));
        bool m2 = false;
        int rc = work.reserve(L.total, B, &m2);
        if (rc != BSW_OK) return rc;
        wl = L;
        work_dirty = true;
        if (moved) *moved = true;
        return BSW_OK;
    }
    int ensure_pinned(size_t bytes)
    {
        if (bytes <= pinned_cap) return BSW_OK;
        if (pinned) cudaFreeHost(pinned);
        pinned = nullptr;
        pinned_cap = 0;
        size_t want = align_up(bytes + bytes / 4, 1 << 20);
        if (fault_hit(BSW_FAULT_ALLOC) || cudaMallocHost(&pinned, want) != cudaSuccess) {
            cudaGetLastError();
            pinned = nullptr;
            return BSW_ENOMEM;
        }
        pinned_cap = want;
        return BSW_OK;
    }
};

// Host-side check of one serving request (small batches; a synchronous host
// batch is checked on the device by stage_host); fills the packed-byte
// extents, the longest query and a bound on the band area.
struct Extents {
    int64_t q_lo = INT64_MAX, q_hi = 0, t_lo = INT64_MAX, t_hi = 0;
    int maxn = 0;
    int64_t est_cells = 0;   // sum of qlen * min(tlen, 2w + 1): a bound on the band area
};

int check_host_batch(const bsw_batch_t *b, const Params &P, Extents *x)
{
    const int64_t N = b->n_pairs;
    for (int64_t k = 0; k < N; ++k) {
        const int32_t n = b->q_len[k], m = b->t_len[k], h0 = b->h0[k];
        const int64_t qo = b->q_off[k], to = b->t_off[k];
        const int32_t w = b->w_override ? b->w_override[k] : P.w;
        if (n < 0 || m < 0 || h0 < 0 || w < 0 || qo < 0 || to < 0 || (qo & 3) || (to & 3)) return BSW_EINVAL;
        if (n > 0 && m > 0) {
            if ((int64_t)h0 + (int64_t)P.a * std::min(n, m) >= (1ll << 30)) return BSW_EINVAL;
            if (n > kLongMax) return BSW_EINVAL;
            x->q_lo = std::min(x->q_lo, qo / 4);
            x->q_hi = std::max(x->q_hi, (qo + n + 3) / 4);
            x->t_lo = std::min(x->t_lo, to / 4);
            x->t_hi = std::max(x->t_hi, (to + m + 3) / 4);
            x->maxn = std::max(x->maxn, n);
            x->est_cells += (int64_t)n * std::min<int64_t>(m, 2 * (int64_t)w + 1);
        }
    }
    if (x->q_lo > x->q_hi) x->q_lo = x->q_hi = 0;
    if (x->t_lo > x->t_hi) x->t_lo = x->t_hi = 0;
    return BSW_OK;
}

// Device layout of a staged serving batch (one contiguous copy from the lane's
// pinned staging).
struct IoLayout {
    size_t q, t, qn, tn, q_off, q_len, t_off, t_len, h0, w, out, cells, status, in_end, total;
};

// N bitmap bytes staged for packed bytes [lo, hi) (two packed bytes per
// bitmap byte; the first bitmap byte holds packed byte lo's bases).
inline int64_t nmask_lo(int64_t lo) { return lo / 2; }
inline int64_t nmask_bytes(int64_t lo, int64_t hi) { return hi > lo ? (hi + 1) / 2 - lo / 2 : 0; }

// qbytes, tbytes: the staged packed bytes; with N bitmaps (has_n) one bitmap
// byte per two packed bytes of each side.
IoLayout io_layout(int64_t N, int64_t qbytes, int64_t tbytes, bool has_n)
{
    IoLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
    L.q = take((size_t)qbytes);
    L.t = take((size_t)tbytes);
    L.qn = take(has_n ? (size_t)(qbytes + 1) / 2 : 0);
    L.tn = take(has_n ? (size_t)(tbytes + 1) / 2 : 0);
    L.q_off = take(8 * (size_t)N);
    L.q_len = take(4 * (size_t)N);
    L.t_off = take(8 * (size_t)N);
    L.t_len = take(4 * (size_t)N);
    L.h0 = take(4 * (size_t)N);
    L.w = take(4 * (size_t)N);
    L.in_end = o;
    L.out = take(sizeof(bsw_result_t) * (size_t)N);
    L.cells = take(8);
    L.status = take(4);
    L.total = o;
    return L;
}

int status_to_rc(uint32_t st) { return st ? BSW_EINVAL : BSW_OK; }

int cuda_rc(cudaError_t e)
{
    if (e == cudaSuccess) return BSW_OK;
    cudaGetLastError();
    return BSW_ECUDA;
}

// ---------------------------------------------------------------- serving

struct Request {
    uint64_t ticket = 0;
    bsw_batch_t b{};
    bsw_result_t *out = nullptr;
    Extents ext;
    std::vector<uint8_t> own;   // owned input copies (BSW_COPY_INPUTS)
    int status = BSW_PENDING;
    int64_t out_pos = 0;        // position of this request's pairs in the merged launch
    int64_t qpos = 0, tpos = 0; // first staged packed byte of its queries / targets
};

// Staged packed bytes of a request's side starting at cursor `pos`: the side
// starts on the parity of its first used byte lo (so base offsets move by a
// multiple of 8 and its N bitmap bytes copy unshifted) and on a bitmap byte
// of its own (so no bitmap byte is shared with the request before it).
inline int64_t stage_start(int64_t pos, int64_t lo) { return ((pos + 1) & ~(int64_t)1) + (lo & 1); }

// Serving counters (bsw_stream_stats) and each launch's device interval,
// in milliseconds from the context's reference event.
struct ServeStats {
    int64_t requests = 0, launches = 0, merged = 0, budget_waits = 0;
    std::vector<std::pair<float, float>> iv;
};
constexpr size_t kStatsIntervals = 1 << 16;   // intervals kept (the most recent)

}  // namespace

struct bsw_ctx {
    Params P{};
    int device = 0;
    int sms = 0;
    Budget budget;
    Lane sync;
    uint32_t *h_status = nullptr;     // pinned
    unsigned long long *h_cells = nullptr;
    Extents32 *h_ext = nullptr;
    DriverCheck *h_chk = nullptr;

    // execution plan (bsw_set_plan / bsw_autotune) and kernel timing
    Plan plan = default_plan();
    bsw_plan_t pub_plan{kShortMax, 0xffu, 0xfu, 0, 8, 2, 0, 0, 0.0f};
    ClassTimer timer{};
    bool timer_ready = false, timer_valid = false;
    cudaEvent_t tune_ev[2] = {nullptr, nullptr};
    int last_launches = 0;

    // seed-extension driver: the reference (bsw_set_reference) and the
    // buffers of a bsw_extend_seeds call
    DevBuf refbuf, drv, drvmeta;     // drvmeta: reads' offsets and lengths, seeds, checks
    int64_t ref_len = -1;
    bool ref_has_n = false;          // refbuf holds an N bitmap after the packed bases

    // suffix array lookup: the uncompressed suffix array and staging
    DevBuf sabuf, salio;
    int64_t sa_n = -1;

    // SMEM search: the FM-index of T = ref + revcomp(ref); staging, and the
    // global lists of reads whose lists overflow shared memory
    DevBuf fmbuf, smemio, smemscratch;
    FmDev fm_t{};
    bool fm_ready = false;

    struct GEntry {
        bsw_batch_t b;
        void *out, *cells;
        cudaGraphExec_t exec;
        int launches;
    };
    std::vector<GEntry> graphs;

    // serving
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> tickets;
    uint64_t next_ticket = 1;
    bool stop = false;
    bool server_started = false;
    std::thread server;
    Lane serve_lane[kServeLanes];
    bool lane_created[kServeLanes] = {false, false, false};
    std::vector<Request *> lane_reqs[kServeLanes];
    int64_t lane_pairs[kServeLanes] = {0, 0, 0};
    size_t lane_out_off[kServeLanes] = {0, 0, 0};
    IoLayout lane_io[kServeLanes];
    bool lane_busy[kServeLanes] = {false, false, false};
    bool lane_has_n[kServeLanes] = {false, false, false};
    bool mem_wait = false;            // an admission waits for memory held by busy lanes
    ServeStats stats;
    cudaEvent_t ref_ev = nullptr;     // reference point of the launch intervals
    bool ref_ok = false;
};

namespace {

void clear_graphs(bsw_ctx *c)
{
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
}

bool same_batch(const bsw_batch_t &a, const bsw_batch_t &b)
{
    return a.n_pairs == b.n_pairs && a.q == b.q && a.q_off == b.q_off && a.q_len == b.q_len && a.t == b.t &&
           a.t_off == b.t_off && a.t_len == b.t_len && a.h0 == b.h0 && a.w_override == b.w_override &&
           a.flags == b.flags && a.q_n == b.q_n && a.t_n == b.t_n;
}

// Enqueue one launch of a device-resident batch on the lane's streams (S.main
// may be replaced by the caller's stream).  Zeroes cells/status first.
cudaError_t enqueue_launch(bsw_ctx *c, Lane &lane, const Streams &S, const Batch &B, Work W, uint32_t flags,
                           bool reset_status, const Plan &L, ClassTimer *T = nullptr)
{
    cudaError_t e;
    Params P = c->P;
    P.flags = flags;
    const bool plain = (flags & (BSW_PLAIN_KERNEL | BSW_PLAIN_GLOBAL)) != 0;
    c->last_launches = plain ? plain_launches(P, L, flags) : batched_launches(L, flags);
    if (lane.work_dirty) {
        if ((e = cudaMemsetAsync(W.hist, 0, 4 * kNumBins, S.main)) != cudaSuccess) return e;
        lane.work_dirty = false;
    }
    if ((e = cudaMemsetAsync(W.cells, 0, 8, S.main)) != cudaSuccess) return e;
    if (reset_status && (e = cudaMemsetAsync(W.status, 0, 4, S.main)) != cudaSuccess) return e;
    if (fault_hit(BSW_FAULT_LAUNCH)) return cudaErrorLaunchFailure;
    return plain ? launch_plain(B, P, W, S.main, c->sms, L) : launch_batched(B, P, W, S, c->sms, L, T);
}

// Timing events for BSW_TIME_KERNELS (created on first use); nullptr when the
// flag is absent or the events cannot be made.
ClassTimer *timer_for(bsw_ctx *c, uint32_t flags)
{
    if (!(flags & BSW_TIME_KERNELS)) return nullptr;
    if (!c->timer_ready) {
        for (int k = 0; k <= kNumClass; ++k)
            if (cudaEventCreate(&c->timer.t0[k]) != cudaSuccess || cudaEventCreate(&c->timer.t1[k]) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
        c->timer_ready = true;
    }
    for (int k = 0; k <= kNumClass; ++k) c->timer.used[k] = false;
    c->timer_valid = true;
    return &c->timer;
}

// Device layout of a host batch staged by stage_host: the per-pair arrays, the
// results and the extents record in the lane's io buffer; the sequences and N
// bitmaps in its seq buffer, sized once the extents are known.
struct StageLayout {
    size_t q_off, q_len, t_off, t_len, h0, w, out, ext, total;
    size_t q, t, qn, tn, seq_total;
};

StageLayout stage_layout(int64_t N, bool has_w)
{
    StageLayout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
    L.q_off = take(8 * (size_t)N);
    L.q_len = take(4 * (size_t)N);
    L.t_off = take(8 * (size_t)N);
    L.t_len = take(4 * (size_t)N);
    L.h0 = take(4 * (size_t)N);
    L.w = take(has_w ? 4 * (size_t)N : 0);
    L.out = take(sizeof(bsw_result_t) * (size_t)N);
    L.ext = take(sizeof(Extents32));
    L.total = o;
    return L;
}

void stage_seq_layout(StageLayout &L, int64_t qbytes, int64_t tbytes, int64_t qnbytes, int64_t tnbytes)
{
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
    L.qn = take((size_t)qnbytes);
    L.tn = take((size_t)tnbytes);
    L.q = take((size_t)qbytes);
    L.t = take((size_t)tbytes);
    L.seq_total = o;
}

// Batches up to this many pairs are checked on the host: below it the host
// loop costs less than the device check's round trip.
constexpr int64_t kHostCheckMax = 32768;

// Stage a host batch on the sync lane (enqueued after `user`, nullable,
// reaches this point): copy the per-pair arrays, check them and reduce their
// extents (on the device with one small read-back, or on the host for small
// batches), then copy only the packed sequence bytes the pairs use; the
// device base pointers are shifted back by the first used byte so the
// caller's offsets stay valid.  Describes the staged batch as a device Batch
// whose results go to the io buffer.
int stage_host(bsw_ctx *c, const bsw_batch_t *b, cudaStream_t user, Batch *out_B, StageLayout *out_L)
{
    const int64_t N = b->n_pairs;
    Lane &lane = c->sync;
    StageLayout L = stage_layout(N, b->w_override != nullptr);
    bool moved = false;
    int rc;
    if ((rc = lane.io.reserve(L.total, c->budget, &moved)) != BSW_OK) return rc;
    uint8_t *d = lane.io.p;
    cudaStream_t st = lane.S.main;
    cudaError_t e;
    if (user) {
        if ((e = cudaEventRecord(lane.done, user)) != cudaSuccess) return cuda_rc(e);
        if ((e = cudaStreamWaitEvent(st, lane.done, 0)) != cudaSuccess) return cuda_rc(e);
    }
    struct Cp { size_t off; const void *src; size_t bytes; };
    const Cp meta[] = {
        {L.q_off, b->q_off, 8 * (size_t)N}, {L.q_len, b->q_len, 4 * (size_t)N},
        {L.t_off, b->t_off, 8 * (size_t)N}, {L.t_len, b->t_len, 4 * (size_t)N},
        {L.h0, b->h0, 4 * (size_t)N}, {L.w, b->w_override, b->w_override ? 4 * (size_t)N : 0}};
    for (const Cp &cp : meta)
        if (cp.bytes && (e = h2d(d + cp.off, cp.src, cp.bytes, st)) != cudaSuccess) return cuda_rc(e);
    const PairMeta M{(const int64_t *)(d + L.q_off), (const int32_t *)(d + L.q_len), (const int64_t *)(d + L.t_off),
                     (const int32_t *)(d + L.t_len), (const int32_t *)(d + L.h0),
                     b->w_override ? (const int32_t *)(d + L.w) : nullptr};
    Extents32 x;
    if (N <= kHostCheckMax) {
        Extents hx;
        if ((rc = check_host_batch(b, c->P, &hx)) != BSW_OK) return rc;
        x = Extents32{(unsigned long long)hx.q_lo, (unsigned long long)hx.t_lo, (unsigned long long)hx.q_hi,
                      (unsigned long long)hx.t_hi, hx.maxn, 0u};
    } else {
        Extents32 *X = reinterpret_cast<Extents32 *>(d + L.ext);
        if ((e = cudaMemsetAsync(X, 0xff, 16, st)) != cudaSuccess) return cuda_rc(e);             // q_lo, t_lo
        if ((e = cudaMemsetAsync(reinterpret_cast<uint8_t *>(X) + 16, 0, sizeof(Extents32) - 16, st)) != cudaSuccess)
            return cuda_rc(e);
        if ((e = launch_extents(M, N, c->P, X, st, c->sms)) != cudaSuccess) return cuda_rc(e);
        if ((e = cudaMemcpyAsync(c->h_ext, X, sizeof(Extents32), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return cuda_rc(e);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_rc(e);
        x = *c->h_ext;
        if (x.inval) return BSW_EINVAL;
    }
    int64_t q_lo = (int64_t)x.q_lo, q_hi = (int64_t)x.q_hi, t_lo = (int64_t)x.t_lo, t_hi = (int64_t)x.t_hi;
    if (x.q_lo > x.q_hi) q_lo = q_hi = 0;                 // no pair with both sides non-empty
    if (x.t_lo > x.t_hi) t_lo = t_hi = 0;
    const int64_t qnb = b->q_n ? nmask_bytes(q_lo, q_hi) : 0, tnb = b->t_n ? nmask_bytes(t_lo, t_hi) : 0;
    stage_seq_layout(L, q_hi - q_lo, t_hi - t_lo, qnb, tnb);
    if ((rc = lane.seq.reserve(L.seq_total, c->budget, &moved)) != BSW_OK) return rc;
    if ((rc = lane.ensure_work(N, std::max((int)x.maxn, kShortMax), c->sms, c->budget, &moved)) != BSW_OK) return rc;
    if (moved) clear_graphs(c);
    uint8_t *sq = lane.seq.p;
    const Cp seqs[] = {
        {L.q, b->q + q_lo, (size_t)(q_hi - q_lo)}, {L.t, b->t + t_lo, (size_t)(t_hi - t_lo)},
        {L.qn, b->q_n ? b->q_n + nmask_lo(q_lo) : nullptr, (size_t)qnb},
        {L.tn, b->t_n ? b->t_n + nmask_lo(t_lo) : nullptr, (size_t)tnb}};
    for (const Cp &cp : seqs)
        if (cp.bytes && (e = h2d(sq + cp.off, cp.src, cp.bytes, st)) != cudaSuccess) return cuda_rc(e);
    *out_B = Batch{N, sq + L.q - q_lo, M.q_off, M.q_len, sq + L.t - t_lo, M.t_off, M.t_len, M.h0, M.w,
                   (bsw_result_t *)(d + L.out), b->q_n ? sq + L.qn - nmask_lo(q_lo) : nullptr,
                   b->t_n ? sq + L.tn - nmask_lo(t_lo) : nullptr};
    *out_L = L;
    return BSW_OK;
}

int extend_host(bsw_ctx *c, const bsw_batch_t *b, bsw_result_t *out, int64_t *cells_out, cudaStream_t user)
{
    Batch B;
    StageLayout L;
    int rc = stage_host(c, b, user, &B, &L);
    if (rc != BSW_OK) return rc;
    const int64_t N = b->n_pairs;
    Lane &lane = c->sync;
    uint8_t *d = lane.io.p;
    cudaStream_t st = lane.S.main;
    cudaError_t e;
    Work W = make_work(lane.work.p, lane.wl);
    if ((e = enqueue_launch(c, lane, lane.S, B, W, b->flags, true, c->plan, timer_for(c, b->flags))) != cudaSuccess) {
        lane.work_dirty = true;
        return cuda_rc(e);
    }
    if ((e = cudaMemcpyAsync(out, d + L.out, sizeof(bsw_result_t) * (size_t)N, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_rc(e);
    if ((e = cudaMemcpyAsync(c->h_cells, W.cells, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_rc(e);
    if ((e = cudaMemcpyAsync(c->h_status, W.status, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_rc(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) { lane.work_dirty = true; return cuda_rc(e); }
    if (cells_out) *cells_out = (int64_t)*c->h_cells;
    return status_to_rc(*c->h_status);
}

int extend_device(bsw_ctx *c, const bsw_batch_t *b, bsw_result_t *out, int64_t *cells_out, cudaStream_t user)
{
    const int64_t N = b->n_pairs;
    Lane &lane = c->sync;
    bool moved = false;
    int rc = lane.ensure_work(N, kLongMax, c->sms, c->budget, &moved);
    if (rc != BSW_OK) return rc;
    if (moved) clear_graphs(c);
    cudaStream_t st = user ? user : lane.S.main;
    Batch B{N, b->q, b->q_off, b->q_len, b->t, b->t_off, b->t_len, b->h0, b->w_override, out, b->q_n, b->t_n};
    Work W = make_work(lane.work.p, lane.wl);
    if (cells_out) W.cells = (unsigned long long *)cells_out;
    cudaError_t e;
    if (b->flags & BSW_NO_GRAPH) {
        Streams S = lane.S;
        S.main = st;
        if ((e = enqueue_launch(c, lane, S, B, W, b->flags, false, c->plan, timer_for(c, b->flags))) != cudaSuccess) {
            lane.work_dirty = true;
            return cuda_rc(e);
        }
        return BSW_OK;
    }
    for (auto &g : c->graphs)
        if (same_batch(g.b, *b) && g.out == (void *)out && g.cells == (void *)cells_out) {
            c->last_launches = g.launches;
            return cuda_rc(cudaGraphLaunch(g.exec, st));
        }
    if (lane.work_dirty) {   // make the zeroing part of the stream order, not of the graph
        if ((e = cudaMemsetAsync(W.hist, 0, 4 * kNumBins, st)) != cudaSuccess) return cuda_rc(e);
        lane.work_dirty = false;
    }
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if ((e = cudaStreamBeginCapture(lane.S.main, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return cuda_rc(e);
    cudaError_t le = enqueue_launch(c, lane, lane.S, B, W, b->flags, false, c->plan);
    e = cudaStreamEndCapture(lane.S.main, &graph);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        lane.work_dirty = true;
        return cuda_rc(le != cudaSuccess ? le : e);
    }
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_rc(e);
    if ((int)c->graphs.size() >= kGraphCache) {
        cudaGraphExecDestroy(c->graphs.front().exec);
        c->graphs.erase(c->graphs.begin());
    }
    c->graphs.push_back({*b, (void *)out, (void *)cells_out, exec, c->last_launches});
    return cuda_rc(cudaGraphLaunch(exec, st));
}

// ------------------------------------------------------------ serving loop

// Stage the lane's requests into pinned memory, copy to the device, launch,
// copy results back.  Called by the server thread without the lock.
int serve_launch(bsw_ctx *c, int li)
{
    Lane &lane = c->serve_lane[li];
    std::vector<Request *> &reqs = c->lane_reqs[li];
    int64_t N = 0, qb = 0, tb = 0;
    int maxn = 0;
    bool has_n = false;
    for (Request *r : reqs) {
        r->out_pos = N;
        N += r->b.n_pairs;
        r->qpos = stage_start(qb, r->ext.q_lo);
        qb = r->qpos + (r->ext.q_hi - r->ext.q_lo);
        r->tpos = stage_start(tb, r->ext.t_lo);
        tb = r->tpos + (r->ext.t_hi - r->ext.t_lo);
        maxn = std::max(maxn, r->ext.maxn);
        has_n |= r->b.q_n != nullptr || r->b.t_n != nullptr;
    }
    IoLayout L = io_layout(N, qb, tb, has_n);
    int rc;
    if ((rc = lane.io.reserve(L.total, c->budget)) != BSW_OK) return rc;
    if ((rc = lane.ensure_work(N, std::max(maxn, kShortMax), c->sms, c->budget, nullptr)) != BSW_OK) return rc;
    if ((rc = lane.ensure_pinned(L.total)) != BSW_OK) return rc;
    uint8_t *h = lane.pinned;
    if (has_n) std::memset(h + L.qn, 0, L.q_off - L.qn);   // both bitmaps: requests without N stage none
    int64_t k0 = 0;
    for (Request *r : reqs) {
        const bsw_batch_t &b = r->b;
        const int64_t n = b.n_pairs;
        std::memcpy(h + L.q + r->qpos, b.q + r->ext.q_lo, (size_t)(r->ext.q_hi - r->ext.q_lo));
        std::memcpy(h + L.t + r->tpos, b.t + r->ext.t_lo, (size_t)(r->ext.t_hi - r->ext.t_lo));
        if (b.q_n)
            std::memcpy(h + L.qn + (r->qpos >> 1), b.q_n + (r->ext.q_lo >> 1),
                        (size_t)(((r->ext.q_hi + 1) >> 1) - (r->ext.q_lo >> 1)));
        if (b.t_n)
            std::memcpy(h + L.tn + (r->tpos >> 1), b.t_n + (r->ext.t_lo >> 1),
                        (size_t)(((r->ext.t_hi + 1) >> 1) - (r->ext.t_lo >> 1)));
        int64_t *qo = (int64_t *)(h + L.q_off) + k0, *to = (int64_t *)(h + L.t_off) + k0;
        const int64_t dq = 4 * (r->qpos - r->ext.q_lo), dt = 4 * (r->tpos - r->ext.t_lo);
        for (int64_t k = 0; k < n; ++k) {
            // pairs that are never read (empty sides) keep a valid offset of 0
            const bool used = b.q_len[k] > 0 && b.t_len[k] > 0;
            qo[k] = used ? b.q_off[k] + dq : 0;
            to[k] = used ? b.t_off[k] + dt : 0;
        }
        std::memcpy((int32_t *)(h + L.q_len) + k0, b.q_len, 4 * (size_t)n);
        std::memcpy((int32_t *)(h + L.t_len) + k0, b.t_len, 4 * (size_t)n);
        std::memcpy((int32_t *)(h + L.h0) + k0, b.h0, 4 * (size_t)n);
        int32_t *wv = (int32_t *)(h + L.w) + k0;
        if (b.w_override) std::memcpy(wv, b.w_override, 4 * (size_t)n);
        else for (int64_t k = 0; k < n; ++k) wv[k] = c->P.w;
        k0 += n;
    }
    cudaStream_t st = lane.S.main;
    uint8_t *d = lane.io.p;
    cudaError_t e;
    if ((e = cudaEventRecord(lane.t_start, st)) != cudaSuccess) return cuda_rc(e);
    if ((e = h2d(d, h, L.in_end, st)) != cudaSuccess) return cuda_rc(e);
    Batch B{N, d + L.q, (const int64_t *)(d + L.q_off), (const int32_t *)(d + L.q_len), d + L.t,
            (const int64_t *)(d + L.t_off), (const int32_t *)(d + L.t_len), (const int32_t *)(d + L.h0),
            (const int32_t *)(d + L.w), (bsw_result_t *)(d + L.out), has_n ? d + L.qn : nullptr,
            has_n ? d + L.tn : nullptr};
    Work W = make_work(lane.work.p, lane.wl);
    if ((e = enqueue_launch(c, lane, lane.S, B, W, 0u, true, c->plan)) != cudaSuccess) {
        lane.work_dirty = true;
        return cuda_rc(e);
    }
    if ((e = cudaMemcpyAsync(h + L.out, d + L.out, sizeof(bsw_result_t) * (size_t)N, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_rc(e);
    if ((e = cudaMemcpyAsync(h + L.status, W.status, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess) return cuda_rc(e);
    if ((e = cudaEventRecord(lane.t_end, st)) != cudaSuccess) return cuda_rc(e);
    if ((e = cudaEventRecord(lane.done, st)) != cudaSuccess) return cuda_rc(e);
    c->lane_io[li] = L;
    c->lane_pairs[li] = N;
    c->lane_has_n[li] = has_n;
    return BSW_OK;
}

// Called with the lock held.  launched: the lane's work reached the device
// (its events are recorded), so its interval is kept.
void finish_lane(bsw_ctx *c, int li, int rc, bool launched)
{
    Lane &lane = c->serve_lane[li];
    const IoLayout &L = c->lane_io[li];
    if (rc == BSW_OK) rc = status_to_rc(*(uint32_t *)(lane.pinned + L.status));
    ServeStats &S = c->stats;
    for (Request *r : c->lane_reqs[li]) {
        if (rc == BSW_OK)
            std::memcpy(r->out, lane.pinned + L.out + sizeof(bsw_result_t) * (size_t)r->out_pos,
                        sizeof(bsw_result_t) * (size_t)r->b.n_pairs);
        r->status = rc;
    }
    S.requests += (int64_t)c->lane_reqs[li].size();
    if (c->lane_reqs[li].size() > 1) S.merged += (int64_t)c->lane_reqs[li].size();
    if (launched) {
        ++S.launches;
        float a = 0.0f, b = 0.0f;
        if (c->ref_ok && cudaEventElapsedTime(&a, c->ref_ev, lane.t_start) == cudaSuccess &&
            cudaEventElapsedTime(&b, c->ref_ev, lane.t_end) == cudaSuccess) {
            try {
                if (S.iv.size() >= kStatsIntervals) S.iv.erase(S.iv.begin(), S.iv.begin() + kStatsIntervals / 2);
                S.iv.emplace_back(a, b);
            } catch (...) {
            }
        } else {
            cudaGetLastError();
        }
    }
    c->lane_reqs[li].clear();
    c->lane_busy[li] = false;
    c->mem_wait = false;   // memory may be free now
}

void server_main(bsw_ctx *c)
{
    cudaSetDevice(c->device);
    std::unique_lock<std::mutex> lk(c->mu);
    if (cudaEventCreate(&c->ref_ev) == cudaSuccess && cudaEventRecord(c->ref_ev, c->sync.S.main) == cudaSuccess &&
        cudaEventSynchronize(c->ref_ev) == cudaSuccess)
        c->ref_ok = true;
    else
        cudaGetLastError();
    for (;;) {
        bool progressed = false;
        // completions
        for (int li = 0; li < kServeLanes; ++li) {
            if (!c->lane_busy[li]) continue;
            cudaError_t q = cudaEventQuery(c->serve_lane[li].done);
            if (q == cudaErrorNotReady) continue;
            finish_lane(c, li, q == cudaSuccess ? BSW_OK : cuda_rc(q), true);
            progressed = true;
        }
        if (progressed) c->cv_done.notify_all();
        // admissions: continuous batching into free lanes (none while an
        // admission waits for memory that busy lanes hold)
        bool any_busy = false;
        for (int li = 0; li < kServeLanes; ++li) any_busy |= c->lane_busy[li];
        if (!any_busy) c->mem_wait = false;
        for (int li = 0; li < kServeLanes && !c->queue.empty() && !c->mem_wait; ++li) {
            if (c->lane_busy[li]) continue;
            if (!c->lane_created[li]) {
                if (c->serve_lane[li].create() != BSW_OK) continue;
                c->lane_created[li] = true;
            }
            std::vector<Request *> &reqs = c->lane_reqs[li];
            int64_t pairs = 0, ecells = 0, qb = 0, tb = 0;
            int maxn = 0;
            bool has_n = false;
            // Whether the merged launch, with request r added, fits the budget
            // on its own (every request alone does: bsw_stream_submit checks).
            auto fits = [&](const Request *r) {
                const bool n2 = has_n || r->b.q_n || r->b.t_n;
                const IoLayout L = io_layout(pairs + r->b.n_pairs, qb + (r->ext.q_hi - r->ext.q_lo) + 2,
                                             tb + (r->ext.t_hi - r->ext.t_lo) + 2, n2);
                const WorkLayout W = work_layout(pairs + r->b.n_pairs,
                                                 slot_bytes_for(std::max(std::max(maxn, r->ext.maxn), kShortMax)),
                                                 warp_slots_needed(c->sms));
                return (int64_t)(L.total + W.total) <= c->budget.cap;
            };
            try {                        // a request moves to the lane only once the lane's list holds it
                while (!c->queue.empty() &&
                       (reqs.empty() || (pairs + c->queue.front()->b.n_pairs <= kMergePairs &&
                                         ecells + c->queue.front()->ext.est_cells <= kMergeCells &&
                                         fits(c->queue.front())))) {
                    if (fault_hit(BSW_FAULT_HOST)) throw std::bad_alloc();
                    const Request *r = c->queue.front();
                    reqs.push_back(c->queue.front());
                    pairs += r->b.n_pairs;
                    ecells += r->ext.est_cells;
                    qb += r->ext.q_hi - r->ext.q_lo + 2;
                    tb += r->ext.t_hi - r->ext.t_lo + 2;
                    maxn = std::max(maxn, r->ext.maxn);
                    has_n |= r->b.q_n || r->b.t_n;
                    c->queue.pop_front();
                }
            } catch (...) {
            }
            if (reqs.empty()) break;     // no memory for the list: try again on the next wake-up
            c->lane_busy[li] = true;
            lk.unlock();
            int rc = serve_launch(c, li);
            lk.lock();
            if (rc == BSW_EBUDGET) {
                bool others = false;
                for (int k = 0; k < kServeLanes; ++k) others |= (k != li && c->lane_busy[k]);
                bool requeued = false;
                if (others) {   // wait for memory held by other lanes
                    try {           // an insert at the front either takes them all or changes nothing
                        c->queue.insert(c->queue.begin(), reqs.begin(), reqs.end());
                        requeued = true;
                    } catch (...) {
                    }
                }
                if (requeued) {
                    reqs.clear();
                    c->lane_busy[li] = false;
                    c->serve_lane[li].io.release(c->budget);
                    c->mem_wait = true;
                    ++c->stats.budget_waits;
                    break;
                }
            }
            if (rc != BSW_OK) {
                finish_lane(c, li, rc, false);
                c->cv_done.notify_all();
            }
            progressed = true;
        }
        bool busy = false;
        for (int li = 0; li < kServeLanes; ++li) busy |= c->lane_busy[li];
        if (c->stop && !busy && c->queue.empty()) break;
        if (!progressed) {
            if (busy) c->cv_work.wait_for(lk, std::chrono::microseconds(50));
            else c->cv_work.wait_for(lk, std::chrono::milliseconds(20));
        }
    }
}

// True when no submitted batch is queued or on the device.
bool serving_idle(bsw_ctx *c)
{
    std::lock_guard<std::mutex> lk(c->mu);
    if (!c->queue.empty()) return false;
    for (int li = 0; li < kServeLanes; ++li)
        if (c->lane_busy[li]) return false;
    return true;
}

}  // namespace

// ------------------------------------------------------------------- C ABI

// No C++ exception crosses the C ABI: the entry points that use the C++
// library's containers or threads run their bodies through guard, which turns
// a failed allocation (or any other exception) into BSW_ENOMEM.
template <class F>
int guard(F &&f)
{
    try {
        return f();
    } catch (...) {
        return BSW_ENOMEM;
    }
}

extern "C" {

const char *bsw_version(void) { return "bsw-gb300 1.0 (sm_103a)"; }

const char *bsw_strerror(int code)
{
    switch (code) {
    case BSW_OK: return "ok";
    case BSW_PENDING: return "pending";
    case BSW_EINVAL: return "invalid argument or input value";
    case BSW_ENOMEM: return "out of memory";
    case BSW_EBUDGET: return "batch exceeds the device-memory budget";
    case BSW_ECUDA: return "CUDA error";
    case BSW_ETIMEOUT: return "timed out";
    case BSW_ENOTFOUND: return "unknown ticket";
    case BSW_ESTATE: return "context cannot accept the call";
    default: return "unknown error code";
    }
}

int bsw_pack_2bit(const uint8_t *in, int64_t n, uint8_t *out)
{
    if (n < 0 || (n > 0 && (!in || !out))) return BSW_EINVAL;
    for (int64_t k = 0; k < (n + 3) / 4; ++k) out[k] = 0;
    for (int64_t k = 0; k < n; ++k) {
        int v;
        switch (in[k]) {
        case 0: case 'A': case 'a': v = 0; break;
        case 1: case 'C': case 'c': v = 1; break;
        case 2: case 'G': case 'g': v = 2; break;
        case 3: case 'T': case 't': v = 3; break;
        default: return BSW_EINVAL;
        }
        out[k >> 2] |= (uint8_t)(v << (2 * (k & 3)));
    }
    return BSW_OK;
}

int bsw_pack_2bit_n(const uint8_t *in, int64_t n, uint8_t *out, uint8_t *out_n)
{
    if (n < 0 || (n > 0 && (!in || !out || !out_n))) return BSW_EINVAL;
    for (int64_t k = 0; k < (n + 3) / 4; ++k) out[k] = 0;
    for (int64_t k = 0; k < (n + 7) / 8; ++k) out_n[k] = 0;
    for (int64_t k = 0; k < n; ++k) {
        int v;
        switch (in[k]) {
        case 0: case 'A': case 'a': v = 0; break;
        case 1: case 'C': case 'c': v = 1; break;
        case 2: case 'G': case 'g': v = 2; break;
        case 3: case 'T': case 't': v = 3; break;
        case 4: case 'N': case 'n': v = 0; out_n[k >> 3] |= (uint8_t)(1u << (k & 7)); break;
        default: return BSW_EINVAL;
        }
        out[k >> 2] |= (uint8_t)(v << (2 * (k & 3)));
    }
    return BSW_OK;
}

int32_t bsw_band_width(const bsw_ctx_t *ctx, int32_t qlen, int32_t w)
{
    if (!ctx || qlen < 0 || w < 0) return -1;
    const Params &P = ctx->P;
    auto cap = [&](int o, int e) {
        long long x = (long long)qlen * P.a + P.end_bonus - o + e;
        long long k = x / e;
        return (int32_t)(k > 1 ? k : 1);
    };
    return std::min(w, std::min(cap(P.o_ins, P.e_ins), cap(P.o_del, P.e_del)));
}

int bsw_partition(const bsw_scoring_t *sc, int32_t w, int32_t end_bonus, const int32_t *q_len, const int32_t *t_len,
                  const int32_t *w_override, int64_t n_pairs, int32_t parts, int64_t *bounds)
{
    if (!sc || !bounds || parts < 1 || n_pairs < 0 || w < 0 || end_bonus < 0) return BSW_EINVAL;
    if (n_pairs > 0 && (!q_len || !t_len)) return BSW_EINVAL;
    if (sc->match <= 0 || sc->e_del <= 0 || sc->e_ins <= 0 || sc->o_del < 0 || sc->o_ins < 0) return BSW_EINVAL;
    auto cap = [&](int32_t n, int o, int e) {
        const long long x = (long long)n * sc->match + end_bonus - o + e;
        const long long k = x / e;
        return k > 1 ? k : 1ll;
    };
    // two passes (the total, then the boundaries) and no per-pair storage
    long double total = 0.0L;
    for (int64_t p = 0; p < n_pairs; ++p) {
        const int32_t n = q_len[p], m = t_len[p], wp = w_override ? w_override[p] : w;
        if (n < 0 || m < 0 || wp < 0) return BSW_EINVAL;
        const long long wb = std::min<long long>(wp, std::min(cap(n, sc->o_ins, sc->e_ins), cap(n, sc->o_del, sc->e_del)));
        total += (long double)n * (long double)std::min<long long>(m, 2 * wb + 1);
    }
    bounds[0] = 0;
    long double run = 0.0L;
    int k = 1;
    for (int64_t p = 0; p < n_pairs && k < parts; ++p) {
        const int32_t n = q_len[p], m = t_len[p], wp = w_override ? w_override[p] : w;
        const long long wb = std::min<long long>(wp, std::min(cap(n, sc->o_ins, sc->e_ins), cap(n, sc->o_del, sc->e_del)));
        run += (long double)n * (long double)std::min<long long>(m, 2 * wb + 1);
        while (k < parts && run * parts >= total * k) bounds[k++] = p + 1;
    }
    while (k <= parts) bounds[k++] = n_pairs;
    return BSW_OK;
}

int bsw_init(const bsw_scoring_t *sc, int32_t w, int32_t zdrop, int32_t end_bonus, int64_t mem_budget_bytes,
             bsw_ctx_t **out)
{
    if (!sc || !out || w < 0 || end_bonus < 0 || mem_budget_bytes <= 0) return BSW_EINVAL;
    if (sc->match <= 0 || sc->match > 127 || sc->mismatch <= 0 || sc->mismatch > 128 || sc->o_del < 0 ||
        sc->o_ins < 0 || sc->e_del <= 0 || sc->e_ins <= 0 || sc->o_del > (1 << 20) || sc->o_ins > (1 << 20) ||
        sc->e_del > (1 << 20) || sc->e_ins > (1 << 20) || end_bonus > (1 << 20))
        return BSW_EINVAL;
    *out = nullptr;
    bsw_ctx *c = new (std::nothrow) bsw_ctx();
    if (!c) return BSW_ENOMEM;
    c->P = Params{sc->match, sc->mismatch, sc->o_del, sc->e_del, sc->o_ins, sc->e_ins, w, zdrop, end_bonus, 0u, kLongMax,
                  1u << 8, 1u << 16, 1u << 24, kShortMax};
    c->budget.cap = mem_budget_bytes;
    int rc = BSW_OK;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        rc = BSW_ECUDA;
    }
    if (rc == BSW_OK) rc = c->sync.create();
    if (rc == BSW_OK && prepare_kernels(c->sms) != cudaSuccess) rc = BSW_ECUDA;
    if (rc == BSW_OK && (cudaMallocHost(&c->h_status, 4) != cudaSuccess ||
                         cudaMallocHost(&c->h_cells, 8) != cudaSuccess ||
                         cudaMallocHost(&c->h_ext, sizeof(Extents32)) != cudaSuccess ||
                         cudaMallocHost(&c->h_chk, sizeof(DriverCheck)) != cudaSuccess))
        rc = BSW_ENOMEM;
    if (rc == BSW_OK && (cudaEventCreate(&c->tune_ev[0]) != cudaSuccess || cudaEventCreate(&c->tune_ev[1]) != cudaSuccess))
        rc = BSW_ECUDA;
    if (rc != BSW_OK) {
        cudaGetLastError();
        bsw_destroy(c);
        return rc;
    }
    *out = c;
    return BSW_OK;
}

int bsw_extend_batch(bsw_ctx_t *ctx, const bsw_batch_t *b, bsw_result_t *out, int64_t *cells_out, void *stream)
{
    return guard([&]() -> int {
        if (!ctx || !b) return BSW_EINVAL;
        if (b->n_pairs < 0 || b->n_pairs > INT32_MAX || (b->flags & ~kKnownFlags)) return BSW_EINVAL;
        const uint32_t forced = b->flags & (BSW_FORCE_I8 | BSW_FORCE_I16 | BSW_FORCE_I32);
        if (forced & (forced - 1)) return BSW_EINVAL;
        const bool dev = (b->flags & BSW_DEVICE_PTRS) != 0;
        // events inside a captured graph would not time this call's kernels
        if (dev && (b->flags & BSW_TIME_KERNELS) && !(b->flags & BSW_NO_GRAPH)) return BSW_EINVAL;
        if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_rc(cudaErrorInvalidDevice);
        if (b->n_pairs == 0) {
            if (cells_out) {
                if (dev) return cuda_rc(cudaMemsetAsync(cells_out, 0, 8, (cudaStream_t)stream));
                *cells_out = 0;
            }
            return BSW_OK;
        }
        if (!b->q || !b->q_off || !b->q_len || !b->t || !b->t_off || !b->t_len || !b->h0 || !out) return BSW_EINVAL;
        if (dev) return extend_device(ctx, b, out, cells_out, (cudaStream_t)stream);
        return extend_host(ctx, b, out, cells_out, (cudaStream_t)stream);
    });
}

int bsw_sync(bsw_ctx_t *ctx, void *stream)
{
    if (!ctx) return BSW_EINVAL;
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->sync.S.main;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_rc(e);
    if (!ctx->sync.work.p) return BSW_OK;
    Work W = make_work(ctx->sync.work.p, ctx->sync.wl);
    if ((e = cudaMemcpy(ctx->h_status, W.status, 4, cudaMemcpyDeviceToHost)) != cudaSuccess) return cuda_rc(e);
    if ((e = cudaMemset(W.status, 0, 4)) != cudaSuccess) return cuda_rc(e);
    return status_to_rc(*ctx->h_status);
}

int bsw_stream_submit(bsw_ctx_t *ctx, const bsw_batch_t *b, bsw_result_t *out, uint64_t *ticket)
{
    return guard([&]() -> int {
        if (!ctx || !b || !ticket) return BSW_EINVAL;
        if (b->n_pairs < 0 || b->n_pairs > INT32_MAX || (b->flags & ~kKnownFlags)) return BSW_EINVAL;
        if (b->flags & (BSW_DEVICE_PTRS | BSW_PLAIN_KERNEL | BSW_PLAIN_GLOBAL | BSW_FORCE_I8 | BSW_FORCE_I16 |
                        BSW_FORCE_I32 | BSW_TIME_KERNELS))
            return BSW_EINVAL;   // the serving loop runs the context's batched plan on host inputs
        if (b->n_pairs > 0 && (!b->q || !b->q_off || !b->q_len || !b->t || !b->t_off || !b->t_len || !b->h0 || !out))
            return BSW_EINVAL;
        std::unique_ptr<Request> holder(new (std::nothrow) Request());
        Request *r = holder.get();
        if (!r) return BSW_ENOMEM;
        r->b = *b;
        r->out = out;
        int rc = check_host_batch(b, ctx->P, &r->ext);
        if (rc == BSW_OK) {
            const int64_t N = b->n_pairs;
            IoLayout L = io_layout(N, r->ext.q_hi - r->ext.q_lo + 2, r->ext.t_hi - r->ext.t_lo + 2,
                                   b->q_n != nullptr || b->t_n != nullptr);
            WorkLayout W = work_layout(N, slot_bytes_for(std::max(r->ext.maxn, kShortMax)), warp_slots_needed(ctx->sms));
            if ((int64_t)(L.total + W.total) > ctx->budget.cap) rc = BSW_EBUDGET;
        }
        if (rc == BSW_OK && (b->flags & BSW_COPY_INPUTS) && b->n_pairs > 0) {
            const int64_t N = b->n_pairs;
            const size_t qb = (size_t)(r->ext.q_hi - r->ext.q_lo), tb = (size_t)(r->ext.t_hi - r->ext.t_lo);
            const size_t qnb = b->q_n ? (size_t)(((r->ext.q_hi + 1) >> 1) - (r->ext.q_lo >> 1)) : 0;
            const size_t tnb = b->t_n ? (size_t)(((r->ext.t_hi + 1) >> 1) - (r->ext.t_lo >> 1)) : 0;
            const size_t total = qb + tb + qnb + tnb + 8 * (size_t)N * 2 + 4 * (size_t)N * (b->w_override ? 4 : 3);
            try {
                r->own.resize(total);
            } catch (...) {
                rc = BSW_ENOMEM;
            }
            if (rc == BSW_OK) {
                uint8_t *p = r->own.data();
                std::memcpy(p, b->q + r->ext.q_lo, qb);
                r->b.q = p - r->ext.q_lo;   // keep the caller's offsets valid
                p += qb;
                std::memcpy(p, b->t + r->ext.t_lo, tb);
                r->b.t = p - r->ext.t_lo;
                p += tb;
                if (qnb) {                  // the N bitmaps' bytes of the copied bases, offsets kept valid too
                    std::memcpy(p, b->q_n + (r->ext.q_lo >> 1), qnb);
                    r->b.q_n = p - (r->ext.q_lo >> 1);
                    p += qnb;
                }
                if (tnb) {
                    std::memcpy(p, b->t_n + (r->ext.t_lo >> 1), tnb);
                    r->b.t_n = p - (r->ext.t_lo >> 1);
                    p += tnb;
                }
                auto dup = [&](const void *src, size_t bytes) { std::memcpy(p, src, bytes); void *d = p; p += bytes; return d; };
                r->b.q_off = (const int64_t *)dup(b->q_off, 8 * (size_t)N);
                r->b.t_off = (const int64_t *)dup(b->t_off, 8 * (size_t)N);
                r->b.q_len = (const int32_t *)dup(b->q_len, 4 * (size_t)N);
                r->b.t_len = (const int32_t *)dup(b->t_len, 4 * (size_t)N);
                r->b.h0 = (const int32_t *)dup(b->h0, 4 * (size_t)N);
                if (b->w_override) r->b.w_override = (const int32_t *)dup(b->w_override, 4 * (size_t)N);
            }
        }
        if (rc != BSW_OK) return rc;
        // Commit under the lock, all or nothing: the server thread is started
        // first, then the ticket and the queue entry go in; if any step
        // throws, what was added is taken out again and no ticket is issued,
        // so the server never sees (or writes the out of) a failed request.
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (ctx->stop) return BSW_ESTATE;
        if (b->n_pairs > 0 && !ctx->server_started) {
            try {
                if (fault_hit(BSW_FAULT_THREAD))
                    throw std::system_error(std::make_error_code(std::errc::resource_unavailable_try_again));
                ctx->server = std::thread(server_main, ctx);
            } catch (...) {
                return BSW_ENOMEM;
            }
            ctx->server_started = true;
        }
        const uint64_t t = ctx->next_ticket;
        r->ticket = t;
        if (b->n_pairs == 0) r->status = BSW_OK;
        try {
            if (fault_hit(BSW_FAULT_HOST)) throw std::bad_alloc();
            ctx->tickets.emplace(t, r);
        } catch (...) {
            return BSW_ENOMEM;
        }
        if (b->n_pairs > 0) {
            try {
                if (fault_hit(BSW_FAULT_HOST)) throw std::bad_alloc();
                ctx->queue.push_back(r);
            } catch (...) {
                ctx->tickets.erase(t);
                return BSW_ENOMEM;
            }
        }
        holder.release();
        ctx->next_ticket = t + 1;
        *ticket = t;
        if (b->n_pairs > 0) ctx->cv_work.notify_one();
        return BSW_OK;
    });
}

int bsw_stream_stats(bsw_ctx_t *ctx, bsw_serve_stats_t *out, int32_t reset)
{
    if (!ctx || !out) return BSW_EINVAL;
    return guard([&]() -> int {
        std::vector<std::pair<float, float>> iv;
        {
            std::lock_guard<std::mutex> lk(ctx->mu);
            const ServeStats &S = ctx->stats;
            out->requests = S.requests;
            out->launches = S.launches;
            out->merged = S.merged;
            out->budget_waits = S.budget_waits;
            iv = S.iv;
            if (reset) ctx->stats = ServeStats();
        }
        // busy: the sum of the launches' intervals; union: the time at least
        // one launch was on the device; the most launches at one moment
        std::sort(iv.begin(), iv.end());
        double busy = 0.0, uni = 0.0, end = -1e30;
        for (const auto &x : iv) {
            busy += x.second - x.first;
            if (x.first > end) { uni += x.second - x.first; end = x.second; }
            else if (x.second > end) { uni += x.second - end; end = x.second; }
        }
        std::vector<std::pair<float, int>> ev;
        ev.reserve(2 * iv.size());
        for (const auto &x : iv) { ev.emplace_back(x.first, 1); ev.emplace_back(x.second, -1); }
        std::sort(ev.begin(), ev.end(), [](const std::pair<float, int> &a, const std::pair<float, int> &b) {
            return a.first < b.first || (a.first == b.first && a.second < b.second);
        });
        int cur = 0, mx = 0;
        for (const auto &e : ev) { cur += e.second; mx = std::max(mx, cur); }
        out->busy_ms = busy;
        out->union_ms = uni;
        out->max_concurrent = mx;
        return BSW_OK;
    });
}

int bsw_fault_inject(const char *spec)
{
    uint32_t sites;
    int32_t skip, count;
    if (!parse_faults(spec, &sites, &skip, &count)) return BSW_EINVAL;
    set_faults(sites, skip, count);
    return BSW_OK;
}

int bsw_stream_poll(bsw_ctx_t *ctx, uint64_t ticket, int32_t timeout_us)
{
    if (!ctx) return BSW_EINVAL;
    std::unique_lock<std::mutex> lk(ctx->mu);
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return BSW_ENOTFOUND;
    Request *r = it->second;
    auto ready = [&] { return r->status != BSW_PENDING; };
    if (!ready()) {
        if (timeout_us < 0) ctx->cv_done.wait(lk, ready);
        else if (timeout_us > 0) ctx->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    }
    if (!ready()) return BSW_PENDING;
    const int rc = r->status;
    ctx->tickets.erase(ticket);
    delete r;
    return rc;
}

int bsw_get_plan(const bsw_ctx_t *ctx, bsw_plan_t *plan)
{
    if (!ctx || !plan) return BSW_EINVAL;
    *plan = ctx->pub_plan;
    return BSW_OK;
}

int bsw_set_plan(bsw_ctx_t *ctx, const bsw_plan_t *plan)
{
    if (!ctx || !plan) return BSW_EINVAL;
    if (plan->packed != 0 && plan->packed != 1) return BSW_EINVAL;
    if (plan->warp_x2 != 0 && plan->warp_x2 != 1) return BSW_EINVAL;
    Plan L;
    if (!make_plan(plan->short_max, plan->u8_bounds, plan->i16_bounds, plan->packed != 0, plan->warp_cols,
                   plan->inter_warps, plan->cta_min, plan->warp_x2 != 0, &L))
        return BSW_EINVAL;
    if (!serving_idle(ctx)) return BSW_ESTATE;
    ctx->plan = L;
    ctx->pub_plan = *plan;
    ctx->pub_plan.u8_bounds |= 1u;
    ctx->pub_plan.i16_bounds |= 1u;
    ctx->pub_plan.ms = 0.0f;
    clear_graphs(ctx);   // captured graphs hold the old plan's launches
    return BSW_OK;
}

int bsw_autotune(bsw_ctx_t *ctx, const bsw_batch_t *b, int64_t sample_pairs, int32_t reps, bsw_plan_t *chosen)
{
    return guard([&]() -> int {
        if (!ctx || !b) return BSW_EINVAL;
        if (b->n_pairs < 0 || b->n_pairs > INT32_MAX || (b->flags & ~BSW_DEVICE_PTRS)) return BSW_EINVAL;
        if (!serving_idle(ctx)) return BSW_ESTATE;
        if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_rc(cudaErrorInvalidDevice);
        const int64_t ns = std::min<int64_t>(b->n_pairs, sample_pairs > 0 ? sample_pairs : kTuneSample);
        if (reps <= 0) reps = 3;
        if (ns == 0) {
            if (chosen) *chosen = ctx->pub_plan;
            return BSW_OK;
        }
        if (!b->q || !b->q_off || !b->q_len || !b->t || !b->t_off || !b->t_len || !b->h0) return BSW_EINVAL;
        bsw_batch_t sb = *b;
        sb.n_pairs = ns;
        Lane &lane = ctx->sync;
        Batch B;
        int rc;
        if (b->flags & BSW_DEVICE_PTRS) {
            bool moved = false;
            if ((rc = lane.ensure_work(ns, kLongMax, ctx->sms, ctx->budget, &moved)) != BSW_OK) return rc;
            if (moved) clear_graphs(ctx);
            if ((rc = lane.io.reserve(sizeof(bsw_result_t) * (size_t)ns, ctx->budget)) != BSW_OK) return rc;
            B = Batch{ns, sb.q, sb.q_off, sb.q_len, sb.t, sb.t_off, sb.t_len, sb.h0, sb.w_override,
                      (bsw_result_t *)lane.io.p, sb.q_n, sb.t_n};
        } else {
            StageLayout L;
            if ((rc = stage_host(ctx, &sb, nullptr, &B, &L)) != BSW_OK) return rc;
        }
        const Work W = make_work(lane.work.p, lane.wl);
        const bool can_pack = packed_scoring_ok(ctx->P);

        // One candidate: a warm-up launch, then the fastest of reps, timed with
        // events on the lane's stream (the batched path joins its side streams
        // back into it).  counts receives the pairs each class held.
        auto time_plan = [&](const bsw_plan_t &k, float *ms, int32_t *counts) -> int {
            Plan L;
            if (!make_plan(k.short_max, k.u8_bounds, k.i16_bounds, k.packed != 0, k.warp_cols, k.inter_warps,
                           k.cta_min, k.warp_x2 != 0, &L))
                return BSW_EINVAL;
            float best = 0.0f;
            for (int r = 0; r <= reps; ++r) {
                cudaError_t e;
                if ((e = cudaEventRecord(ctx->tune_ev[0], lane.S.main)) != cudaSuccess) return cuda_rc(e);
                if ((e = enqueue_launch(ctx, lane, lane.S, B, W, 0u, true, L)) != cudaSuccess) {
                    lane.work_dirty = true;
                    return cuda_rc(e);
                }
                if ((e = cudaEventRecord(ctx->tune_ev[1], lane.S.main)) != cudaSuccess) return cuda_rc(e);
                if ((e = cudaEventSynchronize(ctx->tune_ev[1])) != cudaSuccess) {
                    lane.work_dirty = true;
                    return cuda_rc(e);
                }
                float t = 0.0f;
                if ((e = cudaEventElapsedTime(&t, ctx->tune_ev[0], ctx->tune_ev[1])) != cudaSuccess) return cuda_rc(e);
                if (r == 1 || (r > 1 && t < best)) best = t;
            }
            cudaError_t e = cudaMemcpy(ctx->h_status, W.status, 4, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_rc(e);
            if (*ctx->h_status) return BSW_EINVAL;
            if ((e = cudaMemcpy(counts, W.cls_count, 4 * (kNumClass + 1), cudaMemcpyDeviceToHost)) != cudaSuccess)
                return cuda_rc(e);
            *ms = best;
            return BSW_OK;
        };

        // Coordinate descent.  Knobs that only affect classes the sample leaves
        // empty are not timed (their differences would be noise), and the
        // boundary of a class the sample leaves empty is removed outright (one
        // launch fewer, the same work).
        bsw_plan_t best{kShortMax, 0xffu, 0xfu, 0, 8, 2, 0, 0, 0.0f};
        float tbest = 0.0f;
        int32_t cnt[kNumClass + 1], cnt_best[kNumClass + 1];
        if ((rc = time_plan(best, &tbest, cnt_best)) != BSW_OK) return rc;
        auto consider = [&](const bsw_plan_t &k) -> int {
            float t = 0.0f;
            const int r = time_plan(k, &t, cnt);
            if (r == BSW_OK && t < 0.99f * tbest) {
                best = k;
                tbest = t;
                std::memcpy(cnt_best, cnt, sizeof(cnt));
            }
            return r;
        };
        for (int sm : {192, 128, 96, 64}) {
            bsw_plan_t k = best;
            k.short_max = sm;
            if ((rc = consider(k)) != BSW_OK) return rc;
        }
        auto any = [&](int c0, int c1) {   // classes [c0, c1) hold pairs under the best plan
            for (int c = c0; c < c1; ++c)
                if (cnt_best[c] > 0) return true;
            return false;
        };
        if (any(kClsCTA, kClsW16 + 1)) {
            if (x2_usable(ctx->P)) {
                bsw_plan_t k = best;
                k.warp_x2 = 1;
                if ((rc = consider(k)) != BSW_OK) return rc;
            }
            for (int cols : {4, 16}) {
                if (best.warp_x2) break;
                bsw_plan_t k = best;
                k.warp_cols = cols;
                if ((rc = consider(k)) != BSW_OK) return rc;
            }
            for (int cm : {8192, 4096, 2048, 1024, 512}) {
                bsw_plan_t k = best;
                k.cta_min = cm;
                if ((rc = consider(k)) != BSW_OK) return rc;
            }
        }
        if (can_pack && any(4, 8)) {       // the 8-bit classes of bound 128 and below
            bsw_plan_t k = best;
            k.packed = 1;
            if ((rc = consider(k)) != BSW_OK) return rc;
        }
        if (any(0, kClsW16))
            for (int wp : {1, 4}) {
                bsw_plan_t k = best;
                k.inter_warps = wp;
                if ((rc = consider(k)) != BSW_OK) return rc;
            }
        // Class boundaries: removing boundary c moves class c's pairs into the
        // next larger kept class.
        for (int bit = 1; bit < 8; ++bit) {
            if (!((best.u8_bounds >> bit) & 1u)) continue;
            bsw_plan_t k = best;
            k.u8_bounds &= ~(1u << bit);
            if (cnt_best[bit] == 0) {
                best = k;
                continue;
            }
            if ((rc = consider(k)) != BSW_OK) return rc;
        }
        for (int bit = 1; bit < 4; ++bit) {
            if (!((best.i16_bounds >> bit) & 1u)) continue;
            bsw_plan_t k = best;
            k.i16_bounds &= ~(1u << bit);
            if (cnt_best[8 + bit] == 0) {
                best = k;
                continue;
            }
            if ((rc = consider(k)) != BSW_OK) return rc;
        }
        if ((rc = time_plan(best, &tbest, cnt)) != BSW_OK) return rc;
        make_plan(best.short_max, best.u8_bounds, best.i16_bounds, best.packed != 0, best.warp_cols, best.inter_warps,
                  best.cta_min, best.warp_x2 != 0, &ctx->plan);
        best.ms = tbest;
        ctx->pub_plan = best;
        clear_graphs(ctx);
        if (chosen) *chosen = best;
        return BSW_OK;
    });
}

int bsw_kernel_times(bsw_ctx_t *ctx, bsw_timing_t *out)
{
    if (!ctx || !out) return BSW_EINVAL;
    if (!ctx->timer_valid) return BSW_ESTATE;
    out->launches = ctx->last_launches;
    for (int k = 0; k <= kNumClass; ++k) {
        out->class_ms[k] = 0.0f;
        if (!ctx->timer.used[k]) continue;
        cudaError_t e = cudaEventSynchronize(ctx->timer.t1[k]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&out->class_ms[k], ctx->timer.t0[k], ctx->timer.t1[k]);
        if (e != cudaSuccess) return cuda_rc(e);
    }
    return BSW_OK;
}

int bsw_set_reference_n(bsw_ctx_t *ctx, const uint8_t *ref, const uint8_t *ref_n, int64_t ref_len)
{
    if (!ctx || ref_len < 0 || (ref_len > 0 && !ref)) return BSW_EINVAL;
    if (!serving_idle(ctx)) return BSW_ESTATE;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_rc(cudaErrorInvalidDevice);
    const size_t bytes = (size_t)((ref_len + 3) / 4), nbytes = ref_n ? (size_t)((ref_len + 7) / 8) : 0;
    const size_t n_at = align_up(bytes, 256);                 // the bitmap after the packed bases
    ctx->ref_len = -1;
    ctx->ref_has_n = false;
    int rc = ctx->refbuf.reserve(std::max<size_t>(n_at + nbytes, 1), ctx->budget);
    if (rc != BSW_OK) return rc;
    cudaError_t e;
    if (bytes && (e = cudaMemcpy(ctx->refbuf.p, ref, bytes, cudaMemcpyHostToDevice)) != cudaSuccess) return cuda_rc(e);
    if (nbytes && (e = cudaMemcpy(ctx->refbuf.p + n_at, ref_n, nbytes, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_rc(e);
    ctx->ref_len = ref_len;
    ctx->ref_has_n = nbytes > 0;
    return BSW_OK;
}

int bsw_set_reference(bsw_ctx_t *ctx, const uint8_t *ref, int64_t ref_len)
{
    return bsw_set_reference_n(ctx, ref, nullptr, ref_len);
}

int bsw_extend_seeds(bsw_ctx_t *ctx, int64_t n_reads, const uint8_t *reads, const int64_t *read_off,
                     const int32_t *read_len, int64_t n_seeds, const bsw_seed_t *seeds, int32_t max_band_try,
                     bsw_aln_t *out, int64_t *cells_out)
{
    return bsw_extend_seeds_n(ctx, n_reads, reads, nullptr, read_off, read_len, n_seeds, seeds, max_band_try, out,
                              cells_out);
}

int bsw_extend_seeds_n(bsw_ctx_t *ctx, int64_t n_reads, const uint8_t *reads, const uint8_t *reads_n,
                       const int64_t *read_off, const int32_t *read_len, int64_t n_seeds, const bsw_seed_t *seeds,
                       int32_t max_band_try, bsw_aln_t *out, int64_t *cells_out)
{
    return guard([&]() -> int {
        if (!ctx || n_reads < 0 || n_seeds < 0 || n_seeds > INT32_MAX || max_band_try < 1 || max_band_try > 8)
            return BSW_EINVAL;
        if (n_seeds > 0 && (!reads || !read_off || !read_len || !seeds || !out)) return BSW_EINVAL;
        if (ctx->ref_len < 0) return BSW_ESTATE;
        if (!serving_idle(ctx)) return BSW_ESTATE;
        if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_rc(cudaErrorInvalidDevice);
        if (cells_out) *cells_out = 0;
        if (n_seeds == 0) return BSW_OK;
        const int w = ctx->P.w;
        if ((int64_t)w << (max_band_try - 1) > (1 << 20)) return BSW_EINVAL;

        // Checks on the device (launch_driver_check): reads, seeds inside their
        // read and the reference, each read's seeds consecutive, the score bound;
        // they also give the packed-read extent and the longest read.
        const int64_t N = n_seeds;
        Lane &lane = ctx->sync;
        cudaStream_t st = lane.S.main;
        cudaError_t e;
        size_t om = 0;
        auto take_m = [&](size_t bytes) { size_t r = om; om = align_up(om + bytes, 256); return r; };
        const size_t o_roff = take_m(8 * (size_t)n_reads), o_rlen = take_m(4 * (size_t)n_reads),
                     o_seeds = take_m(sizeof(bsw_seed_t) * (size_t)N), o_runs = take_m(4 * (size_t)n_reads),
                     o_chk = take_m(sizeof(DriverCheck));
        int rc = ctx->drvmeta.reserve(om, ctx->budget);
        if (rc != BSW_OK) return rc;
        uint8_t *dm = ctx->drvmeta.p;
        const struct { size_t off; const void *src; size_t bytes; } meta[] = {
            {o_roff, read_off, 8 * (size_t)n_reads}, {o_rlen, read_len, 4 * (size_t)n_reads},
            {o_seeds, seeds, sizeof(bsw_seed_t) * (size_t)N}};
        for (const auto &cp : meta)
            if (cp.bytes && (e = cudaMemcpyAsync(dm + cp.off, cp.src, cp.bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
                return cuda_rc(e);
        if ((e = cudaMemsetAsync(dm + o_runs, 0, om - o_runs, st)) != cudaSuccess) return cuda_rc(e);   // runs, check
        DriverCheck *chk = (DriverCheck *)(dm + o_chk);
        const DriverIn Dm{(const bsw_seed_t *)(dm + o_seeds), nullptr, (const int64_t *)(dm + o_roff),
                          (const int32_t *)(dm + o_rlen), ctx->refbuf.p, ctx->ref_len, nullptr, nullptr};
        if ((e = launch_driver_check(Dm, n_reads, N, ctx->P.a, (uint32_t *)(dm + o_runs), chk, st, ctx->sms)) != cudaSuccess)
            return cuda_rc(e);
        if ((e = cudaMemcpyAsync(ctx->h_chk, chk, sizeof(DriverCheck), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_rc(e);
        if (ctx->h_chk->inval) return BSW_EINVAL;
        const int64_t read_bytes = (int64_t)ctx->h_chk->read_bytes;
        const int maxrl = ctx->h_chk->maxrl;

        // Device layout: the reads, one side's pairs, the retry batch, the alignments.
        const int qslot = (int)align_up((size_t)std::max(maxrl, 1), 16);
        const int tslot = (int)align_up((size_t)maxrl + (size_t)w + 4, 16);
        size_t o = 0;
        auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
        const size_t o_reads = take((size_t)read_bytes),
                     o_q = take((size_t)N * qslot / 4), o_t = take((size_t)N * tslot / 4), o_qoff = take(8 * (size_t)N),
                     o_toff = take(8 * (size_t)N), o_qlen = take(4 * (size_t)N), o_tlen = take(4 * (size_t)N),
                     o_h0 = take(4 * (size_t)N), o_wcur = take(4 * (size_t)N), o_res = take(sizeof(bsw_result_t) * (size_t)N),
                     o_list = take(4 * (size_t)N), o_count = take(4), o_cqoff = take(8 * (size_t)N),
                     o_ctoff = take(8 * (size_t)N), o_cqlen = take(4 * (size_t)N), o_ctlen = take(4 * (size_t)N),
                     o_ch0 = take(4 * (size_t)N), o_cw = take(4 * (size_t)N),
                     o_cres = take(sizeof(bsw_result_t) * (size_t)N), o_aln = take(sizeof(bsw_aln_t) * (size_t)N),
                     o_cells = take(8 * 2 * (size_t)max_band_try);
        // N bitmaps: the reads' (read_bytes packed bytes hold 2 * read_bytes bitmap
        // bytes' worth of bases: (read_bytes + 1) / 2 bytes) and each side's slots
        const bool has_n = reads_n != nullptr || ctx->ref_has_n;
        const size_t rn_bytes = reads_n ? (size_t)((read_bytes + 1) / 2) : 0;
        const size_t o_rn = take(rn_bytes), o_qn = take(has_n ? (size_t)N * qslot / 8 : 0),
                     o_tn = take(has_n ? (size_t)N * tslot / 8 : 0);
        bool moved = false;
        if ((rc = ctx->drv.reserve(o, ctx->budget)) != BSW_OK) return rc;
        if ((rc = lane.ensure_work(N, std::max(maxrl, kShortMax), ctx->sms, ctx->budget, &moved)) != BSW_OK) return rc;
        if (moved) clear_graphs(ctx);
        uint8_t *d = ctx->drv.p;
        if (read_bytes && (e = cudaMemcpyAsync(d + o_reads, reads, (size_t)read_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_rc(e);
        if (rn_bytes && (e = cudaMemcpyAsync(d + o_rn, reads_n, rn_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_rc(e);
        const DriverIn D{Dm.seeds, d + o_reads, Dm.read_off, Dm.read_len, ctx->refbuf.p, ctx->ref_len,
                         reads_n ? d + o_rn : nullptr,
                         ctx->ref_has_n ? ctx->refbuf.p + align_up((size_t)((ctx->ref_len + 3) / 4), 256) : nullptr};
        const DriverSide S{d + o_q, d + o_t, (int64_t *)(d + o_qoff), (int64_t *)(d + o_toff), (int32_t *)(d + o_qlen),
                           (int32_t *)(d + o_tlen), (int32_t *)(d + o_h0), (int32_t *)(d + o_wcur),
                           (bsw_result_t *)(d + o_res), qslot, tslot, has_n ? d + o_qn : nullptr,
                           has_n ? d + o_tn : nullptr};
        const DriverCompact C{(int64_t *)(d + o_cqoff), (int64_t *)(d + o_ctoff), (int32_t *)(d + o_cqlen),
                              (int32_t *)(d + o_ctlen), (int32_t *)(d + o_ch0), (int32_t *)(d + o_cw),
                              (bsw_result_t *)(d + o_cres)};
        int32_t *list = (int32_t *)(d + o_list);
        uint32_t *count = (uint32_t *)(d + o_count);
        bsw_aln_t *aln = (bsw_aln_t *)(d + o_aln);
        unsigned long long *cells = (unsigned long long *)(d + o_cells);
        int n_runs = 0;
        bool first = true;
        auto extend = [&](const Batch &B) -> int {
            Work W = make_work(lane.work.p, lane.wl);
            W.cells = cells + n_runs++;
            cudaError_t le = enqueue_launch(ctx, lane, lane.S, B, W, 0u, first, ctx->plan);
            first = false;
            if (le != cudaSuccess) {
                lane.work_dirty = true;
                return cuda_rc(le);
            }
            return BSW_OK;
        };
        for (int side = 0; side < 2; ++side) {
            const bool left = side == 0;
            if ((e = launch_side(left, D, S, N, w, ctx->P.a, st, ctx->sms)) != cudaSuccess) return cuda_rc(e);
            if ((rc = extend(Batch{N, S.q, S.q_off, S.q_len, S.t, S.t_off, S.t_len, S.h0, nullptr, S.res, S.q_n, S.t_n})) !=
                BSW_OK)
                return rc;
            for (int t = 1; t < max_band_try; ++t) {
                const int wt = w << (t - 1), wnext = w << t;
                if ((e = cudaMemsetAsync(count, 0, 4, st)) != cudaSuccess) return cuda_rc(e);
                if ((e = launch_retry_select(S, N, wt, list, count, st, ctx->sms)) != cudaSuccess) return cuda_rc(e);
                uint32_t cnt = 0;
                if ((e = cudaMemcpyAsync(ctx->h_status, count, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                    (e = cudaStreamSynchronize(st)) != cudaSuccess)
                    return cuda_rc(e);
                cnt = *ctx->h_status;
                if (cnt == 0) break;
                if ((e = launch_retry_gather(S, list, count, cnt, wnext, C, st, ctx->sms)) != cudaSuccess) return cuda_rc(e);
                if ((rc = extend(Batch{(int64_t)cnt, S.q, C.q_off, C.q_len, S.t, C.t_off, C.t_len, C.h0, C.w, C.res, S.q_n,
                                       S.t_n})) != BSW_OK)
                    return rc;
                if ((e = launch_retry_scatter(S, list, count, cnt, wnext, C, st, ctx->sms)) != cudaSuccess) return cuda_rc(e);
            }
            if ((e = launch_decide(left, D, S, N, ctx->P.end_bonus, aln, st, ctx->sms)) != cudaSuccess) return cuda_rc(e);
        }
        if ((e = launch_filter(D, N, aln, st, ctx->sms)) != cudaSuccess) return cuda_rc(e);
        std::vector<unsigned long long> hc((size_t)n_runs);
        Work W = make_work(lane.work.p, lane.wl);
        if ((e = cudaMemcpyAsync(out, aln, sizeof(bsw_aln_t) * (size_t)N, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(hc.data(), cells, 8 * (size_t)n_runs, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(ctx->h_status, W.status, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_rc(e);
        if (cells_out) {
            unsigned long long tot = 0;
            for (unsigned long long c : hc) tot += c;
            *cells_out = (int64_t)tot;
        }
        return status_to_rc(*ctx->h_status);
    });
}

int bsw_sal_set_index(bsw_ctx_t *ctx, const int32_t *sa, int64_t sa_n)
{
    if (!ctx || sa_n < 0 || (sa_n > 0 && !sa)) return BSW_EINVAL;
    if (!serving_idle(ctx)) return BSW_ESTATE;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_rc(cudaErrorInvalidDevice);
    ctx->sa_n = -1;
    const size_t bytes = 4 * (size_t)sa_n;
    int rc = ctx->sabuf.reserve(bytes > 0 ? bytes : 4, ctx->budget);
    if (rc != BSW_OK) return rc;
    if (bytes) {
        cudaError_t e = cudaMemcpy(ctx->sabuf.p, sa, bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_rc(e);
    }
    ctx->sa_n = sa_n;
    return BSW_OK;
}

int bsw_sal_lookup(bsw_ctx_t *ctx, int64_t n_int, const int64_t *k, const int32_t *cnt, const int64_t *off,
                   int32_t *positions, uint32_t flags, void *cuda_stream)
{
    if (!ctx || n_int < 0 || (flags & ~BSW_DEVICE_PTRS)) return BSW_EINVAL;
    if (ctx->sa_n < 0) return BSW_ESTATE;
    if (n_int == 0) return BSW_OK;
    if (!k || !cnt || !off || !positions) return BSW_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_rc(cudaErrorInvalidDevice);
    const int32_t *sa = (const int32_t *)ctx->sabuf.p;
    cudaError_t e;
    if (flags & BSW_DEVICE_PTRS) {
        // enqueue only; an interval outside the suffix array is reported by bsw_sync
        Lane &lane = ctx->sync;
        bool moved = false;
        int rc = lane.ensure_work(1, kShortMax, ctx->sms, ctx->budget, &moved);
        if (rc != BSW_OK) return rc;
        if (moved) clear_graphs(ctx);
        Work W = make_work(lane.work.p, lane.wl);
        cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : lane.S.main;
        return cuda_rc(launch_sal(sa, ctx->sa_n, k, cnt, off, n_int, positions, W.status, st, ctx->sms));
    }
    // host pointers: check, stage, gather, copy back
    int64_t total = 0;
    for (int64_t t = 0; t < n_int; ++t) {
        if (k[t] < 0 || cnt[t] < 0 || k[t] + cnt[t] > ctx->sa_n || off[t] < 0) return BSW_EINVAL;
        total = std::max(total, off[t] + cnt[t]);
    }
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
    const size_t o_k = take(8 * (size_t)n_int), o_c = take(4 * (size_t)n_int), o_o = take(8 * (size_t)n_int),
                 o_p = take(4 * (size_t)total), o_st = take(4);
    int rc = ctx->salio.reserve(o, ctx->budget);
    if (rc != BSW_OK) return rc;
    uint8_t *d = ctx->salio.p;
    cudaStream_t st = ctx->sync.S.main;
    if ((e = cudaMemcpyAsync(d + o_k, k, 8 * (size_t)n_int, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d + o_c, cnt, 4 * (size_t)n_int, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d + o_o, off, 8 * (size_t)n_int, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(d + o_st, 0, 4, st)) != cudaSuccess)
        return cuda_rc(e);
    if ((e = launch_sal(sa, ctx->sa_n, (const int64_t *)(d + o_k), (const int32_t *)(d + o_c),
                        (const int64_t *)(d + o_o), n_int, (int32_t *)(d + o_p), (uint32_t *)(d + o_st), st,
                        ctx->sms)) != cudaSuccess)
        return cuda_rc(e);
    if ((total && (e = cudaMemcpyAsync(positions, d + o_p, 4 * (size_t)total, cudaMemcpyDeviceToHost, st)) != cudaSuccess) ||
        (e = cudaMemcpyAsync(ctx->h_status, d + o_st, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_rc(e);
    return status_to_rc(*ctx->h_status);
}

int bsw_fm_build(bsw_ctx_t *ctx, const uint8_t *ref, int64_t n)
{
    if (!ctx || n < 1 || n >= (1ll << 30) || !ref) return BSW_EINVAL;
    if (!serving_idle(ctx)) return BSW_ESTATE;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_rc(cudaErrorInvalidDevice);
    ctx->fm_ready = false;
    FmHost ft;
    try {
        std::vector<uint8_t> T((size_t)(2 * n));
        for (int64_t i = 0; i < n; ++i) {
            if (ref[i] > 3) return BSW_EINVAL;
            T[(size_t)i] = ref[i];
            T[(size_t)(2 * n - 1 - i)] = (uint8_t)(3 - ref[i]);   // reverse complement
        }
        std::vector<int32_t> sa((size_t)(2 * n + 1));
        int rc = bsw_sa_build(T.data(), 2 * n, sa.data());
        if (rc != BSW_OK) return rc;
        fm_from_sa(T.data(), 2 * n, sa.data(), ft);
    } catch (const std::bad_alloc &) {
        return BSW_ENOMEM;
    }
    const size_t bt = sizeof(FmEntry) * ft.occ.size();
    int rc = ctx->fmbuf.reserve(bt, ctx->budget);
    if (rc != BSW_OK) return rc;
    cudaError_t e;
    if ((e = cudaMemcpy(ctx->fmbuf.p, ft.occ.data(), bt, cudaMemcpyHostToDevice)) != cudaSuccess) return cuda_rc(e);
    ctx->fm_t = FmDev{(const FmEntry *)ctx->fmbuf.p, ft.n, ft.primary, {ft.C[0], ft.C[1], ft.C[2], ft.C[3], ft.C[4]}};
    ctx->fm_ready = true;
    return BSW_OK;
}

int bsw_smem(bsw_ctx_t *ctx, int64_t n_reads, const uint8_t *reads, const int64_t *read_off,
             const int32_t *read_len, int32_t min_len, bsw_smem_t *out, int64_t out_cap, int64_t *n_out,
             int64_t *first)
{
    return bsw_smem_n(ctx, n_reads, reads, nullptr, read_off, read_len, min_len, out, out_cap, n_out, first);
}

int bsw_smem_n(bsw_ctx_t *ctx, int64_t n_reads, const uint8_t *reads, const uint8_t *reads_n, const int64_t *read_off,
               const int32_t *read_len, int32_t min_len, bsw_smem_t *out, int64_t out_cap, int64_t *n_out,
               int64_t *first)
{
    return guard([&]() -> int {
        if (!ctx || n_reads < 0 || min_len < 1 || out_cap < 0 || !n_out) return BSW_EINVAL;
        if (n_reads > 0 && (!reads || !read_off || !read_len)) return BSW_EINVAL;
        if (!ctx->fm_ready) return BSW_ESTATE;
        if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_rc(cudaErrorInvalidDevice);
        *n_out = 0;
        if (first) first[0] = 0;
        if (n_reads == 0) return BSW_OK;
        int64_t read_bytes = 0;
        int lmax = 0;
        for (int64_t r = 0; r < n_reads; ++r) {
            if (read_off[r] < 0 || (read_off[r] & 3) || read_len[r] < 0 || read_len[r] > kLongMax) return BSW_EINVAL;
            read_bytes = std::max(read_bytes, (read_off[r] + read_len[r] + 3) / 4);
            lmax = std::max(lmax, (int)read_len[r]);
        }
        size_t o = 0;
        auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
        const size_t o_reads = take((size_t)read_bytes), o_roff = take(8 * (size_t)n_reads),
                     o_rlen = take(4 * (size_t)n_reads), o_cnt = take(8 * (size_t)n_reads),
                     o_first = take(8 * (size_t)n_reads), o_ids = take(4 * (size_t)n_reads), o_nids = take(4),
                     o_next = take(4), o_keep = take(sizeof(bsw_smem_t) * kSmemKeep * (size_t)n_reads),
                     o_rn = take(reads_n ? (size_t)((read_bytes + 1) / 2) : 0),
                     o_out = take(sizeof(bsw_smem_t) * (size_t)std::max<int64_t>(out_cap, 1));
        int rc = ctx->smemio.reserve(o, ctx->budget);
        if (rc != BSW_OK) return rc;
        uint8_t *d = ctx->smemio.p;
        cudaStream_t st = ctx->sync.S.main;
        cudaError_t e;
        if ((e = cudaMemcpyAsync(d + o_reads, reads, (size_t)read_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(d + o_roff, read_off, 8 * (size_t)n_reads, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(d + o_rlen, read_len, 4 * (size_t)n_reads, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = cudaMemsetAsync(d + o_nids, 0, 4, st)) != cudaSuccess)
            return cuda_rc(e);
        if (reads_n && read_bytes &&
            (e = cudaMemcpyAsync(d + o_rn, reads_n, (size_t)((read_bytes + 1) / 2), cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_rc(e);
        const SmemIn R{d + o_reads, (const int64_t *)(d + o_roff), (const int32_t *)(d + o_rlen), n_reads, lmax,
                       reads_n ? d + o_rn : nullptr};
        int32_t *ids = (int32_t *)(d + o_ids);
        uint32_t *nids = (uint32_t *)(d + o_nids);
        int64_t *dfirst = (int64_t *)(d + o_first);
        const SmemWork W{(int64_t *)(d + o_cnt), (bsw_smem_t *)(d + o_keep), dfirst, (bsw_smem_t *)(d + o_out),
                         (uint32_t *)(d + o_next), nids, ids};
        auto global_lists = [&](int64_t n_ids, BiIv **lists) -> int {      // lmax + 1 entries hold any list
            const int r2 = ctx->smemscratch.reserve(sizeof(BiIv) * (size_t)n_ids * (size_t)(lmax + 1), ctx->budget);
            *lists = (BiIv *)ctx->smemscratch.p;
            return r2;
        };

        // One search pass: counts, and the records of reads with few; reads whose
        // lists overflow shared memory are searched with lists in global memory.
        if ((e = launch_smem_store(R, ctx->fm_t, min_len, W, st, ctx->sms)) != cudaSuccess ||
            (e = cudaMemcpyAsync(ctx->h_status, nids, 4, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_rc(e);
        const int64_t n_ovf = *ctx->h_status;
        if (n_ovf > 0) {
            BiIv *lists = nullptr;
            if ((rc = global_lists(n_ovf, &lists)) != BSW_OK) return rc;
            if ((e = launch_smem_global(false, R, ctx->fm_t, min_len, W, ids, n_ovf, lists, lmax + 1, st, ctx->sms)) !=
                cudaSuccess)
                return cuda_rc(e);
        }
        std::vector<int64_t> hc((size_t)n_reads), hf((size_t)n_reads + 1);
        if ((e = cudaMemcpyAsync(hc.data(), W.count, 8 * (size_t)n_reads, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_rc(e);
        hf[0] = 0;
        std::vector<int32_t> many;                                        // reads with more records than were kept
        for (int64_t r = 0; r < n_reads; ++r) {
            hf[(size_t)r + 1] = hf[(size_t)r] + hc[(size_t)r];
            if (hc[(size_t)r] > kSmemKeep) many.push_back((int32_t)r);
        }
        const int64_t total = hf[(size_t)n_reads];
        *n_out = total;
        if (first) std::memcpy(first, hf.data(), 8 * ((size_t)n_reads + 1));
        if (total > out_cap) return BSW_EBUDGET;
        if (total == 0) return BSW_OK;
        if ((e = cudaMemcpyAsync(dfirst, hf.data(), 8 * (size_t)n_reads, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
            (e = launch_smem_gather(n_reads, W, st, ctx->sms)) != cudaSuccess)
            return cuda_rc(e);
        if (!many.empty()) {
            BiIv *lists = nullptr;
            if ((rc = global_lists((int64_t)many.size(), &lists)) != BSW_OK) return rc;
            if ((e = cudaMemcpyAsync(ids, many.data(), 4 * many.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
                (e = launch_smem_global(true, R, ctx->fm_t, min_len, W, ids, (int64_t)many.size(), lists, lmax + 1, st,
                                        ctx->sms)) != cudaSuccess)
                return cuda_rc(e);
        }
        if ((e = cudaMemcpyAsync(out, W.out, sizeof(bsw_smem_t) * (size_t)total, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_rc(e);
        return BSW_OK;
    });
}

void bsw_destroy(bsw_ctx_t *ctx)
{
    if (!ctx) return;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->stop = true;
    }
    ctx->cv_work.notify_all();
    if (ctx->server_started) ctx->server.join();
    cudaSetDevice(ctx->device);
    clear_graphs(ctx);
    for (int li = 0; li < kServeLanes; ++li)
        if (ctx->lane_created[li]) ctx->serve_lane[li].destroy(ctx->budget);
    ctx->sync.destroy(ctx->budget);
    ctx->refbuf.release(ctx->budget);
    ctx->drv.release(ctx->budget);
    ctx->drvmeta.release(ctx->budget);
    ctx->sabuf.release(ctx->budget);
    ctx->salio.release(ctx->budget);
    ctx->fmbuf.release(ctx->budget);
    ctx->smemio.release(ctx->budget);
    ctx->smemscratch.release(ctx->budget);
    if (ctx->timer_ready)
        for (int k = 0; k <= kNumClass; ++k) {
            cudaEventDestroy(ctx->timer.t0[k]);
            cudaEventDestroy(ctx->timer.t1[k]);
        }
    for (cudaEvent_t ev : ctx->tune_ev)
        if (ev) cudaEventDestroy(ev);
    for (auto &kv : ctx->tickets) delete kv.second;
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    if (ctx->h_cells) cudaFreeHost(ctx->h_cells);
    if (ctx->h_ext) cudaFreeHost(ctx->h_ext);
    if (ctx->h_chk) cudaFreeHost(ctx->h_chk);
    delete ctx;
}

}  // extern "C"
