// Continuous-batching request server of the GB300 Serial-EMD library.
//
// A host worker thread owns one CUDA stream and a device memory pool of the server's
// byte budget. Requests wait in a FIFO queue; whenever a slot is free and the pool can
// hold a request's working buffers (first-fit), the request is admitted: its signal is
// serialized (Sec. 3.2) and it joins the next sifting pass. Each round runs a few passes
// of the sifting loop (k_pass over the tiles of every admitted request, then k_reduce
// over the requests, Sec. 2.1) for all admitted requests at once; requests admitted in
// different rounds are at different stages of their decompositions within one pass.
// After each round the worker reads the requests' states; a finished request gets its
// residue de-serialized (Sec. 3.3), its result recorded and its memory and slot freed,
// which lets queued requests in. Every request's arithmetic depends only on its own
// data, so its result is bit-identical to decomposing it alone.
#include "semd_runtime.h"

#include <algorithm>
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace semd {

using Clock = std::chrono::steady_clock;

// First-fit allocator of byte ranges in the device pool (256-byte granules).
class PoolAlloc {
  public:
    void init(size_t bytes)
    {
        free_.clear();
        if (bytes)
            free_[0] = bytes;
    }
    bool alloc(size_t bytes, size_t &off)
    {
        bytes = round(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                off = it->first;
                const size_t rest = it->second - bytes;
                free_.erase(it);
                if (rest)
                    free_[off + bytes] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = round(bytes);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    static size_t round(size_t b) { return (b + 255) & ~(size_t)255; }

  private:
    std::map<size_t, size_t> free_; // offset -> length
};

// Per-request device buffers, carved from one pool range.
struct ReqLayout {
    int64_t Lp = 0, nt = 0, rlen = 0;
    size_t h = 0, r = 0, tex = 0, tsol = 0, taux = 0, rscr = 0, kmask = 0, total = 0;
};

static ReqLayout req_layout(int64_t L, size_t elem, int tile)
{
    ReqLayout q;
    q.Lp = (L + 31) & ~(int64_t)31;
    q.nt = (L + tile - 1) / tile;
    q.rlen = reduce_len(q.nt);
    auto R = PoolAlloc::round;
    q.h = R((size_t)q.Lp * elem);
    q.r = R((size_t)q.Lp * 8);
    q.tex = R((size_t)q.nt * 2 * tile_rec_bytes(elem));
    q.tsol = R((size_t)q.nt * 2 * sizeof(TileSolve));
    q.taux = R((size_t)q.nt * sizeof(TileAux));
    q.rscr = R((size_t)(2 * rscr_env_doubles(q.rlen)) * 8);
    q.kmask = R((size_t)q.nt * 32 * sizeof(uint2));
    q.total = 2 * q.h + 2 * q.r + q.tex + q.tsol + q.taux + q.rscr + q.kmask;
    return q;
}

struct Request {
    uint64_t ticket = 0;
    semd_request req{};
    int64_t M = 0, N = 0, D = 0, L = 0;
    ReqLayout lay;
    Clock::time_point t_submit, t_admit;
};

struct Slot {
    bool used = false;
    bool fresh = false; // admitted this round: serialize, then the INIT pass
    Request rq;
    size_t off = 0;
};

} // namespace semd

namespace semd {
// A lane of the server: its own worker thread, stream, requests and launch arrays. Small
// requests and large ones (at least kLargeSamples serialized samples) run in separate
// lanes, so the passes over a large request never hold up the small ones: the small lane's
// stream has the higher priority, and the large lane's pass grid keeps to part of each SM,
// so both lanes' kernels run side by side.
constexpr int64_t kLargeSamples = (int64_t)1 << 21;
struct Lane {
    int max_inflight = 1;
    int tile = kTile;    // pass-kernel tile of the lane's requests
    int ctas_per_sm = 0; // pass-grid cap (0: as many CTAs as fit)
    int64_t cap_tiles = 0;
    Inst *d_inst = nullptr, *h_inst = nullptr;
    State *d_state = nullptr, *h_state = nullptr;
    int32_t *d_tiles = nullptr, *h_tiles = nullptr; // pass launch: tile -> slot
    int32_t *d_list = nullptr, *h_list = nullptr;   // reduce launch: block -> slot
    int32_t *d_active = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    std::vector<Slot> slots;
    std::deque<Request> queue;
    std::thread worker;
};
} // namespace semd

struct semd_server_s {
    semd_params p{};
    size_t budget = 0, elem = 4;
    int64_t Lmax = 0;
    void *pool = nullptr;
    semd::PoolAlloc alloc;
    semd::Lane lanes[2]; // 0: small requests, 1: large requests
    std::mutex mu;
    std::condition_variable cv;      // work for a worker (or stop)
    std::condition_variable cv_done; // a result was recorded
    std::unordered_map<uint64_t, semd_result> results;
    std::unordered_set<uint64_t> pending;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::string err;

    void run(int li);
    bool round(semd::Lane &ln, std::string &e);
    void fail_lane(semd::Lane &ln, int status);
    void release_device();
};

namespace semd {
static thread_local std::string g_server_create_error;

static double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}
} // namespace semd

using namespace semd;

#define SV_CU(call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            e = std::string(#call) + ": " + cudaGetErrorString(e_);                        \
            return false;                                                                  \
        }                                                                                  \
    } while (0)

// One round of a lane: admit, launch a few passes for every admitted request, collect
// finished ones. Returns false on a CUDA error (message in e).
bool semd_server_s::round(Lane &ln, std::string &e)
{
    // admission, FIFO within the lane: a request waits until a slot and pool space are free
    std::vector<int> fresh;
    {
        std::lock_guard<std::mutex> lk(mu);
        while (!ln.queue.empty()) {
            Request &rq = ln.queue.front();
            int si = -1;
            for (int i = 0; i < ln.max_inflight; ++i)
                if (!ln.slots[i].used) {
                    si = i;
                    break;
                }
            size_t off = 0;
            if (si < 0 || !alloc.alloc(rq.lay.total, off))
                break;
            Slot &sl = ln.slots[si];
            sl.used = true;
            sl.fresh = true;
            sl.off = off;
            sl.rq = rq;
            sl.rq.t_admit = Clock::now();
            ln.queue.pop_front();
            fresh.push_back(si);
        }
    }
    // descriptors and tile maps of every admitted request
    int64_t ntiles = 0, max_nt = 0, min_nt = INT64_MAX;
    int nact = 0;
    for (int i = 0; i < ln.max_inflight; ++i) {
        Slot &sl = ln.slots[i];
        if (!sl.used)
            continue;
        const Request &rq = sl.rq;
        const ReqLayout &q = rq.lay;
        char *b = (char *)pool + sl.off;
        Inst in{};
        in.L = rq.L;
        in.M = rq.M;
        in.N = rq.N;
        in.D = rq.D;
        in.tile0 = (int32_t)ntiles;
        in.ntiles = (int32_t)q.nt;
        in.order = rq.req.order;
        in.imf_serialized = 0;
        in.h[0] = b;
        in.h[1] = b + q.h;
        in.r[0] = (double *)(b + 2 * q.h);
        in.r[1] = (double *)(b + 2 * q.h + q.r);
        char *c = b + 2 * q.h + 2 * q.r;
        in.tex = c;
        in.tsol = (TileSolve *)(c + q.tex);
        in.taux = (TileAux *)(c + q.tex + q.tsol);
        in.rscr = (double *)(c + q.tex + q.tsol + q.taux);
        in.kmask = (uint2 *)(c + q.tex + q.tsol + q.taux + q.rscr);
        in.rlen = q.rlen;
        in.x = rq.req.d_x;
        in.imf = rq.req.d_imfs;
        in.res = rq.req.d_residue;
        in.imf_stride = rq.req.rows * rq.req.cols;
        ln.h_inst[i] = in;
        for (int64_t t = 0; t < q.nt; ++t)
            ln.h_tiles[ntiles + t] = i;
        ntiles += q.nt;
        max_nt = std::max<int64_t>(max_nt, q.nt);
        min_nt = std::min<int64_t>(min_nt, q.nt);
        ln.h_list[nact++] = i;
    }
    if (nact == 0)
        return true;
    SV_CU(cudaMemcpyAsync(ln.d_inst, ln.h_inst, (size_t)ln.max_inflight * sizeof(Inst),
                          cudaMemcpyHostToDevice, ln.stream));
    SV_CU(cudaMemcpyAsync(ln.d_tiles, ln.h_tiles, (size_t)ntiles * 4, cudaMemcpyHostToDevice,
                          ln.stream));
    SV_CU(cudaMemcpyAsync(ln.d_list, ln.h_list, (size_t)nact * 4, cudaMemcpyHostToDevice,
                          ln.stream));
    if (!fresh.empty()) {
        // fresh states are zero (MODE_INIT): serialize only those instances
        for (int si : fresh)
            SV_CU(cudaMemsetAsync(ln.d_state + si, 0, sizeof(State), ln.stream));
        launch_serialize_any(elem, ln.d_inst, ln.d_state, ln.d_tiles, ntiles, ln.tile, ln.stream);
    }
    for (int si : fresh)
        ln.slots[si].fresh = false;
    // a few passes per round; fewer while requests are waiting, so they join sooner
    bool waiting, small_busy = false;
    {
        std::lock_guard<std::mutex> lk(mu);
        waiting = !ln.queue.empty();
        for (const Slot &sl : lanes[0].slots)
            small_busy = small_busy || sl.used;
        small_busy = small_busy || !lanes[0].queue.empty();
    }
    const int passes = waiting ? 2 : 8;
    // the large lane leaves room on every SM only while small requests are on the GPU
    const int ctas = (&ln == &lanes[1] && small_busy) ? ln.ctas_per_sm : 0;
    NvtxRange nvtx("server round");
    PassArgs pa{ln.d_inst, ln.d_state, ln.d_tiles, ntiles, p.stop == SEMD_STOP_SD ? 1 : 0,
                p.stop == SEMD_STOP_SNUMBER ? 1 : 0};
    ReduceArgs ra = make_reduce_args(p, ln.d_inst, ln.d_state, ln.d_list, ln.d_active, elem,
                                     min_nt, max_nt);
    for (int it = 0; it < passes; ++it) {
        launch_pass_any(elem, ln.tile, pa, ntiles, ln.stream, ctas);
        launch_reduce_any(elem, ra, nact, ln.stream);
    }
    SV_CU(cudaGetLastError());
    SV_CU(cudaMemcpyAsync(ln.h_state, ln.d_state, (size_t)ln.max_inflight * sizeof(State),
                          cudaMemcpyDeviceToHost, ln.stream));
    SV_CU(cudaEventRecord(ln.ev, ln.stream));
    SV_CU(cudaEventSynchronize(ln.ev));
    // finished requests (state MODE_DONE): residue de-serialization and zero-fill over
    // the same tile map, then release
    std::vector<int> fin;
    for (int k = 0; k < nact; ++k)
        if (ln.h_state[ln.h_list[k]].mode == MODE_DONE)
            fin.push_back(ln.h_list[k]);
    if (fin.empty())
        return true;
    launch_finalize_any(elem, ln.d_inst, ln.d_state, ln.d_tiles, ntiles, ln.tile, p.max_imfs,
                        ln.stream);
    SV_CU(cudaGetLastError());
    SV_CU(cudaEventRecord(ln.ev, ln.stream));
    SV_CU(cudaEventSynchronize(ln.ev));
    const Clock::time_point now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(mu);
        for (int i : fin) {
            Slot &sl = ln.slots[i];
            const State &st = ln.h_state[i];
            semd_result r{};
            r.status = SEMD_OK;
            r.n_imfs = st.imf_count;
            int64_t sifts = 0;
            for (int k = 0; k < st.imf_count && k < KMAX; ++k)
                sifts += st.sifts[k];
            r.sifts = sifts;
            r.queue_ms = ms_between(sl.rq.t_submit, sl.rq.t_admit);
            r.run_ms = ms_between(sl.rq.t_admit, now);
            results[sl.rq.ticket] = r;
            pending.erase(sl.rq.ticket);
            alloc.release(sl.off, sl.rq.lay.total);
            sl.used = false;
        }
    }
    cv_done.notify_all();
    cv.notify_all(); // freed pool space may admit the other lane's requests
    return true;
}

// Ends every request of a lane (admitted or queued) with `status`.
void semd_server_s::fail_lane(Lane &ln, int status)
{
    {
        std::lock_guard<std::mutex> lk(mu);
        auto mark = [&](const Request &rq) {
            semd_result r{};
            r.status = status;
            results[rq.ticket] = r;
            pending.erase(rq.ticket);
        };
        for (auto &sl : ln.slots)
            if (sl.used) {
                mark(sl.rq);
                alloc.release(sl.off, sl.rq.lay.total);
                sl.used = false;
            }
        for (auto &rq : ln.queue)
            mark(rq);
        ln.queue.clear();
    }
    cv_done.notify_all();
}

void semd_server_s::run(int li)
{
    Lane &ln = lanes[li];
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(mu);
            bool busy = false;
            for (auto &sl : ln.slots)
                busy = busy || sl.used;
            if (!busy)
                cv.wait(lk, [&] { return stop || !ln.queue.empty(); });
            if (stop)
                break;
        }
        std::string e;
        if (!round(ln, e)) {
            cudaStreamSynchronize(ln.stream);
            fail_lane(ln, SEMD_ECUDA);
            {
                std::lock_guard<std::mutex> lk(mu);
                err = e;
                stop = true;
            }
            cv.notify_all();
            break;
        }
    }
    cudaStreamSynchronize(ln.stream);
    fail_lane(ln, SEMD_ECANCELED);
}

void semd_server_s::release_device()
{
    for (Lane &ln : lanes) {
        if (ln.ev)
            cudaEventDestroy(ln.ev);
        if (ln.stream)
            cudaStreamDestroy(ln.stream);
        void *dev[] = {ln.d_inst, ln.d_state, ln.d_tiles, ln.d_list, ln.d_active};
        for (void *q : dev)
            if (q)
                cudaFree(q);
        void *host[] = {ln.h_inst, ln.h_state, ln.h_tiles, ln.h_list};
        for (void *q : host)
            if (q)
                cudaFreeHost(q);
    }
    if (pool)
        cudaFree(pool);
}

extern "C" {

semd_status serial_emd_server_create(const semd_params *defaults, size_t mem_budget,
                                     int max_inflight, semd_server_t *out)
{
    std::string &err = g_server_create_error;
    err.clear();
    if (!defaults || !out || mem_budget == 0 || max_inflight < 1) {
        err = "null argument, zero budget or max_inflight < 1";
        return SEMD_EINVAL;
    }
    *out = nullptr;
    if (!validate(*defaults, err))
        return SEMD_EINVAL;
    if (defaults->ensemble_trials > 1) {
        err = "the server decomposes EMD requests; EEMD is served by plans";
        return SEMD_EUNSUPPORTED;
    }
    int64_t M, N, D;
    if (!geometry(*defaults, defaults->rows, defaults->cols, defaults->order, M, N, D, err))
        return SEMD_EINVAL;
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) {
        err = "no CUDA device is available";
        return SEMD_ECUDA;
    }
    semd_server_s *sv = new (std::nothrow) semd_server_s();
    if (!sv) {
        err = "out of host memory";
        return SEMD_ENOMEM;
    }
    sv->p = *defaults;
    sv->budget = mem_budget;
    sv->elem = defaults->precision == SEMD_FP64 ? 8 : 4;
    sv->Lmax = serial_length(M, N, D);
    // every admitted request holds at least (2w + 16) bytes per sample of the pool
    // lane 0 (small requests) keeps most slots; lane 1 (large ones) a few, and its pass
    // grid takes at most two CTAs per SM
    const int nlarge = std::max(1, max_inflight / 8);
    sv->lanes[0].max_inflight = max_inflight;
    sv->lanes[1].max_inflight = nlarge;
    sv->lanes[1].ctas_per_sm = 2;
    // large requests: 512-sample tiles halve their interface systems, the longest step of
    // a sift at millions of samples (measured on a 2048 x 2048 image: 29 instead of 47 ms)
    sv->lanes[1].tile = 512;
    int prio_lo = 0, prio_hi = 0;
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (e == cudaSuccess)
        e = cudaMalloc(&sv->pool, mem_budget);
    for (int li = 0; li < 2 && e == cudaSuccess; ++li) {
        Lane &ln = sv->lanes[li];
        ln.cap_tiles = (int64_t)(mem_budget / ((2 * sv->elem + 16) * (size_t)ln.tile)) +
                       2 * (int64_t)ln.max_inflight;
        ln.slots.resize(ln.max_inflight);
        const size_t ni = (size_t)ln.max_inflight, nt = (size_t)ln.cap_tiles;
        e = cudaMalloc((void **)&ln.d_inst, ni * sizeof(Inst));
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&ln.d_state, ni * sizeof(State));
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&ln.d_tiles, nt * 4);
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&ln.d_list, ni * 4);
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&ln.d_active, 64);
        if (e == cudaSuccess)
            e = cudaMallocHost((void **)&ln.h_inst, ni * sizeof(Inst));
        if (e == cudaSuccess)
            e = cudaMallocHost((void **)&ln.h_state, ni * sizeof(State));
        if (e == cudaSuccess)
            e = cudaMallocHost((void **)&ln.h_tiles, nt * 4);
        if (e == cudaSuccess)
            e = cudaMallocHost((void **)&ln.h_list, ni * 4);
        if (e == cudaSuccess)
            e = cudaStreamCreateWithPriority(&ln.stream, cudaStreamNonBlocking,
                                             li == 0 ? prio_hi : prio_lo);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&ln.ev, cudaEventDisableTiming);
        if (e == cudaSuccess)
            std::memset(ln.h_inst, 0, ni * sizeof(Inst));
    }
    if (e == cudaSuccess)
        e = setup_kernel_attrs(sv->elem);
    if (e != cudaSuccess) {
        err = std::string("server set-up: ") + cudaGetErrorString(e);
        (void)cudaGetLastError(); // a failed allocation must not surface in later calls
        sv->release_device();
        delete sv;
        return e == cudaErrorMemoryAllocation ? SEMD_ENOMEM : SEMD_ECUDA;
    }
    sv->alloc.init(mem_budget);
    for (int li = 0; li < 2; ++li)
        sv->lanes[li].worker = std::thread([sv, li] { sv->run(li); });
    *out = sv;
    return SEMD_OK;
}

semd_status serial_emd_submit(semd_server_t sv, const semd_request *req, uint64_t *ticket)
{
    if (!sv || !req || !ticket)
        return SEMD_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) {
        sv->err = "the server has stopped";
        return SEMD_ECANCELED;
    }
    if (!req->d_x || !req->d_imfs) {
        sv->err = "null input or output pointer";
        return SEMD_EINVAL;
    }
    if (req->order != SEMD_ORDER_ROWS && req->order != SEMD_ORDER_COLS) {
        sv->err = "order must be ROWS or COLS";
        return SEMD_EINVAL;
    }
    Request rq;
    if (!geometry(sv->p, req->rows, req->cols, req->order, rq.M, rq.N, rq.D, sv->err))
        return SEMD_EINVAL;
    rq.L = serial_length(rq.M, rq.N, rq.D);
    const int li = rq.L >= kLargeSamples ? 1 : 0;
    rq.lay = req_layout(rq.L, sv->elem, sv->lanes[li].tile);
    if (rq.L > sv->Lmax || PoolAlloc::round(rq.lay.total) > sv->budget ||
        rq.lay.nt > sv->lanes[li].cap_tiles) {
        sv->err = "the request is larger than the server accepts (" +
                  std::to_string(rq.lay.total) + " bytes of working buffers)";
        return SEMD_EBUDGET;
    }
    rq.req = *req;
    rq.ticket = sv->next_ticket++;
    rq.t_submit = Clock::now();
    sv->pending.insert(rq.ticket);
    sv->lanes[li].queue.push_back(rq);
    *ticket = rq.ticket;
    sv->cv.notify_all();
    return SEMD_OK;
}

semd_status serial_emd_poll(semd_server_t sv, uint64_t ticket, semd_result *out)
{
    if (!sv || !out)
        return SEMD_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->results.find(ticket);
    if (it != sv->results.end()) {
        *out = it->second;
        sv->results.erase(it);
        return SEMD_OK;
    }
    if (sv->pending.count(ticket))
        return SEMD_PENDING;
    sv->err = "unknown ticket (or its result was already returned)";
    return SEMD_EINVAL;
}

semd_status serial_emd_wait(semd_server_t sv, uint64_t ticket, double timeout_ms,
                            semd_result *out)
{
    if (!sv || !out || !(timeout_ms >= 0))
        return SEMD_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    const auto deadline =
        Clock::now() + std::chrono::duration_cast<Clock::duration>(
                           std::chrono::duration<double, std::milli>(timeout_ms));
    for (;;) {
        auto it = sv->results.find(ticket);
        if (it != sv->results.end()) {
            *out = it->second;
            sv->results.erase(it);
            return SEMD_OK;
        }
        if (!sv->pending.count(ticket)) {
            sv->err = "unknown ticket (or its result was already returned)";
            return SEMD_EINVAL;
        }
        if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout &&
            Clock::now() >= deadline) {
            auto again = sv->results.find(ticket);
            if (again != sv->results.end()) {
                *out = again->second;
                sv->results.erase(again);
                return SEMD_OK;
            }
            sv->err = "the request did not finish within the time limit";
            return SEMD_ETIMEOUT;
        }
    }
}

void serial_emd_server_destroy(semd_server_t sv)
{
    if (!sv)
        return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv.notify_all();
    for (Lane &ln : sv->lanes)
        if (ln.worker.joinable())
            ln.worker.join();
    sv->release_device();
    delete sv;
}

const char *serial_emd_server_last_error(semd_server_t sv)
{
    if (!sv)
        return g_server_create_error.c_str();
    std::lock_guard<std::mutex> lk(sv->mu);
    thread_local std::string copy;
    copy = sv->err;
    return copy.c_str();
}

} // extern "C"
