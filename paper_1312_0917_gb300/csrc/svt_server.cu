// svt_server.cu -- serving runtime: continuous batching of independent event
// batches (requests) over a fixed set of device slots.
//
// Each slot owns a context (device buffers sized for one request), a copy
// stream and a compute stream, pinned host staging for the request's words,
// and a track buffer in mapped pinned host memory that the kernel's output
// stage writes directly (over the CPU-GPU link, no device-to-host copy).  A
// request is admitted when a slot is free; its host->device copy (copy
// stream), then its persistent kernel and control-block read (compute
// stream, after the copy's event) are enqueued at once, so requests admitted
// while others run overlap on the device (each kernel takes a share of the
// SMs).  A progress thread watches the slots' events; when a slot's control
// block has arrived its tracks are already in host memory, and the result is
// published.  Latency runs from svt_server_submit to that moment.
//
// A request larger than a slot (more words, events or roads than a slot's
// limits) is cut at event boundaries into chunks that fit, and each chunk is
// admitted like a request of its own as slots free up; the chunks' results
// are joined in stream order (event indices offset) into the request's
// result once the last chunk is done.  Events are independent (the
// hit-warrior's scope is one event), so the joined result is the whole
// request's.
#include "svt_ctx.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

using namespace svt;

static_assert(sizeof(svt_server_config) == 56, "svt_server_config layout");
static_assert(sizeof(svt_server_result) == 48, "svt_server_result layout");

namespace {

using Clock = std::chrono::steady_clock;

enum SlotState { SLOT_FREE = 0, SLOT_RESERVED, SLOT_RUNNING };

struct Slot {
    svt_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;   // compute: kernel and control-block read
    cudaStream_t copy = nullptr;     // host->device copy of the words
    uint32_t *h_words = nullptr;     // pinned staging of the request's words
    uint32_t *d_words = nullptr;     // device copy of the words
    svt_track *h_tracks = nullptr;   // mapped pinned host memory: the kernel writes the tracks here
    cudaEvent_t ev_h2d = nullptr;    // the words are on the device
    cudaEvent_t ev_ctrl = nullptr;   // control block (and so the tracks) in host memory
    int state = SLOT_FREE;
    uint64_t id = 0;
    uint64_t parent = 0;             // the split request this slot runs a chunk of (0 = none)
    unsigned chunk = 0;
    size_t n_tracks = 0;
    int status = SVT_OK;
    Clock::time_point t_submit;
};

struct Result {
    svt_server_result info;
    std::vector<svt_track> tracks;
};

// A request split into chunks: their results until the last one is done.
struct Parent {
    uint64_t id = 0;
    unsigned n_done = 0;
    std::vector<uint32_t> ev_base;                 // event index of each chunk's first event
    std::vector<int> status;                       // per chunk
    std::vector<std::vector<svt_track>> tracks;    // per chunk
    uint64_t n_events = 0, n_comb = 0;
    Clock::time_point t_submit;
};

}  // namespace

struct svt_server {
    int device = 0;
    svt_server_config cfg{};
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv_slot;   // a slot became free
    std::condition_variable cv_done;   // a result is ready
    std::deque<uint64_t> done_order;   // completed, not yet reported by svt_server_wait
    std::list<Result> results;         // completed, not yet taken
    std::list<Parent> parents;         // split requests with chunks in flight
    std::thread progress;
    std::atomic<bool> stop{false};
    uint64_t next_id = 1;
    unsigned in_flight = 0;
};

namespace {

// The last chunk of split request p is done: its joined result.  Called
// with s->mu held.
void publish_parent(svt_server *s, std::list<Parent>::iterator p)
{
    Result r;
    r.info.request_id = p->id;
    r.info.status = SVT_OK;
    for (int st : p->status)   // the first chunk that failed, in stream order
        if (st != SVT_OK) {
            r.info.status = st;
            break;
        }
    r.info.pad = 0;
    r.info.n_events = p->n_events;
    r.info.n_combinations = p->n_comb;
    if (r.info.status == SVT_OK) {
        size_t n = 0;
        for (const auto &t : p->tracks)
            n += t.size();
        r.tracks.reserve(n);
        for (size_t k = 0; k < p->tracks.size(); ++k)
            for (svt_track t : p->tracks[k]) {
                t.event += p->ev_base[k];
                r.tracks.push_back(t);
            }
    }
    r.info.n_tracks = r.tracks.size();
    r.info.latency_ns =
        (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - p->t_submit).count();
    s->results.push_back(std::move(r));
    s->done_order.push_back(p->id);
    s->parents.erase(p);
    s->cv_done.notify_all();
}

void finish(svt_server *s, Slot &sl, int status, size_t n_tracks)
{
    if (sl.parent) {   // a chunk of a split request
        const Ctrl &h = *sl.ctx->h_ctrl;
        std::vector<svt_track> tr;
        if (status == SVT_OK && n_tracks)
            tr.assign(sl.h_tracks, sl.h_tracks + n_tracks);
        if (h.flags & FLAG_TIMEOUT)
            sl.ctx->hash_dirty = true;
        std::lock_guard<std::mutex> lk(s->mu);
        for (auto it = s->parents.begin(); it != s->parents.end(); ++it)
            if (it->id == sl.parent) {
                it->status[sl.chunk] = status;
                it->tracks[sl.chunk] = std::move(tr);
                it->n_events += h.n_events;
                it->n_comb += h.n_comb;
                if (++it->n_done == it->status.size())
                    publish_parent(s, it);
                break;
            }
        sl.state = SLOT_FREE;
        sl.parent = 0;
        --s->in_flight;
        s->cv_slot.notify_all();
        return;
    }
    Result r;
    r.info.request_id = sl.id;
    r.info.status = status;
    r.info.pad = 0;
    r.info.n_tracks = status == SVT_OK ? n_tracks : 0;
    const Ctrl &h = *sl.ctx->h_ctrl;
    r.info.n_events = h.n_events;
    r.info.n_combinations = h.n_comb;
    r.info.latency_ns =
        (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - sl.t_submit).count();
    if (status == SVT_OK && n_tracks)
        r.tracks.assign(sl.h_tracks, sl.h_tracks + n_tracks);
    if (h.flags & FLAG_TIMEOUT)
        sl.ctx->hash_dirty = true;   // the batch may have stopped before clearing its table
    std::lock_guard<std::mutex> lk(s->mu);
    s->results.push_back(std::move(r));
    s->done_order.push_back(sl.id);
    sl.state = SLOT_FREE;
    --s->in_flight;
    s->cv_slot.notify_all();
    s->cv_done.notify_all();
}

// One pass over the slots; returns true if any slot advanced.
bool progress_once(svt_server *s)
{
    bool moved = false;
    for (Slot &sl : s->slots) {
        int state;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            state = sl.state;
        }
        if (state != SLOT_RUNNING)
            continue;
        const cudaError_t q = cudaEventQuery(sl.ev_ctrl);
        if (q == cudaErrorNotReady)
            continue;
        moved = true;
        if (q != cudaSuccess) {
            finish(s, sl, SVT_E_CUDA, 0);
            continue;
        }
        // the kernel wrote the tracks into the slot's mapped host buffer
        int st = ctx_status(sl.ctx);
        const size_t n = (size_t)sl.ctx->h_ctrl->n_out;
        if (st == SVT_OK && n > s->cfg.max_tracks)
            st = SVT_E_CAPACITY;
        finish(s, sl, st, st == SVT_OK ? n : 0);
    }
    return moved;
}

void progress_loop(svt_server *s)
{
    cudaSetDevice(s->device);
    while (!s->stop.load(std::memory_order_acquire)) {
        if (!progress_once(s)) {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->in_flight == 0)
                s->cv_slot.wait_for(lk, std::chrono::milliseconds(1));
            else {
                lk.unlock();
                std::this_thread::yield();
            }
        }
    }
}

void destroy_slots(svt_server *s)
{
    for (Slot &sl : s->slots) {
        if (sl.stream)
            cudaStreamSynchronize(sl.stream);
        if (sl.copy)
            cudaStreamSynchronize(sl.copy);
        if (sl.ev_ctrl)
            cudaEventDestroy(sl.ev_ctrl);
        if (sl.ev_h2d)
            cudaEventDestroy(sl.ev_h2d);
        if (sl.h_words)
            cudaFreeHost(sl.h_words);
        if (sl.h_tracks)
            cudaFreeHost(sl.h_tracks);
        if (sl.d_words)
            cudaFree(sl.d_words);
        if (sl.stream)
            cudaStreamDestroy(sl.stream);
        if (sl.copy)
            cudaStreamDestroy(sl.copy);
        if (sl.ctx)
            svt_destroy(sl.ctx);
        sl = Slot{};
    }
}

}  // namespace

extern "C" {

int svt_server_create(svt_server **out, int device, const svt_server_config *config,
                      const svt_const_set *sets, uint32_t n_sets, int64_t chi2_cut)
{
    if (!out)
        return SVT_E_INVAL;
    *out = nullptr;
    svt_server_config cfg = config ? *config : svt_server_config{};
    if (!cfg.ctas_per_sm) cfg.ctas_per_sm = 1;
    // by default a slot holds any stream of max_words words (a road has three
    // words at least), so only a request of more words is ever split
    if (!cfg.max_words) cfg.max_words = 1ull << 20;
    if (!cfg.max_events) cfg.max_events = (uint32_t)std::min<uint64_t>(cfg.max_words / 3 + 1, 1u << 30);
    if (!cfg.max_roads) cfg.max_roads = (uint32_t)std::min<uint64_t>(cfg.max_words / 3 + 1, 1u << 30);
    if (!cfg.max_tracks) cfg.max_tracks = 1ull << 20;
    if (!cfg.hash_slots) cfg.hash_slots = 1u << 20;
    if ((cfg.mode != SVT_PERSISTENT && cfg.mode != SVT_PLAIN) || cfg.n_slots > 64 ||
        cfg.max_words >= (1ull << 31) || cfg.max_tracks >= (1ull << 32) ||
        (cfg.hash_slots & (cfg.hash_slots - 1)))
        return SVT_E_INVAL;
    if (cudaSetDevice(device) != cudaSuccess)
        return SVT_E_CUDA;
    svt_server *s = new (std::nothrow) svt_server();
    if (!s)
        return SVT_E_INVAL;
    s->device = device;

    svt_limits lim{};
    lim.max_words = cfg.max_words;
    lim.max_events = cfg.max_events;
    lim.max_roads = cfg.max_roads;
    lim.max_tracks = cfg.max_tracks;
    lim.hash_slots = cfg.hash_slots;
    lim.max_combinations = cfg.mode == SVT_PLAIN ? (cfg.max_combinations ? cfg.max_combinations : 1ull << 24) : 1;
    cfg.max_combinations = lim.max_combinations;

    // admission by device memory: without an explicit slot count, take as
    // many slots as a quarter of the free memory holds (at least one)
    unsigned n_slots = cfg.n_slots;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete s;
        return SVT_E_CUDA;
    }
    int st = SVT_OK;
    s->slots.resize(n_slots ? n_slots : 1);
    for (size_t i = 0; i < s->slots.size() && st == SVT_OK; ++i) {
        Slot &sl = s->slots[i];
        size_t before = 0, after = 0, tot = 0;
        cudaMemGetInfo(&before, &tot);
        if ((st = svt_create(&sl.ctx, device, &lim)) != SVT_OK)
            break;
        if ((st = svt_load_constants(sl.ctx, sets, n_sets, chi2_cut, nullptr)) != SVT_OK)
            break;
        if ((st = ctx_prepare(sl.ctx, cfg.mode)) != SVT_OK)
            break;
        sl.ctx->blocks_per_sm = (int)cfg.ctas_per_sm;
        sl.ctx->max_ctas = (int)cfg.max_ctas;
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&sl.copy, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMallocHost(&sl.h_words, sizeof(uint32_t) * cfg.max_words) != cudaSuccess ||
            cudaHostAlloc(&sl.h_tracks, sizeof(svt_track) * cfg.max_tracks, cudaHostAllocMapped) != cudaSuccess ||
            cudaMalloc(&sl.d_words, sizeof(uint32_t) * cfg.max_words) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev_h2d, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev_ctrl, cudaEventDisableTiming) != cudaSuccess) {
            st = SVT_E_CUDA;
            break;
        }
        if ((st = svt_set_track_output(sl.ctx, sl.h_tracks, cfg.max_tracks)) != SVT_OK)   // written in place
            break;
        cudaMemGetInfo(&after, &tot);
        if (!n_slots && i == 0) {   // size the slot count from the first slot's footprint
            const size_t per = before > after ? before - after : 1;
            const size_t want = std::max<size_t>(1, std::min<size_t>(8, free_b / 4 / per));
            s->slots.resize(want);
        }
    }
    if (st != SVT_OK) {
        destroy_slots(s);
        delete s;
        return st;
    }
    cfg.n_slots = (uint32_t)s->slots.size();
    s->cfg = cfg;
    s->progress = std::thread(progress_loop, s);
    *out = s;
    return SVT_OK;
}

void svt_server_destroy(svt_server *s)
{
    if (!s)
        return;
    cudaSetDevice(s->device);
    {
        // wait for the requests in flight
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_slot.wait_for(lk, std::chrono::seconds(10), [s] { return s->in_flight == 0; });
    }
    s->stop.store(true, std::memory_order_release);
    s->cv_slot.notify_all();
    if (s->progress.joinable())
        s->progress.join();
    destroy_slots(s);
    delete s;
}

int svt_server_get_config(svt_server *s, svt_server_config *out)
{
    if (!s || !out)
        return SVT_E_INVAL;
    *out = s->cfg;
    return SVT_OK;
}

}  // extern "C"

namespace {

// EE and EP words among n (a loop the compiler vectorises).
void count_ends(const uint32_t *__restrict w, size_t n, size_t &ee, size_t &ep)
{
    uint64_t a = 0, b = 0;
    for (size_t i = 0; i < n; ++i) {
        a += w[i] >> 31;
        b += (w[i] >> 30) & 1u;
    }
    ee = a;
    ep = b;
}

// Admit one request or chunk to the first free slot (waiting for one) and
// enqueue its copy, kernel and control-block read.  parent != 0: chunk
// `chunk` of that split request.  A request (not a chunk) with more events or
// roads than the slot holds is not admitted: false (the slot is released).
bool admit(svt_server *s, const uint32_t *words, size_t n_words, uint64_t parent, unsigned chunk,
           Clock::time_point t0, uint64_t *id)
{
    Slot *sl = nullptr;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv_slot.wait(lk, [s, &sl] {
            for (Slot &x : s->slots)
                if (x.state == SLOT_FREE) {
                    sl = &x;
                    return true;
                }
            return false;
        });
        sl->state = SLOT_RESERVED;
        sl->id = parent ? 0 : s->next_id++;
        sl->parent = parent;
        sl->chunk = chunk;
        sl->t_submit = t0;
        ++s->in_flight;
    }
    s->cv_slot.notify_all();   // wakes an idle progress thread
    if (n_words)
        std::memcpy(sl->h_words, words, n_words * sizeof(uint32_t));
    // a road has three words at least: only a request of more than three
    // times the slot's event or road limit in words can exceed them
    size_t n_ee = 0, n_ep = 0;
    if (!parent && n_words > 3 * (size_t)std::min(s->cfg.max_events, s->cfg.max_roads))
        count_ends(sl->h_words, n_words, n_ee, n_ep);
    if (!parent && (n_ee > s->cfg.max_events || n_ep > s->cfg.max_roads)) {
        std::lock_guard<std::mutex> lk(s->mu);
        sl->state = SLOT_FREE;
        --s->in_flight;
        s->cv_slot.notify_all();
        return false;
    }
    if (id)
        *id = sl->id;
    int launches = 0;
    bool ok = cudaSetDevice(s->device) == cudaSuccess &&
              (!n_words || cudaMemcpyAsync(sl->d_words, sl->h_words, n_words * sizeof(uint32_t),
                                           cudaMemcpyHostToDevice, sl->copy) == cudaSuccess) &&
              cudaEventRecord(sl->ev_h2d, sl->copy) == cudaSuccess &&
              cudaStreamWaitEvent(sl->stream, sl->ev_h2d, 0) == cudaSuccess &&
              svt_unpack(sl->ctx, sl->d_words, n_words, sl->stream) == SVT_OK &&
              ctx_enqueue(sl->ctx, s->cfg.mode, sl->stream, &launches) == cudaSuccess &&
              cudaMemcpyAsync(sl->ctx->h_ctrl, sl->ctx->d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost,
                              sl->stream) == cudaSuccess &&
              cudaEventRecord(sl->ev_ctrl, sl->stream) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        std::memset(sl->ctx->h_ctrl, 0, sizeof(Ctrl));
        finish(s, *sl, SVT_E_CUDA, 0);   // the failure is the request's status
        return true;
    }
    sl->ctx->ran = true;
    sl->ctx->last_launches = launches;
    std::lock_guard<std::mutex> lk(s->mu);
    sl->state = SLOT_RUNNING;
    return true;
}

// Cut points of a request at event ends (EE words) into chunks of at most
// the slot's words, events and roads (EP words); the words after the last EE
// (a truncated event) go with the last chunk.  Empty if one event alone
// exceeds a slot.
std::vector<size_t> split_points(const svt_server_config &cfg, const uint32_t *w, size_t n)
{
    std::vector<size_t> cuts{0};   // chunk k: words [cuts[k], cuts[k + 1])
    size_t ev_start = 0, chunk_ev = 0, chunk_roads = 0, ev_roads = 0;
    for (size_t i = 0; i < n; ++i) {
        ev_roads += (w[i] >> 30) & 1u;
        if (!(w[i] >> 31) && i + 1 < n)
            continue;
        // an event ends at i (or the stream does)
        const size_t ev_end = i + 1, ev_words = ev_end - ev_start;
        if (ev_words > cfg.max_words || ev_roads > cfg.max_roads)
            return {};
        if (ev_end - cuts.back() > cfg.max_words || chunk_ev + 1 > cfg.max_events ||
            chunk_roads + ev_roads > cfg.max_roads) {
            cuts.push_back(ev_start);
            chunk_ev = 0;
            chunk_roads = 0;
        }
        ++chunk_ev;
        chunk_roads += ev_roads;
        ev_roads = 0;
        ev_start = ev_end;
    }
    cuts.push_back(n);
    return cuts;
}

}  // namespace

extern "C" {

int svt_server_submit(svt_server *s, const uint32_t *words, size_t n_words, uint64_t *request_id)
{
    if (!s || !request_id || (n_words && !words))
        return SVT_E_INVAL;
    *request_id = 0;
    const Clock::time_point t0 = Clock::now();
    // the usual case: the request fits a slot (its words are counted as they
    // are copied to the slot's staging buffer)
    if (n_words <= s->cfg.max_words && admit(s, words, n_words, 0, 0, t0, request_id))
        return SVT_OK;
    // larger than a slot: chunks at event boundaries
    const std::vector<size_t> cuts = split_points(s->cfg, words, n_words);
    if (cuts.size() < 2)
        return SVT_E_CAPACITY;   // one event alone exceeds a slot
    const unsigned n_chunks = (unsigned)(cuts.size() - 1);
    uint64_t pid;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        pid = s->next_id++;
        Parent p;
        p.id = pid;
        p.status.assign(n_chunks, SVT_OK);
        p.tracks.resize(n_chunks);
        p.t_submit = t0;
        uint32_t ev = 0;
        for (unsigned k = 0; k < n_chunks; ++k) {
            p.ev_base.push_back(ev);
            for (size_t i = cuts[k]; i < cuts[k + 1]; ++i)
                ev += words[i] >> 31;
        }
        s->parents.push_back(std::move(p));
    }
    *request_id = pid;
    for (unsigned k = 0; k < n_chunks; ++k)
        admit(s, words + cuts[k], cuts[k + 1] - cuts[k], pid, k, t0, nullptr);
    return SVT_OK;
}

int svt_server_wait(svt_server *s, int64_t timeout_us, svt_server_result *out)
{
    if (!s || !out)
        return SVT_E_INVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [s] { return !s->done_order.empty(); };
    if (timeout_us < 0)
        s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready))
        return SVT_E_TIMEOUT;
    const uint64_t id = s->done_order.front();
    s->done_order.pop_front();
    for (const Result &r : s->results)
        if (r.info.request_id == id) {
            *out = r.info;
            return SVT_OK;
        }
    return SVT_E_STATE;
}

int svt_server_take(svt_server *s, uint64_t request_id, svt_track *out, size_t cap, size_t *n_out)
{
    if (!s || !n_out)
        return SVT_E_INVAL;
    *n_out = 0;
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto it = s->results.begin(); it != s->results.end(); ++it) {
        if (it->info.request_id != request_id)
            continue;
        const size_t n = it->tracks.size();
        *n_out = n;
        if (n > cap)
            return SVT_E_CAPACITY;
        if (n && !out)
            return SVT_E_INVAL;
        if (n)
            std::memcpy(out, it->tracks.data(), n * sizeof(svt_track));
        s->results.erase(it);
        return SVT_OK;
    }
    return SVT_E_STATE;
}

}  // extern "C"
