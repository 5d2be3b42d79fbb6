// svt_api.cu -- the C ABI (include/svt.h): context, buffers, status, launches.
#include "svt_ctx.h"

#include <algorithm>
#include <cstdlib>
#include <vector>
#include <cstring>
#include <new>

using namespace svt;

static_assert(sizeof(svt_const_set) == 96, "svt_const_set layout");
static_assert(sizeof(svt_track) == 40, "svt_track layout");
static_assert(sizeof(svt_road) == 100, "svt_road layout");
static_assert(sizeof(RoadRec) == 16, "RoadRec layout");


namespace {

template <class T>
cudaError_t dalloc(svt_ctx *c, T **p, size_t count)
{
    void *q = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0)
        bytes = 16;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess)
        return e;
    c->allocs[c->n_allocs++] = q;
    *p = static_cast<T *>(q);
    return cudaSuccess;
}

void free_all(svt_ctx *c)
{
    for (int i = 0; i < c->n_allocs; ++i)
        cudaFree(c->allocs[i]);
    c->n_allocs = 0;
    if (c->h_ctrl)
        cudaFreeHost(c->h_ctrl);
    c->h_ctrl = nullptr;
    if (c->gexec)
        cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
}

void drop_graph(svt_ctx *c)
{
    if (c->gexec)
        cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->g_mode = -1;
}

int read_ctrl(svt_ctx *c, cudaStream_t s)
{
    if (cudaMemcpyAsync(c->h_ctrl, c->d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SVT_E_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return SVT_E_CUDA;
    if (c->h_ctrl->flags & FLAG_TIMEOUT)
        c->hash_dirty = true;   // the batch may have stopped before clearing the table
    return SVT_OK;
}

int ensure_plain_buffers(svt_ctx *c)
{
    if (c->d.fit_key)
        return SVT_OK;
    if (dalloc(c, &c->d.fit_key, c->d.max_combs) || dalloc(c, &c->d.fit_p, c->d.max_combs * 3))
        return SVT_E_CUDA;
    return SVT_OK;
}

// Clear the group table on s if a batch stopped before leaving it empty.
cudaError_t clear_if_dirty(svt_ctx *c, cudaStream_t s)
{
    if (!c->hash_dirty)
        return cudaSuccess;
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->d.hash, 0, sizeof(HashSlot) * (size_t)(c->d.hash_mask + 1), s)) ||
        (e = cudaMemsetAsync(c->d.hash_bits, 0, sizeof(uint32_t) * (c->d.hash_mask / 32 + 1), s)))
        return e;
    c->hash_dirty = false;
    return cudaSuccess;
}

// enqueue one batch (ctrl reset + kernels) on s
cudaError_t enqueue(svt_ctx *c, int mode, cudaStream_t s, int *launches)
{
    Dev d = c->d;
    d.wait_ns = c->wait_ns;
    d.skip_arrival = mode == SVT_PERSISTENT ? c->skip_arrival : 0;
    cudaError_t e = cudaMemsetAsync(c->d.ctrl, 0, sizeof(Ctrl), s);
    if (e || (e = clear_if_dirty(c, s)))
        return e;
    if (mode == SVT_PLAIN) {
        if ((e = launch_unpack_plain(d, s, launches)))
            return e;
        return launch_fit_plain(d, s, launches);
    }
    c->skip_arrival = 0;   // the test hook holds for one persistent launch
    return launch_persistent(c->block, d, s, c->blocks_per_sm, c->max_ctas, launches);
}

}  // namespace

namespace svt {
cudaError_t ctx_enqueue(svt_ctx *c, int mode, cudaStream_t s, int *launches)
{
    return enqueue(c, mode, s, launches);
}
int ctx_status(const svt_ctx *c) { return status_of(*c->h_ctrl); }
int ctx_prepare(svt_ctx *c, int mode) { return mode == SVT_PLAIN ? ensure_plain_buffers(c) : SVT_OK; }
}  // namespace svt

extern "C" {

const char *svt_strerror(int code)
{
    switch (code) {
    case SVT_OK: return "ok";
    case SVT_E_INVAL: return "invalid argument";
    case SVT_E_BADWORD: return "malformed input word";
    case SVT_E_TRUNCATED: return "input does not end at an event boundary";
    case SVT_E_LIMIT: return "more than 8 hits on a layer or 256 roads in an event";
    case SVT_E_CAPACITY: return "batch exceeds the context or buffer capacity";
    case SVT_E_CUDA: return "CUDA runtime error";
    case SVT_E_TIMEOUT: return "device-side wait timed out";
    case SVT_E_STATE: return "call out of order";
    default: return "unknown status";
    }
}

int svt_create(svt_ctx **out, int device, const svt_limits *lim)
{
    if (!out)
        return SVT_E_INVAL;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess)
        return SVT_E_CUDA;
    svt_ctx *c = new (std::nothrow) svt_ctx();
    if (!c)
        return SVT_E_INVAL;
    c->device = device;
    svt_limits L = lim ? *lim : svt_limits{};
    if (!L.max_words) L.max_words = 1ull << 24;
    if (!L.max_events) L.max_events = 1u << 16;
    if (!L.max_roads) L.max_roads = 1u << 20;
    if (!L.max_tracks) L.max_tracks = 1ull << 22;
    if (!L.hash_slots) L.hash_slots = 1u << 22;
    if (!L.max_combinations) L.max_combinations = 1ull << 26;
    if ((L.hash_slots & (L.hash_slots - 1)) || L.max_words >= (1ull << 31) ||
        L.max_tracks >= (1ull << 32)) {
        delete c;
        return SVT_E_INVAL;
    }
    c->lim = L;
    Dev &d = c->d;
    d.max_events = L.max_events;
    d.max_roads = L.max_roads;
    d.max_chunks_r = (L.max_roads + ROAD_CHUNK - 1) / ROAD_CHUNK;
    d.max_tracks = L.max_tracks;
    d.max_combs = L.max_combinations;
    d.hash_mask = L.hash_slots - 1;
    d.small_n4 = N4_SMALL_MAX;
    d.run_roads = WARP_ROADS;
    bool ok =
        !dalloc(c, &d.ctrl, 1) && !dalloc(c, const_cast<svt_const_set **>(&d.consts), N_SETS) &&
        !dalloc(c, &d.span_ee, MAX_SPANS + MAX_GRID) && !dalloc(c, &d.span_ep, MAX_SPANS + MAX_GRID) &&
        !dalloc(c, &d.span_seg, MAX_SPANS + MAX_GRID) && !dalloc(c, &d.ev_road_end, L.max_events) && !dalloc(c, &d.ev_big, L.max_events) &&
        !dalloc(c, &d.roads, L.max_roads) && !dalloc(c, &d.coords, (size_t)L.max_roads * 40) &&
        !dalloc(c, &d.xmask, L.max_roads) && !dalloc(c, &d.big_list, L.max_roads) &&
        !dalloc(c, &d.cand_bits, L.max_roads / 32 + 1) && !dalloc(c, &d.fitc, N_SETS * SET_INT4) &&
        !dalloc(c, &d.surv_pool, (size_t)L.max_roads * SURV_SLOTS) &&
        !dalloc(c, &d.surv_cnt, L.max_roads) &&
        !dalloc(c, &d.rchunk_sum, d.max_chunks_r) && !dalloc(c, &d.rchunk_off, d.max_chunks_r) &&
        !dalloc(c, &d.cchunk_sum, d.max_chunks_r) && !dalloc(c, &d.cchunk_off, d.max_chunks_r) &&
        !dalloc(c, &d.hash, L.hash_slots) && !dalloc(c, &d.hash_bits, L.hash_slots / 32 + 1) &&
        !dalloc(c, &d.comb_off, L.max_roads) && !dalloc(c, &d.tracks, L.max_tracks) &&
        cudaMallocHost(&c->h_ctrl, sizeof(Ctrl)) == cudaSuccess &&
        cudaMemset(d.hash, 0, sizeof(HashSlot) * (size_t)L.hash_slots) == cudaSuccess &&
        cudaMemset(d.hash_bits, 0, sizeof(uint32_t) * (L.hash_slots / 32 + 1)) == cudaSuccess &&
        cudaMemset(d.ctrl, 0, sizeof(Ctrl)) == cudaSuccess && cudaDeviceSynchronize() == cudaSuccess;
    c->dev_tracks = d.tracks;
    if (!ok) {
        free_all(c);
        delete c;
        return SVT_E_CUDA;
    }
    *out = c;
    return SVT_OK;
}

void svt_destroy(svt_ctx *c)
{
    if (!c)
        return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    free_all(c);
    delete c;
}

int svt_load_constants(svt_ctx *c, const svt_const_set *sets, uint32_t n_sets, int64_t cut,
                       void *stream)
{
    if (!c || !sets || n_sets != (uint32_t)N_SETS || cut < 0 || !constants_admissible(sets))
        return SVT_E_INVAL;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int32_t> fw((size_t)N_SETS * SET_INT4 * 4);
    fit_words(sets, fw.data());
    if (cudaSetDevice(c->device) ||
        cudaMemcpyAsync(const_cast<svt_const_set *>(c->d.consts), sets, sizeof(svt_const_set) * N_SETS,
                        cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(c->d.fitc, fw.data(), sizeof(int32_t) * fw.size(), cudaMemcpyHostToDevice, s) ||
        cudaStreamSynchronize(s))
        return SVT_E_CUDA;
    c->d.cut = cut;
    c->consts_loaded = true;
    drop_graph(c);
    return SVT_OK;
}

// The device's address of `p`: itself for device (or managed) memory, the
// mapped alias for page-locked host memory; nullptr for memory the device
// cannot address (pageable host memory) or on error.
static const void *device_view(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)
        return p;
    if (a.type == cudaMemoryTypeHost)
        return a.devicePointer;
    return nullptr;
}

int svt_unpack(svt_ctx *c, const uint32_t *d_words, size_t n_words, void *stream)
{
    (void)stream;
    if (!c || (n_words && !d_words) || ((uintptr_t)d_words & 3u))
        return SVT_E_INVAL;
    if (n_words > c->lim.max_words)
        return SVT_E_CAPACITY;
    if (n_words) {
        d_words = static_cast<const uint32_t *>(device_view(d_words));
        if (!d_words)
            return SVT_E_INVAL;
    }
    c->d.words = d_words;
    c->d.n_words = n_words;
    c->bound = true;
    c->roads_valid = false;
    c->ran = false;
    return SVT_OK;
}

int svt_fit_events(svt_ctx *c, int mode, void *stream)
{
    if (!c || (mode != SVT_PLAIN && mode != SVT_PERSISTENT))
        return SVT_E_INVAL;
    if (!c->consts_loaded || !c->bound)
        return SVT_E_STATE;
    if (cudaSetDevice(c->device))
        return SVT_E_CUDA;
    if (mode == SVT_PLAIN && ensure_plain_buffers(c))
        return SVT_E_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int launches = 0;
    cudaError_t e;
    // A batch that stopped early (a barrier timeout) may have left entries
    // in the group table: it is cleared here, outside any graph, so a
    // replayed graph never skips the clear and a captured one never holds it.
    if ((e = clear_if_dirty(c, s)))
        return SVT_E_CUDA;
    // the test hook of svt_debug_wait runs one direct launch, never a graph
    if (c->use_graph && s != nullptr && !(mode == SVT_PERSISTENT && c->skip_arrival)) {
        bool hit = c->gexec && c->g_mode == mode && c->g_words == c->d.words && c->g_n == c->d.n_words &&
                   c->g_stream == s;
        if (!hit) {
            drop_graph(c);
            cudaGraph_t graph = nullptr;
            if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)))
                return SVT_E_CUDA;
            int nl = 0;
            cudaError_t ee = enqueue(c, mode, s, &nl);
            e = cudaStreamEndCapture(s, &graph);
            if (ee || e || !graph) {
                if (graph)
                    cudaGraphDestroy(graph);
                cudaGetLastError();
                return SVT_E_CUDA;
            }
            e = cudaGraphInstantiate(&c->gexec, graph, 0);
            cudaGraphDestroy(graph);
            if (e) {
                c->gexec = nullptr;
                cudaGetLastError();
                return SVT_E_CUDA;
            }
            c->g_mode = mode;
            c->g_words = c->d.words;
            c->g_n = c->d.n_words;
            c->g_stream = s;
            c->g_launches = nl;
        }
        e = cudaGraphLaunch(c->gexec, s);
        launches = c->g_launches;
    } else {
        e = enqueue(c, mode, s, &launches);
    }
    if (e)
        return SVT_E_CUDA;
    c->last_launches = launches;
    c->ran = true;
    c->roads_valid = true;
    return SVT_OK;
}

int svt_set_track_output(svt_ctx *c, svt_track *host, size_t cap)
{
    if (!c || (host && (!cap || ((uintptr_t)host & 7u))))
        return SVT_E_INVAL;
    svt_track *dev = c->dev_tracks;
    size_t n = c->lim.max_tracks;
    if (host) {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, host) != cudaSuccess || a.type != cudaMemoryTypeHost ||
            !a.devicePointer) {
            cudaGetLastError();
            return SVT_E_INVAL;
        }
        dev = static_cast<svt_track *>(a.devicePointer);
        n = std::min(n, cap);
    }
    c->d.tracks = dev;
    c->d.max_tracks = n;
    c->host_out = host;
    c->last_n_out = 0;
    drop_graph(c);
    return SVT_OK;
}

int svt_get_tracks(svt_ctx *c, svt_track *out, size_t cap, size_t *n_out, void *stream)
{
    if (!c || !n_out)
        return SVT_E_INVAL;
    *n_out = 0;
    if (!c->ran)
        return SVT_E_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaSetDevice(c->device))
        return SVT_E_CUDA;
    // The status block and, speculatively, as many tracks as the previous
    // batch had go out together, so a batch like the one before takes one
    // synchronisation; the rest (if any) follows once the count is known.
    // With a host output buffer the tracks are there already: `out` equal to
    // it takes no copy.
    const bool in_place = c->host_out && out == c->host_out;
    const svt_track *src = c->host_out ? c->host_out : c->d.tracks;
    const size_t spec = out && !in_place ? std::min(cap, (size_t)c->last_n_out) : 0;
    if (cudaMemcpyAsync(c->h_ctrl, c->d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s) ||
        (spec && cudaMemcpyAsync(out, src, spec * sizeof(svt_track), cudaMemcpyDefault, s)) ||
        cudaStreamSynchronize(s))
        return SVT_E_CUDA;
    if (c->h_ctrl->flags & FLAG_TIMEOUT)
        c->hash_dirty = true;   // the batch may have stopped before clearing the table
    int st = status_of(*c->h_ctrl);
    if (st)
        return st;
    size_t n = (size_t)c->h_ctrl->n_out;
    *n_out = n;
    c->last_n_out = n;
    if (n > cap)
        return SVT_E_CAPACITY;
    if (in_place)
        return SVT_OK;
    if (n > spec && (!out || cudaMemcpyAsync(out + spec, src + spec, (n - spec) * sizeof(svt_track),
                                             cudaMemcpyDefault, s) ||
                     cudaStreamSynchronize(s)))
        return out ? SVT_E_CUDA : SVT_E_INVAL;
    return SVT_OK;
}

int svt_get_roads(svt_ctx *c, svt_road *out, size_t cap, size_t *n_out, void *stream)
{
    if (!c || !n_out)
        return SVT_E_INVAL;
    *n_out = 0;
    if (!c->bound)
        return SVT_E_STATE;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaSetDevice(c->device))
        return SVT_E_CUDA;
    if (!c->roads_valid) {
        int nl = 0;
        Dev d = c->d;
        if (cudaMemsetAsync(c->d.ctrl, 0, sizeof(Ctrl), s) || launch_unpack_plain(d, s, &nl))
            return SVT_E_CUDA;
        c->roads_valid = true;
    }
    if (!c->d.road_out && dalloc(c, &c->d.road_out, c->lim.max_roads))
        return SVT_E_CUDA;
    if (launch_export_roads(c->d, s) || read_ctrl(c, s))
        return SVT_E_CUDA;
    const Ctrl &h = *c->h_ctrl;
    int st = status_of(h);
    if (st)
        return st;
    size_t n = h.n_roads;
    *n_out = n;
    if (n > cap)
        return SVT_E_CAPACITY;
    if (n && (!out || cudaMemcpyAsync(out, c->d.road_out, n * sizeof(svt_road), cudaMemcpyDefault, s) ||
              cudaStreamSynchronize(s)))
        return out ? SVT_E_CUDA : SVT_E_INVAL;
    return SVT_OK;
}

int svt_get_stats(svt_ctx *c, svt_stats *out, void *stream)
{
    if (!c || !out)
        return SVT_E_INVAL;
    if (cudaSetDevice(c->device) || read_ctrl(c, (cudaStream_t)stream))
        return SVT_E_CUDA;
    const Ctrl &h = *c->h_ctrl;
    std::memset(out, 0, sizeof *out);
    out->n_events = h.n_events;
    out->n_roads = h.n_roads;
    out->n_combinations = h.n_comb;
    out->n_passing = h.n_pass;
    out->n_tracks = h.n_out;
    out->status = status_of(h);
    out->n_groups = h.hash_used;
    out->error_word = h.err_inv ? (~h.err_inv) >> 8 : 0ull;
    for (int k = 0; k < 6; ++k) {
        const unsigned long long t0 = h.t_phase[k], t1 = h.t_phase[k + 1];
        out->phase_ns[k] = (t0 && t1 && t1 >= t0) ? t1 - t0 : 0ull;
    }
    return SVT_OK;
}

static bool launch_ok(const svt_launch &L)
{
    return (L.block == 0 || persistent_block_ok(L.block)) && L.blocks_per_sm >= 0 && L.small_n4 >= 0 &&
           L.small_n4 <= N4_SMALL_MAX && (L.run_roads == 0 || L.run_roads == 4 || L.run_roads == 8 ||
                                          L.run_roads == RUN_ROADS_MAX) && L.max_ctas >= 0;
}

static void apply_launch(svt_ctx *c, const svt_launch &L)
{
    c->block = L.block ? L.block : 256;
    c->blocks_per_sm = L.blocks_per_sm;
    c->d.small_n4 = L.small_n4 ? L.small_n4 : N4_SMALL_MAX;
    c->d.run_roads = L.run_roads ? L.run_roads : WARP_ROADS;
    c->max_ctas = L.max_ctas;
}

static svt_launch current_launch(const svt_ctx *c)
{
    return svt_launch{c->block, c->blocks_per_sm, c->d.small_n4, c->d.run_roads, c->max_ctas};
}

int svt_set_launch(svt_ctx *c, const svt_launch *cfg)
{
    if (!c || !cfg || !launch_ok(*cfg))
        return SVT_E_INVAL;
    apply_launch(c, *cfg);
    drop_graph(c);
    return SVT_OK;
}

int svt_get_launch(svt_ctx *c, svt_launch *out)
{
    if (!c || !out)
        return SVT_E_INVAL;
    *out = current_launch(c);
    if (out->blocks_per_sm == 0) {
        if (cudaSetDevice(c->device))
            return SVT_E_CUDA;
        out->blocks_per_sm = persistent_max_blocks_per_sm(c->block, c->device);
    }
    return SVT_OK;
}

int svt_autotune(svt_ctx *c, int reps, svt_tune_point *points, uint32_t cap, uint32_t *n_points,
                 void *stream)
{
    if (!c || reps < 1 || (cap && !points))
        return SVT_E_INVAL;
    if (n_points)
        *n_points = 0;
    if (!c->consts_loaded || !c->bound)
        return SVT_E_STATE;
    if (cudaSetDevice(c->device))
        return SVT_E_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    static const int kSmall[] = {64, 128, N4_SMALL_MAX};
    static const int kRun[] = {4, WARP_ROADS, RUN_ROADS_MAX};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) || cudaEventCreate(&e1))
        return SVT_E_CUDA;
    const svt_launch old = current_launch(c);
    svt_launch best_cfg = old;
    int st = SVT_OK;
    float best = 0.f;
    uint32_t n = 0;
    std::vector<float> t(reps);
    for (int block : PERSISTENT_BLOCKS) {
        const int maxb = persistent_max_blocks_per_sm(block, c->device);
        if (maxb <= 0) {
            st = SVT_E_CUDA;
            break;
        }
        for (int bps = 1; bps <= maxb && st == SVT_OK; ++bps)
            for (int small : kSmall)
                for (int run : kRun) {
                    if (st != SVT_OK)
                        break;
                    const svt_launch L{block, bps, small, run, old.max_ctas};
                    apply_launch(c, L);
                    int nl = 0;
                    if (enqueue(c, SVT_PERSISTENT, s, &nl) || read_ctrl(c, s)) {   // warm-up
                        st = SVT_E_CUDA;
                        break;
                    }
                    if ((st = status_of(*c->h_ctrl)) != SVT_OK)
                        break;
                    for (int r = 0; r < reps && st == SVT_OK; ++r) {
                        if (cudaEventRecord(e0, s) || enqueue(c, SVT_PERSISTENT, s, &nl) ||
                            cudaEventRecord(e1, s) || cudaEventSynchronize(e1) ||
                            cudaEventElapsedTime(&t[r], e0, e1))
                            st = SVT_E_CUDA;
                    }
                    if (st != SVT_OK)
                        break;
                    std::sort(t.begin(), t.end());
                    const float med = t[reps / 2];
                    if (n < cap)
                        points[n] = svt_tune_point{L, med};
                    ++n;
                    if (best == 0.f || med < best) {
                        best = med;
                        best_cfg = L;
                    }
                }
        if (st != SVT_OK)
            break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    apply_launch(c, st == SVT_OK ? best_cfg : old);
    drop_graph(c);
    if (n_points)
        *n_points = n;
    return st != SVT_OK ? st : n > cap && cap ? SVT_E_CAPACITY : SVT_OK;
}

int svt_use_graph(svt_ctx *c, int enable)
{
    if (!c)
        return SVT_E_INVAL;
    c->use_graph = enable != 0;
    if (!c->use_graph)
        drop_graph(c);
    return SVT_OK;
}

int svt_debug_wait(svt_ctx *c, uint32_t wait_limit_us, int skip_arrival)
{
    if (!c)
        return SVT_E_INVAL;
    if (skip_arrival < 0 || skip_arrival > 2)
        return SVT_E_INVAL;
    const unsigned long long w = wait_limit_us ? (unsigned long long)wait_limit_us * 1000ull : 2000000000ull;
    if (w != c->wait_ns)
        drop_graph(c);   // the wait limit is a kernel argument a graph holds
    c->wait_ns = w;
    c->skip_arrival = skip_arrival;   // never captured: the hook's launch is a direct one
    return SVT_OK;
}

int svt_last_launch_count(svt_ctx *c) { return c ? c->last_launches : 0; }

}  // extern "C"
