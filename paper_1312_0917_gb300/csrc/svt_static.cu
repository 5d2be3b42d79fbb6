// svt_static.cu -- svt_run_static: the whole chain on one batch with no
// allocation at call time.
//
// Some callers cannot allocate device memory when a batch arrives: a process
// whose free device memory is already owned by another allocator (a caching
// allocator that holds the pool, or a budget fixed at start-up), and trigger
// paths where an allocation's latency or failure is not acceptable.  For them
// this entry point runs the persistent kernel over a scratch arena that is a
// file-scope __device__ array of fixed size (ARENA_BYTES), placed by the
// module loader, and writes the tracks into the caller's buffer.
//
// Every call looks up the arena's address with cudaGetSymbolAddress on the
// current device (cheap, and it follows a re-created primary context); the
// first call on a device, and the first after the address changed, clears
// its group table.  There is one arena per device: calls that overlap in time
// (two host threads, or two streams with work in flight) race on it.
#include "svt_ctx.h"

#include <vector>
#include <mutex>

using namespace svt;

namespace {

// limits of one batch in the arena
constexpr unsigned long long S_WORDS = 1ull << 17;
constexpr unsigned S_EVENTS = 1u << 10;
constexpr unsigned S_ROADS = 1u << 13;
constexpr unsigned S_HASH = 1u << 15;
constexpr unsigned S_CHUNKS_R = (S_ROADS + ROAD_CHUNK - 1) / ROAD_CHUNK;

constexpr size_t up256(size_t b) { return (b + 255) / 256 * 256; }

// byte offsets of the arena's regions
constexpr size_t OFF_CTRL = 0;
constexpr size_t OFF_CONSTS = OFF_CTRL + up256(sizeof(Ctrl));
constexpr unsigned S_SPANS = MAX_SPANS + MAX_GRID;   // per-warp word spans, then per-CTA totals
constexpr size_t OFF_SPAN = OFF_CONSTS + up256(sizeof(svt_const_set) * N_SETS);    // 3 x [S_SPANS] u32
constexpr size_t OFF_EV = OFF_SPAN + up256(3 * sizeof(uint32_t) * S_SPANS);         // 2 x [S_EVENTS] u32
constexpr size_t OFF_ROADS = OFF_EV + up256(2 * sizeof(uint32_t) * S_EVENTS);
constexpr size_t OFF_COORDS = OFF_ROADS + up256(sizeof(RoadRec) * S_ROADS);
constexpr size_t OFF_XMASK = OFF_COORDS + up256(sizeof(uint16_t) * 40 * S_ROADS);
constexpr size_t OFF_BIG = OFF_XMASK + up256(sizeof(unsigned long long) * S_ROADS);
constexpr size_t OFF_CAND = OFF_BIG + up256(sizeof(uint32_t) * S_ROADS);
constexpr size_t OFF_FITC = OFF_CAND + up256(sizeof(uint32_t) * (S_ROADS / 32 + 1));
constexpr size_t OFF_SURV = OFF_FITC + up256(sizeof(int4) * SET_INT4 * N_SETS);
constexpr size_t OFF_SCNT = OFF_SURV + up256(sizeof(unsigned long long) * SURV_SLOTS * S_ROADS);
constexpr size_t OFF_RCH = OFF_SCNT + up256(S_ROADS);                                 // 2 x [S_CHUNKS_R] u32
constexpr size_t OFF_CCH = OFF_RCH + up256(2 * sizeof(uint32_t) * S_CHUNKS_R);       // 2 x [S_CHUNKS_R] u64
constexpr size_t OFF_HASH = OFF_CCH + up256(2 * sizeof(unsigned long long) * S_CHUNKS_R);
constexpr size_t OFF_HUSED = OFF_HASH + up256(sizeof(HashSlot) * S_HASH);
constexpr size_t ARENA_BYTES = OFF_HUSED + up256(sizeof(uint32_t) * (S_HASH / 32 + 1));
static_assert(ARENA_BYTES < (8u << 20), "the static arena stays modest (under 8 MB)");

}  // namespace

// The arena.  The first call on a device clears its group table; the kernel
// leaves the table empty after every batch that completes.
static __device__ __align__(256) unsigned char g_arena[ARENA_BYTES];

namespace {

struct DeviceArena {
    unsigned char *base = nullptr;   // the arena's address when the table was last known empty
    bool hash_dirty = true;          // clear the group table before the next batch
};

std::mutex g_mu;
DeviceArena g_dev[64];

}  // namespace

extern "C" int svt_run_static(const uint32_t *d_words, size_t n_words, const svt_const_set *sets,
                              uint32_t n_sets, int64_t chi2_cut, svt_track *d_tracks, size_t cap,
                              size_t *n_out, void *stream)
{
    if (n_out)
        *n_out = 0;
    if (!n_out || !sets || n_sets != (uint32_t)N_SETS || chi2_cut < 0 || (n_words && !d_words) ||
        ((uintptr_t)d_words & 3u) || (cap && !d_tracks) || ((uintptr_t)d_tracks & 7u))
        return SVT_E_INVAL;
    if (n_words > S_WORDS)
        return SVT_E_CAPACITY;
    if (!constants_admissible(sets))
        return SVT_E_INVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return SVT_E_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    // the call waits for its batch, which a stream being captured cannot do
    cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap_st) != cudaSuccess)
        return SVT_E_CUDA;
    if (cap_st != cudaStreamCaptureStatusNone)
        return SVT_E_INVAL;

    DeviceArena *da = &g_dev[dev];
    unsigned char *b = nullptr;
    {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_arena) != cudaSuccess || !p)
            return SVT_E_CUDA;
        b = static_cast<unsigned char *>(p);
        std::lock_guard<std::mutex> lk(g_mu);
        if (da->base != b) {   // first call on this device, or a new context: table state unknown
            da->base = b;
            da->hash_dirty = true;
        }
    }
    Dev d{};
    d.ctrl = reinterpret_cast<Ctrl *>(b + OFF_CTRL);
    d.consts = reinterpret_cast<const svt_const_set *>(b + OFF_CONSTS);
    d.words = d_words;
    d.n_words = n_words;
    d.max_events = S_EVENTS;
    d.max_roads = S_ROADS;
    d.max_chunks_r = S_CHUNKS_R;
    d.max_tracks = cap;
    d.max_combs = 0;
    uint32_t *span = reinterpret_cast<uint32_t *>(b + OFF_SPAN);
    d.span_ee = span;
    d.span_ep = span + S_SPANS;
    d.span_seg = span + 2 * S_SPANS;
    d.ev_road_end = reinterpret_cast<uint32_t *>(b + OFF_EV);
    d.ev_big = d.ev_road_end + S_EVENTS;
    d.roads = reinterpret_cast<RoadRec *>(b + OFF_ROADS);
    d.coords = reinterpret_cast<uint16_t *>(b + OFF_COORDS);
    d.xmask = reinterpret_cast<unsigned long long *>(b + OFF_XMASK);
    d.big_list = reinterpret_cast<uint32_t *>(b + OFF_BIG);
    d.cand_bits = reinterpret_cast<uint32_t *>(b + OFF_CAND);
    d.fitc = reinterpret_cast<int4 *>(b + OFF_FITC);
    d.surv_pool = reinterpret_cast<unsigned long long *>(b + OFF_SURV);
    d.surv_cnt = reinterpret_cast<uint8_t *>(b + OFF_SCNT);
    uint32_t *rch = reinterpret_cast<uint32_t *>(b + OFF_RCH);
    d.rchunk_sum = rch;
    d.rchunk_off = rch + S_CHUNKS_R;
    unsigned long long *cch = reinterpret_cast<unsigned long long *>(b + OFF_CCH);
    d.cchunk_sum = cch;
    d.cchunk_off = cch + S_CHUNKS_R;
    d.hash = reinterpret_cast<HashSlot *>(b + OFF_HASH);
    d.hash_bits = reinterpret_cast<uint32_t *>(b + OFF_HUSED);
    d.hash_mask = S_HASH - 1;
    d.tracks = d_tracks;
    d.cut = chi2_cut;
    d.small_n4 = N4_SMALL_MAX;
    d.run_roads = WARP_ROADS;
    d.wait_ns = 2000000000ull;

    // what must start at zero: the control block every batch, the group
    // table on the first batch and after one that did not finish
    int launches = 0;
    std::vector<int32_t> fw((size_t)N_SETS * SET_INT4 * 4);   // lives until the stream is synchronized below
    fit_words(sets, fw.data());
    if (cudaMemcpyAsync(b + OFF_CONSTS, sets, sizeof(svt_const_set) * N_SETS, cudaMemcpyHostToDevice, s) ||
        cudaMemcpyAsync(d.fitc, fw.data(), sizeof(int32_t) * fw.size(), cudaMemcpyHostToDevice, s) ||
        cudaMemsetAsync(d.ctrl, 0, sizeof(Ctrl), s) ||
        (da->hash_dirty && (cudaMemsetAsync(d.hash, 0, sizeof(HashSlot) * S_HASH, s) ||
                            cudaMemsetAsync(d.hash_bits, 0, sizeof(uint32_t) * (S_HASH / 32 + 1), s))) ||
        launch_persistent(256, d, s, 0, 0, &launches))
        return SVT_E_CUDA;
    Ctrl h;
    if (cudaMemcpyAsync(&h, d.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s) || cudaStreamSynchronize(s))
        return SVT_E_CUDA;
    da->hash_dirty = (h.flags & FLAG_TIMEOUT) != 0;
    const int st = status_of(h);
    // with SVT_E_CAPACITY, the survivors when they did not fit `cap`; 0 when
    // an arena limit (events, roads, group table) was exceeded
    if (st == SVT_OK || (st == SVT_E_CAPACITY && h.n_out > cap))
        *n_out = (size_t)h.n_out;
    return st;
}
