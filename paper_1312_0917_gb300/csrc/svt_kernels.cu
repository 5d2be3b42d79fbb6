// svt_kernels.cu -- sm_103a kernels of the SVT track-fitting chain.
//
// Stages (arXiv:1312.0917, Sec. II-A: unpack, combine, fit), followed by the
// chi-square cut and the hit-warrior:
//
//   P0  word spans (one per warp): count EE / EP words, check every word's fields
//   P1  word spans: decode the roads whose header lies in the span (header,
//       XFT track, hits ranked per layer), enforce the grammar and limits
//   P2  events: flag the hits a road shares with another road of the event
//       that holds its coordinates on >= 3 layers (the cross-road candidates)
//   P3  roads: combinations, fit, chi-square, cut and the road-local part of
//       the hit-warrior; publish cross-road group minima for flagged groups
//   P4  candidate roads: finish the hit-warrior across roads, count survivors
//   P5  road chunks: write the surviving tracks in (event, road, comb) order
//
// SVT_PLAIN runs P0, P1, P2, a combination scan, a fit kernel with one thread
// per combination that stores every key and track parameter in HBM, the
// warrior, P4 and P5 as separate kernels.  SVT_PERSISTENT runs all phases in
// one cooperative kernel separated by grid barriers whose waits are bounded,
// and evaluates each distinct fit once from per-hit partial sums kept in
// shared memory.  Both produce identical tracks.
//
// Integer exactness (the reason the fit runs in 32-bit): svt_load_constants
// admits only constant sets for which every partial and full sum of
// coefficient x input (+ 4096 x offset) stays below 2^31 in magnitude, so
// int32 accumulation equals the int64 sum; an arithmetic right shift by 12
// is floor division by 4096, and floor(s / 4096) + k == floor((s + 4096 k) /
// 4096).  chi2 < 2^38, so the track key (chi2 << 23 | road << 15 | comb)
// is a 61-bit integer ordered like (chi2, road, comb).
//
// The block size of every kernel is SVT_BLOCK (256 unless the including
// file sets it); each block size builds in a namespace of its own, and only
// the 256-thread build holds the plain pipeline.
#include <cstddef>

#include "svt_internal.h"

#ifndef SVT_BLOCK
#define SVT_BLOCK 256
#endif
#if SVT_BLOCK == 128
#define SVT_KNS b128
#elif SVT_BLOCK == 256
#define SVT_KNS b256
#elif SVT_BLOCK == 512
#define SVT_KNS b512
#else
#error "SVT_BLOCK must be 128, 256 or 512"
#endif

namespace svt {
namespace SVT_KNS {

constexpr int BLOCK = SVT_BLOCK;           // threads per CTA, every kernel of this build
constexpr int WARPS = BLOCK / 32;
constexpr int GRID_MAX = MAX_SPANS / WARPS < MAX_GRID ? MAX_SPANS / WARPS : MAX_GRID;

#define FULL_MASK 0xffffffffu

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned warp_id() { return threadIdx.x >> 5; }

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_relaxed(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// loads of data written earlier in the same launch by other CTAs: L2 only
template <class T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }
template <>
__device__ __forceinline__ RoadRec ldcg(const RoadRec *p)
{
    static_assert(sizeof(RoadRec) == 16, "RoadRec is one 16-byte load");
    uint4 v = __ldcg(reinterpret_cast<const uint4 *>(p));
    RoadRec r;
    memcpy(&r, &v, sizeof r);
    return r;
}

__device__ __forceinline__ void report(const Dev &d, unsigned long long pos, unsigned rank)
{
    atomicMax(&d.ctrl->err_inv, ~((pos << 8) | rank));
}

__device__ __forceinline__ void raise_flag(const Dev &d, unsigned f) { atomicOr(&d.ctrl->flags, f); }

// Survivor slot s of road g.  Slots are slot-major, so the first survivors
// of consecutive roads are adjacent (the output stage reads them in road
// order).
__device__ __forceinline__ size_t surv_at(const Dev &d, unsigned g, unsigned s)
{
    return (size_t)s * d.max_roads + g;
}

__device__ __forceinline__ bool word_ok(uint32_t w)
{
    uint32_t type = (w >> 27) & 7u, pl = w & 0x07FFFFFFu;
    if ((w >> 31) && !((w >> 30) & 1u))
        return false;                                   // EE without EP
    if (type <= 4)
        return (pl >> 12) == 0;
    if (type <= 6)
        return (pl >> 16) == 0;
    return (pl >> 10) == 0 && (pl & 15u) < 12 && ((pl >> 4) & 7u) < 6 && ((pl >> 7) & 7u) < 5;
}

// combinations of a road (product of its five hit counts) and its distinct
// fits (product over the four fitted layers: the excluded layer's hit does not
// enter the fit), from RoadRec::pk
// combinations N (at most 8^5) and distinct fits N4 of a road record
__device__ __forceinline__ void road_sizes(uint32_t pk, unsigned &N, unsigned &N4)
{
    const unsigned excl = (pk >> 20) & 7u;
    N = 1;
    N4 = 1;
    for (unsigned l = 0; l < N_LAYERS; ++l) {
        const unsigned n = (pk >> (4 * l)) & 15u;
        N *= n;
        if (l != excl)
            N4 *= n;
    }
}

// floor(x / m) for 1 <= m <= 8 and x < 2^16 with M = ceil(2^31 / m):
// (2x)(2^31 + e) / (m 2^32) = x / m + 2 x e / (m 2^32) with e < m, and
// 2 x e < 2^32, so the high word of 2x * M is the quotient (32-bit
// multiply-high, no 64-bit product).
__device__ __forceinline__ unsigned divm(unsigned x, unsigned M) { return __umulhi(x << 1, M); }
__host__ __device__ constexpr unsigned magic(unsigned m) { return (unsigned)(((1ull << 31) + m - 1) / m); }
// magic(m) for the hit counts m = 1..8 (entry 0 repeats m = 1)
__device__ __constant__ unsigned c_magic[MAX_HITS + 1] = {
    magic(1), magic(1), magic(2), magic(3), magic(4), magic(5), magic(6), magic(7), magic(8)};

template <class T>
__device__ __forceinline__ T warp_sum(T v)
{
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v)
{
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long u = __shfl_xor_sync(FULL_MASK, v, o);
        v = u < v ? u : v;
    }
    return v;
}

// block-wide exclusive scan of one unsigned long long per thread
__device__ unsigned long long block_excl_scan(unsigned long long v, unsigned long long *total)
{
    __shared__ unsigned long long s_w[WARPS + 1];
    unsigned long long inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long n = __shfl_up_sync(FULL_MASK, inc, o);
        if ((int)lane_id() >= o)
            inc += n;
    }
    if (lane_id() == 31)
        s_w[warp_id()] = inc;
    __syncthreads();
    if (warp_id() == 0) {
        unsigned long long x = lane_id() < WARPS ? s_w[lane_id()] : 0, xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long n = __shfl_up_sync(FULL_MASK, xi, o);
            if ((int)lane_id() >= o)
                xi += n;
        }
        if (lane_id() < WARPS)
            s_w[lane_id()] = xi - x;
        if (lane_id() == WARPS - 1)
            s_w[WARPS] = xi;
    }
    __syncthreads();
    unsigned long long r = s_w[warp_id()] + inc - v;
    if (total)
        *total = s_w[WARPS];
    __syncthreads();
    return r;
}

// the same for one unsigned per thread (32-bit sums)
__device__ unsigned block_excl_scan32(unsigned v, unsigned *total)
{
    __shared__ unsigned s_w32[WARPS + 1];
    unsigned inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned n = __shfl_up_sync(FULL_MASK, inc, o);
        if ((int)lane_id() >= o)
            inc += n;
    }
    if (lane_id() == 31)
        s_w32[warp_id()] = inc;
    __syncthreads();
    if (warp_id() == 0) {
        const unsigned x = lane_id() < WARPS ? s_w32[lane_id()] : 0u;
        unsigned xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned n = __shfl_up_sync(FULL_MASK, xi, o);
            if ((int)lane_id() >= o)
                xi += n;
        }
        if (lane_id() < WARPS)
            s_w32[lane_id()] = xi - x;
        if (lane_id() == WARPS - 1)
            s_w32[WARPS] = xi;
    }
    __syncthreads();
    const unsigned r = s_w32[warp_id()] + inc - v;
    *total = s_w32[WARPS];
    __syncthreads();
    return r;
}

// block-wide sums of two unsigned long long per thread, one exchange
__device__ void block_sum2(unsigned long long &a, unsigned long long &b)
{
    __shared__ unsigned long long s_ab[2 * WARPS];   // a of each warp, then b
    a = warp_sum(a);
    b = warp_sum(b);
    if (lane_id() == 0) {
        s_ab[warp_id()] = a;
        s_ab[WARPS + warp_id()] = b;
    }
    __syncthreads();
    a = 0;
    b = 0;
#pragma unroll
    for (unsigned w = 0; w < WARPS; ++w) {
        a += s_ab[w];
        b += s_ab[WARPS + w];
    }
    __syncthreads();
}

__device__ unsigned long long block_sum(unsigned long long v)
{
    unsigned long long t;
    block_excl_scan(v, &t);
    return t;
}

// Exclusive scan of in[0..n) into out[0..n) by one CTA; returns the total.
template <class TI, class TO>
__device__ unsigned long long block_scan_array(const TI *in, TO *out, unsigned n)
{
    unsigned long long carry = 0;
    for (unsigned base = 0; base < n; base += BLOCK) {
        unsigned i = base + threadIdx.x;
        unsigned long long v = i < n ? (unsigned long long)ldcg(in + i) : 0ull, tot;
        unsigned long long ex = block_excl_scan(v, &tot);
        if (i < n)
            out[i] = (TO)(carry + ex);
        carry += tot;
    }
    return carry;
}

// true in the CTA that arrives last at `counter` (all earlier CTAs' writes
// are visible to it)
__device__ bool last_block(unsigned *counter, unsigned nblocks)
{
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(counter, 1u) == nblocks - 1;
    }
    __syncthreads();
    if (s_last)
        __threadfence();
    return s_last;
}

// next item of work queue q for the whole CTA
__device__ unsigned grab(const Dev &d, int q)
{
    __shared__ unsigned s_item;
    __syncthreads();
    if (threadIdx.x == 0)
        s_item = atomicAdd(&d.ctrl->q[q], 1u);
    __syncthreads();
    return s_item;
}

// Work queue q where every CTA's first item is its own index: the queue
// hands out items gridDim.x, gridDim.x + 1, ... (one claim per later item,
// none at the start, when every CTA would claim at once on one counter)
__device__ __forceinline__ unsigned grab_after_first(const Dev &d, int q)
{
    return gridDim.x + grab(d, q);
}

// Grid barrier of the persistent kernel.  All CTAs are co-resident
// (cooperative launch).  The wait is bounded by d.wait_ns; on expiry the CTA
// raises FLAG_TIMEOUT and every CTA that sees the flag stops working.
__device__ bool grid_sync(const Dev &d)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned nb = gridDim.x;
        unsigned old = atomicAdd(&d.ctrl->bar, 1u);
        unsigned target = (old / nb + 1u) * nb;
        unsigned long long t0 = globaltimer_ns();
        int ok = 1;
        // relaxed polls of the counter (the fence below orders what follows);
        // the timeout flag and the clock are looked at every 16th poll
        for (unsigned it = 1; (int)(ld_relaxed(&d.ctrl->bar) - target) < 0; ++it) {
            if ((it & 15u) == 0) {
                if (ld_relaxed(&d.ctrl->flags) & FLAG_TIMEOUT) {
                    ok = 0;
                    break;
                }
                if (globaltimer_ns() - t0 > d.wait_ns) {
                    raise_flag(d, FLAG_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
            __nanosleep(32);
        }
        __threadfence();
        if (ld_acquire(&d.ctrl->flags) & FLAG_TIMEOUT)
            ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// phase timestamp k of the persistent kernel (block 0, thread 0)
__device__ __forceinline__ void stamp(const Dev &d, unsigned k)
{
    if (blockIdx.x == 0 && threadIdx.x == 0)
        d.ctrl->t_phase[k] = globaltimer_ns();
}

// work-queue indices (Ctrl::q)
enum { Q_P0 = 0, Q_P1, Q_P2, Q_BIG, Q_SMALL, Q_P4, Q_P5, Q_CNT, Q_CSC, Q_FIT, Q_P2W };

// ---------------------------------------------------------------------------
// P0 / P1: the word stream, one warp per span.  The stream is cut into
// gridDim.x * WARPS spans of whole 32-word windows; warp w of CTA b owns span
// b * WARPS + w.  P0 counts each span's EE and EP words and the EP words after
// its last EE, and checks every word's fields.  P1 gives each warp the counts
// of the spans before its own (every CTA sums them itself, no CTA scans for
// the others) and decodes the roads whose header lies in the warp's span.
// Ballots over the EP and EE bits of a window (lane i: word i) find the roads
// that start in it, with their road index, event and place in the event;
// each road is then walked by one lane from its header to its EP word,
// which checks the grammar and ranks each hit in its layer.  A warp follows
// its last road past the end of its span.
// ---------------------------------------------------------------------------

constexpr unsigned WIN = 32;               // words per window: one per lane
constexpr unsigned SEG_EE = 0x80000000u;   // segment word: an EE was seen (low bits: EP words since)

// span i of the stream (0 <= i < gridDim.x * WARPS): words [a, e)
__device__ __forceinline__ void span_of(const Dev &d, unsigned i, unsigned long long &a, unsigned long long &e)
{
    const unsigned long long n = (unsigned long long)gridDim.x * WARPS;
    const unsigned long long per = ((d.n_words + n - 1) / n + WIN - 1) / WIN * WIN;
    a = min((unsigned long long)i * per, d.n_words);
    e = min(a + per, d.n_words);
}

// Join of the segment words of two stretches of words, x before y: the EP
// words since the last EE of both (SEG_EE when either holds an EE).  0 is the
// identity.  Counts stay below 2^31 (a batch holds fewer words).
__device__ __forceinline__ unsigned seg_join(unsigned x, unsigned y)
{
    return (y & SEG_EE) ? y : (x & SEG_EE) | ((x & ~SEG_EE) + y);
}

// segment word of one window from its EE and EP lane masks
__device__ __forceinline__ unsigned seg_window(unsigned em, unsigned pm)
{
    return em ? SEG_EE | (unsigned)__popc((pm >> (31 - __clz(em))) >> 1) : (unsigned)__popc(pm);
}

// In-order fold of one segment word per lane (lane i's stretch before lane
// i + 1's); the result in every lane.
__device__ __forceinline__ unsigned warp_seg_fold(unsigned v)
{
    for (unsigned o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_down_sync(FULL_MASK, v, o);
        if (lane_id() + o < 32)
            v = seg_join(v, u);
    }
    return __shfl_sync(FULL_MASK, v, 0);
}

// the same over the CTA (thread t's stretch before thread t + 1's)
__device__ unsigned block_seg_fold(unsigned v)
{
    __shared__ unsigned s_seg[WARPS];
    v = warp_seg_fold(v);
    if (lane_id() == 0)
        s_seg[warp_id()] = v;
    __syncthreads();
    unsigned r = 0;
#pragma unroll
    for (unsigned w = 0; w < WARPS; ++w)
        r = seg_join(r, s_seg[w]);
    __syncthreads();
    return r;
}

__device__ void scan_count(const Dev &d)
{
    const unsigned lane = lane_id(), sp = blockIdx.x * WARPS + warp_id();
    unsigned long long a, e;
    span_of(d, sp, a, e);
    unsigned ee = 0, ep = 0, seg = 0;
    unsigned long long bad = ~0ull;
    constexpr unsigned UNROLL = 8;   // windows whose loads are in flight together
    for (unsigned long long base = a; base < e; base += UNROLL * WIN) {
        uint32_t w[UNROLL];
#pragma unroll
        for (unsigned k = 0; k < UNROLL; ++k) {
            const unsigned long long i = base + k * WIN + lane;
            w[k] = i < e ? __ldg(d.words + i) : 0u;
        }
#pragma unroll
        for (unsigned k = 0; k < UNROLL; ++k) {
            const unsigned long long i = base + k * WIN + lane;
            const unsigned em = __ballot_sync(FULL_MASK, w[k] >> 31);
            const unsigned pm = __ballot_sync(FULL_MASK, (w[k] >> 30) & 1u);
            ee += __popc(em);
            ep += __popc(pm);
            seg = seg_join(seg, seg_window(em, pm));
            if (i < e && bad == ~0ull && !word_ok(w[k]))
                bad = i;
        }
    }
    bad = warp_min_u64(bad);
    __shared__ unsigned s_cnt[3][WARPS];
    if (lane == 0) {
        if (bad != ~0ull)
            report(d, bad, RANK_BAD);
        d.span_ee[sp] = ee;
        d.span_ep[sp] = ep;
        d.span_seg[sp] = seg;
        s_cnt[0][warp_id()] = ee;
        s_cnt[1][warp_id()] = ep;
        s_cnt[2][warp_id()] = seg;
    }
    __syncthreads();
    if (threadIdx.x == 0) {   // the CTA's spans together, after the per-warp entries
        unsigned tee = 0, tep = 0, tseg = 0;
#pragma unroll
        for (unsigned w = 0; w < WARPS; ++w) {
            tee += s_cnt[0][w];
            tep += s_cnt[1][w];
            tseg = seg_join(tseg, s_cnt[2][w]);
        }
        d.span_ee[MAX_SPANS + blockIdx.x] = tee;
        d.span_ep[MAX_SPANS + blockIdx.x] = tep;
        d.span_seg[MAX_SPANS + blockIdx.x] = tseg;
    }
}

// P1 of one warp.  A ballot scan of the span finds the roads that start in
// it (the word after an EP word) with their road index, event and place in
// the event, and queues them in shared memory; each batch of 32 queued roads
// is decoded one road per lane, the lane walking its road's words from the
// header to the EP word (past the span's end if need be).  Each lane builds
// its road's coordinate row in shared memory; the batch's rows (consecutive
// roads) are then copied out with 16-byte stores.
constexpr unsigned P1_AHEAD = 4;                  // windows scanned per step (loads in flight together)
constexpr unsigned P1_Q = (P1_AHEAD + 1) * WIN;  // queued road starts per warp
struct P1Warp {
    uint16_t row[WIN][40];           // coordinate rows of the batch's roads
    uint32_t pos[P1_Q], g[P1_Q], ev[P1_Q], rie[P1_Q];   // queued roads: first word, index, event,
                                                         // roads of the event before it
};
static_assert(sizeof(P1Warp) % 16 == 0, "warp regions of 16-byte multiples");

// the longest road a lane walks: a road of more words breaks a rule within
// its first MAX_ROAD_WORDS words (a ninth hit on some layer at the latest)
constexpr unsigned MAX_ROAD_WORDS = 3 + N_LAYERS * MAX_HITS + 1;

// Decode queued roads [off, off + cnt) (cnt <= 32) one per lane; returns the
// batch's first fault (encoded as in Ctrl::err_inv, ~0 when none).
__device__ __forceinline__ unsigned long long decode_batch(const Dev &d, P1Warp &q, unsigned off, unsigned cnt,
                                                           unsigned n_events)
{
    const unsigned lane = lane_id();
    unsigned long long err = ~0ull;
    bool done = false;   // a complete road (its EP word seen)
    unsigned g = 0;
    if (lane < cnt) {
        const unsigned start = q.pos[off + lane], ev = q.ev[off + lane], rie = q.rie[off + lane];
        g = q.g[off + lane];
        uint16_t *row = q.row[lane];
        unsigned cnt4 = 0;   // hits so far, layer l in bits 4 l .. 4 l + 3 (at most MAX_HITS)
        uint32_t hdr = 0, cw = 0, pw = 0;
        bool ee = false;
        for (unsigned k0 = 0; k0 < MAX_ROAD_WORDS && !done && err == ~0ull; k0 += 8) {
            uint32_t w4[8];
#pragma unroll
            for (unsigned u = 0; u < 8; ++u) {   // eight loads in flight
                const unsigned long long p = (unsigned long long)start + k0 + u;
                w4[u] = p < d.n_words ? __ldg(d.words + p) : 0u;
            }
#pragma unroll
            for (unsigned u = 0; u < 8; ++u) {
                const unsigned k = k0 + u;
                const unsigned long long p = (unsigned long long)start + k;
                if (done || err != ~0ull || k >= MAX_ROAD_WORDS || p >= d.n_words)
                    break;
                const uint32_t w = w4[u];
                const unsigned type = (w >> 27) & 7u;
                const bool ep = (w >> 30) & 1u;
                bool bad;
                if (k == 0) {
                    bad = type != 7 || ep;
                    hdr = w;
                    if (!bad && rie >= (unsigned)MAX_ROADS_EV)
                        err = (p << 8) | RANK_LIMIT;
                } else if (k == 1) {
                    bad = type != 5 || ep;
                    cw = w;
                } else if (k == 2) {
                    bad = type != 6;
                    pw = w;
                } else {
                    bad = type > 4;
                    if (!bad) {
                        const unsigned r = (cnt4 >> (4 * type)) & 15u;
                        if (r >= (unsigned)MAX_HITS) {
                            err = (p << 8) | RANK_LIMIT;
                        } else {
                            row[type * 8 + r] = (uint16_t)(w & 0xFFFu);
                            cnt4 += 1u << (4 * type);
                        }
                    }
                }
                if (bad)
                    err = (p << 8) | RANK_BAD;
                else if (ep && err == ~0ull) {
                    done = true;
                    ee = (w >> 31) != 0;
                }
            }
        }
        if (done && g < d.max_roads) {   // a complete road: its record
            const unsigned pk = cnt4;   // the hit counts, four bits per layer
            const unsigned wedge = min(hdr & 15u, 11u), barrel = min((hdr >> 4) & 7u, 5u);
            const unsigned excl = min((hdr >> 7) & 7u, 4u);
            RoadRec r;
            r.event = ev;
            r.pk = pk | (excl << 20) | (min(rie, 255u) << 24);
            r.curv = (int16_t)(cw & 0xFFFFu);
            r.phi = (int16_t)(pw & 0xFFFFu);
            r.set = (uint16_t)((wedge * 6 + barrel) * 5 + excl);
            r.cta = 0;
            d.roads[g] = r;
            if (ee && ev < d.max_events) {   // the event's last road
                d.ev_road_end[ev] = g + 1;
                if (rie + 1 > (unsigned)P2W_ROADS)   // P2 takes this event with a whole CTA
                    d.ev_big[atomicAdd(&d.ctrl->n_big_ev, 1u)] = ev;
                if (ev + 1 == n_events)
                    d.ctrl->n_roads = g + 1;
            }
        }
    }
    __syncwarp();
    // the rows of the batch's complete roads (consecutive road indices from
    // the first lane's), five 16-byte words each
    const unsigned g0 = __shfl_sync(FULL_MASK, g, 0), dm = __ballot_sync(FULL_MASK, done);
    const uint4 *src = reinterpret_cast<const uint4 *>(&q.row[0][0]);
    uint4 *dst = reinterpret_cast<uint4 *>(d.coords + (size_t)g0 * 40);
    for (unsigned i = lane; i < cnt * N_LAYERS; i += WIN) {
        const unsigned j = i / N_LAYERS;
        if (((dm >> j) & 1u) && g0 + j < d.max_roads)
            dst[i] = src[i];
    }
    __syncwarp();
    return warp_min_u64(err);
}

// P1 for one warp: the roads whose header lies in [a, e).  g, ev: EP and EE
// words before a; rie: EP words since the last EE before a (roads of the open
// event).
__device__ void decode_span(const Dev &d, P1Warp &q, unsigned long long a, unsigned long long e, unsigned g,
                            unsigned ev, unsigned rie, unsigned n_events)
{
    const unsigned lane = lane_id(), lt = lanemask_lt();
    bool prev_ep = a == 0 || ((__ldg(d.words + a - 1) >> 30) & 1u);   // word a starts a road
    unsigned qn = 0;
    unsigned long long err = ~0ull;
    for (unsigned long long W0 = a;; W0 += P1_AHEAD * WIN) {
        const bool more = W0 < e && err == ~0ull;
        if (more) {   // P1_AHEAD windows: their road starts join the queue
            uint32_t wds[P1_AHEAD];
#pragma unroll
            for (unsigned k = 0; k < P1_AHEAD; ++k) {
                const unsigned long long i = W0 + k * WIN + lane;
                wds[k] = i < e ? __ldg(d.words + i) : 0u;
            }
#pragma unroll
            for (unsigned k = 0; k < P1_AHEAD; ++k) {
                const unsigned long long i = W0 + k * WIN + lane;
                const bool in = i < e;
                const uint32_t wd = wds[k];
                const unsigned pm = __ballot_sync(FULL_MASK, in && ((wd >> 30) & 1u));
                const unsigned em = __ballot_sync(FULL_MASK, in && (wd >> 31));
                const unsigned sm = ((pm << 1) | (prev_ep ? 1u : 0u)) & __ballot_sync(FULL_MASK, in);
                if ((sm >> lane) & 1u) {   // a road starts at this word
                    const unsigned j = qn + __popc(sm & lt), em_lt = em & lt;
                    q.pos[j] = (uint32_t)i;
                    q.g[j] = g + __popc(pm & lt);
                    q.ev[j] = ev + __popc(em & lt);
                    q.rie[j] = em_lt ? __popc(pm & lt & ~((2u << (31 - __clz(em_lt))) - 1u)) : rie + __popc(pm & lt);
                }
                qn += __popc(sm);
                g += __popc(pm);
                ev += __popc(em);
                rie = em ? (unsigned)__popc((pm >> (31 - __clz(em))) >> 1) : rie + __popc(pm);
                prev_ep = (pm >> 31) & 1u;
            }
            __syncwarp();
        }
        // full batches of 32 roads, and at the end the rest
        unsigned off = 0;
        while (err == ~0ull && (qn - off >= WIN || (!more && qn > off))) {
            const unsigned c = min(qn - off, WIN);
            err = decode_batch(d, q, off, c, n_events);
            off += c;
        }
        if (!more || err != ~0ull)
            break;
        if (off) {   // fewer than 32 left: to the front of the queue
            const unsigned rest = qn - off;
            uint32_t p0 = 0, p1 = 0, p2 = 0, p3 = 0;
            if (lane < rest) {
                p0 = q.pos[off + lane];
                p1 = q.g[off + lane];
                p2 = q.ev[off + lane];
                p3 = q.rie[off + lane];
            }
            __syncwarp();
            if (lane < rest) {
                q.pos[lane] = p0;
                q.g[lane] = p1;
                q.ev[lane] = p2;
                q.rie[lane] = p3;
            }
            qn = rest;
            __syncwarp();
        }
    }
    if (lane == 0 && err != ~0ull)
        atomicMax(&d.ctrl->err_inv, ~err);   // the first fault of the batch is its status
}

// P1; false when the stream does not fit the context (every CTA sees the
// same totals and stops).  smem: the CTA's shared memory (a P1Warp per warp).
__device__ bool scan_decode(const Dev &d, unsigned char *smem)
{
    const unsigned mine0 = blockIdx.x * WARPS;
    // the CTAs below this one (their aggregates follow the per-warp entries),
    // and all CTAs (the stream's counts)
    const unsigned per = (gridDim.x + BLOCK - 1) / BLOCK;
    const unsigned c0 = min(threadIdx.x * per, gridDim.x), c1 = min(c0 + per, gridDim.x);
    unsigned long long all = 0, below = 0;   // EE << 32 | EP
    unsigned seg = 0;
    for (unsigned c = c0; c < c1; ++c) {
        const unsigned long long v = ((unsigned long long)ldcg(d.span_ee + MAX_SPANS + c) << 32) |
                                     ldcg(d.span_ep + MAX_SPANS + c);
        all += v;
        if (c < blockIdx.x) {
            below += v;
            seg = seg_join(seg, ldcg(d.span_seg + MAX_SPANS + c));
        }
    }
    block_sum2(all, below);
    seg = block_seg_fold(seg);
    const unsigned n_ee = (unsigned)(all >> 32), n_ep = (unsigned)all;
    const bool fits = n_ee <= d.max_events && n_ep <= d.max_roads;
    // the candidate bits of this batch's roads start at zero (P2 sets them)
    if (fits)
        for (unsigned i = blockIdx.x * BLOCK + threadIdx.x; i < n_ep / 32 + 1; i += gridDim.x * BLOCK)
            d.cand_bits[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctrl *c = d.ctrl;
        c->n_events = n_ee;
        c->n_ep = n_ep;
        unsigned tail = 0;
        if (d.n_words > 0 && !(__ldg(d.words + d.n_words - 1) >> 31)) {
            tail = 1;
            report(d, d.n_words, RANK_TRUNC);
        }
        c->has_tail = tail;
        if (!fits)
            raise_flag(d, FLAG_CAPACITY);
        if (n_ee == 0)
            c->n_roads = 0;
    }
    if (!fits)
        return false;
    // the spans of this CTA below this warp
    unsigned g = (unsigned)below, ev = (unsigned)(below >> 32);
    {
        const unsigned j = lane_id(), sp = mine0 + j;
        const bool b4 = j < warp_id();
        g += warp_sum(b4 ? ldcg(d.span_ep + sp) : 0u);
        ev += warp_sum(b4 ? ldcg(d.span_ee + sp) : 0u);
        seg = seg_join(seg, warp_seg_fold(b4 ? ldcg(d.span_seg + sp) : 0u));
    }
    unsigned long long a, e;
    span_of(d, mine0 + warp_id(), a, e);
    P1Warp &q = reinterpret_cast<P1Warp *>(smem)[warp_id()];
    decode_span(d, q, a, e, g, ev, seg & ~SEG_EE, n_ee);
    return true;
}

// ---------------------------------------------------------------------------
// P2: the cross-road flags of each event (a CTA or a warp per event).  A track can
// only be dropped by a track of another road that shares hits with it on
// three layers, so only road pairs with a coordinate in common on >= 3
// layers matter.  The coordinates of the event that appear in two or more
// roads (per-layer bitmaps) get, per road and layer, a 64-bit signature;
// pairs of roads whose signatures meet on >= 3 layers take the exact test,
// which marks the shared hits of both roads.  A road with a marked hit is a
// cross-road candidate; its marked hits are the ones it publishes and looks
// up.  The road records get the candidate bit and their fit path.
//
// In a batch of many events, events of at most P2W_ROADS roads take one warp
// each instead (p2_warp), with the same bitmaps, 32-bit signatures, and a
// lane per road that tests its road against the others and marks its own
// hits (p2_phase chooses).
// ---------------------------------------------------------------------------

constexpr unsigned P2_PAIRS = 1024;   // road pairs queued for the exact test (more: tested in place)

struct P2Smem {
    RoadRec rec[MAX_ROADS_EV];
    uint16_t coord[MAX_ROADS_EV][40];     // [road][layer * 8 + hit]
    unsigned long long sig[MAX_ROADS_EV][N_LAYERS];   // signatures of a road's shared coordinates
    uint32_t seen[N_LAYERS][128];         // coordinate bitmaps of the event
    uint32_t multi[N_LAYERS][128];
    uint32_t xlo[MAX_ROADS_EV];           // hits shared with a road that shares coordinates on
    uint32_t xhi[MAX_ROADS_EV];           //   >= 3 layers: bit 8 l + d (l < 4), layer 4 in xhi
    uint16_t elig[MAX_ROADS_EV];          // roads with shared coordinates on >= 3 layers
    uint32_t cp[P2_PAIRS];                // road pairs whose signatures meet on >= 3 layers (r | t << 16)
    uint8_t rep[MAX_ROADS_EV];            // a coordinate repeated within a layer of the road
    unsigned n_elig, n_cp;
};
static_assert(offsetof(P2Smem, coord) % 16 == 0 && offsetof(P2Smem, rec) % 16 == 0, "16-byte rows");

// signature bit of a coordinate: a multiplicative hash into 0..63
__device__ __forceinline__ unsigned sig_bit(unsigned v) { return (v * 0x9E3779B1u) >> 26; }

__device__ __forceinline__ bool is_multi(const P2Smem &s, unsigned l, unsigned v)
{
    return (s.multi[l][v >> 5] >> (v & 31u)) & 1u;
}

// coordinate x of a layer's row (eight 16-bit coordinates in a uint4); x is
// a constant in the unrolled loops below
__device__ __forceinline__ unsigned row_coord(const uint4 &q, unsigned x)
{
    const unsigned w = x < 2 ? q.x : x < 4 ? q.y : x < 6 ? q.z : q.w;
    return (w >> (16 * (x & 1u))) & 0xFFFFu;
}

// Hits of one layer of a road (row q) whose coordinate was already in the
// event's bitmap when the hit set its bit (bit x of `again`): a coordinate
// of an earlier slot of the same row is a repeat; any other was set by
// another road and gets the multi bit.  So a coordinate gets the multi bit
// exactly when two roads hold it.  True when the row repeats a coordinate.
__device__ __noinline__ bool seen_again(uint32_t *multi, const uint4 &q, unsigned again)
{
    bool rep = false;
#pragma unroll
    for (unsigned x = 0; x < MAX_HITS; ++x) {
        if (!((again >> x) & 1u))
            continue;
        const unsigned v = row_coord(q, x);
        bool dup = false;
#pragma unroll
        for (unsigned y = 0; y < x; ++y)
            dup = dup || row_coord(q, y) == v;
        if (dup)
            rep = true;
        else
            atomicOr(&multi[v >> 5], 1u << (v & 31u));
    }
    return rep;
}

// Roads r and t of the event: the layers on which they hold a common
// coordinate and the hits involved; with three or more such layers, the
// shared hits of both roads are marked.  Only coordinates present in two
// roads can be common.
__device__ void pair_exact(P2Smem &s, unsigned r, unsigned t)
{
    const uint32_t pr = s.rec[r].pk, pt = s.rec[t].pk;
    unsigned lo_r = 0, lo_t = 0, hi_r = 0, hi_t = 0, layers = 0;
#pragma unroll
    for (unsigned l = 0; l < N_LAYERS; ++l) {
        const unsigned nr = (pr >> (4 * l)) & 15u, nt = (pt >> (4 * l)) & 15u;   // <= MAX_HITS
        unsigned br = 0, bt = 0;
        for (unsigned x = 0; x < nr; ++x) {
            const unsigned v = s.coord[r][l * 8 + x];
            if (!is_multi(s, l, v))
                continue;
            for (unsigned y = 0; y < nt; ++y)
                if (s.coord[t][l * 8 + y] == v) {
                    br |= 1u << x;
                    bt |= 1u << y;
                }
        }
        layers += br != 0;
        if (l < 4) {
            lo_r |= br << (8 * l);
            lo_t |= bt << (8 * l);
        } else {
            hi_r = br;
            hi_t = bt;
        }
    }
    if (layers >= 3) {
        atomicOr(&s.xlo[r], lo_r);
        atomicOr(&s.xhi[r], hi_r);
        atomicOr(&s.xlo[t], lo_t);
        atomicOr(&s.xhi[t], hi_t);
    }
}

// The exact test of pair_exact by a whole warp: lane 8 l + x (then lane x
// for layer 4) takes hit x of road r on layer l and compares it with road t's
// hits on that layer.
__device__ void pair_exact_warp(P2Smem &s, unsigned r, unsigned t)
{
    const unsigned lane = lane_id();
    const uint32_t pr = s.rec[r].pk, pt = s.rec[t].pk;
    unsigned m_r[2], m_t[2];   // marked hits of r and t: layers 0..3, then layer 4
#pragma unroll
    for (unsigned pass = 0; pass < 2; ++pass) {
        const unsigned l = pass ? 4u : lane >> 3, x = pass ? lane : lane & 7u;
        const unsigned nr = (pr >> (4 * l)) & 15u, nt = (pt >> (4 * l)) & 15u;   // <= MAX_HITS
        unsigned br = 0, bt = 0;
        if (x < nr && (!pass || lane < 8)) {
            const unsigned v = s.coord[r][l * 8 + x];
            if (is_multi(s, l, v))
                for (unsigned y = 0; y < nt; ++y)
                    if (s.coord[t][l * 8 + y] == v) {
                        br = 1u << x;
                        bt |= 1u << y;
                    }
        }
        const unsigned sh = pass ? 0u : 8 * l;
        m_r[pass] = __reduce_or_sync(FULL_MASK, br << sh);
        m_t[pass] = __reduce_or_sync(FULL_MASK, bt << sh);
    }
    const unsigned layers = ((m_r[0] & 0xFFu) != 0) + ((m_r[0] & 0xFF00u) != 0) + ((m_r[0] & 0xFF0000u) != 0) +
                            ((m_r[0] >> 24) != 0) + (m_r[1] != 0);
    if (layers >= 3 && lane == 0) {
        atomicOr(&s.xlo[r], m_r[0]);
        atomicOr(&s.xhi[r], m_r[1]);
        atomicOr(&s.xlo[t], m_t[0]);
        atomicOr(&s.xhi[t], m_t[1]);
    }
}

// Flags of event e (roads r0 .. r0 + nr - 1); adds its combinations to n_comb.
__device__ void p2_event(const Dev &d, unsigned e, unsigned r0, unsigned nr, unsigned char *smem,
                         unsigned long long &n_comb)
{
    P2Smem &s = *reinterpret_cast<P2Smem *>(smem);
    // the event's roads: records and coordinate rows (16-byte loads)
    for (unsigned k = threadIdx.x; k < nr; k += BLOCK) {
        s.rec[k] = ldcg(d.roads + r0 + k);
        s.rep[k] = 0;
        s.xlo[k] = 0;
        s.xhi[k] = 0;
    }
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(d.coords + (size_t)r0 * 40);
        uint4 *dst = reinterpret_cast<uint4 *>(&s.coord[0][0]);
        for (unsigned i = threadIdx.x; i < nr * N_LAYERS; i += BLOCK)
            dst[i] = ldcg(src + i);
    }
    for (unsigned i = threadIdx.x; i < N_LAYERS * 128; i += BLOCK) {
        (&s.seen[0][0])[i] = 0;
        (&s.multi[0][0])[i] = 0;
    }
    if (threadIdx.x == 0) {
        s.n_elig = 0;
        s.n_cp = 0;
    }
    __syncthreads();
    // coordinates present in >= 2 roads on a layer: each distinct coordinate
    // of a road's layer marks the bitmap, a second road with it the multi bit
    for (unsigned i = threadIdx.x; i < nr * N_LAYERS; i += BLOCK) {
        const unsigned k = i / N_LAYERS, l = i - k * N_LAYERS;
        const unsigned n = (s.rec[k].pk >> (4 * l)) & 15u;
        const uint4 q = *reinterpret_cast<const uint4 *>(&s.coord[k][l * 8]);
        unsigned again = 0;   // bit x: hit x found its bit set
#pragma unroll
        for (unsigned x = 0; x < MAX_HITS; ++x) {
            const unsigned v = row_coord(q, x), bit = 1u << (v & 31u);
            if (x < n && (atomicOr(&s.seen[l][v >> 5], bit) & bit))
                again |= 1u << x;
        }
        if (again && seen_again(s.multi[l], q, again))
            s.rep[k] = 1;
    }
    __syncthreads();
    // signatures of the shared coordinates; roads with >= 3 such layers
    for (unsigned k = threadIdx.x; k < nr; k += BLOCK) {
        unsigned layers = 0;
#pragma unroll
        for (unsigned l = 0; l < N_LAYERS; ++l) {
            const unsigned n = (s.rec[k].pk >> (4 * l)) & 15u;
            unsigned long long sg = 0;
            for (unsigned x = 0; x < n; ++x) {
                const unsigned v = s.coord[k][l * 8 + x];
                if (is_multi(s, l, v))
                    sg |= 1ull << sig_bit(v);
            }
            s.sig[k][l] = sg;
            layers += sg != 0;
        }
        if (layers >= 3)
            s.elig[atomicAdd(&s.n_elig, 1u)] = (uint16_t)k;
    }
    __syncthreads();
    // pairs of eligible roads whose signatures meet on >= 3 layers
    const unsigned ne = s.n_elig;
    for (unsigned a = warp_id(); a < ne; a += WARPS) {
        const unsigned r = s.elig[a];
        const unsigned long long s0 = s.sig[r][0], s1 = s.sig[r][1], s2 = s.sig[r][2], s3 = s.sig[r][3],
                                 s4 = s.sig[r][4];
        for (unsigned b = a + 1 + lane_id(); b < ne; b += 32) {
            const unsigned t = s.elig[b];
            const unsigned c = ((s0 & s.sig[t][0]) != 0) + ((s1 & s.sig[t][1]) != 0) + ((s2 & s.sig[t][2]) != 0) +
                               ((s3 & s.sig[t][3]) != 0) + ((s4 & s.sig[t][4]) != 0);
            if (c >= 3) {   // queued for a warp's exact test (in place when the queue is full)
                const unsigned k = atomicAdd(&s.n_cp, 1u);
                if (k < P2_PAIRS)
                    s.cp[k] = r | (t << 16);
                else
                    pair_exact(s, r, t);
            }
        }
    }
    __syncthreads();
    for (unsigned k = warp_id(); k < min(s.n_cp, P2_PAIRS); k += WARPS)
        pair_exact_warp(s, s.cp[k] & 0xFFFFu, s.cp[k] >> 16);
    __syncthreads();
    // the road records: candidate bit and fit path
    for (unsigned k = threadIdx.x; k < nr; k += BLOCK) {
        const unsigned g = r0 + k;
        RoadRec r = s.rec[k];
        const unsigned long long xm = ((unsigned long long)s.xhi[k] << 32) | s.xlo[k];
        const bool cand = xm != 0ull, rep = s.rep[k] != 0;
        unsigned N, N4;
        road_sizes(r.pk, N, N4);
        // fitted by one warp each (the box path): roads with more distinct
        // fits than a warp's run takes, and cross-road candidates with a
        // repeated coordinate (they publish over canonical hits)
        const bool big = N > 0 && (N4 > (unsigned)d.small_n4 || (cand && rep));
        r.pk |= cand ? (1u << 23) : 0u;
        r.cta = (big ? 1 : 0) | (rep ? 2 : 0);
        d.roads[g] = r;
        d.xmask[g] = xm;
        d.surv_cnt[g] = 0;
        if (big) {
            unsigned i = atomicAdd(&d.ctrl->n_big, 1u);
            if (i < d.max_roads)
                d.big_list[i] = g;
        }
        if (N > 0 && cand)   // checked against the other roads' groups after the fit
            atomicOr(&d.cand_bits[g >> 5], 1u << (g & 31u));
        n_comb += N;
    }
    __syncthreads();   // the shared arrays are refilled for the next event
}

// One warp's state for an event of at most P2W_ROADS roads; the roads'
// coordinate rows stay in global memory (L2), read a road at a time.
struct P2Warp {
    uint32_t seen[N_LAYERS][128];           // coordinate bitmaps of the event (12-bit coordinates)
    uint32_t multi[N_LAYERS][128];          // coordinates present in two or more roads
    uint32_t sig[P2W_ROADS][N_LAYERS];      // 32-bit signatures of a road's shared coordinates
    uint32_t pk[P2W_ROADS];
};
constexpr size_t P2W_BYTES = (sizeof(P2Warp) + 15) / 16 * 16;

// signature bit of a coordinate in a 32-bit signature
__device__ __forceinline__ unsigned sig_bit32(unsigned v) { return (v * 0x9E3779B1u) >> 27; }

// Hits of road g that road h holds too (bit 8 l + x), when they hold common
// coordinates on three layers or more; 0 otherwise.  pg, ph: their records'
// pk words.
__device__ unsigned long long pair_marks(const Dev &d, unsigned g, unsigned h, uint32_t pg, uint32_t ph)
{
    const uint4 *rg = reinterpret_cast<const uint4 *>(d.coords + (size_t)g * 40);
    const uint4 *rh = reinterpret_cast<const uint4 *>(d.coords + (size_t)h * 40);
    unsigned long long m = 0;
    unsigned layers = 0;
    for (unsigned l = 0; l < N_LAYERS; ++l) {
        const unsigned ng = (pg >> (4 * l)) & 15u, nh = (ph >> (4 * l)) & 15u;   // <= MAX_HITS
        const uint4 a = ldcg(rg + l), b = ldcg(rh + l);
        unsigned br = 0;
#pragma unroll
        for (unsigned x = 0; x < MAX_HITS; ++x) {
            const unsigned v = row_coord(a, x);
            bool hit = false;
#pragma unroll
            for (unsigned y = 0; y < MAX_HITS; ++y)
                hit = hit || (y < nh && row_coord(b, y) == v);
            br |= (x < ng && hit) ? 1u << x : 0u;
        }
        layers += br != 0;
        m |= (unsigned long long)br << (8 * l);
    }
    return layers >= 3 ? m : 0ull;
}

// P2 of the event of roads r0 .. r0 + nr - 1 (nr <= P2W_ROADS) by one warp
// with state `w`; lane i owns roads i and i + 32.  The same steps as
// p2_event: coordinates present in two roads (bitmaps), signatures of those
// per road and layer, pairs whose signatures meet on >= 3 layers tested
// exactly.  A lane tests its eligible road against every other eligible road
// (a pair whose signatures meet on >= 3 layers has two) and marks only its
// own road's hits, so each pair is tested from both sides.
__device__ void p2_warp(const Dev &d, unsigned r0, unsigned nr, P2Warp &w, unsigned long long &n_comb)
{
    const unsigned lane = lane_id();
    {
        uint4 *z = reinterpret_cast<uint4 *>(&w.seen[0][0]);   // seen and multi
        for (unsigned i = lane; i < 2 * N_LAYERS * 128 / 4; i += 32)
            z[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    bool rep[2] = {false, false};
#pragma unroll
    for (unsigned h = 0; h < 2; ++h) {
        const unsigned k = lane + 32 * h;
        if (k < nr)
            w.pk[k] = ldcg(&d.roads[r0 + k].pk);
    }
    __syncwarp();
    // each distinct coordinate of a road's layer marks the bitmap once; a
    // second road with it sets the multi bit
#pragma unroll
    for (unsigned h = 0; h < 2; ++h) {
        const unsigned k = lane + 32 * h;
        if (k >= nr)
            continue;
        const uint4 *row = reinterpret_cast<const uint4 *>(d.coords + (size_t)(r0 + k) * 40);
        const uint32_t pk = w.pk[k];
        for (unsigned l = 0; l < N_LAYERS; ++l) {
            const unsigned n = (pk >> (4 * l)) & 15u;
            const uint4 q = ldcg(row + l);
#pragma unroll
            for (unsigned x = 0; x < MAX_HITS; ++x) {
                const unsigned v = row_coord(q, x);
                bool first = x < n;
#pragma unroll
                for (unsigned y = 0; y < x; ++y)
                    first = first && row_coord(q, y) != v;
                if (first) {
                    const unsigned bit = 1u << (v & 31u);
                    if (atomicOr(&w.seen[l][v >> 5], bit) & bit)
                        atomicOr(&w.multi[l][v >> 5], bit);
                }
                rep[h] = rep[h] || (x < n && !first);
            }
        }
    }
    __syncwarp();
    // signatures of the shared coordinates
    unsigned elig = 0;   // bit h: the lane's road h has shared coordinates on >= 3 layers
#pragma unroll
    for (unsigned h = 0; h < 2; ++h) {
        const unsigned k = lane + 32 * h;
        if (k >= nr)
            continue;
        const uint4 *row = reinterpret_cast<const uint4 *>(d.coords + (size_t)(r0 + k) * 40);
        const uint32_t pk = w.pk[k];
        unsigned layers = 0;
        for (unsigned l = 0; l < N_LAYERS; ++l) {
            const unsigned n = (pk >> (4 * l)) & 15u;
            const uint4 q = ldcg(row + l);
            uint32_t sl = 0;
#pragma unroll
            for (unsigned x = 0; x < MAX_HITS; ++x) {
                const unsigned v = row_coord(q, x);
                if (x < n && ((w.multi[l][v >> 5] >> (v & 31u)) & 1u))
                    sl |= 1u << sig_bit32(v);
            }
            w.sig[k][l] = sl;
            layers += sl != 0u;
        }
        elig |= layers >= 3 ? 1u << h : 0u;
    }
    __syncwarp();
    // the other eligible roads t against the lane's eligible roads (their
    // signatures meet on >= 3 layers first)
    unsigned long long xm[2] = {0ull, 0ull};
    unsigned long long em = ((unsigned long long)__ballot_sync(FULL_MASK, (elig >> 1) & 1u) << 32) |
                            __ballot_sync(FULL_MASK, elig & 1u);
    if (__popcll(em) >= 2) {
        for (; em; em &= em - 1) {
            const unsigned t = (unsigned)__ffsll((long long)em) - 1;
#pragma unroll
            for (unsigned h = 0; h < 2; ++h) {
                const unsigned k = lane + 32 * h;
                if (!((elig >> h) & 1u) || k == t)
                    continue;
                unsigned c = 0;
#pragma unroll
                for (unsigned l = 0; l < N_LAYERS; ++l)
                    c += (w.sig[k][l] & w.sig[t][l]) != 0u;
                if (c >= 3)
                    xm[h] |= pair_marks(d, r0 + k, r0 + t, w.pk[k], w.pk[t]);
            }
        }
    }
#pragma unroll
    for (unsigned h = 0; h < 2; ++h) {
        const unsigned k = lane + 32 * h;
        if (k >= nr)
            continue;
        const unsigned g = r0 + k;
        RoadRec r = ldcg(d.roads + g);
        const bool cand = xm[h] != 0ull;
        unsigned N, N4;
        road_sizes(r.pk, N, N4);
        const bool big = N > 0 && (N4 > (unsigned)d.small_n4 || (cand && rep[h]));
        r.pk |= cand ? (1u << 23) : 0u;
        r.cta = (big ? 1 : 0) | (rep[h] ? 2 : 0);
        d.roads[g] = r;
        d.xmask[g] = xm[h];
        d.surv_cnt[g] = 0;
        if (big) {
            unsigned i = atomicAdd(&d.ctrl->n_big, 1u);
            if (i < d.max_roads)
                d.big_list[i] = g;
        }
        if (N > 0 && cand)
            atomicOr(&d.cand_bits[g >> 5], 1u << (g & 31u));
        n_comb += N;
    }
    __syncwarp();   // the state is refilled for the next event
}

// P2 over the events.  A batch of at most P2_CTA_EVENTS events per CTA: a
// CTA per event.  A larger one: first the events of more than P2W_ROADS
// roads (listed in P1), a CTA each from a queue; then every warp takes the
// other events from a second queue, one at a time (a warp takes longer over
// an event than a CTA, but eight of them work at once).  One
// combination-count atomic per CTA.
constexpr unsigned P2_CTA_EVENTS = 4;

__device__ void p2_phase(const Dev &d, unsigned char *smem)
{
    if (ldcg(&d.ctrl->err_inv) != 0ull)
        return;   // a data fault (every CTA reads the same word after the barrier): no tracks
    const unsigned n_events = min(ldcg(&d.ctrl->n_events), d.max_events);
    // survivor totals of the road chunks start at zero (the fit adds to them)
    const unsigned n_chunks = min((ldcg(&d.ctrl->n_roads) + ROAD_CHUNK - 1) / ROAD_CHUNK, d.max_chunks_r);
    for (unsigned i = blockIdx.x * BLOCK + threadIdx.x; i < n_chunks; i += gridDim.x * BLOCK)
        d.rchunk_sum[i] = 0;
    unsigned long long n_comb = 0;
    if (n_events <= P2_CTA_EVENTS * gridDim.x) {
        // few events for the grid: every event a CTA (the shortest time per
        // event); the CTA's first event is its own index, the queue hands
        // out the rest
        for (unsigned e = blockIdx.x; e < n_events; e = grab_after_first(d, Q_P2)) {
            const unsigned r0 = e == 0 ? 0u : min(ldcg(d.ev_road_end + e - 1), d.max_roads);
            const unsigned r1 = min(ldcg(d.ev_road_end + e), d.max_roads);
            p2_event(d, e, r0, min(r1 - min(r0, r1), (unsigned)MAX_ROADS_EV), smem, n_comb);
        }
        n_comb = block_sum(n_comb);
        if (threadIdx.x == 0 && n_comb)
            atomicAdd(&d.ctrl->n_comb, n_comb);
        return;
    }
    const unsigned n_big_ev = min(ldcg(&d.ctrl->n_big_ev), n_events);
    for (unsigned i = blockIdx.x; i < n_big_ev; i = grab_after_first(d, Q_P2)) {
        const unsigned e = min(ldcg(d.ev_big + i), n_events - 1);
        const unsigned r0 = e == 0 ? 0u : min(ldcg(d.ev_road_end + e - 1), d.max_roads);
        const unsigned r1 = min(ldcg(d.ev_road_end + e), d.max_roads);
        // an event of more than MAX_ROADS_EV roads is a fault (reported in P1)
        p2_event(d, e, r0, min(r1 - min(r0, r1), (unsigned)MAX_ROADS_EV), smem, n_comb);
    }
    __syncthreads();   // the shared memory becomes the warps' regions
    {
        P2Warp &w = *reinterpret_cast<P2Warp *>(smem + warp_id() * P2W_BYTES);
        const unsigned n_warps = gridDim.x * WARPS;
        for (unsigned e = blockIdx.x * WARPS + warp_id(); e < n_events;) {
            const unsigned r0 = e == 0 ? 0u : min(ldcg(d.ev_road_end + e - 1), d.max_roads);
            const unsigned r1 = min(ldcg(d.ev_road_end + e), d.max_roads);
            const unsigned nr = r1 - min(r0, r1);
            if (nr <= (unsigned)P2W_ROADS)   // the others were listed
                p2_warp(d, r0, nr, w, n_comb);
            unsigned ne = 0;
            if (lane_id() == 0)
                ne = n_warps + atomicAdd(&d.ctrl->q[Q_P2W], 1u);
            e = __shfl_sync(FULL_MASK, ne, 0);
        }
    }
    n_comb = block_sum(n_comb);
    if (threadIdx.x == 0 && n_comb)
        atomicAdd(&d.ctrl->n_comb, n_comb);
}

// ---------------------------------------------------------------------------
// P3: fit + cut + road-local hit-warrior: runs of roads per warp (the flat
// path), the roads listed in P2 one per warp (the box path)
// ---------------------------------------------------------------------------

// the same triples as constants the compiler folds in unrolled loops: layer
// k of triple t
__device__ __forceinline__ unsigned triple_l(unsigned t, unsigned k)
{
    return (unsigned)(((k == 0 ? 0x2111000000ull : k == 1 ? 0x3322322111ull : 0x4443443432ull) >> (4 * t)) & 15u);
}

__device__ __forceinline__ unsigned long long make_key(long long chi2, unsigned rie, unsigned comb)
{
    return ((unsigned long long)chi2 << 23) | ((unsigned long long)rie << 15) | comb;
}

__device__ __forceinline__ long long sq(int a) { return (long long)a * a; }

// hash of a group key (splitmix64 finaliser)
__device__ __forceinline__ unsigned hash_slot(unsigned long long k, unsigned mask)
{
    k ^= k >> 30;
    k *= 0xBF58476D1CE4E5B9ull;
    k ^= k >> 27;
    k *= 0x94D049BB133111EBull;
    k ^= k >> 31;
    return (unsigned)k & mask;
}

// The group table is probed linearly from a group's home slot, at most
// HASH_PROBES slots, and may be filled to three quarters of its slots: a
// batch that needs more raises FLAG_CAPACITY (SVT_E_CAPACITY, no tracks)
// instead of probing on.
constexpr unsigned HASH_PROBES = 64;

__device__ __forceinline__ unsigned hash_probes(const Dev &d) { return min(HASH_PROBES, d.hash_mask + 1); }

__device__ void hash_min(const Dev &d, unsigned long long gk, unsigned long long key)
{
    unsigned h = hash_slot(gk, d.hash_mask);
    const unsigned slots = d.hash_mask + 1;
    for (unsigned probe = 0; probe < hash_probes(d); ++probe) {
        unsigned long long prev = atomicCAS(&d.hash[h].key, 0ull, gk);
        if (prev == 0ull) {   // a new slot: marked for clearing (no value awaited)
            atomicOr(&d.hash_bits[h >> 5], 1u << (h & 31u));
            if (atomicAdd(&d.ctrl->hash_used, 1u) >= slots - slots / 4)
                raise_flag(d, FLAG_CAPACITY);
        }
        if (prev == 0ull || prev == gk) {
            atomicMax(&d.hash[h].val_inv, ~key);
            return;
        }
        h = (h + 1) & d.hash_mask;
    }
    raise_flag(d, FLAG_CAPACITY);
}

// lookup after the table is complete (no writer in flight): a slot's key and
// value are read by one 16-byte load
__device__ unsigned long long hash_get(const Dev &d, unsigned long long gk)
{
    static_assert(sizeof(HashSlot) == 16, "one 16-byte load per slot");
    unsigned h = hash_slot(gk, d.hash_mask);
    for (unsigned probe = 0; probe < hash_probes(d); ++probe) {
        const ulonglong2 sl = __ldcg(reinterpret_cast<const ulonglong2 *>(d.hash + h));
        if (sl.x == gk)
            return ~sl.y;
        if (sl.x == 0ull)
            return NO_KEY;
        h = (h + 1) & d.hash_mask;
    }
    return NO_KEY;
}

__device__ __forceinline__ unsigned long long group_key(unsigned event, unsigned t, unsigned v0,
                                                        unsigned v1, unsigned v2)
{
    return ((unsigned long long)(event + 1) << 40) | ((unsigned long long)t << 36) |
           ((unsigned long long)v0 << 24) | ((unsigned long long)v1 << 12) | v2;
}

__device__ __forceinline__ unsigned nth_bit(unsigned mask, unsigned n)
{
    for (unsigned i = 0; i < n; ++i)
        mask &= mask - 1;
    return __ffs(mask) - 1;
}

// ---------------------------------------------------------------------------
// P3, flat path: a warp fits a run of small roads together, one lane per
// table entry across the roads of the run (fit, pair tables, survivors), so
// the per-road work is spread over the lanes instead of repeated per road.
// A coordinate repeated within a fitted layer makes the pair tables take
// canonical hits (the lowest index with the same coordinate); a cross-road
// candidate with a repeated coordinate goes through the box path.
// ---------------------------------------------------------------------------

constexpr unsigned FLAT_K = N4_SMALL_MAX, FLAT_Q = QTAB_SMALL, FLAT_A = 64;

// One road of a run, in the warp's shared memory.  The fields the per-entry
// passes read are grouped in 16-byte words (vector loads).
struct alignas(16) FlatRoad {
    unsigned kb, ab, qb, key_hi;  // first key, partial sum and pair-table entry; road bits of a key
    unsigned m[4], st[4], SL[4], aoff[4];   // aoff: first partial sum of fitted slot j
    unsigned off[6];              // first entry of pair table p (aoff and off are rebased on the
                                  // sub-run's tables in the shared copy)
    unsigned M[3];                // magic divisors of m[0..2]
    unsigned xl;                  // excluded layer (bits 0..2), cross-road candidate (bit 3), hits
                                  // of the excluded layer (bits 4..7), layer of fitted slot j
                                  // (bits 8 + 3j .. 10 + 3j)
    unsigned g, N4, E, set;
    unsigned event, nl, Se;       // nl: hits per layer, 4 bits each; Se: comb stride of excl
    int curv, phi;
    unsigned pad;
    unsigned cm[4];               // canonical hit (the lowest index with the same coordinate) of
                                  // each hit of fitted slot j, 3 bits each
    unsigned long long cb;        // plain mode: first combination of the road
    unsigned long long xm;        // cross-road candidates: the road's flagged hits (xmask)
};
static_assert(offsetof(FlatRoad, m) % 16 == 0 && offsetof(FlatRoad, off) % 16 == 0 &&
                  offsetof(FlatRoad, cm) % 16 == 0,
              "16-byte groups");
__device__ __forceinline__ unsigned fr_excl(const FlatRoad &r) { return r.xl & 7u; }
__device__ __forceinline__ unsigned fr_ne(const FlatRoad &r) { return (r.xl >> 4) & 15u; }
__device__ __forceinline__ unsigned fr_layer(const FlatRoad &r, unsigned j) { return (r.xl >> (8 + 3 * j)) & 7u; }
constexpr unsigned CANON_ID = 0xFAC688u;   // hit x -> x for x < 8, 3 bits each

struct P3Flat {
    int4 A[FLAT_A];                       // partial chi-square sums, [aoff[j] + hit]
    unsigned long long K[FLAT_K];         // keys of distinct fits, [kb + f]
    unsigned Qh[FLAT_Q], Ql[FLAT_Q];      // pair tables, [qb + off[p] + x * m_b + y]: high and
                                          // low word of the minimum key (all ones = none)
    uint16_t dig[FLAT_K];                 // the fit's four slot hits (3 bits each), its road's lane
    FlatRoad rd[WARP_ROADS];
    uint16_t co[WARP_ROADS][40];
    unsigned cnt[WARP_ROADS];             // survivors found so far
};
static_assert(offsetof(P3Flat, co) % 16 == 0, "coordinate rows are copied in 16-byte words");

// the six pairs of fitted slots (a, b)
__device__ __forceinline__ unsigned pair_a(unsigned p) { return (0x211000u >> (4 * p)) & 15u; }
__device__ __forceinline__ unsigned pair_b(unsigned p) { return (0x332321u >> (4 * p)) & 15u; }

// The roads of a sub-run, in order, are the set bits of `sub` (lanes of the
// run).  A table over the sub-run packs the first entry of its k-th road in
// half-word k of w (0xFFFF past the last road) and the road's lane in nibble
// k of `lanes`.
struct FlatIndex {
    unsigned w[4], lanes;
    // lane of the road that owns entry t
    __device__ unsigned owner(unsigned t) const
    {
        unsigned k = t >= (w[0] >> 16);
#pragma unroll
        for (unsigned q = 1; q < 4; ++q)
            k += (t >= (w[q] & 0xFFFFu)) + (t >= (w[q] >> 16));
        return (lanes >> (4 * k)) & 15u;
    }
};

// Build the index from each road lane's first entry (every lane calls it).
__device__ __forceinline__ FlatIndex flat_index(unsigned first, unsigned sub)
{
    FlatIndex x{{0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, 0u};
    unsigned rest = sub;
#pragma unroll
    for (unsigned k = 0; k < WARP_ROADS; ++k) {
        const unsigned ln = rest ? __ffs(rest) - 1 : 0u;
        const unsigned v = __shfl_sync(FULL_MASK, first, ln) & 0xFFFFu;
        if (rest) {
            const unsigned sh = 16 * (k & 1u);
            x.w[k >> 1] = (x.w[k >> 1] & ~(0xFFFFu << sh)) | (v << sh);
            x.lanes |= ln << (4 * k);
        }
        rest &= rest - 1;
    }
    return x;
}

// Publish, for road ri of a flat sub-run (no repeated coordinate in a layer,
// so every hit index is canonical), the minimum key of every group (layer
// triple, three coordinates) whose three hits are flagged as shared with
// another road of the event.  The whole warp takes the groups.
__device__ void flat_publish(const Dev &d, const P3Flat &F, unsigned ri)
{
    const FlatRoad &r = F.rd[ri];
    const unsigned excl = fr_excl(r);
    // flagged hits of layer l: byte l of flp (no arrays indexed at run time)
    unsigned long long flp = 0;
#pragma unroll
    for (unsigned l = 0; l < N_LAYERS; ++l) {
        const unsigned n = (r.nl >> (4 * l)) & 15u;
        flp |= (r.xm & ((unsigned long long)((1u << n) - 1u) << (8 * l)));
    }
    const auto fl = [flp](unsigned l) { return (unsigned)(flp >> (8 * l)) & 0xFFu; };
    const auto groups = [&fl](unsigned t) {   // groups of triple t
        return __popc(fl(triple_l(t, 0))) * __popc(fl(triple_l(t, 1))) * __popc(fl(triple_l(t, 2)));
    };
    unsigned total = 0;
#pragma unroll
    for (unsigned t = 0; t < 10; ++t)
        total += groups(t);
    for (unsigned gi = lane_id(); gi < total; gi += 32) {
        unsigned t = 0, rem = gi;
        bool found = false;
#pragma unroll
        for (unsigned tt = 0; tt < 10; ++tt) {   // the triple of group gi
            const unsigned c = groups(tt);
            if (!found) {
                if (rem < c) {
                    t = tt;
                    found = true;
                } else {
                    rem -= c;
                }
            }
        }
        const unsigned lt[3] = {triple_l(t, 0), triple_l(t, 1), triple_l(t, 2)};
        const unsigned f0 = fl(lt[0]), f1 = fl(lt[1]), f2 = fl(lt[2]);
        const unsigned p0 = __popc(f0), p1 = __popc(f1);
        const unsigned dsel[3] = {nth_bit(f0, rem % p0), nth_bit(f1, (rem / p0) % p1), nth_bit(f2, rem / (p0 * p1))};
        unsigned long long mn = NO_KEY;
        if (lt[0] != excl && lt[1] != excl && lt[2] != excl) {
            // the free fitted slot runs over its hits, the three others are fixed
            unsigned fb = 0, free_slot = 0 + 1 + 2 + 3;
#pragma unroll
            for (unsigned q = 0; q < 3; ++q) {
                const unsigned sq_ = lt[q] - (lt[q] > excl);
                free_slot -= sq_;
                fb += dsel[q] * r.st[sq_];
            }
            for (unsigned z = 0; z < r.m[free_slot]; ++z) {
                const unsigned long long k = F.K[r.kb + fb + z * r.st[free_slot]];
                mn = k < mn ? k : mn;
            }
        } else {
            // the excluded layer in the triple: its lowest hit index of the
            // coordinate (the index itself, canonical) and the pair table
            unsigned de = 0, fa = 4, fb = 4, da = 0, db = 0;
#pragma unroll
            for (unsigned q = 0; q < 3; ++q) {
                if (lt[q] == excl) {
                    de = dsel[q];
                } else if (fa == 4) {
                    fa = lt[q] - (lt[q] > excl);
                    da = dsel[q];
                } else {
                    fb = lt[q] - (lt[q] > excl);
                    db = dsel[q];
                }
            }
            unsigned p = 0;
            while (p < 5 && !(pair_a(p) == fa && pair_b(p) == fb))
                ++p;
            const unsigned idx = r.off[p] + da * r.m[fb] + db;
            mn = ((unsigned long long)F.Qh[idx] << 32) | F.Ql[idx];
            if (mn != NO_KEY)
                mn += (unsigned long long)de * r.Se;
        }
        if (mn != NO_KEY)
            hash_min(d, group_key(r.event, t, F.co[ri][lt[0] * 8 + dsel[0]], F.co[ri][lt[1] * 8 + dsel[1]],
                                  F.co[ri][lt[2] * 8 + dsel[2]]),
                     mn);
    }
    __syncwarp();
}

// Survivors of one pass of a flat sub-run (every lane of the warp calls it):
// lane flags `surv` with its key and its road's lane ri (entries in order).
// A road's survivors take its slots in entry order.
__device__ __forceinline__ void flat_emit(const Dev &d, P3Flat &F, bool surv, unsigned ri,
                                          unsigned long long key)
{
    const unsigned lane = lane_id();
    if (!surv)
        ri = WARP_ROADS + lane;   // distinct per lane unless a survivor
    const unsigned sv = __ballot_sync(FULL_MASK, surv);
    if (!sv)
        return;
    const unsigned same = __match_any_sync(FULL_MASK, ri) & sv;
    unsigned pos = 0;
    if (surv)
        pos = F.cnt[ri] + __popc(same & lanemask_lt());
    __syncwarp();
    if (surv) {
        if (pos < SURV_SLOTS)
            d.surv_pool[surv_at(d, F.rd[ri].g, pos)] = key;
        else
            raise_flag(d, FLAG_INTERNAL);
        if ((same >> lane) == 1u)   // the last survivor of its road in this pass
            F.cnt[ri] = pos + 1;
    }
    __syncwarp();
}

// Fit roads g0 .. g0 + R - 1 (R <= WARP_ROADS) with one warp; `region` is
// the warp's shared memory.  Roads marked in P2 for a whole CTA are skipped.
template <bool PLAIN>
__device__ void fit_run(const Dev &d, unsigned char *region, unsigned g0, unsigned R,
                        unsigned long long &npass)
{
    P3Flat &F = *reinterpret_cast<P3Flat *>(region);
    const unsigned lane = lane_id();
    unsigned np32 = 0;   // passing combinations of the run (at most 8 x 256 x 8)

    // the run's records and coordinates
    RoadRec rec = {};
    unsigned N = 0, N4 = 0;
    if (lane < R) {
        rec = ldcg(d.roads + g0 + lane);
        road_sizes(rec.pk, N, N4);
    }
    {   // 80 bytes per road, five 16-byte words
        const uint4 *src = reinterpret_cast<const uint4 *>(d.coords + (size_t)g0 * 40);
        uint4 *dst = reinterpret_cast<uint4 *>(&F.co[0][0]);
        for (unsigned idx = lane; idx < R * N_LAYERS; idx += 32)
            dst[idx] = ldcg(src + idx);
    }
    __syncwarp();

    // lane i < R: the shape of road i (a road the CTAs fit is skipped),
    // written straight into the road's record in shared memory (slot i in
    // every sub-run), so that no per-lane array needs local memory
    const bool small = lane < R && N > 0 && !(rec.cta & 1u);
    unsigned E = 0, asum = 0, xl = 0;
    bool flat = false, dup_fit = false;
    if (small) {
        FlatRoad &w = F.rd[lane];
        const uint32_t pk = rec.pk;
        const unsigned excl = min((pk >> 20) & 7u, 4u);
        // fitted slots: the layers other than excl, in order.  Canonical hits
        // of each fitted layer: a repeated coordinate makes the pair tables
        // take canonical indices (dup_fit)
        unsigned S = 1, Se = 1, ne = 0, j = 0, st = 1;
        xl = excl | (((pk >> 23) & 1u) << 3);
        for (unsigned l = 0; l < N_LAYERS; ++l) {
            const unsigned nl_ = min((pk >> (4 * l)) & 15u, (unsigned)MAX_HITS);
            if (l == excl) {
                Se = S;
                ne = nl_;
            } else {
                xl |= l << (8 + 3 * j);
                unsigned map = CANON_ID;
                for (unsigned x = 1; x < ((rec.cta & 2u) ? nl_ : 0u); ++x) {   // P2 flags repeated coordinates
                    unsigned c = x;
                    for (unsigned y = x; y-- > 0;)   // the lowest equal index wins
                        c = F.co[lane][l * 8 + x] == F.co[lane][l * 8 + y] ? y : c;
                    map = (map & ~(7u << (3 * x))) | (c << (3 * x));
                }
                w.cm[j] = map;
                dup_fit = dup_fit || map != CANON_ID;
                w.m[j] = nl_;
                w.st[j] = st;
                w.SL[j] = S;
                w.aoff[j] = asum;
                asum += nl_;
                st *= nl_;
                ++j;
            }
            S *= nl_;
        }
        xl |= ne << 4;
        for (unsigned p = 0; p < 6; ++p) {
            w.off[p] = E;
            E += w.m[pair_a(p)] * w.m[pair_b(p)];
        }
        for (unsigned q = 0; q < 3; ++q)
            w.M[q] = c_magic[w.m[q]];
        w.g = g0 + lane;
        w.event = rec.event;
        w.xl = xl;
        w.nl = pk & 0xFFFFFu;
        w.Se = Se;
        w.N4 = N4;
        w.E = E;
        w.key_hi = rec.pk >> 24;
        w.set = min((unsigned)rec.set, (unsigned)(N_SETS - 1));
        w.curv = rec.curv;
        w.phi = rec.phi;
        w.cb = PLAIN ? ldcg(d.comb_off + g0 + lane) : 0ull;
        w.xm = ((pk >> 23) & 1u) ? ldcg(d.xmask + g0 + lane) : 0ull;   // loaded with the run
        // every road a warp takes fits the tables: N4 <= small_n4 <= FLAT_K,
        // and then E <= QTAB_SMALL and asum <= 32
        flat = N4 <= FLAT_K && E <= FLAT_Q && asum <= FLAT_A;
        if (!flat)
            raise_flag(d, FLAG_INTERNAL);
    }

    // flat sub-runs: a prefix of the remaining flat roads that fits the tables
    unsigned todo = __ballot_sync(FULL_MASK, flat);
    while (todo) {
        const bool mine = (todo >> lane) & 1u;
        unsigned ik = mine ? N4 : 0u, iq = mine ? E : 0u, ia = mine ? asum : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {   // inclusive prefix sums over the lanes
            const unsigned uk = __shfl_up_sync(FULL_MASK, ik, o);
            const unsigned uq = __shfl_up_sync(FULL_MASK, iq, o);
            const unsigned ua = __shfl_up_sync(FULL_MASK, ia, o);
            if ((int)lane >= o) {
                ik += uk;
                iq += uq;
                ia += ua;
            }
        }
        const bool take = mine && ik <= FLAT_K && iq <= FLAT_Q && ia <= FLAT_A;
        const unsigned sub = __ballot_sync(FULL_MASK, take);   // the first roads left
        const bool sdup = __any_sync(FULL_MASK, take && dup_fit);
        const unsigned s1 = 31 - __clz(sub);
        const unsigned nk = __shfl_sync(FULL_MASK, ik, s1), nq = __shfl_sync(FULL_MASK, iq, s1),
                       na = __shfl_sync(FULL_MASK, ia, s1);
        if (take) {   // the road's record joins the sub-run: offsets rebased on its tables
            FlatRoad &w = F.rd[lane];
            const unsigned qb = iq - E, ab = ia - asum;
            w.kb = ik - N4;
            w.qb = qb;
            w.ab = ab;
#pragma unroll
            for (unsigned p = 0; p < 6; ++p)
                w.off[p] += qb;
#pragma unroll
            for (unsigned jj = 0; jj < 4; ++jj)
                w.aoff[jj] += ab;
            F.cnt[lane] = 0;
        }
        const FlatIndex xk = flat_index(ik - N4, sub), xa = flat_index(ia - asum, sub);
        __syncwarp();

        // partial chi-square sums of every fitted hit of every road
        if (!PLAIN) {
            for (unsigned t = lane; t < na; t += 32) {
                const unsigned ri = xa.owner(t);
                const FlatRoad &r = F.rd[ri];
                const unsigned j = (t >= r.aoff[1]) + (t >= r.aoff[2]) + (t >= r.aoff[3]);
                const unsigned dd = t - r.aoff[j];
                const int h = F.co[ri][fr_layer(r, j) * 8 + dd];
                // column j of the set's C (one 16-byte load; columns 4, 5 and k for slot 0)
                const int4 *cc = d.fitc + SET_INT4 * r.set + SET_C;
                const int4 cj = __ldg(cc + j);
                int4 a;
                a.x = cj.x * h;
                a.y = cj.y * h;
                a.z = cj.z * h;
                a.w = 0;
                if (j == 0) {   // curvature, phi and 4096 * offset ride on slot 0
                    const int4 c4 = __ldg(cc + 4), c5 = __ldg(cc + 5), kk = __ldg(cc + 6);
                    a.x += c4.x * r.curv + c5.x * r.phi + 4096 * kk.x;
                    a.y += c4.y * r.curv + c5.y * r.phi + 4096 * kk.y;
                    a.z += c4.z * r.curv + c5.z * r.phi + 4096 * kk.z;
                }
                F.A[t] = a;
            }
            __syncwarp();
        }

        // pair tables start empty (the low words once they are needed)
        for (unsigned t = lane; t < nq; t += 32)
            F.Qh[t] = 0xFFFFFFFFu;
        __syncwarp();

        // keys of the distinct fits.  The pair tables hold the minimum key of
        // the fits with the same hits on two fitted slots; a 64-bit minimum
        // is taken in two 32-bit steps: the high words here, then, only if
        // a table has two keys with its minimum high word (a tie), the low
        // words of the keys whose high word is the minimum.  A key that
        // finds a lower high word already in one of its tables cannot be a
        // table's minimum there; the others ("maybe" keys) are listed in
        // entry order over the low words, unused until a tie.  The second
        // of two keys with the minimum high word of a table always finds
        // it there, so every tie at a minimum is seen.
        const long long cut = d.cut;
        uint16_t *ml = reinterpret_cast<uint16_t *>(F.Ql);
        static_assert(sizeof(F.Ql) >= FLAT_K * sizeof(uint16_t), "maybe list fits over Ql");
        unsigned nmaybe = 0;
        bool tie = false;
        for (unsigned base = 0; base < nk; base += 32) {
            const unsigned t = base + lane;
            bool maybe = false;
            if (t < nk) {
                const unsigned ri = xk.owner(t);
                const FlatRoad &r = F.rd[ri];
                const unsigned f = t - r.kb;
                const unsigned q0 = divm(f, r.M[0]), f0 = f - q0 * r.m[0];
                const unsigned q1 = divm(q0, r.M[1]), f1 = q0 - q1 * r.m[1];
                const unsigned f3 = divm(q1, r.M[2]), f2 = q1 - f3 * r.m[2];
                const unsigned comb = f0 * r.SL[0] + f1 * r.SL[1] + f2 * r.SL[2] + f3 * r.SL[3];
                unsigned long long key;
                if (PLAIN) {
                    key = ldcg(d.fit_key + r.cb + comb);
                } else {
                    const int4 a0 = F.A[r.aoff[0] + f0], a1 = F.A[r.aoff[1] + f1];
                    const int4 a2 = F.A[r.aoff[2] + f2], a3 = F.A[r.aoff[3] + f3];
                    const int sx = a0.x + a1.x + a2.x + a3.x;
                    const int sy = a0.y + a1.y + a2.y + a3.y;
                    const int sz = a0.z + a1.z + a2.z + a3.z;
                    const long long chi2 = sq(sx >> 12) + sq(sy >> 12) + sq(sz >> 12);
                    const bool pass = chi2 <= cut;
                    np32 += pass ? fr_ne(r) : 0u;
                    key = pass ? make_key(chi2, r.key_hi, comb) : NO_KEY;
                }
                // pair tables take canonical hits (a sub-run with a repeated
                // coordinate maps them; elsewhere they are the hits)
                unsigned fd[4] = {f0, f1, f2, f3};
                if (sdup) {
#pragma unroll
                    for (unsigned jj = 0; jj < 4; ++jj)
                        fd[jj] = (r.cm[jj] >> (3 * fd[jj])) & 7u;
                }
                F.K[t] = key;
                F.dig[t] = (uint16_t)(fd[0] | (fd[1] << 3) | (fd[2] << 6) | (fd[3] << 9) | (ri << 12));
                if (key != NO_KEY) {
                    const unsigned hi = (unsigned)(key >> 32);
                    maybe = true;
#pragma unroll
                    for (unsigned p = 0; p < 6; ++p) {
                        const unsigned a = pair_a(p), b = pair_b(p);
                        const unsigned old = atomicMin(&F.Qh[r.off[p] + fd[a] * r.m[b] + fd[b]], hi);
                        maybe = maybe && old >= hi;
                        tie = tie || old == hi;
                    }
                }
            }
            const unsigned mb = __ballot_sync(FULL_MASK, maybe);
            if (maybe)
                ml[nmaybe + __popc(mb & lanemask_lt())] = (uint16_t)t;
            nmaybe += __popc(mb);
        }
        const bool ties = __any_sync(FULL_MASK, tie);
        __syncwarp();

        // candidates: keys whose high word is the minimum of all six
        // tables.  Without a tie a candidate is a survivor and is written at
        // once; after a tie the candidates are listed in entry order over the
        // partial sums (no longer needed) for the low-word test.
        uint16_t *cl = reinterpret_cast<uint16_t *>(F.A);
        static_assert(sizeof(F.A) >= FLAT_K * sizeof(uint16_t), "candidate list fits over A");
        unsigned ncand = 0;
        if (!ties) {
            for (unsigned base = 0; base < nmaybe; base += 32) {
                const unsigned i = base + lane;
                bool cand = false;
                unsigned t = 0;
                unsigned long long key = NO_KEY;
                unsigned ri = 0;
                if (i < nmaybe) {
                    t = ml[i];
                    key = F.K[t];
                    const unsigned hi = (unsigned)(key >> 32);
                    const unsigned dg = F.dig[t];
                    ri = dg >> 12;
                    const FlatRoad &r = F.rd[ri];
                    const unsigned fd[4] = {dg & 7u, (dg >> 3) & 7u, (dg >> 6) & 7u, (dg >> 9) & 7u};
                    cand = true;
#pragma unroll
                    for (unsigned p = 0; p < 6; ++p) {
                        const unsigned a = pair_a(p), b = pair_b(p);
                        cand = cand && F.Qh[r.off[p] + fd[a] * r.m[b] + fd[b]] == hi;
                    }
                }
                // without a tie a candidate is a survivor: written now (the
                // maybe keys are in entry order)
                flat_emit(d, F, cand, ri, key);
            }
        } else {
            // a tie: the low words start empty (the list over them is
            // dropped) and every key with a table's minimum high word
            // takes part in that table's low-word minimum
            for (unsigned t = lane; t < nq; t += 32)
                F.Ql[t] = 0xFFFFFFFFu;
            __syncwarp();
            for (unsigned base = 0; base < nk; base += 32) {
                const unsigned t = base + lane;
                bool cand = false;
                if (t < nk) {
                    const unsigned long long key = F.K[t];
                    if (key != NO_KEY) {
                        const unsigned dg = F.dig[t];
                        const FlatRoad &r = F.rd[dg >> 12];
                        const unsigned fd[4] = {dg & 7u, (dg >> 3) & 7u, (dg >> 6) & 7u, (dg >> 9) & 7u};
                        const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
                        cand = true;
#pragma unroll
                        for (unsigned p = 0; p < 6; ++p) {
                            const unsigned a = pair_a(p), b = pair_b(p);
                            const unsigned idx = r.off[p] + fd[a] * r.m[b] + fd[b];
                            if (F.Qh[idx] == hi)
                                atomicMin(&F.Ql[idx], lo);
                            else
                                cand = false;
                        }
                    }
                }
                const unsigned cb = __ballot_sync(FULL_MASK, cand);
                if (cand)
                    cl[ncand + __popc(cb & lanemask_lt())] = (uint16_t)t;
                ncand += __popc(cb);
            }
        }
        __syncwarp();

        // after a tie: survivors are the candidates that also hold the low
        // word of all six tables (in entry order)
        for (unsigned base = 0; base < ncand; base += 32) {
            const unsigned i = base + lane;
            unsigned ri = 0;
            bool surv = false;
            unsigned long long key = NO_KEY;
            if (i < ncand) {
                const unsigned t = cl[i];
                const unsigned dg = F.dig[t];
                ri = dg >> 12;
                const FlatRoad &r = F.rd[ri];
                const unsigned fd[4] = {dg & 7u, (dg >> 3) & 7u, (dg >> 6) & 7u, (dg >> 9) & 7u};
                key = F.K[t];
                const unsigned lo = (unsigned)key;
                surv = true;
#pragma unroll
                for (unsigned p = 0; p < 6; ++p) {
                    const unsigned a = pair_a(p), b = pair_b(p);
                    surv = surv && F.Ql[r.off[p] + fd[a] * r.m[b] + fd[b]] == lo;
                }
            }
            flat_emit(d, F, surv, ri, key);
        }
        {
            // survivor counts of the sub-run's roads, and their sums per road
            // chunk (a run spans at most two chunks)
            const bool in_sub = (sub >> lane) & 1u;
            const unsigned v = in_sub ? min(F.cnt[lane], (unsigned)SURV_SLOTS) : 0u;
            if (in_sub)
                d.surv_cnt[g0 + lane] = (uint8_t)v;
            const unsigned ch0 = g0 / ROAD_CHUNK;
            const bool second = (g0 + lane) / ROAD_CHUNK != ch0;
            const unsigned s0 = __reduce_add_sync(FULL_MASK, second ? 0u : v);
            const unsigned s1 = __reduce_add_sync(FULL_MASK, second ? v : 0u);
            if (lane == 0 && s0)
                atomicAdd(&d.rchunk_sum[ch0], s0);
            if (lane == 0 && s1)
                atomicAdd(&d.rchunk_sum[ch0 + 1], s1);
        }
        // cross-road candidates of the sub-run publish their group minima,
        // which read whole keys from the pair tables.  Without a tie the low
        // words were not taken: each table's minimum high word belongs to
        // one key, which writes its low word.
        const unsigned cands = __ballot_sync(FULL_MASK, ((sub >> lane) & 1u) && (xl & 8u));
        if (cands && !ties) {
            for (unsigned t = lane; t < nq; t += 32)
                F.Ql[t] = 0xFFFFFFFFu;
            __syncwarp();
            for (unsigned t = lane; t < nk; t += 32) {
                const unsigned long long key = F.K[t];
                if (key == NO_KEY)
                    continue;
                const unsigned dg = F.dig[t];
                const FlatRoad &r = F.rd[dg >> 12];
                const unsigned fd[4] = {dg & 7u, (dg >> 3) & 7u, (dg >> 6) & 7u, (dg >> 9) & 7u};
                const unsigned hi = (unsigned)(key >> 32);
#pragma unroll
                for (unsigned p = 0; p < 6; ++p) {
                    const unsigned a = pair_a(p), b = pair_b(p);
                    const unsigned idx = r.off[p] + fd[a] * r.m[b] + fd[b];
                    if (F.Qh[idx] == hi)
                        F.Ql[idx] = (unsigned)key;
                }
            }
            __syncwarp();
        }
        for (unsigned c = cands; c; c &= c - 1)
            flat_publish(d, F, __ffs(c) - 1);
        todo &= ~sub;
        __syncwarp();
    }
    npass += np32;
}

// shared memory of one warp in the warp part of P3
constexpr size_t P3_WARP_BYTES = (sizeof(P3Flat) + 15) / 16 * 16;

// ---------------------------------------------------------------------------
// P3, box path: one warp fits one listed road (more distinct fits than
// small_n4, or a cross-road candidate with a repeated coordinate).
//
// Hits with one coordinate in one layer are one hit for the warrior (hits
// are shared by value), and among fits with the same coordinates the lowest
// hit index has the lowest comb.  So every pair-table minimum and every
// road-local survivor takes canonical hits only (the lowest index of each
// coordinate), and the warp works on the box of canonical fits.  The four
// fitted slots get roles (a, b, c, e); in pass p, lane t = 32 p + lane takes
// the pair (x, y) = (t mod m_a, t div m_a) of slots a and b and loops over
// (z, w) of slots c and e.  Of the six pair tables (minimum key over the
// fits with the same canonical hits on two slots) that loop makes three:
//   T_ab[x][y]  the lane's minimum over its own fits
//   T_ac, T_bc  the lane's minimum over w at each z, folded over the lanes
// A pair's minimum that holds T_ac and T_bc (about one per road) is then
// checked against the other three, taken on demand by a warp-wide minimum
// over the other two slots' hits (box_min2), as are the entries the
// publish step reads:
//   T_ae, T_be, T_ce  (folding T_ae and T_be in the loop held sixteen more
//               registers there and measured slower)
// The lane minima are folded by 32-bit shared-memory atomics without a
// return value, each pass into tables of its own: the high words first,
// then, after the warp has synchronised, the low words of the lanes whose
// high word is the minimum.  That is the exact minimum of the 64-bit keys
// over the pass (every lane of the pass takes part in the same steps); the
// survivor check takes the smaller of the two passes' entries.  (64-bit
// atomic minima, and folds through scratch rows or warp shuffles, measured
// slower.)
// A fit survives the road-local warrior iff its key is the minimum of all
// six (see the flat path); it is then the minimum of its pair (x, y), so a
// pair has at most one candidate and a road at most 64 survivors.
// ---------------------------------------------------------------------------

enum { T_AB = 0, T_CE, T_AC, T_BC, T_AE, T_BE, N_TAB };
// table row stride: rows 9 entries apart put the entries [u][v] of
// different u in different banks
constexpr unsigned TS = 9;

struct P3Box {
    unsigned long long T[2][8 * TS];   // T_ab, T_ce: [u * TS + v] (u: the first role's hit); T_ce
                                       // only where needed (box_tce)
    unsigned H[2][4][8 * TS];          // T_ac, T_bc of pass 0 and pass 1: high words; T_ae, T_be:
                                       // the entries taken on demand for the publish step (pass 0)
    unsigned L[2][4][8 * TS];          // and low words (of the keys with the minimum high word)
    int4 A[4][8];                      // slot j, canonical hit k: chi-square partial sums (x, y,
                                       // z) and comb part (w); slot 0 also carries curvature, phi,
                                       // 4096 k and the road bits of the key
    uint16_t co[40];                   // the road's coordinates, [layer * 8 + hit]
    uint8_t raw[4][8];                 // raw hit index of canonical hit k of slot j
    uint8_t rank[4][8];                // canonical hit (class) of raw hit d of slot j
    uint8_t mult[4][8];                // raw hits sharing the coordinate of canonical hit k
};
static_assert(offsetof(P3Box, A) % 16 == 0 && offsetof(P3Box, co) % 16 == 0, "16-byte rows");

__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b)
{
    return b < a ? b : a;
}

// entry idx of pair table tab: T_ab and T_ce as stored, the others the
// smaller of the two passes' (high, low) entries
__device__ __forceinline__ unsigned long long box_get(const P3Box &B, unsigned tab, unsigned idx)
{
    if (tab < 2)
        return B.T[tab][idx];
    const unsigned t = tab - 2;
    return umin64(((unsigned long long)B.H[0][t][idx] << 32) | B.L[0][t][idx],
                  ((unsigned long long)B.H[1][t][idx] << 32) | B.L[1][t][idx]);
}

// Fold v into entry idx of table t of pass q, stage 1 (high word); stage 2
// (low word) runs after the warp has synchronised: only lanes whose high
// word is then the minimum take part.
__device__ __forceinline__ void fold_hi(P3Box &B, unsigned q, unsigned t, unsigned idx, unsigned long long v)
{
    atomicMin(&B.H[q][t][idx], (unsigned)(v >> 32));
}
__device__ __forceinline__ void fold_lo(P3Box &B, unsigned q, unsigned t, unsigned idx, unsigned long long v)
{
    if ((unsigned)(v >> 32) == B.H[q][t][idx])
        atomicMin(&B.L[q][t][idx], (unsigned)v);
}

// hits of layer l of a road record (clamped to the format limit)
__device__ __forceinline__ unsigned hits_of(uint32_t pk, unsigned l)
{
    return min((pk >> (4 * l)) & 15u, (unsigned)MAX_HITS);
}

// Key of a fit from its summed partials s: (chi2, road bits and comb), or
// NO_KEY when it fails the cut.  s.x, s.y, s.z are 4096 times the three
// chi-square components before the floor (exact in int32, see the header);
// s.w is road << 15 | comb.
__device__ __forceinline__ unsigned long long box_key(const int4 &s, long long cut, bool &pass)
{
    const long long chi2 = sq(s.x >> 12) + sq(s.y >> 12) + sq(s.z >> 12);
    pass = chi2 <= cut;
    return pass ? (((unsigned long long)chi2 << 23) | (unsigned)s.w) : NO_KEY;
}

__device__ __forceinline__ int4 add4(const int4 &a, const int4 &b)
{
    return make_int4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// Shape of a road in the box path, the same in every lane.
struct BoxShape {
    unsigned mpk;              // canonical hits of fitted slot j in bits 4j .. 4j + 3
    unsigned ra, rb, rc, re;   // the slots in roles a, b, c, e
    unsigned ma, mb, mc, me;   // their canonical hits
    unsigned ne;               // raw hits of the excluded layer
    unsigned long long cb;     // plain mode: first combination of the road
    __device__ unsigned m(unsigned s) const { return (mpk >> (4 * s)) & 15u; }
};

// Key of the fit with summed partials s (without the comb) and comb part
// cw, or NO_KEY when it fails the cut or `live` is false.  The comb occupies
// bits below the chi-square's shifted bits, so it is added, not or-ed.
__device__ __forceinline__ unsigned long long box_key2(const int4 &s, unsigned cw, long long cut, bool live,
                                                       bool &ok)
{
    const long long chi2 = sq(s.x >> 12) + sq(s.y >> 12) + sq(s.z >> 12);
    ok = live && chi2 <= cut;
    const unsigned hi = (unsigned)((unsigned long long)chi2 >> 9);
    const unsigned lo = ((unsigned)chi2 << 23) + cw;
    return ok ? ((unsigned long long)hi << 32) | lo : NO_KEY;
}

// The key of a fit without the cut: chi2 << 23 | cw (the cut is key < kb).
__device__ __forceinline__ unsigned long long box_key_raw(const int4 &s, unsigned cw)
{
    const long long chi2 = sq(s.x >> 12) + sq(s.y >> 12) + sq(s.z >> 12);
    const unsigned hi = (unsigned)((unsigned long long)chi2 >> 9);
    const unsigned lo = ((unsigned)chi2 << 23) + cw;
    return ((unsigned long long)hi << 32) | lo;
}

// One pass over the pairs (x, y) of slots a and b: lane t = 32 p + lane.
// The inner loop over the hits of slot e has ME (4 or 8, at least me) steps,
// unrolled and predicated, so a step has no branch.  DUP: the road has
// repeated coordinates (passing counts are weighted by the raw fits each
// canonical fit stands for).  T_ce is not made here (see box_tce).
template <bool PLAIN, bool DUP, unsigned ME, bool FULLW>
__device__ void box_pass(const Dev &d, P3Box &B, const BoxShape &sh, unsigned p, unsigned &np)
{
    const unsigned lane = lane_id();
    const unsigned ma = sh.ma, mb = sh.mb, mc = sh.mc, me = sh.me;
    const unsigned t = p * 32 + lane;
    const bool act = t < ma * mb;
    const unsigned y = act ? divm(t, c_magic[ma]) : 0u, x = act ? t - y * ma : 0u;
    const int4 pab = add4(B.A[sh.ra][x], B.A[sh.rb][y]);
    const unsigned wab = DUP ? (unsigned)B.mult[sh.ra][x] * B.mult[sh.rb][y] : 1u;
    const long long cut = d.cut;
    // full passes compare raw keys with kb: chi2 <= cut iff key < kb; a
    // minimum of kb or more means no passing fit (NO_KEY when stored)
    const unsigned long long kb = cut < 0 ? 0ull : (unsigned long long)(min(cut, 1ll << 40) + 1) << 23;
    const auto cut_min = [kb](unsigned long long v) { return FULLW && v >= kb ? NO_KEY : v; };
    const int4 *Ae = B.A[sh.re];
    bool live[ME];
#pragma unroll
    for (unsigned w = 0; w < ME; ++w)
        live[w] = FULLW || (act && w < me);   // full passes of 8-hit slots e: every lane, every w
    unsigned long long qab = NO_KEY;
    for (unsigned z = 0; z < mc; ++z) {
        const int4 pz = add4(pab, B.A[sh.rc][z]);
        const unsigned wz = DUP ? wab * B.mult[sh.rc][z] : 1u;
        unsigned long long rz = NO_KEY;
#pragma unroll
        for (unsigned w = 0; w < ME; ++w) {
            const int4 aw = Ae[w];
            unsigned long long key;
            if (PLAIN) {
                key = live[w] ? ldcg(d.fit_key + sh.cb + (unsigned)(pz.w + aw.w)) : NO_KEY;
            } else {
                const int4 s = make_int4(pz.x + aw.x, pz.y + aw.y, pz.z + aw.z, 0);
                if (FULLW) {
                    key = box_key_raw(s, (unsigned)pz.w + (unsigned)aw.w);
                    np += key < kb;
                } else {
                    bool ok;
                    key = box_key2(s, (unsigned)pz.w + (unsigned)aw.w, cut, live[w], ok);
                    if (DUP)
                        np += ok ? wz * B.mult[sh.re][w] : 0u;
                    else
                        np += ok;
                }
            }
            rz = umin64(rz, key);
        }
        qab = umin64(qab, rz);
        rz = cut_min(rz);
        const unsigned q = p & 1u;
        if (act) {
            fold_hi(B, q, T_AC - 2, x * TS + z, rz);
            fold_hi(B, q, T_BC - 2, y * TS + z, rz);
        }
        __syncwarp();
        if (act) {
            fold_lo(B, q, T_AC - 2, x * TS + z, rz);
            fold_lo(B, q, T_BC - 2, y * TS + z, rz);
        }
    }
    if (act)
        B.T[T_AB][x * TS + y] = cut_min(qab);
    __syncwarp();
}

// The minimum key over the fits with canonical hit kp of slot sp and kq of
// slot sq (sp != sq), taken on demand by the warp: lanes over the canonical
// hits of the other two slots (every lane calls it with the same arguments;
// the result is the same in every lane).  Gives T_ae, T_be and T_ce, which
// the passes do not fold.
template <bool PLAIN>
__device__ unsigned long long box_min2(const Dev &d, const P3Box &B, const BoxShape &sh, unsigned sp, unsigned kp,
                                       unsigned sq, unsigned kq)
{
    const unsigned lane = lane_id();
    const unsigned rest = 0xFu & ~(1u << sp) & ~(1u << sq);
    const unsigned su = __ffs(rest) - 1, sv = 31 - __clz(rest);
    const unsigned mu = sh.m(su), mv = sh.m(sv);
    const int4 pf = add4(B.A[sp][kp], B.A[sq][kq]);
    unsigned long long mn = NO_KEY;
    for (unsigned t = lane; t < mu * mv; t += 32) {
        const unsigned iv = divm(t, c_magic[mu]), iu = t - iv * mu;
        const int4 s = add4(pf, add4(B.A[su][iu], B.A[sv][iv]));
        unsigned long long key;
        if (PLAIN) {
            key = ldcg(d.fit_key + sh.cb + (unsigned)s.w);
        } else {
            bool ok;
            key = box_key2(s, (unsigned)s.w, d.cut, true, ok);
        }
        mn = umin64(mn, key);
    }
    const unsigned hi = (unsigned)(mn >> 32);
    const unsigned mh = __reduce_min_sync(FULL_MASK, hi);
    const unsigned ml = __reduce_min_sync(FULL_MASK, hi == mh ? (unsigned)mn : 0xFFFFFFFFu);
    return ((unsigned long long)mh << 32) | ml;
}

// T_ce[z][w]: the minimum key over every pair (x, y) at hits z, w of slots c and e
template <bool PLAIN>
__device__ __forceinline__ unsigned long long box_tce(const Dev &d, const P3Box &B, const BoxShape &sh, unsigned z,
                                                      unsigned w)
{
    return box_min2<PLAIN>(d, B, sh, sh.rc, z, sh.re, w);
}

// the table holding the minima over slots p and q (p != q) and the index of
// canonical hits (kp, kq) in it
__device__ __forceinline__ unsigned box_tab(const BoxShape &sh, unsigned p, unsigned kp, unsigned q, unsigned kq,
                                            unsigned &idx)
{
    const auto role = [&sh](unsigned s) {
        return s == sh.ra ? 0u : s == sh.rb ? 1u : s == sh.rc ? 2u : 3u;
    };
    unsigned r1 = role(p), r2 = role(q), k1 = kp, k2 = kq;
    if (r1 > r2) {
        const unsigned tr = r1, tk = k1;
        r1 = r2;
        k1 = k2;
        r2 = tr;
        k2 = tk;
    }
    idx = k1 * TS + k2;
    // role pairs (0,1) ab, (2,3) ce, (0,2) ac, (1,2) bc, (0,3) ae, (1,3) be
    return r1 == 0 && r2 == 1 ? T_AB : r1 == 2 ? T_CE : r2 == 2 ? (r1 == 0 ? T_AC : T_BC) : (r1 == 0 ? T_AE : T_BE);
}

// Fit road g with one warp (see above); adds its passing combinations to npass.
template <bool PLAIN>
__device__ void box_road(const Dev &d, unsigned char *region, unsigned g, unsigned long long &npass)
{
    P3Box &B = *reinterpret_cast<P3Box *>(region);
    const unsigned lane = lane_id();
    const RoadRec rec = ldcg(d.roads + g);
    const uint32_t pk = rec.pk;
    const unsigned excl = min((pk >> 20) & 7u, 4u);
    __syncwarp();   // the region's previous user is done
    if (lane < N_LAYERS)   // 80 bytes of coordinates, five 16-byte words
        reinterpret_cast<uint4 *>(B.co)[lane] = ldcg(reinterpret_cast<const uint4 *>(d.coords + (size_t)g * 40) + lane);
    for (unsigned i = lane; i < 2 * 8 * TS; i += 32)
        (&B.T[0][0])[i] = NO_KEY;
    for (unsigned i = lane; i < 2 * 2 * 4 * 8 * TS; i += 32)   // H and L
        (&B.H[0][0][0])[i] = 0xFFFFFFFFu;
    __syncwarp();

    // lane 8 j + h: raw hit h of fitted slot j.  Canonical hits, their ranks
    // and multiplicities, and the partial sums of the canonical hits.
    const unsigned j = lane >> 3, h = lane & 7u;
    const unsigned L = j + (j >= excl);
    const unsigned nj = hits_of(pk, L);
    const bool valid = h < nj;
    unsigned cls = h;   // the lowest index with the same coordinate
    if (valid) {
        const unsigned v = B.co[L * 8 + h];
        for (unsigned x = h; x-- > 0;)
            cls = B.co[L * 8 + x] == v ? x : cls;
    }
    const bool canon = valid && cls == h;
    const unsigned cm = __ballot_sync(FULL_MASK, canon);
    const bool dup = __ballot_sync(FULL_MASK, valid) != cm;
    const unsigned mine = (cm >> (8 * j)) & 0xFFu;
    const unsigned same = __match_any_sync(FULL_MASK, valid ? j * 8 + cls : 32u + lane);
    const unsigned k = __popc(mine & ((1u << h) - 1u));
    if (valid)
        B.rank[j][h] = (uint8_t)__popc(mine & ((1u << cls) - 1u));
    BoxShape sh;
    sh.mpk = 0;
#pragma unroll
    for (unsigned s = 0; s < 4; ++s)
        sh.mpk |= (unsigned)__popc((cm >> (8 * s)) & 0xFFu) << (4 * s);
    sh.ne = hits_of(pk, excl);
    sh.cb = PLAIN ? ldcg(d.comb_off + g) : 0ull;
    if (canon) {
        unsigned SL = 1;   // comb stride of layer L
        for (unsigned l = 0; l < L; ++l)
            SL *= hits_of(pk, l);
        B.raw[j][k] = (uint8_t)h;
        B.mult[j][k] = (uint8_t)__popc(same);
        int4 a = make_int4(0, 0, 0, (int)(h * SL));
        if (!PLAIN) {
            const int4 *cc = d.fitc + SET_INT4 * min((unsigned)rec.set, (unsigned)(N_SETS - 1)) + SET_C;
            const int4 cj = __ldg(cc + j);
            const int hv = B.co[L * 8 + h];
            a.x = cj.x * hv;
            a.y = cj.y * hv;
            a.z = cj.z * hv;
            if (j == 0) {   // curvature, phi, 4096 * offset and the road bits ride on slot 0
                const int4 c4 = __ldg(cc + 4), c5 = __ldg(cc + 5), kk = __ldg(cc + 6);
                a.x += c4.x * rec.curv + c5.x * rec.phi + 4096 * kk.x;
                a.y += c4.y * rec.curv + c5.y * rec.phi + 4096 * kk.y;
                a.z += c4.z * rec.curv + c5.z * rec.phi + 4096 * kk.z;
                a.w += (int)((pk >> 24) << 15);
            }
        }
        B.A[j][k] = a;
    }
    // roles: the pair (a, b) that needs the fewest lane steps, then c before
    // e with e (the unrolled inner loop) the larger
    {
        const unsigned n4 = sh.m(0) * sh.m(1) * sh.m(2) * sh.m(3);
        unsigned best = ~0u, ba = 0, bb = 1;
#pragma unroll
        for (unsigned q = 0; q < 6; ++q) {
            const unsigned pa = pair_a(q), pb = pair_b(q);
            const unsigned prod = sh.m(pa) * sh.m(pb);
            const unsigned cost = (prod + 31) / 32 * (n4 / prod);
            if (cost < best) {
                best = cost;
                ba = pa;
                bb = pb;
            }
        }
        const unsigned rest = 0xFu & ~(1u << ba) & ~(1u << bb);
        const unsigned r0 = __ffs(rest) - 1, r1 = 31 - __clz(rest);
        const bool sw = sh.m(r0) > sh.m(r1);
        sh.ra = ba;
        sh.rb = bb;
        sh.rc = sw ? r1 : r0;
        sh.re = sw ? r0 : r1;
        sh.ma = sh.m(sh.ra);
        sh.mb = sh.m(sh.rb);
        sh.mc = sh.m(sh.rc);
        sh.me = sh.m(sh.re);
    }
    __syncwarp();

    // the loop over the box: every table but T_ce
    const unsigned ma = sh.ma, mb = sh.mb, me = sh.me;
    const unsigned passes = (ma * mb + 31) / 32;   // 1 or 2
    unsigned np = 0;
    // full passes and all eight hits of slot e (every 8^4 road): no per-step predicate
    const bool fullw = (ma * mb) % 32 == 0 && me == 8 && !dup;
    for (unsigned p = 0; p < passes; ++p) {
        if (fullw)
            box_pass<PLAIN, false, 8, true>(d, B, sh, p, np);
        else if (me > 4) {
            if (dup)
                box_pass<PLAIN, true, 8, false>(d, B, sh, p, np);
            else
                box_pass<PLAIN, false, 8, false>(d, B, sh, p, np);
        } else {
            if (dup)
                box_pass<PLAIN, true, 4, false>(d, B, sh, p, np);
            else
                box_pass<PLAIN, false, 4, false>(d, B, sh, p, np);
        }
    }
    __syncwarp();
    if (!PLAIN)
        npass += (unsigned long long)np * sh.ne;

    // road-local survivors: the minimum of pair (x, y) survives iff it is
    // also the minimum of its other five tables; T_ce (the minimum over all
    // pairs at its hits of slots c and e) is taken last, for the pairs that
    // pass the other four, by the whole warp
    unsigned long long sk[2] = {NO_KEY, NO_KEY};
    bool sv[2] = {false, false};
    unsigned zw[2] = {0u, 0u};
#pragma unroll
    for (unsigned p = 0; p < 2; ++p) {
        const unsigned t = p * 32 + lane;
        if (p < passes && t < ma * mb) {
            const unsigned y = divm(t, c_magic[ma]), x = t - y * ma;
            const unsigned long long key = B.T[T_AB][x * TS + y];
            if (key != NO_KEY) {
                // raw hits of the layers of slots c and e from the comb
                unsigned rest = (unsigned)(key & 0x7FFFu), dc = 0, de = 0;
                const unsigned Lc = sh.rc + (sh.rc >= excl), Le = sh.re + (sh.re >= excl);
#pragma unroll
                for (unsigned l = 0; l < N_LAYERS; ++l) {
                    const unsigned n = max(hits_of(pk, l), 1u);
                    const unsigned q = divm(rest, c_magic[n]);
                    const unsigned dl = rest - q * n;
                    rest = q;
                    dc = l == Lc ? dl : dc;
                    de = l == Le ? dl : de;
                }
                const unsigned z = B.rank[sh.rc][dc], w = B.rank[sh.re][de];
                sv[p] = box_get(B, T_AC, x * TS + z) == key && box_get(B, T_BC, y * TS + z) == key;
                sk[p] = key;
                zw[p] = x | (y << 3) | (z << 6) | (w << 9);
            }
        }
    }
#pragma unroll
    for (unsigned p = 0; p < 2; ++p) {
        for (unsigned bits = __ballot_sync(FULL_MASK, sv[p]); bits; bits &= bits - 1) {
            const unsigned src = __ffs(bits) - 1;
            const unsigned e = __shfl_sync(FULL_MASK, zw[p], src);
            const unsigned long long key = __shfl_sync(FULL_MASK, sk[p], src);
            const unsigned x = e & 7u, y = (e >> 3) & 7u, z = (e >> 6) & 7u, w = e >> 9;
            // T_ae, T_be, T_ce of the candidate, on demand (each one only if
            // the ones before hold the key)
            bool ok = box_min2<PLAIN>(d, B, sh, sh.ra, x, sh.re, w) == key;
            ok = ok && box_min2<PLAIN>(d, B, sh, sh.rb, y, sh.re, w) == key;
            ok = ok && box_tce<PLAIN>(d, B, sh, z, w) == key;
            if (lane == src)
                sv[p] = ok;
        }
    }
    // survivors in comb order: each finds its rank among the others
    const unsigned s0 = __ballot_sync(FULL_MASK, sv[0]), s1 = __ballot_sync(FULL_MASK, sv[1]);
    const unsigned n_surv = __popc(s0) + __popc(s1);
    unsigned rk[2] = {0u, 0u};
    const unsigned my0 = (unsigned)(sk[0] & 0x7FFFu), my1 = (unsigned)(sk[1] & 0x7FFFu);
    for (unsigned q = 0; q < 2; ++q) {
        for (unsigned bits = q ? s1 : s0; bits; bits &= bits - 1) {
            const unsigned src = __ffs(bits) - 1;
            const unsigned other = __shfl_sync(FULL_MASK, q ? my1 : my0, src);
            rk[0] += other < my0;
            rk[1] += other < my1;
        }
    }
#pragma unroll
    for (unsigned p = 0; p < 2; ++p)
        if (sv[p])
            d.surv_pool[surv_at(d, g, rk[p])] = sk[p];
    if (lane == 0) {
        d.surv_cnt[g] = (uint8_t)n_surv;
        if (n_surv)
            atomicAdd(&d.rchunk_sum[g / ROAD_CHUNK], n_surv);
    }

    // cross-road candidates: the minimum key of every group (layer triple,
    // three coordinates) whose three hits are canonical and flagged as
    // present in another road of the event
    if ((pk >> 23) & 1u) {
        // canonical hits of the excluded layer (lanes 0..7)
        unsigned xc = lane;
        const bool xv = lane < sh.ne;
        if (xv) {
            const unsigned v = B.co[excl * 8 + lane];
            for (unsigned x = lane; x-- > 0;)
                xc = B.co[excl * 8 + x] == v ? x : xc;
        }
        const unsigned cmx = __ballot_sync(FULL_MASK, xv && xc == lane) & 0xFFu;
        const unsigned long long xm = ldcg(d.xmask + g);
        unsigned long long flp = 0;
#pragma unroll
        for (unsigned l = 0; l < N_LAYERS; ++l) {
            const unsigned cl = l == excl ? cmx : (cm >> (8 * (l - (l > excl)))) & 0xFFu;
            flp |= (unsigned long long)((unsigned)(xm >> (8 * l)) & cl) << (8 * l);
        }
        const auto fl = [flp](unsigned l) { return (unsigned)(flp >> (8 * l)) & 0xFFu; };
        const auto groups = [&fl](unsigned t) {
            return __popc(fl(triple_l(t, 0))) * __popc(fl(triple_l(t, 1))) * __popc(fl(triple_l(t, 2)));
        };
        unsigned total = 0;
#pragma unroll
        for (unsigned t = 0; t < 10; ++t)
            total += groups(t);
        {   // the entries of the tables the passes do not fold (T_ae, T_be,
            // T_ce) that groups of (excluded layer, slot p, slot e) read
            if (fl(excl)) {
                const unsigned Le = sh.re + (sh.re >= excl), fe = fl(Le);
#pragma unroll
                for (unsigned q = 0; q < 3; ++q) {
                    const unsigned sp = q == 0 ? sh.ra : q == 1 ? sh.rb : sh.rc;
                    const unsigned Lp = sp + (sp >= excl);
                    for (unsigned bp = fl(Lp); bp; bp &= bp - 1)
                        for (unsigned be = fe; be; be &= be - 1) {
                            const unsigned kp = B.rank[sp][__ffs(bp) - 1], w = B.rank[sh.re][__ffs(be) - 1];
                            const unsigned long long m = box_min2<PLAIN>(d, B, sh, sp, kp, sh.re, w);
                            if (lane == 0) {
                                if (q == 2) {
                                    B.T[T_CE][kp * TS + w] = m;
                                } else {   // read by box_get as the first pass's entry
                                    B.H[0][q == 0 ? T_AE - 2 : T_BE - 2][kp * TS + w] = (unsigned)(m >> 32);
                                    B.L[0][q == 0 ? T_AE - 2 : T_BE - 2][kp * TS + w] = (unsigned)m;
                                }
                            }
                        }
                }
            }
            __syncwarp();
        }
        unsigned Se = 1;   // comb stride of the excluded layer
        for (unsigned l = 0; l < excl; ++l)
            Se *= hits_of(pk, l);
        for (unsigned gi = lane; gi < total; gi += 32) {
            unsigned t = 0, rem = gi;
            bool found = false;
#pragma unroll
            for (unsigned tt = 0; tt < 10; ++tt) {
                const unsigned c = groups(tt);
                if (!found) {
                    if (rem < c) {
                        t = tt;
                        found = true;
                    } else {
                        rem -= c;
                    }
                }
            }
            const unsigned lt[3] = {triple_l(t, 0), triple_l(t, 1), triple_l(t, 2)};
            const unsigned f0 = fl(lt[0]), f1 = fl(lt[1]), f2 = fl(lt[2]);
            const unsigned p0 = __popc(f0), p1 = __popc(f1);
            const unsigned dsel[3] = {nth_bit(f0, rem % p0), nth_bit(f1, (rem / p0) % p1),
                                      nth_bit(f2, rem / (p0 * p1))};
            unsigned long long mn = NO_KEY;
            if (lt[0] != excl && lt[1] != excl && lt[2] != excl) {
                // three fitted slots fixed; the fourth runs over its canonical hits
                int4 base = make_int4(0, 0, 0, 0);
                unsigned free_slot = 0 + 1 + 2 + 3;
#pragma unroll
                for (unsigned q = 0; q < 3; ++q) {
                    const unsigned s = lt[q] - (lt[q] > excl);
                    free_slot -= s;
                    base = add4(base, B.A[s][B.rank[s][dsel[q]]]);
                }
                for (unsigned z = 0; z < sh.m(free_slot); ++z) {
                    const int4 s = add4(base, B.A[free_slot][z]);
                    unsigned long long key;
                    if (PLAIN) {
                        key = ldcg(d.fit_key + sh.cb + (unsigned)s.w);
                    } else {
                        bool pass;
                        key = box_key(s, d.cut, pass);
                    }
                    mn = umin64(mn, key);
                }
            } else {
                // the excluded layer in the triple: the pair table of the two
                // fitted slots, then the excluded hit's comb
                unsigned de = 0, sa = 4, sb = 4, da = 0, db = 0;
#pragma unroll
                for (unsigned q = 0; q < 3; ++q) {
                    if (lt[q] == excl) {
                        de = dsel[q];
                    } else if (sa == 4) {
                        sa = lt[q] - (lt[q] > excl);
                        da = dsel[q];
                    } else {
                        sb = lt[q] - (lt[q] > excl);
                        db = dsel[q];
                    }
                }
                unsigned idx;
                const unsigned tab = box_tab(sh, sa, B.rank[sa][da], sb, B.rank[sb][db], idx);
                mn = box_get(B, tab, idx);
                if (mn != NO_KEY)
                    mn += (unsigned long long)de * Se;
            }
            if (mn != NO_KEY)
                hash_min(d, group_key(rec.event, t, B.co[lt[0] * 8 + dsel[0]], B.co[lt[1] * 8 + dsel[1]],
                                      B.co[lt[2] * 8 + dsel[2]]),
                         mn);
        }
    }
    __syncwarp();
}

static_assert(sizeof(P3Box) <= P3_WARP_BYTES, "the box path uses a warp's region of the flat path");

// The roads listed in P2 (more than small_n4 distinct fits, or a cross-road
// candidate with a repeated coordinate) are fitted first, one warp each
// (box_road); then every warp claims runs of d.run_roads consecutive roads
// (4, 8 or 16) and fits the others itself, WARP_ROADS at a time (fit_run).
// Each warp works in its own region of shared memory, so no stage of P3
// waits for the whole CTA.
template <bool PLAIN>
__device__ void p3_phase(const Dev &d, unsigned char *smem, int qbig, int qsmall)
{
    const unsigned n_big = min(ldcg(&d.ctrl->n_big), d.max_roads);
    const unsigned n_roads = min(ldcg(&d.ctrl->n_roads), d.max_roads);
    unsigned long long npass = 0;
    unsigned char *region = smem + warp_id() * P3_WARP_BYTES;
    // a warp's first item of each queue is its own index; the queue hands out the rest
    const unsigned n_warps = gridDim.x * WARPS;
    for (unsigned i = blockIdx.x * WARPS + warp_id(); i < n_big;) {
        box_road<PLAIN>(d, region, min(ldcg(d.big_list + i), d.max_roads - 1), npass);
        unsigned ni = 0;
        if (lane_id() == 0)
            ni = n_warps + atomicAdd(&d.ctrl->q[qbig], 1u);
        i = __shfl_sync(FULL_MASK, ni, 0);
    }
    __syncwarp();
    {
        const unsigned rr = (unsigned)d.run_roads;
        const unsigned n_runs = (n_roads + rr - 1) / rr;
        for (unsigned c = blockIdx.x * WARPS + warp_id(); c < n_runs;) {
            const unsigned ge = min(c * rr + rr, n_roads);
            for (unsigned g0 = c * rr; g0 < ge; g0 += WARP_ROADS)
                fit_run<PLAIN>(d, region, g0, min((unsigned)WARP_ROADS, ge - g0), npass);
            unsigned nc = 0;
            if (lane_id() == 0)
                nc = n_warps + atomicAdd(&d.ctrl->q[qsmall], 1u);
            c = __shfl_sync(FULL_MASK, nc, 0);
        }
    }
    npass = block_sum(npass);
    if (!PLAIN && threadIdx.x == 0 && npass)
        atomicAdd(&d.ctrl->n_pass, npass);
}

// ---------------------------------------------------------------------------
// P4: cross-road hit-warrior and survivor counts, P5: output
// ---------------------------------------------------------------------------

__device__ unsigned cross_check(const Dev &d, unsigned g, unsigned cnt)
{
    const RoadRec rec = ldcg(d.roads + g);
    const unsigned long long xm = ldcg(d.xmask + g);
    unsigned n[N_LAYERS];
#pragma unroll
    for (unsigned l = 0; l < N_LAYERS; ++l)
        n[l] = max(min((rec.pk >> (4 * l)) & 15u, (unsigned)MAX_HITS), 1u);
    const uint16_t *co = d.coords + (size_t)g * 40;
    unsigned kept = 0;
    for (unsigned i = 0; i < cnt; ++i) {
        unsigned long long key = ldcg(d.surv_pool + surv_at(d, g, i));
        unsigned t = (unsigned)(key & 0x7FFFu);
        unsigned dl[N_LAYERS], v[N_LAYERS];
#pragma unroll
        for (unsigned l = 0; l < N_LAYERS; ++l) {   // mixed-radix digits of comb
            const unsigned q = divm(t, c_magic[n[l]]);
            dl[l] = t - q * n[l];
            t = q;
            v[l] = ldcg(co + l * 8 + dl[l]);
        }
        bool dropped = false;
#pragma unroll
        for (unsigned t = 0; t < 10; ++t) {
            if (dropped)
                break;
            const unsigned l0 = triple_l(t, 0), l1 = triple_l(t, 1), l2 = triple_l(t, 2);
            bool flagged = ((xm >> (8 * l0 + dl[l0])) & 1ull) && ((xm >> (8 * l1 + dl[l1])) & 1ull) &&
                           ((xm >> (8 * l2 + dl[l2])) & 1ull);
            if (flagged && hash_get(d, group_key(rec.event, t, v[l0], v[l1], v[l2])) < key)
                dropped = true;
        }
        if (!dropped)
            d.surv_pool[surv_at(d, g, kept++)] = key;
    }
    return kept;
}

__device__ void p4_item(const Dev &d, unsigned c, unsigned n_roads)
{
    unsigned g = c * ROAD_CHUNK + threadIdx.x;
    unsigned cnt = 0;
    if (g < n_roads) {
        cnt = ldcg(d.surv_cnt + g);
        if (cnt && ((ldcg(&d.roads[g].pk) >> 23) & 1u)) {
            cnt = cross_check(d, g, cnt);
            d.surv_cnt[g] = (uint8_t)cnt;
        }
    }
    unsigned long long tot = block_sum(cnt);
    if (threadIdx.x == 0)
        d.rchunk_sum[c] = (uint32_t)tot;
}

__device__ void p4_finish(const Dev &d, unsigned n_chunks)
{
    unsigned long long total = block_scan_array(d.rchunk_sum, d.rchunk_off, n_chunks);
    if (threadIdx.x == 0) {
        d.ctrl->n_out = total;
        if (total > d.max_tracks)
            raise_flag(d, FLAG_CAPACITY);
        __threadfence();
    }
}

// hit d (0..7) of a layer's eight 16-bit coordinates held in one uint4
__device__ __forceinline__ unsigned coord_of(const uint4 &r, unsigned d)
{
    const unsigned w = d < 4 ? (d < 2 ? r.x : r.y) : (d < 6 ? r.z : r.w);
    return (w >> (16 * (d & 1u))) & 0xFFFFu;
}

// The track of key `key` of road g (record rec, coordinate row rw: the
// road's 40 coordinates as five 16-byte words), written to output slot pos.
// The loops are unrolled (registers, no local arrays).
template <bool PLAIN>
__device__ void build_track(const Dev &d, unsigned g, const RoadRec &rec, const uint4 (&rw)[N_LAYERS],
                            unsigned long long key, unsigned long long pos)
{
    int F[3][6], q[3];
    if (!PLAIN) {   // six 16-byte loads of the set's F and q
        const int4 *fc = d.fitc + SET_INT4 * min((unsigned)rec.set, (unsigned)(N_SETS - 1));
        int4 v[6];
#pragma unroll
        for (unsigned i = 0; i < 6; ++i)
            v[i] = __ldg(fc + i);
        const int f[24] = {v[0].x, v[0].y, v[0].z, v[0].w, v[1].x, v[1].y, v[1].z, v[1].w,
                           v[2].x, v[2].y, v[2].z, v[2].w, v[3].x, v[3].y, v[3].z, v[3].w,
                           v[4].x, v[4].y, v[4].z, v[4].w, v[5].x, v[5].y, v[5].z, v[5].w};
#pragma unroll
        for (unsigned k = 0; k < 3; ++k) {
#pragma unroll
            for (unsigned jj = 0; jj < 6; ++jj)
                F[k][jj] = f[6 * k + jj];
            q[k] = f[18 + k];
        }
    }
    const unsigned excl = min((rec.pk >> 20) & 7u, 4u);
    const unsigned comb = (unsigned)(key & 0x7FFFu);
    unsigned v[N_LAYERS];
    unsigned rest = comb;
#pragma unroll
    for (unsigned l = 0; l < N_LAYERS; ++l) {   // mixed-radix digits of comb
        const unsigned n = max(min((rec.pk >> (4 * l)) & 15u, (unsigned)MAX_HITS), 1u);
        const unsigned qq = divm(rest, c_magic[n]);
        const unsigned dl = rest - qq * n;
        rest = qq;
        v[l] = coord_of(rw[l], dl);
    }
    svt_track t;
    t.event = rec.event;
    t.road = (uint16_t)(rec.pk >> 24);
    t.comb = (uint16_t)comb;
    t.pad = 0;
    t.chi2 = (long long)(key >> 23);
    unsigned long long hits = 0;
#pragma unroll
    for (unsigned l = 0; l < N_LAYERS; ++l)
        hits |= (unsigned long long)v[l] << (12 * l);
    t.hits = hits;
    if (PLAIN) {
        const unsigned long long ci = ldcg(d.comb_off + g) + comb;
        t.p[0] = ldcg(d.fit_p + 3 * ci);
        t.p[1] = ldcg(d.fit_p + 3 * ci + 1);
        t.p[2] = ldcg(d.fit_p + 3 * ci + 2);
    } else {
        // the fit's inputs: the four layers other than excl, in order, then
        // curvature and phi
        const int x[6] = {(int)(excl == 0 ? v[1] : v[0]), (int)(excl <= 1 ? v[2] : v[1]),
                          (int)(excl <= 2 ? v[3] : v[2]), (int)(excl <= 3 ? v[4] : v[3]), rec.curv, rec.phi};
#pragma unroll
        for (unsigned k = 0; k < 3; ++k) {
            int acc = 0;
#pragma unroll
            for (unsigned jj = 0; jj < 6; ++jj)
                acc += F[k][jj] * x[jj];
            t.p[k] = (acc >> 12) + q[k];
        }
    }
    if (pos < d.max_tracks)
        d.tracks[pos] = t;
}

// Track of survivor idx of road g, written to output slot pos: the road's
// record, the key and the coordinate row go out together (none depends on
// another).
template <bool PLAIN>
__device__ void emit_track(const Dev &d, unsigned g, unsigned idx, unsigned long long pos)
{
    static_assert(sizeof(uint16_t) * 40 == N_LAYERS * sizeof(uint4), "a coordinate row is five 16-byte words");
    const RoadRec rec = ldcg(d.roads + g);
    const unsigned long long key = ldcg(d.surv_pool + surv_at(d, g, idx));
    const uint4 *row = reinterpret_cast<const uint4 *>(d.coords + (size_t)g * 40);
    uint4 rw[N_LAYERS];
#pragma unroll
    for (unsigned l = 0; l < N_LAYERS; ++l)
        rw[l] = ldcg(row + l);
    build_track<PLAIN>(d, g, rec, rw, key, pos);
}

// road of survivor i of a chunk: the last r with s_first[r] <= i (a road
// with survivors; s_first holds the chunk's exclusive scan of counts)
__device__ __forceinline__ unsigned chunk_road(const unsigned *s_first, unsigned i)
{
    unsigned lo = 0, hi = ROAD_CHUNK;
    while (hi - lo > 1) {
        const unsigned mid = (lo + hi) >> 1;
        if (s_first[mid] <= i)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

#if SVT_BLOCK == 256   // the plain pipeline's output stage
// Output of one chunk of ROAD_CHUNK roads (plain kernels): a block scan of
// the survivor counts gives each road's first output slot; then each thread
// takes survivors (not roads), so roads with many survivors are spread out.
template <bool PLAIN>
__device__ void p5_item(const Dev &d, unsigned c, unsigned n_roads, unsigned *s_first)
{
    // s_first: ROAD_CHUNK + 1 shared words, the first survivor of each road
    static_assert(ROAD_CHUNK == BLOCK, "one thread per road of a chunk");
    const unsigned g_me = c * ROAD_CHUNK + threadIdx.x;
    const unsigned cnt_me = g_me < n_roads ? ldcg(d.surv_cnt + g_me) : 0u;
    unsigned long long total;
    const unsigned ex = (unsigned)block_excl_scan(cnt_me, &total);
    s_first[threadIdx.x] = ex;
    if (threadIdx.x == 0)
        s_first[ROAD_CHUNK] = (unsigned)total;
    const unsigned long long base = ldcg(d.rchunk_off + c);
    __syncthreads();
    for (unsigned i = threadIdx.x; i < (unsigned)total; i += BLOCK) {
        const unsigned r = chunk_road(s_first, i);
        emit_track<PLAIN>(d, c * ROAD_CHUNK + r, i - s_first[r], base + i);
    }
    __syncthreads();   // s_first is reused by the next chunk
}
#endif

// P4 of the persistent kernel: the cross-road hit-warrior over the
// candidate roads only (P2 sets their bits; the others keep their
// survivors).  One warp per word of candidate bits, one lane per road, so
// every candidate road checks its survivors at once; bit word w goes to CTA
// w % grid, so that a few candidates are spread out.  A road that loses
// survivors takes them off its chunk's total.
__device__ void p4_cand_phase(const Dev &d)
{
    const unsigned n_roads = min(ldcg(&d.ctrl->n_roads), d.max_roads);
    const unsigned n_words = (n_roads + 31) / 32;
    const unsigned lane = lane_id();
    for (unsigned w = warp_id() * gridDim.x + blockIdx.x; w < n_words; w += gridDim.x * WARPS) {
        const unsigned bits = ldcg(d.cand_bits + w);
        const unsigned g = w * 32 + lane;
        if (!((bits >> lane) & 1u) || g >= n_roads)
            continue;   // not a candidate, or a road of the truncated tail (not fitted)
        const unsigned cnt = ldcg(d.surv_cnt + g);
        if (!cnt)
            continue;
        const unsigned kept = cross_check(d, g, cnt);
        if (kept != cnt) {
            d.surv_cnt[g] = (uint8_t)kept;
            atomicSub(&d.rchunk_sum[g / ROAD_CHUNK], cnt - kept);
        }
    }
}

// P5 of the persistent kernel: the tracks in road order, split evenly over
// the CTAs.  Every CTA scans the chunk totals itself (no CTA scans for the
// others) and takes survivors [S b / grid, S (b + 1) / grid) of the S in all.
// The survivor counts of the roads that hold them are loaded at once, eight
// roads per thread (P5_GROUP chunks at a time), and scanned into a table of
// first survivors, which places each survivor at its road.
constexpr unsigned P5_PER_THREAD = 8;
constexpr unsigned P5_ROADS = BLOCK * P5_PER_THREAD;
constexpr unsigned P5_GROUP = P5_ROADS / ROAD_CHUNK;   // chunks per pass
static_assert(P5_ROADS % ROAD_CHUNK == 0, "whole chunks per pass");
static_assert(P5_GROUP <= 32, "a lane per chunk of a pass");

constexpr unsigned P5_STAGE = 448;   // roads whose records and coordinates are staged at once

struct P5Smem {
    unsigned first[P5_ROADS + 1];   // first survivor of each road of the pass, from its start
    unsigned long long at[2];       // the chunk holding survivor lo, and its first survivor
    RoadRec rec[P5_STAGE];          // staged roads: records
    uint4 row[P5_STAGE * N_LAYERS]; // and coordinate rows
};

// the last road r of [lo, hi) with first[r] <= k (the road of survivor k)
__device__ __forceinline__ unsigned p5_road(const unsigned *first, unsigned lo, unsigned hi, unsigned k)
{
    while (hi - lo > 1) {
        const unsigned mid = (lo + hi) >> 1;
        if (first[mid] <= k)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// survivor counts of roads g .. g + 7 (0 from n_roads on), one byte each
__device__ __forceinline__ unsigned long long load_counts8(const Dev &d, unsigned g, unsigned n_roads)
{
    if (g + P5_PER_THREAD <= n_roads)
        return ldcg(reinterpret_cast<const unsigned long long *>(d.surv_cnt + g));
    unsigned long long v = 0;
    for (unsigned k = 0; k < P5_PER_THREAD && g + k < n_roads; ++k)
        v |= (unsigned long long)ldcg(d.surv_cnt + g + k) << (8 * k);
    return v;
}

__device__ void p5_phase(const Dev &d, unsigned char *smem)
{
    P5Smem &s = *reinterpret_cast<P5Smem *>(smem);
    const unsigned n_roads = min(ldcg(&d.ctrl->n_roads), d.max_roads);
    const unsigned n_chunks = min((n_roads + ROAD_CHUNK - 1) / ROAD_CHUNK, d.max_chunks_r);
    // each thread sums a contiguous range of chunk totals
    const unsigned per = (n_chunks + BLOCK - 1) / BLOCK;
    const unsigned c0 = min(threadIdx.x * per, n_chunks), c1 = min(c0 + per, n_chunks);
    unsigned long long mine = 0;
    for (unsigned c = c0; c < c1; ++c)
        mine += ldcg(d.rchunk_sum + c);
    unsigned long long S;
    const unsigned long long ex = block_excl_scan(mine, &S);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        d.ctrl->n_out = S;
        if (S > d.max_tracks)
            raise_flag(d, FLAG_CAPACITY);
    }
    if (S > d.max_tracks)
        return;
    const unsigned long long lo = S * blockIdx.x / gridDim.x, hi = S * (blockIdx.x + 1) / gridDim.x;
    if (lo == hi)
        return;
    // the chunk holding survivor lo lies in one thread's range
    if (ex <= lo && lo < ex + mine) {
        unsigned c = c0;
        unsigned long long pre = ex;
        for (unsigned long long t = ldcg(d.rchunk_sum + c); pre + t <= lo; t = ldcg(d.rchunk_sum + c)) {
            pre += t;
            ++c;
        }
        s.at[0] = c;
        s.at[1] = pre;
    }
    __syncthreads();
    unsigned c = (unsigned)s.at[0];
    unsigned long long pre = s.at[1];   // first survivor of chunk c
    while (pre < hi && c < n_chunks) {
        const unsigned g0 = c * ROAD_CHUNK, gt = g0 + threadIdx.x * P5_PER_THREAD;
        const unsigned long long cnt8 = load_counts8(d, gt, n_roads);
        unsigned mysum = 0;
#pragma unroll
        for (unsigned k = 0; k < P5_PER_THREAD; ++k)
            mysum += (unsigned)(cnt8 >> (8 * k)) & 0xFFu;
        unsigned long long tot;
        unsigned run = (unsigned)block_excl_scan(mysum, &tot);
#pragma unroll
        for (unsigned k = 0; k < P5_PER_THREAD; ++k) {
            s.first[threadIdx.x * P5_PER_THREAD + k] = run;
            run += (unsigned)(cnt8 >> (8 * k)) & 0xFFu;
        }
        if (warp_id() == 0) {   // the counts and the chunk totals agree (a lane per chunk)
            const unsigned k = lane_id();
            const unsigned long long chk =
                warp_sum(k < P5_GROUP && c + k < n_chunks ? ldcg(d.rchunk_sum + c + k) : 0ull);
            if (k == 0) {
                s.first[P5_ROADS] = (unsigned)tot;
                if (chk != tot)
                    raise_flag(d, FLAG_INTERNAL);
            }
        }
        __syncthreads();
        const unsigned long long a = lo > pre ? lo : pre, b = hi < pre + tot ? hi : pre + tot;
        if (a < b) {
            // survivors ka .. kb of the pass lie in roads r_lo .. r_hi; their
            // records and coordinate rows are staged with coalesced loads,
            // P5_STAGE roads at a time
            const unsigned ka = (unsigned)(a - pre), kb = (unsigned)(b - 1 - pre);
            const unsigned r_lo = p5_road(s.first, 0, P5_ROADS, ka), r_hi = p5_road(s.first, 0, P5_ROADS, kb);
            for (unsigned rb = r_lo; rb <= r_hi; rb += P5_STAGE) {
                const unsigned re = min(rb + P5_STAGE, r_hi + 1), nr = re - rb;
                // the thread's first survivor of the stage: its key is loaded
                // together with the stage
                const unsigned k0 = max(ka, s.first[rb]), k1 = min(kb + 1, s.first[re]);
                const unsigned kf = k0 + threadIdx.x;
                unsigned rf = 0;
                unsigned long long keyf = 0;
                if (kf < k1) {
                    rf = p5_road(s.first, rb, re, kf);
                    keyf = ldcg(d.surv_pool + surv_at(d, g0 + rf, kf - s.first[rf]));
                }
                for (unsigned j = threadIdx.x; j < nr; j += BLOCK)
                    s.rec[j] = ldcg(d.roads + g0 + rb + j);
                const uint4 *rows = reinterpret_cast<const uint4 *>(d.coords + (size_t)(g0 + rb) * 40);
                for (unsigned j = threadIdx.x; j < nr * N_LAYERS; j += BLOCK)
                    s.row[j] = ldcg(rows + j);
                __syncthreads();
                for (unsigned k = kf; k < k1; k += BLOCK) {
                    const unsigned r = k == kf ? rf : p5_road(s.first, rb, re, k), g = g0 + r;
                    const unsigned long long key =
                        k == kf ? keyf : ldcg(d.surv_pool + surv_at(d, g, k - s.first[r]));
                    uint4 rw[N_LAYERS];
#pragma unroll
                    for (unsigned l = 0; l < N_LAYERS; ++l)
                        rw[l] = s.row[(r - rb) * N_LAYERS + l];
                    build_track<false>(d, g, s.rec[r - rb], rw, key, pre + k);
                }
                __syncthreads();   // the stage is refilled next
            }
        }
        pre += tot;
        c += P5_GROUP;
        __syncthreads();   // the table is refilled next
    }
}

// Leave the group table empty: every claimed slot (its bit) is cleared, with
// its bit.  Run by the whole grid once every lookup is done.
__device__ void clear_hash(const Dev &d)
{
    if (ldcg(&d.ctrl->hash_used) == 0)
        return;
    const unsigned n_words = d.hash_mask / 32 + 1;
    for (unsigned w = blockIdx.x * BLOCK + threadIdx.x; w < n_words; w += gridDim.x * BLOCK) {
        unsigned bits = ldcg(d.hash_bits + w);
        if (!bits)
            continue;
        d.hash_bits[w] = 0;
        for (; bits; bits &= bits - 1) {
            const unsigned h = w * 32 + (unsigned)(__ffs(bits) - 1);
            d.hash[h].key = 0ull;
            d.hash[h].val_inv = 0ull;
        }
    }
}

// ---------------------------------------------------------------------------
// the persistent fused kernel
// ---------------------------------------------------------------------------


__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_persistent(Dev d)
{
    extern __shared__ __align__(16) unsigned char smem[];
    if (d.skip_arrival == 1 && blockIdx.x == 0)
        return;   // test hook: this CTA never arrives at the first barrier
    stamp(d, 0);

    scan_count(d);
    if (!grid_sync(d))
        return;
    stamp(d, 1);
    if (!scan_decode(d, smem))
        return;
    if (!grid_sync(d))
        return;
    stamp(d, 2);

    p2_phase(d, smem);
    if (!grid_sync(d))
        return;
    stamp(d, 3);
    if (ldcg(&d.ctrl->err_inv) != 0ull)
        return;   // a data fault: no tracks

    p3_phase<false>(d, smem, Q_BIG, Q_SMALL);
    if (d.skip_arrival == 2 && blockIdx.x == 0)
        return;   // test hook: this CTA leaves after publishing, the others' waits run out
    if (!grid_sync(d))
        return;
    stamp(d, 4);

    p4_cand_phase(d);
    if (!grid_sync(d))
        return;
    stamp(d, 5);
    p5_phase(d, smem);
    // every lookup is done (barrier above): leave the group table empty
    clear_hash(d);
    if (threadIdx.x == 0)
        atomicMax(&d.ctrl->t_phase[6], globaltimer_ns());
}

#if SVT_BLOCK == 256
// ---------------------------------------------------------------------------
// plain per-stage kernels
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(BLOCK) k_p0(Dev d) { scan_count(d); }

__global__ void __launch_bounds__(BLOCK) k_p1(Dev d)
{
    extern __shared__ __align__(16) unsigned char smem[];
    scan_decode(d, smem);
}

__global__ void __launch_bounds__(BLOCK) k_p2(Dev d)
{
    extern __shared__ __align__(16) unsigned char smem[];
    if (ldcg(&d.ctrl->flags) & FLAG_CAPACITY)
        return;
    p2_phase(d, smem);
}

__device__ __forceinline__ bool stop_after_unpack(const Dev &d)
{
    return ldcg(&d.ctrl->err_inv) != 0ull || (ldcg(&d.ctrl->flags) & FLAG_CAPACITY);
}

// combinations per road -> exclusive offsets (the "combine" stage)
__global__ void __launch_bounds__(BLOCK) k_comb_count(Dev d)
{
    if (stop_after_unpack(d))
        return;
    const unsigned n_roads = ldcg(&d.ctrl->n_roads);
    const unsigned n_chunks = (n_roads + ROAD_CHUNK - 1) / ROAD_CHUNK;
    for (unsigned c = grab(d, Q_CNT); c < n_chunks; c = grab(d, Q_CNT)) {
        unsigned g = c * ROAD_CHUNK + threadIdx.x;
        unsigned long long N = 0;
        if (g < n_roads) {
            uint32_t pk = ldcg(&d.roads[g].pk);
            N = 1;
            for (unsigned l = 0; l < N_LAYERS; ++l)
                N *= (pk >> (4 * l)) & 15u;
        }
        unsigned long long t = block_sum(N);
        if (threadIdx.x == 0)
            d.cchunk_sum[c] = t;
    }
    if (last_block(&d.ctrl->done[2], gridDim.x)) {
        unsigned long long total = block_scan_array(d.cchunk_sum, d.cchunk_off, n_chunks);
        if (threadIdx.x == 0 && total > d.max_combs)
            raise_flag(d, FLAG_CAPACITY);
    }
}

__global__ void __launch_bounds__(BLOCK) k_comb_scatter(Dev d)
{
    if (stop_after_unpack(d))
        return;
    const unsigned n_roads = ldcg(&d.ctrl->n_roads);
    const unsigned n_chunks = (n_roads + ROAD_CHUNK - 1) / ROAD_CHUNK;
    for (unsigned c = grab(d, Q_CSC); c < n_chunks; c = grab(d, Q_CSC)) {
        unsigned g = c * ROAD_CHUNK + threadIdx.x;
        unsigned long long N = 0;
        if (g < n_roads) {
            uint32_t pk = ldcg(&d.roads[g].pk);
            N = 1;
            for (unsigned l = 0; l < N_LAYERS; ++l)
                N *= (pk >> (4 * l)) & 15u;
        }
        unsigned long long ex = block_excl_scan(N, nullptr);
        if (g < n_roads)
            d.comb_off[g] = ldcg(d.cchunk_off + c) + ex;
    }
}

// one thread per combination: the paper's fit kernel (Sec. II-A)
__global__ void __launch_bounds__(BLOCK) k_fit_plain(Dev d)
{
    if (stop_after_unpack(d))
        return;
    const unsigned n_roads = ldcg(&d.ctrl->n_roads);
    const unsigned long long n_comb = ldcg(&d.ctrl->n_comb);
    unsigned long long npass = 0;
    const unsigned long long stride = (unsigned long long)gridDim.x * BLOCK;
    for (unsigned long long base = (unsigned long long)blockIdx.x * BLOCK; base < n_comb; base += stride) {
        unsigned long long i = base + threadIdx.x;
        if (i < n_comb) {
            // road: last g with comb_off[g] <= i
            unsigned lo = 0, hi = n_roads;
            while (hi - lo > 1) {
                unsigned mid = (lo + hi) >> 1;
                if (ldcg(d.comb_off + mid) <= i)
                    lo = mid;
                else
                    hi = mid;
            }
            unsigned g = lo;
            RoadRec rec = ldcg(d.roads + g);
            unsigned comb = (unsigned)(i - ldcg(d.comb_off + g));
            const unsigned excl = min((rec.pk >> 20) & 7u, 4u);
            const uint16_t *co = d.coords + (size_t)g * 40;
            int x[6];
            unsigned t = comb, j = 0;
            for (unsigned l = 0; l < N_LAYERS; ++l) {
                unsigned nl = max(min((rec.pk >> (4 * l)) & 15u, (unsigned)MAX_HITS), 1u);
                unsigned q = divm(t, c_magic[nl]);
                unsigned dl = t - q * nl;
                t = q;
                if (l != excl)
                    x[j++] = ldcg(co + l * 8 + dl);
            }
            x[4] = rec.curv;
            x[5] = rec.phi;
            const svt_const_set *cs = d.consts + min((unsigned)rec.set, (unsigned)(N_SETS - 1));
            long long chi2 = 0;
            for (unsigned k = 0; k < 3; ++k) {
                int acc = 0;
                for (unsigned jj = 0; jj < 6; ++jj)
                    acc += (int)__ldg(&cs->C[k][jj]) * x[jj];
                chi2 += sq((acc >> 12) + __ldg(&cs->k[k]));
            }
            for (unsigned k = 0; k < 3; ++k) {
                int acc = 0;
                for (unsigned jj = 0; jj < 6; ++jj)
                    acc += (int)__ldg(&cs->F[k][jj]) * x[jj];
                d.fit_p[3 * i + k] = (acc >> 12) + __ldg(&cs->q[k]);
            }
            bool pass = chi2 <= d.cut;
            npass += pass;
            d.fit_key[i] = pass ? make_key(chi2, rec.pk >> 24, comb) : NO_KEY;
        }
    }
    npass = block_sum(npass);
    if (threadIdx.x == 0 && npass)
        atomicAdd(&d.ctrl->n_pass, npass);
}

__global__ void __launch_bounds__(BLOCK) k_warrior_plain(Dev d)
{
    extern __shared__ __align__(16) unsigned char smem[];
    if (stop_after_unpack(d))
        return;
    p3_phase<true>(d, smem, Q_BIG, Q_SMALL);
}

__global__ void __launch_bounds__(BLOCK) k_p4(Dev d)
{
    if (stop_after_unpack(d))
        return;
    const unsigned n_roads = ldcg(&d.ctrl->n_roads);
    const unsigned n_chunks = (n_roads + ROAD_CHUNK - 1) / ROAD_CHUNK;
    for (unsigned c = grab(d, Q_P4); c < n_chunks; c = grab(d, Q_P4))
        p4_item(d, c, n_roads);
    if (last_block(&d.ctrl->done[1], gridDim.x))
        p4_finish(d, n_chunks);
}

__global__ void __launch_bounds__(BLOCK) k_p5(Dev d)
{
    __shared__ unsigned s_first[ROAD_CHUNK + 1];
    const unsigned n_roads = ldcg(&d.ctrl->n_roads);
    const unsigned n_chunks = (n_roads + ROAD_CHUNK - 1) / ROAD_CHUNK;
    if (!stop_after_unpack(d))
        for (unsigned c = grab(d, Q_P5); c < n_chunks; c = grab(d, Q_P5))
            p5_item<true>(d, c, n_roads, s_first);
    // the previous kernels' lookups are done: leave the group table empty
    clear_hash(d);
}

__global__ void __launch_bounds__(BLOCK) k_export_roads(Dev d)
{
    const unsigned n_roads = min(ldcg(&d.ctrl->n_roads), d.max_roads);
    for (unsigned g = blockIdx.x * BLOCK + threadIdx.x; g < n_roads; g += gridDim.x * BLOCK) {
        RoadRec rec = ldcg(d.roads + g);
        svt_road o;
        o.event = rec.event;
        o.road = (uint16_t)(rec.pk >> 24);
        unsigned set = rec.set, excl = set % 5, wb = set / 5;
        o.wedge = (uint8_t)(wb / 6);
        o.barrel = (uint8_t)(wb % 6);
        o.excl = (uint8_t)excl;
        for (unsigned l = 0; l < N_LAYERS; ++l)
            o.n[l] = (uint8_t)((rec.pk >> (4 * l)) & 15u);
        o.pad[0] = o.pad[1] = 0;
        o.curv = rec.curv;
        o.phi = rec.phi;
        for (unsigned j = 0; j < 40; ++j)   // slots beyond a layer's hits hold no coordinate
            o.coord[j >> 3][j & 7] = (j & 7u) < o.n[j >> 3] ? ldcg(d.coords + (size_t)g * 40 + j) : (uint16_t)0;
        d.road_out[g] = o;
    }
}

#endif   // the plain per-stage kernels

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

static size_t p1_smem() { return WARPS * sizeof(P1Warp); }
static size_t p2_smem() { return sizeof(P2Smem) > WARPS * P2W_BYTES ? sizeof(P2Smem) : WARPS * P2W_BYTES; }
static size_t p3_smem() { return WARPS * P3_WARP_BYTES; }

size_t persistent_smem_bytes()
{
    size_t a = p2_smem(), b = p3_smem(), c = p1_smem(), e = sizeof(P5Smem);   // p2_smem: both P2 paths
    a = a > b ? a : b;
    a = a > c ? a : c;
    return a > e ? a : e;
}

static cudaError_t set_smem_attrs()
{
    static bool done = false;
    if (done)
        return cudaSuccess;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)persistent_smem_bytes())))
        return e;
#if SVT_BLOCK == 256
    if ((e = cudaFuncSetAttribute(k_p2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p2_smem())))
        return e;
    if ((e = cudaFuncSetAttribute(k_p1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p1_smem())))
        return e;
    if ((e = cudaFuncSetAttribute(k_warrior_plain, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)p3_smem())))
        return e;
#endif
    done = true;
    return cudaSuccess;
}

int persistent_max_blocks_per_sm(int device)
{
    (void)device;
    if (set_smem_attrs() != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persistent, BLOCK,
                                                      persistent_smem_bytes()) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_persistent(const Dev &d, cudaStream_t s, int blocks_per_sm, int max_ctas, int *n_launches)
{
    cudaError_t e = set_smem_attrs();
    if (e)
        return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int maxb = persistent_max_blocks_per_sm(dev);
    if (maxb <= 0)
        return cudaErrorInvalidConfiguration;
    int bps = blocks_per_sm > 0 && blocks_per_sm < maxb ? blocks_per_sm : maxb;
    Dev dd = d;
    void *args[] = {&dd};
    cudaLaunchConfig_t cfg = {};
    int grid = sms * bps;
    if (max_ctas > 0 && max_ctas < grid)
        grid = max_ctas;
    if (grid > GRID_MAX)   // the word spans (one per warp) and the per-CTA totals are sized for this
        grid = GRID_MAX;
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(BLOCK);
    cfg.dynamicSmemBytes = persistent_smem_bytes();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelExC(&cfg, (const void *)k_persistent, args);
    *n_launches += 1;
    return e;
}

#if SVT_BLOCK == 256
static int plain_grid()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms * 4 < GRID_MAX ? sms * 4 : GRID_MAX;
}

cudaError_t launch_unpack_plain(const Dev &d, cudaStream_t s, int *n_launches)
{
    cudaError_t e = set_smem_attrs();
    if (e)
        return e;
    const int g = plain_grid();   // the same grid for P0 and P1: the word spans follow it
    k_p0<<<g, BLOCK, 0, s>>>(d);
    k_p1<<<g, BLOCK, p1_smem(), s>>>(d);
    k_p2<<<g, BLOCK, p2_smem(), s>>>(d);
    *n_launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_fit_plain(const Dev &d, cudaStream_t s, int *n_launches)
{
    cudaError_t e = set_smem_attrs();
    if (e)
        return e;
    int g = plain_grid();
    k_comb_count<<<g, BLOCK, 0, s>>>(d);
    k_comb_scatter<<<g, BLOCK, 0, s>>>(d);
    k_fit_plain<<<g * 4, BLOCK, 0, s>>>(d);
    k_warrior_plain<<<g, BLOCK, p3_smem(), s>>>(d);
    k_p4<<<g, BLOCK, 0, s>>>(d);
    k_p5<<<g, BLOCK, 0, s>>>(d);
    *n_launches += 6;
    return cudaGetLastError();
}

cudaError_t launch_export_roads(const Dev &d, cudaStream_t s)
{
    k_export_roads<<<plain_grid(), BLOCK, 0, s>>>(d);
    return cudaGetLastError();
}
#endif

}  // namespace SVT_KNS
}  // namespace svt
