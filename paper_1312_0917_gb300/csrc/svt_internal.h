// svt_internal.h -- definitions shared by the library's kernels and its C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "svt.h"

namespace svt {

constexpr int MAX_GRID = 4096;             // CTAs of any kernel over the word spans at most
constexpr int MAX_SPANS = MAX_GRID * 8;    // word spans (one per warp of the grid): a grid of
                                           // b threads per CTA has at most MAX_SPANS * 32 / b CTAs
constexpr int MAX_ROADS_EV = 256;          // format limit: roads per event
constexpr int MAX_HITS = 8;                // format limit: hits per layer per road
constexpr int N_LAYERS = 5;
constexpr int N_SETS = 360;                // 12 wedges x 6 barrels x 5 excluded layers
constexpr int SURV_SLOTS = 64;             // survivors per road are <= 64 (see box_road)
constexpr int ROAD_CHUNK = 256;            // roads per output work item
constexpr int WARP_ROADS = 8;              // roads a fitting warp takes into its tables at once
constexpr int P2W_ROADS = 64;              // events of at most this many roads: one warp each in P2
constexpr int RUN_ROADS_MAX = 16;          // roads per queue claim of a fitting warp (run_roads)
constexpr int N4_SMALL_MAX = 256;          // largest road a single warp takes
constexpr int QTAB_SMALL = 160;            // the same sum for any road with N4 <= 256
constexpr unsigned long long NO_KEY = ~0ull;

// fault ranks: at one word a format/grammar fault outranks a limit fault;
// truncation is reported at position n_words, after every word
enum : unsigned { RANK_BAD = 1, RANK_LIMIT = 2, RANK_TRUNC = 3 };
enum : unsigned { FLAG_CAPACITY = 1, FLAG_TIMEOUT = 2, FLAG_INTERNAL = 4 };

// The kernels' copy of each set's constants as int32 in 16-byte words, 14
// per set: words 0..5 hold F row by row, then q and three zeros (the output
// stage's six loads); words 6..11 hold column j of C, (C[0][j], C[1][j],
// C[2][j], 0); word 12 holds (k[0], k[1], k[2], 0); word 13 is zero.
constexpr int SET_INT4 = 14;
constexpr int SET_C = 6;   // first word of the C columns
inline void fit_words(const svt_const_set *sets, int32_t *out)
{
    for (int s = 0; s < N_SETS; ++s) {
        int32_t *o = out + s * SET_INT4 * 4;
        for (int j = 0; j < SET_INT4 * 4; ++j)
            o[j] = 0;
        for (int j = 0; j < 18; ++j)
            o[j] = sets[s].F[j / 6][j % 6];
        for (int j = 0; j < 3; ++j)
            o[18 + j] = sets[s].q[j];
        for (int j = 0; j < 6; ++j)
            for (int r = 0; r < 3; ++r)
                o[4 * (SET_C + j) + r] = sets[s].C[r][j];
        for (int r = 0; r < 3; ++r)
            o[4 * (SET_C + 6) + r] = sets[s].k[r];
    }
}

// Per-batch control block in device memory; zeroed by the host before each
// batch.  Queue counters hand out work items; `bar` counts grid-barrier
// arrivals of the persistent kernel.
struct Ctrl {
    unsigned long long err_inv;   // max over faults of ~((pos << 8) | rank); 0 = none
    unsigned int flags;           // FLAG_*
    unsigned int n_events;        // complete events (EE words)
    unsigned int n_ep;            // EP words in the stream
    unsigned int has_tail;        // words after the last EE
    unsigned int n_roads;         // roads of complete events
    unsigned int n_big;           // roads fitted by a whole CTA (list length)
    unsigned int n_big_ev;        // events of more than P2W_ROADS roads (list length)
    unsigned int hash_used;       // claimed slots of the group table
    unsigned int q[12];           // work-queue heads
    unsigned int bar;             // grid barrier arrivals
    unsigned int done[4];         // last-block-done counters
    unsigned int pad0;
    unsigned long long n_comb, n_pass, n_out;
    unsigned long long pad1[2];
    unsigned long long t_phase[8];   // persistent kernel: globaltimer at its start, after each
                                     // barrier (block 0) and at the last CTA's exit (max)
};

// Unpacked road, 16 bytes.  pk: n[l] in bits 4l..4l+3 (l < 5), excluded layer
// in bits 20..22, cross-road candidate in bit 23, road-in-event in bits 24..31.
struct RoadRec {
    uint32_t event;
    uint32_t pk;
    int16_t curv, phi;
    uint16_t set;
    uint16_t cta;   // bit 0: fitted by a whole CTA (listed in big_list), not by a warp's run;
                    // bit 1: a coordinate repeated within a layer
};

// Cross-road group table slot: key = (event + 1, triple, three coordinates),
// val_inv = ~(lowest track key of the group), 0 = empty.
struct HashSlot {
    unsigned long long key, val_inv;
};

// Everything a kernel needs, passed by value.
struct Dev {
    Ctrl *ctrl;
    const svt_const_set *consts;
    const uint32_t *words;
    unsigned long long n_words;
    unsigned int max_events, max_roads, max_chunks_r;
    unsigned long long max_tracks, max_combs;
    uint32_t *span_ee, *span_ep, *span_seg;   // [MAX_SPANS + MAX_GRID] per word span (one per warp),
                                              // then per CTA (its spans together): EE and EP words,
                                              // EP words since its last EE (SEG_EE set when it holds one)
    uint32_t *ev_road_end;                    // [max_events] roads up to the end of each event
    uint32_t *ev_big;                         // [max_events] events of more than P2W_ROADS roads
    RoadRec *roads;                                               // [max_roads]
    uint16_t *coords;                                             // [max_roads][5][8]
    unsigned long long *xmask;                                    // [max_roads]
    uint32_t *big_list;                                           // [max_roads]
    int4 *fitc;            // [N_SETS][SET_INT4]: the constants as int32 in 16-byte words, written
                           // with the constants (fit_words); read-only in the kernels
    uint32_t *cand_bits;                                          // [max_roads / 32 + 1] cross-road
                                                                  // candidate roads, one bit each
    unsigned long long *surv_pool;                                // [SURV_SLOTS][max_roads] road survivors
                                                                  // (slot-major: see surv_at)
    uint8_t *surv_cnt;                                            // [max_roads]
    uint32_t *rchunk_sum, *rchunk_off;                            // [max_chunks_r]
    unsigned long long *cchunk_sum, *cchunk_off;                  // [max_chunks_r]
    HashSlot *hash;
    uint32_t *hash_bits;   // [hash_mask / 32 + 1] claimed slots of the group table, one bit each
    uint32_t hash_mask;
    unsigned long long *comb_off;                                 // plain: [max_roads]
    unsigned long long *fit_key;                                  // plain: [max_combs]
    int32_t *fit_p;                                               // plain: [max_combs][3]
    svt_track *tracks;                                            // [max_tracks]
    svt_road *road_out;                                           // [max_roads] (svt_get_roads)
    long long cut;
    int small_n4;
    int run_roads;         // roads per queue claim of the fit stage's runs: 4, 8 or 16
    int skip_arrival;
    unsigned long long wait_ns;
};

// Launchers.  svt_kernels.cu is compiled once per block size of the
// persistent kernel, each build in its own namespace: b256 (svt_kernels.cu,
// also the plain pipeline), b128 (svt_kernels_b128.cu), b512
// (svt_kernels_b512.cu).
#define SVT_PERSISTENT_DECLS                                                                          \
    cudaError_t launch_persistent(const Dev &d, cudaStream_t s, int blocks_per_sm, int max_ctas,      \
                                  int *n_launches);                                                   \
    int persistent_max_blocks_per_sm(int device);                                                     \
    size_t persistent_smem_bytes();
namespace b128 { SVT_PERSISTENT_DECLS }
namespace b512 { SVT_PERSISTENT_DECLS }
namespace b256 {
SVT_PERSISTENT_DECLS
cudaError_t launch_unpack_plain(const Dev &d, cudaStream_t s, int *n_launches);
cudaError_t launch_fit_plain(const Dev &d, cudaStream_t s, int *n_launches);
cudaError_t launch_export_roads(const Dev &d, cudaStream_t s);
}
#undef SVT_PERSISTENT_DECLS
using b256::launch_unpack_plain;
using b256::launch_fit_plain;
using b256::launch_export_roads;

constexpr int PERSISTENT_BLOCKS[3] = {128, 256, 512};   // the block sizes built
inline bool persistent_block_ok(int block) { return block == 128 || block == 256 || block == 512; }

// the persistent kernel at `block` threads per CTA (128, 256 or 512)
inline cudaError_t launch_persistent(int block, const Dev &d, cudaStream_t s, int blocks_per_sm, int max_ctas,
                                     int *n_launches)
{
    return block == 128   ? b128::launch_persistent(d, s, blocks_per_sm, max_ctas, n_launches)
           : block == 512 ? b512::launch_persistent(d, s, blocks_per_sm, max_ctas, n_launches)
                          : b256::launch_persistent(d, s, blocks_per_sm, max_ctas, n_launches);
}
inline int persistent_max_blocks_per_sm(int block, int device)
{
    return block == 128   ? b128::persistent_max_blocks_per_sm(device)
           : block == 512 ? b512::persistent_max_blocks_per_sm(device)
                          : b256::persistent_max_blocks_per_sm(device);
}

}  // namespace svt
