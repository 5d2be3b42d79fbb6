// svt_ctx.h -- the context behind the opaque svt_ctx handle, and the host
// helpers that the C ABI (svt_api.cu) and the serving runtime
// (svt_server.cu) share.
#pragma once
#include "svt_internal.h"

#include <cstdlib>

struct svt_ctx {
    int device = 0;
    svt_limits lim{};
    svt::Dev d{};
    svt::Ctrl *h_ctrl = nullptr;          // pinned mirror of the control block
    bool consts_loaded = false;
    bool bound = false;              // a batch is bound by svt_unpack
    bool roads_valid = false;        // the road table holds the bound batch
    bool ran = false;                // svt_fit_events ran on the bound batch
    int block = 256;                 // threads per CTA of the persistent kernel (128, 256, 512)
    int blocks_per_sm = 0;
    int max_ctas = 0;                // persistent grid cap (0 = all SMs x blocks_per_sm)
    int last_launches = 0;
    unsigned long long wait_ns = 2000000000ull;
    int skip_arrival = 0;
    bool hash_dirty = false;         // a batch stopped before clearing its group table
    unsigned long long last_n_out = 0;   // tracks of the last batch read (svt_get_tracks' first copy)
    svt_track *dev_tracks = nullptr;     // the context's own track buffer (device memory)
    svt_track *host_out = nullptr;       // host buffer the output stage writes (svt_set_track_output)
    // CUDA graph of one svt_fit_events enqueue
    bool use_graph = false;
    cudaGraphExec_t gexec = nullptr;
    int g_mode = -1;
    const uint32_t *g_words = nullptr;
    unsigned long long g_n = 0;
    cudaStream_t g_stream = nullptr;
    int g_launches = 0;
    unsigned long long g_key = 0;
    void *allocs[40] = {};
    int n_allocs = 0;
};

namespace svt {

// Bound on |sum_j coef_j x_j + 4096 offset| over every admissible input: hits
// are at most 4095, curvature and phi at most 32768 in magnitude.
inline long long bound_row(const int16_t *coef, int32_t off)
{
    long long b = 0;
    for (int j = 0; j < 6; ++j)
        b += (long long)std::llabs(coef[j]) * (j < 4 ? 4095 : 32768);
    return b + 4096ll * std::llabs((long long)off);
}

// The admission rule of constant sets (svt_load_constants, svt_run_static):
// every row's bound below 2^31 (the fit's 32-bit sums are exact) and the
// chi-square bound below 2^38 (the track key's 61 bits).
inline bool constants_admissible(const svt_const_set *sets)
{
    for (int s = 0; s < N_SETS; ++s) {
        long long chi_bound = 0;
        for (int k = 0; k < 3; ++k) {
            const long long bf = bound_row(sets[s].F[k], sets[s].q[k]);
            const long long bc = bound_row(sets[s].C[k], sets[s].k[k]);
            if (bf >= (1ll << 31) || bc >= (1ll << 31))
                return false;
            const long long a = bc / 4096 + 1;
            chi_bound += a * a;
        }
        if (chi_bound >= (1ll << 38))
            return false;
    }
    return true;
}

// Status of a batch from its control block (after the kernels).
inline int status_of(const Ctrl &c)
{
    if (c.flags & FLAG_TIMEOUT)
        return SVT_E_TIMEOUT;
    if (c.flags & FLAG_CAPACITY)
        return SVT_E_CAPACITY;
    if (c.err_inv != 0ull) {
        unsigned rank = (unsigned)(~c.err_inv & 0xFFull);
        return rank == RANK_BAD ? SVT_E_BADWORD : rank == RANK_LIMIT ? SVT_E_LIMIT : SVT_E_TRUNCATED;
    }
    if (c.flags & FLAG_INTERNAL)
        return SVT_E_CUDA;
    return SVT_OK;
}

// Enqueue one batch of the words bound to c (control block reset, kernels)
// on s; adds the kernel launches to *launches.
cudaError_t ctx_enqueue(svt_ctx *c, int mode, cudaStream_t s, int *launches);

// Status of the batch whose control block is in c->h_ctrl (after a copy).
int ctx_status(const svt_ctx *c);

// Allocate what `mode` needs beyond svt_create (SVT_PLAIN's per-combination
// buffers); SVT_OK or SVT_E_CUDA.
int ctx_prepare(svt_ctx *c, int mode);

}  // namespace svt
