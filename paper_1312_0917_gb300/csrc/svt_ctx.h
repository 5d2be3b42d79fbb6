// svt_ctx.h -- the context behind the opaque svt_ctx handle, and the host
// helpers that the C ABI (svt_api.cu) and the serving runtime
// (svt_server.cu) share.
#pragma once
#include "svt_internal.h"

struct svt_ctx {
    int device = 0;
    svt_limits lim{};
    svt::Dev d{};
    svt::Ctrl *h_ctrl = nullptr;          // pinned mirror of the control block
    bool consts_loaded = false;
    bool bound = false;              // a batch is bound by svt_unpack
    bool roads_valid = false;        // the road table holds the bound batch
    bool ran = false;                // svt_fit_events ran on the bound batch
    int blocks_per_sm = 0;
    int max_ctas = 0;                // persistent grid cap (0 = all SMs x blocks_per_sm)
    int last_launches = 0;
    unsigned long long wait_ns = 2000000000ull;
    int skip_arrival = 0;
    bool hash_dirty = false;         // a batch stopped before clearing its group table
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

// Enqueue one batch of the words bound to c (control block reset, kernels)
// on s; adds the kernel launches to *launches.
cudaError_t ctx_enqueue(svt_ctx *c, int mode, cudaStream_t s, int *launches);

// Status of the batch whose control block is in c->h_ctrl (after a copy).
int ctx_status(const svt_ctx *c);

// Allocate what `mode` needs beyond svt_create (SVT_PLAIN's per-combination
// buffers); SVT_OK or SVT_E_CUDA.
int ctx_prepare(svt_ctx *c, int mode);

}  // namespace svt
