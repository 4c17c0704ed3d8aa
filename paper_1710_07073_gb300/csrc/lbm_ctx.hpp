// Host-side definition of the context shared by the C-ABI translation units
// (lbm_capi.cu, lbm_adjoint.cu).  Not part of the public interface.
#pragma once

#include <string>
#include <utility>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.cuh"

struct AdjointTape;   // lbm_adjoint.cu

using lbm::Bins;
using lbm::BubbleDev;
using lbm::SmallBins;
using lbm::SwarmBins;

struct lbm_ctx {
    int nx = 0, ny = 0, nz = 0;
    unsigned walls = 0;
    double omega = 1.0;
    int storage = LBM_STORE_F32;
    double scale = 1.0;
    lbm_params p{};
    cudaStream_t stream = nullptr;
    lbm_alloc_fn af = nullptr;
    lbm_free_fn ff = nullptr;
    void* au = nullptr;

    bool dev_ready = false;
    int device = 0;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    int* flag_d = nullptr;
    int* flag_h = nullptr;       // pinned
    bool unstable = false;

    // bubbles
    BubbleDev bub{};
    int nb_cap = 0;
    double hwmax = 0.0;          // largest window half-width of the bubbles
    // bins: the large path (count, scan, fill, sort) or, for few pairs, the
    // single-launch small path
    Bins bins{};
    SmallBins small{};
    bool use_small = false;
    bool bins_valid = false;
    // Number of the next step for the overlap guard (small.safe holds two
    // tag sets of ntz, by step parity).  Any change of the bubble state
    // outside a step moves it past every stored tag (guard_invalidate), so
    // stale tags never clear a layer.
    unsigned epoch = 1;
    // Large path: whether the tile lists (bins) and spreading records are
    // those of the current centres.
    bool cover_valid = false;
    // Large path: interpolation parts, list positions and binning scratch.
    SwarmBins swarm{};
    // Large path, split sweep: a step forks from `stream` into a high-priority
    // stream for the bubble side (update, binning, the sweep of the z blocks
    // bubbles can reach) and a low-priority one for the sweep of the others,
    // and joins again.  The blocks bubbles can reach come from the binning's
    // z range of SPLIT_LAG steps before (read back into pinned memory), widened
    // by the distance a bubble may move since.
    static constexpr int SPLIT_RING = 4;
    static constexpr int SPLIT_LAG = 2;
    cudaStream_t side_hi = nullptr, side_lo = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_hi = nullptr, ev_lo = nullptr;
    cudaEvent_t ev_rb[SPLIT_RING] = {};
    int* zr_host = nullptr;                 // pinned [2 * SPLIT_RING]
    long long rb_step[SPLIT_RING] = {-1, -1, -1, -1};
    long long swarm_step = 0;               // steps with bubbles enqueued
    long long swarm_valid_from = 0;         // readbacks before this step are stale
    int sms = 0;                            // SM count (the split interpolation's grid)

    // timing of the collide-stream launches
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    size_t events_used = 0;

    long long launches = 0;      // kernels enqueued by this context

    AdjointTape* adj = nullptr;   // forward record of lbm_adj_forward

    std::vector<std::pair<void*, size_t>> allocs;
    std::string err;
};


int fail(lbm_ctx* c, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int cuda_fail(lbm_ctx* c, cudaError_t e, const char* what);
void* dalloc(lbm_ctx* c, size_t bytes);
void dfree(lbm_ctx* c, void* p);
size_t elem_size(int storage);
lbm::Geo geo_of(const lbm_ctx* c);
lbm::CollideParams collide_params(const lbm_ctx* c);
lbm::BubbleConst bubble_const(const lbm_ctx* c);
int ensure_device(lbm_ctx* c);
// One coupled step on the context stream (the body of lbm_step's loop).
int enqueue_one_step(lbm_ctx* c);
// The bubble state changed outside a step: no stored guard tag may clear a
// layer for the next step.
void guard_invalidate(lbm_ctx* c);
int finish_steps(lbm_ctx* c);
void adjoint_free(lbm_ctx* c);

#define LBM_CUDA(call, what)                                  \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)
