// Host side of the batch C ABI (include/lbm.h, lbm_batch_*): many independent
// columns -- each with its own size, relaxation frequency, walls and bubbles --
// advanced together.  One coupled step of the batch is two launches: the
// bubble update of every column (with the binning fused behind it) and one
// persistent collide-stream launch over all columns' work items.  Pairs of
// steps are captured once into a CUDA graph and replayed.  An autotuner picks
// the CTA tile shape (z-planes per CTA), the work-item depth and the
// persistent grid size by timing candidates on the batch itself, with the
// state saved and restored around the trials.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.cuh"

using namespace lbm;

struct lbm_batch {
    int ncols = 0;
    std::vector<int> dims;          // 3 per column
    std::vector<double> omega;
    std::vector<unsigned> walls;
    std::vector<BatchColumn> cols;  // host copy
    int storage = LBM_STORE_F32;
    double scale = 1.0;
    lbm_params p{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    lbm_alloc_fn af = nullptr;
    lbm_free_fn ff = nullptr;
    void* au = nullptr;

    bool dev_ready = false;
    unsigned long long total_elems = 0;   // 19 * sum of sites
    long long total_sites = 0;
    int total_tiles = 0;
    int total_items = 0;                  // for the current depth
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    BatchColumn* cols_d = nullptr;
    double* col_nu_d = nullptr;
    int* flag_d = nullptr;
    int* flag_h = nullptr;
    int* work_counter = nullptr;
    bool unstable = false;

    BubbleDev bub{};
    int* bubble_col_d = nullptr;
    SmallBins small{};

    // launch shape (autotuned)
    int planes = SWEEP_PZ;   // z-planes per CTA: the CTA tile is 32 x 4 x planes nodes
    int depth = 2;           // z-blocks (of `planes` planes) per work item
    int grid = 0;            // persistent CTAs
    bool grid_fixed = false; // grid set by lbm_batch_set_launch_shape
    bool tuned = false;

    cudaGraphExec_t graph = nullptr;
    bool graph_dirty = true;

    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    size_t events_used = 0;
    long long launches = 0;

    std::vector<std::pair<void*, size_t>> allocs;
    std::string err;
};

namespace {

int bfail(lbm_batch* b, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int bfail(lbm_batch* b, int code, const char* fmt, ...) {
    if (b) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        b->err = buf;
    }
    return code;
}

#define LBM_BCUDA(call, what)                                                                \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return bfail(b, LBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e_));          \
    } while (0)

void* balloc(lbm_batch* b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* ptr = nullptr;
    if (b->af) {
        ptr = b->af(bytes, b->au);
    } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
    }
    if (ptr) b->allocs.emplace_back(ptr, bytes);
    return ptr;
}

void bfree(lbm_batch* b, void* ptr) {
    if (!ptr) return;
    for (size_t i = 0; i < b->allocs.size(); ++i) {
        if (b->allocs[i].first == ptr) {
            if (b->ff) b->ff(ptr, b->allocs[i].second, b->au);
            else cudaFree(ptr);
            b->allocs.erase(b->allocs.begin() + (long)i);
            return;
        }
    }
}

size_t elem_bytes(int storage) { return storage == LBM_STORE_F32 ? 4 : 2; }

BubbleConst batch_bubble_const(const lbm_batch* b) {
    BubbleConst bc;
    bc.g = b->p.g;
    bc.rho_l = b->p.rho_l;
    bc.rho_b = b->p.rho_ratio * b->p.rho_l;
    bc.sigma = b->p.sigma;
    bc.c_am = b->p.c_added_mass;
    bc.drag_scale = b->p.drag_scale;
    bc.sn_coeff = b->p.sn_coeff;
    bc.sn_exp = b->p.sn_exp;
    bc.nu = 0.0;   // per column
    bc.dt_l = 1.0;
    bc.dt_b = 1.0 / b->p.substeps;
    split_f2(bc.dt_b, bc.dt_bh, bc.dt_bl);
    bc.substeps = b->p.substeps;
    bc.lift = (b->p.forces & LBM_FORCE_LIFT) ? 1 : 0;
    bc.stress = (b->p.forces & LBM_FORCE_STRESS) ? 1 : 0;
    bc.point = b->p.mapping == LBM_MAP_POINT ? 1 : 0;
    bc.reaction_all = b->p.reaction == LBM_REACTION_ALL ? 1 : 0;
    return bc;
}

// Column table for the current work-item depth.
void layout_columns(lbm_batch* b) {
    unsigned long long off = 0;
    int tile = 0, item = 0;
    const int pz = b->planes;
    b->cols.resize(b->ncols);
    for (int c = 0; c < b->ncols; ++c) {
        BatchColumn& col = b->cols[c];
        const int nx = b->dims[3 * c], ny = b->dims[3 * c + 1], nz = b->dims[3 * c + 2];
        col.g.nx = nx;
        col.g.ny = ny;
        col.g.nz = nz;
        col.g.walls = b->walls[c];
        col.g.S = (long long)nx * ny * nz;
        col.g.ntx = (nx + TX - 1) / TX;
        col.g.nty = (ny + TY - 1) / TY;
        col.g.ntz = (nz + TZ - 1) / TZ;
        col.cp.omega = (float)b->omega[c];
        col.cp.pref = (float)(1.0 - 0.5 * b->omega[c]);
        col.cp.rho0 = (float)b->p.rho_l;
        col.cp.scale = (float)b->scale;
        col.cp.inv_scale = (float)(1.0 / b->scale);
        col.cp.point = b->p.mapping == LBM_MAP_POINT ? 1 : 0;
        col.pop_offset = off;
        col.tile_base = tile;
        col.item_base = item;
        off += (unsigned long long)Q * (unsigned long long)col.g.S;
        tile += col.g.ntx * col.g.nty * col.g.ntz;
        const int nbz = (nz + pz - 1) / pz;
        item += col.g.ntx * col.g.nty * ((nbz + b->depth - 1) / b->depth);
    }
    b->total_elems = off;
    b->total_tiles = tile;
    b->total_items = item;
}

int upload_columns(lbm_batch* b) {
    LBM_BCUDA(cudaMemcpyAsync(b->cols_d, b->cols.data(), sizeof(BatchColumn) * b->cols.size(),
                              cudaMemcpyHostToDevice, b->stream), "upload columns");
    return LBM_OK;
}

int ensure_device(lbm_batch* b) {
    if (b->dev_ready) return LBM_OK;
    if (!b->stream) {
        LBM_BCUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "stream");
        b->own_stream = true;
    }
    layout_columns(b);
    const size_t bytes = (size_t)b->total_elems * elem_bytes(b->storage);
    for (int k = 0; k < 2; ++k) b->f[k] = balloc(b, bytes);
    b->cols_d = (BatchColumn*)balloc(b, sizeof(BatchColumn) * b->ncols);
    b->col_nu_d = (double*)balloc(b, sizeof(double) * b->ncols);
    b->flag_d = (int*)balloc(b, sizeof(int));
    b->work_counter = (int*)balloc(b, sizeof(int));
    SmallBins& sb = b->small;
    sb.T = b->total_tiles;
    sb.start = (int*)balloc(b, sizeof(int) * (size_t)sb.T);
    sb.count = (int*)balloc(b, sizeof(int) * (size_t)sb.T);
    sb.items = (int*)balloc(b, sizeof(int) * SMALL_MAX_PAIRS);
    sb.prev_tiles = (int*)balloc(b, sizeof(int) * SMALL_MAX_PAIRS);
    sb.prev_n = (int*)balloc(b, sizeof(int));
    sb.overflow = (int*)balloc(b, sizeof(int));
    sb.done = (int*)balloc(b, sizeof(int));
    if (!b->f[0] || !b->f[1] || !b->cols_d || !b->col_nu_d || !b->flag_d || !b->work_counter ||
        !sb.start || !sb.count || !sb.items || !sb.prev_tiles || !sb.prev_n || !sb.overflow ||
        !sb.done) {
        // All or nothing: free what this call allocated so that the batch
        // stays destroyable and a later call may retry.
        void** owned[] = {&b->f[0], &b->f[1], (void**)&b->cols_d, (void**)&b->col_nu_d,
                          (void**)&b->flag_d, (void**)&b->work_counter, (void**)&sb.start,
                          (void**)&sb.count, (void**)&sb.items, (void**)&sb.prev_tiles,
                          (void**)&sb.prev_n, (void**)&sb.overflow, (void**)&sb.done};
        for (void** q : owned) {
            bfree(b, *q);
            *q = nullptr;
        }
        return bfail(b, LBM_ERR_ALLOC, "batch device state (%zu bytes per population buffer)",
                     bytes);
    }
    if (!b->flag_h) LBM_BCUDA(cudaMallocHost((void**)&b->flag_h, sizeof(int)), "cudaMallocHost");
    cudaStream_t s = b->stream;
    LBM_BCUDA(cudaMemsetAsync(b->f[0], 0, bytes, s), "memset f");
    LBM_BCUDA(cudaMemsetAsync(b->flag_d, 0, sizeof(int), s), "flag");
    LBM_BCUDA(cudaMemsetAsync(b->work_counter, 0, sizeof(int), s), "counter");
    LBM_BCUDA(cudaMemsetAsync(sb.count, 0, sizeof(int) * (size_t)sb.T, s), "count");
    LBM_BCUDA(cudaMemsetAsync(sb.prev_n, 0, sizeof(int), s), "prev_n");
    LBM_BCUDA(cudaMemsetAsync(sb.overflow, 0, sizeof(int), s), "overflow");
    LBM_BCUDA(cudaMemsetAsync(sb.done, 0, sizeof(int), s), "done");
    std::vector<double> nu(b->ncols);
    for (int c = 0; c < b->ncols; ++c) nu[c] = (2.0 / b->omega[c] - 1.0) / 6.0;   // Eq. 9
    LBM_BCUDA(cudaMemcpyAsync(b->col_nu_d, nu.data(), sizeof(double) * nu.size(),
                              cudaMemcpyHostToDevice, s), "nu");
    int rc = upload_columns(b);
    if (rc) return rc;
    LBM_BCUDA(cudaStreamSynchronize(s), "batch init");
    int dev = 0, sms = 0;
    LBM_BCUDA(cudaGetDevice(&dev), "device");
    LBM_BCUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    if (!b->grid_fixed) b->grid = sms * batch_min_blocks(b->storage, b->planes);
    b->dev_ready = true;
    return LBM_OK;
}

// Enqueue one coupled step of every column on the batch stream.
int enqueue_step(lbm_batch* b, bool time_it) {
    cudaStream_t s = b->stream;
    const bool bubbles = b->bub.nb > 0;
    if (bubbles) {
        LBM_BCUDA(launch_bubbles_batch(b->storage, b->f[b->cur], b->cols_d, b->bubble_col_d, b->bub,
                                       batch_bubble_const(b), b->flag_d, b->small, s),
                  "batch bubble update");
        ++b->launches;
    }
    LBM_BCUDA(cudaMemsetAsync(b->work_counter, 0, sizeof(int), s), "work counter");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (time_it) {
        if (b->events_used == b->events.size()) {
            cudaEvent_t x, y;
            LBM_BCUDA(cudaEventCreate(&x), "event");
            LBM_BCUDA(cudaEventCreate(&y), "event");
            b->events.emplace_back(x, y);
        }
        e0 = b->events[b->events_used].first;
        e1 = b->events[b->events_used].second;
        ++b->events_used;
        LBM_BCUDA(cudaEventRecord(e0, s), "event");
    }
    TileLists tl{b->small.start, b->small.count, b->small.items, SMALL_MAX_PAIRS};
    const bool two_way = bubbles && b->p.two_way;
    TileLists none{nullptr, nullptr, nullptr, 0};
    LBM_BCUDA(launch_collide_batch(b->storage, b->f[b->cur], b->f[b->cur ^ 1], b->cols_d, b->ncols,
                                   b->total_items, b->depth, b->grid, b->planes,
                                   b->work_counter,
                                   two_way ? tl : none, b->bub.rec, b->bub.nb, b->flag_d, s),
              "batch collide-stream");
    ++b->launches;
    if (time_it) LBM_BCUDA(cudaEventRecord(e1, s), "event");
    b->cur ^= 1;
    return LBM_OK;
}

void drop_graph(lbm_batch* b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_dirty = true;
}

// Capture two steps (A -> B -> A) into a graph.
int build_graph(lbm_batch* b) {
    drop_graph(b);
    cudaGraph_t g = nullptr;
    const int cur0 = b->cur;
    const long long l0 = b->launches;
    LBM_BCUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    int rc = enqueue_step(b, false);
    if (!rc) rc = enqueue_step(b, false);
    cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    b->cur = cur0;          // capture does not run anything
    b->launches = l0;
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "end capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "instantiate: %s", cudaGetErrorString(e));
    b->graph_dirty = false;
    return LBM_OK;
}

int check_flag(lbm_batch* b) {
    LBM_BCUDA(cudaMemcpyAsync(b->flag_h, b->flag_d, sizeof(int), cudaMemcpyDeviceToHost, b->stream),
              "flag");
    LBM_BCUDA(cudaStreamSynchronize(b->stream), "step");
    if (*b->flag_h) {
        b->unstable = true;
        return bfail(b, LBM_ERR_UNSTABLE,
                     "non-finite value or |u| >= 0.3 in a column, or a bubble faster than %d "
                     "cells per step", GUARD_CELLS);
    }
    int ov = 0;
    LBM_BCUDA(cudaMemcpy(&ov, b->small.overflow, sizeof(int), cudaMemcpyDeviceToHost), "overflow");
    if (ov) return bfail(b, LBM_ERR_STATE, "tile list capacity exceeded");
    return LBM_OK;
}

int run_steps(lbm_batch* b, int nsteps) {
    if (b->timing) {
        for (int s = 0; s < nsteps; ++s) {
            int rc = enqueue_step(b, true);
            if (rc) return rc;
        }
        return LBM_OK;
    }
    if (nsteps >= 2 && b->graph_dirty) {
        int rc = build_graph(b);
        if (rc) return rc;
    }
    int s = 0;
    for (; s + 2 <= nsteps; s += 2) {
        LBM_BCUDA(cudaGraphLaunch(b->graph, b->stream), "graph launch");
        b->launches += b->bub.nb > 0 ? 4 : 2;
    }
    if (s < nsteps) {
        int rc = enqueue_step(b, false);
        if (rc) return rc;
        // The graph is captured for buffer A as the start; an odd step flips it.
        drop_graph(b);
    }
    return LBM_OK;
}

void free_bubbles(lbm_batch* b) {
    void* ptrs[] = {b->bub.k, b->bub.xh, b->bub.xl, b->bub.u, b->bub.d, b->bub.n,
                    b->bub.ulprev, b->bub.ul, b->bub.out64, b->bub.psi, b->bub.has_prev,
                    b->bub.active, b->bub.spread, b->bub.cell, b->bub.rec, b->bubble_col_d,
                    b->small.part, b->small.arrive};
    for (void* ptr : ptrs) bfree(b, ptr);
    b->bub = BubbleDev{};
    b->bubble_col_d = nullptr;
    b->small.part = nullptr;
    b->small.arrive = nullptr;
    b->small.parts = 0;
}

int axis_tile_bound(double n, int T) {
    const int cells = (int)std::ceil(2.0 * n) + 1;
    return (cells + T - 1) / T + 1;
}

}  // namespace

extern "C" {

int lbm_batch_create(int ncols, const int* dims3, const double* omegas, const unsigned* walls,
                     int storage, double scale, lbm_batch** out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (ncols <= 0 || ncols > 256 || !dims3 || !omegas) return LBM_ERR_ARG;
    if (storage < LBM_STORE_F32 || storage > LBM_STORE_BF16) return LBM_ERR_ARG;
    if (storage != LBM_STORE_F32 && !(scale > 0.0 && std::isfinite(scale))) return LBM_ERR_ARG;
    unsigned long long elems = 0;
    for (int c = 0; c < ncols; ++c) {
        const int nx = dims3[3 * c], ny = dims3[3 * c + 1], nz = dims3[3 * c + 2];
        if (nx <= 0 || ny <= 0 || nz <= 0 || (nx & 1)) return LBM_ERR_ARG;
        if (!(omegas[c] > 0.0 && omegas[c] < 2.0)) return LBM_ERR_ARG;
        const unsigned w = walls ? walls[c] : (unsigned)LBM_WALL_ALL;
        if (w & ~0x7Fu) return LBM_ERR_ARG;
        for (int a = 0; a < 3; ++a)
            if (!(w & (1u << (2 * a))) != !(w & (1u << (2 * a + 1)))) return LBM_ERR_ARG;
        if ((w & WALL_TOP_FREE) && !(w & 0x20u)) return LBM_ERR_ARG;
        const unsigned long long S = (unsigned long long)nx * ny * nz;
        if (S * Q >= (1ULL << 32)) return LBM_ERR_ARG;
        elems += S * Q;
    }
    lbm_batch* b = new lbm_batch();
    b->ncols = ncols;
    b->dims.assign(dims3, dims3 + 3 * ncols);
    b->omega.assign(omegas, omegas + ncols);
    b->walls.resize(ncols);
    for (int c = 0; c < ncols; ++c) b->walls[c] = walls ? walls[c] : (unsigned)LBM_WALL_ALL;
    b->storage = storage;
    b->scale = storage == LBM_STORE_F32 ? 1.0 : scale;
    lbm_default_params(&b->p);
    long long sites = 0;
    for (int c = 0; c < ncols; ++c) sites += (long long)dims3[3 * c] * dims3[3 * c + 1] * dims3[3 * c + 2];
    b->total_sites = sites;
    (void)elems;
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    if (b->dev_ready) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (auto& e : b->events) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    while (!b->allocs.empty()) bfree(b, b->allocs.back().first);
    if (b->flag_h) cudaFreeHost(b->flag_h);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

int lbm_batch_set_stream(lbm_batch* b, void* stream) {
    if (!b) return LBM_ERR_ARG;
    if (!stream) return bfail(b, LBM_ERR_ARG, "a batch needs a non-default stream (graphs)");
    if (b->dev_ready) LBM_BCUDA(cudaStreamSynchronize(b->stream), "sync");
    if (b->own_stream) {
        cudaStreamDestroy(b->stream);
        b->own_stream = false;
    }
    b->stream = (cudaStream_t)stream;
    drop_graph(b);
    return LBM_OK;
}

int lbm_batch_set_allocator(lbm_batch* b, lbm_alloc_fn alloc, lbm_free_fn free_fn, void* user) {
    if (!b) return LBM_ERR_ARG;
    if (b->dev_ready) return bfail(b, LBM_ERR_STATE, "allocator must be set before first device use");
    if ((alloc == nullptr) != (free_fn == nullptr)) return LBM_ERR_ARG;
    b->af = alloc;
    b->ff = free_fn;
    b->au = user;
    return LBM_OK;
}

int lbm_batch_set_params(lbm_batch* b, const lbm_params* p) {
    if (!b || !p) return LBM_ERR_ARG;
    if (!(p->g >= 0.0) || !(p->rho_l > 0.0) || !(p->rho_ratio >= 0.0 && p->rho_ratio < 1.0) ||
        !(p->sigma > 0.0) || !(p->c_added_mass >= 0.0) || !(p->drag_scale >= 0.0) ||
        !(p->sn_coeff >= 0.0) || !(p->sn_exp > 0.0) || !(p->width_factor > 0.0) ||
        p->substeps < 1 || p->substeps > 10000 || p->rho_ratio + p->c_added_mass <= 0.0 ||
        (p->forces & ~(LBM_FORCE_LIFT | LBM_FORCE_STRESS)) ||
        (p->mapping != LBM_MAP_CELL && p->mapping != LBM_MAP_POINT) ||
        (p->reaction != LBM_REACTION_DRAG_LIFT && p->reaction != LBM_REACTION_ALL))
        return bfail(b, LBM_ERR_ARG, "parameter out of range");
    if (b->bub.nb > 0 && ((p->forces ^ b->p.forces) & LBM_FORCE_LIFT))
        return bfail(b, LBM_ERR_STATE, "switch lift before lbm_batch_set_bubbles");
    if (b->bub.nb > 0 && p->width_factor != b->p.width_factor)
        return bfail(b, LBM_ERR_STATE, "set width_factor before lbm_batch_set_bubbles");
    if (b->bub.nb > 0 && p->mapping != b->p.mapping)
        return bfail(b, LBM_ERR_STATE, "set the mapping before lbm_batch_set_bubbles");
    if (b->dev_ready && p->rho_l != b->p.rho_l)
        return bfail(b, LBM_ERR_STATE, "rho_l is the storage reference; set it before first use");
    const bool remap = b->dev_ready && p->mapping != b->p.mapping;
    b->p = *p;
    if (remap) {   // the column table carries the mapping mode
        layout_columns(b);
        int rc = upload_columns(b);
        if (rc) return rc;
    }
    if (b->bub.nb > 0)
        LBM_BCUDA(launch_bubble_constants_batch(b->bub, batch_bubble_const(b), b->col_nu_d,
                                                b->bubble_col_d, b->stream), "bubble constants");
    drop_graph(b);
    return LBM_OK;
}

int lbm_batch_set_bubbles(lbm_batch* b, const int* counts, const double* pos3, const double* vel3,
                          const double* diam) {
    if (!b || !counts) return LBM_ERR_ARG;
    int n = 0;
    for (int c = 0; c < b->ncols; ++c) {
        if (counts[c] < 0) return LBM_ERR_ARG;
        n += counts[c];
    }
    if (n > 0 && (!pos3 || !diam)) return bfail(b, LBM_ERR_ARG, "pos3 and diam are required");
    std::vector<int> col_of(n);
    double dmax = 0.0;
    for (int c = 0, k = 0; c < b->ncols; ++c) {
        const int L[3] = {b->dims[3 * c], b->dims[3 * c + 1], b->dims[3 * c + 2]};
        for (int i = 0; i < counts[c]; ++i, ++k) {
            col_of[k] = c;
            const double d = diam[k];
            if (!(d > 0.0 && d <= LBM_MAX_DIAMETER))
                return bfail(b, LBM_ERR_ARG, "bubble %d: diameter out of range", k);
            const double hw = b->p.width_factor * d;
            if (hw > MAX_HALF_WIDTH) return bfail(b, LBM_ERR_ARG, "bubble %d: window too wide", k);
            if (b->p.mapping == LBM_MAP_POINT && !(hw > 0.5))
                return bfail(b, LBM_ERR_ARG, "bubble %d: the point-sampled map needs a window "
                             "half-width above 1/2", k);
            dmax = std::fmax(dmax, d);
            for (int a = 0; a < 3; ++a) {
                const double x = pos3[3 * k + a];
                if (!(x >= 0.0 && x < (double)L[a]))
                    return bfail(b, LBM_ERR_ARG, "bubble %d: centre outside its column", k);
                const bool periodic = !(b->walls[c] & (1u << (2 * a)));
                const double halo = (b->p.forces & LBM_FORCE_LIFT) ? 2.0 : 0.0;
                if (periodic && 2.0 * hw + 2.0 + halo > (double)L[a])
                    return bfail(b, LBM_ERR_ARG, "bubble %d: window wraps onto itself", k);
                if (!periodic && d >= (double)L[a])
                    return bfail(b, LBM_ERR_ARG, "bubble %d: wider than its column", k);
            }
        }
    }
    const double hwmax = b->p.width_factor * dmax;
    const int pad = (b->p.forces & LBM_FORCE_LIFT) ? 1 : 0;   // the lift's vorticity halo
    const long long per = (long long)axis_tile_bound(hwmax + pad, TX) *
                          axis_tile_bound(hwmax + pad, TY) * axis_tile_bound(hwmax + pad, TZ);
    if (per * n > SMALL_MAX_PAIRS)
        return bfail(b, LBM_ERR_ARG, "a batch bins at most %d (tile, bubble) pairs; %lld needed",
                     SMALL_MAX_PAIRS, per * n);
    int rc = ensure_device(b);
    if (rc) return rc;
    LBM_BCUDA(cudaStreamSynchronize(b->stream), "sync");
    free_bubbles(b);
    drop_graph(b);
    SmallBins& sb = b->small;
    cudaStream_t s = b->stream;
    LBM_BCUDA(cudaMemsetAsync(sb.count, 0, sizeof(int) * (size_t)sb.T, s), "count");
    LBM_BCUDA(cudaMemsetAsync(sb.prev_n, 0, sizeof(int), s), "prev_n");
    if (n == 0) return LBM_OK;
    BubbleDev& B = b->bub;
    const size_t f3 = sizeof(float) * 3 * (size_t)n, v1 = sizeof(double) * (size_t)n,
                 i1 = sizeof(int) * (size_t)n;
    B.k = (BubbleK*)balloc(b, sizeof(BubbleK) * (size_t)n);
    B.xh = (float*)balloc(b, f3);
    B.xl = (float*)balloc(b, f3);
    B.u = (float*)balloc(b, f3);
    B.d = (double*)balloc(b, v1);
    B.n = (double*)balloc(b, v1);
    B.ulprev = (float*)balloc(b, f3);
    B.ul = (float*)balloc(b, f3);
    B.psi = (float*)balloc(b, f3);
    B.out64 = (double*)balloc(b, sizeof(double) * 12 * (size_t)n);
    B.has_prev = (int*)balloc(b, i1);
    B.active = (int*)balloc(b, i1);
    B.spread = (int*)balloc(b, i1);
    B.cell = (int*)balloc(b, i1);
    B.rec = (BubbleRec*)balloc(b, sizeof(BubbleRec) * (size_t)n);
    b->bubble_col_d = (int*)balloc(b, i1);
    sb.parts = window_parts(hwmax, pad);
    sb.part = (float*)balloc(b, sizeof(float) * WIN_VALS_LIFT * WINDOW_CHUNKS_MAX * (size_t)n);
    sb.arrive = (int*)balloc(b, i1);
    if (!B.k || !B.xh || !B.xl || !B.u || !B.d || !B.n || !B.ulprev || !B.ul || !B.psi || !B.out64 ||
        !B.has_prev || !B.active || !B.spread || !B.cell || !B.rec || !b->bubble_col_d ||
        !sb.part || !sb.arrive) {
        free_bubbles(b);
        return bfail(b, LBM_ERR_ALLOC, "bubble state");
    }
    B.nb = n;
    std::vector<double> hn(n);
    for (int k = 0; k < n; ++k) hn[k] = b->p.width_factor * diam[k];
    std::vector<int> ones(n, 1), izero(n, 0), minus(n, -1);
    LBM_BCUDA(upload_bubble_state(B, n, pos3, vel3, s), "bubbles");
    LBM_BCUDA(cudaMemcpyAsync(B.d, diam, v1, cudaMemcpyHostToDevice, s), "diam");
    LBM_BCUDA(cudaMemcpyAsync(B.n, hn.data(), v1, cudaMemcpyHostToDevice, s), "n");
    LBM_BCUDA(cudaMemcpyAsync(B.has_prev, izero.data(), i1, cudaMemcpyHostToDevice, s), "has_prev");
    LBM_BCUDA(cudaMemcpyAsync(B.active, ones.data(), i1, cudaMemcpyHostToDevice, s), "active");
    LBM_BCUDA(cudaMemcpyAsync(B.spread, izero.data(), i1, cudaMemcpyHostToDevice, s), "spread");
    LBM_BCUDA(cudaMemcpyAsync(B.cell, minus.data(), i1, cudaMemcpyHostToDevice, s), "cell");
    LBM_BCUDA(cudaMemcpyAsync(b->bubble_col_d, col_of.data(), i1, cudaMemcpyHostToDevice, s), "col");
    LBM_BCUDA(cudaMemsetAsync(B.rec, 0, sizeof(BubbleRec) * (size_t)n, s), "rec");
    LBM_BCUDA(cudaMemsetAsync(sb.arrive, 0, i1, s), "arrive");
    LBM_BCUDA(launch_bubble_constants_batch(B, batch_bubble_const(b), b->col_nu_d, b->bubble_col_d, s),
              "bubble constants");
    LBM_BCUDA(cudaStreamSynchronize(s), "bubble upload");
    return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int nsteps) {
    if (!b || nsteps < 0) return LBM_ERR_ARG;
    int rc = ensure_device(b);
    if (rc) return rc;
    if (b->unstable) return bfail(b, LBM_ERR_UNSTABLE, "a column is unstable (sticky)");
    rc = run_steps(b, nsteps);
    if (rc) return rc;
    return check_flag(b);
}

int lbm_batch_tune(lbm_batch* b, int trial_steps, int* depth_out, int* grid_out) {
    if (!b || trial_steps < 2) return LBM_ERR_ARG;
    int rc = ensure_device(b);
    if (rc) return rc;
    if (b->unstable) return bfail(b, LBM_ERR_UNSTABLE, "a column is unstable (sticky)");
    trial_steps += trial_steps & 1;
    cudaStream_t s = b->stream;
    // Save the state the trials will advance: populations, bubbles, bins.
    const size_t fbytes = (size_t)b->total_elems * elem_bytes(b->storage);
    void* f_save = balloc(b, fbytes);
    const int n = b->bub.nb;
    const size_t bub_bytes = (size_t)n * (sizeof(float) * 18 + sizeof(int) * 4 + sizeof(BubbleRec));
    const size_t bin_bytes = sizeof(int) * ((size_t)b->small.T * 2 + 2 * SMALL_MAX_PAIRS + 1);
    char* aux = (char*)balloc(b, bub_bytes + bin_bytes + 16);
    if (!f_save || !aux) {
        bfree(b, f_save);
        bfree(b, aux);
        return bfail(b, LBM_ERR_ALLOC, "tuning backup");
    }
    struct Blob { void* p; size_t bytes; };
    const BubbleDev& B = b->bub;
    const SmallBins& sb = b->small;
    const Blob blobs[] = {
        {B.xh, sizeof(float) * 3 * (size_t)n}, {B.xl, sizeof(float) * 3 * (size_t)n},
        {B.u, sizeof(float) * 3 * (size_t)n}, {B.ulprev, sizeof(float) * 3 * (size_t)n},
        {B.ul, sizeof(float) * 3 * (size_t)n}, {B.psi, sizeof(float) * 3 * (size_t)n},
        {B.has_prev, sizeof(int) * (size_t)n},
        {B.active, sizeof(int) * (size_t)n}, {B.spread, sizeof(int) * (size_t)n},
        {B.cell, sizeof(int) * (size_t)n}, {B.rec, sizeof(BubbleRec) * (size_t)n},
        {sb.start, sizeof(int) * (size_t)sb.T}, {sb.count, sizeof(int) * (size_t)sb.T},
        {sb.items, sizeof(int) * SMALL_MAX_PAIRS}, {sb.prev_tiles, sizeof(int) * SMALL_MAX_PAIRS},
        {sb.prev_n, sizeof(int)}};
    const int cur0 = b->cur;
    LBM_BCUDA(cudaMemcpyAsync(f_save, b->f[cur0], fbytes, cudaMemcpyDeviceToDevice, s), "save f");
    size_t off = 0;
    for (const Blob& bl : blobs) {
        if (bl.p && bl.bytes)
            LBM_BCUDA(cudaMemcpyAsync(aux + off, bl.p, bl.bytes, cudaMemcpyDeviceToDevice, s), "save");
        off += bl.bytes;
    }
    int dev = 0, sms = 0;
    LBM_BCUDA(cudaGetDevice(&dev), "device");
    LBM_BCUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    // Candidates: CTA tiles of 32 x 4 x {1, 2, 4} nodes; work items of
    // {1, 2, 4, 8} z-blocks; half, one and two times the resident CTAs per SM
    // the kernel is compiled for.  Work items span the same planes whatever
    // the tile, so only the hand-out granularity and the CTA shape change.
    const int planes_c[] = {1, 2, 4};
    const int depths[] = {1, 2, 4, 8};
    cudaEvent_t t0, t1;
    LBM_BCUDA(cudaEventCreate(&t0), "event");
    LBM_BCUDA(cudaEventCreate(&t1), "event");
    float best = 1e30f;
    int best_planes = b->planes, best_depth = b->depth, best_grid = b->grid;
    const bool timing = b->timing;
    b->timing = false;
    for (int pl : planes_c) {
        const int maxb = batch_min_blocks(b->storage, pl);
        const int per_sm[] = {maxb / 2, maxb, 2 * maxb};
        for (int d : depths) {
            for (int k : per_sm) {
                b->planes = pl;
                b->depth = d;
                b->grid = sms * k;
                layout_columns(b);
                rc = upload_columns(b);
                if (!rc) rc = build_graph(b);
                if (!rc) rc = run_steps(b, 2);   // warm
                if (rc) break;
                cudaEventRecord(t0, s);
                rc = run_steps(b, trial_steps);
                cudaEventRecord(t1, s);
                if (rc) break;
                LBM_BCUDA(cudaEventSynchronize(t1), "trial");
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, t0, t1);
                if (ms < best) {
                    best = ms;
                    best_planes = pl;
                    best_depth = d;
                    best_grid = b->grid;
                }
            }
            if (rc) break;
        }
        if (rc) break;
    }
    b->timing = timing;
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    // Restore the state and keep the winner.
    b->planes = best_planes;
    b->depth = best_depth;
    b->grid = best_grid;
    layout_columns(b);
    int rc2 = upload_columns(b);
    b->cur = cur0;
    LBM_BCUDA(cudaMemcpyAsync(b->f[cur0], f_save, fbytes, cudaMemcpyDeviceToDevice, s), "restore f");
    off = 0;
    for (const Blob& bl : blobs) {
        if (bl.p && bl.bytes)
            LBM_BCUDA(cudaMemcpyAsync(bl.p, aux + off, bl.bytes, cudaMemcpyDeviceToDevice, s), "restore");
        off += bl.bytes;
    }
    LBM_BCUDA(cudaMemsetAsync(b->flag_d, 0, sizeof(int), s), "flag");
    LBM_BCUDA(cudaStreamSynchronize(s), "restore");
    bfree(b, f_save);
    bfree(b, aux);
    drop_graph(b);
    if (rc) return rc;
    if (rc2) return rc2;
    b->unstable = false;
    b->tuned = true;
    if (depth_out) *depth_out = best_depth;
    if (grid_out) *grid_out = best_grid;
    return LBM_OK;
}

int lbm_batch_set_launch_shape(lbm_batch* b, int planes, int depth, int grid) {
    if (!b) return LBM_ERR_ARG;
    if ((planes != 1 && planes != 2 && planes != 4) || depth < 1 || depth > 64 || grid < 0 ||
        grid > (1 << 20))
        return bfail(b, LBM_ERR_ARG, "launch shape out of range (planes 1, 2 or 4)");
    b->planes = planes;
    b->depth = depth;
    if (grid > 0) {
        b->grid = grid;
    } else if (b->dev_ready) {
        int dev = 0, sms = 0;
        LBM_BCUDA(cudaGetDevice(&dev), "device");
        LBM_BCUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
        b->grid = sms * batch_min_blocks(b->storage, planes);
    }
    if (b->dev_ready) {
        layout_columns(b);
        int rc = upload_columns(b);
        if (rc) return rc;
    }
    drop_graph(b);
    b->grid_fixed = grid > 0;
    return LBM_OK;
}

int lbm_batch_launch_shape(const lbm_batch* b, int* planes, int* depth, int* grid) {
    if (!b) return LBM_ERR_ARG;
    if (planes) *planes = b->planes;
    if (depth) *depth = b->depth;
    if (grid) *grid = b->grid;
    return LBM_OK;
}

int lbm_batch_get_fields(lbm_batch* b, int col, double* rho, double* u3) {
    if (!b || col < 0 || col >= b->ncols) return LBM_ERR_ARG;
    int rc = ensure_device(b);
    if (rc) return rc;
    if (!rho && !u3) return LBM_OK;
    const BatchColumn& c = b->cols[col];
    const size_t S = (size_t)c.g.S;
    double* rd = rho ? (double*)balloc(b, sizeof(double) * S) : nullptr;
    double* ud = u3 ? (double*)balloc(b, sizeof(double) * 3 * S) : nullptr;
    if ((rho && !rd) || (u3 && !ud)) {
        bfree(b, rd);
        bfree(b, ud);
        return bfail(b, LBM_ERR_ALLOC, "field staging");
    }
    const char* base = (const char*)b->f[b->cur] + (size_t)c.pop_offset * elem_bytes(b->storage);
    cudaError_t e = launch_fields(b->storage, base, c.g, c.cp, rd, ud, b->stream);
    if (e == cudaSuccess && rho)
        e = cudaMemcpyAsync(rho, rd, sizeof(double) * S, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess && u3)
        e = cudaMemcpyAsync(u3, ud, sizeof(double) * 3 * S, cudaMemcpyDeviceToHost, b->stream);
    cudaError_t e2 = cudaStreamSynchronize(b->stream);
    bfree(b, rd);
    bfree(b, ud);
    if (e != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "get fields: %s", cudaGetErrorString(e));
    if (e2 != cudaSuccess) return bfail(b, LBM_ERR_CUDA, "get fields: %s", cudaGetErrorString(e2));
    return LBM_OK;
}

int lbm_batch_get_bubbles(lbm_batch* b, int cap, int* n, double* pos3, double* vel3, double* ul3,
                          double* psi3, int* active) {
    if (!b || cap < 0) return LBM_ERR_ARG;
    const int nb = b->bub.nb;
    if (n) *n = nb;
    const int k = nb < cap ? nb : cap;
    if (k == 0) return LBM_OK;
    cudaStream_t s = b->stream;
    LBM_BCUDA(download_bubble_state(b->bub, k, pos3, vel3, ul3, psi3, s), "bubbles");
    if (active)
        LBM_BCUDA(cudaMemcpyAsync(active, b->bub.active, sizeof(int) * (size_t)k,
                                  cudaMemcpyDeviceToHost, s), "active");
    LBM_BCUDA(cudaStreamSynchronize(s), "get bubbles");
    return LBM_OK;
}

long long lbm_batch_sites(const lbm_batch* b) { return b ? b->total_sites : 0; }

int lbm_batch_set_kernel_timing(lbm_batch* b, int on) {
    if (!b) return LBM_ERR_ARG;
    if (b->dev_ready) LBM_BCUDA(cudaStreamSynchronize(b->stream), "sync");
    b->timing = on != 0;
    b->events_used = 0;
    return LBM_OK;
}

int lbm_batch_get_kernel_time(lbm_batch* b, double* ms, int* launches) {
    if (!b) return LBM_ERR_ARG;
    if (b->dev_ready) LBM_BCUDA(cudaStreamSynchronize(b->stream), "sync");
    double total = 0.0;
    for (size_t i = 0; i < b->events_used; ++i) {
        float t = 0.0f;
        LBM_BCUDA(cudaEventElapsedTime(&t, b->events[i].first, b->events[i].second), "elapsed");
        total += t;
    }
    if (ms) *ms = total;
    if (launches) *launches = (int)b->events_used;
    b->events_used = 0;
    return LBM_OK;
}

long long lbm_batch_launch_count(const lbm_batch* b) { return b ? b->launches : 0; }

int lbm_batch_sync(lbm_batch* b) {
    if (!b) return LBM_ERR_ARG;
    if (!b->dev_ready) return LBM_OK;
    LBM_BCUDA(cudaStreamSynchronize(b->stream), "sync");
    return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : "null batch"; }

}  // extern "C"
