// Host side of the C ABI declared in include/lbm.h: argument checks, device
// state, and the order of launches of one coupled step (Algorithm 1 of
// arXiv:1710.07073).
#include <algorithm>
#include <climits>
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

#include "lbm_ctx.hpp"

int fail(lbm_ctx* c, int code, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

int cuda_fail(lbm_ctx* c, cudaError_t e, const char* what) {
    return fail(c, LBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void* dalloc(lbm_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (c->af) {
        p = c->af(bytes, c->au);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->allocs.emplace_back(p, bytes);
    return p;
}

void dfree(lbm_ctx* c, void* p) {
    if (!p) return;
    for (size_t i = 0; i < c->allocs.size(); ++i) {
        if (c->allocs[i].first == p) {
            if (c->ff) c->ff(p, c->allocs[i].second, c->au);
            else cudaFree(p);
            c->allocs.erase(c->allocs.begin() + (long)i);
            return;
        }
    }
}

size_t elem_size(int storage) { return storage == LBM_STORE_F32 ? 4 : 2; }

Geo geo_of(const lbm_ctx* c) {
    Geo g;
    g.nx = c->nx;
    g.ny = c->ny;
    g.nz = c->nz;
    g.walls = c->walls;
    g.S = (long long)c->nx * c->ny * c->nz;
    g.ntx = (c->nx + TX - 1) / TX;
    g.nty = (c->ny + TY - 1) / TY;
    g.ntz = (c->nz + TZ - 1) / TZ;
    return g;
}

CollideParams collide_params(const lbm_ctx* c) {
    CollideParams cp;
    cp.omega = (float)c->omega;
    cp.pref = (float)(1.0 - 0.5 * c->omega);
    cp.rho0 = (float)c->p.rho_l;
    cp.scale = (float)c->scale;
    cp.inv_scale = (float)(1.0 / c->scale);
    cp.point = c->p.mapping == LBM_MAP_POINT ? 1 : 0;
    return cp;
}

BubbleConst bubble_const(const lbm_ctx* c) {
    BubbleConst bc;
    bc.g = c->p.g;
    bc.rho_l = c->p.rho_l;
    bc.rho_b = c->p.rho_ratio * c->p.rho_l;
    bc.sigma = c->p.sigma;
    bc.c_am = c->p.c_added_mass;
    bc.drag_scale = c->p.drag_scale;
    bc.sn_coeff = c->p.sn_coeff;
    bc.sn_exp = c->p.sn_exp;
    bc.nu = (2.0 / c->omega - 1.0) / 6.0;     // Eq. 9
    bc.dt_l = 1.0;
    bc.dt_b = 1.0 / c->p.substeps;            // Table 2: dt_b = dt_l / substeps
    split_f2(bc.dt_b, bc.dt_bh, bc.dt_bl);
    bc.substeps = c->p.substeps;
    bc.lift = (c->p.forces & LBM_FORCE_LIFT) ? 1 : 0;
    bc.stress = (c->p.forces & LBM_FORCE_STRESS) ? 1 : 0;
    bc.point = c->p.mapping == LBM_MAP_POINT ? 1 : 0;
    bc.reaction_all = c->p.reaction == LBM_REACTION_ALL ? 1 : 0;
    return bc;
}

// Device state of a context, allocated on first use.  All or nothing: if
// any allocation fails, what this call allocated is freed again, so the
// context stays destroyable and a later call may retry.
int ensure_device(lbm_ctx* c) {
    if (c->dev_ready) return LBM_OK;
    LBM_CUDA(cudaGetDevice(&c->device), "cudaGetDevice");
    const Geo g = geo_of(c);
    const size_t bytes = (size_t)Q * (size_t)g.S * elem_size(c->storage);
    c->bins.T = g.ntx * g.nty * g.ntz;
    c->bins.nblocks = scan_blocks(c->bins.T);
    for (int k = 0; k < 2; ++k) c->f[k] = dalloc(c, bytes);
    c->flag_d = (int*)dalloc(c, sizeof(int));
    c->bins.cnt = (int*)dalloc(c, sizeof(int) * (size_t)c->bins.T);
    c->bins.off = (int*)dalloc(c, sizeof(int) * ((size_t)c->bins.T + 1));
    c->bins.block_sums = (int*)dalloc(c, sizeof(int) * (size_t)c->bins.nblocks);
    c->bins.overflow = (int*)dalloc(c, sizeof(int));
    if (!c->f[0] || !c->f[1] || !c->flag_d || !c->bins.cnt || !c->bins.off ||
        !c->bins.block_sums || !c->bins.overflow) {
        void** owned[] = {&c->f[0], &c->f[1], (void**)&c->flag_d, (void**)&c->bins.cnt,
                          (void**)&c->bins.off, (void**)&c->bins.block_sums,
                          (void**)&c->bins.overflow};
        for (void** q : owned) {
            dfree(c, *q);
            *q = nullptr;
        }
        return fail(c, LBM_ERR_ALLOC, "device state of the column (%zu bytes per population "
                    "buffer)", bytes);
    }
    if (!c->flag_h) LBM_CUDA(cudaMallocHost((void**)&c->flag_h, sizeof(int)), "cudaMallocHost");
    // Rest state f = f^eq(rho_l, 0) has zero shifted value in every format.
    LBM_CUDA(cudaMemsetAsync(c->f[0], 0, bytes, c->stream), "memset f");
    LBM_CUDA(cudaMemsetAsync(c->flag_d, 0, sizeof(int), c->stream), "memset flag");
    c->cur = 0;
    LBM_CUDA(cudaMemsetAsync(c->bins.overflow, 0, sizeof(int), c->stream), "memset overflow");
    c->bins.items = nullptr;
    c->bins.cap = 0;
    c->dev_ready = true;
    return LBM_OK;
}

namespace {

int check_walls(unsigned walls) {
    if (walls & ~0x7Fu) return 0;
    for (int a = 0; a < 3; ++a) {
        bool lo = walls & (1u << (2 * a)), hi = walls & (1u << (2 * a + 1));
        if (lo != hi) return 0;
    }
    if ((walls & WALL_TOP_FREE) && !(walls & 0x20)) return 0;   // a free-slip top bounds z
    return 1;
}

// Tiles a window of half-width n can touch along an axis of tile size T.
int axis_tile_bound(double n, int T) {
    int cells = (int)std::ceil(2.0 * n) + 1;
    return (cells + T - 1) / T + 1;
}

void free_bubbles(lbm_ctx* c) {
    BubbleDev& b = c->bub;
    SmallBins& sb = c->small;
    SwarmBins& sw = c->swarm;
    void* ptrs[] = {b.k, b.xh, b.xl, b.u, b.d, b.n, b.ulprev, b.ul, b.psi, b.out64, b.has_prev,
                    b.active, b.spread, b.cell, b.rec, c->bins.items, sb.start, sb.count, sb.items,
                    sb.prev_tiles, sb.prev_n, sb.overflow, sb.done, sb.part, sb.arrive, sb.safe,
                    sb.zperm, sb.zrange, sw.bar, sw.cursor, sw.kidx, sw.slots, sw.ntile, sw.partial, sw.cover,
                    sw.ncover, sw.chunk_sums, sw.zrange};
    for (void* p : ptrs) dfree(c, p);
    c->cover_valid = false;
    b = BubbleDev{};
    sb = SmallBins{};
    sw = SwarmBins{};
    c->bins.items = nullptr;
    c->bins.cap = 0;
    c->nb_cap = 0;
    c->use_small = false;
    guard_invalidate(c);
}

}  // namespace

void guard_invalidate(lbm_ctx* c) {
    c->epoch += 1;
    c->swarm_valid_from = c->swarm_step;   // older z ranges say nothing of the new state
}

namespace {

// Two tag sets of ntz (zero: no layer cleared) and two sweep orders of nbz z
// blocks (identity), by step parity.
int alloc_guard(lbm_ctx* c, unsigned** safe, int** zperm, int* nbz, int** zrange) {
    const Geo g = geo_of(c);
    *nbz = sweep_z_blocks(g.nz);
    *safe = (unsigned*)dalloc(c, 2 * sizeof(unsigned) * (size_t)g.ntz);
    *zperm = (int*)dalloc(c, 2 * sizeof(int) * (size_t)*nbz);
    *zrange = (int*)dalloc(c, 2 * sizeof(int));
    if (!*safe || !*zperm || !*zrange) return LBM_ERR_ALLOC;
    std::vector<int> ident(2 * (size_t)*nbz);
    for (int k = 0; k < 2 * *nbz; ++k) ident[k] = k % *nbz;
    LBM_CUDA(cudaMemsetAsync(*safe, 0, 2 * sizeof(unsigned) * (size_t)g.ntz, c->stream), "guard");
    LBM_CUDA(cudaMemcpyAsync(*zperm, ident.data(), sizeof(int) * ident.size(),
                             cudaMemcpyHostToDevice, c->stream), "sweep order");
    return LBM_OK;
}

}  // namespace

// Interpolation CTAs per SM while the sweep of the blocks no bubble reaches
// runs beside it (GB300, swarm 384x384x768: 2 gives the shortest step; 4,
// the interpolation's own occupancy, leaves the sweep no room; 1 starves it).
#ifndef LBM_SPLIT_INTERP_PER_SM
#define LBM_SPLIT_INTERP_PER_SM 2
#endif

// Few bubbles: the split pays only where the sweep is long against the
// step's extra host and stream work (fork, join, read-back, a third launch):
// on GB300 256x256x512 gains (FP16 step 0.460 -> 0.445 ms), 128x128x256
// loses (0.102 -> 0.120 s for 1000 forward steps).
#ifndef LBM_FEW_SPLIT_MIN_SITES
#define LBM_FEW_SPLIT_MIN_SITES (1LL << 24)
#endif


namespace {

// Streams, events and pinned slots of the split sweep, made on first use.
int ensure_split(lbm_ctx* c) {
    if (c->side_hi) return LBM_OK;
    int least = 0, greatest = 0;
    LBM_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest), "stream priorities");
    LBM_CUDA(cudaStreamCreateWithPriority(&c->side_hi, cudaStreamNonBlocking, greatest), "stream");
    LBM_CUDA(cudaStreamCreateWithPriority(&c->side_lo, cudaStreamNonBlocking, least), "stream");
    LBM_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming), "event");
    LBM_CUDA(cudaEventCreateWithFlags(&c->ev_hi, cudaEventDisableTiming), "event");
    LBM_CUDA(cudaEventCreateWithFlags(&c->ev_lo, cudaEventDisableTiming), "event");
    for (int k = 0; k < lbm_ctx::SPLIT_RING; ++k) {
        LBM_CUDA(cudaEventCreateWithFlags(&c->ev_rb[k], cudaEventDisableTiming), "event");
        c->rb_step[k] = -1;
    }
    LBM_CUDA(cudaHostAlloc((void**)&c->zr_host, 2 * sizeof(int) * lbm_ctx::SPLIT_RING,
                           cudaHostAllocDefault), "pinned z range");
    int dev = 0;
    LBM_CUDA(cudaGetDevice(&dev), "device");
    LBM_CUDA(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    return LBM_OK;
}

void destroy_split(lbm_ctx* c) {
    if (c->side_hi) cudaStreamSynchronize(c->side_hi);
    if (c->side_lo) cudaStreamSynchronize(c->side_lo);
    if (c->side_hi) cudaStreamDestroy(c->side_hi);
    if (c->side_lo) cudaStreamDestroy(c->side_lo);
    for (cudaEvent_t e : {c->ev_fork, c->ev_hi, c->ev_lo})
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_rb)
        if (e) cudaEventDestroy(e);
    if (c->zr_host) cudaFreeHost(c->zr_host);
}

// The z blocks [*b0, *b1) that bubble forces may reach in step n, from the z
// range read back SPLIT_LAG steps before (the many-bubble binning's lists, or
// the few-bubble update's guarded layers, which already reach one step on): a
// bubble moves at most GUARD_CELLS = TZ cells, one tile layer, per step (else
// the step is flagged unstable).  Returns false if no such read-back is at
// hand.
bool guarded_blocks(lbm_ctx* c, const Geo& g, int* b0, int* b1, int* rc) {
    *rc = LBM_OK;
    const long long n = c->swarm_step, m = n - lbm_ctx::SPLIT_LAG;
    if (!c->side_hi || m < 0 || m < c->swarm_valid_from) return false;
    const int slot = (int)(m % lbm_ctx::SPLIT_RING);
    if (c->rb_step[slot] != m) return false;
    const cudaError_t e = cudaEventSynchronize(c->ev_rb[slot]);
    if (e != cudaSuccess) {
        *rc = cuda_fail(c, e, "z range read-back");
        return false;
    }
    static_assert(GUARD_CELLS <= TZ, "a bubble crosses at most one tile layer per step");
    const int zlo = c->zr_host[2 * slot], zhi = c->zr_host[2 * slot + 1];
    const int nbz = sweep_z_blocks(g.nz);
    if (zhi < zlo) {
        *b0 = *b1 = 0;
        return true;
    }
    const int widen = (int)(n - m) + 1;
    const int l0 = std::max(0, zlo - widen), l1 = std::min(g.ntz - 1, zhi + widen);
    *b0 = std::min(nbz, l0 * TZ / SWEEP_PZ);
    *b1 = std::min(nbz, (l1 + 1) * TZ / SWEEP_PZ);
    return true;
}

}  // namespace

int enqueue_one_step(lbm_ctx* c) {
    const Geo g = geo_of(c);
    const CollideParams cp = collide_params(c);
    const bool bubbles = c->bub.nb > 0;
    const bool two_way = bubbles && c->p.two_way;
    // Two-way coupling on even rows: the update and the sweep overlap
    // (programmatic dependent launches), guarded by the tags the update before
    // wrote.  Timed launches keep plain stream order so that the sweep's
    // events time the sweep alone.
    unsigned* const safe = c->use_small ? c->small.safe : nullptr;
    int* const zperm = c->use_small ? c->small.zperm : nullptr;
    const int nbz = c->small.nbz;
    const bool overlap = two_way && safe != nullptr && !c->timing && (g.nx & 1) == 0;
    if (c->epoch >= 0xFFFFFF00u) {
        // Before the step number wraps: no stored tag may match a later one.
        if (safe)
            LBM_CUDA(cudaMemsetAsync(safe, 0, 2 * sizeof(unsigned) * (size_t)g.ntz, c->stream),
                     "guard reset");
        c->epoch = 1;
    }
    const unsigned epoch = c->epoch++;
    // Tag sets and sweep orders by step parity: this step's sweep reads set
    // (epoch & 1) while its update writes the next step's into the other.
    const size_t now = epoch & 1u, next = (epoch + 1u) & 1u;
    const unsigned* safe_now = safe ? safe + now * (size_t)g.ntz : nullptr;
    const int* zperm_now = zperm ? zperm + now * (size_t)nbz : nullptr;
    const int pad = (c->p.forces & LBM_FORCE_LIFT) ? 1 : 0;   // the vorticity halo
    // Split step (wall-bounded z, even rows): the update and the sweep of the
    // z blocks bubble forces can reach run on a high-priority side stream
    // while the other blocks are swept (without forces) on a low-priority
    // one; the step then joins on c->stream.  The per-node arithmetic is the
    // same, so are the results.  Many bubbles take the z range of the
    // binning's lists, few bubbles that of the update's guarded layers.
    const bool many = bubbles && !c->use_small;
    const bool few_split = c->use_small && g.S >= LBM_FEW_SPLIT_MIN_SITES;
    const int* zrange_d = many ? c->swarm.zrange : (few_split ? c->small.zrange : nullptr);
    const bool split_able = bubbles && zrange_d != nullptr && two_way && !c->timing &&
                            (g.nx & 1) == 0 && (c->walls & 0x30) == 0x30;
    int gb0 = 0, gb1 = 0;
    bool split = false;
    if (split_able) {
        int rc = ensure_split(c);
        if (rc) return rc;
        split = guarded_blocks(c, g, &gb0, &gb1, &rc);
        if (rc) return rc;
    }
    cudaStream_t st = c->stream;   // the update and the guarded sweep
    if (split) {
        const int nbz = sweep_z_blocks(g.nz);
        LBM_CUDA(cudaEventRecord(c->ev_fork, c->stream), "fork");
        LBM_CUDA(cudaStreamWaitEvent(c->side_hi, c->ev_fork, 0), "fork");
        LBM_CUDA(cudaStreamWaitEvent(c->side_lo, c->ev_fork, 0), "fork");
        const ZSpan free_span{0, nbz - (gb1 - gb0), gb0, gb1 - gb0};
        LBM_CUDA(launch_collide_stream(c->storage, c->f[c->cur], c->f[c->cur ^ 1], g, cp, nullptr,
                                       c->bub.rec, c->bub.nb, c->flag_d, nullptr, epoch, false,
                                       nullptr, c->side_lo, &free_span),
                 "collide-stream (no bubble reaches)");
        LBM_CUDA(cudaEventRecord(c->ev_lo, c->side_lo), "join");
        if (free_span.count > 0) c->launches += 1;
        st = c->side_hi;
    }
    if (bubbles) {
        if (c->use_small) {
            SmallBins sb = c->small;
            sb.parts = window_parts(c->hwmax, pad);
            if (sb.safe) sb.safe += next * (size_t)g.ntz;
            if (sb.zperm) sb.zperm += next * (size_t)nbz;
            sb.safe_epoch = epoch + 1;   // the update clears layers for the next step
            LBM_CUDA(launch_bubbles(c->storage, c->f[c->cur], g, cp, c->bub, bubble_const(c),
                                    c->flag_d, sb, overlap && !split, st),
                     "bubble update");
            c->launches += 1;   // binning fused into the bubble update
        } else {
            // The tile lists of the current centres and their spreading
            // records: left by the previous step, else made here from
            // `active` (first step after the bubbles were set).
            if (!c->cover_valid) {
                LBM_CUDA(launch_bubble_records(g, c->bub, st), "records");
                LBM_CUDA(cudaMemsetAsync(c->bins.cnt, 0, sizeof(int) * (size_t)c->bins.T, st),
                         "cover counts");
                LBM_CUDA(cudaMemsetAsync(c->swarm.ncover, 0, sizeof(int), st), "cover list");
                SwarmBins sw = c->swarm;
                sw.pad = pad;
                LBM_CUDA(launch_swarm_binning(g, c->bub, c->bins, sw, c->bub.active, c->flag_d, st),
                         "cover");
                c->launches += 2;
            }
            SwarmBins sw = c->swarm;
            sw.pad = pad;
            // Split: the persistent interpolation leaves room on every SM for
            // the sweep of the blocks bubbles do not reach.
            if (split && c->sms > 0)
                sw.interp_grid = std::min(sw.interp_grid, c->sms * LBM_SPLIT_INTERP_PER_SM);
            LBM_CUDA(launch_swarm_update(c->storage, c->f[c->cur], g, cp, c->bub, bubble_const(c),
                                         c->flag_d, c->bins, sw, st),
                     "bubble update");
            c->launches += SWARM_LAUNCHES;   // interpolation by tiles; update; binning
            c->cover_valid = true;
        }
        if (split_able) {
            // This step's z range, for the split SPLIT_LAG steps on.
            const int slot = (int)(c->swarm_step % lbm_ctx::SPLIT_RING);
            LBM_CUDA(cudaMemcpyAsync(c->zr_host + 2 * slot, zrange_d, 2 * sizeof(int),
                                     cudaMemcpyDeviceToHost, st), "z range");
            LBM_CUDA(cudaEventRecord(c->ev_rb[slot], st), "z range");
            c->rb_step[slot] = c->swarm_step;
        }
        c->swarm_step += 1;
        c->bins_valid = true;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->timing) {
        if (c->events_used == c->events.size()) {
            cudaEvent_t a, b;
            LBM_CUDA(cudaEventCreate(&a), "event");
            LBM_CUDA(cudaEventCreate(&b), "event");
            c->events.emplace_back(a, b);
        }
        e0 = c->events[c->events_used].first;
        e1 = c->events[c->events_used].second;
        ++c->events_used;
        LBM_CUDA(cudaEventRecord(e0, c->stream), "event record");
    }
    TileLists tl{};
    if (c->use_small) tl = TileLists{c->small.start, c->small.count, c->small.items, SMALL_MAX_PAIRS};
    else tl = TileLists{c->bins.off, c->bins.cnt, c->bins.items, c->bins.cap};
    if (split) {
        const ZSpan guarded{gb0, gb1 - gb0, INT_MAX, 0};
        LBM_CUDA(launch_collide_stream(c->storage, c->f[c->cur], c->f[c->cur ^ 1], g, cp, &tl,
                                       c->bub.rec, c->bub.nb, c->flag_d, nullptr, epoch, false,
                                       nullptr, st, &guarded),
                 "collide-stream (bubbles reach)");
        LBM_CUDA(cudaEventRecord(c->ev_hi, st), "join");
        LBM_CUDA(cudaStreamWaitEvent(c->stream, c->ev_hi, 0), "join");
        LBM_CUDA(cudaStreamWaitEvent(c->stream, c->ev_lo, 0), "join");
        if (guarded.count > 0) c->launches += 1;
        c->cur ^= 1;
        return LBM_OK;
    }
    LBM_CUDA(launch_collide_stream(c->storage, c->f[c->cur], c->f[c->cur ^ 1], g, cp,
                                   two_way ? &tl : nullptr, c->bub.rec, c->bub.nb, c->flag_d,
                                   overlap ? safe_now : nullptr, epoch, overlap,
                                   two_way ? zperm_now : nullptr, c->stream),
             "collide-stream");
    if (c->timing) LBM_CUDA(cudaEventRecord(e1, c->stream), "event record");
    c->launches += 1;
    c->cur ^= 1;
    return LBM_OK;
}

// Wait for the enqueued steps and report the instability flag / overflow.
int finish_steps(lbm_ctx* c) {
    LBM_CUDA(cudaMemcpyAsync(c->flag_h, c->flag_d, sizeof(int), cudaMemcpyDeviceToHost,
                             c->stream), "read flag");
    LBM_CUDA(cudaStreamSynchronize(c->stream), "step");
    if (*c->flag_h & 8) {
        // A grid barrier of the many-bubble update gave up waiting: its
        // arrival counter may be left part-way, so it starts again at zero.
        c->unstable = true;
        if (c->swarm.bar)
            LBM_CUDA(cudaMemsetAsync(c->swarm.bar, 0, 2 * sizeof(unsigned), c->stream), "barrier");
        LBM_CUDA(cudaStreamSynchronize(c->stream), "barrier reset");
        return fail(c, LBM_ERR_TIMEOUT,
                    "a device-wide wait of the bubble update ran out (more than 1 s)");
    }
    if (*c->flag_h) {
        c->unstable = true;
        return fail(c, LBM_ERR_UNSTABLE,
                    "non-finite value or |u| >= 0.3 in the liquid, or a bubble faster than %d "
                    "cells per step", GUARD_CELLS);
    }
    if (c->bins_valid) {
        int ov = 0;
        LBM_CUDA(cudaMemcpy(&ov, c->use_small ? c->small.overflow : c->bins.overflow, sizeof(int),
                            cudaMemcpyDeviceToHost), "overflow");
        if (ov) return fail(c, LBM_ERR_STATE, "tile list capacity exceeded");
    }
    return LBM_OK;
}

extern "C" {

void lbm_default_params(lbm_params* p) {
    if (!p) return;
    p->g = 1e-5;
    p->rho_l = 1.0;
    p->rho_ratio = 1e-3;
    p->sigma = 5.84e-6;
    p->c_added_mass = 0.5;
    p->drag_scale = 1.0;
    p->sn_coeff = 0.15;
    p->sn_exp = 0.687;
    p->width_factor = 1.5;
    p->substeps = 10;
    p->two_way = 1;
    p->forces = 0;
    p->mapping = LBM_MAP_CELL;
    p->reaction = LBM_REACTION_DRAG_LIFT;
}

void lbm_velocity_set(int* c57, double* w19) {
    for (int j = 0; j < Q; ++j) {
        if (c57) {
            c57[3 * j] = cx(j);
            c57[3 * j + 1] = cy(j);
            c57[3 * j + 2] = cz(j);
        }
        if (w19) w19[j] = wd(j);
    }
}

// Appendix A: lattice-per-physical factors from Delta x_lu = Delta t_lu = 1
// and rho_pu = rho_lu LCF^3 / MCF; each quantity scales by its dimensions.
int lbm_units_from_physical(const lbm_physical* ph, lbm_units* u, lbm_params* p,
                            double* omega) {
    if (!ph || !u) return LBM_ERR_ARG;
    const double v[8] = {ph->dx, ph->dt, ph->rho_l, ph->rho_b, ph->mu_l, ph->sigma, ph->g,
                         ph->rho_l_lu};
    for (int i = 0; i < 8; ++i)
        if (!std::isfinite(v[i]) || v[i] < 0.0) return LBM_ERR_ARG;
    if (!(ph->dx > 0.0 && ph->dt > 0.0 && ph->rho_l > 0.0 && ph->mu_l > 0.0 &&
          ph->sigma > 0.0 && ph->rho_l_lu > 0.0) || !(ph->rho_b < ph->rho_l))
        return LBM_ERR_ARG;
    const double lcf = 1.0 / ph->dx, tcf = 1.0 / ph->dt;
    const double mcf = ph->rho_l_lu * lcf * lcf * lcf / ph->rho_l;
    const double nu_lu = ph->mu_l / ph->rho_l * lcf * lcf / tcf;
    u->lcf = lcf;
    u->tcf = tcf;
    u->mcf = mcf;
    if (p) {
        p->g = ph->g * lcf / (tcf * tcf);
        p->rho_l = ph->rho_l_lu;
        p->rho_ratio = ph->rho_b / ph->rho_l;
        p->sigma = ph->sigma * mcf / (tcf * tcf);
    }
    if (omega) *omega = 1.0 / (3.0 * nu_lu + 0.5);   // Eq. 9
    return LBM_OK;
}

int lbm_create_storage(int nx, int ny, int nz, double omega, unsigned walls, int storage,
                       double scale, lbm_ctx** out) {
    if (!out) return LBM_ERR_ARG;
    *out = nullptr;
    if (nx <= 0 || ny <= 0 || nz <= 0) return LBM_ERR_ARG;
    if ((long long)nx * ny * nz * Q >= (1LL << 32)) return LBM_ERR_ARG;   // 32-bit indices
    if (!(omega > 0.0 && omega < 2.0)) return LBM_ERR_ARG;
    if (!check_walls(walls)) return LBM_ERR_ARG;
    if (storage < LBM_STORE_F32 || storage > LBM_STORE_BF16) return LBM_ERR_ARG;
    if (storage != LBM_STORE_F32 && !(scale > 0.0 && std::isfinite(scale))) return LBM_ERR_ARG;
    lbm_ctx* c = new lbm_ctx();
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->walls = walls;
    c->omega = omega;
    c->storage = storage;
    c->scale = storage == LBM_STORE_F32 ? 1.0 : scale;
    lbm_default_params(&c->p);
    *out = c;
    return LBM_OK;
}

int lbm_create(int nx, int ny, int nz, double omega, unsigned walls, lbm_ctx** out) {
    return lbm_create_storage(nx, ny, nz, omega, walls, LBM_STORE_F32, 1.0, out);
}

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    if (c->dev_ready) cudaStreamSynchronize(c->stream);
    destroy_split(c);
    adjoint_free(c);
    for (auto& e : c->events) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    while (!c->allocs.empty()) dfree(c, c->allocs.back().first);
    if (c->flag_h) cudaFreeHost(c->flag_h);
    delete c;
}

int lbm_set_stream(lbm_ctx* c, void* stream) {
    if (!c) return LBM_ERR_ARG;
    c->stream = (cudaStream_t)stream;
    return LBM_OK;
}

int lbm_set_allocator(lbm_ctx* c, lbm_alloc_fn alloc, lbm_free_fn free_fn, void* user) {
    if (!c) return LBM_ERR_ARG;
    if (c->dev_ready) return fail(c, LBM_ERR_STATE, "allocator must be set before first device use");
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(c, LBM_ERR_ARG, "alloc and free must both be set or both be NULL");
    c->af = alloc;
    c->ff = free_fn;
    c->au = user;
    return LBM_OK;
}

int lbm_set_params(lbm_ctx* c, const lbm_params* p) {
    if (!c || !p) return LBM_ERR_ARG;
    if (!(p->g >= 0.0) || !(p->rho_l > 0.0) || !(p->rho_ratio >= 0.0 && p->rho_ratio < 1.0) ||
        !(p->sigma > 0.0) || !(p->c_added_mass >= 0.0) || !(p->drag_scale >= 0.0) ||
        !(p->sn_coeff >= 0.0) || !(p->sn_exp > 0.0) || !(p->width_factor > 0.0) ||
        p->substeps < 1 || p->substeps > 10000 ||
        (p->forces & ~(LBM_FORCE_LIFT | LBM_FORCE_STRESS)) ||
        (p->mapping != LBM_MAP_CELL && p->mapping != LBM_MAP_POINT) ||
        (p->reaction != LBM_REACTION_DRAG_LIFT && p->reaction != LBM_REACTION_ALL))
        return fail(c, LBM_ERR_ARG, "parameter out of range");
    if (p->rho_ratio + p->c_added_mass <= 0.0)
        return fail(c, LBM_ERR_ARG, "effective bubble mass must be positive");
    if (c->bub.nb > 0) {
        std::vector<double> d(c->bub.nb);
        LBM_CUDA(cudaMemcpy(d.data(), c->bub.d, sizeof(double) * d.size(), cudaMemcpyDeviceToHost),
                 "read diameters");
        const int pad = (p->forces & LBM_FORCE_LIFT) ? 1 : 0;
        const int L[3] = {c->nx, c->ny, c->nz};
        for (double v : d) {
            if (p->width_factor * v > MAX_HALF_WIDTH)
                return fail(c, LBM_ERR_ARG, "width_factor too large for the current bubbles");
            for (int a = 0; a < 3; ++a)
                if (!(c->walls & (1u << (2 * a))) &&
                    2.0 * p->width_factor * v + 2.0 + 2.0 * pad > (double)L[a])
                    return fail(c, LBM_ERR_ARG, "a window with the lift's halo wraps onto itself "
                                "on axis %d", a);
        }
        if (p->width_factor != c->p.width_factor)
            return fail(c, LBM_ERR_STATE, "set width_factor before lbm_set_bubbles");
        if (p->mapping != c->p.mapping)
            return fail(c, LBM_ERR_STATE, "set the mapping before lbm_set_bubbles");
    }
    adjoint_free(c);
    if ((p->forces ^ c->p.forces) & LBM_FORCE_LIFT) c->cover_valid = false;   // lists change reach
    c->p = *p;
    guard_invalidate(c);
    if (c->bub.nb > 0)
        LBM_CUDA(launch_bubble_constants(c->bub, bubble_const(c), c->stream), "bubble constants");
    return LBM_OK;
}

int lbm_get_params(const lbm_ctx* c, lbm_params* p) {
    if (!c || !p) return LBM_ERR_ARG;
    *p = c->p;
    return LBM_OK;
}

int lbm_set_fields(lbm_ctx* c, const double* rho, const double* u3) {
    if (!c) return LBM_ERR_ARG;
    adjoint_free(c);
    int rc = ensure_device(c);
    if (rc) return rc;
    const Geo g = geo_of(c);
    double* rho_d = nullptr;
    double* u_d = nullptr;
    if (rho) {
        rho_d = (double*)dalloc(c, sizeof(double) * (size_t)g.S);
        if (!rho_d) return fail(c, LBM_ERR_ALLOC, "rho staging");
        LBM_CUDA(cudaMemcpyAsync(rho_d, rho, sizeof(double) * (size_t)g.S, cudaMemcpyHostToDevice,
                                 c->stream), "upload rho");
    }
    if (u3) {
        u_d = (double*)dalloc(c, sizeof(double) * 3 * (size_t)g.S);
        if (!u_d) {
            dfree(c, rho_d);
            return fail(c, LBM_ERR_ALLOC, "u staging");
        }
        LBM_CUDA(cudaMemcpyAsync(u_d, u3, sizeof(double) * 3 * (size_t)g.S, cudaMemcpyHostToDevice,
                                 c->stream), "upload u");
    }
    cudaError_t e = launch_set_equilibrium(c->storage, rho_d, u_d, c->f[c->cur], g,
                                           collide_params(c), c->stream);
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    dfree(c, rho_d);
    dfree(c, u_d);
    if (e != cudaSuccess) return cuda_fail(c, e, "set equilibrium");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "set equilibrium (sync)");
    LBM_CUDA(cudaMemsetAsync(c->flag_d, 0, sizeof(int), c->stream), "memset flag");
    c->unstable = false;
    return LBM_OK;
}

int lbm_set_populations(lbm_ctx* c, const double* f) {
    if (!c || !f) return LBM_ERR_ARG;
    adjoint_free(c);
    int rc = ensure_device(c);
    if (rc) return rc;
    const Geo g = geo_of(c);
    const size_t bytes = sizeof(double) * Q * (size_t)g.S;
    double* fd = (double*)dalloc(c, bytes);
    if (!fd) return fail(c, LBM_ERR_ALLOC, "population staging");
    cudaError_t e = cudaMemcpyAsync(fd, f, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = launch_set_populations(c->storage, fd, c->f[c->cur], g, collide_params(c), c->stream);
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    dfree(c, fd);
    if (e != cudaSuccess) return cuda_fail(c, e, "set populations");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "set populations (sync)");
    LBM_CUDA(cudaMemsetAsync(c->flag_d, 0, sizeof(int), c->stream), "memset flag");
    c->unstable = false;
    return LBM_OK;
}

int lbm_get_populations(lbm_ctx* c, double* f) {
    if (!c || !f) return LBM_ERR_ARG;
    int rc = ensure_device(c);
    if (rc) return rc;
    const Geo g = geo_of(c);
    const size_t bytes = sizeof(double) * Q * (size_t)g.S;
    double* fd = (double*)dalloc(c, bytes);
    if (!fd) return fail(c, LBM_ERR_ALLOC, "population staging");
    cudaError_t e = launch_get_populations(c->storage, c->f[c->cur], g, collide_params(c), fd,
                                           c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, fd, bytes, cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    dfree(c, fd);
    if (e != cudaSuccess) return cuda_fail(c, e, "get populations");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "get populations (sync)");
    return LBM_OK;
}

int lbm_set_bubbles(lbm_ctx* c, int n, const double* pos3, const double* vel3,
                    const double* diam) {
    if (!c || n < 0) return LBM_ERR_ARG;
    if (n > 0 && (!pos3 || !diam)) return fail(c, LBM_ERR_ARG, "pos3 and diam are required");
    const int L[3] = {c->nx, c->ny, c->nz};
    for (int b = 0; b < n; ++b) {
        const double d = diam[b];
        if (!(d > 0.0 && d <= LBM_MAX_DIAMETER))
            return fail(c, LBM_ERR_ARG, "bubble %d: diameter %g outside (0, %g]", b, d,
                        (double)LBM_MAX_DIAMETER);
        const double hw = c->p.width_factor * d;
        if (hw > MAX_HALF_WIDTH)
            return fail(c, LBM_ERR_ARG, "bubble %d: window half-width %g exceeds %g", b, hw,
                        MAX_HALF_WIDTH);
        if (c->p.mapping == LBM_MAP_POINT && !(hw > 0.5))
            return fail(c, LBM_ERR_ARG, "bubble %d: the point-sampled map needs a window "
                        "half-width above 1/2 (got %g)", b, hw);
        const double halo = (c->p.forces & LBM_FORCE_LIFT) ? 2.0 : 0.0;
        for (int a = 0; a < 3; ++a) {
            const double x = pos3[3 * b + a];
            if (!(x >= 0.0 && x < (double)L[a]))
                return fail(c, LBM_ERR_ARG, "bubble %d: centre outside the box", b);
            const bool periodic = !(c->walls & (1u << (2 * a)));
            if (periodic && 2.0 * hw + 2.0 + halo > (double)L[a])
                return fail(c, LBM_ERR_ARG, "bubble %d: window wraps onto itself on axis %d", b, a);
            if (!periodic && d >= (double)L[a])
                return fail(c, LBM_ERR_ARG, "bubble %d: wider than the box on axis %d", b, a);
            if (vel3 && !std::isfinite(vel3[3 * b + a]))
                return fail(c, LBM_ERR_ARG, "bubble %d: non-finite velocity", b);
        }
    }
    int rc = ensure_device(c);
    if (rc) return rc;
    adjoint_free(c);
    LBM_CUDA(cudaStreamSynchronize(c->stream), "sync before bubble reset");
    free_bubbles(c);
    c->bins_valid = false;
    if (n == 0) return LBM_OK;

    BubbleDev& B = c->bub;
    const size_t f3 = sizeof(float) * 3 * (size_t)n, v1 = sizeof(double) * (size_t)n,
                 i1 = sizeof(int) * (size_t)n;
    B.xh = (float*)dalloc(c, f3);
    B.xl = (float*)dalloc(c, f3);
    B.u = (float*)dalloc(c, f3);
    B.d = (double*)dalloc(c, v1);
    B.n = (double*)dalloc(c, v1);
    B.ulprev = (float*)dalloc(c, f3);
    B.ul = (float*)dalloc(c, f3);
    B.psi = (float*)dalloc(c, f3);
    B.out64 = (double*)dalloc(c, sizeof(double) * 12 * (size_t)n);
    B.has_prev = (int*)dalloc(c, i1);
    B.active = (int*)dalloc(c, i1);
    B.spread = (int*)dalloc(c, i1);
    B.cell = (int*)dalloc(c, i1);
    B.rec = (BubbleRec*)dalloc(c, sizeof(BubbleRec) * (size_t)n);
    B.k = (BubbleK*)dalloc(c, sizeof(BubbleK) * (size_t)n);
    // Upper bound of (tile, bubble) pairs from the largest window, with the
    // one-cell halo lift may add.
    double dmax = 0.0;
    for (int b = 0; b < n; ++b) dmax = std::fmax(dmax, diam[b]);
    const double hwmax = c->p.width_factor * dmax;
    const long long per = (long long)axis_tile_bound(hwmax + 1.0, TX) *
                          axis_tile_bound(hwmax + 1.0, TY) * axis_tile_bound(hwmax + 1.0, TZ);
    const long long cap = per * n;
    if (cap >= (1LL << 31)) {
        free_bubbles(c);
        return fail(c, LBM_ERR_ARG, "too many bubbles for the tile lists");
    }
    bool lists_ok = true;
    c->use_small = cap <= SMALL_MAX_PAIRS;
    if (c->use_small) {
        SmallBins& sb = c->small;
        sb.T = c->bins.T;
        sb.start = (int*)dalloc(c, sizeof(int) * (size_t)sb.T);
        sb.count = (int*)dalloc(c, sizeof(int) * (size_t)sb.T);
        sb.items = (int*)dalloc(c, sizeof(int) * SMALL_MAX_PAIRS);
        sb.prev_tiles = (int*)dalloc(c, sizeof(int) * SMALL_MAX_PAIRS);
        sb.prev_n = (int*)dalloc(c, sizeof(int));
        sb.overflow = (int*)dalloc(c, sizeof(int));
        sb.done = (int*)dalloc(c, sizeof(int));
        sb.parts = window_parts(hwmax, 0);   // set per step (the lift's halo)
        sb.part = (float*)dalloc(c, sizeof(float) * WIN_VALS_LIFT * WINDOW_CHUNKS_MAX * (size_t)n);
        sb.arrive = (int*)dalloc(c, sizeof(int) * (size_t)n);
        lists_ok = sb.start && sb.count && sb.items && sb.prev_tiles && sb.prev_n && sb.overflow &&
                   sb.done && sb.part && sb.arrive;
        // Overlap guard: tags and sweep orders, one set per step parity.
        if (c->bins.T > 0 && geo_of(c).ntz <= GUARD_LAYERS_MAX) {
            int rc = alloc_guard(c, &sb.safe, &sb.zperm, &sb.nbz, &sb.zrange);
            if (rc == LBM_ERR_CUDA) {
                free_bubbles(c);
                return rc;
            }
            lists_ok = lists_ok && rc == LBM_OK;
        }
    } else {
        c->bins.cap = (int)cap;
        c->bins.items = (int*)dalloc(c, sizeof(int) * (size_t)cap);
        SwarmBins& sw = c->swarm;
        sw.grid = swarm_grid(c->storage);
        if (sw.grid < 1) {
            free_bubbles(c);
            return fail(c, LBM_ERR_CUDA, "occupancy of the bubble binning");
        }
        sw.per = (int)per;
        sw.interp_grid = interp_grid(c->storage);
        if (sw.interp_grid < 1) {
            free_bubbles(c);
            return fail(c, LBM_ERR_CUDA, "occupancy of the interpolation");
        }
        sw.bar = (unsigned*)dalloc(c, 2 * sizeof(unsigned));
        sw.cursor = (int*)dalloc(c, sizeof(int) * (size_t)c->bins.T);
        sw.kidx = (int*)dalloc(c, sizeof(int) * (size_t)cap);
        sw.slots = (int*)dalloc(c, sizeof(int) * (size_t)cap);   // n * per
        sw.ntile = (int*)dalloc(c, sizeof(int) * (size_t)n);
        sw.partial = (float*)dalloc(c, WIN_VALS_LIFT * sizeof(float) * (size_t)cap);
        sw.cover = (int*)dalloc(c, sizeof(int) * (size_t)c->bins.T);
        sw.ncover = (int*)dalloc(c, sizeof(int));
        sw.chunk_sums = (int*)dalloc(c, sizeof(int) * (size_t)sw.grid);
        sw.zrange = (int*)dalloc(c, 2 * sizeof(int));
        lists_ok = c->bins.items && sw.bar && sw.cursor && sw.kidx && sw.slots && sw.ntile &&
                   sw.partial && sw.cover && sw.ncover && sw.chunk_sums && sw.zrange;
        if (lists_ok)
            LBM_CUDA(cudaMemsetAsync(sw.bar, 0, 2 * sizeof(unsigned), c->stream), "barrier");
    }
    if (!B.k || !B.xh || !B.xl || !B.u || !B.d || !B.n || !B.ulprev || !B.ul || !B.psi ||
        !B.out64 || !B.has_prev || !B.active || !B.spread || !B.cell || !B.rec || !lists_ok) {
        free_bubbles(c);
        return fail(c, LBM_ERR_ALLOC, "bubble state");
    }
    if (c->use_small) {
        SmallBins& sb = c->small;
        LBM_CUDA(cudaMemsetAsync(sb.count, 0, sizeof(int) * (size_t)sb.T, c->stream), "count");
        LBM_CUDA(cudaMemsetAsync(sb.prev_n, 0, sizeof(int), c->stream), "prev_n");
        LBM_CUDA(cudaMemsetAsync(sb.overflow, 0, sizeof(int), c->stream), "overflow");
        LBM_CUDA(cudaMemsetAsync(sb.done, 0, sizeof(int), c->stream), "done");
        LBM_CUDA(cudaMemsetAsync(sb.arrive, 0, sizeof(int) * (size_t)n, c->stream), "arrive");
    }
    B.nb = n;
    std::vector<double> hn(n);
    for (int b = 0; b < n; ++b) hn[b] = c->p.width_factor * diam[b];
    std::vector<int> ones(n, 1), izero(n, 0), minus(n, -1);
    cudaStream_t s = c->stream;
    LBM_CUDA(upload_bubble_state(B, n, pos3, vel3, s), "upload bubbles");
    LBM_CUDA(cudaMemcpyAsync(B.d, diam, v1, cudaMemcpyHostToDevice, s), "upload diam");
    LBM_CUDA(cudaMemcpyAsync(B.n, hn.data(), v1, cudaMemcpyHostToDevice, s), "upload n");
    LBM_CUDA(cudaMemcpyAsync(B.has_prev, izero.data(), i1, cudaMemcpyHostToDevice, s), "has_prev");
    LBM_CUDA(cudaMemcpyAsync(B.active, ones.data(), i1, cudaMemcpyHostToDevice, s), "active");
    LBM_CUDA(cudaMemcpyAsync(B.spread, izero.data(), i1, cudaMemcpyHostToDevice, s), "spread");
    LBM_CUDA(cudaMemcpyAsync(B.cell, minus.data(), i1, cudaMemcpyHostToDevice, s), "cell");
    LBM_CUDA(cudaMemsetAsync(B.rec, 0, sizeof(BubbleRec) * (size_t)n, s), "rec");
    LBM_CUDA(launch_bubble_constants(B, bubble_const(c), s), "bubble constants");
    LBM_CUDA(cudaStreamSynchronize(s), "bubble upload");
    c->nb_cap = n;
    c->hwmax = hwmax;
    return LBM_OK;
}

int lbm_step(lbm_ctx* c, int nsteps) {
    if (!c || nsteps < 0) return LBM_ERR_ARG;
    adjoint_free(c);
    int rc = ensure_device(c);
    if (rc) return rc;
    if (c->unstable) return fail(c, LBM_ERR_UNSTABLE, "liquid solver is unstable (sticky)");
    for (int s = 0; s < nsteps; ++s) {
        rc = enqueue_one_step(c);
        if (rc) return rc;
    }
    return finish_steps(c);
}

int lbm_get_fields(lbm_ctx* c, double* rho, double* u3) {
    if (!c) return LBM_ERR_ARG;
    int rc = ensure_device(c);
    if (rc) return rc;
    if (!rho && !u3) return LBM_OK;
    const Geo g = geo_of(c);
    double* rd = rho ? (double*)dalloc(c, sizeof(double) * (size_t)g.S) : nullptr;
    double* ud = u3 ? (double*)dalloc(c, sizeof(double) * 3 * (size_t)g.S) : nullptr;
    if ((rho && !rd) || (u3 && !ud)) {
        dfree(c, rd);
        dfree(c, ud);
        return fail(c, LBM_ERR_ALLOC, "field staging");
    }
    cudaError_t e = launch_fields(c->storage, c->f[c->cur], g, collide_params(c), rd, ud, c->stream);
    if (e == cudaSuccess && rho)
        e = cudaMemcpyAsync(rho, rd, sizeof(double) * (size_t)g.S, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && u3)
        e = cudaMemcpyAsync(u3, ud, sizeof(double) * 3 * (size_t)g.S, cudaMemcpyDeviceToHost,
                            c->stream);
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    dfree(c, rd);
    dfree(c, ud);
    if (e != cudaSuccess) return cuda_fail(c, e, "get fields");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "get fields (sync)");
    return LBM_OK;
}

int lbm_get_bubbles(lbm_ctx* c, int cap, int* n, double* pos3, double* vel3, double* ul3,
                    double* psi3, int* active) {
    if (!c || cap < 0) return LBM_ERR_ARG;
    const int nb = c->bub.nb;
    if (n) *n = nb;
    const int k = nb < cap ? nb : cap;
    if (k == 0) return LBM_OK;
    cudaStream_t s = c->stream;
    LBM_CUDA(download_bubble_state(c->bub, k, pos3, vel3, ul3, psi3, s), "get bubbles");
    if (active)
        LBM_CUDA(cudaMemcpyAsync(active, c->bub.active, sizeof(int) * (size_t)k,
                                 cudaMemcpyDeviceToHost, s), "active");
    LBM_CUDA(cudaStreamSynchronize(s), "get bubbles");
    return LBM_OK;
}

int lbm_get_totals(lbm_ctx* c, double* out4) {
    if (!c || !out4) return LBM_ERR_ARG;
    int rc = ensure_device(c);
    if (rc) return rc;
    const Geo g = geo_of(c);
    const int np = totals_partials(g);
    double* part = (double*)dalloc(c, sizeof(double) * 4 * (size_t)np + sizeof(double) * 4);
    if (!part) return fail(c, LBM_ERR_ALLOC, "totals scratch");
    double* out_d = part + 4 * (size_t)np;
    cudaError_t e = launch_totals(c->storage, c->f[c->cur], g, collide_params(c), part, np, out_d,
                                  c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out4, out_d, sizeof(double) * 4, cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e2 = cudaStreamSynchronize(c->stream);
    dfree(c, part);
    if (e != cudaSuccess) return cuda_fail(c, e, "totals");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "totals (sync)");
    return LBM_OK;
}

int lbm_get_bins(lbm_ctx* c, int* cell, int* tile3, int* ntiles, int* offsets, int* items,
                 int cap_items, int* nitems) {
    if (!c || cap_items < 0) return LBM_ERR_ARG;
    if (tile3) {
        tile3[0] = TX;
        tile3[1] = TY;
        tile3[2] = TZ;
    }
    const Geo g = geo_of(c);
    const int T = g.ntx * g.nty * g.ntz;
    if (ntiles) *ntiles = T;
    if (!c->bins_valid) {
        if (nitems) *nitems = 0;
        if (offsets) std::memset(offsets, 0, sizeof(int) * ((size_t)T + 1));
        if (cell)
            for (int b = 0; b < c->bub.nb; ++b) cell[b] = -1;
        return LBM_OK;
    }
    cudaStream_t s = c->stream;
    LBM_CUDA(cudaStreamSynchronize(s), "bins sync");
    int total = 0;
    const int* items_d = c->use_small ? c->small.items : c->bins.items;
    if (c->use_small) {
        // Offsets are the running sum of the per-tile counts (pairs are
        // sorted by tile, so the runs are in tile order).
        std::vector<int> cnt((size_t)T);
        LBM_CUDA(cudaMemcpy(cnt.data(), c->small.count, sizeof(int) * (size_t)T,
                            cudaMemcpyDeviceToHost), "bins counts");
        if (offsets) offsets[0] = 0;
        for (int t = 0; t < T; ++t) {
            total += cnt[t];
            if (offsets) offsets[t + 1] = total;
        }
    } else {
        LBM_CUDA(cudaMemcpy(&total, c->bins.off + T, sizeof(int), cudaMemcpyDeviceToHost),
                 "bins total");
        if (offsets)
            LBM_CUDA(cudaMemcpy(offsets, c->bins.off, sizeof(int) * ((size_t)T + 1),
                                cudaMemcpyDeviceToHost), "bins offsets");
    }
    if (nitems) *nitems = total;
    if (items) {
        const int k = total < cap_items ? total : cap_items;
        if (k > 0)
            LBM_CUDA(cudaMemcpy(items, items_d, sizeof(int) * (size_t)k, cudaMemcpyDeviceToHost),
                     "bins items");
    }
    if (cell && c->bub.nb > 0)
        LBM_CUDA(cudaMemcpy(cell, c->bub.cell, sizeof(int) * (size_t)c->bub.nb,
                            cudaMemcpyDeviceToHost), "bins cells");
    return LBM_OK;
}

long long lbm_sites(const lbm_ctx* c) { return c ? (long long)c->nx * c->ny * c->nz : 0; }

int lbm_bytes_per_site(const lbm_ctx* c) { return c ? (int)(2 * Q * elem_size(c->storage)) : 0; }

int lbm_set_kernel_timing(lbm_ctx* c, int on) {
    if (!c) return LBM_ERR_ARG;
    if (c->dev_ready) LBM_CUDA(cudaStreamSynchronize(c->stream), "timing sync");
    c->timing = on != 0;
    c->events_used = 0;
    return LBM_OK;
}

int lbm_get_kernel_time(lbm_ctx* c, double* ms, int* launches) {
    if (!c) return LBM_ERR_ARG;
    if (c->dev_ready) LBM_CUDA(cudaStreamSynchronize(c->stream), "timing sync");
    double total = 0.0;
    for (size_t i = 0; i < c->events_used; ++i) {
        float t = 0.0f;
        LBM_CUDA(cudaEventElapsedTime(&t, c->events[i].first, c->events[i].second), "elapsed");
        total += t;
    }
    if (ms) *ms = total;
    if (launches) *launches = (int)c->events_used;
    c->events_used = 0;
    return LBM_OK;
}

long long lbm_launch_count(const lbm_ctx* c) { return c ? c->launches : 0; }

const char* lbm_sweep_kernel(const lbm_ctx* c) {
    if (!c) return "";
    // The choice launch_collide_stream makes for this context's next step.
    static const char* const pair[3][2] = {
        {"k_collide_stream_pair<0,0>", "k_collide_stream_pair<0,1>"},
        {"k_collide_stream_pair<1,0>", "k_collide_stream_pair<1,1>"},
        {"k_collide_stream_pair<2,0>", "k_collide_stream_pair<2,1>"}};
    static const char* const single[3] = {"k_collide_stream<0>", "k_collide_stream<1>",
                                          "k_collide_stream<2>"};
    static const char* const free_[3] = {"k_collide_stream_free<0>", "k_collide_stream_free<1>",
                                         "k_collide_stream_free<2>"};
    const int st = c->storage < 0 || c->storage > 2 ? 0 : c->storage;
    if (c->nx & 1) return single[st];
    if (!(c->bub.nb > 0 && c->p.two_way)) return free_[st];   // no tile lists
    return pair[st][c->use_small ? 0 : 1];
}

int lbm_sync(lbm_ctx* c) {
    if (!c) return LBM_ERR_ARG;
    if (!c->dev_ready) return LBM_OK;
    LBM_CUDA(cudaStreamSynchronize(c->stream), "sync");
    return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : "null context"; }

const char* lbm_status_string(int s) {
    switch (s) {
        case LBM_OK: return "LBM_OK";
        case LBM_ERR_ARG: return "LBM_ERR_ARG";
        case LBM_ERR_ALLOC: return "LBM_ERR_ALLOC";
        case LBM_ERR_UNSTABLE: return "LBM_ERR_UNSTABLE";
        case LBM_ERR_TIMEOUT: return "LBM_ERR_TIMEOUT";
        case LBM_ERR_CUDA: return "LBM_ERR_CUDA";
        case LBM_ERR_STATE: return "LBM_ERR_STATE";
        default: return "LBM_UNKNOWN";
    }
}

}  // extern "C"
