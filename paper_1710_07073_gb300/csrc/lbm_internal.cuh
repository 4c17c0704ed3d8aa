// Internal declarations shared by the CUDA translation units of liblbm.so.
//
// D3Q19 direction order used by this library (Eq. 7-8 of arXiv:1710.07073,
// renumbered with the rest velocity first):
//   0: (0,0,0)
//   1,2: (+-1,0,0)   3,4: (0,+-1,0)   5,6: (0,0,+-1)
//   7: (+1,+1,0) 8: (-1,-1,0) 9: (+1,-1,0) 10: (-1,+1,0)
//   11: (+1,0,+1) 12: (-1,0,-1) 13: (+1,0,-1) 14: (-1,0,+1)
//   15: (0,+1,+1) 16: (0,-1,-1) 17: (0,+1,-1) 18: (0,-1,+1)
// Opposite directions come in consecutive pairs (2k-1, 2k).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int Q = 19;
// Binning tile; the collide-stream CTA covers TX x TY sites of one z-plane, so
// all threads of a CTA share one tile.
constexpr int TX = 32, TY = 4, TZ = 4;
constexpr int MAX_AXIS_TILES = 8;   // per-axis tiles a window may touch (n <= 9)
// z planes per CTA of the two-node collide-stream sweep (divides TZ); a
// compile-time knob of the sweep's launch shape.
#ifndef LBM_PAIR_PZ
#define LBM_PAIR_PZ 2
#endif
constexpr int SWEEP_PZ = LBM_PAIR_PZ;
// Resident CTAs per SM of the many-bubble binning launch.
#ifndef LBM_SWARM_CTAS_PER_SM
#define LBM_SWARM_CTAS_PER_SM 4
#endif
constexpr double MAX_HALF_WIDTH = 9.0;

__host__ __device__ __forceinline__ constexpr int cx(int j) {
    return (j == 1 || j == 7 || j == 9 || j == 11 || j == 13) ? 1
         : (j == 2 || j == 8 || j == 10 || j == 12 || j == 14) ? -1 : 0;
}
__host__ __device__ __forceinline__ constexpr int cy(int j) {
    return (j == 3 || j == 7 || j == 10 || j == 15 || j == 17) ? 1
         : (j == 4 || j == 8 || j == 9 || j == 16 || j == 18) ? -1 : 0;
}
__host__ __device__ __forceinline__ constexpr int cz(int j) {
    return (j == 5 || j == 11 || j == 14 || j == 15 || j == 18) ? 1
         : (j == 6 || j == 12 || j == 13 || j == 16 || j == 17) ? -1 : 0;
}
__host__ __device__ __forceinline__ constexpr int opp(int j) {
    return j == 0 ? 0 : ((j & 1) ? j + 1 : j - 1);
}
// The direction with the same tangential components and c_z reversed
// (specular reflection at a z face).
__host__ __device__ __forceinline__ constexpr int mirz(int j) {
    return j == 5 ? 6 : j == 6 ? 5 : j == 11 ? 13 : j == 13 ? 11 : j == 12 ? 14 : j == 14 ? 12
         : j == 15 ? 17 : j == 17 ? 15 : j == 16 ? 18 : j == 18 ? 16 : j;
}
// walls bit: the +z face (bounded, bit 0x20 set too) is a free-slip plane
// (specular reflection) instead of a no-slip wall (LBM_TOP_FREE_SLIP).
constexpr unsigned WALL_TOP_FREE = 0x40;
// Eq. 8 weights and their reciprocals.
__host__ __device__ __forceinline__ constexpr float wf(int j) {
    return j == 0 ? (1.0f / 3.0f) : (j <= 6 ? (1.0f / 18.0f) : (1.0f / 36.0f));
}
__host__ __device__ __forceinline__ constexpr double wd(int j) {
    return j == 0 ? (1.0 / 3.0) : (j <= 6 ? (1.0 / 18.0) : (1.0 / 36.0));
}
__host__ __device__ __forceinline__ constexpr float inv_wf(int j) {
    return j == 0 ? 3.0f : (j <= 6 ? 18.0f : 36.0f);
}

struct Geo {
    int nx, ny, nz;
    unsigned walls;        // LBM_WALL_* bits
    long long S;           // sites
    int ntx, nty, ntz;     // tiles per axis
};

struct CollideParams {
    float omega;           // 1/tau
    float pref;            // 1 - omega/2 (Eq. 12)
    float rho0;            // storage shift reference density
    float scale;           // 16-bit storage: stored = g * scale / w_j
    float inv_scale;
    int point;             // bubble weights by point samples (lbm_params.mapping)
};

// What the collide-stream sweep needs to spread one bubble (Eq. 21): the
// integer anchor cell and FP32 offset of the centre, the window in units of
// the half-width, and psi_b divided by the window normalisation.
struct __align__(16) BubbleRec {
    int ax, ay, az, pad;
    float fx, fy, fz, inv_n;
    float px, py, pz, h;   // h = 0.5 * inv_n
};

// Per-bubble constants of the closures (Table 1) and of the mapping window,
// derived from the diameter and the parameters whenever either changes.
// Lengths used against positions come as two floats (hi + lo, |lo| <=
// ulp(hi)/2), like the positions themselves.
struct BubbleK {
    double r;           // d / 2
    float rh, rl;       // r as two floats (wall tests)
    float nh, nl;       // n = width_factor * d as two floats (window bounds)
    float inv_nf;       // 1 / n
    float kdt;          // dt_b / m_eff, m_eff = (rho_b + C_A rho_l) V_b
    float fb;           // (rho_l - rho_b) V_b g
    float drag_pref;    // 1/2 rho_l pi r^2 * drag_scale
    float fvm_coef_dt;  // C_A rho_l V_b / dt_l
    float visc_a0;      // 24 nu / d
    float visc_b;       // 48 nu / d
    float re_per_speed; // d / nu
    float eo_term;      // 8/3 Eo / (Eo + 4)
    // Lift (Table 1): C_L = cl_tanh ? min(0.288 tanh(0.121 Re), cl_f) : cl_f,
    // F_L = -C_L lift_pref (u_b - u_l) x (curl u_l); lift_pref = rho_l V_b,
    // 0 with lift off.
    float lift_pref;
    float cl_f;
    int cl_tanh;
    float fs_coef_dt;   // rho_l V_b / dt_l for F_S = rho_l V_b D_t u_l (0: off)
    // Mapping weights (Eq. 19): h = 1/(2n) takes the cell integral of Z,
    // h = -1/(2n) the point sample at the node (cell_poly).
    float hmap;
    // Reaction -sum F (Sec. 3.2): psi = react_ca F_B - react_mb (mean F_D +
    // F_L + F_S + C_A rho_l V_b D_t u_l), react_ca = C_A rho_l V_b / m_eff,
    // react_mb = m_b / m_eff.
    float react_ca, react_mb;
};

// Bubble state on the device.  A context keeps the centres as two floats
// (xh + xl: about 48 significant bits, enough for the 1e-5 moves of a
// sub-step at positions of hundreds) and velocities, u_l and psi in FP32, so
// that the per-bubble update runs on the FP32 pipe; the host converts from
// and to the FP64 arrays of the C ABI.  `x` (FP64 centres) is set only by
// callers that bin FP64 input directly and is null in a context.
struct BubbleDev {
    int nb;
    BubbleK* k;       // [nb]
    double* x;        // [3*nb] FP64 centres (binning of caller input only)
    float* xh;        // [3*nb] interleaved centre, high part
    float* xl;        // [3*nb] low part
    float* u;         // [3*nb] velocity
    double* d;        // [nb] diameter
    double* n;        // [nb] window half-width
    float* ulprev;    // [3*nb] interpolated liquid velocity of the previous step
    float* ul;        // [3*nb] interpolated liquid velocity of the last step
    float* psi;       // [3*nb] reaction of the last step
    int* has_prev;    // [nb]
    int* active;      // [nb]
    int* spread;      // [nb] 1 if the bubble spread in the last step
    int* cell;        // [nb] containing cell after the last update (-1 inactive)
    BubbleRec* rec;   // [nb]
    double* out64;    // [12*nb] FP64 staging for exports to the host
};

struct BubbleConst {
    double g, rho_l, rho_b, sigma, c_am, drag_scale, sn_coeff, sn_exp, nu, dt_b, dt_l;
    float dt_bh, dt_bl;   // dt_b as two floats
    int substeps;
    int lift;             // F_L of Table 1 on (the windows then carry the vorticity halo)
    int stress;           // F_S of Table 1 on
    int point;            // mapping by point samples of Z instead of cell integrals
    int reaction_all;     // psi_b = -sum of the interphase forces (Sec. 3.2)
};

// Values a window sum carries per bubble: the Eq. 20 velocity (3) and, with
// lift, six sums that give the interpolated vorticity (by summation by parts:
// the central differences of Eq. 10 velocities, interpolated with Eq. 19
// weights, are sums of the velocities times per-axis difference weights).
constexpr int WIN_VALS_LIFT = 9;
__host__ __device__ constexpr int win_vals(bool lift) { return lift ? WIN_VALS_LIFT : 3; }

// A double as two floats (h = v rounded, l = the rest rounded) and back.
__host__ __device__ inline void split_f2(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}
__host__ __device__ inline double join_f2(float h, float l) { return (double)h + (double)l; }

struct Bins {
    int T;             // tiles
    int* cnt;          // [T] counts, then fill cursors
    int* off;          // [T+1]
    int* items;        // [cap]
    int cap;
    int* block_sums;   // scan scratch [nblocks]
    int nblocks;
    int* overflow;     // set to 1 if items would exceed cap
};

// Per-tile bubble lists as the collide-stream sweep reads them: tile t holds
// items[start[t] .. start[t] + count[t]) (start is only read when count > 0).
struct TileLists {
    const int* start;
    const int* count;
    const int* items;
    int cap;
};

// Single-launch binning for few (tile, bubble) pairs: pairs are sorted by
// (tile, bubble) in shared memory; only the tiles touched by the previous step
// are cleared, so no work scales with the tile count.
constexpr int SMALL_MAX_PAIRS = 4096;
// A bubble window is reduced in chunks of WINDOW_CHUNK nodes (two per thread
// of a 256-thread bubble CTA): at most (2 MAX_HALF_WIDTH + 2)^3 / WINDOW_CHUNK
// rounded up.
constexpr int WINDOW_CELLS_MAX = 2 * (int)MAX_HALF_WIDTH + 4;   // + a halo cell each side (lift)
constexpr int WINDOW_CHUNK = 512;
constexpr int WINDOW_CHUNKS_MAX =
    (WINDOW_CELLS_MAX * WINDOW_CELLS_MAX * WINDOW_CELLS_MAX + WINDOW_CHUNK - 1) / WINDOW_CHUNK;
struct SmallBins {
    int T;
    int* start;        // [T]
    int* count;        // [T], zero except on tiles listed in prev_tiles
    int* items;        // [SMALL_MAX_PAIRS]
    int* prev_tiles;   // [SMALL_MAX_PAIRS] tile of each pair of the last binning
    int* prev_n;       // [1] number of pairs of the last binning
    int* overflow;     // [1]
    int* done;         // [1] bubbles the update has finished (0 between launches)
    int parts;         // CTAs per bubble in the update, 1..WINDOW_CHUNKS_MAX
    float* part;       // [nb * WINDOW_CHUNKS_MAX * WIN_VALS_LIFT] chunk sums (parts > 1)
    int* arrive;       // [nb] CTAs of a bubble that have finished (0 between launches)
    // Overlap guard (single column): safe[l] = e states that no bubble force
    // reaches z tile layer l in the step numbered e.  The update writes
    // safe_epoch (the next step's number) into the layers that no active
    // bubble's support, widened by GUARD_CELLS, touches; the context keeps
    // one set of ntz tags per step parity, so an update never rewrites the
    // set its own sweep reads.  Null: not kept.
    unsigned* safe;    // [ntz] (the set this launch writes)
    unsigned safe_epoch;
    // Order of the next sweep's z blocks (PZ planes each): the blocks of
    // cleared layers first, then the guarded ones, each in ascending order,
    // so that the sweep reaches the layers that wait for the update last.
    // Null: not kept.
    int* zperm;        // [nbz] (the set this launch writes)
    int nbz;
    // The first and last z tile layer the update marks as guarded (last <
    // first: none), for the host's split of later sweeps.  Null: not kept.
    int* zrange;       // [2]
};

// Many bubbles: the bubble side of a step in three launches
// (launch_swarm_update), with the binning done by one persistent launch whose
// phases are separated by grid barriers over CTAs that are all resident.
// Besides the tile lists of `Bins`, the binning records where each bubble sits
// in each of its tiles' lists (slots), so that the next step's interpolation
// can be summed per tile and gathered per bubble in a fixed order.
struct SwarmBins {
    unsigned* bar;        // [2] grid barrier: arrivals, generation (zero between launches)
    int* cursor;          // [T] fill cursors of the counting sort
    int* kidx;            // [cap] for each list entry: which of its bubble's tiles it is
    int* slots;           // [nb * per] list position of bubble b's k-th tile
    int* ntile;           // [nb] tiles of bubble b in the last binning (0: not binned)
    int per;              // tiles a bubble's window can touch at most
    float* partial;       // [WIN_VALS_LIFT * cap] Eq. 20 sums of each (tile, bubble) entry
    int pad;              // cells the lists reach beyond the supports (1 with lift)
    int* cover;           // [T] the tiles with a non-empty list (any order)
    int* ncover;          // [1] their number
    int* zrange;          // [2] lowest and highest z tile layer of any list (empty: lo > hi)
    int interp_grid;      // CTAs of the interpolation launch
    int* chunk_sums;      // [grid] per-CTA count totals (scan)
    int grid;             // CTAs of the binning launch (all resident)
};

// A bubble moves at most this many cells along an axis per liquid step (a
// lattice speed of 4 is far past any stable state); a faster one raises the
// instability flag (bit 4).  The overlap guard relies on it.
constexpr int GUARD_CELLS = 4;
// Tile layers the guard covers (nz <= 4 GUARD_LAYERS_MAX); taller columns keep
// no guard.
constexpr int GUARD_LAYERS_MAX = 2048;

// One column of a batch: its geometry and relaxation, where its populations
// start in the batch buffers (elements), and the first global tile and work
// item that belong to it.
struct BatchColumn {
    Geo g;
    CollideParams cp;
    unsigned long long pop_offset;
    int tile_base;
    int item_base;
};

// ---- launchers (defined in the kernel translation units) -------------------
// The sweep.  With `safe` set it is launched as a programmatic dependent of
// the bubble update before it (`overlap`): CTAs whose z tile layer holds
// safe[layer] == epoch run without waiting for the update; the others (and
// CTA 0) wait for it before reading the tile lists.
// zperm (may be null): the order of the z blocks (PZ planes each) in which
// the CTAs are handed out, a permutation of 0 .. ceil(nz / PZ) - 1.
// A subset of the sweep's z blocks (PZ planes each): CTA z-index i sweeps
// block first + i, moved past the hole [hole, hole + skip) when it reaches it;
// `count` blocks in all.
struct ZSpan {
    int first, count, hole, skip;
};

cudaError_t launch_collide_stream(int storage, const void* fin, void* fout, const Geo& g,
                                  const CollideParams& cp, const TileLists* tl,
                                  const BubbleRec* recs, int nb, int* flag, const unsigned* safe,
                                  unsigned epoch, bool overlap, const int* zperm,
                                  cudaStream_t st, const ZSpan* span = nullptr);

// Bubble update with the few-pair binning in the same launch (sb.parts CTAs
// per bubble).  `overlap`: launched as a programmatic dependent of the sweep
// before it; it waits for that sweep, then lets the next sweep start.
cudaError_t launch_bubbles(int storage, const void* f, const Geo& g, const CollideParams& cp,
                           const BubbleDev& b, const BubbleConst& bc, int* flag,
                           const SmallBins& sb, bool overlap, cudaStream_t st);
// CTAs per bubble for windows of half-width up to max_half_width, widened by
// `pad` cells each side: one per WINDOW_CHUNK nodes of the largest window.
int window_parts(double max_half_width, int pad);
cudaError_t launch_bubble_constants(const BubbleDev& b, const BubbleConst& bc, cudaStream_t st);
// Host: FP64 centres and velocities of n bubbles into the device state
// (vel3 may be null: at rest); u_l, its previous value and psi are zeroed.
// Synchronises the stream.
cudaError_t upload_bubble_state(const BubbleDev& B, int n, const double* pos3, const double* vel3,
                                cudaStream_t st);
// Host: the first k bubbles' state as FP64 arrays (null pointers are
// skipped), converted on the device into B.out64.  Synchronises the stream.
cudaError_t download_bubble_state(const BubbleDev& B, int k, double* pos3, double* vel3,
                                  double* ul3, double* psi3, cudaStream_t st);
// Many bubbles, three launches per step, in stream order:
//   1. per tile the current binning lists (persistent over the list of
//      covered tiles): the Eq. 10 velocity of its nodes, and for each listed
//      bubble the part of its Eq. 20 sum over the tile (weights from the
//      bubble's spreading record, which holds the current centre);
//   2. per bubble (a thread each): its parts added in tile order, the Table 1
//      forces and Eq. 4 sub-steps, the reaction and the new record;
//   3. the binning of the updated bubbles (one persistent launch, sw.grid
//      CTAs): tile lists, list positions and the list of covered tiles.
// A grid barrier that waits longer than a second sets flag bit 8.
constexpr int SWARM_LAUNCHES = 3;
cudaError_t launch_swarm_update(int storage, const void* f, const Geo& g,
                                const CollideParams& cp, const BubbleDev& b,
                                const BubbleConst& bc, int* flag, const Bins& bins,
                                const SwarmBins& sw, cudaStream_t st);
// Many bubbles: the binning alone, of the bubbles with select[b] != 0 (the
// first step's lists of the current centres); bins.cnt and *sw.ncover must
// be zero.
cudaError_t launch_swarm_binning(const Geo& g, const BubbleDev& b, const Bins& bins,
                                 const SwarmBins& sw, const int* select, int* flag,
                                 cudaStream_t st);
// Spreading records (anchor cell, offset, window) of the current centres,
// with the current reaction.
cudaError_t launch_bubble_records(const Geo& g, const BubbleDev& b, cudaStream_t st);
// CTAs of the many-bubble binning launch that are resident at once on this
// device, and of the interpolation launch (persistent over the covered tiles).
int swarm_grid(int storage);
int interp_grid(int storage);
// Sweep z blocks (planes per CTA of the pair sweep) for nz planes.
int sweep_z_blocks(int nz);
// Kernels launched by one launch_binning call (count, 3-pass scan, fill, sort).
// Bubbles b with select[b] != 0 are binned; select defaults to b.spread.
constexpr int BINNING_LAUNCHES = 6;
cudaError_t launch_binning(const Geo& g, const BubbleDev& b, const Bins& bins, cudaStream_t st,
                           const int* select = nullptr);
cudaError_t launch_fields(int storage, const void* f, const Geo& g, const CollideParams& cp,
                          double* rho, double* u, cudaStream_t st);
cudaError_t launch_get_populations(int storage, const void* f, const Geo& g,
                                   const CollideParams& cp, double* out, cudaStream_t st);
cudaError_t launch_set_populations(int storage, const double* fin, void* f, const Geo& g,
                                   const CollideParams& cp, cudaStream_t st);
cudaError_t launch_set_equilibrium(int storage, const double* rho, const double* u, void* f,
                                   const Geo& g, const CollideParams& cp, cudaStream_t st);
cudaError_t launch_totals(int storage, const void* f, const Geo& g, const CollideParams& cp,
                          double* partials, int npartials, double* out4, cudaStream_t st);
cudaError_t launch_collide_batch(int storage, const void* fin, void* fout,
                                 const BatchColumn* cols, int ncols, int total_items, int depth,
                                 int grid, int planes, int* work_counter, const TileLists& tl,
                                 const BubbleRec* recs, int nb, int* flag, cudaStream_t st);
cudaError_t launch_bubbles_batch(int storage, const void* f, const BatchColumn* cols,
                                 const int* bubble_col, const BubbleDev& b, const BubbleConst& bc,
                                 int* flag, const SmallBins& sb, cudaStream_t st);
cudaError_t launch_bubble_constants_batch(const BubbleDev& b, const BubbleConst& bc,
                                          const double* col_nu, const int* bubble_col,
                                          cudaStream_t st);
// Resident CTAs per SM the batch sweep is compiled for, with `planes` z-planes
// per CTA (1, 2 or 4; the same threads per SM for each).
int batch_min_blocks(int storage, int planes);
int totals_partials(const Geo& g);
int scan_blocks(int T);

}  // namespace lbm
