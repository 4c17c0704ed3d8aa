// Bubble binning that allocates nothing.
//
// The coupled step bins bubbles with per-tile counters and scan block sums
// that live in buffers the context allocates.  Some callers cannot allocate
// device memory at the point where they want the binning: code that runs while
// a stream is being captured into a CUDA graph in global capture mode (where
// cudaMalloc is an error), runtimes that hand all device memory to their own
// pool when they start, and tight loops that cannot afford the device-wide
// synchronisation a cudaMalloc implies.  lbm_bin_bubbles_noalloc runs the same
// binning kernels with that scratch taken from a fixed array compiled into the
// library, so the caller only passes its own inputs and outputs.
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_internal.cuh"

using namespace lbm;

namespace {

static_assert(LBM_NOALLOC_MAX_HALF_WIDTH == MAX_HALF_WIDTH,
              "the header's half-width limit is the one the binning kernels check");

constexpr int NOALLOC_SCAN_CHUNK = 1024;   // counts per scan block (matches scan_blocks)
constexpr int NOALLOC_MAX_BLOCKS =
    (LBM_NOALLOC_MAX_TILES + NOALLOC_SCAN_CHUNK - 1) / NOALLOC_SCAN_CHUNK;

// Scratch of every call: LBM_NOALLOC_MAX_TILES tile counters followed by the
// scan's block sums (1 MiB + 1 KiB).  Each GPU that loads the library holds
// one copy until the process exits.
static __device__ __align__(256) int g_bin_scratch[LBM_NOALLOC_MAX_TILES + NOALLOC_MAX_BLOCKS];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
int* g_scratch_ptr[MAX_DEVICES] = {};

// Device address of g_bin_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device with that device current.
cudaError_t scratch_address(int** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        int* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_bin_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int lbm_bin_bubbles_noalloc(int nx, int ny, int nz, unsigned walls, int n,
                                       const double* pos3, const double* half_width,
                                       const int* active, int* tile_offsets, int* tile_items,
                                       int cap_items, int* status, void* stream) {
    if (nx <= 0 || ny <= 0 || nz <= 0 || n < 0 || cap_items < 0) return LBM_ERR_ARG;
    if ((long long)nx * ny * nz * 19 >= (1LL << 32)) return LBM_ERR_ARG;
    if (walls & ~0x7Fu) return LBM_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(walls & (1u << (2 * a))) != !(walls & (1u << (2 * a + 1)))) return LBM_ERR_ARG;
    if ((walls & WALL_TOP_FREE) && !(walls & 0x20u)) return LBM_ERR_ARG;
    Geo g;
    g.nx = nx;
    g.ny = ny;
    g.nz = nz;
    g.walls = walls;
    g.S = (long long)nx * ny * nz;
    g.ntx = (nx + TX - 1) / TX;
    g.nty = (ny + TY - 1) / TY;
    g.ntz = (nz + TZ - 1) / TZ;
    const long long T = (long long)g.ntx * g.nty * g.ntz;
    if (T > LBM_NOALLOC_MAX_TILES) return LBM_ERR_ARG;   // scratch holds this many tiles
    if (!tile_offsets || !status || (n > 0 && (!pos3 || !half_width || !active)) ||
        (cap_items > 0 && !tile_items))
        return LBM_ERR_ARG;
    int* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return LBM_ERR_CUDA;

    BubbleDev b{};
    b.nb = n;
    b.x = const_cast<double*>(pos3);
    b.n = const_cast<double*>(half_width);
    b.spread = const_cast<int*>(active);
    Bins bins{};
    bins.T = (int)T;
    bins.cnt = scratch;                              // cleared by launch_binning
    bins.block_sums = scratch + LBM_NOALLOC_MAX_TILES;
    bins.nblocks = scan_blocks(bins.T);
    bins.off = tile_offsets;
    bins.items = tile_items;
    bins.cap = cap_items;
    bins.overflow = status;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return LBM_ERR_CUDA;
    if (launch_binning(g, b, bins, st) != cudaSuccess) return LBM_ERR_CUDA;
    return LBM_OK;
}
