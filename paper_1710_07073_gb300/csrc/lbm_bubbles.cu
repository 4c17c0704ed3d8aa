// Bubble side of the coupled step and the field utilities.
//
//  k_bubbles      one warp per bubble: forward coupling (Eq. 19-20) of the bare
//                 Eq. 10 liquid velocity, Table 1 forces, sub-stepped Newton
//                 update (Eq. 4, Table 2), reaction psi_b = -mean F_D
//                 (Algorithm 1 step 6) and the spreading record for the sweep.
//  binning        bubble windows to lattice tiles (Algorithm 1 step 2):
//                 integer counting sort, then each tile's list in bubble order.
//  field kernels  initialisation to f^eq (Eq. 6), population I/O, Eq. 10
//                 moments and FP64 totals.
#include "lbm_device.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// Bubble update
// ---------------------------------------------------------------------------

// Window normalisation along one axis: the integral of the mapping over the
// in-box part of [-n, n] (without 15/16); the full 16/15 on a periodic axis.
__device__ __forceinline__ float axis_norm(double xa, float inv_n, int L, bool periodic) {
    if (periodic) return 16.0f / 15.0f;
    const float lo = (float)(-xa) * inv_n, hi = (float)((double)L - xa) * inv_n;
    const float a = fmaxf(lo, -1.0f), b = fminf(hi, 1.0f);
    if (!(b > a)) return 0.0f;
    const float a2 = a * a, b2 = b * b, ab = a * b;
    const float p4 = b2 * b2 + b2 * ab + ab * ab + ab * a2 + a2 * a2;
    return (b - a) * (p4 * 0.2f - (b2 + ab + a2) * (2.0f / 3.0f) + 1.0f);
}

__device__ __forceinline__ void make_record(const double* xb, float inv_n, const Geo& g,
                                            const float* psi, BubbleRec& r) {
    int anc[3];
    float fr[3];
    float norm = 1.0f;
    const int L[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a) {
        const double fl = floor(xb[a]);
        anc[a] = (int)fl;
        fr[a] = (float)(xb[a] - fl);
        norm *= axis_norm(xb[a], inv_n, L[a], !(g.walls & (1u << (2 * a))));
    }
    const float inv_norm = 1.0f / norm;
    r.ax = anc[0];
    r.ay = anc[1];
    r.az = anc[2];
    r.pad = 0;
    r.fx = fr[0];
    r.fy = fr[1];
    r.fz = fr[2];
    r.inv_n = inv_n;
    r.h = 0.5f * inv_n;
    r.px = psi[0] * inv_norm;
    r.py = psi[1] * inv_norm;
    r.pz = psi[2] * inv_norm;
}

// One CTA of BUBBLE_THREADS threads per bubble: the threads stride over the
// window's nodes for the forward coupling, thread 0 integrates the bubble.
//
// Precision: positions are integrated in FP64 (they reach hundreds of lattice
// units and move by 1e-5 per sub-step); velocities, forces and the mapping
// weights are FP32.  FP64 latency on this GPU is long, so only the position
// update, the window bounds and the wall tests use it.
constexpr int BUBBLE_THREADS = 256;

template <int ST>
__device__ void bubble_update(const typename Store<ST>::T* __restrict__ f, const Geo& g,
                              const CollideParams& cp, const BubbleDev& B, const BubbleConst& bc,
                              int* __restrict__ flag, int b, float (*red)[BUBBLE_THREADS / 32]) {
    const int tid = threadIdx.x;
    if (b >= B.nb) return;
    if (!B.active[b]) {
        if (tid == 0) {
            B.spread[b] = 0;
            B.cell[b] = -1;
        }
        return;
    }
    const int L[3] = {g.nx, g.ny, g.nz};
    double xb[3] = {B.x[3 * b], B.x[3 * b + 1], B.x[3 * b + 2]};
    const double n = B.n[b];
    const BubbleK K = B.k[b];
    if (!(isfinite(xb[0]) && isfinite(xb[1]) && isfinite(xb[2]))) {
        // A non-finite centre can only come from an unstable liquid: stop
        // coupling this bubble and report the instability.
        if (tid == 0) {
            B.active[b] = 0;
            B.spread[b] = 0;
            B.cell[b] = -1;
            atomicOr(flag, 2);
        }
        return;
    }

    // Window cells per axis (Algorithm 1 step 2): cells overlapping (x - n, x + n).
    const float inv_n = K.inv_nf, hh = 0.5f * K.inv_nf;
    int lo[3], cnt[3], anc[3];
    float fr[3];
    float norm = 1.0f;
    for (int a = 0; a < 3; ++a) {
        const bool periodic = !(g.walls & (1u << (2 * a)));
        int l = (int)floor(xb[a] - n);
        int h = (int)ceil(xb[a] + n) - 1;
        if (!periodic) {
            l = max(l, 0);
            h = min(h, L[a] - 1);
        }
        lo[a] = l;
        cnt[a] = min(max(h - l + 1, 0), 2 * (int)MAX_HALF_WIDTH + 2);
        const double fl = floor(xb[a]);
        anc[a] = (int)fl;
        fr[a] = (float)(xb[a] - fl);
        norm *= axis_norm(xb[a], inv_n, L[a], periodic);
    }

    // Forward coupling (Eq. 20): threads stride over the window's nodes and
    // weight the bare Eq. 10 velocity of the current populations.
    float ax = 0.0f, ay = 0.0f, az = 0.0f;
    const int M = cnt[0] * cnt[1] * cnt[2];
    for (int m = tid; m < M; m += BUBBLE_THREADS) {
        const int ix = m % cnt[0];
        const int rest = m / cnt[0];
        const int iy = rest % cnt[1];
        const int iz = rest / cnt[1];
        const int i = lo[0] + ix, j = lo[1] + iy, k = lo[2] + iz;
        const float w = cell_poly(((float)(i - anc[0]) + 0.5f - fr[0]) * inv_n, hh) *
                        cell_poly(((float)(j - anc[1]) + 0.5f - fr[1]) * inv_n, hh) *
                        cell_poly(((float)(k - anc[2]) + 0.5f - fr[2]) * inv_n, hh);
        const int iw = (i % g.nx + g.nx) % g.nx;
        const int jw = (j % g.ny + g.ny) % g.ny;
        const int kw = (k % g.nz + g.nz) % g.nz;
        float gv[Q];
        gather<ST>(f, g, cp, iw, jw, kw, gv);
        float drho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            drho += gv[q];
            if (cx(q) != 0) jx += (float)cx(q) * gv[q];
            if (cy(q) != 0) jy += (float)cy(q) * gv[q];
            if (cz(q) != 0) jz += (float)cz(q) * gv[q];
        }
        const float inv_rho = 1.0f / (cp.rho0 + drho);
        ax = fmaf(w, jx * inv_rho, ax);
        ay = fmaf(w, jy * inv_rho, ay);
        az = fmaf(w, jz * inv_rho, az);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
    }
    if ((tid & 31) == 0) {
        red[0][tid >> 5] = ax;
        red[1][tid >> 5] = ay;
        red[2][tid >> 5] = az;
    }
    __syncthreads();
    if (tid != 0) return;
    ax = ay = az = 0.0f;
    for (int w = 0; w < BUBBLE_THREADS / 32; ++w) {
        ax += red[0][w];
        ay += red[1][w];
        az += red[2][w];
    }

    const float inv_norm = 1.0f / norm;
    const float ul[3] = {ax * inv_norm, ay * inv_norm, az * inv_norm};
    float fvm[3] = {0.0f, 0.0f, 0.0f};   // C_A rho_l V_b D_t u_l
    if (B.has_prev[b]) {
        for (int a = 0; a < 3; ++a)
            fvm[a] = K.fvm_coef_dt * (ul[a] - (float)B.ulprev[3 * b + a]);
    }

    // Table 1 forces and the Newton update of Eq. 4 with the added mass on
    // the left (m_eff), sub-stepped with dt_b (Table 2).
    const double dt_b = bc.dt_b;
    const double r = K.r;
    const float sn_coeff = (float)bc.sn_coeff, sn_exp = (float)bc.sn_exp;
    const float fb[3] = {0.0f, 0.0f, K.fb};
    float u[3] = {(float)B.u[3 * b], (float)B.u[3 * b + 1], (float)B.u[3 * b + 2]};
    float fd_sum[3] = {0.0f, 0.0f, 0.0f};
    for (int k = 0; k < bc.substeps; ++k) {
        const float v0 = u[0] - ul[0], v1 = u[1] - ul[1], v2 = u[2] - ul[2];
        const float speed = sqrtf(v0 * v0 + v1 * v1 + v2 * v2);
        const float re = speed * K.re_per_speed;
        const float visc_a = K.visc_a0 * (1.0f + sn_coeff * __powf(re, sn_exp));
        const float cdv = fmaxf(fminf(visc_a, K.visc_b), K.eo_term * speed);   // C_D |v|
        const float kd = -K.drag_pref * cdv;
        const float fd[3] = {kd * v0, kd * v1, kd * v2};
        for (int a = 0; a < 3; ++a) {
            fd_sum[a] += fd[a];
            u[a] = fmaf(fb[a] + fd[a] + fvm[a], K.kdt, u[a]);
            xb[a] = fma((double)u[a], dt_b, xb[a]);
            if (g.walls & (1u << (2 * a))) {
                if (xb[a] < r) {
                    xb[a] = r;
                    u[a] = fmaxf(u[a], 0.0f);
                }
                if (xb[a] > (double)L[a] - r) {
                    xb[a] = (double)L[a] - r;
                    u[a] = fminf(u[a], 0.0f);
                }
            } else {
                xb[a] = __dsub_rn(xb[a], __dmul_rn((double)L[a], floor(xb[a] / (double)L[a])));
            }
        }
    }
    float psi[3];
    const float inv_sub = 1.0f / (float)bc.substeps;
    for (int a = 0; a < 3; ++a) {
        psi[a] = -fd_sum[a] * inv_sub;
        B.x[3 * b + a] = xb[a];
        B.u[3 * b + a] = u[a];
        B.ul[3 * b + a] = ul[a];
        B.ulprev[3 * b + a] = ul[a];
        B.psi[3 * b + a] = psi[a];
    }
    B.has_prev[b] = 1;
    if (!(isfinite(xb[0]) && isfinite(xb[1]) && isfinite(xb[2]) && isfinite(u[0]) &&
          isfinite(u[1]) && isfinite(u[2]) && isfinite(psi[0]) && isfinite(psi[1]) &&
          isfinite(psi[2]))) {
        B.active[b] = 0;
        B.spread[b] = 0;
        B.cell[b] = -1;
        atomicOr(flag, 2);
        return;
    }
    B.spread[b] = 1;
    int ci[3];
    for (int a = 0; a < 3; ++a) ci[a] = min(max((int)floor(xb[a]), 0), L[a] - 1);
    B.cell[b] = (ci[2] * g.ny + ci[1]) * g.nx + ci[0];
    make_record(xb, inv_n, g, psi, B.rec[b]);
    // Algorithm 1: the bubble stops once it reaches the top of the liquid.
    if ((g.walls & 0x20) && xb[2] >= (double)g.nz - r) B.active[b] = 0;
}

template <int ST>
__global__ void __launch_bounds__(BUBBLE_THREADS)
k_bubbles(const typename Store<ST>::T* __restrict__ f, Geo g, CollideParams cp, BubbleDev B,
          BubbleConst bc, int* __restrict__ flag) {
    __shared__ float red[3][BUBBLE_THREADS / 32];
    bubble_update<ST>(f, g, cp, B, bc, flag, blockIdx.x, red);
}

// Table 1 / Eq. 3 constants of each bubble (FP64).
__global__ void k_bubble_constants(BubbleDev B, BubbleConst bc, double width_factor) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B.nb) return;
    const double d = B.d[b];
    const double r = 0.5 * d;
    const double vol = M_PI * d * d * d / 6.0;
    const double eo = (bc.rho_l - bc.rho_b) * bc.g * d * d / bc.sigma;   // Eq. 3 with d^2
    BubbleK K;
    K.inv_nf = (float)(1.0 / B.n[b]);
    K.r = r;
    K.kdt = (float)(bc.dt_b / ((bc.rho_b + bc.c_am * bc.rho_l) * vol));
    K.fb = (float)((bc.rho_l - bc.rho_b) * vol * bc.g);
    K.drag_pref = (float)(0.5 * bc.rho_l * M_PI * r * r * bc.drag_scale);
    K.fvm_coef_dt = (float)(bc.c_am * bc.rho_l * vol / bc.dt_l);
    K.visc_a0 = (float)(24.0 * bc.nu / d);
    K.visc_b = (float)(48.0 * bc.nu / d);
    K.re_per_speed = (float)(d / bc.nu);
    K.eo_term = (float)(8.0 / 3.0 * eo / (eo + 4.0));
    B.k[b] = K;
    (void)width_factor;
}

cudaError_t launch_bubble_constants(const BubbleDev& b, const BubbleConst& bc, cudaStream_t st) {
    if (b.nb == 0) return cudaSuccess;
    k_bubble_constants<<<(b.nb + 127) / 128, 128, 0, st>>>(b, bc, 0.0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Binning (Algorithm 1 step 2): bubble windows -> tiles, deterministic lists
// ---------------------------------------------------------------------------

// Tiles of one axis holding at least one window cell, ascending.
__device__ int axis_tiles(double xa, double n, int L, bool periodic, int T,
                          int out[MAX_AXIS_TILES]) {
    int lo = (int)floor(xa - n);
    int hi = (int)ceil(xa + n) - 1;
    int cnt = 0;
    if (!periodic) {
        lo = max(lo, 0);
        hi = min(hi, L - 1);
        for (int t = lo / T; t <= hi / T && cnt < MAX_AXIS_TILES; ++t) out[cnt++] = t;
        return cnt;
    }
    for (int c = lo; c <= hi; ++c) {
        const int t = ((c % L + L) % L) / T;
        bool seen = false;
        for (int q = 0; q < cnt; ++q) seen |= (out[q] == t);
        if (!seen && cnt < MAX_AXIS_TILES) out[cnt++] = t;
    }
    for (int i = 1; i < cnt; ++i) {   // insertion sort, at most a few entries
        int v = out[i], k = i - 1;
        while (k >= 0 && out[k] > v) {
            out[k + 1] = out[k];
            --k;
        }
        out[k + 1] = v;
    }
    return cnt;
}

template <bool FILL>
__global__ void k_bin(Geo g, BubbleDev B, Bins bins) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B.nb || !B.spread[b]) return;
    const int L[3] = {g.nx, g.ny, g.nz};
    const int T[3] = {TX, TY, TZ};
    int tl[3][MAX_AXIS_TILES];
    int nt[3];
    const double n = B.n[b];
    for (int a = 0; a < 3; ++a)
        nt[a] = axis_tiles(B.x[3 * b + a], n, L[a], !(g.walls & (1u << (2 * a))), T[a], tl[a]);
    for (int iz = 0; iz < nt[2]; ++iz)
        for (int iy = 0; iy < nt[1]; ++iy)
            for (int ix = 0; ix < nt[0]; ++ix) {
                const int t = (tl[2][iz] * g.nty + tl[1][iy]) * g.ntx + tl[0][ix];
                const int pos = atomicAdd(&bins.cnt[t], 1);
                if (FILL) {
                    const int at = bins.off[t] + pos;
                    if (at < bins.cap) bins.items[at] = b;
                    else atomicOr(bins.overflow, 1);
                }
            }
}

// Sort each tile's list by bubble id so the gather order is fixed.
__global__ void k_bin_sort(Bins bins) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= bins.T) return;
    const int beg = bins.off[t], end = min(bins.off[t + 1], bins.cap);
    for (int i = beg + 1; i < end; ++i) {
        const int v = bins.items[i];
        int k = i - 1;
        while (k >= beg && bins.items[k] > v) {
            bins.items[k + 1] = bins.items[k];
            --k;
        }
        bins.items[k + 1] = v;
    }
}

// Exclusive scan of counts into offsets (3 passes, 1024 counts per block).
constexpr int SCAN_BLOCK = 256, SCAN_ITEMS = 4, SCAN_CHUNK = SCAN_BLOCK * SCAN_ITEMS;

int scan_blocks(int T) { return (T + SCAN_CHUNK - 1) / SCAN_CHUNK; }

__device__ int block_exclusive_scan(int v, int* warp_sums, int& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
        int si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += t;
        }
        if (lane < (int)(blockDim.x >> 5)) warp_sums[lane] = si - s;
        if (lane == (int)(blockDim.x >> 5) - 1) warp_sums[32] = si;
    }
    __syncthreads();
    const int res = warp_sums[wid] + incl - v;
    total = warp_sums[32];
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_local(const int* cnt, int* off, int T,
                                                            int* block_sums) {
    __shared__ int ws[33];
    const int base = blockIdx.x * SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = (base + k < T) ? cnt[base + k] : 0;
        s += v[k];
    }
    int total;
    int ex = block_exclusive_scan(s, ws, total);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < T) off[base + k] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_sums(int* block_sums, int nblocks, int* off,
                                                           int T) {
    __shared__ int ws[33];
    int carry = 0;
    for (int c0 = 0; c0 < nblocks; c0 += SCAN_BLOCK) {
        const int i = c0 + threadIdx.x;
        const int v = i < nblocks ? block_sums[i] : 0;
        int total;
        const int ex = block_exclusive_scan(v, ws, total);
        if (i < nblocks) block_sums[i] = ex + carry;
        carry += total;
    }
    if (threadIdx.x == 0) off[T] = carry;
}

__global__ void __launch_bounds__(SCAN_BLOCK) k_scan_add(int* off, int T, const int* block_sums) {
    const int base = blockIdx.x * SCAN_CHUNK + threadIdx.x * SCAN_ITEMS;
    const int add = block_sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < T) off[base + k] += add;
}

cudaError_t launch_binning(const Geo& g, const BubbleDev& b, const Bins& bins, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(bins.cnt, 0, sizeof(int) * (size_t)bins.T, st);
    if (e != cudaSuccess) return e;
    const int tb = 128;
    const int bb = (b.nb + tb - 1) / tb;
    if (b.nb > 0) k_bin<false><<<bb, tb, 0, st>>>(g, b, bins);
    k_scan_local<<<bins.nblocks, SCAN_BLOCK, 0, st>>>(bins.cnt, bins.off, bins.T, bins.block_sums);
    k_scan_sums<<<1, SCAN_BLOCK, 0, st>>>(bins.block_sums, bins.nblocks, bins.off, bins.T);
    k_scan_add<<<bins.nblocks, SCAN_BLOCK, 0, st>>>(bins.off, bins.T, bins.block_sums);
    e = cudaMemsetAsync(bins.cnt, 0, sizeof(int) * (size_t)bins.T, st);
    if (e != cudaSuccess) return e;
    if (b.nb > 0) k_bin<true><<<bb, tb, 0, st>>>(g, b, bins);
    k_bin_sort<<<(bins.T + 127) / 128, 128, 0, st>>>(bins);
    return cudaGetLastError();
}

// Few pairs: one CTA enumerates every (tile, bubble) pair, sorts the keys
// (tile << 32 | bubble) with a bitonic network in shared memory and writes the
// runs.  The per-tile counts stay valid between calls because only the tiles
// the previous call touched are cleared first.  The bubble state is read with
// __ldcg: it was written by other CTAs of the same launch.
// With `cols` set (a batch), bubble b lives in column bubble_col[b], whose
// tiles are numbered from cols[c].tile_base in the shared tile space.
__device__ void bin_small_block(const Geo& g, const BubbleDev& B, const SmallBins& sb,
                                unsigned long long* keys, int* s_n,
                                const BatchColumn* cols = nullptr,
                                const int* bubble_col = nullptr) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int prev = min(max(__ldcg(sb.prev_n), 0), SMALL_MAX_PAIRS);
    for (int i = tid; i < prev; i += nt) {
        const int t = __ldcg(sb.prev_tiles + i);
        if (t >= 0 && t < sb.T) sb.count[t] = 0;
    }
    if (tid == 0) *s_n = 0;
    __syncthreads();
    const int T[3] = {TX, TY, TZ};
    for (int b = tid; b < B.nb; b += nt) {
        if (!__ldcg(B.spread + b)) continue;
        const Geo& gb = cols ? cols[bubble_col[b]].g : g;
        const int base = cols ? cols[bubble_col[b]].tile_base : 0;
        const int L[3] = {gb.nx, gb.ny, gb.nz};
        int tl[3][MAX_AXIS_TILES];
        int ntl[3];
        const double n = __ldcg(B.n + b);
        for (int a = 0; a < 3; ++a)
            ntl[a] = axis_tiles(__ldcg(B.x + 3 * b + a), n, L[a], !(gb.walls & (1u << (2 * a))),
                                T[a], tl[a]);
        for (int iz = 0; iz < ntl[2]; ++iz)
            for (int iy = 0; iy < ntl[1]; ++iy)
                for (int ix = 0; ix < ntl[0]; ++ix) {
                    const unsigned t = (unsigned)(base + (tl[2][iz] * gb.nty + tl[1][iy]) * gb.ntx +
                                                  tl[0][ix]);
                    const int k = atomicAdd(s_n, 1);
                    if (k < SMALL_MAX_PAIRS) keys[k] = ((unsigned long long)t << 32) | (unsigned)b;
                    else atomicOr(sb.overflow, 1);
                }
    }
    __syncthreads();
    const int n = min(*s_n, SMALL_MAX_PAIRS);
    int p2 = 1;
    while (p2 < n) p2 <<= 1;
    for (int i = n + tid; i < p2; i += nt) keys[i] = ~0ull;
    __syncthreads();
    for (int k = 2; k <= p2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < p2; i += nt) {
                const int l = i ^ j;
                if (l > i) {
                    const unsigned long long a = keys[i], c = keys[l];
                    const bool up = (i & k) == 0;
                    if ((a > c) == up) {
                        keys[i] = c;
                        keys[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < n; i += nt) {
        const int t = (int)(keys[i] >> 32);
        sb.items[i] = (int)(keys[i] & 0xffffffffu);
        sb.prev_tiles[i] = t;
        if (i == 0 || (int)(keys[i - 1] >> 32) != t) sb.start[t] = i;
        atomicAdd(&sb.count[t], 1);
    }
    if (tid == 0) *sb.prev_n = n;
}

// Bubble update with the few-pair binning fused behind it: every CTA updates
// its bubble, then counts itself done; the CTA that finds all others done
// (no waiting: it is simply the last to arrive) bins all bubbles.
template <int ST>
__global__ void __launch_bounds__(BUBBLE_THREADS)
k_bubbles_binned(const typename Store<ST>::T* __restrict__ f, Geo g, CollideParams cp,
                 BubbleDev B, BubbleConst bc, int* __restrict__ flag, SmallBins sb) {
    __shared__ float red[3][BUBBLE_THREADS / 32];
    __shared__ unsigned long long keys[SMALL_MAX_PAIRS];
    __shared__ int s_n, s_last;
    bubble_update<ST>(f, g, cp, B, bc, flag, blockIdx.x, red);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();                                 // publish this bubble's state
        s_last = atomicAdd(sb.done, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    bin_small_block(g, B, sb, keys, &s_n);
    if (threadIdx.x == 0) *sb.done = 0;                  // ready for the next launch
}

cudaError_t launch_bubbles(int storage, const void* f, const Geo& g, const CollideParams& cp,
                           const BubbleDev& b, const BubbleConst& bc, int* flag,
                           const SmallBins* fused, cudaStream_t st) {
    if (b.nb == 0) return cudaSuccess;
    if (fused) {
        switch (storage) {
            case 0:
                k_bubbles_binned<0><<<b.nb, BUBBLE_THREADS, 0, st>>>((const float*)f, g, cp, b, bc,
                                                                     flag, *fused);
                break;
            case 1:
                k_bubbles_binned<1><<<b.nb, BUBBLE_THREADS, 0, st>>>((const __half*)f, g, cp, b, bc,
                                                                     flag, *fused);
                break;
            default:
                k_bubbles_binned<2><<<b.nb, BUBBLE_THREADS, 0, st>>>(
                    (const __nv_bfloat16*)f, g, cp, b, bc, flag, *fused);
                break;
        }
        return cudaGetLastError();
    }
    switch (storage) {
        case 0:
            k_bubbles<0><<<b.nb, BUBBLE_THREADS, 0, st>>>((const float*)f, g, cp, b, bc, flag);
            break;
        case 1:
            k_bubbles<1><<<b.nb, BUBBLE_THREADS, 0, st>>>((const __half*)f, g, cp, b, bc, flag);
            break;
        default:
            k_bubbles<2><<<b.nb, BUBBLE_THREADS, 0, st>>>((const __nv_bfloat16*)f, g, cp, b, bc,
                                                          flag);
            break;
    }
    return cudaGetLastError();
}

// Bubble update of a batch: bubble b moves in column bubble_col[b]; the
// few-pair binning of all columns is fused behind it as for one column.
template <int ST>
__global__ void __launch_bounds__(BUBBLE_THREADS)
k_bubbles_batch(const typename Store<ST>::T* __restrict__ f, const BatchColumn* __restrict__ cols,
                const int* __restrict__ bubble_col, BubbleDev B, BubbleConst bc,
                int* __restrict__ flag, SmallBins sb) {
    __shared__ float red[3][BUBBLE_THREADS / 32];
    __shared__ unsigned long long keys[SMALL_MAX_PAIRS];
    __shared__ int s_n, s_last;
    const int b = blockIdx.x;
    const BatchColumn& col = cols[bubble_col[b]];
    bubble_update<ST>(f + col.pop_offset, col.g, col.cp, B, bc, flag, b, red);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(sb.done, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    bin_small_block(col.g, B, sb, keys, &s_n, cols, bubble_col);
    if (threadIdx.x == 0) *sb.done = 0;
}

cudaError_t launch_bubbles_batch(int storage, const void* f, const BatchColumn* cols,
                                 const int* bubble_col, const BubbleDev& b, const BubbleConst& bc,
                                 int* flag, const SmallBins& sb, cudaStream_t st) {
    if (b.nb == 0) return cudaSuccess;
    switch (storage) {
        case 0:
            k_bubbles_batch<0><<<b.nb, BUBBLE_THREADS, 0, st>>>((const float*)f, cols, bubble_col,
                                                                b, bc, flag, sb);
            break;
        case 1:
            k_bubbles_batch<1><<<b.nb, BUBBLE_THREADS, 0, st>>>((const __half*)f, cols, bubble_col,
                                                                b, bc, flag, sb);
            break;
        default:
            k_bubbles_batch<2><<<b.nb, BUBBLE_THREADS, 0, st>>>((const __nv_bfloat16*)f, cols,
                                                                bubble_col, b, bc, flag, sb);
            break;
    }
    return cudaGetLastError();
}

// Per-bubble closure constants for a batch: nu from each bubble's column.
__global__ void k_bubble_constants_batch(BubbleDev B, BubbleConst bc, const double* col_nu,
                                         const int* bubble_col) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B.nb) return;
    BubbleConst c = bc;
    c.nu = col_nu[bubble_col[b]];
    const double d = B.d[b];
    const double r = 0.5 * d;
    const double vol = M_PI * d * d * d / 6.0;
    const double eo = (c.rho_l - c.rho_b) * c.g * d * d / c.sigma;
    BubbleK K;
    K.inv_nf = (float)(1.0 / B.n[b]);
    K.r = r;
    K.kdt = (float)(c.dt_b / ((c.rho_b + c.c_am * c.rho_l) * vol));
    K.fb = (float)((c.rho_l - c.rho_b) * vol * c.g);
    K.drag_pref = (float)(0.5 * c.rho_l * M_PI * r * r * c.drag_scale);
    K.fvm_coef_dt = (float)(c.c_am * c.rho_l * vol / c.dt_l);
    K.visc_a0 = (float)(24.0 * c.nu / d);
    K.visc_b = (float)(48.0 * c.nu / d);
    K.re_per_speed = (float)(d / c.nu);
    K.eo_term = (float)(8.0 / 3.0 * eo / (eo + 4.0));
    B.k[b] = K;
}

cudaError_t launch_bubble_constants_batch(const BubbleDev& b, const BubbleConst& bc,
                                          const double* col_nu, const int* bubble_col,
                                          cudaStream_t st) {
    if (b.nb == 0) return cudaSuccess;
    k_bubble_constants_batch<<<(b.nb + 127) / 128, 128, 0, st>>>(b, bc, col_nu, bubble_col);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Field utilities
// ---------------------------------------------------------------------------

// Eq. 10 moments of the pre-collision populations, FP64.
template <int ST>
__global__ void k_fields(const typename Store<ST>::T* __restrict__ f, Geo g, CollideParams cp,
                         double* __restrict__ rho, double* __restrict__ u) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.S) return;
    const int x = (int)(s % g.nx), y = (int)((s / g.nx) % g.ny), z = (int)(s / ((long long)g.nx * g.ny));
    float gv[Q];
    gather<ST>(f, g, cp, x, y, z, gv);
    double drho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        drho += gv[j];
        jx += cx(j) * (double)gv[j];
        jy += cy(j) * (double)gv[j];
        jz += cz(j) * (double)gv[j];
    }
    const double r = (double)cp.rho0 + drho;
    if (rho) rho[s] = r;
    if (u) {
        u[s] = jx / r;
        u[g.S + s] = jy / r;
        u[2 * g.S + s] = jz / r;
    }
}

template <int ST>
__global__ void k_get_pop(const typename Store<ST>::T* __restrict__ f, Geo g, CollideParams cp,
                          double* __restrict__ out) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.S) return;
    const int x = (int)(s % g.nx), y = (int)((s / g.nx) % g.ny), z = (int)(s / ((long long)g.nx * g.ny));
    float gv[Q];
    gather<ST>(f, g, cp, x, y, z, gv);
#pragma unroll
    for (int j = 0; j < Q; ++j) out[(size_t)j * g.S + s] = wd(j) * (double)cp.rho0 + (double)gv[j];
}

// Where the stored (post-collision) value of direction j at node y comes
// from: the population j of node y + c_j, or -- if that link crosses a
// wall -- the population opp(j) of node y itself (inverse of the pull).
__device__ __forceinline__ void push_target(const Geo& g, int j, int x, int y, int z, int& dir,
                                            long long& node) {
    int tx = x + cx(j), ty = y + cy(j), tz = z + cz(j);
    bool bounce = false;
    if (cx(j) != 0 && (tx < 0 || tx >= g.nx)) {
        if (g.walls & 0x01) bounce = true;
        else tx = tx < 0 ? tx + g.nx : tx - g.nx;
    }
    if (cy(j) != 0 && (ty < 0 || ty >= g.ny)) {
        if (g.walls & 0x04) bounce = true;
        else ty = ty < 0 ? ty + g.ny : ty - g.ny;
    }
    if (cz(j) != 0 && (tz < 0 || tz >= g.nz)) {
        if (g.walls & 0x10) bounce = true;
        else tz = tz < 0 ? tz + g.nz : tz - g.nz;
    }
    if (bounce) {
        dir = opp(j);
        node = site_index(g, x, y, z);
    } else {
        dir = j;
        node = site_index(g, tx, ty, tz);
    }
}

template <int ST>
__global__ void k_set_pop(const double* __restrict__ fin, typename Store<ST>::T* __restrict__ f,
                          Geo g, CollideParams cp) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.S) return;
    const int x = (int)(s % g.nx), y = (int)((s / g.nx) % g.ny), z = (int)(s / ((long long)g.nx * g.ny));
    for (int j = 0; j < Q; ++j) {
        int dir;
        long long node;
        push_target(g, j, x, y, z, dir, node);
        const double v = fin[(size_t)dir * g.S + node] - wd(dir) * (double)cp.rho0;
        f[(size_t)j * g.S + s] = Store<ST>::from_double(v, j, cp);
    }
}

// f = f^eq(rho, u) of Eq. 6, stored shifted: g^eq_j = w_j [drho + rho (3cu + 4.5cu^2 - 1.5u^2)].
template <int ST>
__global__ void k_set_feq(const double* __restrict__ rho, const double* __restrict__ u,
                          typename Store<ST>::T* __restrict__ f, Geo g, CollideParams cp) {
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.S) return;
    const int x = (int)(s % g.nx), y = (int)((s / g.nx) % g.ny), z = (int)(s / ((long long)g.nx * g.ny));
    for (int j = 0; j < Q; ++j) {
        int dir;
        long long node;
        push_target(g, j, x, y, z, dir, node);
        const double r = rho ? rho[node] : (double)cp.rho0;
        const double ux = u ? u[node] : 0.0, uy = u ? u[g.S + node] : 0.0,
                     uz = u ? u[2 * g.S + node] : 0.0;
        const double cu = cx(dir) * ux + cy(dir) * uy + cz(dir) * uz;
        const double usq = ux * ux + uy * uy + uz * uz;
        const double v = wd(dir) * ((r - (double)cp.rho0) + r * (3.0 * cu + 4.5 * cu * cu - 1.5 * usq));
        f[(size_t)j * g.S + s] = Store<ST>::from_double(v, j, cp);
    }
}

// FP64 totals: per-block partial sums in fixed order, then one block.
constexpr int TOT_BLOCK = 256;

int totals_partials(const Geo& g) {
    long long blocks = (g.S + TOT_BLOCK - 1) / TOT_BLOCK;
    return (int)(blocks < 4096 ? blocks : 4096);
}

__device__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;
}

template <int ST>
__global__ void __launch_bounds__(TOT_BLOCK)
k_totals(const typename Store<ST>::T* __restrict__ f, Geo g, CollideParams cp, double* partials) {
    __shared__ double sh[32];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.S;
         s += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(s % g.nx), y = (int)((s / g.nx) % g.ny),
                  z = (int)(s / ((long long)g.nx * g.ny));
        float gv[Q];
        gather<ST>(f, g, cp, x, y, z, gv);
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            acc[0] += gv[j];
            acc[1] += cx(j) * (double)gv[j];
            acc[2] += cy(j) * (double)gv[j];
            acc[3] += cz(j) * (double)gv[j];
        }
    }
    for (int k = 0; k < 4; ++k) {
        const double t = block_sum(acc[k], sh);
        if (threadIdx.x == 0) partials[4 * blockIdx.x + k] = t;
    }
}

__global__ void k_totals_final(const double* partials, int np, double mass0, double* out4) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < np; ++i)
        for (int k = 0; k < 4; ++k) t[k] += partials[4 * i + k];
    out4[0] = mass0 + t[0];
    out4[1] = t[1];
    out4[2] = t[2];
    out4[3] = t[3];
}

static unsigned site_blocks(const Geo& g) { return (unsigned)((g.S + 255) / 256); }

cudaError_t launch_fields(int storage, const void* f, const Geo& g, const CollideParams& cp,
                          double* rho, double* u, cudaStream_t st) {
    switch (storage) {
        case 0: k_fields<0><<<site_blocks(g), 256, 0, st>>>((const float*)f, g, cp, rho, u); break;
        case 1: k_fields<1><<<site_blocks(g), 256, 0, st>>>((const __half*)f, g, cp, rho, u); break;
        default:
            k_fields<2><<<site_blocks(g), 256, 0, st>>>((const __nv_bfloat16*)f, g, cp, rho, u);
    }
    return cudaGetLastError();
}

cudaError_t launch_get_populations(int storage, const void* f, const Geo& g,
                                   const CollideParams& cp, double* out, cudaStream_t st) {
    switch (storage) {
        case 0: k_get_pop<0><<<site_blocks(g), 256, 0, st>>>((const float*)f, g, cp, out); break;
        case 1: k_get_pop<1><<<site_blocks(g), 256, 0, st>>>((const __half*)f, g, cp, out); break;
        default:
            k_get_pop<2><<<site_blocks(g), 256, 0, st>>>((const __nv_bfloat16*)f, g, cp, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_set_populations(int storage, const double* fin, void* f, const Geo& g,
                                   const CollideParams& cp, cudaStream_t st) {
    switch (storage) {
        case 0: k_set_pop<0><<<site_blocks(g), 256, 0, st>>>(fin, (float*)f, g, cp); break;
        case 1: k_set_pop<1><<<site_blocks(g), 256, 0, st>>>(fin, (__half*)f, g, cp); break;
        default: k_set_pop<2><<<site_blocks(g), 256, 0, st>>>(fin, (__nv_bfloat16*)f, g, cp);
    }
    return cudaGetLastError();
}

cudaError_t launch_set_equilibrium(int storage, const double* rho, const double* u, void* f,
                                   const Geo& g, const CollideParams& cp, cudaStream_t st) {
    switch (storage) {
        case 0: k_set_feq<0><<<site_blocks(g), 256, 0, st>>>(rho, u, (float*)f, g, cp); break;
        case 1: k_set_feq<1><<<site_blocks(g), 256, 0, st>>>(rho, u, (__half*)f, g, cp); break;
        default:
            k_set_feq<2><<<site_blocks(g), 256, 0, st>>>(rho, u, (__nv_bfloat16*)f, g, cp);
    }
    return cudaGetLastError();
}

cudaError_t launch_totals(int storage, const void* f, const Geo& g, const CollideParams& cp,
                          double* partials, int npartials, double* out4, cudaStream_t st) {
    switch (storage) {
        case 0: k_totals<0><<<npartials, TOT_BLOCK, 0, st>>>((const float*)f, g, cp, partials); break;
        case 1: k_totals<1><<<npartials, TOT_BLOCK, 0, st>>>((const __half*)f, g, cp, partials); break;
        default:
            k_totals<2><<<npartials, TOT_BLOCK, 0, st>>>((const __nv_bfloat16*)f, g, cp, partials);
    }
    k_totals_final<<<1, 32, 0, st>>>(partials, npartials, (double)g.S * (double)cp.rho0, out4);
    return cudaGetLastError();
}

}  // namespace lbm
