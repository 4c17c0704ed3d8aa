// Bubble side of the coupled step and the field utilities.
//
//  k_bubbles_binned  few bubbles: the window of each bubble is reduced by one
//                    or more CTAs (gathered Eq. 10 velocity, Eq. 19-20); the
//                    CTA completing a bubble does the Table 1 forces, the
//                    sub-stepped Newton update (Eq. 4, Table 2), the reaction
//                    psi_b = -mean F_D (Algorithm 1 step 6) and the spreading
//                    record; the last one bins all bubbles.
//  k_tile_interp,    many bubbles: per listed tile, the Eq. 10 velocity of its
//  k_swarm_tail,     nodes and each listed bubble's Eq. 20 sum over it; per
//  k_swarm_bin       bubble, the parts added and the update; the binning in
//                    one persistent launch.
//  binning           bubble windows to lattice tiles (Algorithm 1 step 2):
//                    integer counting sort, then each tile's list in bubble
//                    order.
//  field kernels     initialisation to f^eq (Eq. 6), population I/O, Eq. 10
//                    moments and FP64 totals.
#include <climits>
#include <algorithm>
#include <cmath>
#include <vector>

#include "lbm_device.cuh"

namespace lbm {

// ---------------------------------------------------------------------------
// Bubble update
// ---------------------------------------------------------------------------

// ---- positions in two floats ------------------------------------------------
// A position is carried through the sub-steps as hi + lo, two floats with
// |lo| <= ulp(hi)/2 (about 48 significant bits), so the 10 sub-steps use the
// FP32 pipe: FP64 issue is slow on this GPU and the bubble update is one
// serial thread.  Sums use Knuth's TwoSum; the product error of u dt_b comes
// from one FMA (the exact-product property of fused multiply-add).
struct F2 {
    float h, l;
};

__device__ __forceinline__ F2 f2_from(double v) {
    const float h = (float)v;
    return F2{h, (float)(v - (double)h)};
}

__device__ __forceinline__ double f2_to(F2 a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return F2{s, (a - (s - bb)) + (b - bb)};
}

// (a.h + a.l) + (bh + bl)
__device__ __forceinline__ F2 f2_add(F2 a, float bh, float bl) {
    const F2 s = two_sum(a.h, bh);
    return two_sum(s.h, s.l + (a.l + bl));
}

__device__ __forceinline__ bool f2_lt(F2 a, F2 b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }

// floor of hi + lo and the fraction (hi + lo) - floor in [0, 1].
__device__ __forceinline__ int f2_floor(F2 a, float& frac) {
    float f = floorf(a.h);
    if (f == a.h && a.l < 0.0f) f -= 1.0f;
    frac = (a.h - f) + a.l;
    return (int)f;
}

// floor and ceil of hi + lo.  With |lo| <= ulp(hi)/2 the sum can cross an
// integer only when hi itself is one, so lo decides only then.
__device__ __forceinline__ int f2_floor_int(F2 a) {
    float f = floorf(a.h);
    if (f == a.h && a.l < 0.0f) f -= 1.0f;
    return (int)f;
}

__device__ __forceinline__ int f2_ceil_int(F2 a) {
    float c = ceilf(a.h);
    if (c == a.h && a.l > 0.0f) c += 1.0f;
    return (int)c;
}

// Window normalisation along one axis: the sum of the axis weights over the
// in-box cells.  For cell integrals (h > 0) that is the integral of the
// mapping over the in-box part of [-n, n] (without 15/16), for the two-float
// coordinate xa, and the full 16/15 on a periodic axis.  For point samples
// (h < 0) it is the sum of the node samples themselves, evaluated as the
// weights are (cell_poly of the offset from the anchor cell anc, fraction fr)
// over the cells within n + 1 of the centre.
__device__ __forceinline__ float axis_norm(F2 xa, int anc, float fr, float inv_n, float h, int L,
                                           bool periodic) {
    if (h < 0.0f) {
        const int K = (int)ceilf(1.0f / inv_n) + 1;
        float sum = 0.0f;
        for (int k = -K; k <= K; ++k) {
            const int c = anc + k;
            if (!periodic && (c < 0 || c >= L)) continue;
            sum += cell_poly(((float)k + 0.5f - fr) * inv_n, h);
        }
        return sum;
    }
    if (periodic) return 16.0f / 15.0f;
    const float lo = (-xa.h - xa.l) * inv_n, hi = (((float)L - xa.h) - xa.l) * inv_n;
    const float a = fmaxf(lo, -1.0f), b = fminf(hi, 1.0f);
    if (!(b > a)) return 0.0f;
    const float a2 = a * a, b2 = b * b, ab = a * b;
    const float p4 = b2 * b2 + b2 * ab + ab * ab + ab * a2 + a2 * a2;
    return (b - a) * (p4 * 0.2f - (b2 + ab + a2) * (2.0f / 3.0f) + 1.0f);
}

__device__ __forceinline__ void make_record(const F2* xb, const BubbleK& K, const Geo& g,
                                            const float* psi, BubbleRec& r) {
    const float inv_n = K.inv_nf;
    int anc[3];
    float fr[3];
    float norm = 1.0f;
    const int L[3] = {g.nx, g.ny, g.nz};
    for (int a = 0; a < 3; ++a) {
        anc[a] = f2_floor(xb[a], fr[a]);
        norm *= axis_norm(xb[a], anc[a], fr[a], inv_n, K.hmap, L[a],
                          !(g.walls & (1u << (2 * a))));
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
    r.h = K.hmap;
    r.px = psi[0] * inv_norm;
    r.py = psi[1] * inv_norm;
    r.pz = psi[2] * inv_norm;
}

// Bare Eq. 10 velocity u = sum_j c_j g_j / (rho0 + sum_j g_j) of shifted
// pre-collision populations.
__device__ __forceinline__ void node_velocity(const float gv[Q], const CollideParams& cp,
                                              float u[3]) {
    float drho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
        drho += gv[q];
        if (cx(q) != 0) jx += (float)cx(q) * gv[q];
        if (cy(q) != 0) jy += (float)cy(q) * gv[q];
        if (cz(q) != 0) jz += (float)cz(q) * gv[q];
    }
    const float inv_rho = 1.0f / (cp.rho0 + drho);
    u[0] = jx * inv_rho;
    u[1] = jy * inv_rho;
    u[2] = jz * inv_rho;
}

// Precision: positions are integrated in FP64 (they reach hundreds of lattice
// units and move by 1e-5 per sub-step); velocities, forces and the mapping
// weights are FP32.  FP64 latency on this GPU is long, so only the position
// update, the window bounds and the wall tests use it.
constexpr int BUBBLE_THREADS = 256;

// The interpolation window of one bubble (Algorithm 1 step 2): the cells
// overlapping (x - n, x + n) per axis, the anchor cell and fraction of the
// centre, and the in-domain weight sum used to renormalise.
struct Window {
    int lo[3], cnt[3], anc[3];
    float fr[3];
    float norm;
    float h;  // cell_poly's h: 1/(2n) for cell integrals, -1/(2n) for point samples
    int M;   // nodes in the window
};

enum { BUBBLE_LIVE = 0, BUBBLE_IDLE = 1, BUBBLE_NONFINITE = 2 };

// The state of one bubble that an update reads, loaded in one round trip at
// the start of the kernel (the integration part only by the thread that will
// integrate, `full`).
struct BubbleIn {
    F2 x[3];
    BubbleK k;
    float u[3], ulprev[3];
    int active, has_prev;
};

// The state the previous update wrote is read through L2 (ld.global.cg): that
// update may have run as an overlapped launch.
__device__ __forceinline__ void load_bubble(const BubbleDev& B, int b, bool full, BubbleIn& in) {
    in.active = __ldcg(B.active + b);
    for (int a = 0; a < 3; ++a) in.x[a] = F2{__ldcg(B.xh + 3 * b + a), __ldcg(B.xl + 3 * b + a)};
    in.k = B.k[b];
    in.has_prev = full ? __ldcg(B.has_prev + b) : 0;
    for (int a = 0; a < 3; ++a) {
        in.u[a] = full ? __ldcg(B.u + 3 * b + a) : 0.0f;
        in.ulprev[a] = full ? __ldcg(B.ulprev + 3 * b + a) : 0.0f;
    }
}

// First and last cell of the support (x - n, x + n) on one axis, before
// clipping: floor(x - n) and ceil(x + n) - 1, from the two-float centre and
// half-width.
__device__ __forceinline__ void support_cells(F2 x, float nh, float nl, int& lo, int& hi) {
    lo = f2_floor_int(f2_add(x, -nh, -nl));
    hi = f2_ceil_int(f2_add(x, nh, nl)) - 1;
}

// pad: cells added beyond the support on each side (the vorticity halo of
// lift), clipped to the box on wall axes.
__device__ int bubble_window(const Geo& g, const BubbleIn& in, Window& w, int pad = 0) {
    const F2* xb = in.x;
    const float inv_n = in.k.inv_nf;
    if (!in.active) return BUBBLE_IDLE;
    const int L[3] = {g.nx, g.ny, g.nz};
    // A non-finite centre can only come from an unstable liquid.
    if (!(isfinite(xb[0].h) && isfinite(xb[1].h) && isfinite(xb[2].h))) return BUBBLE_NONFINITE;
    w.norm = 1.0f;
    w.h = in.k.hmap;
    for (int a = 0; a < 3; ++a) {
        const bool periodic = !(g.walls & (1u << (2 * a)));
        int l, h;
        support_cells(xb[a], in.k.nh, in.k.nl, l, h);
        l -= pad;
        h += pad;
        if (!periodic) {
            l = max(l, 0);
            h = min(h, L[a] - 1);
        }
        w.lo[a] = l;
        w.cnt[a] = min(max(h - l + 1, 0), WINDOW_CELLS_MAX);
        w.anc[a] = f2_floor(xb[a], w.fr[a]);
        w.norm *= axis_norm(xb[a], w.anc[a], w.fr[a], inv_n, w.h, L[a], periodic);
    }
    w.M = w.cnt[0] * w.cnt[1] * w.cnt[2];
    return BUBBLE_LIVE;
}

// Weight and wrapped lattice coordinates of window node m (x fastest).
// m / d for 0 <= m < 2^13 and 1 <= d <= WINDOW_CELLS_MAX, through the float
// reciprocal: (m + 0.5) / d lies at least 1/(2d) from an integer, far more
// than the rounding of the product, so the truncation is exact.
__device__ __forceinline__ int div_small(int m, int d) {
    return (int)(((float)m + 0.5f) * (1.0f / (float)d));
}

// A window coordinate wrapped into [0, L) (windows are narrower than the box).
__device__ __forceinline__ int wrap_axis(int i, int L) {
    return i < 0 ? i + L : (i >= L ? i - L : i);
}

__device__ __forceinline__ float window_node(const Geo& g, const Window& w, float inv_n, int m,
                                             int& iw, int& jw, int& kw) {
    const float hh = w.h;
    const int rest = div_small(m, w.cnt[0]);
    const int ix = m - rest * w.cnt[0];
    const int iz = div_small(rest, w.cnt[1]);
    const int iy = rest - iz * w.cnt[1];
    const int i = w.lo[0] + ix, j = w.lo[1] + iy, k = w.lo[2] + iz;
    iw = wrap_axis(i, g.nx);
    jw = wrap_axis(j, g.ny);
    kw = wrap_axis(k, g.nz);
    return cell_poly(((float)(i - w.anc[0]) + 0.5f - w.fr[0]) * inv_n, hh) *
           cell_poly(((float)(j - w.anc[1]) + 0.5f - w.fr[1]) * inv_n, hh) *
           cell_poly(((float)(k - w.anc[2]) + 0.5f - w.fr[2]) * inv_n, hh);
}

// Lift: the four weights of window node m -- W = wx wy wz (Eq. 19) and the
// difference weights Gx = dx wy wz, Gy = wx dy wz, Gz = wx wy dz (axis_wd) --
// and its wrapped lattice coordinates.
__device__ __forceinline__ void window_node_lift(const Geo& g, const Window& w, float inv_n,
                                                 int m, int& iw, int& jw, int& kw, float wt[4]) {
    const float hh = w.h;
    const int rest = div_small(m, w.cnt[0]);
    const int ix = m - rest * w.cnt[0];
    const int iz = div_small(rest, w.cnt[1]);
    const int iy = rest - iz * w.cnt[1];
    const int c[3] = {w.lo[0] + ix, w.lo[1] + iy, w.lo[2] + iz};
    const int L[3] = {g.nx, g.ny, g.nz};
    float ww[3], dd[3];
    for (int a = 0; a < 3; ++a)
        axis_wd(c[a], w.anc[a], w.fr[a], inv_n, hh, L[a], !(g.walls & (1u << (2 * a))),
                a == 2 && (g.walls & WALL_TOP_FREE), ww[a], dd[a]);
    iw = wrap_axis(c[0], g.nx);
    jw = wrap_axis(c[1], g.ny);
    kw = wrap_axis(c[2], g.nz);
    wt[0] = ww[0] * ww[1] * ww[2];
    wt[1] = dd[0] * ww[1] * ww[2];
    wt[2] = ww[0] * dd[1] * ww[2];
    wt[3] = ww[0] * ww[1] * dd[2];
}

// Adds node velocity u with weights wt (LIFT) or weight wt[0] into acc:
// acc[0..2] the Eq. 20 velocity sums; with lift acc[3..8] = Gx u_y, Gx u_z,
// Gy u_x, Gy u_z, Gz u_x, Gz u_y (the interpolated central differences
// d(u_y)/dx, d(u_z)/dx, d(u_x)/dy, d(u_z)/dy, d(u_x)/dz, d(u_y)/dz).
template <bool LIFT>
__device__ __forceinline__ void add_window_node(const float wt[4], const float u[3], float* acc) {
    acc[0] = fmaf(wt[0], u[0], acc[0]);
    acc[1] = fmaf(wt[0], u[1], acc[1]);
    acc[2] = fmaf(wt[0], u[2], acc[2]);
    if (LIFT) {
        acc[3] = fmaf(wt[1], u[1], acc[3]);
        acc[4] = fmaf(wt[1], u[2], acc[4]);
        acc[5] = fmaf(wt[2], u[0], acc[5]);
        acc[6] = fmaf(wt[2], u[2], acc[6]);
        acc[7] = fmaf(wt[3], u[0], acc[7]);
        acc[8] = fmaf(wt[3], u[1], acc[8]);
    }
}

// Eq. 20 partial sums of one chunk: nodes m0 + tid and m0 + tid + nt (below
// m1), both gathered before either is used so their loads overlap.
template <int ST, bool LIFT>
__device__ __forceinline__ void chunk_sum2(const typename Store<ST>::T* __restrict__ f,
                                           const Geo& g, const CollideParams& cp, const Window& w,
                                           float inv_n, int m0, int m1, int tid, int nt,
                                           float* acc) {
    const int ma = m0 + tid, mb = ma + nt;
    const bool ha = ma < m1, hb = mb < m1;
    int ia, ja, ka, ib, jb, kb;
    float wa[4], wb[4];
    if (LIFT) {
        window_node_lift(g, w, inv_n, ha ? ma : m0, ia, ja, ka, wa);
        window_node_lift(g, w, inv_n, hb ? mb : m0, ib, jb, kb, wb);
    } else {
        wa[0] = window_node(g, w, inv_n, ha ? ma : m0, ia, ja, ka);
        wb[0] = window_node(g, w, inv_n, hb ? mb : m0, ib, jb, kb);
    }
    typename Store<ST>::T ra[Q], rb[Q];
    gather_issue<ST>(f, g, ia, ja, ka, ra);
    gather_issue<ST>(f, g, ib, jb, kb, rb);
    float ga[Q], gb[Q];
    gather_finish<ST>(ra, cp, ga);
    gather_finish<ST>(rb, cp, gb);
    float ua[3], ub[3];
    node_velocity(ga, cp, ua);
    node_velocity(gb, cp, ub);
    if (ha) add_window_node<LIFT>(wa, ua, acc);
    if (hb) add_window_node<LIFT>(wb, ub, acc);
}

__device__ __forceinline__ void warp_sum3(float& ax, float& ay, float& az) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
    }
}

// Sum of v[0..N) over the CTA's BUBBLE_THREADS threads, in thread 0 (fixed
// order: warp shuffles, then warps in order).
template <int N>
__device__ __forceinline__ void block_sum_n(float* v, float (*red)[BUBBLE_THREADS / 32]) {
#pragma unroll
    for (int q = 0; q < N; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
    const int tid = threadIdx.x;
    if ((tid & 31) == 0)
#pragma unroll
        for (int q = 0; q < N; ++q) red[q][tid >> 5] = v[q];
    __syncthreads();
    if (tid == 0) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            v[q] = 0.0f;
            for (int k = 0; k < BUBBLE_THREADS / 32; ++k) v[q] += red[q][k];
        }
    }
}

// One thread: everything after the window sums (ax, ay, az) of bubble b.
// An idle bubble leaves the coupling; a non-finite one is deactivated and
// flags the instability; a live one takes the Table 1 forces and the Newton
// update of Eq. 4 with the added mass on the left (m_eff), sub-stepped with
// dt_b (Table 2), then its reaction psi (Algorithm 1) and spreading record.
// acc: the window sums, acc[0..2] the Eq. 20 velocity and, with lift,
// acc[3..8] the vorticity sums (add_window_node).
__device__ void bubble_tail(const Geo& g, const BubbleDev& B, const BubbleConst& bc,
                            int* __restrict__ flag, int b, int state, const Window& w,
                            const float* acc, const BubbleIn& in) {
    if (state != BUBBLE_LIVE) {
        if (state == BUBBLE_NONFINITE) {
            B.active[b] = 0;
            atomicOr(flag, 2);
        }
        B.spread[b] = 0;
        B.cell[b] = -1;
        return;
    }
    const int L[3] = {g.nx, g.ny, g.nz};
    F2 xb[3] = {in.x[0], in.x[1], in.x[2]};
    const BubbleK& K = in.k;
    const float inv_norm = 1.0f / w.norm;
    const float ul[3] = {acc[0] * inv_norm, acc[1] * inv_norm, acc[2] * inv_norm};
    // Interpolated vorticity (lift): curl from the difference sums.
    float om[3] = {0.0f, 0.0f, 0.0f};
    if (bc.lift) {
        om[0] = (acc[6] - acc[8]) * inv_norm;   // d(u_z)/dy - d(u_y)/dz
        om[1] = (acc[7] - acc[4]) * inv_norm;   // d(u_x)/dz - d(u_z)/dx
        om[2] = (acc[3] - acc[5]) * inv_norm;   // d(u_y)/dx - d(u_x)/dy
    }
    // C_A rho_l V_b D_t u_l (virtual mass, liquid part) plus, with the
    // stress-gradient force, rho_l V_b D_t u_l (F_S).
    float fvm[3] = {0.0f, 0.0f, 0.0f};
    if (in.has_prev) {
        for (int a = 0; a < 3; ++a)
            fvm[a] = (K.fvm_coef_dt + K.fs_coef_dt) * (ul[a] - in.ulprev[a]);
    }
    const F2 dt_b{bc.dt_bh, bc.dt_bl};
    const F2 r{K.rh, K.rl};
    F2 top[3];   // L - r
    for (int a = 0; a < 3; ++a) top[a] = f2_add(F2{(float)L[a], 0.0f}, -r.h, -r.l);
    const float sn_coeff = (float)bc.sn_coeff, sn_exp = (float)bc.sn_exp;
    const float fb[3] = {0.0f, 0.0f, K.fb};
    float u[3] = {in.u[0], in.u[1], in.u[2]};
    float fd_sum[3] = {0.0f, 0.0f, 0.0f};
    bool wrap_far = false;   // a periodic coordinate left [-L, 2L): folded through FP64 below
    for (int k = 0; k < bc.substeps; ++k) {
        const float v0 = u[0] - ul[0], v1 = u[1] - ul[1], v2 = u[2] - ul[2];
        const float speed = sqrtf(v0 * v0 + v1 * v1 + v2 * v2);
        const float re = speed * K.re_per_speed;
        // Re^b with the accurate powf (the adjoint replays the same value).
        const float visc_a = K.visc_a0 * (1.0f + sn_coeff * powf(re, sn_exp));
        const float cdv = fmaxf(fminf(visc_a, K.visc_b), K.eo_term * speed);   // C_D |v|
        const float kd = -K.drag_pref * cdv;
        float fd[3] = {kd * v0, kd * v1, kd * v2};
        if (bc.lift) {
            // F_L = -C_L rho_l V_b v x omega (Table 1), with the drag in the
            // reaction (Algorithm 1 step 6).
            const float cl = K.cl_tanh ? fminf(0.288f * tanhf(0.121f * re), K.cl_f) : K.cl_f;
            const float kl = -cl * K.lift_pref;
            fd[0] = fmaf(kl, v1 * om[2] - v2 * om[1], fd[0]);
            fd[1] = fmaf(kl, v2 * om[0] - v0 * om[2], fd[1]);
            fd[2] = fmaf(kl, v0 * om[1] - v1 * om[0], fd[2]);
        }
        for (int a = 0; a < 3; ++a) {
            fd_sum[a] += fd[a];
            u[a] = fmaf(fb[a] + fd[a] + fvm[a], K.kdt, u[a]);
            // x += u dt_b: the product as hi + lo (FMA error term), then TwoSum.
            const float ph = u[a] * dt_b.h;
            const float pl = fmaf(u[a], dt_b.h, -ph) + u[a] * dt_b.l;
            xb[a] = f2_add(xb[a], ph, pl);
            if (g.walls & (1u << (2 * a))) {
                if (f2_lt(xb[a], r)) {
                    xb[a] = r;
                    u[a] = fmaxf(u[a], 0.0f);
                }
                if (f2_lt(top[a], xb[a])) {
                    xb[a] = top[a];
                    u[a] = fminf(u[a], 0.0f);
                }
            } else {
                const float La = (float)L[a];
                if (f2_lt(xb[a], F2{0.0f, 0.0f})) xb[a] = f2_add(xb[a], La, 0.0f);
                else if (!f2_lt(xb[a], F2{La, 0.0f})) xb[a] = f2_add(xb[a], -La, 0.0f);
                if (!(xb[a].h >= 0.0f && xb[a].h <= La)) wrap_far = true;
            }
        }
    }
    if (wrap_far) {
        // Only reachable with runaway or non-finite velocities: fold in FP64.
        for (int a = 0; a < 3; ++a) {
            if (g.walls & (1u << (2 * a))) continue;
            double v = f2_to(xb[a]);
            v = __dsub_rn(v, __dmul_rn((double)L[a], floor(v / (double)L[a])));
            xb[a] = f2_from(v);
        }
    }
    // A bubble that moved more than GUARD_CELLS cells along an axis in one
    // step (lattice speed > 4) flags the instability.
    bool too_fast = false;
    for (int a = 0; a < 3; ++a) {
        float d = (xb[a].h - in.x[a].h) + (xb[a].l - in.x[a].l);
        if (!(g.walls & (1u << (2 * a)))) {
            const float La = (float)L[a];
            if (d > 0.5f * La) d -= La;
            else if (d < -0.5f * La) d += La;
        }
        too_fast |= !(fabsf(d) <= (float)GUARD_CELLS);
    }
    if (too_fast) atomicOr(flag, 4);
    // Reaction: -(F_D + F_L) averaged over the sub-steps (Algorithm 1 step
    // 6), or -sum F over the interphase forces (Sec. 3.2).  The latter adds
    // F_S and F_VM = C_A rho_l V_b (D_t u_l - a_k); with m_eff a_k = F_B +
    // F_D + F_L + F_S + C_A rho_l V_b D_t u_l its sub-step mean is
    // react_mb (mean F_D + F_L + fvm) - react_ca F_B, fvm = F_S + C_A rho_l
    // V_b D_t u_l.
    float psi[3];
    const float inv_sub = 1.0f / (float)bc.substeps;
    for (int a = 0; a < 3; ++a) {
        psi[a] = bc.reaction_all
                     ? K.react_ca * fb[a] - K.react_mb * fmaf(fd_sum[a], inv_sub, fvm[a])
                     : -fd_sum[a] * inv_sub;
        B.xh[3 * b + a] = xb[a].h;
        B.xl[3 * b + a] = xb[a].l;
        B.u[3 * b + a] = u[a];
        B.ul[3 * b + a] = ul[a];
        B.ulprev[3 * b + a] = ul[a];
        B.psi[3 * b + a] = psi[a];
    }
    B.has_prev[b] = 1;
    if (!(isfinite(xb[0].h) && isfinite(xb[1].h) && isfinite(xb[2].h) && isfinite(u[0]) &&
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
    for (int a = 0; a < 3; ++a) {
        float fr;
        ci[a] = min(max(f2_floor(xb[a], fr), 0), L[a] - 1);
    }
    B.cell[b] = (ci[2] * g.ny + ci[1]) * g.nx + ci[0];
    make_record(xb, K, g, psi, B.rec[b]);
    // Algorithm 1: the bubble stops once it reaches the top of the liquid.
    if ((g.walls & 0x20) && !f2_lt(xb[2], top[2])) B.active[b] = 0;
}

// Table 1 / Eq. 3 constants of a bubble of diameter d and window half-width n
// (FP64), with the closure parameters bc (nu: the bubble's column).
__device__ BubbleK bubble_constants(double d, double n, const BubbleConst& bc) {
    const double r = 0.5 * d;
    const double vol = M_PI * d * d * d / 6.0;
    const double eo = (bc.rho_l - bc.rho_b) * bc.g * d * d / bc.sigma;   // Eq. 3 with d^2
    BubbleK K;
    K.inv_nf = (float)(1.0 / n);
    K.r = r;
    split_f2(r, K.rh, K.rl);
    split_f2(n, K.nh, K.nl);
    K.kdt = (float)(bc.dt_b / ((bc.rho_b + bc.c_am * bc.rho_l) * vol));
    K.fb = (float)((bc.rho_l - bc.rho_b) * vol * bc.g);
    K.drag_pref = (float)(0.5 * bc.rho_l * M_PI * r * r * bc.drag_scale);
    K.fvm_coef_dt = (float)(bc.c_am * bc.rho_l * vol / bc.dt_l);
    K.visc_a0 = (float)(24.0 * bc.nu / d);
    K.visc_b = (float)(48.0 * bc.nu / d);
    K.re_per_speed = (float)(d / bc.nu);
    K.eo_term = (float)(8.0 / 3.0 * eo / (eo + 4.0));
    // Lift coefficient (Table 1): Eo_d = Eo / E^(2/3), E = 1 / (1 + 0.163
    // Eo^0.757); f(Eo_d) with the published constant 0.474.
    const double e = 1.0 / (1.0 + 0.163 * pow(eo, 0.757));
    const double eo_d = eo / pow(e, 2.0 / 3.0);
    const double fl = 0.00105 * eo_d * eo_d * eo_d - 0.0159 * eo_d * eo_d - 0.0204 * eo_d + 0.474;
    K.cl_tanh = eo_d < 4.0 ? 1 : 0;
    K.cl_f = (float)(eo_d <= 10.0 ? fl : -0.29);
    K.lift_pref = bc.lift ? (float)(bc.rho_l * vol) : 0.0f;
    K.fs_coef_dt = bc.stress ? (float)(bc.rho_l * vol / bc.dt_l) : 0.0f;
    K.hmap = (float)((bc.point ? -0.5 : 0.5) / n);
    const double meff_per_vol = bc.rho_b + bc.c_am * bc.rho_l;
    K.react_ca = (float)(bc.c_am * bc.rho_l / meff_per_vol);
    K.react_mb = (float)(bc.rho_b / meff_per_vol);
    return K;
}

__global__ void k_bubble_constants(BubbleDev B, BubbleConst bc) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B.nb) return;
    B.k[b] = bubble_constants(B.d[b], B.n[b], bc);
}

cudaError_t launch_bubble_constants(const BubbleDev& b, const BubbleConst& bc, cudaStream_t st) {
    if (b.nb == 0) return cudaSuccess;
    k_bubble_constants<<<(b.nb + 127) / 128, 128, 0, st>>>(b, bc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Binning (Algorithm 1 step 2): bubble windows -> tiles, deterministic lists
// ---------------------------------------------------------------------------

// Tiles of one axis holding at least one window cell, ascending.
// lo, hi: the first and last support cell, floor(x - n) and ceil(x + n) - 1.
__device__ int axis_tiles(int lo, int hi, int L, bool periodic, int T, int out[MAX_AXIS_TILES]) {
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
__global__ void k_bin(Geo g, BubbleDev B, Bins bins, const int* __restrict__ select) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B.nb || !select[b]) return;
    const int L[3] = {g.nx, g.ny, g.nz};
    const int T[3] = {TX, TY, TZ};
    if (B.x) {
        // FP64 centres and half-widths from the caller (binning without a
        // context) never passed lbm_set_bubbles' checks: a non-finite value,
        // a half-width outside (0, MAX_HALF_WIDTH] or a centre outside the
        // box skips the bubble and sets bit 2 of the status word.
        const double n = B.n[b];
        bool ok = isfinite(n) && n > 0.0 && n <= MAX_HALF_WIDTH;
        for (int a = 0; a < 3; ++a) {
            const double xa = B.x[3 * b + a];
            ok = ok && isfinite(xa) && xa >= 0.0 && xa < (double)L[a];
        }
        if (!ok) {
            atomicOr(bins.overflow, 2);
            return;
        }
    }
    int tl[3][MAX_AXIS_TILES];
    int nt[3];
    for (int a = 0; a < 3; ++a) {
        int lo, hi;
        if (B.x) {
            const double xa = B.x[3 * b + a], n = B.n[b];
            lo = (int)floor(xa - n);
            hi = (int)ceil(xa + n) - 1;
        } else {
            const BubbleK& K = B.k[b];
            support_cells(F2{B.xh[3 * b + a], B.xl[3 * b + a]}, K.nh, K.nl, lo, hi);
        }
        nt[a] = axis_tiles(lo, hi, L[a], !(g.walls & (1u << (2 * a))), T[a], tl[a]);
    }
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

cudaError_t launch_binning(const Geo& g, const BubbleDev& b, const Bins& bins, cudaStream_t st,
                           const int* select) {
    if (!select) select = b.spread;
    cudaError_t e = cudaMemsetAsync(bins.cnt, 0, sizeof(int) * (size_t)bins.T, st);
    if (e != cudaSuccess) return e;
    const int tb = 128;
    const int bb = (b.nb + tb - 1) / tb;
    if (b.nb > 0) k_bin<false><<<bb, tb, 0, st>>>(g, b, bins, select);
    k_scan_local<<<bins.nblocks, SCAN_BLOCK, 0, st>>>(bins.cnt, bins.off, bins.T, bins.block_sums);
    k_scan_sums<<<1, SCAN_BLOCK, 0, st>>>(bins.block_sums, bins.nblocks, bins.off, bins.T);
    k_scan_add<<<bins.nblocks, SCAN_BLOCK, 0, st>>>(bins.off, bins.T, bins.block_sums);
    e = cudaMemsetAsync(bins.cnt, 0, sizeof(int) * (size_t)bins.T, st);
    if (e != cudaSuccess) return e;
    if (b.nb > 0) k_bin<true><<<bb, tb, 0, st>>>(g, b, bins, select);
    k_bin_sort<<<(bins.T + 127) / 128, 128, 0, st>>>(bins);
    return cudaGetLastError();
}

// The per-tile counts of the previous binning back to zero (only the tiles it
// listed), so that the counts stay valid between calls without a sweep over
// all tiles.
__device__ void clear_prev_tiles(const SmallBins& sb) {
    // The first entries are read together with the count (one round trip);
    // prev_tiles holds SMALL_MAX_PAIRS entries, so the read is in bounds.
    const int first = (int)threadIdx.x < SMALL_MAX_PAIRS ? __ldcg(sb.prev_tiles + threadIdx.x) : -1;
    const int prev = min(max(__ldcg(sb.prev_n), 0), SMALL_MAX_PAIRS);
    if ((int)threadIdx.x < prev && first >= 0 && first < sb.T) sb.count[first] = 0;
    for (int i = threadIdx.x + blockDim.x; i < prev; i += blockDim.x) {
        const int t = __ldcg(sb.prev_tiles + i);
        if (t >= 0 && t < sb.T) sb.count[t] = 0;
    }
}

// Few pairs: one CTA enumerates every (tile, bubble) pair, sorts the keys
// (tile << 32 | bubble) with a bitonic network in shared memory and writes the
// runs.  The per-tile counts stay valid between calls because only the tiles
// the previous call touched are cleared first.  The bubble state is read with
// __ldcg: it was written by other CTAs of the same launch.
// With `cols` set (a batch), bubble b lives in column bubble_col[b], whose
// tiles are numbered from cols[c].tile_base in the shared tile space.
__device__ void bin_small_block(const Geo& g, const BubbleDev& B, const SmallBins& sb,
                                unsigned long long* keys, int* s_n, int pad,
                                const BatchColumn* cols = nullptr,
                                const int* bubble_col = nullptr) {
    const int tid = threadIdx.x, nt = blockDim.x;
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
        const float nh = __ldcg(&B.k[b].nh), nl = __ldcg(&B.k[b].nl);
        for (int a = 0; a < 3; ++a) {
            int lo, hi;
            support_cells(F2{__ldcg(B.xh + 3 * b + a), __ldcg(B.xl + 3 * b + a)}, nh, nl, lo, hi);
            ntl[a] = axis_tiles(lo - pad, hi + pad, L[a], !(gb.walls & (1u << (2 * a))), T[a],
                                tl[a]);
        }
        // One reservation per bubble; its pairs come out in ascending tile
        // order (each axis list is ascending).
        int k = atomicAdd(s_n, ntl[0] * ntl[1] * ntl[2]);
        for (int iz = 0; iz < ntl[2]; ++iz)
            for (int iy = 0; iy < ntl[1]; ++iy)
                for (int ix = 0; ix < ntl[0]; ++ix, ++k) {
                    const unsigned t = (unsigned)(base + (tl[2][iz] * gb.nty + tl[1][iy]) * gb.ntx +
                                                  tl[0][ix]);
                    if (k < SMALL_MAX_PAIRS) keys[k] = ((unsigned long long)t << 32) | (unsigned)b;
                    else atomicOr(sb.overflow, 1);
                }
    }
    __syncthreads();
    const int n = min(*s_n, SMALL_MAX_PAIRS);
    // Keys already in order (one bubble, or bubbles that happened to reserve
    // in order) skip the sort.
    int unsorted = 0;
    for (int i = tid + 1; i < n; i += nt) unsorted |= keys[i - 1] > keys[i];
    if (__syncthreads_or(unsorted)) {   // uniform over the CTA
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

__device__ __forceinline__ int floor_div(int a, int b) {
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

// Sweep order of the z blocks for the next step, written by one CTA (every
// thread calls it): the blocks whose tile layer is not marked in `lay` (bit
// l: layer l is guarded), ascending, then the guarded ones, ascending.  Each
// thread places a contiguous run of blocks; a block-wide scan of the cleared
// counts gives every run's first slot.
__device__ void write_zperm(int nbz, const unsigned* lay, int* __restrict__ zperm) {
    __shared__ int ws[33];
    const int tid = threadIdx.x, nt = blockDim.x;
    const int per = (nbz + nt - 1) / nt;
    const int b0 = min(tid * per, nbz), b1 = min(b0 + per, nbz);
    int cleared = 0;
    for (int bz = b0; bz < b1; ++bz) {
        const int l = (bz * SWEEP_PZ) / TZ;
        cleared += !((lay[l >> 5] >> (l & 31)) & 1u);
    }
    int total;
    const int before = block_exclusive_scan(cleared, ws, total);
    int sc = before, sg = total + (b0 - before);   // guarded blocks before b0: b0 - before
    for (int bz = b0; bz < b1; ++bz) {
        const int l = (bz * SWEEP_PZ) / TZ;
        if ((lay[l >> 5] >> (l & 31)) & 1u) zperm[sg++] = bz;
        else zperm[sc++] = bz;
    }
}

// The z tile layers the support of an active bubble, widened by GUARD_CELLS
// cells, reaches: bits of `lay` (atomicOr; shared or global memory).
__device__ __forceinline__ void mark_guarded_layers(const Geo& g, F2 z, float nh, float nl,
                                                    unsigned* lay) {
    const int ntz = g.ntz;
    const bool periodic = !(g.walls & 0x10);
    int lo, hi;
    support_cells(z, nh, nl, lo, hi);
    lo = max(lo, -2 * g.nz) - GUARD_CELLS;
    hi = min(hi, 3 * g.nz) + GUARD_CELLS;
    int l0, l1;
    if (!periodic) {
        lo = max(lo, 0);
        hi = min(hi, g.nz - 1);
        if (hi < lo) return;
        l0 = lo / TZ;
        l1 = hi / TZ;
    } else if (hi - lo + 1 >= g.nz) {
        l0 = 0;
        l1 = ntz - 1;
    } else {
        l0 = floor_div(lo, TZ);
        l1 = floor_div(hi, TZ);
    }
    for (int l = l0; l <= l1; ++l) {
        int lw = l % ntz;
        if (lw < 0) lw += ntz;
        atomicOr(&lay[lw >> 5], 1u << (lw & 31));
    }
}

// Overlap guard for the next step (single column): safe[l] = sb.safe_epoch
// for every z tile layer l that the support of no active bubble, widened by
// GUARD_CELLS cells, reaches.  Next step's forces lie inside those supports
// unless a bubble moves more than GUARD_CELLS cells, which flags the
// instability.  Every thread of the CTA calls it.
__device__ void write_safe_layers(const Geo& g, const BubbleDev& B, const SmallBins& sb) {
    __shared__ unsigned s_lay[GUARD_LAYERS_MAX / 32];
    __shared__ int s_zr[2];   // first and last guarded layer
    const int tid = threadIdx.x, nt = blockDim.x;
    const int ntz = g.ntz;
    if (ntz > GUARD_LAYERS_MAX) {
        // No tags kept: every layer counts as guarded.
        if (sb.zrange != nullptr && tid == 0) {
            sb.zrange[0] = 0;
            sb.zrange[1] = ntz - 1;
        }
        return;
    }
    for (int i = tid; i < GUARD_LAYERS_MAX / 32; i += nt) s_lay[i] = 0u;
    if (tid == 0) {
        s_zr[0] = INT_MAX;
        s_zr[1] = -1;
    }
    __syncthreads();
    for (int b = tid; b < B.nb; b += nt) {
        if (!__ldcg(B.active + b)) continue;
        mark_guarded_layers(g, F2{__ldcg(B.xh + 3 * b + 2), __ldcg(B.xl + 3 * b + 2)},
                            __ldcg(&B.k[b].nh), __ldcg(&B.k[b].nl), s_lay);
    }
    __syncthreads();
    for (int l = tid; l < ntz; l += nt) {
        if (!((s_lay[l >> 5] >> (l & 31)) & 1u)) {
            sb.safe[l] = sb.safe_epoch;
        } else {
            atomicMin(&s_zr[0], l);
            atomicMax(&s_zr[1], l);
        }
    }
    if (sb.zperm != nullptr) write_zperm(sb.nbz, s_lay, sb.zperm);
    __syncthreads();
    if (sb.zrange != nullptr && tid == 0) {
        sb.zrange[0] = s_zr[0];
        sb.zrange[1] = s_zr[1];
    }
}

// Bubble update with the few-pair binning fused behind it.
//
// The window of a bubble is cut into chunks of WINDOW_CHUNK nodes (node m of
// chunk k is m = k WINDOW_CHUNK + thread or + thread + BUBBLE_THREADS), and
// sb.parts CTAs share a bubble, CTA p taking chunks p, p + parts, ...  Each
// chunk is reduced in a fixed order and the chunk sums are added in chunk
// order, so the result does not depend on `parts`: a bubble gives the same
// bits in a column of its own and in a batch.  The CTA that completes a
// bubble's chunks (the last to arrive; nothing waits) integrates it; the CTA
// that completes the last bubble bins all bubbles.  CTA 0 first clears the
// previous binning's tile counts; that is ordered before the new binning by
// the same arrive / done counters.  With `cols` set (a batch), bubble b lives
// in column bubble_col[b].
//
// Launched to overlap with the sweep before it, the update first waits for
// that sweep (whose populations it reads and whose tile lists it rewrites),
// then lets the next sweep start: that sweep runs alongside the rest of the
// update and waits for it only in the z layers the guard does not clear.
// LIFT: the window carries the vorticity halo and nine sums (add_window_node).
template <int ST, bool LIFT>
__global__ void __launch_bounds__(BUBBLE_THREADS, 1)
k_bubbles_binned(const typename Store<ST>::T* __restrict__ f, Geo g, CollideParams cp,
                 BubbleDev B, BubbleConst bc, int* __restrict__ flag, SmallBins sb,
                 const BatchColumn* __restrict__ cols, const int* __restrict__ bubble_col) {
    constexpr int NV = win_vals(LIFT);
    __shared__ float red[NV][BUBBLE_THREADS / 32];
    __shared__ unsigned long long keys[SMALL_MAX_PAIRS];
    __shared__ int s_n, s_last;
    const int parts = sb.parts;
    const int b = blockIdx.x / parts, p = blockIdx.x - b * parts;
    const bool alone = gridDim.x == 1;   // one bubble, one CTA: nothing to publish
    pdl_wait();
    pdl_trigger();
    BubbleIn in;
    load_bubble(B, b, threadIdx.x == 0, in);
    if (blockIdx.x == 0) {
        clear_prev_tiles(sb);
        if (!alone) __threadfence();
    }
    if (cols) {
        const BatchColumn& col = cols[bubble_col[b]];
        f += col.pop_offset;
        g = col.g;
        cp = col.cp;
    }
    Window w;
    const int state = bubble_window(g, in, w, LIFT ? 1 : 0);
    const int nchunks = state == BUBBLE_LIVE ? (w.M + WINDOW_CHUNK - 1) / WINDOW_CHUNK : 0;
    const float inv_n = in.k.inv_nf;
    float sum[NV];   // thread 0: running sum over this CTA's chunks
#pragma unroll
    for (int q = 0; q < NV; ++q) sum[q] = 0.0f;
    for (int k = p; k < nchunks; k += parts) {
        float acc[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) acc[q] = 0.0f;
        const int m0 = k * WINDOW_CHUNK;
        chunk_sum2<ST, LIFT>(f, g, cp, w, inv_n, m0, min(m0 + WINDOW_CHUNK, w.M), threadIdx.x,
                             BUBBLE_THREADS, acc);
        block_sum_n<NV>(acc, red);
        if (threadIdx.x == 0) {
            if (parts == 1) {
#pragma unroll
                for (int q = 0; q < NV; ++q) sum[q] += acc[q];
            } else {
                float* slot = sb.part + WIN_VALS_LIFT * ((size_t)b * WINDOW_CHUNKS_MAX + k);
#pragma unroll
                for (int q = 0; q < NV; ++q) slot[q] = acc[q];
            }
        }
        __syncthreads();   // `red` is reused by the next chunk
    }
    __syncthreads();       // CTA 0's clearing is complete before thread 0 arrives
    if (threadIdx.x == 0) {
        bool mine = true;
        if (parts > 1) {
            __threadfence();                                 // publish this CTA's chunk sums
            mine = atomicAdd(sb.arrive + b, 1) == parts - 1;
            if (mine) {
                __threadfence();
                const float* q = sb.part + WIN_VALS_LIFT * (size_t)b * WINDOW_CHUNKS_MAX;
                for (int k = 0; k < nchunks; ++k)
#pragma unroll
                    for (int v = 0; v < NV; ++v) sum[v] += __ldcg(q + WIN_VALS_LIFT * k + v);
                sb.arrive[b] = 0;                            // ready for the next launch
            }
        }
        s_last = 0;
        if (mine) {
            bubble_tail(g, B, bc, flag, b, state, w, sum, in);
            if (alone) {
                s_last = 1;
            } else {
                __threadfence();                             // publish this bubble's state
                s_last = atomicAdd(sb.done, 1) == B.nb - 1;
            }
        }
    }
    __syncthreads();
    if (!s_last) return;
    if (!alone) __threadfence();
    bin_small_block(g, B, sb, keys, &s_n, LIFT ? 1 : 0, cols, bubble_col);
    if (sb.safe != nullptr && cols == nullptr) write_safe_layers(g, B, sb);
    if (threadIdx.x == 0 && !alone) *sb.done = 0;        // ready for the next launch
}

int window_parts(double max_half_width, int pad) {
    const int cells =
        std::min((int)std::ceil(2.0 * max_half_width) + 1 + 2 * pad, WINDOW_CELLS_MAX);
    const int nodes = cells * cells * cells;
    return std::max(1, std::min((nodes + WINDOW_CHUNK - 1) / WINDOW_CHUNK, WINDOW_CHUNKS_MAX));
}

namespace {
template <int ST>
cudaError_t launch_binned(const void* f, const Geo& g, const CollideParams& cp,
                          const BubbleDev& b, const BubbleConst& bc, int* flag,
                          const SmallBins& sb, const BatchColumn* cols, const int* bubble_col,
                          bool overlap, cudaStream_t st) {
    using T = typename Store<ST>::T;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b.nb * sb.parts);
    cfg.blockDim = dim3(BUBBLE_THREADS);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = overlap ? 1 : 0;
    if (bc.lift)
        return cudaLaunchKernelEx(&cfg, k_bubbles_binned<ST, true>, (const T*)f, g, cp, b, bc,
                                  flag, sb, cols, bubble_col);
    return cudaLaunchKernelEx(&cfg, k_bubbles_binned<ST, false>, (const T*)f, g, cp, b, bc, flag,
                              sb, cols, bubble_col);
}
}  // namespace

cudaError_t launch_bubbles(int storage, const void* f, const Geo& g, const CollideParams& cp,
                           const BubbleDev& b, const BubbleConst& bc, int* flag,
                           const SmallBins& sb, bool overlap, cudaStream_t st) {
    if (b.nb == 0) return cudaSuccess;
    if (sb.parts < 1 || sb.parts > WINDOW_CHUNKS_MAX) return cudaErrorInvalidValue;
    switch (storage) {
        case 0: return launch_binned<0>(f, g, cp, b, bc, flag, sb, nullptr, nullptr, overlap, st);
        case 1: return launch_binned<1>(f, g, cp, b, bc, flag, sb, nullptr, nullptr, overlap, st);
        default: return launch_binned<2>(f, g, cp, b, bc, flag, sb, nullptr, nullptr, overlap, st);
    }
}

cudaError_t launch_bubbles_batch(int storage, const void* f, const BatchColumn* cols,
                                 const int* bubble_col, const BubbleDev& b, const BubbleConst& bc,
                                 int* flag, const SmallBins& sb, cudaStream_t st) {
    if (b.nb == 0) return cudaSuccess;
    if (sb.parts < 1 || sb.parts > WINDOW_CHUNKS_MAX) return cudaErrorInvalidValue;
    // Geometry and relaxation come from each bubble's column.
    const Geo g0{};
    const CollideParams cp0{};
    switch (storage) {
        case 0: return launch_binned<0>(f, g0, cp0, b, bc, flag, sb, cols, bubble_col, false, st);
        case 1: return launch_binned<1>(f, g0, cp0, b, bc, flag, sb, cols, bubble_col, false, st);
        default: return launch_binned<2>(f, g0, cp0, b, bc, flag, sb, cols, bubble_col, false, st);
    }
}

// ---------------------------------------------------------------------------
// Many bubbles: interpolation by tiles, update per bubble, binning in one
// persistent launch
// ---------------------------------------------------------------------------
// The window sum of Eq. 20 splits over the lattice tiles a bubble's window
// touches.  The binning of the current centres lists, per tile, the bubbles
// whose windows touch it; k_tile_interp forms per tile the Eq. 10 velocity of
// its 512 nodes once, in shared memory, and for each listed bubble the part
// of its sum over the tile (a separable tensor product: x-rows first, then the
// y and z weights).  k_swarm_tail adds a bubble's parts in the order of its
// tiles (ascending) and runs the update; k_swarm_bin bins the updated
// bubbles and records, for every bubble and tile, the list position of the
// pair, where the next step's parts are written and read.  All sums run in a
// fixed order, so the results do not depend on scheduling.

constexpr int INTERP_THREADS = TX * TY * 2;   // two of a tile's TZ planes per thread
constexpr int INTERP_CHUNK = 32;              // listed bubbles per pass
constexpr int INTERP_ROWS = TY * TZ;          // (y, z) rows of a tile: 16
static_assert(INTERP_THREADS % INTERP_ROWS == 0 && TZ == 4, "tile shape of the interpolation");
// Resident CTAs per SM the interpolation is compiled for: 16-bit storage on
// even rows at 5 (48 registers; its swarm step ran 1 % shorter than at 4, at
// 6 longer); FP32 at 4 (at 5 it spills 96 bytes and its step was longer), as
// odd rows (whose two-node gather spills 172 bytes at 48 registers).
template <int ST, bool PAIR> struct InterpOccupancy {
    static constexpr int kMinBlocks = (ST != 0 && PAIR) ? 5 : 4;
};

// The list head of a covered tile: its list range [beg, end) and this
// thread's entry of the first chunk (-1 beyond it).  The interpolation loads
// a tile's head one tile ahead: the chain cover -> count and offset -> entry
// is three dependent loads.
struct TileHead {
    int t, beg, end, id;
};

// One covered tile h.t: the Eq. 10 velocity of its nodes, then for each listed
// bubble the part of its Eq. 20 sum over the tile, written at the bubble's
// list position.  Every thread of the CTA calls it.  Once the first chunk's
// tables are made, the next tile's first list entry is loaded into next.id
// (next.beg and next.end were loaded a tile before).
template <int ST, bool PAIR, bool LIFT>
__device__ __forceinline__ void tile_interp(const typename Store<ST>::T* __restrict__ f,
                                            const Geo& g, const CollideParams& cp,
                                            const TileHead& h, TileHead& next,
                                            const int* __restrict__ items,
                                            const BubbleRec* __restrict__ recs, int nb,
                                            float* __restrict__ partial) {
    const int t = h.t;
    constexpr int NAX = TX + TY + TZ;
    __shared__ float s_u[3][INTERP_ROWS][TX + 1];   // node velocities by (z, y) row, padded
    __shared__ float s_w[INTERP_CHUNK][NAX];         // per-axis cell integrals per bubble
    __shared__ BubbleRec s_rec[INTERP_CHUNK];
    __shared__ int s_xlo[INTERP_CHUNK], s_xhi[INTERP_CHUNK];   // non-zero x weights
    __shared__ float s_d[LIFT ? INTERP_CHUNK : 1][NAX];          // lift: difference weights
    const int tid = threadIdx.x;
    const int bx = t % g.ntx, by = (t / g.ntx) % g.nty, bz = t / (g.ntx * g.nty);
    const int xb0 = bx * TX, yb0 = by * TY, zb0 = bz * TZ;
    // The population loads go out first; the list and the first chunk's
    // records (a chain of dependent loads) are fetched while they are in
    // flight.  PAIR (even nx): thread (px, y, z) gathers the x-pair
    // (2 px, 2 px + 1) of row (y, z) with aligned 2-wide row loads; else
    // thread (x, y, zp) gathers nodes (x, y, zp) and (x, y, zp + 2).
    const int tx = tid % TX, ty = (tid / TX) % TY, zp = tid / (TX * TY);
    const int x = xb0 + tx, y = yb0 + ty, za = zb0 + zp, zb = zb0 + zp + 2;
    const bool inxy = x < g.nx && y < g.ny;
    const bool ina = inxy && za < g.nz, inb = inxy && zb < g.nz;
    const int ppx = tid % (TX / 2), py2 = (tid / (TX / 2)) % TY, pz2 = tid / ((TX / 2) * TY);
    const int px0 = xb0 + 2 * ppx, pyy = yb0 + py2, pzz = zb0 + pz2;
    const bool inp = px0 < g.nx && pyy < g.ny && pzz < g.nz;
    typename Store<ST>::T ra[PAIR ? 1 : Q], rb[PAIR ? 1 : Q];
    typename Raw2<ST>::T rp[PAIR ? Q : 1];
    if (PAIR) {
        gather_pair<ST>(f, g, inp ? px0 : 0, inp ? pyy : 0, inp ? pzz : 0, rp);
    } else {
        gather_issue<ST>(f, g, ina ? x : 0, ina ? y : 0, ina ? za : 0, ra);
        gather_issue<ST>(f, g, inb ? x : 0, inb ? y : 0, inb ? zb : 0, rb);
    }
    const int beg = h.beg, end = h.end;
    BubbleRec rec0{0, 0, 0, 0, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (h.id >= 0 && h.id < nb) rec0 = load_rec(recs + h.id);
    if (PAIR) {
        // Eq. 10 velocity of the pair (zero for nodes beyond the box).
        float2 drho, jx, jy, jz;
        pair_moments<ST>(rp, cp, drho, jx, jy, jz);
        const float ra0 = 1.0f / (cp.rho0 + drho.x), ra1 = 1.0f / (cp.rho0 + drho.y);
        const int row = pz2 * TY + py2;
        s_u[0][row][2 * ppx] = inp ? jx.x * ra0 : 0.0f;
        s_u[0][row][2 * ppx + 1] = inp ? jx.y * ra1 : 0.0f;
        s_u[1][row][2 * ppx] = inp ? jy.x * ra0 : 0.0f;
        s_u[1][row][2 * ppx + 1] = inp ? jy.y * ra1 : 0.0f;
        s_u[2][row][2 * ppx] = inp ? jz.x * ra0 : 0.0f;
        s_u[2][row][2 * ppx + 1] = inp ? jz.y * ra1 : 0.0f;
    } else {
        // Eq. 10 velocity of the tile's nodes (zero for nodes beyond the box).
        float gv[Q], u[3];
        gather_finish<ST>(ra, cp, gv);
        node_velocity(gv, cp, u);
        for (int c = 0; c < 3; ++c) s_u[c][zp * TY + ty][tx] = ina ? u[c] : 0.0f;
        gather_finish<ST>(rb, cp, gv);
        node_velocity(gv, cp, u);
        for (int c = 0; c < 3; ++c) s_u[c][(zp + 2) * TY + ty][tx] = inb ? u[c] : 0.0f;
    }
    const bool px = !(g.walls & 0x01), py = !(g.walls & 0x04), pz = !(g.walls & 0x10);
    for (int c0 = beg; c0 < end; c0 += INTERP_CHUNK) {
        const int cntc = min(INTERP_CHUNK, end - c0);
        __syncthreads();
        if (tid < cntc) {
            if (c0 == beg) {
                s_rec[tid] = rec0;
            } else {
                const int id = __ldcg(items + c0 + tid);
                if (id >= 0 && id < nb) s_rec[tid] = load_rec(recs + id);
                else s_rec[tid] = BubbleRec{0, 0, 0, 0, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            }
            s_xlo[tid] = TX;
            s_xhi[tid] = -1;
        }
        __syncthreads();
        // The mapping mode is the same for every bubble: one loop per mode.
        auto tabulate = [&](auto mode) {
            constexpr int PM = decltype(mode)::value;
            for (int e = tid; e < cntc * NAX; e += INTERP_THREADS) {
                const int k = e / NAX, q = e - k * NAX;
                const BubbleRec& r = s_rec[k];
                if (LIFT) {
                    float w, dw;
                    if (q < TX)
                        axis_wd<PM>(xb0 + q, r.ax, r.fx, r.inv_n, r.h, g.nx, px, false, w, dw);
                    else if (q < TX + TY)
                        axis_wd<PM>(yb0 + q - TX, r.ay, r.fy, r.inv_n, r.h, g.ny, py, false, w, dw);
                    else
                        axis_wd<PM>(zb0 + q - TX - TY, r.az, r.fz, r.inv_n, r.h, g.nz, pz,
                                    (g.walls & WALL_TOP_FREE) != 0, w, dw);
                    s_w[k][q] = w;
                    s_d[k][q] = dw;
                    if (q < TX && (w != 0.0f || dw != 0.0f)) {
                        atomicMin(&s_xlo[k], q);
                        atomicMax(&s_xhi[k], q);
                    }
                } else if (q < TX) {
                    const float w = axis_weight<PM>(r, xb0 + q, r.ax, r.fx, g.nx, px);
                    s_w[k][q] = w;
                    if (w != 0.0f) {
                        atomicMin(&s_xlo[k], q);
                        atomicMax(&s_xhi[k], q);
                    }
                } else if (q < TX + TY) {
                    s_w[k][q] = axis_weight<PM>(r, yb0 + q - TX, r.ay, r.fy, g.ny, py);
                } else {
                    s_w[k][q] = axis_weight<PM>(r, zb0 + q - TX - TY, r.az, r.fz, g.nz, pz);
                }
            }
        };
        if (cp.point) tabulate(MapMode<MAP_POINT>{});
        else tabulate(MapMode<MAP_CELL>{});
        __syncthreads();
        if (c0 == beg && tid < min(INTERP_CHUNK, next.end - next.beg))
            next.id = __ldcg(items + next.beg + tid);
        // INTERP_ROWS threads per bubble, one (z, y) row each; the row sums
        // are added over the rows by shuffles (fixed order).
        for (int k0 = 0; k0 < cntc; k0 += INTERP_THREADS / INTERP_ROWS) {
            const int k = k0 + tid / INTERP_ROWS, row = tid % INTERP_ROWS;
            constexpr int NV = win_vals(LIFT);
            float v[NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) v[q] = 0.0f;
            if (k < cntc) {
                const float wy = s_w[k][TX + row % TY], wz = s_w[k][TX + TY + row / TY];
                const float dy = LIFT ? s_d[k][TX + row % TY] : 0.0f;
                const float dz = LIFT ? s_d[k][TX + TY + row / TY] : 0.0f;
                const float wyz = wy * wz;
                if (wyz != 0.0f || (LIFT && (dy * wz != 0.0f || wy * dz != 0.0f))) {
                    // Only the x columns with a non-zero weight: zero terms
                    // add nothing.  Row sums sum_x w_x u (and, with lift,
                    // sum_x d_x u_y and sum_x d_x u_z).
                    float ax = 0.0f, ay = 0.0f, az = 0.0f, bxy = 0.0f, bxz = 0.0f;
                    const int xe = s_xhi[k];
                    for (int x = s_xlo[k]; x <= xe; ++x) {
                        const float wx = s_w[k][x];
                        ax = fmaf(wx, s_u[0][row][x], ax);
                        ay = fmaf(wx, s_u[1][row][x], ay);
                        az = fmaf(wx, s_u[2][row][x], az);
                        if (LIFT) {
                            const float dx = s_d[k][x];
                            bxy = fmaf(dx, s_u[1][row][x], bxy);
                            bxz = fmaf(dx, s_u[2][row][x], bxz);
                        }
                    }
                    v[0] = ax * wyz;
                    v[1] = ay * wyz;
                    v[2] = az * wyz;
                    if (LIFT) {
                        // Gx u_y, Gx u_z, Gy u_x, Gy u_z, Gz u_x, Gz u_y
                        v[3] = bxy * wyz;
                        v[4] = bxz * wyz;
                        v[5] = ax * (dy * wz);
                        v[6] = az * (dy * wz);
                        v[7] = ax * (wy * dz);
                        v[8] = ay * (wy * dz);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < NV; ++q)
#pragma unroll
                for (int o = INTERP_ROWS / 2; o > 0; o >>= 1)
                    v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
            if (row == 0 && k < cntc) {
                float* q = partial + WIN_VALS_LIFT * (size_t)(c0 + k);
#pragma unroll
                for (int i = 0; i < NV; ++i) q[i] = v[i];
            }
        }
    }
}

// Persistent over the list of covered tiles, a tile per CTA in turn.
template <int ST, bool PAIR, bool LIFT>
__global__ void __launch_bounds__(INTERP_THREADS, InterpOccupancy<ST, PAIR>::kMinBlocks)
k_tile_interp(const typename Store<ST>::T* __restrict__ f, Geo g, CollideParams cp,
              const int* __restrict__ cnt, const int* __restrict__ off,
              const int* __restrict__ items, int cap, const BubbleRec* __restrict__ recs, int nb,
              const int* __restrict__ cover, const int* __restrict__ ncover,
              float* __restrict__ partial) {
    const int ntiles = __ldcg(ncover);
    const int step = (int)gridDim.x;
    int i = (int)blockIdx.x;
    if (i >= ntiles) return;
    // The head of the CTA's first tile, and the index of the one after it.
    auto head = [&](int t) {
        TileHead h{t, 0, 0, -1};
        if (t >= 0) {
            h.beg = __ldcg(off + t);
            h.end = min(h.beg + __ldcg(cnt + t), cap);
        }
        return h;
    };
    TileHead h = head(__ldcg(cover + i));
    if (threadIdx.x < min(INTERP_CHUNK, h.end - h.beg)) h.id = __ldcg(items + h.beg + threadIdx.x);
    int tn = i + step < ntiles ? __ldcg(cover + i + step) : -1;
    for (; i < ntiles; i += step) {
        // The next tile's count and offset go out now; its first list entry
        // during this tile; the index of the tile after it.
        TileHead next = head(tn);
        const int tnn = i + 2 * step < ntiles ? __ldcg(cover + i + 2 * step) : -1;
        __syncthreads();   // the shared tables of the previous tile are done with
        tile_interp<ST, PAIR, LIFT>(f, g, cp, h, next, items, recs, nb, partial);
        h = next;
        tn = tnn;
    }
}

// The update, a thread per bubble: its Eq. 20 sum is the parts of its tiles
// added in tile order.  The tile counts and the list of covered tiles start
// again for the binning after it.
constexpr int TAIL_THREADS = 128;

__global__ void __launch_bounds__(TAIL_THREADS)
k_swarm_tail(Geo g, BubbleDev B, BubbleConst bc, int* __restrict__ flag, Bins bins,
             SwarmBins sw) {
    const int tid = threadIdx.x;
    const int gtid = blockIdx.x * TAIL_THREADS + tid, nthreads = gridDim.x * TAIL_THREADS;
    for (int t = gtid; t < bins.T; t += nthreads) bins.cnt[t] = 0;
    if (gtid == 0) {
        *sw.ncover = 0;
        if (sw.zrange) {
            sw.zrange[0] = INT_MAX;
            sw.zrange[1] = -1;
        }
    }
    const int b = gtid;
    if (b < B.nb) {
        BubbleIn in;
        load_bubble(B, b, true, in);
        Window w;
        const int state = bubble_window(g, in, w);
        const int nv = win_vals(bc.lift != 0);
        float acc[WIN_VALS_LIFT];
        for (int q = 0; q < WIN_VALS_LIFT; ++q) acc[q] = 0.0f;
        if (state == BUBBLE_LIVE) {
            const int n = min(__ldcg(sw.ntile + b), sw.per);
            const int* sl = sw.slots + (size_t)b * sw.per;
            for (int k = 0; k < n; ++k) {
                const int p = __ldcg(sl + k);
                if (p < 0 || p >= bins.cap) continue;
                const float* q = sw.partial + WIN_VALS_LIFT * (size_t)p;
                for (int v = 0; v < nv; ++v) acc[v] += __ldcg(q + v);
            }
        }
        bubble_tail(g, B, bc, flag, b, state, w, acc, in);
    }
}

// Binning of the updated bubbles in one persistent launch, phases separated
// by grid barriers (all its CTAs are resident):
//   1. count: every selected bubble adds itself to the tiles its window
//      touches (Algorithm 1 step 2);
//   2. scan of the counts (per-CTA chunk totals, then offsets), and the list
//      of covered tiles;
//   3. fill: each bubble takes slots through per-tile cursors, noting which
//      of its tiles each is;
//   4. each tile's list ordered by bubble id (a warp per tile: an id's rank
//      is the number of smaller ids in the list), and the list positions
//      recorded per bubble.
// The counts, offsets and lists are those of launch_binning.  Everything
// written earlier in the launch is read through L2 (ld.global.cg).
constexpr int SWARM_THREADS = 256;
constexpr int SWARM_WARPS = SWARM_THREADS / 32;
constexpr int SWARM_SORT_MAX = 128;   // longer tile lists are ordered by one thread
// A grid barrier that waits longer than this (a CTA that never arrives) gives
// up: flag bit 8, and the launch ends.
constexpr unsigned long long SWARM_WAIT_NS = 1000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier over the launch's CTAs (bar[0] arrivals, bar[1] generation).
// The last CTA to arrive resets the arrivals before it advances the
// generation, so the counter is zero again for the next barrier and launch.
// Returns false (in every thread of the CTA) if the wait ran out.
__device__ bool grid_barrier(unsigned* bar, int* flag) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* vbar = bar;
        const unsigned gen = vbar[1];
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (vbar[1] == gen) {
                __nanosleep(64);
                if (global_ns() - t0 > SWARM_WAIT_NS) {
                    atomicOr(flag, 8);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Sum over the CTA (fixed order), returned in every thread.
__device__ __forceinline__ int block_sum_int(int v, int* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    int t = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    __syncthreads();
    return t;
}

// The tiles bubble b's window touches, per axis (ascending), as k_bin finds
// them; returns false for a bubble that is not selected.
__device__ __forceinline__ bool bubble_tiles(const Geo& g, const BubbleDev& B, const int* select,
                                             int pad, int b, int tl[3][MAX_AXIS_TILES],
                                             int nt[3]) {
    if (!__ldcg(select + b)) return false;
    const int L[3] = {g.nx, g.ny, g.nz};
    const int T[3] = {TX, TY, TZ};
    const float nh = B.k[b].nh, nl = B.k[b].nl;
    for (int a = 0; a < 3; ++a) {
        int lo, hi;
        support_cells(F2{__ldcg(B.xh + 3 * b + a), __ldcg(B.xl + 3 * b + a)}, nh, nl, lo, hi);
        nt[a] = axis_tiles(lo - pad, hi + pad, L[a], !(g.walls & (1u << (2 * a))), T[a], tl[a]);
    }
    return true;
}

__global__ void __launch_bounds__(SWARM_THREADS)
k_swarm_bin(Geo g, BubbleDev B, Bins bins, SwarmBins sw, const int* __restrict__ select,
            int* __restrict__ flag) {
    __shared__ int s_red[SWARM_WARPS];
    __shared__ int s_id[SWARM_WARPS][SWARM_SORT_MAX];
    __shared__ int s_k[SWARM_WARPS][SWARM_SORT_MAX];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nthreads = gridDim.x * SWARM_THREADS;
    const int gtid = blockIdx.x * SWARM_THREADS + tid;
    const int T = bins.T;

    // 1. Count; and the z tile layers the lists reach (for the next steps'
    // split of the sweep).
    int zlo = INT_MAX, zhi = -1;
    for (int b = gtid; b < B.nb; b += nthreads) {
        int tl[3][MAX_AXIS_TILES], nt[3];
        int n = 0;
        if (bubble_tiles(g, B, select, sw.pad, b, tl, nt)) {
            for (int iz = 0; iz < nt[2]; ++iz) {
                zlo = min(zlo, tl[2][iz]);
                zhi = max(zhi, tl[2][iz]);
                for (int iy = 0; iy < nt[1]; ++iy)
                    for (int ix = 0; ix < nt[0]; ++ix)
                        atomicAdd(&bins.cnt[(tl[2][iz] * g.nty + tl[1][iy]) * g.ntx + tl[0][ix]], 1);
            }
            n = nt[0] * nt[1] * nt[2];
        }
        sw.ntile[b] = n;
    }
    if (sw.zrange) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            zlo = min(zlo, __shfl_xor_sync(0xffffffffu, zlo, o));
            zhi = max(zhi, __shfl_xor_sync(0xffffffffu, zhi, o));
        }
        if (lane == 0 && zhi >= 0) {
            atomicMin(sw.zrange, zlo);
            atomicMax(sw.zrange + 1, zhi);
        }
    }
    if (!grid_barrier(sw.bar, flag)) return;

    // 2. Scan, chunk totals.
    const int chunk = (T + gridDim.x - 1) / gridDim.x;
    const int c0 = min(blockIdx.x * chunk, T), c1 = min(c0 + chunk, T);
    int part = 0;
    for (int t = c0 + tid; t < c1; t += SWARM_THREADS) part += __ldcg(bins.cnt + t);
    part = block_sum_int(part, s_red);
    if (tid == 0) sw.chunk_sums[blockIdx.x] = part;
    if (!grid_barrier(sw.bar, flag)) return;

    // Scan, offsets (and the fill cursors).
    int prefix = 0;
    for (int c = tid; c < (int)blockIdx.x; c += SWARM_THREADS) prefix += __ldcg(sw.chunk_sums + c);
    prefix = block_sum_int(prefix, s_red);
    {
        __shared__ int ws[33];
        int carry = prefix;
        for (int base = c0; base < c1; base += SWARM_THREADS) {
            const int t = base + tid;
            const int v = t < c1 ? __ldcg(bins.cnt + t) : 0;
            int total;
            const int ex = block_exclusive_scan(v, ws, total);
            if (t < c1) {
                bins.off[t] = carry + ex;
                sw.cursor[t] = carry + ex;
            }
            // The tiles with a non-empty list, appended a warp at a time.
            const unsigned m = __ballot_sync(0xffffffffu, v > 0);
            if (m) {
                int at = 0;
                if (lane == 0) at = atomicAdd(sw.ncover, __popc(m));
                at = __shfl_sync(0xffffffffu, at, 0);
                if (v > 0) sw.cover[at + __popc(m & ((1u << lane) - 1u))] = t;
            }
            carry += total;
        }
        if (c1 == T && c0 < c1 && tid == 0) bins.off[T] = carry;
    }
    if (!grid_barrier(sw.bar, flag)) return;

    // 3. Fill.
    for (int b = gtid; b < B.nb; b += nthreads) {
        int tl[3][MAX_AXIS_TILES], nt[3];
        if (!bubble_tiles(g, B, select, sw.pad, b, tl, nt)) continue;
        int k = 0;
        for (int iz = 0; iz < nt[2]; ++iz)
            for (int iy = 0; iy < nt[1]; ++iy)
                for (int ix = 0; ix < nt[0]; ++ix, ++k) {
                    const int t = (tl[2][iz] * g.nty + tl[1][iy]) * g.ntx + tl[0][ix];
                    const int at = atomicAdd(&sw.cursor[t], 1);
                    if (at < bins.cap) {
                        bins.items[at] = b;
                        sw.kidx[at] = k;
                    } else {
                        atomicOr(bins.overflow, 1);
                    }
                }
    }
    if (!grid_barrier(sw.bar, flag)) return;

    // 4. Each tile's list in bubble order, and each bubble's list positions.
    // A bubble is listed at most once per tile, so the ids of a list are
    // distinct and their ranks are the positions.
    int* ids = s_id[warp];
    int* ks = s_k[warp];
    for (int t = blockIdx.x * SWARM_WARPS + warp; t < T; t += gridDim.x * SWARM_WARPS) {
        const int n = __ldcg(bins.cnt + t);
        if (n == 0) continue;   // uniform over the warp
        const int beg = __ldcg(bins.off + t);
        const int end = min(beg + n, bins.cap);
        const int m = end - beg;
        if (m <= SWARM_SORT_MAX) {
            for (int i = lane; i < m; i += 32) {
                ids[i] = __ldcg(bins.items + beg + i);
                ks[i] = __ldcg(sw.kidx + beg + i);
            }
            __syncwarp();
            for (int i = lane; i < m; i += 32) {
                const int v = ids[i];
                int rank = 0;
                for (int j = 0; j < m; ++j) rank += ids[j] < v;
                bins.items[beg + rank] = v;
                sw.slots[(size_t)v * sw.per + min(ks[i], sw.per - 1)] = beg + rank;
            }
            __syncwarp();
        } else if (lane == 0) {
            for (int i = beg + 1; i < end; ++i) {
                const int v = __ldcg(bins.items + i), kv = __ldcg(sw.kidx + i);
                int j = i - 1;
                while (j >= beg) {
                    const int w = __ldcg(bins.items + j);
                    if (w <= v) break;
                    bins.items[j + 1] = w;
                    sw.kidx[j + 1] = __ldcg(sw.kidx + j);
                    --j;
                }
                bins.items[j + 1] = v;
                sw.kidx[j + 1] = kv;
            }
            for (int i = beg; i < end; ++i) {
                const int v = __ldcg(bins.items + i);
                sw.slots[(size_t)v * sw.per + min(__ldcg(sw.kidx + i), sw.per - 1)] = i;
            }
        }
        __syncwarp();
    }
}

// Spreading records of the current centres (with the current reaction).
__global__ void k_bubble_records(Geo g, BubbleDev B) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B.nb) return;
    const F2 xb[3] = {F2{B.xh[3 * b], B.xl[3 * b]}, F2{B.xh[3 * b + 1], B.xl[3 * b + 1]},
                      F2{B.xh[3 * b + 2], B.xl[3 * b + 2]}};
    const float psi[3] = {B.psi[3 * b], B.psi[3 * b + 1], B.psi[3 * b + 2]};
    make_record(xb, B.k[b], g, psi, B.rec[b]);
}

cudaError_t launch_bubble_records(const Geo& g, const BubbleDev& b, cudaStream_t st) {
    if (b.nb == 0) return cudaSuccess;
    k_bubble_records<<<(b.nb + 127) / 128, 128, 0, st>>>(g, b);
    return cudaGetLastError();
}

int swarm_grid(int /*storage*/) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_swarm_bin, SWARM_THREADS, 0) !=
            cudaSuccess || per < 1)
        return 0;
    return sms * std::min(per, LBM_SWARM_CTAS_PER_SM);
}

int interp_grid(int storage) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    cudaError_t e;
    switch (storage) {
        case 0: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tile_interp<0, true, true>, INTERP_THREADS, 0); break;
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tile_interp<1, true, true>, INTERP_THREADS, 0); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_tile_interp<2, true, true>, INTERP_THREADS, 0); break;
    }
    if (e != cudaSuccess || per < 1) return 0;
    return sms * per;
}

namespace {
template <int ST, bool PAIR, bool LIFT>
cudaError_t launch_interp_as(const void* f, const Geo& g, const CollideParams& cp,
                             const Bins& bins, const BubbleDev& b, const SwarmBins& sw,
                             cudaStream_t st) {
    using T = typename Store<ST>::T;
    k_tile_interp<ST, PAIR, LIFT><<<sw.interp_grid, INTERP_THREADS, 0, st>>>(
        (const T*)f, g, cp, bins.cnt, bins.off, bins.items, bins.cap, b.rec, b.nb, sw.cover,
        sw.ncover, sw.partial);
    return cudaGetLastError();
}

// Two-node gathers with aligned row loads on even rows; the vorticity sums
// with lift.
template <int ST>
cudaError_t launch_interp(const void* f, const Geo& g, const CollideParams& cp, const Bins& bins,
                          const BubbleDev& b, const SwarmBins& sw, bool lift, cudaStream_t st) {
    if (lift)
        return (g.nx & 1) == 0 ? launch_interp_as<ST, true, true>(f, g, cp, bins, b, sw, st)
                               : launch_interp_as<ST, false, true>(f, g, cp, bins, b, sw, st);
    return (g.nx & 1) == 0 ? launch_interp_as<ST, true, false>(f, g, cp, bins, b, sw, st)
                           : launch_interp_as<ST, false, false>(f, g, cp, bins, b, sw, st);
}

bool swarm_ready(const SwarmBins& sw) {
    return sw.grid >= 1 && sw.interp_grid >= 1 && sw.bar && sw.cursor && sw.kidx && sw.slots &&
           sw.ntile && sw.per >= 1 && sw.partial && sw.cover && sw.ncover && sw.chunk_sums;
}
}  // namespace

cudaError_t launch_swarm_update(int storage, const void* f, const Geo& g,
                                const CollideParams& cp, const BubbleDev& b,
                                const BubbleConst& bc, int* flag, const Bins& bins,
                                const SwarmBins& sw, cudaStream_t st) {
    if (b.nb == 0) return cudaSuccess;
    if (!swarm_ready(sw)) return cudaErrorInvalidValue;
    cudaError_t e;
    switch (storage) {
        case 0: e = launch_interp<0>(f, g, cp, bins, b, sw, bc.lift != 0, st); break;
        case 1: e = launch_interp<1>(f, g, cp, bins, b, sw, bc.lift != 0, st); break;
        default: e = launch_interp<2>(f, g, cp, bins, b, sw, bc.lift != 0, st); break;
    }
    if (e != cudaSuccess) return e;
    k_swarm_tail<<<(b.nb + TAIL_THREADS - 1) / TAIL_THREADS, TAIL_THREADS, 0, st>>>(g, b, bc, flag,
                                                                                   bins, sw);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_swarm_binning(g, b, bins, sw, b.spread, flag, st);
}

cudaError_t launch_swarm_binning(const Geo& g, const BubbleDev& b, const Bins& bins,
                                 const SwarmBins& sw, const int* select, int* flag,
                                 cudaStream_t st) {
    if (b.nb == 0) return cudaSuccess;
    if (!swarm_ready(sw)) return cudaErrorInvalidValue;
    k_swarm_bin<<<sw.grid, SWARM_THREADS, 0, st>>>(g, b, bins, sw, select, flag);
    return cudaGetLastError();
}

// Per-bubble closure constants for a batch: nu from each bubble's column.
__global__ void k_bubble_constants_batch(BubbleDev B, BubbleConst bc, const double* col_nu,
                                         const int* bubble_col) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B.nb) return;
    BubbleConst c = bc;
    c.nu = col_nu[bubble_col[b]];
    B.k[b] = bubble_constants(B.d[b], B.n[b], c);
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

// Node coordinates of site s (x fastest); 19 S < 2^32, so 32-bit arithmetic.
__device__ __forceinline__ void site_coords(const Geo& g, unsigned s, int& x, int& y, int& z) {
    const unsigned xy = s / (unsigned)g.nx;
    x = (int)(s - xy * (unsigned)g.nx);
    y = (int)(xy % (unsigned)g.ny);
    z = (int)(xy / (unsigned)g.ny);
}

// rho and the bare Eq. 10 velocity of the current populations, summed in
// FP64 over the stored values (the same sums as the FP64 totals).
template <int ST>
__global__ void k_fields(const typename Store<ST>::T* __restrict__ f, Geo g, CollideParams cp,
                         double* __restrict__ rho, double* __restrict__ u) {
    const unsigned s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= (unsigned)g.S) return;
    int x, y, z;
    site_coords(g, s, x, y, z);
    float gv[Q];
    gather<ST>(f, g, cp, x, y, z, gv);
    double drho = 0.0, jx = 0.0, jy = 0.0, jz = 0.0;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const double v = gv[j];
        drho += v;
        if (cx(j) != 0) jx += cx(j) > 0 ? v : -v;
        if (cy(j) != 0) jy += cy(j) > 0 ? v : -v;
        if (cz(j) != 0) jz += cz(j) > 0 ? v : -v;
    }
    const double r = (double)cp.rho0 + drho;
    if (rho) rho[s] = r;
    if (u) {
        const double inv_r = 1.0 / r;
        u[s] = jx * inv_r;
        u[g.S + s] = jy * inv_r;
        u[2 * g.S + s] = jz * inv_r;
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
// from: the population j of node y + c_j; if that link crosses a no-slip
// wall, the population opp(j) of node y itself; if it crosses only a
// free-slip top, the population mirz(j) of the top-layer node one
// tangential step along (inverse of the pull).
__device__ __forceinline__ void push_target(const Geo& g, int j, int x, int y, int z, int& dir,
                                            long long& node) {
    int tx = x + cx(j), ty = y + cy(j), tz = z + cz(j);
    bool bounce = false, specular = false;
    if (cx(j) != 0 && (tx < 0 || tx >= g.nx)) {
        if (g.walls & 0x01) bounce = true;
        else tx = tx < 0 ? tx + g.nx : tx - g.nx;
    }
    if (cy(j) != 0 && (ty < 0 || ty >= g.ny)) {
        if (g.walls & 0x04) bounce = true;
        else ty = ty < 0 ? ty + g.ny : ty - g.ny;
    }
    if (cz(j) != 0 && (tz < 0 || tz >= g.nz)) {
        if (tz >= g.nz && (g.walls & WALL_TOP_FREE)) specular = true;
        else if (g.walls & 0x10) bounce = true;
        else tz = tz < 0 ? tz + g.nz : tz - g.nz;
    }
    if (bounce) {
        dir = opp(j);
        node = site_index(g, x, y, z);
    } else if (specular) {
        dir = mirz(j);
        node = site_index(g, tx, ty, z);
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
    // Each node writes its 19 equilibria (Eq. 6) to the places the first
    // step's pull will read them from (pull_offset; a bijection, so no two
    // threads write the same place).  FP32 arithmetic on the shifted value;
    // rho - rho0 is formed in FP64 first.
    const unsigned s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= (unsigned)g.S) return;
    int x, y, z;
    site_coords(g, s, x, y, z);
    const double rd = rho ? rho[s] : (double)cp.rho0;
    const float dr = (float)(rd - (double)cp.rho0), r = (float)rd;
    const float ux = u ? (float)u[s] : 0.0f, uy = u ? (float)u[g.S + s] : 0.0f,
                uz = u ? (float)u[2 * g.S + s] : 0.0f;
    const float usq15 = 1.5f * (ux * ux + uy * uy + uz * uz);
#define LBM_FEQ(J)                                                                            \
    {                                                                                         \
        const float cu = (float)cx(J) * ux + (float)cy(J) * uy + (float)cz(J) * uz;           \
        const float v = wf(J) * (dr + r * (cu * (3.0f + 4.5f * cu) - usq15));                 \
        Store<ST>::template store<J>(f + pull_offset<J>(g, x, y, z), v, cp);                  \
    }
    LBM_FEQ(0); LBM_FEQ(1); LBM_FEQ(2); LBM_FEQ(3); LBM_FEQ(4); LBM_FEQ(5); LBM_FEQ(6);
    LBM_FEQ(7); LBM_FEQ(8); LBM_FEQ(9); LBM_FEQ(10); LBM_FEQ(11); LBM_FEQ(12); LBM_FEQ(13);
    LBM_FEQ(14); LBM_FEQ(15); LBM_FEQ(16); LBM_FEQ(17); LBM_FEQ(18);
#undef LBM_FEQ
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

namespace lbm {

// ---------------------------------------------------------------------------
// Host conversion of the bubble state between the C ABI's FP64 arrays and the
// device format (two-float centres, FP32 velocities).
// ---------------------------------------------------------------------------
cudaError_t upload_bubble_state(const BubbleDev& B, int n, const double* pos3, const double* vel3,
                                cudaStream_t st) {
    const size_t m = 3 * (size_t)n;
    std::vector<float> xh(m), xl(m), u(m, 0.0f), zeros(m, 0.0f);
    for (size_t i = 0; i < m; ++i) {
        split_f2(pos3[i], xh[i], xl[i]);
        if (vel3) u[i] = (float)vel3[i];
    }
    const size_t bytes = sizeof(float) * m;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(B.xh, xh.data(), bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(B.xl, xl.data(), bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(B.u, u.data(), bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(B.ulprev, zeros.data(), bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(B.ul, zeros.data(), bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(B.psi, zeros.data(), bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
    // The staging vectors go out of scope: let the copies finish first.
    return cudaStreamSynchronize(st);
}

// FP64 copies of the first k bubbles' state: out = [x | u | u_l | psi], each
// 3k values.
__global__ void k_export_bubbles(BubbleDev B, int k, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t m = 3 * (size_t)k;
    if (i >= (int)m) return;
    out[i] = join_f2(B.xh[i], B.xl[i]);
    out[m + i] = B.u[i];
    out[2 * m + i] = B.ul[i];
    out[3 * m + i] = B.psi[i];
}

cudaError_t download_bubble_state(const BubbleDev& B, int k, double* pos3, double* vel3,
                                  double* ul3, double* psi3, cudaStream_t st) {
    double* const stage = B.out64;
    const size_t m = 3 * (size_t)k, bytes = sizeof(double) * m;
    k_export_bubbles<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(B, k, stage);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double* dst[4] = {pos3, vel3, ul3, psi3};
    for (int q = 0; q < 4; ++q)
        if (dst[q] && (e = cudaMemcpyAsync(dst[q], stage + q * m, bytes, cudaMemcpyDeviceToHost,
                                           st)) != cudaSuccess)
            return e;
    return cudaStreamSynchronize(st);
}

}  // namespace lbm
