// Reverse mode of the coupled step (hand-written adjoint), with checkpointed
// recomputation.
//
// Objective: L = (ubar - target)^2, ubar the mean over bubbles and over the
// last `window` steps of the bubble rise velocity u_b,z.  Gradients: with
// respect to the drag scale s_D (Table 1 drag times s_D), each bubble's
// diameter d_b (through its volume, mass, buoyancy, drag closure and mapping
// window n = width_factor d_b), and the initial liquid velocity field u0 (with
// the initial populations f = f^eq(rho, u0), Algorithm 1 initialisation).
//
// One forward step n maps (f^n, bubble state) to (f^{n+1}, bubble state'):
//   bubble update   u_l = sum_j W_j(x^n) u(f^n)_j (Eq. 20), sub-stepped
//                   Newton update (Eq. 4, Table 1), psi = -mean F_D;
//   spreading       F(y) = sum_b W_y(x^{n+1}_b) psi_b (Eq. 21);
//   liquid          f^{n+1} = Stream(Collide(f^n, F)) (Eq. 12-16).
// The reverse step (step n, newest first):
//   k_adj_liquid    Lambda^n = C_f^T S^T Lambda^{n+1} per node (transposed
//                   streaming with bounce-back, linearised forced BGK);
//   k_adj_bubbles_ab (a CTA per bubble, on a second stream alongside
//                   k_adj_liquid: both read only Lambda^{n+1} and f^n)
//                   spreading adjoint and the reverse of the sub-steps;
//   k_adj_bubbles_c (after both, one CTA, bubbles in order)
//                   the interpolation adjoint.
//   In all:         per bubble: spreading adjoint (Lambda_psi, Lambda_x^{n+1},
//                   Lambda_n from the force adjoint at the window nodes),
//                   reverse of the sub-steps, interpolation adjoint (adds to
//                   Lambda^n at the window nodes, Lambda_x^n, Lambda_n).
// Liquid adjoints are FP32 (like the forward sweep); the bubble adjoint and
// the accumulated parameter gradients are FP64.
#include <cmath>
#include <vector>

#include "lbm_ctx.hpp"
#include "lbm_device.cuh"

using namespace lbm;

namespace {

constexpr int ADJ_MAX_BUBBLES = 256;
constexpr int ADJ_THREADS = 256;
constexpr int ADJ_MAX_SUB = 64;

// Bubble state snapshot: before a step (x, u, q = u_l history, h, active) and
// after it (ul = u_l of the step, psi, x', u', rec = spreading record).
struct BubbleSnap {
    double x[3], u[3], q[3], ul[3], psi[3];
    float xh[3], xl[3];   // the centre as stored (x = xh + xl), for an exact restore
    int h, active;
    BubbleRec rec;
};

// Per-bubble adjoint state carried between reverse steps.
struct BubbleAdj {
    double lx[3], lu[3], lq[3];
};

// Closure constants in FP64 together with their d-derivatives (Table 1, Eq. 3).
struct AdjConst {
    double nu, dt_b, dt_l, sn_coeff, sn_exp, width_factor, drag_scale;
    double rho_l, rho_b, g, sigma, c_am;
    int substeps, two_way;
};

__global__ void k_snapshot(BubbleDev B, BubbleSnap* out, int post) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B.nb) return;
    BubbleSnap& s = out[b];
    for (int a = 0; a < 3; ++a) {
        s.xh[a] = B.xh[3 * b + a];
        s.xl[a] = B.xl[3 * b + a];
        s.x[a] = join_f2(s.xh[a], s.xl[a]);
        s.u[a] = B.u[3 * b + a];
        if (post) {
            s.ul[a] = B.ul[3 * b + a];
            s.psi[a] = B.psi[3 * b + a];
        } else {
            s.q[a] = B.ulprev[3 * b + a];
        }
    }
    if (post) {
        s.rec = B.rec[b];
        s.active = B.spread[b];   // 1 if it took part in the step
    } else {
        s.h = B.has_prev[b];
        s.active = B.active[b];
    }
}

__global__ void k_restore(BubbleDev B, const BubbleSnap* in) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B.nb) return;
    const BubbleSnap& s = in[b];
    for (int a = 0; a < 3; ++a) {
        B.xh[3 * b + a] = s.xh[a];
        B.xl[3 * b + a] = s.xl[a];
        B.u[3 * b + a] = (float)s.u[a];
        B.ulprev[3 * b + a] = (float)s.q[a];
    }
    B.has_prev[b] = s.h;
    B.active[b] = s.active;
}

__global__ void k_record_uz(BubbleDev B, double* uz) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B.nb) uz[b] = B.u[3 * b + 2];
}

// ubar over the last `window` steps; out = {ubar, loss}.
__global__ void k_adj_loss(const double* uz, int nsteps, int nb, int window, double target,
                           double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int n = nsteps - window; n < nsteps; ++n)
        for (int b = 0; b < nb; ++b) s += uz[(size_t)n * nb + b];
    const double ubar = s / ((double)window * nb);
    out[0] = ubar;
    out[1] = (ubar - target) * (ubar - target);
}

// ---- mapping weights and their derivatives, normalised units --------------
// z(t) = t^4 - 2 t^2 + 1 on [-1, 1] (Eq. 18 without 15/(16 n)); the cell
// integral of Z is 15/16 of the integral of z over the clipped cell.
__device__ __forceinline__ float zpoly(float t) {
    const float t2 = t * t;
    return (t2 - 2.0f) * t2 + 1.0f;
}

// Integral of z over [a, b] (clipped to [-1, 1]) and its derivatives with
// respect to the bubble coordinate x and the half-width n, for the cell
// [s0, s0 + 1] relative to the bubble (a = s0/n, b = (s0+1)/n).
struct AxisW {
    float w, dx, dn;
};

__device__ __forceinline__ AxisW axis_weight(float s0, float s1, float inv_n) {
    const float a = fmaxf(s0 * inv_n, -1.0f), b = fminf(s1 * inv_n, 1.0f);
    AxisW r{0.0f, 0.0f, 0.0f};
    if (!(b > a)) return r;
    const float a2 = a * a, b2 = b * b, ab = a * b;
    const float p4 = b2 * b2 + b2 * ab + ab * ab + ab * a2 + a2 * a2;
    r.w = (b - a) * (p4 * 0.2f - (b2 + ab + a2) * (2.0f / 3.0f) + 1.0f);
    const float za = zpoly(a), zb = zpoly(b);
    r.dx = -inv_n * (zb - za);                 // d/dx, s = i - x
    r.dn = -inv_n * (b * zb - a * za);         // d/dn
    return r;
}

// Per-axis normalisation over the in-box part of the window (walls) and its
// derivatives; 16/15 and zero derivatives on a periodic axis.
__device__ __forceinline__ AxisW axis_norm_d(double x, int L, float inv_n, bool periodic) {
    if (periodic) return AxisW{16.0f / 15.0f, 0.0f, 0.0f};
    return axis_weight((float)(-x), (float)((double)L - x), inv_n);
}

// Window of one bubble at centre x: cells per axis and the normalisation.
struct Window {
    int lo[3], cnt[3];
    double x[3];
    float inv_n;
    AxisW norm[3];
};

__device__ __forceinline__ void make_window(const Geo& g, const double* x, double n, Window& w) {
    const int L[3] = {g.nx, g.ny, g.nz};
    w.inv_n = (float)(1.0 / n);
    for (int a = 0; a < 3; ++a) {
        const bool periodic = !(g.walls & (1u << (2 * a)));
        int l = (int)floor(x[a] - n);
        int h = (int)ceil(x[a] + n) - 1;
        if (!periodic) {
            l = max(l, 0);
            h = min(h, L[a] - 1);
        }
        w.lo[a] = l;
        w.cnt[a] = min(max(h - l + 1, 0), 2 * (int)MAX_HALF_WIDTH + 2);
        w.x[a] = x[a];
        w.norm[a] = axis_norm_d(x[a], L[a], w.inv_n, periodic);
    }
}

// Weight W of window node m and its derivatives dW/dx (3) and dW/dn; the
// node's wrapped lattice coordinates in (i, j, k).
__device__ __forceinline__ float window_node(const Geo& g, const Window& w, int m, float dWdx[3],
                                             float& dWdn, int& i, int& j, int& k) {
    const int ix = m % w.cnt[0], rest = m / w.cnt[0];
    const int iy = rest % w.cnt[1], iz = rest / w.cnt[1];
    const int c[3] = {w.lo[0] + ix, w.lo[1] + iy, w.lo[2] + iz};
    AxisW ax[3];
    for (int a = 0; a < 3; ++a) {
        const float s0 = (float)((double)c[a] - w.x[a]);
        ax[a] = axis_weight(s0, s0 + 1.0f, w.inv_n);
    }
    const float nrm = w.norm[0].w * w.norm[1].w * w.norm[2].w;
    const float W = ax[0].w * ax[1].w * ax[2].w / nrm;
    dWdn = 0.0f;
    for (int a = 0; a < 3; ++a) {
        const int b1 = (a + 1) % 3, b2 = (a + 2) % 3;
        const float others = ax[b1].w * ax[b2].w / nrm;
        dWdx[a] = ax[a].dx * others - W * w.norm[a].dx / w.norm[a].w;
        dWdn += ax[a].dn * others - W * w.norm[a].dn / w.norm[a].w;
    }
    i = (c[0] % g.nx + g.nx) % g.nx;
    j = (c[1] % g.ny + g.ny) % g.ny;
    k = (c[2] % g.nz + g.nz) % g.nz;
    return W;
}

__device__ __forceinline__ int node_index(const Geo& g, int i, int j, int k) {
    return (k * g.ny + j) * g.nx + i;
}

// Adjoint of the post-collision values gathered back through streaming:
// a_j(y) = Lambda^{n+1} at the node and direction that out_j(y) streams to.
// Element offset of the adjoint of population J leaving node (x,y,z): plane J
// at x + c_J, or, when that link crosses a wall, plane opp(J) at the node
// itself (the adjoint of half-way bounce-back); periodic axes wrap.  Written
// with selects so that a gather issues all 19 loads before using any.
template <int J>
__device__ __forceinline__ unsigned push_offset(const Geo& g, int x, int y, int z) {
    int tx = x + cx(J), ty = y + cy(J), tz = z + cz(J);
    bool bounce = false;
    if (cx(J) != 0) {
        const bool out = (unsigned)tx >= (unsigned)g.nx;
        bounce = bounce || (out && (g.walls & 0x01));
        tx = out ? (tx < 0 ? tx + g.nx : tx - g.nx) : tx;
    }
    if (cy(J) != 0) {
        const bool out = (unsigned)ty >= (unsigned)g.ny;
        bounce = bounce || (out && (g.walls & 0x04));
        ty = out ? (ty < 0 ? ty + g.ny : ty - g.ny) : ty;
    }
    if (cz(J) != 0) {
        const bool out = (unsigned)tz >= (unsigned)g.nz;
        bounce = bounce || (out && (g.walls & 0x10));
        tz = out ? (tz < 0 ? tz + g.nz : tz - g.nz) : tz;
    }
    const unsigned S = (unsigned)g.S;
    return bounce ? (unsigned)opp(J) * S + (unsigned)node_index(g, x, y, z)
                  : (unsigned)J * S + (unsigned)node_index(g, tx, ty, tz);
}

__device__ __forceinline__ void gather_push(const float* __restrict__ lam, const Geo& g, int x,
                                            int y, int z, float a[Q]) {
    unsigned o[Q];
#define LBM_PO(J) o[J] = push_offset<J>(g, x, y, z)
    LBM_PO(0); LBM_PO(1); LBM_PO(2); LBM_PO(3); LBM_PO(4); LBM_PO(5); LBM_PO(6);
    LBM_PO(7); LBM_PO(8); LBM_PO(9); LBM_PO(10); LBM_PO(11); LBM_PO(12); LBM_PO(13);
    LBM_PO(14); LBM_PO(15); LBM_PO(16); LBM_PO(17); LBM_PO(18);
#undef LBM_PO
#pragma unroll
    for (int j = 0; j < Q; ++j) a[j] = __ldg(lam + o[j]);
}

// Force at a node from all spreading records of the step (Eq. 21).
__device__ __forceinline__ void force_at(const Geo& g, const BubbleRec* recs, const int* spread,
                                         int nb, int x, int y, int z, float F[3]) {
    F[0] = F[1] = F[2] = 0.0f;
    for (int b = 0; b < nb; ++b) {
        if (!spread[b]) continue;
        const BubbleRec& r = recs[b];
        float rr[3] = {(float)(x - r.ax) + 0.5f - r.fx, (float)(y - r.ay) + 0.5f - r.fy,
                       (float)(z - r.az) + 0.5f - r.fz};
        const int L[3] = {g.nx, g.ny, g.nz};
        bool outside = false;
        for (int a = 0; a < 3; ++a) {
            if (!(g.walls & (1u << (2 * a)))) {
                if (rr[a] > 0.5f * L[a]) rr[a] -= (float)L[a];
                else if (rr[a] < -0.5f * L[a]) rr[a] += (float)L[a];
            }
            // cell_poly is zero once the cell [s - h, s + h] is outside [-1, 1]
            outside = outside || fabsf(rr[a] * r.inv_n) >= 1.0f + r.h;
        }
        if (outside) continue;
        float w = 1.0f;
        for (int a = 0; a < 3; ++a) w *= cell_poly(rr[a] * r.inv_n, r.h);
        F[0] = fmaf(w, r.px, F[0]);
        F[1] = fmaf(w, r.py, F[1]);
        F[2] = fmaf(w, r.pz, F[2]);
    }
}

// Linearised forced BGK at one node, transposed.  g: shifted pre-collision
// populations; a: adjoint of the post-collision values.  Returns the adjoint
// of the pre-collision populations in lam and of the force in lamF.
//   rho = rho0 + sum g, u = (sum c g + F/2) / rho
//   out_j = (1 - w) f_j + w f^eq_j(rho, u) + G_j(u, F)
//   dL/df_k = (1 - w) a_k + A_rho + A_u . (c_k - u) / rho
//   A_rho = w sum_j a_j w_j (1 + 3 cu + 9/2 cu^2 - 3/2 u^2)
//   A_u   = sum_j a_j [w w_j rho (3 c_j + 9 cu_j c_j - 3 u) + pref w_j (9 cF_j c_j - 3 F)]
//   dL/dF = A_u / (2 rho) + sum_j a_j pref w_j (3 (c_j - u) + 9 cu_j c_j)
__device__ __forceinline__ void collide_adjoint(const float g[Q], const float F[3], float rho0,
                                                float omega, float pref, const float a[Q],
                                                float lam[Q], float lamF[3]) {
    float drho = 0.0f, m[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        drho += g[j];
        if (cx(j) != 0) m[0] += (float)cx(j) * g[j];
        if (cy(j) != 0) m[1] += (float)cy(j) * g[j];
        if (cz(j) != 0) m[2] += (float)cz(j) * g[j];
    }
    const float rho = rho0 + drho, inv_rho = 1.0f / rho;
    const float u[3] = {(m[0] + 0.5f * F[0]) * inv_rho, (m[1] + 0.5f * F[1]) * inv_rho,
                        (m[2] + 0.5f * F[2]) * inv_rho};
    const float usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    // With aw_j = a_j w_j, the sums over j that the adjoint needs:
    //   S0 = sum aw, S1 = sum aw c, S2 = sum aw (c.u) c, S3 = sum aw (c.F) c,
    //   Su = sum aw (c.u), Su2 = sum aw (c.u)^2.
    float S0 = 0.0f, Su = 0.0f, Su2 = 0.0f;
    float S1[3] = {0.0f, 0.0f, 0.0f}, S2[3] = {0.0f, 0.0f, 0.0f}, S3[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        const int c[3] = {cx(j), cy(j), cz(j)};
        float cu = 0.0f, cF = 0.0f;
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (c[d] != 0) {
                cu += (float)c[d] * u[d];
                cF += (float)c[d] * F[d];
            }
        const float aw = a[j] * wf(j), awcu = aw * cu, awcF = aw * cF;
        S0 += aw;
        Su += awcu;
        Su2 = fmaf(awcu, cu, Su2);
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (c[d] != 0) {
                S1[d] += (float)c[d] * aw;
                S2[d] += (float)c[d] * awcu;
                S3[d] += (float)c[d] * awcF;
            }
    }
    // The density and velocity adjoints of the forced equilibrium (Eq. 6, 14,
    // 15): sum_j aw_j times the derivatives of f^eq_j and of the Guo term.
    const float A_rho = omega * (S0 * (1.0f - 1.5f * usq) + 3.0f * Su + 4.5f * Su2);
    float Au[3], base = A_rho;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float A_u = omega * rho * (3.0f * S1[d] + 9.0f * S2[d] - 3.0f * u[d] * S0) +
                          pref * (9.0f * S3[d] - 3.0f * F[d] * S0);
        const float G_F = pref * (3.0f * S1[d] - 3.0f * u[d] * S0 + 9.0f * S2[d]);
        Au[d] = A_u * inv_rho;
        base -= u[d] * Au[d];
        lamF[d] = 0.5f * Au[d] + G_F;
    }
    // lam_k = (1 - omega) a_k + A_rho + (c_k - u) . A_u / rho
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        float cA = base;
        if (cx(k) != 0) cA += (float)cx(k) * Au[0];
        if (cy(k) != 0) cA += (float)cy(k) * Au[1];
        if (cz(k) != 0) cA += (float)cz(k) * Au[2];
        lam[k] = (1.0f - omega) * a[k] + cA;
    }
}

// Lambda^n = C_f^T S^T Lambda^{n+1} at every node.
__global__ void __launch_bounds__(128)
k_adj_liquid(const float* __restrict__ fn, const float* __restrict__ lam_next,
             float* __restrict__ lam, Geo g, CollideParams cp, const BubbleSnap* __restrict__ post,
             int nb, int two_way) {
    __shared__ BubbleRec srec[ADJ_MAX_BUBBLES];
    __shared__ int sspread[ADJ_MAX_BUBBLES];
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        srec[b] = post[b].rec;
        sspread[b] = two_way ? post[b].active : 0;
    }
    __syncthreads();
    const unsigned s = blockIdx.x * blockDim.x + threadIdx.x;   // 19 S < 2^32
    if (s >= (unsigned)g.S) return;
    const unsigned xy = s / (unsigned)g.nx;
    const int x = (int)(s - xy * (unsigned)g.nx), y = (int)(xy % (unsigned)g.ny),
              z = (int)(xy / (unsigned)g.ny);
    float gv[Q], a[Q], out[Q], F[3], lamF[3];
    gather<0>(fn, g, cp, x, y, z, gv);
    gather_push(lam_next, g, x, y, z, a);
    force_at(g, srec, sspread, nb, x, y, z, F);
    collide_adjoint(gv, F, cp.rho0, cp.omega, cp.pref, a, out, lamF);
#pragma unroll
    for (int j = 0; j < Q; ++j) lam[(size_t)j * g.S + s] = out[j];
}

// Sums of N values over the CTA, in thread 0 only (per value: warp shuffles,
// then the warps in order).  The N chains interleave, so the FP64 latency is
// paid once rather than N times.
template <int N>
__device__ __forceinline__ void block_sum_dn(double v[N], double (*sh)[8]) {
    static_assert(N <= 8, "at most 8 values");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    __syncthreads();   // the previous user of sh is done
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < N; ++i) sh[wid][i] = v[i];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
#pragma unroll
            for (int i = 0; i < N; ++i) v[i] += sh[w][i];
    }
}

// One replayed sub-step (FP32, like the forward): slip v = u - u_l, |v|, Re,
// C_D |v|, the drag, Re^sn_exp and 1/|v|.
struct SubRec {
    float v[3], s, re, cdv, fd[3];
    float pw;        // Re^sn_exp
    float inv_s;     // 1 / |v| (0 at rest)
    int branch;      // 0: 8/3 Eo/(Eo+4) |v|, 1: 24 nu/d (1 + a Re^e), 2: 48 nu/d
    int xclamp[3], uclamp[3];
};

// Phases A and B of one reverse step, a CTA per bubble (blockIdx.x).  They
// read f^n, Lambda^{n+1} and the step's snapshots only, so they run alongside
// k_adj_liquid; each CTA writes its own bubble's adjoint state, diameter
// gradient, drag-scale gradient part and interpolation seed lul_out.
__global__ void __launch_bounds__(ADJ_THREADS)
k_adj_bubbles_ab(const float* __restrict__ fn, const float* __restrict__ lam_next, Geo g,
                 CollideParams cp, const BubbleSnap* __restrict__ pre,
                 const BubbleSnap* __restrict__ post, const double* __restrict__ diam, int nb,
                 AdjConst ac, BubbleAdj* __restrict__ adj, double* __restrict__ grad_sD,
                 double* __restrict__ grad_d, double* __restrict__ lul_out, double loss_seed) {
    __shared__ BubbleRec srec[ADJ_MAX_BUBBLES];
    __shared__ int sspread[ADJ_MAX_BUBBLES];
    __shared__ double shn[ADJ_THREADS / 32][8];
    __shared__ SubRec sub[ADJ_MAX_SUB];
    const int tid = threadIdx.x;
    const int b = blockIdx.x;
    if (!pre[b].active) {
        // Not updated this step: its adjoint state passes through unchanged.
        if (tid == 0 && loss_seed != 0.0) adj[b].lu[2] += loss_seed;
        return;
    }
    for (int k = tid; k < nb; k += blockDim.x) {
        srec[k] = post[k].rec;
        sspread[k] = ac.two_way ? post[k].active : 0;
    }
    __syncthreads();
    {
        const double d = diam[b];
        const double n = ac.width_factor * d;

        // -- Phase A: spreading adjoint at x^{n+1} ------------------------------
        double lpsi[3] = {0.0, 0.0, 0.0}, gx[3] = {0.0, 0.0, 0.0}, gn = 0.0;
        if (sspread[b]) {
            Window w;
            make_window(g, post[b].x, n, w);
            const double psi[3] = {post[b].psi[0], post[b].psi[1], post[b].psi[2]};
            const int M = w.cnt[0] * w.cnt[1] * w.cnt[2];
            for (int m = tid; m < M; m += blockDim.x) {
                float dWdx[3], dWdn;
                int i, j, k;
                const float W = window_node(g, w, m, dWdx, dWdn, i, j, k);
                float gv[Q], a[Q], out[Q], F[3], lamF[3];
                gather<0>(fn, g, cp, i, j, k, gv);
                gather_push(lam_next, g, i, j, k, a);
                force_at(g, srec, sspread, nb, i, j, k, F);
                collide_adjoint(gv, F, cp.rho0, cp.omega, cp.pref, a, out, lamF);
                const double pl = psi[0] * lamF[0] + psi[1] * lamF[1] + psi[2] * lamF[2];
                for (int c = 0; c < 3; ++c) {
                    lpsi[c] += (double)W * lamF[c];
                    gx[c] += pl * dWdx[c];
                }
                gn += pl * dWdn;
            }
        }
        {
            double sums[7] = {lpsi[0], lpsi[1], lpsi[2], gx[0], gx[1], gx[2], gn};
            block_sum_dn<7>(sums, shn);   // results in thread 0, which runs Phase B
            for (int c = 0; c < 3; ++c) {
                lpsi[c] = sums[c];
                gx[c] = sums[3 + c];
            }
            gn = sums[6];
        }

        // -- Phase B: reverse of the sub-stepped update (thread 0) ---------------
        // The closure constants and their d-derivatives are FP64, once per step.
        // The sub-step replay and the per-sub-step terms of its reverse run in
        // FP32, the precision of the forward they differentiate, because FP64
        // issue is slow on this GPU.  The centre (wall clamps) and the adjoint
        // state carried between sub-steps and steps stay FP64.
        if (tid == 0) {
            const int K = min(ac.substeps, ADJ_MAX_SUB);
            const double r = 0.5 * d, vol = M_PI * d * d * d / 6.0, dvol = 0.5 * M_PI * d * d;
            const double meff = (ac.rho_b + ac.c_am * ac.rho_l) * vol;
            const double kdt = ac.dt_b / meff, dkdt = -kdt / vol * dvol;
            const double fb = (ac.rho_l - ac.rho_b) * vol * ac.g, dfb = (ac.rho_l - ac.rho_b) * ac.g * dvol;
            const double P = 0.5 * ac.rho_l * M_PI * r * r * ac.drag_scale;
            const double dP = 0.25 * ac.rho_l * M_PI * d * ac.drag_scale;
            const double A0 = 24.0 * ac.nu / d, dA0 = -A0 / d;
            const double Bv = 48.0 * ac.nu / d, dBv = -Bv / d;
            const double Eo = (ac.rho_l - ac.rho_b) * ac.g * d * d / ac.sigma, dEo = 2.0 * Eo / d;
            const double E = 8.0 / 3.0 * Eo / (Eo + 4.0), dE = 8.0 / 3.0 * 4.0 / ((Eo + 4.0) * (Eo + 4.0)) * dEo;
            const double Cf = ac.c_am * ac.rho_l * vol / ac.dt_l, dCf = ac.c_am * ac.rho_l * dvol / ac.dt_l;
            const float kdt_f = (float)kdt, fb_f = (float)fb, P_f = (float)P, A0_f = (float)A0,
                        Bv_f = (float)Bv, E_f = (float)E;
            const float sn_coeff = (float)ac.sn_coeff, sn_exp = (float)ac.sn_exp;
            const float re_per_s = (float)(d / ac.nu), nu_over_d = (float)(ac.nu / d),
                        inv_nu = (float)(1.0 / ac.nu), inv_K = 1.0f / (float)K;
            const double* ul = post[b].ul;
            const double* q = pre[b].q;
            const int h = pre[b].h;
            float ulf[3], fvm[3];
            for (int c = 0; c < 3; ++c) {
                ulf[c] = (float)ul[c];
                fvm[c] = h ? (float)(Cf * (ul[c] - q[c])) : 0.0f;
            }
            const int L[3] = {g.nx, g.ny, g.nz};
            // forward replay
            float u[3] = {(float)pre[b].u[0], (float)pre[b].u[1], (float)pre[b].u[2]};
            double x[3] = {pre[b].x[0], pre[b].x[1], pre[b].x[2]};
            for (int kk = 0; kk < K; ++kk) {
                SubRec& sr = sub[kk];
                float s2 = 0.0f;
                for (int c = 0; c < 3; ++c) {
                    sr.v[c] = u[c] - ulf[c];
                    s2 = fmaf(sr.v[c], sr.v[c], s2);
                }
                sr.s = sqrtf(s2);
                sr.inv_s = sr.s > 0.0f ? 1.0f / sr.s : 0.0f;
                sr.re = sr.s * re_per_s;
                sr.pw = sr.re > 0.0f ? powf(sr.re, sn_exp) : 0.0f;
                const float A = A0_f * (1.0f + sn_coeff * sr.pw);
                const float vis = fminf(A, Bv_f);
                if (E_f * sr.s >= vis) {
                    sr.cdv = E_f * sr.s;
                    sr.branch = 0;
                } else {
                    sr.cdv = vis;
                    sr.branch = A <= Bv_f ? 1 : 2;
                }
                for (int c = 0; c < 3; ++c) {
                    sr.fd[c] = -P_f * sr.cdv * sr.v[c];
                    const float fz = c == 2 ? fb_f : 0.0f;
                    u[c] = u[c] + (fz + sr.fd[c] + fvm[c]) * kdt_f;
                    x[c] = x[c] + (double)u[c] * ac.dt_b;
                    sr.xclamp[c] = 0;
                    sr.uclamp[c] = 0;
                    if (g.walls & (1u << (2 * c))) {
                        if (x[c] < r) {
                            x[c] = r;
                            sr.xclamp[c] = 1;
                            if (u[c] < 0.0f) { u[c] = 0.0f; sr.uclamp[c] = 1; }
                        }
                        if (x[c] > (double)L[c] - r) {
                            x[c] = (double)L[c] - r;
                            sr.xclamp[c] = 1;
                            if (u[c] > 0.0f) { u[c] = 0.0f; sr.uclamp[c] = 1; }
                        }
                    }
                }
            }
            // reverse
            double lx[3], lu[3], lul[3], lq[3];
            float lfvm[3] = {0.0f, 0.0f, 0.0f}, lpsi_f[3];
            float lP = 0.0f, lkdt = 0.0f, lfb = 0.0f, lA0 = 0.0f, lB = 0.0f, lE = 0.0f, ld_re = 0.0f;
            for (int c = 0; c < 3; ++c) {
                lx[c] = adj[b].lx[c] + gx[c];
                lu[c] = adj[b].lu[c];
                lul[c] = adj[b].lq[c];   // u_l of this step is the next step's history
                lq[c] = 0.0;
                lpsi_f[c] = (float)lpsi[c];
            }
            lu[2] += loss_seed;
            for (int kk = K - 1; kk >= 0; --kk) {
                const SubRec& sr = sub[kk];
                double lpre[3];
                for (int c = 0; c < 3; ++c) {
                    // x_{k+1} = clamp(x_k + u_{k+1} dt_b), u_{k+1} = clamp(u_k + du)
                    double lu_next = lu[c];
                    if (!sr.xclamp[c]) lu_next += lx[c] * ac.dt_b;
                    else lx[c] = 0.0;
                    lpre[c] = sr.uclamp[c] ? 0.0 : lu_next;
                }
                float lfd[3];
                for (int c = 0; c < 3; ++c) {
                    const float lp = (float)lpre[c];
                    lfd[c] = lp * kdt_f - lpsi_f[c] * inv_K;
                    lfvm[c] += lp * kdt_f;
                    lkdt += lp * ((c == 2 ? fb_f : 0.0f) + sr.fd[c] + fvm[c]);
                    if (c == 2) lfb += lp * kdt_f;
                    lu[c] = lpre[c];
                }
                // fd = -P cdv v
                const float lfd_v = lfd[0] * sr.v[0] + lfd[1] * sr.v[1] + lfd[2] * sr.v[2];
                const float lcdv = -P_f * lfd_v;
                lP += -sr.cdv * lfd_v;
                float lv[3] = {-P_f * sr.cdv * lfd[0], -P_f * sr.cdv * lfd[1], -P_f * sr.cdv * lfd[2]};
                float ls = 0.0f;
                if (sr.branch == 0) {
                    lE += lcdv * sr.s;
                    ls += lcdv * E_f;
                } else if (sr.branch == 1) {
                    lA0 += lcdv * (1.0f + sn_coeff * sr.pw);
                    if (sr.re > 0.0f) {
                        // d(Re^e)/dRe = e Re^e / Re, with 1/Re = nu / (d |v|)
                        const float lre = lcdv * A0_f * sn_coeff * sn_exp * sr.pw * nu_over_d * sr.inv_s;
                        ls += lre * re_per_s;
                        ld_re += lre * sr.s * inv_nu;
                    }
                } else {
                    lB += lcdv;
                }
                if (sr.s > 0.0f)
                    for (int c = 0; c < 3; ++c) lv[c] += ls * sr.v[c] * sr.inv_s;
                for (int c = 0; c < 3; ++c) {
                    lu[c] += lv[c];
                    lul[c] -= lv[c];
                }
            }
            double lCf = 0.0;
            if (h)
                for (int c = 0; c < 3; ++c) {
                    lul[c] += lfvm[c] * Cf;
                    lq[c] -= lfvm[c] * Cf;
                    lCf += lfvm[c] * (ul[c] - q[c]);
                }
            const double gdd = lP * dP + lkdt * dkdt + lfb * dfb + lA0 * dA0 + lB * dBv + lE * dE +
                               ld_re + lCf * dCf + gn * ac.width_factor;
            grad_d[b] += gdd;
            grad_sD[b] += lP * P / ac.drag_scale;   // summed over bubbles at the end
            for (int c = 0; c < 3; ++c) {
                adj[b].lx[c] = lx[c];
                adj[b].lu[c] = lu[c];
                adj[b].lq[c] = lq[c];
                lul_out[3 * b + c] = lul[c];
            }
        }
    }
}

// Phase C of one reverse step, after k_adj_liquid and k_adj_bubbles_ab: the
// interpolation adjoint of every active bubble, one bubble after another in
// one CTA (windows may overlap, and Lambda^n is updated in place in bubble
// order).
__global__ void __launch_bounds__(ADJ_THREADS)
k_adj_bubbles_c(const float* __restrict__ fn, float* __restrict__ lam, Geo g, CollideParams cp,
                const BubbleSnap* __restrict__ pre, const double* __restrict__ diam, int nb,
                AdjConst ac, BubbleAdj* __restrict__ adj, double* __restrict__ grad_d,
                const double* __restrict__ lul_in) {
    __shared__ double shn[ADJ_THREADS / 32][8];
    const int tid = threadIdx.x;
    for (int b = 0; b < nb; ++b) {
        if (!pre[b].active) continue;
        const double n = ac.width_factor * diam[b];
        // -- Phase C: interpolation adjoint at x^n --------------------------------
        {
            Window w;
            make_window(g, pre[b].x, n, w);
            const double lul[3] = {lul_in[3 * b], lul_in[3 * b + 1], lul_in[3 * b + 2]};
            double gx0[3] = {0.0, 0.0, 0.0}, gn0 = 0.0;
            const int M = w.cnt[0] * w.cnt[1] * w.cnt[2];
            for (int m = tid; m < M; m += blockDim.x) {
                float dWdx[3], dWdn;
                int i, j, k;
                const float W = window_node(g, w, m, dWdx, dWdn, i, j, k);
                float gv[Q];
                gather<0>(fn, g, cp, i, j, k, gv);
                float drho = 0.0f, mm[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int q2 = 0; q2 < Q; ++q2) {
                    drho += gv[q2];
                    mm[0] += (float)cx(q2) * gv[q2];
                    mm[1] += (float)cy(q2) * gv[q2];
                    mm[2] += (float)cz(q2) * gv[q2];
                }
                const float rho = cp.rho0 + drho, inv_rho = 1.0f / rho;
                const float uj[3] = {mm[0] * inv_rho, mm[1] * inv_rho, mm[2] * inv_rho};
                const double lu_u = lul[0] * uj[0] + lul[1] * uj[1] + lul[2] * uj[2];
                for (int c = 0; c < 3; ++c) gx0[c] += lu_u * dWdx[c];
                gn0 += lu_u * dWdn;
                // u(j) = m/rho: d u / d f_k = (c_k - u) / rho
                const int node = node_index(g, i, j, k);
                const float lw[3] = {(float)(W * lul[0]) * inv_rho, (float)(W * lul[1]) * inv_rho,
                                     (float)(W * lul[2]) * inv_rho};
                // Each window node belongs to one thread: load its 19 values
                // first, so that the read-modify-writes do not serialise.
                float cur[Q];
#pragma unroll
                for (int q2 = 0; q2 < Q; ++q2) cur[q2] = lam[(size_t)q2 * g.S + node];
#pragma unroll
                for (int q2 = 0; q2 < Q; ++q2) {
                    const float add = ((float)cx(q2) - uj[0]) * lw[0] + ((float)cy(q2) - uj[1]) * lw[1] +
                                      ((float)cz(q2) - uj[2]) * lw[2];
                    lam[(size_t)q2 * g.S + node] = cur[q2] + add;
                }
            }
            double sums[4] = {gx0[0], gx0[1], gx0[2], gn0};
            block_sum_dn<4>(sums, shn);   // results in thread 0
            for (int c = 0; c < 3; ++c) gx0[c] = sums[c];
            gn0 = sums[3];
            if (tid == 0) {
                for (int c = 0; c < 3; ++c) adj[b].lx[c] += gx0[c];
                grad_d[b] += gn0 * ac.width_factor;
            }
        }
        __syncthreads();
    }
}

// dL/du0 at every node for f^0 = f^eq(rho, u0):
//   dL/du0 = sum_j Lambda^0_j w_j rho (3 c_j + 9 (c_j . u0) c_j - 3 u0).
__global__ void k_adj_init(const float* __restrict__ f0, const float* __restrict__ lam, Geo g,
                           CollideParams cp, double* __restrict__ du0) {
    const unsigned s = blockIdx.x * blockDim.x + threadIdx.x;   // 19 S < 2^32
    if (s >= (unsigned)g.S) return;
    const unsigned xy = s / (unsigned)g.nx;
    const int x = (int)(s - xy * (unsigned)g.nx), y = (int)(xy % (unsigned)g.ny),
              z = (int)(xy / (unsigned)g.ny);
    float gv[Q];
    gather<0>(f0, g, cp, x, y, z, gv);
    double drho = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < Q; ++j) {
        drho += gv[j];
        m[0] += cx(j) * (double)gv[j];
        m[1] += cy(j) * (double)gv[j];
        m[2] += cz(j) * (double)gv[j];
    }
    const double rho = (double)cp.rho0 + drho;
    const double u[3] = {m[0] / rho, m[1] / rho, m[2] / rho};
    double out[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < Q; ++j) {
        const double c[3] = {(double)cx(j), (double)cy(j), (double)cz(j)};
        const double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
        const double lw = (double)lam[(size_t)j * g.S + s] * wd(j) * rho;
        for (int d = 0; d < 3; ++d) out[d] += lw * (3.0 * c[d] + 9.0 * cu * c[d] - 3.0 * u[d]);
    }
    for (int d = 0; d < 3; ++d) du0[(size_t)d * g.S + s] = out[d];
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side: forward record with checkpoints, reverse sweep over segments.
// ---------------------------------------------------------------------------
struct AdjointTape {
    int nsteps = 0, every = 0, window = 0, nb = 0;
    double target = 0.0, ubar = 0.0, loss = 0.0;
    long long version = -1;         // ctx state version at the end of the forward
    size_t fbytes = 0;
    std::vector<void*> ck_f;        // populations at steps 0, every, 2 every, ...
    std::vector<BubbleSnap*> ck_b;  // bubble state there
    int cur0 = 0;                   // buffer index at step 0
    double* uz = nullptr;           // [nsteps * nb] u_b,z after each step
    double* lossbuf = nullptr;      // {ubar, loss}
    void* final_f = nullptr;        // state after the forward, restored after backward
    BubbleSnap* final_b = nullptr;
    int final_cur = 0;
};

void adjoint_free(lbm_ctx* c) {
    AdjointTape* t = c->adj;
    if (!t) return;
    for (void* p : t->ck_f) dfree(c, p);
    for (BubbleSnap* p : t->ck_b) dfree(c, p);
    dfree(c, t->uz);
    dfree(c, t->lossbuf);
    dfree(c, t->final_f);
    dfree(c, t->final_b);
    delete t;
    c->adj = nullptr;
}

extern "C" int lbm_adj_forward(lbm_ctx* c, int nsteps, int checkpoint_every, int window,
                               double target, double* loss) {
    if (!c || nsteps < 1 || checkpoint_every < 1 || window < 1 || window > nsteps)
        return LBM_ERR_ARG;
    int rc = ensure_device(c);
    if (rc) return rc;
    const bool timing = c->timing;   // forward launches are not timed
    c->timing = false;
    struct Restore { lbm_ctx* c; bool t; ~Restore() { c->timing = t; } } restore_timing{c, timing};
    if (c->storage != LBM_STORE_F32)
        return fail(c, LBM_ERR_STATE, "the adjoint needs FP32 population storage");
    if (c->walls & WALL_TOP_FREE)
        return fail(c, LBM_ERR_STATE, "the adjoint covers no-slip and periodic faces only");
    if (c->p.forces != 0)
        return fail(c, LBM_ERR_STATE, "the adjoint covers buoyancy, drag and virtual mass only");
    if (c->p.mapping != LBM_MAP_CELL || c->p.reaction != LBM_REACTION_DRAG_LIFT)
        return fail(c, LBM_ERR_STATE, "the adjoint covers the cell-integral map and the "
                    "-(F_D + F_L) reaction only");
    const int nb = c->bub.nb;
    if (nb < 1 || nb > ADJ_MAX_BUBBLES)
        return fail(c, LBM_ERR_STATE, "the adjoint needs 1..%d bubbles", ADJ_MAX_BUBBLES);
    if (c->p.substeps > ADJ_MAX_SUB)
        return fail(c, LBM_ERR_STATE, "the adjoint supports at most %d sub-steps", ADJ_MAX_SUB);
    if (c->unstable) return fail(c, LBM_ERR_UNSTABLE, "liquid solver is unstable (sticky)");
    adjoint_free(c);
    AdjointTape* t = new AdjointTape();
    c->adj = t;
    t->nsteps = nsteps;
    t->every = checkpoint_every;
    t->window = window;
    t->target = target;
    t->nb = nb;
    const Geo g = geo_of(c);
    t->fbytes = (size_t)Q * (size_t)g.S * sizeof(float);
    t->uz = (double*)dalloc(c, sizeof(double) * (size_t)nsteps * nb);
    t->lossbuf = (double*)dalloc(c, sizeof(double) * 2);
    t->final_f = dalloc(c, t->fbytes);
    t->final_b = (BubbleSnap*)dalloc(c, sizeof(BubbleSnap) * nb);
    if (!t->uz || !t->lossbuf || !t->final_f || !t->final_b) {
        adjoint_free(c);
        return fail(c, LBM_ERR_ALLOC, "adjoint tape");
    }
    const int sb = (nb + 127) / 128;
    cudaStream_t s = c->stream;
    t->cur0 = c->cur;
    for (int n = 0; n < nsteps; ++n) {
        if (n % checkpoint_every == 0) {
            void* ck = dalloc(c, t->fbytes);
            BubbleSnap* cb = (BubbleSnap*)dalloc(c, sizeof(BubbleSnap) * nb);
            if (!ck || !cb) {
                dfree(c, ck);
                dfree(c, cb);
                adjoint_free(c);
                return fail(c, LBM_ERR_ALLOC, "checkpoint of %zu bytes", t->fbytes);
            }
            t->ck_f.push_back(ck);
            t->ck_b.push_back(cb);
            LBM_CUDA(cudaMemcpyAsync(ck, c->f[c->cur], t->fbytes, cudaMemcpyDeviceToDevice, s),
                     "checkpoint");
            k_snapshot<<<sb, 128, 0, s>>>(c->bub, cb, 0);
            c->launches += 1;
        }
        rc = enqueue_one_step(c);
        if (rc) return rc;
        k_record_uz<<<sb, 128, 0, s>>>(c->bub, t->uz + (size_t)n * nb);
        c->launches += 1;
    }
    LBM_CUDA(cudaMemcpyAsync(t->final_f, c->f[c->cur], t->fbytes, cudaMemcpyDeviceToDevice, s),
             "final state");
    k_snapshot<<<sb, 128, 0, s>>>(c->bub, t->final_b, 0);
    t->final_cur = c->cur;
    k_adj_loss<<<1, 32, 0, s>>>(t->uz, nsteps, nb, window, target, t->lossbuf);
    c->launches += 2;   // the final snapshot and the loss
    LBM_CUDA(cudaGetLastError(), "adjoint forward");
    rc = finish_steps(c);
    if (rc) return rc;
    double lb[2];
    LBM_CUDA(cudaMemcpy(lb, t->lossbuf, sizeof(lb), cudaMemcpyDeviceToHost), "loss");
    t->ubar = lb[0];
    t->loss = lb[1];
    if (loss) *loss = t->loss;
    return LBM_OK;
}

extern "C" int lbm_adj_backward(lbm_ctx* c, double dloss, double* grad_drag_scale,
                                double* grad_diam, double* grad_u0) {
    if (!c) return LBM_ERR_ARG;
    AdjointTape* t = c->adj;
    if (!t) return fail(c, LBM_ERR_STATE, "lbm_adj_backward needs a preceding lbm_adj_forward");
    const Geo g = geo_of(c);
    const CollideParams cp = collide_params(c);
    const int nb = t->nb, N = t->nsteps, K = t->every;
    cudaStream_t s = c->stream;
    const int sb = (nb + 127) / 128;
    // Scratch: the segment's populations and bubble snapshots, two adjoint fields.
    const size_t fb = t->fbytes;
    std::vector<void*> seg_f(K, nullptr);
    for (int k = 0; k < K; ++k) seg_f[k] = dalloc(c, fb);
    BubbleSnap* seg_pre = (BubbleSnap*)dalloc(c, sizeof(BubbleSnap) * (size_t)K * nb);
    BubbleSnap* seg_post = (BubbleSnap*)dalloc(c, sizeof(BubbleSnap) * (size_t)K * nb);
    float* lam[2] = {(float*)dalloc(c, fb), (float*)dalloc(c, fb)};
    BubbleAdj* adj = (BubbleAdj*)dalloc(c, sizeof(BubbleAdj) * nb);
    // grads[0, nb): dL/dd_b; grads[nb, 2 nb): each bubble's part of dL/ds_D
    // (summed over the bubbles in order at the end); lul: the interpolation
    // seed phase B hands to phase C.
    double* grads = (double*)dalloc(c, sizeof(double) * 2 * (size_t)nb);
    double* lul = (double*)dalloc(c, sizeof(double) * 3 * (size_t)nb);
    double* du0 = grad_u0 ? (double*)dalloc(c, sizeof(double) * 3 * (size_t)g.S) : nullptr;
    auto release = [&]() {
        for (void* p : seg_f) dfree(c, p);
        dfree(c, seg_pre);
        dfree(c, seg_post);
        dfree(c, lam[0]);
        dfree(c, lam[1]);
        dfree(c, adj);
        dfree(c, grads);
        dfree(c, lul);
        dfree(c, du0);
    };
    bool ok = seg_pre && seg_post && lam[0] && lam[1] && adj && grads && lul && (!grad_u0 || du0);
    for (void* p : seg_f) ok = ok && p;
    if (!ok) {
        release();
        return fail(c, LBM_ERR_ALLOC, "adjoint segment storage");
    }
    AdjConst ac;
    ac.nu = (2.0 / c->omega - 1.0) / 6.0;   // Eq. 9
    ac.dt_l = 1.0;
    ac.dt_b = 1.0 / c->p.substeps;
    ac.sn_coeff = c->p.sn_coeff;
    ac.sn_exp = c->p.sn_exp;
    ac.width_factor = c->p.width_factor;
    ac.drag_scale = c->p.drag_scale;
    ac.rho_l = c->p.rho_l;
    ac.rho_b = c->p.rho_ratio * c->p.rho_l;
    ac.g = c->p.g;
    ac.sigma = c->p.sigma;
    ac.c_am = c->p.c_added_mass;
    ac.substeps = c->p.substeps;
    ac.two_way = c->p.two_way;
    const double seed = dloss * 2.0 * (t->ubar - t->target) / ((double)t->window * nb);
    // Kernel timing covers the adjoint sweep only, not the recomputed forward.
    const bool time_adjoint = c->timing;
    c->timing = false;
    struct Restore { lbm_ctx* c; bool t; ~Restore() { c->timing = t; } } restore_timing{c, time_adjoint};
    int lc = 0;   // lam[lc] holds Lambda^{n+1}
    int rc = LBM_OK;
    auto step_rc = [&](cudaError_t e, const char* what) {
        if (e != cudaSuccess && rc == LBM_OK) rc = cuda_fail(c, e, what);
    };
    step_rc(cudaMemsetAsync(lam[lc], 0, fb, s), "lambda");
    step_rc(cudaMemsetAsync(adj, 0, sizeof(BubbleAdj) * nb, s), "bubble adjoint");
    step_rc(cudaMemsetAsync(grads, 0, sizeof(double) * 2 * (size_t)nb, s), "grads");
    // Phases A and B of the bubble adjoint run on a second stream alongside
    // the liquid adjoint; phase C joins both.
    cudaStream_t s2 = nullptr;
    cudaEvent_t ev_in = nullptr, ev_ab = nullptr;
    step_rc(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking), "adjoint stream");
    step_rc(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming), "event");
    step_rc(cudaEventCreateWithFlags(&ev_ab, cudaEventDisableTiming), "event");
    struct Side {
        cudaStream_t& s2;
        cudaEvent_t& a;
        cudaEvent_t& b;
        ~Side() {
            if (s2) {
                cudaStreamSynchronize(s2);
                cudaStreamDestroy(s2);
            }
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } side{s2, ev_in, ev_ab};
    const unsigned blocks = (unsigned)((g.S + 127) / 128);
    const int nseg = (N + K - 1) / K;
    for (int seg = nseg - 1; seg >= 0 && rc == LBM_OK; --seg) {
        const int n0 = seg * K, n1 = std::min(N, n0 + K);
        // Recompute the segment forward from its checkpoint.  Step n reads its
        // populations from slot n - n0 and writes slot n - n0 + 1 directly, so
        // no state is copied per step; the last step writes into a context
        // buffer, which the final restore overwrites.
        void* const f_ctx[2] = {c->f[0], c->f[1]};
        step_rc(cudaMemcpyAsync(seg_f[0], t->ck_f[seg], fb, cudaMemcpyDeviceToDevice, s), "restore");
        k_restore<<<sb, 128, 0, s>>>(c->bub, t->ck_b[seg]);
        c->launches += 1;
        c->cover_valid = false;
        guard_invalidate(c);
        for (int n = n0; n < n1 && rc == LBM_OK; ++n) {
            c->cur = 0;
            c->f[0] = seg_f[n - n0];
            c->f[1] = n + 1 < n1 ? seg_f[n + 1 - n0] : f_ctx[0];
            k_snapshot<<<sb, 128, 0, s>>>(c->bub, seg_pre + (size_t)(n - n0) * nb, 0);
            int r2 = enqueue_one_step(c);
            if (r2) rc = r2;
            k_snapshot<<<sb, 128, 0, s>>>(c->bub, seg_post + (size_t)(n - n0) * nb, 1);
            c->launches += 2;   // the two snapshots around the recomputed step
        }
        c->f[0] = f_ctx[0];
        c->f[1] = f_ctx[1];
        // Reverse through the segment.
        for (int n = n1 - 1; n >= n0 && rc == LBM_OK; --n) {
            const float* fn = (const float*)seg_f[n - n0];
            const BubbleSnap* pre = seg_pre + (size_t)(n - n0) * nb;
            const BubbleSnap* post = seg_post + (size_t)(n - n0) * nb;
            cudaEvent_t e1 = nullptr;
            if (time_adjoint) {
                if (c->events_used == c->events.size()) {
                    cudaEvent_t ea, eb;
                    step_rc(cudaEventCreate(&ea), "event");
                    step_rc(cudaEventCreate(&eb), "event");
                    c->events.emplace_back(ea, eb);
                }
                step_rc(cudaEventRecord(c->events[c->events_used].first, s), "event");
                e1 = c->events[c->events_used].second;
                ++c->events_used;
            }
            const double ls = n >= N - t->window ? seed : 0.0;
            step_rc(cudaEventRecord(ev_in, s), "event");
            step_rc(cudaStreamWaitEvent(s2, ev_in, 0), "event wait");
            k_adj_bubbles_ab<<<nb, ADJ_THREADS, 0, s2>>>(fn, lam[lc], g, cp, pre, post, c->bub.d, nb,
                                                          ac, adj, grads + nb, grads, lul, ls);
            step_rc(cudaGetLastError(), "bubble adjoint");
            step_rc(cudaEventRecord(ev_ab, s2), "event");
            k_adj_liquid<<<blocks, 128, 0, s>>>(fn, lam[lc], lam[lc ^ 1], g, cp, post, nb, ac.two_way);
            if (e1) step_rc(cudaEventRecord(e1, s), "event");
            step_rc(cudaStreamWaitEvent(s, ev_ab, 0), "event wait");
            k_adj_bubbles_c<<<1, ADJ_THREADS, 0, s>>>(fn, lam[lc ^ 1], g, cp, pre, c->bub.d, nb, ac, adj,
                                                       grads, lul);
            step_rc(cudaGetLastError(), "adjoint step");
            c->launches += 3;
            lc ^= 1;
        }
    }
    if (rc == LBM_OK && du0) {
        k_adj_init<<<blocks, 128, 0, s>>>((const float*)t->ck_f[0], lam[lc], g, cp, du0);
        c->launches += 1;
        step_rc(cudaGetLastError(), "initial-field adjoint");
        step_rc(cudaMemcpyAsync(grad_u0, du0, sizeof(double) * 3 * (size_t)g.S, cudaMemcpyDeviceToHost, s),
                "du0");
    }
    std::vector<double> hg(2 * (size_t)nb, 0.0);
    if (rc == LBM_OK)
        step_rc(cudaMemcpyAsync(hg.data(), grads, sizeof(double) * 2 * (size_t)nb,
                                cudaMemcpyDeviceToHost, s),
                "grads");
    // Back to the state after the forward.
    c->cur = t->final_cur;
    step_rc(cudaMemcpyAsync(c->f[c->cur], t->final_f, fb, cudaMemcpyDeviceToDevice, s), "final");
    k_restore<<<sb, 128, 0, s>>>(c->bub, t->final_b);
    c->launches += 1;
    c->cover_valid = false;
    guard_invalidate(c);
    step_rc(cudaStreamSynchronize(s), "adjoint");
    if (s2) step_rc(cudaStreamSynchronize(s2), "adjoint side stream");
    release();
    if (rc) return rc;
    if (grad_drag_scale) {
        double sum = 0.0;
        for (int b = 0; b < nb; ++b) sum += hg[nb + b];
        *grad_drag_scale = sum;
    }
    if (grad_diam)
        for (int b = 0; b < nb; ++b) grad_diam[b] = hg[b];
    return LBM_OK;
}
