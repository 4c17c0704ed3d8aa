// Fused collide-stream sweep (one liquid step of Sec. 2.2 with the bubble
// reaction force of Sec. 3.2).
//
// One thread per lattice node, pull scheme on two structure-of-arrays buffers:
// the thread gathers the 19 populations arriving at its node (Eq. 16 with
// half-way bounce-back, Sec. 3.3), gathers the node's force Phi from the
// bubbles binned to its tile (Eq. 21, fixed order, no atomics), applies the
// first forcing (Eq. 13), BGK collision towards Eq. 6 (Eq. 14) and the second
// forcing with the Guo term (Eq. 12, 15), and writes the post-collision
// populations of its own node.  All arithmetic is FP32 on populations shifted
// by w_j rho0.
//
// The sweep is bound by issue as much as by HBM, so the common case is kept
// short: nodes away from the box faces address their 19 sources with one
// 32-bit offset each, tiles without bubbles skip the forcing terms, and each
// pair of opposite directions shares its equilibrium terms.
#include <climits>
#include "lbm_device.cuh"

namespace lbm {

// Force Phi at node (x,y,z) from one bubble record: tensor product of cell
// integrals (Eq. 19) times psi_b / normalisation.
__device__ __forceinline__ void add_bubble_force(const BubbleRec& r, const Geo& g, int x, int y,
                                                 int z, float& Fx, float& Fy, float& Fz) {
    float rx = (float)(x - r.ax) + 0.5f - r.fx;
    float ry = (float)(y - r.ay) + 0.5f - r.fy;
    float rz = (float)(z - r.az) + 0.5f - r.fz;
    if (!(g.walls & 0x01)) {
        if (rx > 0.5f * g.nx) rx -= (float)g.nx;
        else if (rx < -0.5f * g.nx) rx += (float)g.nx;
    }
    if (!(g.walls & 0x04)) {
        if (ry > 0.5f * g.ny) ry -= (float)g.ny;
        else if (ry < -0.5f * g.ny) ry += (float)g.ny;
    }
    if (!(g.walls & 0x10)) {
        if (rz > 0.5f * g.nz) rz -= (float)g.nz;
        else if (rz < -0.5f * g.nz) rz += (float)g.nz;
    }
    float wx = cell_poly(rx * r.inv_n, r.h);
    if (wx == 0.0f) return;
    float wy = cell_poly(ry * r.inv_n, r.h);
    if (wy == 0.0f) return;
    float wz = cell_poly(rz * r.inv_n, r.h);
    float w = wx * wy * wz;
    Fx = fmaf(w, r.px, Fx);
    Fy = fmaf(w, r.py, Fy);
    Fz = fmaf(w, r.pz, Fz);
}

// Offset of the source of direction J from the receiving node, x fastest.
template <int J>
__device__ __forceinline__ unsigned src_delta(unsigned nx, unsigned nxy) {
    return (unsigned)cx(J) + (unsigned)cy(J) * nx + (unsigned)cz(J) * nxy;
}

// Pull-gather of raw stored values for a node whose y and z neighbours are
// inside the box (all rows but the first and last of each face).  Indices are
// 32-bit (19 S < 2^32 is enforced at creation): the source of J is
// J*S + site - (c_J . (1, nx, nx ny)).  A node on an x face takes its
// x-crossing populations from the opposite plane at its own site (wall) or
// from the other end of the row (periodic), by selects rather than branches.
template <int ST, int J>
__device__ __forceinline__ float pull_raw(const typename Store<ST>::T* __restrict__ f,
                                          unsigned S, unsigned site, unsigned nx, unsigned nxy,
                                          bool xlo, bool xhi, bool wallx) {
    unsigned idx = (unsigned)J * S + site - src_delta<J>(nx, nxy);
    if (cx(J) == 1 && xlo) idx = wallx ? (unsigned)opp(J) * S + site : idx + nx;
    if (cx(J) == -1 && xhi) idx = wallx ? (unsigned)opp(J) * S + site : idx - nx;
    return Store<ST>::load_raw(f + idx);
}

template <int ST>
__device__ __forceinline__ void gather_rows(const typename Store<ST>::T* __restrict__ f,
                                            unsigned S, unsigned site, unsigned nx,
                                            unsigned nxy, bool xlo, bool xhi, bool wallx,
                                            float rv[Q]) {
#define LBM_PULL(J) rv[J] = pull_raw<ST, J>(f, S, site, nx, nxy, xlo, xhi, wallx)
    LBM_PULL(0); LBM_PULL(1); LBM_PULL(2); LBM_PULL(3); LBM_PULL(4);
    LBM_PULL(5); LBM_PULL(6); LBM_PULL(7); LBM_PULL(8); LBM_PULL(9);
    LBM_PULL(10); LBM_PULL(11); LBM_PULL(12); LBM_PULL(13); LBM_PULL(14);
    LBM_PULL(15); LBM_PULL(16); LBM_PULL(17); LBM_PULL(18);
#undef LBM_PULL
}

// General pull-gather of raw values (any node, any walls).
template <int ST, int J>
__device__ __forceinline__ float pull_raw_any(const typename Store<ST>::T* __restrict__ f,
                                              const Geo& g, int x, int y, int z) {
    int plane, idx;
    pull_source<J>(g, x, y, z, plane, idx);
    return Store<ST>::load_raw(f + (size_t)plane * (size_t)g.S + idx);
}

template <int ST>
__device__ __forceinline__ void gather_any(const typename Store<ST>::T* __restrict__ f,
                                           const Geo& g, int x, int y, int z, float rv[Q]) {
#define LBM_PULL(J) rv[J] = pull_raw_any<ST, J>(f, g, x, y, z)
    LBM_PULL(0); LBM_PULL(1); LBM_PULL(2); LBM_PULL(3); LBM_PULL(4);
    LBM_PULL(5); LBM_PULL(6); LBM_PULL(7); LBM_PULL(8); LBM_PULL(9);
    LBM_PULL(10); LBM_PULL(11); LBM_PULL(12); LBM_PULL(13); LBM_PULL(14);
    LBM_PULL(15); LBM_PULL(16); LBM_PULL(17); LBM_PULL(18);
#undef LBM_PULL
}

// One pair of opposite directions (J, J+1 = opp(J)) in raw storage units.
// Eq. 6 is split into its even part (shared by the pair) and odd part (sign
// flips); g^eq_j / w_j = base + 9/2 rho cu^2 +- 3 rho cu.  BGK relaxation
// (Eq. 14) is r' = (1 - omega) r + C [omega g^eq / w], and the Guo term of
// Eq. 12 adds C pref [(9 cu cF - 3 u.F) +- 3 cF], where C = w_J for FP32
// storage and C = scale for the 16-bit formats (r = g scale / w).
template <int ST, int J, bool FORCED>
__device__ __forceinline__ void relax_pair(typename Store<ST>::T* __restrict__ fout, unsigned S,
                                           unsigned site, const float rv[Q], float base,
                                           float rho, float ux, float uy, float uz, float Fx,
                                           float Fy, float Fz, float uF,
                                           const CollideParams& cp) {
    const float C = Store<ST>::kScaled ? cp.scale : wf(J);
    const float cu = (float)cx(J) * ux + (float)cy(J) * uy + (float)cz(J) * uz;
    float even = cp.omega * fmaf(4.5f * rho * cu, cu, base);
    float odd = cp.omega * 3.0f * rho * cu;
    if (FORCED) {
        const float cF = (float)cx(J) * Fx + (float)cy(J) * Fy + (float)cz(J) * Fz;
        even = fmaf(cp.pref, 9.0f * cu * cF - 3.0f * uF, even);
        odd = fmaf(cp.pref, 3.0f * cF, odd);
    }
    const float om1 = 1.0f - cp.omega;
    Store<ST>::store_raw(fout + ((unsigned)J * S + site), fmaf(om1, rv[J], C * (even + odd)));
    Store<ST>::store_raw(fout + ((unsigned)(J + 1) * S + site),
                         fmaf(om1, rv[J + 1], C * (even - odd)));
}

template <int ST, bool FORCED>
__device__ __forceinline__ void collide_store(typename Store<ST>::T* __restrict__ fout,
                                              unsigned S, unsigned site, const float rv[Q],
                                              float Fx, float Fy, float Fz,
                                              const CollideParams& cp, int* flag) {
    // Eq. 10 / Eq. 13 moments of g = r k, k = 1 (FP32) or w_j / scale
    // (16-bit); sum_j w_j c_j = 0 so the shift drops out of the momentum.
    const float s_rest = rv[0];
    const float s_axis = (rv[1] + rv[2]) + (rv[3] + rv[4]) + (rv[5] + rv[6]);
    const float s_edge = ((rv[7] + rv[8]) + (rv[9] + rv[10])) + ((rv[11] + rv[12]) + (rv[13] + rv[14])) +
                         ((rv[15] + rv[16]) + (rv[17] + rv[18]));
    const float ax_x = rv[1] - rv[2], ax_y = rv[3] - rv[4], ax_z = rv[5] - rv[6];
    const float ed_x = (rv[7] - rv[8]) + (rv[9] - rv[10]) + (rv[11] - rv[12]) + (rv[13] - rv[14]);
    const float ed_y = (rv[7] - rv[8]) + (rv[10] - rv[9]) + (rv[15] - rv[16]) + (rv[17] - rv[18]);
    const float ed_z = (rv[11] - rv[12]) + (rv[14] - rv[13]) + (rv[15] - rv[16]) + (rv[18] - rv[17]);
    float drho, jx, jy, jz;
    if (Store<ST>::kScaled) {
        const float k0 = wf(0) * cp.inv_scale, ka = wf(1) * cp.inv_scale, ke = wf(7) * cp.inv_scale;
        drho = fmaf(k0, s_rest, fmaf(ka, s_axis, ke * s_edge));
        jx = fmaf(ka, ax_x, ke * ed_x);
        jy = fmaf(ka, ax_y, ke * ed_y);
        jz = fmaf(ka, ax_z, ke * ed_z);
    } else {
        drho = s_rest + s_axis + s_edge;
        jx = ax_x + ed_x;
        jy = ax_y + ed_y;
        jz = ax_z + ed_z;
    }
    const float rho = cp.rho0 + drho;
    const float inv_rho = 1.0f / rho;
    float ux, uy, uz;
    if (FORCED) {
        ux = fmaf(0.5f, Fx, jx) * inv_rho;
        uy = fmaf(0.5f, Fy, jy) * inv_rho;
        uz = fmaf(0.5f, Fz, jz) * inv_rho;
    } else {
        ux = jx * inv_rho;
        uy = jy * inv_rho;
        uz = jz * inv_rho;
    }
    const float usq = ux * ux + uy * uy + uz * uz;
    if (!(usq < 0.09f)) atomicOr(flag, 1);   // non-finite or beyond |u| = 0.3
    const float uF = FORCED ? (ux * Fx + uy * Fy + uz * Fz) : 0.0f;
    // Common part of g^eq_j / w_j: drho - 3/2 rho u^2.
    const float base = fmaf(-1.5f * rho, usq, drho);
    float e0 = cp.omega * base;
    if (FORCED) e0 = fmaf(cp.pref, -3.0f * uF, e0);   // Eq. 12 with c_0 = 0
    const float C0 = Store<ST>::kScaled ? cp.scale : wf(0);
    Store<ST>::store_raw(fout + site, fmaf(1.0f - cp.omega, rv[0], C0 * e0));
#define LBM_PAIR(J) relax_pair<ST, J, FORCED>(fout, S, site, rv, base, rho, ux, uy, uz, Fx, Fy, Fz, uF, cp)
    LBM_PAIR(1); LBM_PAIR(3); LBM_PAIR(5); LBM_PAIR(7); LBM_PAIR(9);
    LBM_PAIR(11); LBM_PAIR(13); LBM_PAIR(15); LBM_PAIR(17);
#undef LBM_PAIR
}

template <int ST>
__global__ void __launch_bounds__(TX * TY, 8)
k_collide_stream(const typename Store<ST>::T* __restrict__ fin,
                 typename Store<ST>::T* __restrict__ fout, Geo g, CollideParams cp,
                 const int* __restrict__ tile_start, const int* __restrict__ tile_count,
                 const int* __restrict__ items, int cap, const BubbleRec* __restrict__ recs,
                 int nb, int* __restrict__ flag) {
    __shared__ BubbleRec srec[TX * TY];
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    const int z = blockIdx.z;
    const bool inside = (x < g.nx) && (y < g.ny);

    float Fx = 0.0f, Fy = 0.0f, Fz = 0.0f;
    bool forced = false;   // uniform over the CTA
    if (tile_count != nullptr) {
        const int t = ((z / TZ) * g.nty + blockIdx.y) * g.ntx + blockIdx.x;
        const int n_t = tile_count[t];
        if (n_t > 0) {
            forced = true;
            const int beg = tile_start[t];
            const int end = min(beg + n_t, cap);
            const int tid = threadIdx.y * TX + threadIdx.x;
            for (int c0 = beg; c0 < end; c0 += TX * TY) {
                const int cnt = min(TX * TY, end - c0);
                __syncthreads();
                if (tid < cnt) {
                    const int id = items[c0 + tid];
                    if (id >= 0 && id < nb) srec[tid] = recs[id];
                    else srec[tid] = BubbleRec{0, 0, 0, 0, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                }
                __syncthreads();
                if (inside)
                    for (int k = 0; k < cnt; ++k) add_bubble_force(srec[k], g, x, y, z, Fx, Fy, Fz);
            }
        }
    }
    if (!inside) return;

    const unsigned S = (unsigned)g.S;
    const unsigned nx = (unsigned)g.nx, nxy = (unsigned)g.nx * (unsigned)g.ny;
    const unsigned site = (unsigned)z * nxy + (unsigned)y * nx + (unsigned)x;
    float rv[Q];
    // Rows away from the y and z faces (uniform over a warp, which is one row).
    if (y > 0 && y < g.ny - 1 && z > 0 && z < g.nz - 1)
        gather_rows<ST>(fin, S, site, nx, nxy, x == 0, x == g.nx - 1, (g.walls & 0x01) != 0, rv);
    else
        gather_any<ST>(fin, g, x, y, z, rv);

    if (forced) collide_store<ST, true>(fout, S, site, rv, Fx, Fy, Fz, cp, flag);
    else collide_store<ST, false>(fout, S, site, rv, 0.0f, 0.0f, 0.0f, cp, flag);
}

// ---------------------------------------------------------------------------
// Two nodes per thread (even nx).  Each thread owns the x-pair (x0, x0 + 1),
// x0 even, so every plane row is read and written with aligned 2-wide vector
// accesses (float2, half2, bfloat162) and the collision runs on packed FP32
// pairs (FFMA2 / FADD2 / FMUL2).  A CTA is 16 x 4 x 2 threads = 32 x 4 x 2
// nodes, inside one binning tile.
// ---------------------------------------------------------------------------
// Resident CTAs per SM the register budget is sized for: FP32 rows move twice
// the bytes per thread and keep more registers; the 16-bit formats need more
// warps in flight to cover memory latency.  Measured on GB300 (FP16 sweep,
// 256x256x512, rows kept packed until use): 8 CTAs (64 registers) 0.439 ms,
// 7 CTAs 0.448 ms, 9 CTAs 0.461 ms.
#ifndef LBM_PAIR_MINB_16
#define LBM_PAIR_MINB_16 8
#endif
template <int ST> struct PairOccupancy {
    static constexpr int kMinBlocks = ST == 0 ? 6 : LBM_PAIR_MINB_16;
};
constexpr int PX = TX / 2;   // threads along x
// Bubbles staged per pass of the sweep's force gather (records and per-axis
// weight tables in shared memory).
constexpr int FORCE_CHUNK = 32;
constexpr int PZ = SWEEP_PZ;      // z-planes per CTA (divides TZ)
static_assert(TZ % PZ == 0, "a CTA's z-planes must lie in one binning tile");


// Force of one bubble record on the pair (x0, x0 + 1) at (y, z), Eq. 19 and 21.
__device__ __forceinline__ void add_bubble_force_pair(const BubbleRec& r, const Geo& g, int x0,
                                                      int y, int z, float2& Fx, float2& Fy,
                                                      float2& Fz) {
    float ry = (float)(y - r.ay) + 0.5f - r.fy;
    float rz = (float)(z - r.az) + 0.5f - r.fz;
    if (!(g.walls & 0x04)) {
        if (ry > 0.5f * g.ny) ry -= (float)g.ny;
        else if (ry < -0.5f * g.ny) ry += (float)g.ny;
    }
    if (!(g.walls & 0x10)) {
        if (rz > 0.5f * g.nz) rz -= (float)g.nz;
        else if (rz < -0.5f * g.nz) rz += (float)g.nz;
    }
    const float wy = cell_poly(ry * r.inv_n, r.h);
    if (wy == 0.0f) return;
    const float wyz = wy * cell_poly(rz * r.inv_n, r.h);
    if (wyz == 0.0f) return;
    float w[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        float rx = (float)(x0 + k - r.ax) + 0.5f - r.fx;
        if (!(g.walls & 0x01)) {
            if (rx > 0.5f * g.nx) rx -= (float)g.nx;
            else if (rx < -0.5f * g.nx) rx += (float)g.nx;
        }
        w[k] = cell_poly(rx * r.inv_n, r.h) * wyz;
    }
    const float2 wv = make_float2(w[0], w[1]);
    Fx = fma2(wv, f2(r.px), Fx);
    Fy = fma2(wv, f2(r.py), Fy);
    Fz = fma2(wv, f2(r.pz), Fz);
}

// c_j . v for direction J (J odd; J + 1 is its opposite), written with adds
// only: no multiply by +-1.
template <int J>
__device__ __forceinline__ float2 c_dot(float2 vx, float2 vy, float2 vz) {
    constexpr int X = cx(J), Y = cy(J), Z = cz(J);
    static_assert((J & 1) && (X == 1 || (X == 0 && Y == 1) || (X == 0 && Y == 0 && Z == 1)),
                  "odd directions lead with a +1 component");
    if (Y == 0 && Z == 0) return vx;                    // J = 1 (+x)
    if (X == 0 && Z == 0) return vy;                    // J = 3 (+y)
    if (X == 0 && Y == 0) return vz;                    // J = 5 (+z)
    if (Z == 0) return Y > 0 ? add2(vx, vy) : sub2(vx, vy);
    if (Y == 0) return Z > 0 ? add2(vx, vz) : sub2(vx, vz);
    return Z > 0 ? add2(vy, vz) : sub2(vy, vz);
}

// Per-class coefficients of the relaxation in stored units: with K = C omega
// (C = w_j for FP32, the storage scale for 16 bits), the post-collision value
// of J and of its opposite is
//   (1 - omega) r_{J or J+1} + K base + 4.5 K rho (c.u)^2  +-  3 K rho (c.u)
// (Eq. 6 and 14 with f^eq - w rho0 written around base = drho - 1.5 rho u^2).
struct RelaxK {
    float2 base, r45, r3;
};

__device__ __forceinline__ RelaxK relax_k(float K, float2 base, float2 rho) {
    return RelaxK{mul2(f2(K), base), mul2(f2(4.5f * K), rho), mul2(f2(3.0f * K), rho)};
}

// Where a collided pair goes: the pair kernels store it 2-wide in plane J at
// site0.
template <int ST>
struct PairStore {
    typename Store<ST>::T* fout;
    unsigned S, site0;
    bool store;
    template <int J>
    __device__ __forceinline__ void put(float2 v) const {
        if (store) Vec2<ST>::store(fout + ((unsigned)J * S + site0), v);
    }
};

template <int ST, int J, bool FORCED, class Sink>
__device__ __forceinline__ void relax_pair2(Sink& sink, const typename Raw2<ST>::T rv[Q],
                                            const RelaxK& k,
                                            float2 ux, float2 uy, float2 uz, float2 Fx, float2 Fy,
                                            float2 Fz, float2 uF, const CollideParams& cp) {
    const float2 cu = c_dot<J>(ux, uy, uz);
    float2 even = fma2(mul2(k.r45, cu), cu, k.base);
    float2 odd = mul2(k.r3, cu);
    if (FORCED) {
        // Guo term (Eq. 15), (1 - omega/2) w_j [3 (c - u) + 9 (c.u) c] . F
        const float C = Store<ST>::kScaled ? cp.scale : wf(J);
        const float2 cF = c_dot<J>(Fx, Fy, Fz);
        even = fma2(f2(C * cp.pref), fma2(mul2(f2(9.0f), cu), cF, mul2(f2(-3.0f), uF)), even);
        odd = fma2(f2(3.0f * C * cp.pref), cF, odd);
    }
    const float2 om1 = f2(1.0f - cp.omega);
    sink.template put<J>(fma2(om1, Raw2<ST>::widen(rv[J]), add2(even, odd)));
    sink.template put<J + 1>(fma2(om1, Raw2<ST>::widen(rv[J + 1]), sub2(even, odd)));
}

// Collision of one x-pair of nodes (Eq. 13, 6, 14, 12, 15) from its
// pre-collision values rr (stored units, as loaded); `live` pairs take part in
// the stability flag.
template <int ST, bool FORCED, class Sink>
__device__ __forceinline__ void collide_pair(Sink& sink, const typename Raw2<ST>::T rr[Q],
                                             float2 Fx, float2 Fy, float2 Fz,
                                             const CollideParams& cp, int* flag, bool live) {
    float2 drho, jx, jy, jz;
    pair_moments<ST>(rr, cp, drho, jx, jy, jz);
    const float2 rho = add2(f2(cp.rho0), drho);
    const float2 inv_rho = make_float2(1.0f / rho.x, 1.0f / rho.y);
    float2 ux, uy, uz;
    if (FORCED) {
        ux = mul2(fma2(f2(0.5f), Fx, jx), inv_rho);
        uy = mul2(fma2(f2(0.5f), Fy, jy), inv_rho);
        uz = mul2(fma2(f2(0.5f), Fz, jz), inv_rho);
    } else {
        ux = mul2(jx, inv_rho);
        uy = mul2(jy, inv_rho);
        uz = mul2(jz, inv_rho);
    }
    const float2 usq = fma2(ux, ux, fma2(uy, uy, mul2(uz, uz)));
    if (live && !(usq.x < 0.09f && usq.y < 0.09f)) atomicOr(flag, 1);
    const float2 uF = FORCED ? fma2(ux, Fx, fma2(uy, Fy, mul2(uz, Fz))) : f2(0.0f);
    const float2 base = fma2(mul2(f2(-1.5f), rho), usq, drho);
    float2 e0 = mul2(f2(cp.omega), base);
    if (FORCED) e0 = fma2(f2(-3.0f * cp.pref), uF, e0);
    const float C0 = Store<ST>::kScaled ? cp.scale : wf(0);
    sink.template put<0>(fma2(f2(1.0f - cp.omega), Raw2<ST>::widen(rr[0]), mul2(f2(C0), e0)));
    // One coefficient class for the 16-bit formats (C = scale); FP32 has
    // the axis and the diagonal weights.
    const RelaxK ka = relax_k((Store<ST>::kScaled ? cp.scale : wf(1)) * cp.omega, base, rho);
    const RelaxK ke = Store<ST>::kScaled ? ka : relax_k(wf(7) * cp.omega, base, rho);
#define LBM_PAIR2(J, K) relax_pair2<ST, J, FORCED>(sink, rr, K, ux, uy, uz, Fx, Fy, Fz, uF, cp)
    LBM_PAIR2(1, ka); LBM_PAIR2(3, ka); LBM_PAIR2(5, ka); LBM_PAIR2(7, ke); LBM_PAIR2(9, ke);
    LBM_PAIR2(11, ke); LBM_PAIR2(13, ke); LBM_PAIR2(15, ke); LBM_PAIR2(17, ke);
#undef LBM_PAIR2
}

// Eq. 21 at the pair (x0, x0 + 1), (y, z) of a block whose tile lists n_t > 0
// bubbles, for long tile lists (many bubbles).  Every thread of the CTA calls
// it (it synchronises the CTA).
struct Force2 {
    float2 x, y, z;
};

template <int ST>
__device__ __forceinline__ Force2 gather_force_tab(const Geo& g, const int* __restrict__ tile_start,
                                                 const int* __restrict__ items, int cap,
                                                 const BubbleRec* __restrict__ recs, int nb,
                                                 int n_t, int bx, int by, int bz, int x0, int y,
                                                 int z, bool active, BubbleRec* srec, bool point) {
    float2 Fx = f2(0.0f), Fy = f2(0.0f), Fz = f2(0.0f);
    // Chunks of FB bubbles: the CTA first tabulates each bubble's per-axis
    // cell integrals over the block (TX columns, TY rows, PZ planes), then
    // every node forms wx (wy wz) from the tables.  Same products, zero test
    // and order as add_bubble_force_pair.
    constexpr int FB = FORCE_CHUNK, NAX = TX + TY + PZ;
    __shared__ float s_w[FB][NAX];   // x: [0, TX), y: [TX, TX + TY), z: the rest
    const int t = (((bz * PZ) / TZ) * g.nty + by) * g.ntx + bx;
    const int beg = __ldcg(tile_start + t);
    const int end = min(beg + n_t, cap);
    const int tid = (threadIdx.z * TY + threadIdx.y) * PX + threadIdx.x;
    constexpr int NT = PX * TY * PZ;
    const int xb0 = bx * TX, yb0 = by * TY, zb0 = bz * PZ;
    for (int c0 = beg; c0 < end; c0 += FB) {
        const int cnt = min(FB, end - c0);
        __syncthreads();
        if (tid < cnt) {
            const int id = __ldcg(items + c0 + tid);
            if (id >= 0 && id < nb) srec[tid] = load_rec(recs + id);
            else srec[tid] = BubbleRec{0, 0, 0, 0, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        }
        __syncthreads();
        // The mapping mode is the same for every bubble: one loop per mode.
        auto tabulate = [&](auto mode) {
            constexpr int PM = decltype(mode)::value;
            for (int e = tid; e < cnt * NAX; e += NT) {
                const int k = e / NAX, q = e - k * NAX;
                const BubbleRec& r = srec[k];
                if (q < TX)
                    s_w[k][q] = axis_weight<PM>(r, xb0 + q, r.ax, r.fx, g.nx, !(g.walls & 0x01));
                else if (q < TX + TY)
                    s_w[k][q] = axis_weight<PM>(r, yb0 + q - TX, r.ay, r.fy, g.ny, !(g.walls & 0x04));
                else
                    s_w[k][q] =
                        axis_weight<PM>(r, zb0 + q - TX - TY, r.az, r.fz, g.nz, !(g.walls & 0x10));
            }
        };
        // (FP32 keeps the one loop with the mode read per weight: its sweep
        // has the slack, and the smaller code measured faster.)
        if (ST == 0) tabulate(MapMode<MAP_ANY>{});
        else if (point) tabulate(MapMode<MAP_POINT>{});
        else tabulate(MapMode<MAP_CELL>{});
        __syncthreads();
        if (active) {
            const int xi = 2 * threadIdx.x, yi = TX + threadIdx.y, zi = TX + TY + threadIdx.z;
            for (int k = 0; k < cnt; ++k) {
                const float wyz = s_w[k][yi] * s_w[k][zi];
                if (wyz == 0.0f) continue;
                const float2 wv = make_float2(s_w[k][xi] * wyz, s_w[k][xi + 1] * wyz);
                const BubbleRec& r = srec[k];
                Fx = fma2(wv, f2(r.px), Fx);
                Fy = fma2(wv, f2(r.py), Fy);
                Fz = fma2(wv, f2(r.pz), Fz);
            }
        }
    }
    __syncthreads();   // srec and s_w are reused by the CTA's next block
    return Force2{Fx, Fy, Fz};
}

// One CTA's block of the sweep: x-pairs of 32 nodes, TY rows, PZV planes at
// block coordinates (bx, by, bz).  `srec` is the CTA's staging of bubble
// records; every thread of the CTA must call this with the same block.
template <int ST, bool TAB, int PZV = PZ>
__device__ __forceinline__ void sweep_block(const typename Store<ST>::T* __restrict__ fin,
                                            typename Store<ST>::T* __restrict__ fout,
                                            const Geo& g, const CollideParams& cp,
                                            const int* __restrict__ tile_start,
                                            const int* __restrict__ tile_count,
                                            const int* __restrict__ items, int cap,
                                            const BubbleRec* __restrict__ recs, int nb,
                                            int* __restrict__ flag, int bx, int by, int bz,
                                            BubbleRec* srec, const unsigned* safe = nullptr,
                                            unsigned epoch = 0, bool lead = false) {
    static_assert(TZ % PZV == 0 && (!TAB || PZV == PZ), "a block lies in one tile layer");
    const int x0 = bx * TX + 2 * threadIdx.x;
    const int y = by * TY + threadIdx.y;
    const int z = bz * PZV + threadIdx.z;
    const bool active = (x0 < g.nx) && (y < g.ny) && (z < g.nz);
    // Inactive threads gather at a valid node and store nothing.
    const int xa = active ? x0 : 0;
    const int ya = min(y, g.ny - 1), za = min(z, g.nz - 1);

    const int t = (((bz * PZV) / TZ) * g.nty + by) * g.ntx + bx;
    // Read before the population loads: in plain stream order the tile count;
    // overlapped with the bubble update, the guard tag of this z layer (written
    // by the update before, which has completed).  The launch's first CTA
    // (`lead`) never skips, so the sweep cannot complete before the update.
    int n_t = 0;
    bool skip = false;
    if (tile_count != nullptr) {
        if (safe == nullptr) n_t = __ldcg(tile_count + t);
        else skip = !lead && __ldcg(safe + (bz * PZV) / TZ) == epoch;
    }

    const unsigned S = (unsigned)g.S;
    const unsigned nx = (unsigned)g.nx, nxy = (unsigned)g.nx * (unsigned)g.ny;
    const unsigned site0 = (unsigned)za * nxy + (unsigned)ya * nx + (unsigned)xa;
    typename Raw2<ST>::T rv[Q];
    gather_pair<ST>(fin, g, xa, ya, za, rv);
    if (tile_count != nullptr && safe != nullptr && !skip) {
        // Overlapped, and the update before did not clear this layer: wait
        // for this step's update, then read its tile lists.
        pdl_wait();
        n_t = __ldcg(tile_count + t);
    }
    // The force gather (Eq. 21) runs after the population loads are issued,
    // so the tile-list lookup does not delay them.
    float2 Fx = f2(0.0f), Fy = f2(0.0f), Fz = f2(0.0f);
    const bool forced = n_t > 0;   // uniform over the CTA (one tile)
    if (forced && TAB) {
        const Force2 F = gather_force_tab<ST>(g, tile_start, items, cap, recs, nb, n_t, bx, by, bz,
                                          x0, y, z, active, srec, cp.point != 0);
        Fx = F.x;
        Fy = F.y;
        Fz = F.z;
    } else if (forced) {
        // Few bubbles per tile: each node evaluates its listed bubbles directly.
        const int beg = __ldcg(tile_start + t);
        const int end = min(beg + n_t, cap);
        const int tid = (threadIdx.z * TY + threadIdx.y) * PX + threadIdx.x;
        for (int c0 = beg; c0 < end; c0 += FORCE_CHUNK) {
            const int cnt = min(FORCE_CHUNK, end - c0);
            __syncthreads();
            if (tid < cnt) {
                const int id = __ldcg(items + c0 + tid);
                if (id >= 0 && id < nb) srec[tid] = load_rec(recs + id);
                else srec[tid] = BubbleRec{0, 0, 0, 0, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            }
            __syncthreads();
            if (active)
                for (int k = 0; k < cnt; ++k)
                    add_bubble_force_pair(srec[k], g, x0, y, z, Fx, Fy, Fz);
        }
        __syncthreads();   // srec is reused by the CTA's next block
    }

    PairStore<ST> sink{fout, S, site0, active};
    if (forced) collide_pair<ST, true>(sink, rv, Fx, Fy, Fz, cp, flag, active);
    else collide_pair<ST, false>(sink, rv, Fx, Fy, Fz, cp, flag, active);
}

// TAB: the force gather of long tile lists (per-axis weight tables).
template <int ST, bool TAB>
__global__ void __launch_bounds__(PX * TY * PZ, PairOccupancy<ST>::kMinBlocks)
k_collide_stream_pair(const typename Store<ST>::T* __restrict__ fin,
                      typename Store<ST>::T* __restrict__ fout, Geo g, CollideParams cp,
                      const int* tile_start, const int* tile_count, const int* items, int cap,
                      const BubbleRec* recs, int nb, int* __restrict__ flag,
                      const unsigned* safe, unsigned epoch, const int* zperm, ZSpan zs) {
    __shared__ BubbleRec srec[FORCE_CHUNK];
    // The next bubble update may be scheduled once every CTA of the sweep has
    // started; it waits for the sweep to complete before it reads anything.
    pdl_trigger();
    // z blocks in the order the bubble update before chose (cleared layers
    // first; written by an update that has completed), else the span's.
    int bz = zs.first + (int)blockIdx.z;
    if (bz >= zs.hole) bz += zs.skip;
    if (zperm != nullptr) bz = __ldcg(zperm + blockIdx.z);
    const bool lead = (blockIdx.x | blockIdx.y | blockIdx.z) == 0;
    sweep_block<ST, TAB>(fin, fout, g, cp, tile_start, tile_count, items, cap, recs, nb, flag,
                         blockIdx.x, blockIdx.y, bz, srec, safe, epoch, lead);
}

// Sweeps without tile lists (no two-way coupling, or the blocks no bubble
// force reaches): the same gather and the same collision without force
// (collide_pair<ST, false>, as k_collide_stream_pair runs it for a block with
// an empty list), in a kernel without the force-gather code: the 16-bit
// sweep runs about 3 % faster in it than in k_collide_stream_pair.
template <int ST>
__global__ void __launch_bounds__(PX * TY * PZ, PairOccupancy<ST>::kMinBlocks)
k_collide_stream_free(const typename Store<ST>::T* __restrict__ fin,
                      typename Store<ST>::T* __restrict__ fout, Geo g, CollideParams cp,
                      int* __restrict__ flag, ZSpan zs) {
    int bz = zs.first + (int)blockIdx.z;
    if (bz >= zs.hole) bz += zs.skip;
    const int x0 = blockIdx.x * TX + 2 * threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    const int z = bz * PZ + threadIdx.z;
    const bool active = (x0 < g.nx) && (y < g.ny) && (z < g.nz);
    // Inactive threads gather at a valid node and store nothing.
    const int xa = active ? x0 : 0;
    const int ya = min(y, g.ny - 1), za = min(z, g.nz - 1);
    const unsigned nx = (unsigned)g.nx, nxy = (unsigned)g.nx * (unsigned)g.ny;
    const unsigned site0 = (unsigned)za * nxy + (unsigned)ya * nx + (unsigned)xa;
    typename Raw2<ST>::T rv[Q];
    gather_pair<ST>(fin, g, xa, ya, za, rv);
    PairStore<ST> sink{fout, (unsigned)g.S, site0, active};
    collide_pair<ST, false>(sink, rv, f2(0.0f), f2(0.0f), f2(0.0f), cp, flag, active);
}

// ---------------------------------------------------------------------------
// Batched sweep: many independent columns in one persistent launch.  Each CTA
// takes work items -- `depth` consecutive z-blocks of one (column, x-block,
// y-block) -- from a global counter until all are done; columns keep their
// own size, omega and walls.  Results do not depend on which CTA takes which
// item.
// ---------------------------------------------------------------------------
constexpr int MAX_BATCH_COLUMNS = 256;

template <int ST, int PZV>
__global__ void __launch_bounds__(PX * TY * PZV, PairOccupancy<ST>::kMinBlocks * PZ / PZV)
k_collide_batch(const typename Store<ST>::T* __restrict__ fin,
                typename Store<ST>::T* __restrict__ fout, const BatchColumn* __restrict__ cols,
                int ncols, int total_items, int depth, int* __restrict__ work_counter,
                const int* __restrict__ tile_start, const int* __restrict__ tile_count,
                const int* __restrict__ items, int cap, const BubbleRec* __restrict__ recs,
                int nb, int* __restrict__ flag) {
    __shared__ BubbleRec srec[FORCE_CHUNK];
    __shared__ int s_item_base[MAX_BATCH_COLUMNS + 1];
    __shared__ int s_item;
    const int tid = (threadIdx.z * TY + threadIdx.y) * PX + threadIdx.x;
    for (int c = tid; c <= ncols; c += PX * TY * PZV)
        s_item_base[c] = c < ncols ? cols[c].item_base : total_items;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(work_counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total_items) break;
        int lo = 0, hi = ncols - 1;   // column with item_base <= item < next base
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_item_base[mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const BatchColumn& col = cols[lo];
        const int local = item - s_item_base[lo];
        const int bx = local % col.g.ntx;
        const int rest = local / col.g.ntx;
        const int by = rest % col.g.nty;
        const int bz0 = (rest / col.g.nty) * depth;
        const int nbz = (col.g.nz + PZV - 1) / PZV;
        for (int bz = bz0; bz < min(bz0 + depth, nbz); ++bz)
            sweep_block<ST, false, PZV>(fin + col.pop_offset, fout + col.pop_offset, col.g, col.cp,
                            tile_start + col.tile_base, tile_count + col.tile_base, items, cap,
                            recs, nb, flag, bx, by, bz, srec);
    }
}

cudaError_t launch_collide_batch(int storage, const void* fin, void* fout,
                                 const BatchColumn* cols, int ncols, int total_items, int depth,
                                 int grid, int planes, int* work_counter, const TileLists& tl,
                                 const BubbleRec* recs, int nb, int* flag, cudaStream_t st) {
    if (ncols > MAX_BATCH_COLUMNS) return cudaErrorInvalidValue;
    switch (storage * 8 + planes) {
#define LBM_LAUNCH_BATCH(SI, PV, T)                                                               \
    case SI * 8 + PV:                                                                             \
        k_collide_batch<SI, PV><<<grid, dim3(PX, TY, PV), 0, st>>>(                               \
            (const T*)fin, (T*)fout, cols, ncols, total_items, depth, work_counter, tl.start,    \
            tl.count, tl.items, tl.cap, recs, nb, flag);                                         \
        break;
        LBM_LAUNCH_BATCH(0, 1, float)
        LBM_LAUNCH_BATCH(0, 2, float)
        LBM_LAUNCH_BATCH(0, 4, float)
        LBM_LAUNCH_BATCH(1, 1, __half)
        LBM_LAUNCH_BATCH(1, 2, __half)
        LBM_LAUNCH_BATCH(1, 4, __half)
        LBM_LAUNCH_BATCH(2, 1, __nv_bfloat16)
        LBM_LAUNCH_BATCH(2, 2, __nv_bfloat16)
        LBM_LAUNCH_BATCH(2, 4, __nv_bfloat16)
#undef LBM_LAUNCH_BATCH
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

int sweep_z_blocks(int nz) { return (nz + PZ - 1) / PZ; }
int batch_min_blocks(int storage, int planes) {
    const int k = storage == 0 ? PairOccupancy<0>::kMinBlocks : PairOccupancy<1>::kMinBlocks;
    return k * PZ / planes;
}

cudaError_t launch_collide_stream(int storage, const void* fin, void* fout, const Geo& g,
                                  const CollideParams& cp, const TileLists* tl,
                                  const BubbleRec* recs, int nb, int* flag, const unsigned* safe,
                                  unsigned epoch, bool overlap, const int* zperm,
                                  cudaStream_t st, const ZSpan* span) {
    const int* start = tl ? tl->start : nullptr;
    const int* count = tl ? tl->count : nullptr;
    const int* items = tl ? tl->items : nullptr;
    const int cap = tl ? tl->cap : 0;
    if (overlap && (safe == nullptr || tl == nullptr)) return cudaErrorInvalidValue;
    if (!overlap) safe = nullptr;
    const int nbz = (g.nz + PZ - 1) / PZ;
    ZSpan zs{0, nbz, INT_MAX, 0};
    if (span) {
        if ((g.nx & 1) || zperm || span->count < 0 || span->first < 0 || span->skip < 0 ||
            span->first + span->count + span->skip > nbz)
            return cudaErrorInvalidValue;
        zs = *span;
        if (zs.count == 0) return cudaSuccess;
    }
    if ((g.nx & 1) == 0) {
        // Even rows: two nodes per thread with aligned vector accesses.  Tile
        // lists longer than the few-bubble path's (many bubbles per tile)
        // take the tabulated force gather.
        cudaLaunchConfig_t cfg = {};
        cfg.blockDim = dim3(PX, TY, PZ);
        cfg.gridDim = dim3((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, (unsigned)zs.count);
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = overlap ? 1 : 0;
        if (tl == nullptr && zperm == nullptr && !overlap) {
            // No bubble force reaches these blocks.
            switch (storage) {
                case 0:
                    return cudaLaunchKernelEx(&cfg, k_collide_stream_free<0>, (const float*)fin,
                                              (float*)fout, g, cp, flag, zs);
                case 1:
                    return cudaLaunchKernelEx(&cfg, k_collide_stream_free<1>, (const __half*)fin,
                                              (__half*)fout, g, cp, flag, zs);
                default:
                    return cudaLaunchKernelEx(&cfg, k_collide_stream_free<2>,
                                              (const __nv_bfloat16*)fin, (__nv_bfloat16*)fout, g,
                                              cp, flag, zs);
            }
        }
        const bool tab = tl != nullptr && tl->cap > SMALL_MAX_PAIRS;
        switch (storage * 2 + (tab ? 1 : 0)) {
#define LBM_LAUNCH_PAIR(SI, TB, T)                                                                \
    case SI * 2 + TB:                                                                             \
        return cudaLaunchKernelEx(&cfg, k_collide_stream_pair<SI, TB>, (const T*)fin, (T*)fout,   \
                                  g, cp, start, count, items, cap, recs, nb, flag, safe, epoch,  \
                                  zperm, zs);
            LBM_LAUNCH_PAIR(0, 0, float)
            LBM_LAUNCH_PAIR(0, 1, float)
            LBM_LAUNCH_PAIR(1, 0, __half)
            LBM_LAUNCH_PAIR(1, 1, __half)
            LBM_LAUNCH_PAIR(2, 0, __nv_bfloat16)
            LBM_LAUNCH_PAIR(2, 1, __nv_bfloat16)
#undef LBM_LAUNCH_PAIR
            default:
                return cudaErrorInvalidValue;
        }
    }
    if (overlap) return cudaErrorInvalidValue;   // odd rows: plain stream order only
    dim3 block(TX, TY, 1);
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, g.nz);
    switch (storage) {
        case 0:
            k_collide_stream<0><<<grid, block, 0, st>>>((const float*)fin, (float*)fout, g, cp,
                                                        start, count, items, cap, recs, nb, flag);
            break;
        case 1:
            k_collide_stream<1><<<grid, block, 0, st>>>((const __half*)fin, (__half*)fout, g, cp,
                                                        start, count, items, cap, recs, nb, flag);
            break;
        default:
            k_collide_stream<2><<<grid, block, 0, st>>>((const __nv_bfloat16*)fin,
                                                        (__nv_bfloat16*)fout, g, cp, start, count,
                                                        items, cap, recs, nb, flag);
            break;
    }
    return cudaGetLastError();
}

}  // namespace lbm
