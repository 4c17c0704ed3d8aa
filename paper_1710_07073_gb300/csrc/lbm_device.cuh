// Device helpers shared by the kernel translation units: population storage
// formats, the pull-gather with half-way bounce-back, and the cell integral of
// the clipped fourth-order polynomial mapping.
#pragma once

#include "lbm_internal.cuh"

namespace lbm {

// ---- programmatic dependent launch -----------------------------------------
// pdl_wait: block until the grids this one was launched to overlap with have
// completed and their writes are visible (returns at once for a grid launched
// in plain stream order).  pdl_trigger: this CTA no longer holds back the
// launch of the grid queued after this one.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---- population storage ------------------------------------------------------
// Stored value of population j is the shifted deviation g_j = f_j - w_j rho0:
// as is for FP32, times scale / w_j for the 16-bit formats.  load/store convert
// to and from g_j; load_raw/store_raw move the stored value itself (the
// "raw" value, r_j = g_j for FP32 and g_j scale / w_j for 16 bits).
template <int ST> struct Store;

template <> struct Store<0> {
    using T = float;
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ T ld(const T* p) { return __ldg(p); }
    template <int J>
    static __device__ __forceinline__ float widen(T v, const CollideParams&) { return v; }
    static __device__ __forceinline__ float load_raw(const T* p) { return __ldg(p); }
    static __device__ __forceinline__ void store_raw(T* p, float v) { __stcs(p, v); }
    template <int J>
    static __device__ __forceinline__ float load(const T* p, const CollideParams&) {
        return __ldg(p);
    }
    template <int J>
    static __device__ __forceinline__ void store(T* p, float v, const CollideParams&) {
        __stcs(p, v);
    }
    static __host__ __device__ __forceinline__ T from_double(double v, int, const CollideParams&) {
        return (float)v;
    }
    static __host__ __device__ __forceinline__ double to_double(T v, int, const CollideParams&) {
        return (double)v;
    }
};

template <> struct Store<1> {
    using T = __half;
    static constexpr bool kScaled = true;
    static __device__ __forceinline__ T ld(const T* p) { return __ldg(p); }
    template <int J>
    static __device__ __forceinline__ float widen(T v, const CollideParams& cp) {
        return __half2float(v) * (wf(J) * cp.inv_scale);
    }
    static __device__ __forceinline__ float load_raw(const T* p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ void store_raw(T* p, float v) {
        __stcs(p, __float2half_rn(v));
    }
    template <int J>
    static __device__ __forceinline__ float load(const T* p, const CollideParams& cp) {
        return __half2float(__ldg(p)) * (wf(J) * cp.inv_scale);
    }
    template <int J>
    static __device__ __forceinline__ void store(T* p, float v, const CollideParams& cp) {
        __stcs(p, __float2half_rn(v * (cp.scale * inv_wf(J))));
    }
    static __device__ __forceinline__ T from_double(double v, int j, const CollideParams& cp) {
        return __double2half(v * (double)cp.scale / wd(j));
    }
    static __device__ __forceinline__ double to_double(T v, int j, const CollideParams& cp) {
        return (double)__half2float(v) * wd(j) / (double)cp.scale;
    }
};

template <> struct Store<2> {
    using T = __nv_bfloat16;
    static constexpr bool kScaled = true;
    static __device__ __forceinline__ T ld(const T* p) { return __ldg(p); }
    template <int J>
    static __device__ __forceinline__ float widen(T v, const CollideParams& cp) {
        return __bfloat162float(v) * (wf(J) * cp.inv_scale);
    }
    static __device__ __forceinline__ float load_raw(const T* p) {
        return __bfloat162float(__ldg(p));
    }
    static __device__ __forceinline__ void store_raw(T* p, float v) {
        __stcs(p, __float2bfloat16_rn(v));
    }
    template <int J>
    static __device__ __forceinline__ float load(const T* p, const CollideParams& cp) {
        return __bfloat162float(__ldg(p)) * (wf(J) * cp.inv_scale);
    }
    template <int J>
    static __device__ __forceinline__ void store(T* p, float v, const CollideParams& cp) {
        __stcs(p, __float2bfloat16_rn(v * (cp.scale * inv_wf(J))));
    }
    static __device__ __forceinline__ T from_double(double v, int j, const CollideParams& cp) {
        return __double2bfloat16(v * (double)cp.scale / wd(j));
    }
    static __device__ __forceinline__ double to_double(T v, int j, const CollideParams& cp) {
        return (double)__bfloat162float(v) * wd(j) / (double)cp.scale;
    }
};

__device__ __forceinline__ int site_index(const Geo& g, int x, int y, int z) {
    return (z * g.ny + y) * g.nx + x;
}

// Source of population j arriving at node (x,y,z) under streaming (Eq. 16):
// the node x - c_j, wrapped on periodic axes.  If the link crosses a no-slip
// wall the population is the opposite one leaving the same node (half-way
// bounce-back).  If it crosses only a free-slip top (Sec. 3.3), it is the
// z-mirrored population leaving the top layer one tangential step back
// (specular reflection).  `plane` and `idx` say where to read it.
template <int J>
__device__ __forceinline__ void pull_source(const Geo& g, int x, int y, int z, int& plane,
                                            int& idx) {
    int sx = x - cx(J), sy = y - cy(J), sz = z - cz(J);
    bool bounce = false, specular = false;
    if (cx(J) != 0 && (sx < 0 || sx >= g.nx)) {
        if (g.walls & 0x01) bounce = true;
        else sx = sx < 0 ? sx + g.nx : sx - g.nx;
    }
    if (cy(J) != 0 && (sy < 0 || sy >= g.ny)) {
        if (g.walls & 0x04) bounce = true;
        else sy = sy < 0 ? sy + g.ny : sy - g.ny;
    }
    if (cz(J) != 0 && (sz < 0 || sz >= g.nz)) {
        if (sz >= g.nz && (g.walls & WALL_TOP_FREE)) specular = true;
        else if (g.walls & 0x10) bounce = true;
        else sz = sz < 0 ? sz + g.nz : sz - g.nz;
    }
    if (bounce) {
        plane = opp(J);
        idx = site_index(g, x, y, z);
    } else if (specular) {
        plane = mirz(J);
        idx = site_index(g, sx, sy, z);
    } else {
        plane = J;
        idx = site_index(g, sx, sy, sz);
    }
}

// Element offset (plane j S + site) of the population j arriving at node
// (x,y,z) under Eq. 16, with the wrap and the half-way bounce-back of
// pull_source written as selects: no branches, so that a gather can compute
// all 19 offsets, then issue all 19 loads, then use them.
template <int J>
__device__ __forceinline__ unsigned pull_offset(const Geo& g, int x, int y, int z) {
    int sx = x - cx(J), sy = y - cy(J), sz = z - cz(J);
    bool bounce = false, specular = false;
    if (cx(J) != 0) {
        const bool out = (unsigned)sx >= (unsigned)g.nx;
        bounce = bounce || (out && (g.walls & 0x01));
        sx = out ? (sx < 0 ? sx + g.nx : sx - g.nx) : sx;
    }
    if (cy(J) != 0) {
        const bool out = (unsigned)sy >= (unsigned)g.ny;
        bounce = bounce || (out && (g.walls & 0x04));
        sy = out ? (sy < 0 ? sy + g.ny : sy - g.ny) : sy;
    }
    if (cz(J) != 0) {
        const bool out = (unsigned)sz >= (unsigned)g.nz;
        specular = cz(J) < 0 && out && (g.walls & WALL_TOP_FREE);
        bounce = bounce || (out && !specular && (g.walls & 0x10));
        sz = out ? (specular ? z : (sz < 0 ? sz + g.nz : sz - g.nz)) : sz;
    }
    const unsigned S = (unsigned)g.S;
    const unsigned own = (unsigned)site_index(g, x, y, z);
    const unsigned src = (unsigned)site_index(g, sx, sy, sz);
    // The stored scale of a bounced or mirrored population is that of its own
    // plane; the 16-bit formats share w_j between opposite and mirrored
    // directions, so J's scale holds.
    return bounce ? (unsigned)opp(J) * S + own
                  : (specular ? (unsigned)mirz(J) * S + src : (unsigned)J * S + src);
}

// Stored pre-collision values at one node: the 19 loads, issued together.
template <int ST>
__device__ __forceinline__ void gather_issue(const typename Store<ST>::T* __restrict__ f,
                                             const Geo& g, int x, int y, int z,
                                             typename Store<ST>::T raw[Q]) {
    unsigned o[Q];
#define LBM_OFF(J) o[J] = pull_offset<J>(g, x, y, z)
    LBM_OFF(0); LBM_OFF(1); LBM_OFF(2); LBM_OFF(3); LBM_OFF(4); LBM_OFF(5); LBM_OFF(6);
    LBM_OFF(7); LBM_OFF(8); LBM_OFF(9); LBM_OFF(10); LBM_OFF(11); LBM_OFF(12); LBM_OFF(13);
    LBM_OFF(14); LBM_OFF(15); LBM_OFF(16); LBM_OFF(17); LBM_OFF(18);
#undef LBM_OFF
#pragma unroll
    for (int q = 0; q < Q; ++q) raw[q] = Store<ST>::ld(f + o[q]);
}

// Stored values to shifted populations f_j - w_j rho0.
template <int ST>
__device__ __forceinline__ void gather_finish(const typename Store<ST>::T raw[Q],
                                              const CollideParams& cp, float gv[Q]) {
#define LBM_WID(J) gv[J] = Store<ST>::template widen<J>(raw[J], cp)
    LBM_WID(0); LBM_WID(1); LBM_WID(2); LBM_WID(3); LBM_WID(4); LBM_WID(5); LBM_WID(6);
    LBM_WID(7); LBM_WID(8); LBM_WID(9); LBM_WID(10); LBM_WID(11); LBM_WID(12); LBM_WID(13);
    LBM_WID(14); LBM_WID(15); LBM_WID(16); LBM_WID(17); LBM_WID(18);
#undef LBM_WID
}

// Pre-collision populations f_j(x, t) - w_j rho0 at one node (Eq. 16 pull).
template <int ST>
__device__ __forceinline__ void gather(const typename Store<ST>::T* __restrict__ f, const Geo& g,
                                       const CollideParams& cp, int x, int y, int z,
                                       float gv[Q]) {
    typename Store<ST>::T raw[Q];
    gather_issue<ST>(f, g, x, y, z, raw);
    gather_finish<ST>(raw, cp, gv);
}

// Integral of the mapping function over [s - h, s + h] in units of the
// half-width n (s = r/n, h = 1/(2n)), without the constant 15/16:
//   int_a^b (t^4 - 2 t^2 + 1) dt
//     = (b - a) [ (b^4 + b^3 a + b^2 a^2 + b a^3 + a^4)/5 - 2 (b^2 + a b + a^2)/3 + 1 ]
// with a, b clipped to the window [-1, 1] (Eq. 18-19).  The factored form
// avoids the cancellation of a difference of antiderivatives.
// A negative h selects the point-sampled map: Z at the node times the cell
// width, 2|h| (1 - s^2)^2, zero outside the window.  PM fixes the mode at
// compile time (MAP_CELL, MAP_POINT) for loops whose mode is known uniform;
// MAP_ANY reads it from the sign of h.
constexpr int MAP_ANY = -1, MAP_CELL = 0, MAP_POINT = 1;
template <int P> struct MapMode { static constexpr int value = P; };

template <int PM = MAP_ANY>
__device__ __forceinline__ float cell_poly(float s, float h) {
    if (PM == MAP_POINT || (PM == MAP_ANY && h < 0.0f)) {
        const float t = fminf(fabsf(s), 1.0f);
        const float q = fmaf(-t, t, 1.0f);
        return -2.0f * h * q * q;
    }
    float a = fmaxf(s - h, -1.0f);
    float b = fminf(s + h, 1.0f);
    if (!(b > a)) return 0.0f;
    float a2 = a * a, b2 = b * b, ab = a * b;
    float p4 = b2 * b2 + b2 * ab + ab * ab + ab * a2 + a2 * a2;
    float p2 = b2 + ab + a2;
    return (b - a) * (p4 * 0.2f - p2 * (2.0f / 3.0f) + 1.0f);
}

// Cell integral of the mapping along one axis for lattice coordinate c, with
// the record's anchor cell `anc` and offset `fr` (Eq. 19), wrapped on a
// periodic axis of length L to the nearer image.  The sweep's force gather and
// the many-bubble interpolation both take their weights from it.
template <int PM = MAP_ANY>
__device__ __forceinline__ float axis_weight(const BubbleRec& r, int c, int anc, float fr, int L,
                                             bool periodic) {
    float rc = (float)(c - anc) + 0.5f - fr;
    if (periodic) {
        if (rc > 0.5f * L) rc -= (float)L;
        else if (rc < -0.5f * L) rc += (float)L;
    }
    return cell_poly<PM>(rc * r.inv_n, r.h);
}

// Per-axis factors for the interpolated vorticity (lift), by summation by
// parts.  The central difference of the node velocity, (u(c+1) - u(c-1))/2,
// interpolated with the Eq. 19 weights w, is a sum of the velocities u(c)
// times d(c) = (w(c-1) - w(c+1))/2 (w zero beyond a wall face), plus the
// ghost terms of the face nodes: the ghost beyond a no-slip wall is -u (+w/2
// at the low face, -w/2 at the high face), beyond the free-slip top +u for
// the tangential components the curl differentiates (+w/2).  Periodic axes
// wrap the distance to the nearer image.  Returns w(c) and d(c) for the
// cell c, anchor cell anc and offset fr of the centre.
template <int PM = MAP_ANY>
__device__ __forceinline__ void axis_wd(int c, int anc, float fr, float inv_n, float hh, int L,
                                        bool periodic, bool free_hi, float& w, float& d) {
    float rc = (float)(c - anc) + 0.5f - fr;
    if (periodic) {
        if (rc > 0.5f * L) rc -= (float)L;
        else if (rc < -0.5f * L) rc += (float)L;
    }
    const float s = rc * inv_n;
    w = cell_poly<PM>(s, hh);
    const float wm = (!periodic && c - 1 < 0) ? 0.0f : cell_poly<PM>(s - inv_n, hh);
    const float wp = (!periodic && c + 1 > L - 1) ? 0.0f : cell_poly<PM>(s + inv_n, hh);
    d = 0.5f * (wm - wp);
    if (!periodic) {
        if (c == 0) d += 0.5f * w;
        if (c == L - 1) d += free_hi ? 0.5f * w : -0.5f * w;
    }
}

// The tile lists and records are read through L2 (ld.global.cg): with the
// sweep overlapping the bubble update, they are written while the sweep runs,
// so the read-only cache path is not used for them.
__device__ __forceinline__ BubbleRec load_rec(const BubbleRec* p) {
    const int4* q = reinterpret_cast<const int4*>(p);
    const int4 a = __ldcg(q), b = __ldcg(q + 1), c = __ldcg(q + 2);
    return BubbleRec{a.x, a.y, a.z, a.w,
                     __int_as_float(b.x), __int_as_float(b.y), __int_as_float(b.z),
                     __int_as_float(b.w), __int_as_float(c.x), __int_as_float(c.y),
                     __int_as_float(c.z), __int_as_float(c.w)};
}

// ---- two nodes per thread (even nx) -----------------------------------------
// A thread owns the x-pair (x0, x0 + 1), x0 even, so every plane row is read
// with one aligned 2-wide access (float2, half2, bfloat162) and the moments
// run on packed FP32 pairs (FFMA2 / FADD2 / FMUL2).
template <int ST> struct Vec2;
template <> struct Vec2<0> {
    static __device__ __forceinline__ void store(float* p, float2 v) {
        __stcs(reinterpret_cast<float2*>(p), v);
    }
};
template <> struct Vec2<1> {
    static __device__ __forceinline__ void store(__half* p, float2 v) {
        __stcs(reinterpret_cast<__half2*>(p), __floats2half2_rn(v.x, v.y));
    }
};
template <> struct Vec2<2> {
    static __device__ __forceinline__ void store(__nv_bfloat16* p, float2 v) {
        __stcs(reinterpret_cast<__nv_bfloat162*>(p), __floats2bfloat162_rn(v.x, v.y));
    }
};

// The stored values of one direction at an x-pair, as loaded.  FP32 keeps the
// float2; the 16-bit formats keep both nodes packed in one 32-bit register
// (node x0 in the low half) and widen at each use, which halves the registers
// the 19 loaded rows hold while the moments and the relaxation run.
template <int ST> struct Raw2 {
    using T = unsigned;
    using T1 = unsigned;
    static __device__ __forceinline__ T load(const typename Store<ST>::T* p) {
        return __ldg(reinterpret_cast<const unsigned*>(p));
    }
    static __device__ __forceinline__ T1 load1(const typename Store<ST>::T* p) {
        return (unsigned)__ldg(reinterpret_cast<const unsigned short*>(p));
    }
    // (a, P.x) and (P.y, a)
    static __device__ __forceinline__ T lo_from(T1 a, T P) { return __byte_perm(a, P, 0x5410); }
    static __device__ __forceinline__ T hi_from(T P, T1 a) { return __byte_perm(P, a, 0x5432); }
    static __device__ __forceinline__ T join(T1 a, T1 b) { return __byte_perm(a, b, 0x5410); }
    static __device__ __forceinline__ float2 widen(T v);
};
template <> __device__ __forceinline__ float2 Raw2<1>::widen(unsigned v) {
    return __half22float2(*reinterpret_cast<const __half2*>(&v));
}
template <> __device__ __forceinline__ float2 Raw2<2>::widen(unsigned v) {
    return make_float2(__uint_as_float(v << 16), __uint_as_float(v & 0xffff0000u));
}
template <> struct Raw2<0> {
    using T = float2;
    using T1 = float;
    static __device__ __forceinline__ T load(const float* p) {
        return __ldg(reinterpret_cast<const float2*>(p));
    }
    static __device__ __forceinline__ T1 load1(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ T lo_from(T1 a, T P) { return make_float2(a, P.x); }
    static __device__ __forceinline__ T hi_from(T P, T1 a) { return make_float2(P.y, a); }
    static __device__ __forceinline__ T join(T1 a, T1 b) { return make_float2(a, b); }
    static __device__ __forceinline__ float2 widen(T v) { return v; }
};

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.0f), a); }

// Raw values of direction J arriving at the pair (x0, x0 + 1) of a row whose
// y and z neighbours are inside the box.  The aligned pair of the source row
// covers one of the two; the population crossing x for the other node is one
// scalar load, at x0 - 1 or x0 + 2 of the source row, or, on an x face, at the
// opposite plane of the node itself (wall) or the other end of the row
// (periodic).  Every lane issues the same loads, so none waits on another.
template <int ST, int J>
__device__ __forceinline__ typename Raw2<ST>::T pull_pair(const typename Store<ST>::T* __restrict__ f,
                                                          unsigned S, unsigned site0, unsigned nx,
                                                          unsigned nxy, int x0, bool wallx) {
    const unsigned row = (unsigned)J * S + site0 - ((unsigned)cy(J) * nx + (unsigned)cz(J) * nxy);
    const typename Raw2<ST>::T P = Raw2<ST>::load(f + row);   // the source row at (x0, x0 + 1)
    if (cx(J) == 0) return P;
    if (cx(J) == 1) {
        // node x0 receives x0 - 1, node x0 + 1 receives x0
        unsigned a = row - 1u;
        if (x0 == 0) a = wallx ? (unsigned)opp(J) * S + site0 : row + nx - 1u;
        return Raw2<ST>::lo_from(Raw2<ST>::load1(f + a), P);
    }
    // cx == -1: node x0 receives x0 + 1, node x0 + 1 receives x0 + 2
    unsigned a = row + 2u;
    if ((unsigned)x0 + 2u >= nx) a = wallx ? (unsigned)opp(J) * S + site0 + 1u : row - (unsigned)x0;
    return Raw2<ST>::hi_from(P, Raw2<ST>::load1(f + a));
}

template <int ST, int J>
__device__ __forceinline__ typename Raw2<ST>::T pull_pair_any(
    const typename Store<ST>::T* __restrict__ f, const Geo& g, int x0, int y, int z) {
    int p0, i0, p1, i1;
    pull_source<J>(g, x0, y, z, p0, i0);
    pull_source<J>(g, x0 + 1, y, z, p1, i1);
    return Raw2<ST>::join(Raw2<ST>::load1(f + (size_t)p0 * (size_t)g.S + i0),
                          Raw2<ST>::load1(f + (size_t)p1 * (size_t)g.S + i1));
}

// Eq. 10 moments of an x-pair from its raw stored values (as loaded):
// drho = sum_j g_j and j = sum_j c_j g_j of the shifted populations, on packed
// FP32 pairs.  The sum order is fixed (the sweep and the many-bubble
// interpolation share it).
template <int ST>
__device__ __forceinline__ void pair_moments(const typename Raw2<ST>::T rr[Q],
                                             const CollideParams& cp, float2& drho, float2& jx,
                                             float2& jy, float2& jz) {
    float2 rv[Q];
#pragma unroll
    for (int j = 0; j < Q; ++j) rv[j] = Raw2<ST>::widen(rr[j]);
    const float2 s_axis = add2(add2(add2(rv[1], rv[2]), add2(rv[3], rv[4])), add2(rv[5], rv[6]));
    const float2 s_edge = add2(add2(add2(add2(rv[7], rv[8]), add2(rv[9], rv[10])),
                                    add2(add2(rv[11], rv[12]), add2(rv[13], rv[14]))),
                               add2(add2(rv[15], rv[16]), add2(rv[17], rv[18])));
    const float2 ax_x = sub2(rv[1], rv[2]), ax_y = sub2(rv[3], rv[4]), ax_z = sub2(rv[5], rv[6]);
    const float2 d78 = sub2(rv[7], rv[8]), d910 = sub2(rv[9], rv[10]);
    const float2 d1112 = sub2(rv[11], rv[12]), d1314 = sub2(rv[13], rv[14]);
    const float2 d1516 = sub2(rv[15], rv[16]), d1718 = sub2(rv[17], rv[18]);
    const float2 ed_x = add2(add2(d78, d910), add2(d1112, d1314));
    const float2 ed_y = add2(sub2(d78, d910), add2(d1516, d1718));
    const float2 ed_z = add2(sub2(d1112, d1314), sub2(d1516, d1718));
    if (Store<ST>::kScaled) {
        const float2 k0 = f2(wf(0) * cp.inv_scale), ka = f2(wf(1) * cp.inv_scale),
                     ke = f2(wf(7) * cp.inv_scale);
        drho = fma2(k0, rv[0], fma2(ka, s_axis, mul2(ke, s_edge)));
        jx = fma2(ka, ax_x, mul2(ke, ed_x));
        jy = fma2(ka, ax_y, mul2(ke, ed_y));
        jz = fma2(ka, ax_z, mul2(ke, ed_z));
    } else {
        drho = add2(rv[0], add2(s_axis, s_edge));
        jx = add2(ax_x, ed_x);
        jy = add2(ax_y, ed_y);
        jz = add2(ax_z, ed_z);
    }
}

// The raw values of all 19 directions arriving at the pair (x0, x0 + 1) of
// row (y, z) (x0 even, x0 + 1 < nx): the aligned-row gather inside, the
// general one on the y and z faces.
template <int ST>
__device__ __forceinline__ void gather_pair(const typename Store<ST>::T* __restrict__ f,
                                            const Geo& g, int x0, int y, int z,
                                            typename Raw2<ST>::T rv[Q]) {
    if (y > 0 && y < g.ny - 1 && z > 0 && z < g.nz - 1) {
        const unsigned S = (unsigned)g.S;
        const unsigned nx = (unsigned)g.nx, nxy = (unsigned)g.nx * (unsigned)g.ny;
        const unsigned site0 = (unsigned)z * nxy + (unsigned)y * nx + (unsigned)x0;
        const bool wallx = (g.walls & 0x01) != 0;
#define LBM_PP(J) rv[J] = pull_pair<ST, J>(f, S, site0, nx, nxy, x0, wallx)
        LBM_PP(0); LBM_PP(1); LBM_PP(2); LBM_PP(3); LBM_PP(4);
        LBM_PP(5); LBM_PP(6); LBM_PP(7); LBM_PP(8); LBM_PP(9);
        LBM_PP(10); LBM_PP(11); LBM_PP(12); LBM_PP(13); LBM_PP(14);
        LBM_PP(15); LBM_PP(16); LBM_PP(17); LBM_PP(18);
#undef LBM_PP
    } else {
#define LBM_PA(J) rv[J] = pull_pair_any<ST, J>(f, g, x0, y, z)
        LBM_PA(0); LBM_PA(1); LBM_PA(2); LBM_PA(3); LBM_PA(4);
        LBM_PA(5); LBM_PA(6); LBM_PA(7); LBM_PA(8); LBM_PA(9);
        LBM_PA(10); LBM_PA(11); LBM_PA(12); LBM_PA(13); LBM_PA(14);
        LBM_PA(15); LBM_PA(16); LBM_PA(17); LBM_PA(18);
#undef LBM_PA
    }
}

}  // namespace lbm
