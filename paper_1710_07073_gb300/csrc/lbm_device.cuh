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
// the node x - c_j, wrapped on periodic axes.  If the link crosses a wall the
// population is the opposite one leaving the same node (half-way
// bounce-back); `plane` and `idx` say where to read it.
template <int J>
__device__ __forceinline__ void pull_source(const Geo& g, int x, int y, int z, int& plane,
                                            int& idx) {
    int sx = x - cx(J), sy = y - cy(J), sz = z - cz(J);
    bool bounce = false;
    if (cx(J) != 0 && (sx < 0 || sx >= g.nx)) {
        if (g.walls & 0x01) bounce = true;
        else sx = sx < 0 ? sx + g.nx : sx - g.nx;
    }
    if (cy(J) != 0 && (sy < 0 || sy >= g.ny)) {
        if (g.walls & 0x04) bounce = true;
        else sy = sy < 0 ? sy + g.ny : sy - g.ny;
    }
    if (cz(J) != 0 && (sz < 0 || sz >= g.nz)) {
        if (g.walls & 0x10) bounce = true;
        else sz = sz < 0 ? sz + g.nz : sz - g.nz;
    }
    if (bounce) {
        plane = opp(J);
        idx = site_index(g, x, y, z);
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
    bool bounce = false;
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
        bounce = bounce || (out && (g.walls & 0x10));
        sz = out ? (sz < 0 ? sz + g.nz : sz - g.nz) : sz;
    }
    const unsigned S = (unsigned)g.S;
    const unsigned own = (unsigned)site_index(g, x, y, z);
    const unsigned src = (unsigned)site_index(g, sx, sy, sz);
    // The stored scale of a bounced population is that of its own plane; the
    // 16-bit formats share w_j between opposite directions, so J's scale holds.
    return bounce ? (unsigned)opp(J) * S + own : (unsigned)J * S + src;
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
__device__ __forceinline__ float cell_poly(float s, float h) {
    float a = fmaxf(s - h, -1.0f);
    float b = fminf(s + h, 1.0f);
    if (!(b > a)) return 0.0f;
    float a2 = a * a, b2 = b * b, ab = a * b;
    float p4 = b2 * b2 + b2 * ab + ab * ab + ab * a2 + a2 * a2;
    float p2 = b2 + ab + a2;
    return (b - a) * (p4 * 0.2f - p2 * (2.0f / 3.0f) + 1.0f);
}

__device__ __forceinline__ double cell_poly_d(double a, double b) {
    a = fmax(a, -1.0);
    b = fmin(b, 1.0);
    if (!(b > a)) return 0.0;
    double a2 = a * a, b2 = b * b, ab = a * b;
    double p4 = b2 * b2 + b2 * ab + ab * ab + ab * a2 + a2 * a2;
    double p2 = b2 + ab + a2;
    return (b - a) * (p4 * 0.2 - p2 * (2.0 / 3.0) + 1.0);
}

}  // namespace lbm
