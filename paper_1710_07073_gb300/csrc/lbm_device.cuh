// Device helpers shared by the kernel translation units: population storage
// formats, the pull-gather with half-way bounce-back, and the cell integral of
// the clipped fourth-order polynomial mapping.
#pragma once

#include "lbm_internal.cuh"

namespace lbm {

// ---- population storage ------------------------------------------------------
// Stored value of population j is the shifted deviation g_j = f_j - w_j rho0:
// as is for FP32, times scale / w_j for the 16-bit formats.  load/store convert
// to and from g_j; load_raw/store_raw move the stored value itself (the
// "raw" value, r_j = g_j for FP32 and g_j scale / w_j for 16 bits).
template <int ST> struct Store;

template <> struct Store<0> {
    using T = float;
    static constexpr bool kScaled = false;
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

template <int ST, int J>
__device__ __forceinline__ float pull_one(const typename Store<ST>::T* __restrict__ f,
                                          const Geo& g, const CollideParams& cp, int x, int y,
                                          int z) {
    int plane, idx;
    pull_source<J>(g, x, y, z, plane, idx);
    // The stored scale of a bounced population is that of its own plane; the
    // 16-bit formats share w_j between opposite directions, so J's scale holds.
    return Store<ST>::template load<J>(f + (size_t)plane * (size_t)g.S + idx, cp);
}

// Pre-collision populations f_j(x, t) - w_j rho0 at one node (Eq. 16 pull).
template <int ST>
__device__ __forceinline__ void gather(const typename Store<ST>::T* __restrict__ f, const Geo& g,
                                       const CollideParams& cp, int x, int y, int z,
                                       float gv[Q]) {
    gv[0] = pull_one<ST, 0>(f, g, cp, x, y, z);
    gv[1] = pull_one<ST, 1>(f, g, cp, x, y, z);
    gv[2] = pull_one<ST, 2>(f, g, cp, x, y, z);
    gv[3] = pull_one<ST, 3>(f, g, cp, x, y, z);
    gv[4] = pull_one<ST, 4>(f, g, cp, x, y, z);
    gv[5] = pull_one<ST, 5>(f, g, cp, x, y, z);
    gv[6] = pull_one<ST, 6>(f, g, cp, x, y, z);
    gv[7] = pull_one<ST, 7>(f, g, cp, x, y, z);
    gv[8] = pull_one<ST, 8>(f, g, cp, x, y, z);
    gv[9] = pull_one<ST, 9>(f, g, cp, x, y, z);
    gv[10] = pull_one<ST, 10>(f, g, cp, x, y, z);
    gv[11] = pull_one<ST, 11>(f, g, cp, x, y, z);
    gv[12] = pull_one<ST, 12>(f, g, cp, x, y, z);
    gv[13] = pull_one<ST, 13>(f, g, cp, x, y, z);
    gv[14] = pull_one<ST, 14>(f, g, cp, x, y, z);
    gv[15] = pull_one<ST, 15>(f, g, cp, x, y, z);
    gv[16] = pull_one<ST, 16>(f, g, cp, x, y, z);
    gv[17] = pull_one<ST, 17>(f, g, cp, x, y, z);
    gv[18] = pull_one<ST, 18>(f, g, cp, x, y, z);
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
