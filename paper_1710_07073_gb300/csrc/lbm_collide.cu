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

template <int ST, int J>
__device__ __forceinline__ void relax_store(typename Store<ST>::T* __restrict__ fout, size_t S,
                                            int site, float gj, float drho, float rho, float ux,
                                            float uy, float uz, float usq, float Fx, float Fy,
                                            float Fz, float uF, const CollideParams& cp) {
    constexpr float w = wf(J);
    float cu = (float)cx(J) * ux + (float)cy(J) * uy + (float)cz(J) * uz;
    float cF = (float)cx(J) * Fx + (float)cy(J) * Fy + (float)cz(J) * Fz;
    // Eq. 6 shifted by w_j rho0: g^eq = w_j [drho + rho (3 cu + 9/2 cu^2 - 3/2 u^2)]
    float geq = w * (drho + rho * (3.0f * cu + 4.5f * cu * cu - 1.5f * usq));
    // Eq. 14 then Eq. 15 with the Guo term of Eq. 12.
    float out = gj - cp.omega * (gj - geq) + cp.pref * w * (3.0f * (cF - uF) + 9.0f * cu * cF);
    Store<ST>::template store<J>(fout + (size_t)J * S + site, out, cp);
}

template <int ST>
__global__ void __launch_bounds__(TX * TY, 8)
k_collide_stream(const typename Store<ST>::T* __restrict__ fin,
                 typename Store<ST>::T* __restrict__ fout, Geo g, CollideParams cp,
                 const int* __restrict__ tile_off, const int* __restrict__ items, int cap,
                 const BubbleRec* __restrict__ recs, int nb, int* __restrict__ flag) {
    __shared__ BubbleRec srec[TX * TY];
    const int x = blockIdx.x * TX + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    const int z = blockIdx.z;
    const bool inside = (x < g.nx) && (y < g.ny);

    float Fx = 0.0f, Fy = 0.0f, Fz = 0.0f;
    if (tile_off != nullptr) {
        const int t = ((z / TZ) * g.nty + blockIdx.y) * g.ntx + blockIdx.x;
        const int beg = tile_off[t], end = min(tile_off[t + 1], cap);
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
    if (!inside) return;

    float gv[Q];
    gather<ST>(fin, g, cp, x, y, z, gv);

    // Eq. 10 / Eq. 13 moments on shifted populations (sum_j w_j c_j = 0).
    float drho = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int j = 0; j < Q; ++j) {
        drho += gv[j];
        if (cx(j) != 0) jx += (float)cx(j) * gv[j];
        if (cy(j) != 0) jy += (float)cy(j) * gv[j];
        if (cz(j) != 0) jz += (float)cz(j) * gv[j];
    }
    const float rho = cp.rho0 + drho;
    const float inv_rho = 1.0f / rho;
    const float ux = (jx + 0.5f * Fx) * inv_rho;
    const float uy = (jy + 0.5f * Fy) * inv_rho;
    const float uz = (jz + 0.5f * Fz) * inv_rho;
    const float usq = ux * ux + uy * uy + uz * uz;
    if (!(usq < 0.09f)) atomicOr(flag, 1);   // non-finite or beyond |u| = 0.3
    const float uF = ux * Fx + uy * Fy + uz * Fz;

    const size_t S = (size_t)g.S;
    const int site = site_index(g, x, y, z);
#define LBM_RELAX(J) relax_store<ST, J>(fout, S, site, gv[J], drho, rho, ux, uy, uz, usq, Fx, Fy, Fz, uF, cp)
    LBM_RELAX(0); LBM_RELAX(1); LBM_RELAX(2); LBM_RELAX(3); LBM_RELAX(4);
    LBM_RELAX(5); LBM_RELAX(6); LBM_RELAX(7); LBM_RELAX(8); LBM_RELAX(9);
    LBM_RELAX(10); LBM_RELAX(11); LBM_RELAX(12); LBM_RELAX(13); LBM_RELAX(14);
    LBM_RELAX(15); LBM_RELAX(16); LBM_RELAX(17); LBM_RELAX(18);
#undef LBM_RELAX
}

cudaError_t launch_collide_stream(int storage, const void* fin, void* fout, const Geo& g,
                                  const CollideParams& cp, const Bins* bins,
                                  const BubbleRec* recs, int nb, int* flag, cudaStream_t st) {
    dim3 block(TX, TY, 1);
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, g.nz);
    const int* off = bins ? bins->off : nullptr;
    const int* items = bins ? bins->items : nullptr;
    const int cap = bins ? bins->cap : 0;
    switch (storage) {
        case 0:
            k_collide_stream<0><<<grid, block, 0, st>>>((const float*)fin, (float*)fout, g, cp, off,
                                                        items, cap, recs, nb, flag);
            break;
        case 1:
            k_collide_stream<1><<<grid, block, 0, st>>>((const __half*)fin, (__half*)fout, g, cp,
                                                        off, items, cap, recs, nb, flag);
            break;
        default:
            k_collide_stream<2><<<grid, block, 0, st>>>((const __nv_bfloat16*)fin,
                                                        (__nv_bfloat16*)fout, g, cp, off, items,
                                                        cap, recs, nb, flag);
            break;
    }
    return cudaGetLastError();
}

}  // namespace lbm
