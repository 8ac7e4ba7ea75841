// lbm_conv.cuh -- the phases of the cell conversions (Sec. 2.2 of the paper, Fig.
// cellConversions) as device functions over compact worklists, shared by the conversion
// kernel and the fused end-of-step kernel; and the fill-level stencils.
//
// Every phase is called by all warps of a thread-block cluster with its warp index wid among
// nw warps; the phases are separated by cluster_sync (every later phase reads what the earlier
// ones wrote).
#pragma once
#include "lbm_internal.cuh"

namespace lbm {

__device__ __forceinline__ uint32_t list_len(const uint32_t* cnt, int cap) {
    const uint32_t n = *(volatile const uint32_t*)cnt;
    return n < (uint32_t)cap ? n : (uint32_t)cap;
}

// fill level seen by the normal and curvature stencils: interface -> phi, liquid -> 1,
// gas -> 0, obstacle and beyond a wall -> 1 (perfect wetting, Sec. 2.2)
__device__ __forceinline__ float fill_seen(const Dev& d, const float* phi, int x, int y, int z, int dx, int dy, int dz) {
    size_t j;
    if (!nbr(d, x, y, z, dx, dy, dz, j)) return 1.f;
    const uint8_t t = d.flags[j] & F_TYPE;
    if (t & F_IF) return phi[j];
    if (t & F_GAS) return 0.f;
    return 1.f;
}

// Parker-Youngs gradient of the fill level (points into the liquid): central difference
// smoothed with [1,2,1] x [1,2,1] / 16 over the 3x3x3 block
__device__ inline void py_gradient(const Dev& d, const float* phi, int x, int y, int z, float n[3]) {
    float v[27];
#pragma unroll
    for (int c = -1; c <= 1; c++)
#pragma unroll
        for (int b = -1; b <= 1; b++)
#pragma unroll
            for (int a = -1; a <= 1; a++)
                v[(c + 1) * 9 + (b + 1) * 3 + (a + 1)] = (a == 0 && b == 0 && c == 0) ? 0.f : fill_seen(d, phi, x, y, z, a, b, c);
    const float w1[3] = {1.f, 2.f, 1.f};
    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
    for (int p = 0; p < 3; p++)
#pragma unroll
        for (int r = 0; r < 3; r++) {
            const float w = w1[p] * w1[r];
            gx += w * (v[r * 9 + p * 3 + 2] - v[r * 9 + p * 3 + 0]);
            gy += w * (v[r * 9 + 2 * 3 + p] - v[r * 9 + 0 * 3 + p]);
            gz += w * (v[2 * 9 + r * 3 + p] - v[0 * 9 + r * 3 + p]);
        }
    n[0] = gx / 32.f;
    n[1] = gy / 32.f;
    n[2] = gz / 32.f;
}

template <int S>
__device__ float cell_rho(const Dev& d, const typename Store<S>::T* f, size_t i) {
    float dr = 0.f;
#pragma unroll
    for (int q = 0; q < kQ; q++) dr += Store<S>::get_nc(f, (size_t)q * d.N + i);
    return 1.f + dr;
}

// Every conversion kernel runs one warp per listed cell: lane q (1..18) handles the D3Q19
// neighbour x + c_q, lane 0 the cell itself, and warp shuffles combine what they find.

// density of cell i from grid f (deviations), summed over the warp's lanes 0..18
template <int S>
__device__ __forceinline__ float warp_cell_rho(const Dev& d, const typename Store<S>::T* f, size_t i, int lane) {
    const float v = lane < kQ ? Store<S>::get_nc(f, (size_t)lane * d.N + i) : 0.f;
    return 1.f + warp_sum(v);
}

// (ii) + (iii) in one phase.  Filled cells: gas neighbours become new interface cells (mass
// 0 from the start).  Emptied cells: an emptied cell with a filled neighbour stays an
// interface cell (filling wins: it clears its own mark); otherwise its liquid neighbours
// become interface cells with m = rho, the smallest bubble id among their emptied neighbours
// becoming theirs.  The filled marks are final before this phase (written by the sweep).
template <int S>
__device__ void conv_filled_emptied(const Dev& d, const int nxt, const uint32_t wid, const uint32_t nw) {
    using T = typename Store<S>::T;
    const T* f = static_cast<const T*>(d.f[nxt]);
    const uint32_t n = list_len(&d.sc->n_conv, d.wl_cap);
    const int lane = threadIdx.x & 31;
    for (uint32_t e = wid; e < n; e += nw) {
        const size_t i = d.wl_conv[e];
        const uint8_t mk = d.mark[i];
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        size_t j = 0;
        const bool has = lane >= 1 && lane < kQ && nbr(d, x, y, z, cx(lane), cy(lane), cz(lane), j);
        if (mk & K_FILLED) {
            if (!has) continue;
            if (d.flags[j] & F_GAS) {
                const uint8_t old = mark_or(d.mark, j, K_NEWIF);
                if (!(old & K_NEWIF)) {
                    d.mass[j] = 0.f;
                    wl_push(d.wl_newif, &d.sc->n_newif, (uint32_t)d.wl_cap, (uint32_t)j, &d.sc->status);
                }
            }
        } else if (mk & K_EMPTIED) {
            const bool filled_nbr = __any_sync(0xffffffffu, has && (d.mark[j] & K_FILLED));
            if (filled_nbr) {
                if (lane == 0) mark_and(d.mark, i, K_EMPTIED);
                continue;
            }
            if (!has || !(d.flags[j] & F_LIQ)) continue;
            const uint32_t b = d.owner[i];
            const uint8_t old = mark_or(d.mark, j, K_FROMLIQ);
            if (!(old & K_FROMLIQ)) {
                float dr = 0.f;
                for (int q = 0; q < kQ; q++) dr += Store<S>::get_nc(f, (size_t)q * d.N + j);
                d.mass[j] = 1.f + dr;
                wl_push(d.wl_fromliq, &d.sc->n_fromliq, (uint32_t)d.wl_cap, (uint32_t)j, &d.sc->status);
            }
            atomicMin(&d.owner[j], b);
        }
    }
}

// (iv) new interface cells from gas: f* = e(mean rho, mean u) over the neighbours that carry
// PDFs (liquid, interface not emptied, filled); their m = 0 was set when they were marked
template <int S>
__device__ void conv_newif(const Dev& d, const int nxt, const uint32_t wid, const uint32_t nw) {
    using T = typename Store<S>::T;
    T* f = static_cast<T*>(d.f[nxt]);
    const uint32_t n = list_len(&d.sc->n_newif, d.wl_cap);
    const int lane = threadIdx.x & 31;
    for (uint32_t e = wid; e < n; e += nw) {
        const size_t i = d.wl_newif[e];
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        float r = 0.f, u[3] = {0.f, 0.f, 0.f};
        int c = 0;
        size_t j;
        if (lane >= 1 && lane < kQ && nbr(d, x, y, z, cx(lane), cy(lane), cz(lane), j) &&
            (d.flags[j] & F_ACTIVE) && !(d.mark[j] & K_EMPTIED)) {
            post_moments<S>(d, f, j, (d.flags[j] & F_IF) ? d.phi[nxt][j] : 1.f, r, u);
            c = 1;
        }
        const int cnt = warp_sum(c);
        const float rs = warp_sum(r), ux = warp_sum(u[0]), uy = warp_sum(u[1]), uz = warp_sum(u[2]);
        const float rb = cnt ? rs / cnt : 1.f;
        const float ub[3] = {cnt ? ux / cnt : 0.f, cnt ? uy / cnt : 0.f, cnt ? uz / cnt : 0.f};
        if (lane < kQ) Store<S>::put(f, (size_t)lane * d.N + i, equilibrium_dev(lane, rb, ub));
        if (lane == 0 && d.rho[nxt]) d.rho[nxt][i] = rb;
    }
}

// (v) excess mass of converting cells to the neighbours that will be interface cells,
// weighted along the interface normal pointing into the gas (-grad phi): filled cells push
// along it, emptied cells against it; uniform if all weights vanish; to the global pool if
// no neighbour can take it.  The Parker-Youngs gradient is taken over the 3x3x3 block, lane l
// (0..26) holding the fill level of offset (l%3-1, l/3%3-1, l/9-1).
template <int S>
__device__ void conv_excess(const Dev& d, const int nxt, const uint32_t wid, const uint32_t nw) {
    using T = typename Store<S>::T;
    const T* f = static_cast<const T*>(d.f[nxt]);
    const float* phi = d.phi[nxt];
    const uint32_t n = list_len(&d.sc->n_conv, d.wl_cap);
    const int lane = threadIdx.x & 31;
    for (uint32_t e = wid; e < n; e += nw) {
        const size_t i = d.wl_conv[e];
        const uint8_t mk = d.mark[i] & (K_FILLED | K_EMPTIED);
        if (!mk) continue;
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        // Parker-Youngs: central difference smoothed by [1,2,1] x [1,2,1] / 16 (into the liquid)
        float gxl = 0.f, gyl = 0.f, gzl = 0.f;
        if (lane < 27 && lane != 13) {
            const int a = lane % 3 - 1, b = (lane / 3) % 3 - 1, c = lane / 9 - 1;
            const float v = fill_seen(d, phi, x, y, z, a, b, c);
            const float wa = a == 0 ? 2.f : 1.f, wb = b == 0 ? 2.f : 1.f, wc = c == 0 ? 2.f : 1.f;
            gxl = a * wb * wc * v;
            gyl = b * wa * wc * v;
            gzl = c * wa * wb * v;
        }
        const float ngx = -warp_sum(gxl) / 32.f, ngy = -warp_sum(gyl) / 32.f, ngz = -warp_sum(gzl) / 32.f;
        const float r = warp_cell_rho<S>(d, f, i, lane);
        const float m0 = d.mass[i];
        const float mex = (mk & K_FILLED) ? m0 - r : m0;
        size_t j = 0;
        bool rec = false;
        float w = 0.f;
        if (lane >= 1 && lane < kQ && nbr(d, x, y, z, cx(lane), cy(lane), cz(lane), j)) {
            const uint8_t mj = d.mark[j];
            rec = ((d.flags[j] & F_IF) && !(mj & (K_FILLED | K_EMPTIED))) || (mj & (K_NEWIF | K_FROMLIQ));
            if (rec) {
                const float nc = ngx * cx(lane) + ngy * cy(lane) + ngz * cz(lane);
                w = (mk & K_FILLED) ? fmaxf(nc, 0.f) : fmaxf(-nc, 0.f);
            }
        }
        // the lanes' weights in q order, as a serial sum would take them
        float W = 0.f;
        int nr = 0;
        for (int q = 1; q < kQ; q++) {
            W += __shfl_sync(0xffffffffu, w, q);
            nr += __shfl_sync(0xffffffffu, (int)rec, q);
        }
        if (lane == 0) {
            d.mass[i] = (mk & K_FILLED) ? r : 0.f;
            if (nr == 0) atomicAdd(&d.sc->pool_acc, (double)mex);
        }
        if (rec) {
            atomicAdd(&d.mass[j], W > 0.f ? mex * (w / W) : mex / (float)nr);
            mark_or(d.mark, j, K_RECV);
        }
    }
}

// (vi) final types; fill level of every interface cell whose mass changed in this phase
template <int S>
__device__ void conv_finalize(const Dev& d, const int nxt, const uint32_t wid, const uint32_t nw) {
    using T = typename Store<S>::T;
    const T* f = static_cast<const T*>(d.f[nxt]);
    float* phi = d.phi[nxt];
    const uint32_t n1 = list_len(&d.sc->n_conv, d.wl_cap);
    const uint32_t n2 = list_len(&d.sc->n_newif, d.wl_cap);
    const uint32_t n3 = list_len(&d.sc->n_fromliq, d.wl_cap);
    const int lane = threadIdx.x & 31;
    // every change of type or fill level also updates the bubble volumes (interface part
    // 1 - phi, gas cells) and the interface count
    for (uint32_t e = wid; e < n1 + n2 + n3; e += nw) {
        if (e < n1) {
            const size_t i = d.wl_conv[e];
            const uint8_t mk = d.mark[i];
            if (lane == 0 && (mk & (K_FILLED | K_EMPTIED))) {
                const uint32_t b = d.owner[i];
                const double was = 1.0 - (double)phi[i];
                if (mk & K_FILLED) {
                    d.flags[i] = F_LIQ;
                    d.owner[i] = kNone;
                    vol_change(d, b, -was, 0, -1);
                } else {
                    d.flags[i] = F_GAS;
                    vol_change(d, b, -was, 1, -1);
                }
            }
            if (lane == 0 || lane >= kQ) continue;
            int x, y, z;
            cell_xyz(d, i, x, y, z);
            size_t j;
            if (!nbr(d, x, y, z, cx(lane), cy(lane), cz(lane), j)) continue;
            // a receiving interface cell is claimed once (it may neighbour several converting
            // cells): its fill level from its new mass
            const uint8_t mj = mark_and(d.mark, j, K_RECV);
            if ((mj & K_RECV) && !(mj & (K_NEWIF | K_FROMLIQ))) {
                float dr = 0.f;
                for (int q = 0; q < kQ; q++) dr += Store<S>::get_nc(f, (size_t)q * d.N + j);
                const float was = phi[j];
                const float now = d.mass[j] / (1.f + dr);
                phi[j] = now;
                vol_change(d, d.owner[j], (double)was - (double)now, 0, 0);
            }
        } else {
            const bool newif = e < n1 + n2;
            const size_t i = newif ? d.wl_newif[e - n1] : d.wl_fromliq[e - n1 - n2];
            const float r = warp_cell_rho<S>(d, f, i, lane);
            if (lane == 0) {
                d.flags[i] = F_IF;
                const float now = d.mass[i] / r;
                phi[i] = now;
                vol_change(d, d.owner[i], 1.0 - (double)now, newif ? -1 : 0, 1);
            }
        }
    }
}

// (vii) BULK bits of every cell whose type changed and of its neighbours (the boundary list
// and the fix list follow); marks cleared
__device__ inline void conv_bulk(const Dev& d, const uint32_t wid, const uint32_t nw) {
    const uint32_t n1 = list_len(&d.sc->n_conv, d.wl_cap);
    const uint32_t n2 = list_len(&d.sc->n_newif, d.wl_cap);
    const uint32_t n3 = list_len(&d.sc->n_fromliq, d.wl_cap);
    const int lane = threadIdx.x & 31;
    for (uint32_t e = wid; e < n1 + n2 + n3; e += nw) {
        const size_t i = e < n1 ? d.wl_conv[e] : (e < n1 + n2 ? d.wl_newif[e - n1] : d.wl_fromliq[e - n1 - n2]);
        if (lane >= kQ) continue;
        size_t j = i;
        if (lane > 0) {
            int x, y, z;
            cell_xyz(d, i, x, y, z);
            if (!nbr(d, x, y, z, cx(lane), cy(lane), cz(lane), j)) continue;
            merge_check(d, i, j);   // a changed cell against each neighbour
        }
        set_bulk(d, j);
        d.mark[j] = 0;
    }
}


}  // namespace lbm
