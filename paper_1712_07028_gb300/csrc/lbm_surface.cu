// lbm_surface.cu -- free-surface bookkeeping after the sweep (Sec. 2.2 of the paper):
// cell conversions with layer closure, equilibrium initialisation of new interface cells,
// excess-mass redistribution, the bubble model, curvature, initial fields and exports.
//
// Conversions run as phases over compact worklists (the sweep appends every interface cell
// whose fill level crossed a threshold), so their cost scales with the number of converting
// cells, not with the grid.  Marks live in a separate byte array that is all zero outside
// this phase; every phase that a later phase depends on ends at a kernel boundary.
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
__device__ void py_gradient(const Dev& d, const float* phi, int x, int y, int z, float n[3]) {
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
            post_moments<S>(d, f, j, r, u);
            c = 1;
        }
        const int cnt = warp_sum(c);
        const float rs = warp_sum(r), ux = warp_sum(u[0]), uy = warp_sum(u[1]), uz = warp_sum(u[2]);
        const float rb = cnt ? rs / cnt : 1.f;
        const float ub[3] = {cnt ? ux / cnt : 0.f, cnt ? uy / cnt : 0.f, cnt ? uz / cnt : 0.f};
        if (lane < kQ) Store<S>::put(f, (size_t)lane * d.N + i, equilibrium_dev(lane, rb, ub));
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
    for (uint32_t e = wid; e < n1 + n2 + n3; e += nw) {
        if (e < n1) {
            const size_t i = d.wl_conv[e];
            const uint8_t mk = d.mark[i];
            if (lane == 0) {
                if (mk & K_FILLED) { d.flags[i] = F_LIQ; d.owner[i] = kNone; }
                else if (mk & K_EMPTIED) { d.flags[i] = F_GAS; }
            }
            if (lane == 0 || lane >= kQ) continue;
            int x, y, z;
            cell_xyz(d, i, x, y, z);
            size_t j;
            if (!nbr(d, x, y, z, cx(lane), cy(lane), cz(lane), j)) continue;
            const uint8_t mj = d.mark[j];
            if ((mj & K_RECV) && !(mj & (K_NEWIF | K_FROMLIQ))) {
                float dr = 0.f;
                for (int q = 0; q < kQ; q++) dr += Store<S>::get_nc(f, (size_t)q * d.N + j);
                phi[j] = d.mass[j] / (1.f + dr);
            }
        } else {
            const size_t i = e < n1 + n2 ? d.wl_newif[e - n1] : d.wl_fromliq[e - n1 - n2];
            const float r = warp_cell_rho<S>(d, f, i, lane);
            if (lane == 0) {
                d.flags[i] = F_IF;
                phi[i] = d.mass[i] / r;
            }
        }
    }
}

// (vii) BULK bits of every cell whose type changed and of its neighbours; marks cleared
__device__ void conv_bulk(const Dev& d, const uint32_t wid, const uint32_t nw) {
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
        }
        set_bulk(d, j);
        d.mark[j] = 0;
    }
}

// barrier of all threads of the thread-block cluster, ordering their global-memory writes
// before the reads that follow (release / acquire at cluster scope); a hardware barrier, not a
// spin on memory
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// all conversion phases in one launch: one cluster of kClusterCtas blocks, the phases separated
// by cluster barriers (every thread reaches every barrier)
constexpr int kClusterCtas = 8;
constexpr int kClusterThreads = 1024;
template <int S>
__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kClusterThreads) conversions_kernel(const Dev d, const int nxt) {
    const uint32_t wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    // the fix list of the last step has been consumed by the sweep's fix pass; this step's
    // BULK updates (here and in the cover kernels after this launch) fill it again
    if (blockIdx.x == 0 && threadIdx.x == 0) { d.sc->n_fix = 0; d.sc->fix_all = 0; }
    conv_filled_emptied<S>(d, nxt, wid, nw);
    cluster_sync();
    // new-interface initialisation writes only the new cells' PDFs; the excess phase reads
    // only converting cells' PDFs and adds to masses: the two share a phase
    conv_newif<S>(d, nxt, wid, nw);
    conv_excess<S>(d, nxt, wid, nw);
    cluster_sync();
    conv_finalize<S>(d, nxt, wid, nw);
    cluster_sync();
    conv_bulk(d, wid, nw);
    // the boundary list of this step has been consumed by the sweep; the end-of-step scan
    // fills it again
    if (blockIdx.x == 0 && threadIdx.x == 0) d.sc->n_slow = 0;
}

void launch_conversions(const Dev& d, int nxt, cudaStream_t s) {
    switch (d.storage) {
        case LBM_STORE_F32: conversions_kernel<LBM_STORE_F32><<<kClusterCtas, kClusterThreads, 0, s>>>(d, nxt); break;
        case LBM_STORE_F16DEV: conversions_kernel<LBM_STORE_F16DEV><<<kClusterCtas, kClusterThreads, 0, s>>>(d, nxt); break;
        default: conversions_kernel<LBM_STORE_BF16DEV><<<kClusterCtas, kClusterThreads, 0, s>>>(d, nxt); break;
    }
}

// --------------------------------------------------------- end of step: one scan
// One pass over the cell types as the step leaves them: the active cells the bulk sweep
// leaves to the boundary sweep are listed for the next step; each bubble's volume
// V_b = #gas cells + sum over its interface cells of (1 - phi) is summed in FP64 (bubble
// model, Sec. 2.2) and the interface cells are counted.  The last block to finish then
// sets rho_g,b = rho_g0 V_b(0) / V_b (isothermal gas of conserved mass), moves the excess
// pool and the share the next sweep spreads over the interface cells, and resets counters.
__global__ void end_scan_kernel(const Dev d, const int cur, const int set_reference) {
    extern __shared__ unsigned char smem_raw[];
    double* sV = reinterpret_cast<double*>(smem_raw);
    unsigned long long* sG = reinterpret_cast<unsigned long long*>(sV + d.max_bub);
    __shared__ unsigned int sIf;
    __shared__ bool last;
    for (int b = threadIdx.x; b < d.nbub; b += blockDim.x) { sV[b] = 0.0; sG[b] = 0ull; }
    if (threadIdx.x == 0) sIf = 0;
    __syncthreads();
    const float* phi = d.phi[cur];
    const size_t nvec = d.N / 16;
    const size_t total = nvec + (d.N % 16 ? 1 : 0);
    const uint4* fl4 = reinterpret_cast<const uint4*>(d.flags);
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    unsigned int nif = 0;
    uint32_t cb = kNone;
    double cv = 0.0;
    unsigned long long cg = 0ull;
    // every thread of the block runs the same number of rounds (warp collectives below)
    for (size_t base = blockIdx.x * (size_t)blockDim.x; base < total; base += (size_t)gridDim.x * blockDim.x) {
        const size_t v = base + threadIdx.x;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (v < nvec) {
            const uint4 p = fl4[v];
            w[0] = p.x; w[1] = p.y; w[2] = p.z; w[3] = p.w;
        } else if (v < total) {
            for (size_t c = v * 16; c < d.N; c++) w[(c - v * 16) / 4] |= (uint32_t)d.flags[c] << (8 * ((c - v * 16) % 4));
        }
        // boundary cells (active, not BULK): one append per warp
        uint32_t sel = 0u;
#pragma unroll
        for (int c = 0; c < 16; c++) {
            const uint32_t t = (w[c / 4] >> (8 * (c % 4))) & 0xffu;
            sel |= ((t & F_ACTIVE) && !(t & F_BULK)) ? (1u << c) : 0u;
        }
        const uint32_t cnt = __popc(sel);
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(full, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t tot = __shfl_sync(full, incl, 31);
        uint32_t base_slot = 0;
        if (lane == 31 && tot) base_slot = atomicAdd(&d.sc->n_slow, tot);
        base_slot = __shfl_sync(full, base_slot, 31);
        uint32_t slot = base_slot + incl - cnt;
        while (sel) {
            const int c = __ffs(sel) - 1;
            sel &= sel - 1;
            if (slot < (uint32_t)d.N) d.wl_slow[slot] = (uint32_t)(v * 16 + c);
            slot++;
        }
        // bubble volumes: owners and fill levels of the chunk's gas / interface cells
        if (!((w[0] | w[1] | w[2] | w[3]) & 0x06060606u)) continue;
        uint32_t ob[16];
        float pv[16];
#pragma unroll
        for (int c = 0; c < 16; c++) {
            const uint8_t t = (uint8_t)(w[c / 4] >> (8 * (c % 4)));
            ob[c] = (t & (F_IF | F_GAS)) ? d.owner[v * 16 + c] : kNone;
            pv[c] = (t & F_IF) ? phi[v * 16 + c] : 0.f;
        }
#pragma unroll
        for (int c = 0; c < 16; c++) {
            const uint8_t t = (uint8_t)(w[c / 4] >> (8 * (c % 4)));
            if (!(t & (F_IF | F_GAS))) continue;
            const uint32_t b = ob[c];
            if (t & F_IF) nif++;
            if (b >= (uint32_t)d.nbub) continue;
            if (b != cb) {
                if (cb != kNone) {
                    if (cv != 0.0) atomicAdd(&sV[cb], cv);
                    if (cg) atomicAdd(&sG[cb], cg);
                }
                cb = b;
                cv = 0.0;
                cg = 0ull;
            }
            if (t & F_IF) cv += 1.0 - (double)pv[c];
            else cg++;
        }
    }
    if (cb != kNone) {
        if (cv != 0.0) atomicAdd(&sV[cb], cv);
        if (cg) atomicAdd(&sG[cb], cg);
    }
    if (nif) atomicAdd(&sIf, nif);
    // the spheres' bins of this step are emptied (filled again by the next step)
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < d.nsph && d.bin_cnt) {
        const Sphere& sp = d.sph[t];
        d.bin_cnt[bin_index(d, bin_coord(d, 0, sp.x0[0]), bin_coord(d, 1, sp.x0[1]), bin_coord(d, 2, sp.x0[2]))] = 0;
    }
    __syncthreads();
    for (int b = threadIdx.x; b < d.nbub; b += blockDim.x) {
        if (sV[b] != 0.0) atomicAdd(&d.bub[b].Vif, sV[b]);
        if (sG[b]) atomicAdd(&d.bub[b].ngas, sG[b]);
    }
    if (threadIdx.x == 0 && sIf) atomicAdd(&d.sc->n_iface_acc, sIf);
    // the last block to finish sees every block's sums
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&d.sc->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int b = threadIdx.x; b < d.nbub; b += blockDim.x) {
        Bubble& B = d.bub[b];
        const double V = (double)*(volatile unsigned long long*)&B.ngas + *(volatile double*)&B.Vif;
        B.V = V;
        if (set_reference) { B.V0 = V; B.rho_g = (double)d.rho_g0; }
        else if (V > 0.0) B.rho_g = (double)d.rho_g0 * B.V0 / V;
        else atomicOr(&d.sc->status, S_BUBBLE_GONE);
        B.rho_gf = (float)B.rho_g;
        B.ngas = 0ull;
        B.Vif = 0.0;
    }
    if (threadIdx.x == 0) {
        Scalars& c = *d.sc;
        if (c.share != 0.0) c.pool = 0.0;
        c.pool += c.pool_acc;
        c.pool_acc = 0.0;
        c.n_iface = *(volatile uint32_t*)&c.n_iface_acc;
        c.n_iface_acc = 0;
        c.share = (c.pool != 0.0 && c.n_iface > 0) ? c.pool / (double)c.n_iface : 0.0;
        c.share_f = (float)c.share;
        c.n_conv = c.n_newif = c.n_fromliq = c.n_touch = c.n_uncov = 0;
        c.ticket = 0;
    }
}

void launch_end_scan(const Dev& d, int cur, int set_reference, cudaStream_t s) {
    const size_t shm = (size_t)d.max_bub * (sizeof(double) + sizeof(unsigned long long));
    const size_t nvec = d.N / 16 + 1;
    int blocks = (int)((nvec + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    const int need = (d.nsph + 255) / 256;   // one thread per sphere for the bin reset
    if (blocks < need) blocks = need;
    end_scan_kernel<<<blocks, 256, shm, s>>>(d, cur, set_reference);
}

// ---------------------------------------------------------------------- curvature
// kappa = -(1/2) div(n^) of the Parker-Youngs unit normal (central differences; beyond a
// wall the cell's own normal), the mean curvature: -1/R on a gas sphere of radius R
__device__ void unit_normal(const Dev& d, const float* phi, int x, int y, int z, float nh[3]) {
    float n[3];
    py_gradient(d, phi, x, y, z, n);
    const float l = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    nh[0] = l > 0.f ? n[0] / l : 0.f;
    nh[1] = l > 0.f ? n[1] / l : 0.f;
    nh[2] = l > 0.f ? n[2] / l : 0.f;
}

__global__ void curvature_kernel(const Dev d, const int nxt) {
    const float* phi = d.phi[nxt];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < d.N; i += (size_t)gridDim.x * blockDim.x) {
        if (!(d.flags[i] & F_IF)) continue;
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        float n0[3];
        unit_normal(d, phi, x, y, z, n0);
        float div = 0.f;
        for (int k = 0; k < 3; k++) {
            const int dx = k == 0, dy = k == 1, dz = k == 2;
            float np[3], nm[3];
            size_t j;
            if (nbr(d, x, y, z, dx, dy, dz, j)) {
                int a, b, c;
                cell_xyz(d, j, a, b, c);
                unit_normal(d, phi, a, b, c, np);
            } else { np[0] = n0[0]; np[1] = n0[1]; np[2] = n0[2]; }
            if (nbr(d, x, y, z, -dx, -dy, -dz, j)) {
                int a, b, c;
                cell_xyz(d, j, a, b, c);
                unit_normal(d, phi, a, b, c, nm);
            } else { nm[0] = n0[0]; nm[1] = n0[1]; nm[2] = n0[2]; }
            div += 0.5f * (np[k] - nm[k]);
        }
        d.kappa[i] = -0.5f * div;
    }
}

void launch_curvature(const Dev& d, int nxt, cudaStream_t s) {
    curvature_kernel<<<152 * 8, 256, 0, s>>>(d, nxt);
}

// --------------------------------------------------------------------- initial state
// phi = prod_b clamp(|x - c_b| - (r_b - 1/2), 0, 1); gas / liquid / interface; liquid cells
// with a gas neighbour become interface cells (phi = 1) with that gas cell's bubble; f* =
// e(1,0), m = phi; then cells covered by a sphere (lowest id) become obstacle cells.
__device__ void bubble_fill(const Dev& d, const double* geo, int x, int y, int z, float& ph, uint32_t& own) {
    double v = 1.0;
    own = kNone;
    for (int b = 0; b < d.nbub; b++) {
        const double ddx = min_image(d, 0, (double)x, geo[4 * b + 0]);
        const double ddy = min_image(d, 1, (double)y, geo[4 * b + 1]);
        const double ddz = min_image(d, 2, (double)z, geo[4 * b + 2]);
        double c = sqrt(ddx * ddx + ddy * ddy + ddz * ddz) - (geo[4 * b + 3] - 0.5);
        c = c < 0.0 ? 0.0 : (c > 1.0 ? 1.0 : c);
        if (c < 1.0 && own == kNone) own = (uint32_t)b;
        v *= c;
    }
    ph = (float)v;
}

template <int S>
__global__ void init_kernel(const Dev d, const double* geo) {
    using T = typename Store<S>::T;
    T* f = static_cast<T*>(d.f[0]);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < d.N; i += (size_t)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        float ph;
        uint32_t own;
        bubble_fill(d, geo, x, y, z, ph, own);
        uint8_t t = ph <= 0.f ? F_GAS : (ph >= 1.f ? F_LIQ : F_IF);
        if (t == F_LIQ && d.nbub > 0) {   // layer closure
            for (int q = 1; q < kQ; q++) {
                size_t j;
                if (!nbr(d, x, y, z, cx(q), cy(q), cz(q), j)) continue;
                int a, b, c;
                cell_xyz(d, j, a, b, c);
                float pj;
                uint32_t oj;
                bubble_fill(d, geo, a, b, c, pj, oj);
                if (pj <= 0.f) { t = F_IF; ph = 1.f; own = oj; break; }
            }
        }
        if (t == F_LIQ) own = kNone;
        float m = ph;
        if (d.nsph > 0) {
            const uint32_t P = covering_sphere(d, x, y, z);
            if (P != kNone) { t = F_OBS; own = P; m = 0.f; ph = 1.f; }
        }
        d.flags[i] = t;
        d.owner[i] = own;
        d.mass[i] = m;
        d.phi[0][i] = ph;
        d.phi[1][i] = ph;
        if (d.kappa) d.kappa[i] = 0.f;
        for (int q = 0; q < kQ; q++) Store<S>::put(f, (size_t)q * d.N + i, 0.f);   // e(1, 0) - w = 0
    }
}

void launch_init(const Dev& d, const double* geo, cudaStream_t s) {
    switch (d.storage) {
        case LBM_STORE_F32: init_kernel<LBM_STORE_F32><<<152 * 16, 256, 0, s>>>(d, geo); break;
        case LBM_STORE_F16DEV: init_kernel<LBM_STORE_F16DEV><<<152 * 16, 256, 0, s>>>(d, geo); break;
        default: init_kernel<LBM_STORE_BF16DEV><<<152 * 16, 256, 0, s>>>(d, geo); break;
    }
}

__global__ void bulk_all_kernel(const Dev d) {   // initial BULK bits (nothing to fix)
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < d.N; i += (size_t)gridDim.x * blockDim.x)
        set_bulk(d, i, false);
}

void launch_bulk_all(const Dev& d, cudaStream_t s) { bulk_all_kernel<<<152 * 16, 256, 0, s>>>(d); }

// ------------------------------------------------------------------------- exports
template <int S>
__global__ void fields_kernel(const Dev d, const int cur, float* rho, float* u, float* phi, uint8_t* flags) {
    using T = typename Store<S>::T;
    const T* f = static_cast<const T*>(d.f[cur]);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < d.N; i += (size_t)gridDim.x * blockDim.x) {
        const uint8_t t = d.flags[i] & F_TYPE;
        if (rho || u) {
            float r = 0.f, v[3] = {0.f, 0.f, 0.f};
            if (t & F_ACTIVE) post_moments<S>(d, f, i, r, v);
            if (rho) rho[i] = r;
            if (u) { u[i] = v[0]; u[d.N + i] = v[1]; u[2 * d.N + i] = v[2]; }
        }
        if (phi) phi[i] = (t & F_IF) ? d.phi[cur][i] : ((t & F_GAS) ? 0.f : 1.f);
        if (flags) flags[i] = t;
    }
}

template <int S>
__global__ void export_kernel(const Dev d, const int cur, float* f, uint8_t* flags, float* m, float* phi, int32_t* owner, float* kappa) {
    using T = typename Store<S>::T;
    const T* fs = static_cast<const T*>(d.f[cur]);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < d.N; i += (size_t)gridDim.x * blockDim.x) {
        const uint8_t t = d.flags[i] & F_TYPE;
        if (f)
            for (int q = 0; q < kQ; q++) f[(size_t)q * d.N + i] = Store<S>::get_nc(fs, (size_t)q * d.N + i);
        if (flags) flags[i] = t;
        if (m) m[i] = (t & F_IF) ? d.mass[i] : 0.f;
        if (phi) phi[i] = (t & F_IF) ? d.phi[cur][i] : ((t & F_GAS) ? 0.f : 1.f);
        if (owner) owner[i] = d.owner[i] == kNone ? -1 : (int32_t)d.owner[i];
        if (kappa) kappa[i] = d.kappa ? d.kappa[i] : 0.f;
    }
}

#define LBM_DISPATCH(KERNEL, GRID, BLOCK, STREAM, ...)                                              \
    switch (d.storage) {                                                                            \
        case LBM_STORE_F32: KERNEL<LBM_STORE_F32><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;    \
        case LBM_STORE_F16DEV: KERNEL<LBM_STORE_F16DEV><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break; \
        default: KERNEL<LBM_STORE_BF16DEV><<<GRID, BLOCK, 0, STREAM>>>(__VA_ARGS__); break;         \
    }

void launch_fields(const Dev& d, int cur, float* rho, float* u, float* phi, uint8_t* flags, cudaStream_t s) {
    LBM_DISPATCH(fields_kernel, 152 * 8, 256, s, d, cur, rho, u, phi, flags);
}

void launch_export(const Dev& d, int cur, float* f, uint8_t* flags, float* m, float* phi, int32_t* owner, float* kappa, cudaStream_t s) {
    LBM_DISPATCH(export_kernel, 152 * 8, 256, s, d, cur, f, flags, m, phi, owner, kappa);
}

// total liquid mass sum_liquid rho + sum_interface m, in FP64
template <int S>
__global__ void mass_kernel(const Dev d, const int cur) {
    using T = typename Store<S>::T;
    const T* f = static_cast<const T*>(d.f[cur]);
    double acc = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < d.N; i += (size_t)gridDim.x * blockDim.x) {
        const uint8_t t = d.flags[i] & F_TYPE;
        if (t & F_LIQ) {
            double dr = 0.0;
            for (int q = 0; q < kQ; q++) dr += (double)Store<S>::get_nc(f, (size_t)q * d.N + i);
            acc += 1.0 + dr;
        } else if (t & F_IF) {
            acc += (double)d.mass[i];
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&d.sc->mass, acc);
}

void launch_mass(const Dev& d, int cur, cudaStream_t s) {
    LBM_DISPATCH(mass_kernel, 152 * 8, 256, s, d, cur);
}

}  // namespace lbm
