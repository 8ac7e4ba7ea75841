// lbm_surface.cu -- free-surface bookkeeping after the sweep (Sec. 2.2 of the paper):
// cell conversions with layer closure, equilibrium initialisation of new interface cells,
// excess-mass redistribution, the bubble model, curvature, initial fields and exports.
//
// Conversions run as phases over compact worklists (the sweep appends every interface cell
// whose fill level crossed a threshold), so their cost scales with the number of converting
// cells, not with the grid.  Marks live in a separate byte array that is all zero outside
// this phase; every phase that a later phase depends on ends at a kernel boundary.
#include "lbm_conv.cuh"

namespace lbm {


// all conversion phases in one launch: one cluster of kClusterCtas blocks, the phases separated
// by cluster barriers (every thread reaches every barrier)
constexpr int kClusterCtas = 8;
constexpr int kClusterThreads = 1024;
template <int S>
__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kClusterThreads) conversions_kernel(const Dev d, const int nxt, const int close) {
    const uint32_t wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    // the fix list of the last step has been consumed by the sweep's fix pass; this step's
    // BULK updates (here and in the cover kernels after this launch) fill it again
    if (blockIdx.x == 0 && threadIdx.x == 0) { d.sc->n_fix = 0; d.sc->fix_all = 0; }
    // no interface cell crossed a threshold: nothing converts (every thread reads the same
    // count: it is reset only by a step close, which no thread reaches before all have read it)
    if (*(volatile const uint32_t*)&d.sc->n_conv == 0u) {
        if (close) step_close(d, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, false, ClusterSync{});
        return;
    }
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
    if (close) {   // no cover kernel follows: this launch closes the step (the same for all threads)
        cluster_sync();
        step_close(d, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x, false, ClusterSync{});
    }
}

void launch_conversions(const Dev& d, int nxt, bool close, cudaStream_t s) {
    const int c = close ? 1 : 0;
    switch (d.storage) {
        case LBM_STORE_F32: conversions_kernel<LBM_STORE_F32><<<kClusterCtas, kClusterThreads, 0, s>>>(d, nxt, c); break;
        case LBM_STORE_F16DEV: conversions_kernel<LBM_STORE_F16DEV><<<kClusterCtas, kClusterThreads, 0, s>>>(d, nxt, c); break;
        default: conversions_kernel<LBM_STORE_BF16DEV><<<kClusterCtas, kClusterThreads, 0, s>>>(d, nxt, c); break;
    }
}

// --------------------------------------------------------- boundary list
// Append the boundary cells (active, not BULK) of the 16 cells from v * 16, whose types are
// the bytes of w, to the boundary list: interface cells and cells on a free-slip or open face
// to the general segment, the other liquid cells to the liquid segment (from the back).  The
// two counts of a thread are packed in one word (16 bits each: a block of at most 1024
// threads has at most 16384 cells of each kind), scanned over the warp, summed over the block
// and appended with one atomic per segment and block.  Every thread of the block calls it.
__device__ __forceinline__ void blist_append(const Dev& d, size_t v, const uint32_t (&w)[4], uint32_t* sWarp, uint32_t* sBase) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    uint32_t sg = 0u, sl = 0u;
#pragma unroll
    for (int c = 0; c < 16; c++) {
        const uint32_t t = (w[c / 4] >> (8 * (c % 4))) & 0xffu;
        if (!(t & F_ACTIVE) || (t & F_BULK)) continue;
        bool liq = (t & F_LIQ) != 0;
        if (liq && d.special) {
            int x, y, z;
            cell_xyz(d, v * 16 + c, x, y, z);
            liq = !at_special_face(d, x, y, z);
        }
        if (liq) sl |= 1u << c;
        else sg |= 1u << c;
    }
    const uint32_t cnt = (uint32_t)__popc(sg) | ((uint32_t)__popc(sl) << 16);
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) sWarp[threadIdx.x >> 5] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) {
            const uint32_t x = sWarp[k];
            sWarp[k] = acc;
            acc += x;
        }
        sBase[0] = (acc & 0xffffu) ? atomicAdd(&d.sc->n_slow, acc & 0xffffu) : 0u;
        sBase[1] = (acc >> 16) ? atomicAdd(&d.sc->n_liq, acc >> 16) : 0u;
    }
    __syncthreads();
    const uint32_t pre = sWarp[threadIdx.x >> 5] + incl - cnt;
    uint32_t slot = sBase[0] + (pre & 0xffffu);
    uint32_t slotl = sBase[1] + (pre >> 16);
    __syncthreads();   // sWarp / sBase are rewritten by the next call
    const uint32_t N = (uint32_t)d.N;
    while (sg) {
        const int c = __ffs(sg) - 1;
        sg &= sg - 1;
        if (slot < N) d.wl_slow[slot] = (uint32_t)(v * 16 + c);
        slot++;
    }
    while (sl) {
        const int c = __ffs(sl) - 1;
        sl &= sl - 1;
        if (slotl < N) d.wl_slow[N - 1u - slotl] = (uint32_t)(v * 16 + c);
        slotl++;
    }
}

// --------------------------------------------------------- initial scan
// One pass over the initial cell types: the active cells the bulk sweep leaves to the
// boundary sweep form the first boundary list; each bubble's gas cells are counted and V_b(0) = #gas cells + sum over its interface cells
// of (1 - phi) is summed in FP64 (bubble model, Sec. 2.2); the interface cells are counted.
// The last block to finish sets the reference volumes and rho_g = rho_g0.
__global__ void init_scan_kernel(const Dev d) {
    extern __shared__ unsigned char smem_raw[];
    double* sV = reinterpret_cast<double*>(smem_raw);
    unsigned long long* sG = reinterpret_cast<unsigned long long*>(sV + d.max_bub);
    __shared__ unsigned int sIf;
    __shared__ bool last;
    __shared__ uint32_t sWarp[32];
    __shared__ uint32_t sBase[2];
    for (int b = threadIdx.x; b < d.nbub; b += blockDim.x) { sV[b] = 0.0; sG[b] = 0ull; }
    if (threadIdx.x == 0) sIf = 0;
    __syncthreads();
    const float* phi = d.phi[0];
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
        blist_append(d, v, w, sWarp, sBase);   // boundary cells
        // bubble volumes: owners and fill levels of the chunk's gas / interface cells
        if (!((w[0] | w[1] | w[2] | w[3]) & 0x06060606u)) continue;
        // bubbles that touch from the start (the steps check every cell that changes)
#pragma unroll 1
        for (int c = 0; c < 16; c++) {
            const uint8_t t = (uint8_t)(w[c / 4] >> (8 * (c % 4)));
            if (!(t & (F_IF | F_GAS))) continue;
            const size_t ic = v * 16 + c;
            int x, y, z;
            cell_xyz(d, ic, x, y, z);
            for (int q = 1; q < kQ; q++) {
                size_t j;
                if (nbr(d, x, y, z, cx(q), cy(q), cz(q), j)) merge_check(d, ic, j);
            }
        }
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
    // the lanes' last partial sums: summed over the warp first when the lanes agree on the
    // bubble (the common case: one shared atomic per warp instead of one per lane)
    const uint32_t lead = __reduce_min_sync(full, cb);
    if (__all_sync(full, cb == lead || cb == kNone)) {
        const double sv = warp_sum(cb == kNone ? 0.0 : cv);
        const unsigned sg = __reduce_add_sync(full, cb == kNone ? 0u : (unsigned)cg);
        if (lane == 0 && lead != kNone) {
            if (sv != 0.0) atomicAdd(&sV[lead], sv);
            if (sg) atomicAdd(&sG[lead], (unsigned long long)sg);
        }
    } else if (cb != kNone) {
        if (cv != 0.0) atomicAdd(&sV[cb], cv);
        if (cg) atomicAdd(&sG[cb], cg);
    }
    const unsigned nifw = __reduce_add_sync(full, nif);
    if (lane == 0 && nifw) atomicAdd(&sIf, nifw);
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
    // V0 = V and rho_g = rho_g0; bubbles that touch from the start are merged.  The gas count
    // carries over; the sweep sums the interface part afresh
    bubbles_close(d, threadIdx.x, blockDim.x, true, BlockSync{});
    if (threadIdx.x == 0) {
        Scalars& c = *d.sc;
        c.n_iface = *(volatile uint32_t*)&c.n_iface_acc;
        c.n_iface_acc = 0;
        c.share = 0.0;
        c.share_f = 0.f;
        c.ticket = 0;
    }
}

void launch_init_scan(const Dev& d, cudaStream_t s) {
    const size_t shm = (size_t)d.max_bub * (sizeof(double) + sizeof(unsigned long long));
    const size_t nvec = d.N / 16 + 1;
    int blocks = (int)((nvec + 511) / 512);
    if (blocks > 152 * 4) blocks = 152 * 4;
    init_scan_kernel<<<blocks, 512, shm, s>>>(d);
}

// One pass over the cell types as the step leaves them: the active cells that are not BULK,
// in scan order (blocks of 8192 consecutive cells appended whole), are the next boundary
// sweep's list, split into its general and liquid segments.  Scan order keeps the boundary sweep's accesses local: a list kept by
// appending cells in the order they changed made it ~40 % slower.  The list length is zero
// on entry (the step close resets it).
__global__ void list_rescan_kernel(const Dev d) {
    __shared__ uint32_t sWarp[32];
    __shared__ uint32_t sBase[2];
    const size_t nvec = d.N / 16;
    const size_t total = nvec + (d.N % 16 ? 1 : 0);
    const uint4* fl4 = reinterpret_cast<const uint4*>(d.flags);
    // every thread of the block runs the same number of rounds (block collectives below)
    for (size_t base = blockIdx.x * (size_t)blockDim.x; base < total; base += (size_t)gridDim.x * blockDim.x) {
        const size_t v = base + threadIdx.x;
        uint32_t w[4] = {0u, 0u, 0u, 0u};
        if (v < nvec) {
            const uint4 p = fl4[v];
            w[0] = p.x; w[1] = p.y; w[2] = p.z; w[3] = p.w;
        } else if (v < total) {
            for (size_t c = v * 16; c < d.N; c++) w[(c - v * 16) / 4] |= (uint32_t)d.flags[c] << (8 * ((c - v * 16) % 4));
        }
        blist_append(d, v, w, sWarp, sBase);
    }
}

void launch_list_rescan(const Dev& d, cudaStream_t s) {   // after the step close (list length 0)
    const size_t nvec = d.N / 16 + 1;
    int blocks = (int)((nvec + 511) / 512);
    if (blocks > 152 * 2) blocks = 152 * 2;   // (beside the bulk sweep: a share of the SMs' warp slots)
    list_rescan_kernel<<<blocks, 512, 0, s>>>(d);
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
// With g32 (the bubbles' centres and r - 1/2 in FP32, where no bubble nears half a periodic
// period), a bubble whose FP32 distance clears the blend shell c in [0, 1] by a margin of 1e-3
// (four times the FP32 error of coordinates up to 4096) contributes its clamped factor, 1 or 0,
// without FP64;
// FP64 decides the cells near the shell, so the result is the FP64 formula's.  *minc (if given)
// receives the smallest FP32 c over the bubbles.
__device__ void bubble_fill(const Dev& d, const double* geo, const float4* g32, int x, int y, int z, float& ph,
                            uint32_t& own, float* minc = nullptr) {
    double v = 1.0;
    own = kNone;
    float mc = 3.0e38f;
    for (int b = 0; b < d.ngeo; b++) {
        if (g32) {
            const float4 gb = g32[b];
            float dx = (float)x - gb.x, dy = (float)y - gb.y, dz = (float)z - gb.z;
            if (d.bc[0]) dx -= (float)d.nx * rintf(dx / (float)d.nx);
            if (d.bc[1]) dy -= (float)d.ny * rintf(dy / (float)d.ny);
            if (d.bc[2]) dz -= (float)d.nz * rintf(dz / (float)d.nz);
            const float c32 = sqrtf(dx * dx + dy * dy + dz * dz) - gb.w;
            mc = fminf(mc, c32);
            if (c32 > 1.001f) continue;   // factor 1
            if (c32 < -0.001f) {          // factor 0
                if (own == kNone) own = (uint32_t)b;
                v = 0.0;
                continue;
            }
        }
        const double ddx = min_image(d, 0, (double)x, geo[4 * b + 0]);
        const double ddy = min_image(d, 1, (double)y, geo[4 * b + 1]);
        const double ddz = min_image(d, 2, (double)z, geo[4 * b + 2]);
        double c = sqrt(ddx * ddx + ddy * ddy + ddz * ddz) - (geo[4 * b + 3] - 0.5);
        c = c < 0.0 ? 0.0 : (c > 1.0 ? 1.0 : c);
        if (c < 1.0 && own == kNone) own = (uint32_t)b;
        v *= c;
    }
    ph = (float)v;
    if (minc) *minc = mc;
}

template <int S>
__global__ void init_kernel(const Dev d, const double* geo, const int use32) {
    using T = typename Store<S>::T;
    T* f = static_cast<T*>(d.f[0]);
    extern __shared__ float4 sg32[];   // (with use32) the bubbles' centres and r - 1/2 in FP32
    if (use32) {
        for (int b = threadIdx.x; b < d.ngeo; b += blockDim.x)
            sg32[b] = make_float4((float)geo[4 * b], (float)geo[4 * b + 1], (float)geo[4 * b + 2], (float)(geo[4 * b + 3] - 0.5));
        __syncthreads();
    }
    const float4* g32 = use32 ? sg32 : nullptr;
    // every bubble its own root; its initial gas density: rho_gas0, or (hydrostatic start) the
    // liquid's pressure at its centre plus the Laplace jump 2 sigma / r, as a density (p = rho/3)
    // (rows beyond the given bubbles, room for splitting, start free: no cells, no gas)
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < d.nbub; b += gridDim.x * blockDim.x) {
        d.bub[b].root = b;
        d.bub[b].rho_g = d.hydrostatic && b < d.ngeo
                             ? exp(3.0 * d.gz * (geo[4 * b + 2] - (d.nz - 0.5))) + 6.0 * (double)d.sigma / geo[4 * b + 3]
                             : (double)d.rho_g0;
        d.bub[b].rho_gf = (float)d.bub[b].rho_g;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) d.sc->nbub_hw = (uint32_t)d.ngeo;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < d.N; i += (size_t)gridDim.x * blockDim.x) {
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        float ph, minc;
        uint32_t own;
        bubble_fill(d, geo, g32, x, y, z, ph, own, &minc);
        uint8_t t = ph <= 0.f ? F_GAS : (ph >= 1.f ? F_LIQ : F_IF);
        // layer closure (a neighbour, at most sqrt 2 away, can be gas only where some bubble's c
        // is below sqrt 2: with the FP32 distances, a margin beyond that)
        if (t == F_LIQ && d.nbub > 0 && (!g32 || minc < 1.5f)) {
            for (int q = 1; q < kQ; q++) {
                size_t j;
                if (!nbr(d, x, y, z, cx(q), cy(q), cz(q), j)) continue;
                int a, b, c;
                cell_xyz(d, j, a, b, c);
                float pj;
                uint32_t oj;
                bubble_fill(d, geo, g32, a, b, c, pj, oj);
                if (pj <= 0.f) { t = F_IF; ph = 1.f; own = oj; break; }
            }
        }
        if (t == F_LIQ) own = kNone;
        // initial density: 1, or the hydrostatic profile below the open top's plane nz - 1/2
        const float rho = d.hydrostatic ? (float)exp(3.0 * d.gz * ((double)z - (d.nz - 0.5))) : 1.f;
        float m = ph * rho;
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
        for (int q = 0; q < kQ; q++) Store<S>::put(f, (size_t)q * d.N + i, wgt(q) * (rho - 1.f));   // e(rho, 0) - w
        if (d.rho[0]) d.rho[0][i] = rho;
    }
}

template <int S>
__global__ void rho_of_grid_kernel(const Dev d, const int g) {
    using T = typename Store<S>::T;
    const T* f = static_cast<const T*>(d.f[g]);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < d.N; i += (size_t)gridDim.x * blockDim.x) {
        if (!(d.flags[i] & F_ACTIVE)) continue;
        float dr = 0.f;
        for (int q = 0; q < kQ; q++) dr += Store<S>::get_nc(f, (size_t)q * d.N + i);
        d.rho[g][i] = 1.f + dr;
    }
}
void launch_rho_of_grid(const Dev& d, int g, cudaStream_t s) {
    switch (d.storage) {
        case LBM_STORE_F32: rho_of_grid_kernel<LBM_STORE_F32><<<152 * 16, 256, 0, s>>>(d, g); break;
        case LBM_STORE_F16DEV: rho_of_grid_kernel<LBM_STORE_F16DEV><<<152 * 16, 256, 0, s>>>(d, g); break;
        default: rho_of_grid_kernel<LBM_STORE_BF16DEV><<<152 * 16, 256, 0, s>>>(d, g); break;
    }
}

void launch_init(const Dev& d, const double* geo, cudaStream_t s) {
    // the FP32 prefilter of the fill levels: its table in shared memory, and no bubble within two
    // cells of half a periodic period (where an FP32 minimum image could pick another image)
    bool use32 = d.ngeo > 0 && d.ngeo <= 2048 && d.nx <= 4096 && d.ny <= 4096 && d.nz <= 4096;
    if (use32 && d.geo_rmax + 2.0 >= 0.5 * (double)std::min(d.bc[0] ? d.nx : 1 << 30,
                                                              std::min(d.bc[1] ? d.ny : 1 << 30, d.bc[2] ? d.nz : 1 << 30)))
        use32 = false;
    const size_t shm = use32 ? sizeof(float4) * (size_t)d.ngeo : 0;
    switch (d.storage) {
        case LBM_STORE_F32: init_kernel<LBM_STORE_F32><<<152 * 16, 256, shm, s>>>(d, geo, use32 ? 1 : 0); break;
        case LBM_STORE_F16DEV: init_kernel<LBM_STORE_F16DEV><<<152 * 16, 256, shm, s>>>(d, geo, use32 ? 1 : 0); break;
        default: init_kernel<LBM_STORE_BF16DEV><<<152 * 16, 256, shm, s>>>(d, geo, use32 ? 1 : 0); break;
    }
}

__global__ void bulk_all_kernel(const Dev d) {   // initial BULK bits (nothing to fix)
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < d.N; i += (size_t)gridDim.x * blockDim.x)
        set_bulk_init(d, i);
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
            if (t & F_ACTIVE) post_moments<S>(d, f, i, (t & F_IF) ? d.phi[cur][i] : 1.f, r, v);
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
