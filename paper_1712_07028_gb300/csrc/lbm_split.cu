// lbm_split.cu -- bubble splitting: a bubble is one connected gas region (Sec. 2.2).
//
// Every split_every steps, after the step close (the bubble model), six launches on the
// end-of-step stream (the host enqueues them only in the steps that split; each also checks
// the step counter and returns at once on any other step).
//   canon    every gas / interface cell takes its bubble's root id (its gas count moves with
//            it) and is listed; its union-find label starts at its lowest-indexed neighbour of
//            the same bubble (or itself); cells per id are counted; the part table is cleared
//            (the passes below walk the list)
//   hook     each pair of D3Q19 neighbours of one bubble is joined: union-find over the cell
//            indices, the larger root linked under the smaller by compare-and-swap, finds
//            with path halving, so a part's final label is its lowest cell index
//   compress labels point at their roots; each part's lowest cell enters the part table
//   volume   each part's volume (gas cell 1, interface cell 1 - phi) in FP64
//   decide   one block: ids without cells are freed; for each bubble (increasing id) with
//            several parts the largest keeps the id (volumes within 1e-9 of each other: the
//            part with the lower lowest index) and every other part of non-zero volume, in
//            the order of the parts' lowest indices, takes the lowest free id, gas mass and
//            reference volume in proportion to the parts' volumes
//   relabel  the cells of those parts take their new ids (their gas counts move too)
// Finds and unions are bounded; one that runs past the bound, or a part table that fills,
// marks the step as failed: its canonical ids stay, nothing splits, status S_SPLIT.
#include "lbm_internal.cuh"

namespace lbm {

// a label is never above its cell's index (links go from the larger root to the smaller, path
// halving only skips to ancestors), so finds end within a part's size and unions retry only
// while their roots are linked elsewhere; the bounds only guard against the unforeseen
constexpr uint32_t kFindBound = 1u << 24;
constexpr uint32_t kUnionBound = 1u << 20;

__device__ __forceinline__ bool split_due(const Dev& d) {
    return d.split_every > 0 && (*(volatile const uint32_t*)&d.sc->steps) % (uint32_t)d.split_every == 0u;
}

// the cell is a gas or interface cell of a bubble id in the table: its bubble id, else kNone
__device__ __forceinline__ uint32_t split_owner(const Dev& d, size_t i) {
    const uint8_t t = d.flags[i];
    if (!(t & (F_IF | F_GAS))) return kNone;
    const uint32_t b = d.owner[i];
    return b < (uint32_t)d.nbub ? b : kNone;
}

// (plain, L1-cached loads: a stale label is still an ancestor, and a stale root is corrected by
// the union's compare-and-swap, which goes to L2 and returns the root's current parent)
__device__ uint32_t uf_find(uint32_t* lab, uint32_t x, uint32_t* fail) {
    for (uint32_t it = 0; it < kFindBound; it++) {
        const uint32_t p = lab[x];
        if (p == x) return x;
        const uint32_t gp = lab[p];
        if (gp != p) __stcg(lab + x, gp);   // path halving: gp is an ancestor of x
        x = gp;
    }
    atomicExch(fail, 1u);
    return x;
}

// a find that writes nothing: while every thread stores its cell's root, a path-halving store
// could put back an ancestor over a root already stored
__device__ uint32_t uf_root(const uint32_t* lab, uint32_t x, uint32_t* fail) {
    for (uint32_t it = 0; it < kFindBound; it++) {
        const uint32_t p = __ldcg(lab + x);
        if (p == x) return x;
        x = p;
    }
    atomicExch(fail, 1u);
    return x;
}

__device__ void uf_union(uint32_t* lab, uint32_t a, uint32_t b, uint32_t* fail) {
    for (uint32_t it = 0; it < kUnionBound; it++) {
        a = uf_find(lab, a, fail);
        b = uf_find(lab, b, fail);
        if (a == b) return;
        if (a < b) { const uint32_t t = a; a = b; b = t; }   // a: the larger root
        const uint32_t old = atomicCAS(lab + a, a, b);
        if (old == a) return;
        a = old;   // a was linked meanwhile: carry on from where it went
    }
    atomicExch(fail, 1u);
}

__device__ __forceinline__ uint32_t part_hash(uint32_t rep) { return (rep * 2654435761u) & (uint32_t)(kPartCap - 1); }

__device__ __forceinline__ int part_slot(const Dev& d, uint32_t rep) {
    uint32_t h = part_hash(rep);
    for (int p = 0; p < kPartCap; p++) {
        const uint32_t k = __ldcg(&d.part_key[h]);
        if (k == rep + 1u) return (int)h;
        if (k == 0u) return -1;
        h = (h + 1u) & (uint32_t)(kPartCap - 1);
    }
    return -1;
}

__global__ void split_canon_kernel(const Dev d) {
    if (!split_due(d)) return;
    const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, nt = (size_t)gridDim.x * blockDim.x;
    for (size_t k = t0; k < (size_t)kPartCap; k += nt) {
        d.part_key[k] = 0u;
        d.part_V[k] = 0.0;
        d.part_new[k] = -1;
    }
    if (t0 == 0) d.sc->split_fail = 0u;
    const int lane = threadIdx.x & 31;
    for (size_t i = t0; i < d.N; i += nt) {
        const uint32_t b = split_owner(d, i);
        if (b == kNone) continue;
        uint32_t r = b;
        for (int it = 0; it < 64 && d.bub[r].root != (int)r; it++) r = (uint32_t)d.bub[r].root;
        if (r != b) {
            d.owner[i] = r;
            if (d.flags[i] & F_GAS) {
                atomicAdd(&d.bub[b].ngas, ~0ull);   // - 1
                atomicAdd(&d.bub[r].ngas, 1ull);
            }
        }
        // the first label: the lowest-indexed neighbour of the same bubble, if lower than the cell
        // (a real link of the part, so the forest starts mostly joined and the hook pass finds
        // most pairs already together; neighbours may still carry a member id of the bubble)
        uint32_t l = (uint32_t)i;
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        for (int q = 1; q < kQ; q++) {
            size_t j;
            if (!nbr(d, x, y, z, cx(q), cy(q), cz(q), j) || j >= l) continue;
            uint32_t rj = split_owner(d, j);
            if (rj == kNone) continue;
            for (int it = 0; it < 64 && d.bub[rj].root != (int)rj; it++) rj = (uint32_t)d.bub[rj].root;
            if (rj == r) l = (uint32_t)j;
        }
        d.lab[i] = l;
        const unsigned same = __match_any_sync(__activemask(), r);   // one atomic per bubble and warp
        if (lane == __ffs(same) - 1) atomicAdd(&d.bub_cnt[r], (uint32_t)__popc(same));
        wl_push(d.split_list, &d.sc->n_split_cells, (uint32_t)d.N, (uint32_t)i, &d.sc->status);
    }
}

__device__ __forceinline__ uint32_t split_cells(const Dev& d) {
    return min(*(volatile const uint32_t*)&d.sc->n_split_cells, (uint32_t)d.N);
}

// one thread per listed cell and direction: a union is a chain of dependent loads, so the
// pairs are spread over threads rather than walked one after another by each cell's thread
__global__ void split_hook_kernel(const Dev d) {
    if (!split_due(d)) return;
    const uint64_t n = (uint64_t)split_cells(d) * (kQ - 1);
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
        const size_t i = d.split_list[k / (kQ - 1)];
        const int q = 1 + (int)(k % (kQ - 1));
        const uint32_t r = split_owner(d, i);
        if (r == kNone) continue;
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        size_t j;
        if (!nbr(d, x, y, z, cx(q), cy(q), cz(q), j) || j <= i) continue;   // each pair once
        if (split_owner(d, j) != r) continue;
        uf_union(d.lab, (uint32_t)i, (uint32_t)j, &d.sc->split_fail);
    }
}

__global__ void split_compress_kernel(const Dev d) {
    if (!split_due(d)) return;
    const uint32_t n = split_cells(d);
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const size_t i = d.split_list[k];
        const uint32_t r = split_owner(d, i);
        if (r == kNone) continue;
        const uint32_t rep = uf_root(d.lab, (uint32_t)i, &d.sc->split_fail);
        __stcg(&d.lab[i], rep);
        if (rep != (uint32_t)i) continue;
        uint32_t h = part_hash(rep);   // the part's lowest cell enters the table
        bool in = false;
        for (int p = 0; p < kPartCap && !in; p++) {
            if (atomicCAS(&d.part_key[h], 0u, rep + 1u) == 0u) {
                d.part_root[h] = r;
                in = true;
            }
            h = (h + 1u) & (uint32_t)(kPartCap - 1);
        }
        if (!in) atomicExch(&d.sc->split_fail, 1u);
    }
}

__global__ void split_volume_kernel(const Dev d, const int g) {
    if (!split_due(d) || *(volatile const uint32_t*)&d.sc->split_fail) return;
    const float* phi = d.phi[g];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    // every warp runs the same number of rounds: a warp whose cells all belong to one part (the
    // common case) sums them first, one FP64 atomic instead of 32 on the same address
    const uint32_t n = split_cells(d);
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t k = base + threadIdx.x;
        const size_t i = k < n ? d.split_list[k] : 0;
        int s = -1;
        double v = 0.0;
        if (k < n && split_owner(d, i) != kNone) {
            s = part_slot(d, __ldcg(&d.lab[i]));
            if (s >= 0) v = (d.flags[i] & F_GAS) ? 1.0 : 1.0 - (double)phi[i];
        }
        const unsigned has = __ballot_sync(full, s >= 0);
        if (!has) continue;
        const int s0 = __shfl_sync(full, s, __ffs(has) - 1);
        if (__all_sync(full, s < 0 || s == s0)) {
            const double w = warp_sum(v);
            if (lane == 0) atomicAdd(&d.part_V[s0], w);
        } else if (s >= 0) {
            atomicAdd(&d.part_V[s], v);
        }
    }
}

// one block of kDecideThreads threads
constexpr int kDecideThreads = 256;
__global__ void __launch_bounds__(kDecideThreads) split_decide_kernel(const Dev d) {
    if (!split_due(d)) return;
    __shared__ uint32_t sSlot[kPartCap];    // used slots, then in (bubble, lowest index) order
    __shared__ uint32_t sOrder[kPartCap];
    __shared__ uint32_t sN;
    const int tid = threadIdx.x;
    const bool fail = *(volatile const uint32_t*)&d.sc->split_fail != 0u;
    // ids without cells are free rows
    for (int b = tid; b < d.nbub; b += blockDim.x) {
        if (__ldcg(&d.bub_cnt[b]) != 0u) continue;
        Bubble& B = d.bub[b];
        B.V0 = B.V = B.Vif = B.mg = 0.0;
        B.ngas = 0ull;
        B.root = b;
        B.Vtot[0] = B.Vtot[1] = 0.0;
        B.rho_g = (double)d.rho_g0;
        B.rho_gf = d.rho_g0;
    }
    if (tid == 0) sN = 0u;
    __syncthreads();
    if (!fail) {
        for (int s = tid; s < kPartCap; s += blockDim.x)
            if (__ldcg(&d.part_key[s]) != 0u) sSlot[atomicAdd(&sN, 1u)] = (uint32_t)s;
    }
    __syncthreads();
    const uint32_t n = sN;
    // rank of each part by (bubble, lowest cell index)
    for (uint32_t a = tid; a < n; a += blockDim.x) {
        const uint32_t sa = sSlot[a];
        const unsigned long long ka = ((unsigned long long)__ldcg(&d.part_root[sa]) << 32) | __ldcg(&d.part_key[sa]);
        uint32_t rank = 0;
        for (uint32_t e = 0; e < n; e++) {
            const uint32_t se = sSlot[e];
            const unsigned long long ke = ((unsigned long long)__ldcg(&d.part_root[se]) << 32) | __ldcg(&d.part_key[se]);
            rank += ke < ka;
        }
        sOrder[rank] = sa;
    }
    __syncthreads();
    if (tid == 0) {
        if (fail) atomicOr(&d.sc->status, S_SPLIT);
        uint32_t next_free = 0;
        for (uint32_t a = 0; a < n;) {
            const uint32_t r = __ldcg(&d.part_root[sOrder[a]]);
            uint32_t e_end = a;
            while (e_end < n && __ldcg(&d.part_root[sOrder[e_end]]) == r) e_end++;
            uint32_t keep = a;
            double Vr = 0.0;
            for (uint32_t e = a; e < e_end; e++) {
                const double V = __ldcg(&d.part_V[sOrder[e]]);
                Vr += V;
                if (V > __ldcg(&d.part_V[sOrder[keep]]) * (1.0 + 1e-9)) keep = e;
            }
            if (e_end - a >= 2 && Vr > 0.0) {
                Bubble& R = d.bub[r];
                const double V0r = R.V0, mgr = R.mg;
                double kept = 1.0;
                for (uint32_t e = a; e < e_end; e++) {
                    const double V = __ldcg(&d.part_V[sOrder[e]]);
                    if (e == keep || !(V > 0.0)) continue;
                    while (next_free < (uint32_t)d.nbub && __ldcg(&d.bub_cnt[next_free]) != 0u) next_free++;
                    if (next_free >= (uint32_t)d.nbub) {
                        atomicOr(&d.sc->status, S_SPLIT);
                        continue;
                    }
                    const uint32_t id = next_free;
                    d.bub_cnt[id] = 1u;   // taken
                    const double share = V / Vr;
                    Bubble& F = d.bub[id];
                    F.root = (int)id;
                    F.V0 = V0r * share;
                    F.mg = mgr * share;
                    F.V = V;
                    F.rho_g = F.mg / V;
                    F.rho_gf = (float)F.rho_g;
                    F.Vif = 0.0;
                    F.ngas = 0ull;
                    F.Vtot[0] = F.Vtot[1] = 0.0;
                    d.part_new[sOrder[e]] = (int32_t)id;
                    kept -= share;
                    d.sc->n_split++;
                    if (id + 1u > d.sc->nbub_hw) d.sc->nbub_hw = id + 1u;
                }
                R.V0 = V0r * kept;
                R.mg = mgr * kept;
                R.V = Vr * kept;
                if (R.V > 0.0) R.rho_g = R.mg / R.V;
                R.rho_gf = (float)R.rho_g;
            }
            a = e_end;
        }
    }
    __syncthreads();
    for (int b = tid; b < d.nbub; b += blockDim.x) d.bub_cnt[b] = 0u;
}

__global__ void split_relabel_kernel(const Dev d) {
    if (!split_due(d) || *(volatile const uint32_t*)&d.sc->split_fail) return;
    const uint32_t n = split_cells(d);
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const size_t i = d.split_list[k];
        const uint32_t b = split_owner(d, i);
        if (b == kNone) continue;
        const int s = part_slot(d, __ldcg(&d.lab[i]));
        if (s < 0) continue;
        const int32_t F = __ldcg(&d.part_new[s]);
        if (F < 0) continue;
        d.owner[i] = (uint32_t)F;
        if (d.flags[i] & F_GAS) {
            atomicAdd(&d.bub[b].ngas, ~0ull);
            atomicAdd(&d.bub[F].ngas, 1ull);
        }
    }
}

// the split step's kernels on stream s (grid g: the one the step wrote)
void launch_split(const Dev& d, int g, cudaStream_t s) {
    if (d.split_every <= 0) return;
    // small grids: these passes run beside the bulk sweep, whose blocks hold most SM slots, and
    // a grid of a few hundred blocks gets its slots sooner than one of thousands
    const int tb = 256;
    cudaMemsetAsync(&d.sc->n_split_cells, 0, sizeof(uint32_t), s);   // the canon pass lists afresh
    split_canon_kernel<<<152 * 4, tb, 0, s>>>(d);
    split_hook_kernel<<<152 * 4, tb, 0, s>>>(d);
    split_compress_kernel<<<152, tb, 0, s>>>(d);
    split_volume_kernel<<<152, tb, 0, s>>>(d, g);
    split_decide_kernel<<<1, kDecideThreads, 0, s>>>(d);
    split_relabel_kernel<<<152, tb, 0, s>>>(d);
}

}  // namespace lbm
