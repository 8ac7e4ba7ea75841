// lbm_internal.cuh -- device-side definitions shared by the CUDA translation units of the
// free-surface LBM library (sm_103a).  Nothing here is shared with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/lbm.h"

namespace lbm {

// D3Q19, q = 0 rest, 1..6 the faces (+x,-x,+y,-y,+z,-z), 7..18 the edges; the opposite of
// q >= 1 is q+1 for odd q and q-1 for even q.
constexpr int kQ = 19;
__host__ __device__ constexpr int cx(int q) {
    return (q == 1 || q == 7 || q == 9 || q == 11 || q == 13) ? 1
         : (q == 2 || q == 8 || q == 10 || q == 12 || q == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int q) {
    return (q == 3 || q == 7 || q == 10 || q == 15 || q == 17) ? 1
         : (q == 4 || q == 8 || q == 9 || q == 16 || q == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int q) {
    return (q == 5 || q == 11 || q == 14 || q == 15 || q == 18) ? 1
         : (q == 6 || q == 12 || q == 13 || q == 16 || q == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }
__host__ __device__ constexpr float wgt(int q) { return q == 0 ? (1.0f / 3.0f) : (q <= 6 ? (1.0f / 18.0f) : (1.0f / 36.0f)); }
// 72 w_q as an integer (24, 4, 2): the constant part of a bounce-back link's momentum
__host__ __device__ constexpr int w72(int q) { return q == 0 ? 24 : (q <= 6 ? 4 : 2); }

// c_q . v, and a + c v for one component c of c_q, with the zero components of c_q left out.
// Under IEEE rules a product with 0.0f cannot be folded away (it turns a NaN or an infinity
// into a NaN), so the plain forms cost a multiply-add per zero component; these cost only the
// additions the lattice needs.  For finite operands the results are those of the plain forms
// (products with +-1 are exact), up to the sign of a zero.
__device__ __forceinline__ float cdot(int q, float vx, float vy, float vz) {
    float r = 0.f;
    bool any = false;
    if (cx(q) != 0) { r = cx(q) > 0 ? vx : -vx; any = true; }
    if (cy(q) != 0) { r = any ? (cy(q) > 0 ? r + vy : r - vy) : (cy(q) > 0 ? vy : -vy); any = true; }
    if (cz(q) != 0) r = any ? (cz(q) > 0 ? r + vz : r - vz) : (cz(q) > 0 ? vz : -vz);
    return r;
}
__device__ __forceinline__ float cacc(int c, float a, float v) { return c > 0 ? a + v : (c < 0 ? a - v : a); }

// cell flag byte: type bits, plus BULK = liquid cell whose 18 neighbours all exist and are
// liquid or interface (it then streams without looking at its neighbours)
enum : uint8_t { F_LIQ = 1, F_IF = 2, F_GAS = 4, F_OBS = 8, F_BULK = 16, F_TYPE = 15 };
enum : uint8_t { F_ACTIVE = F_LIQ | F_IF };
// kinds of the faces of non-periodic axes
enum : uint8_t { FACE_WALL = 0, FACE_SLIP = 1, FACE_OPEN = 2 };
// conversion / covering marks (separate byte array, zero outside the conversion phase)
enum : uint8_t { K_FILLED = 1, K_EMPTIED = 2, K_NEWIF = 4, K_FROMLIQ = 8, K_RECV = 16, K_TOUCH = 32, K_UNCOV = 64 };

constexpr uint32_t kNone = 0xffffffffu;

// ---------------------------------------------------------------- PDF storage traits
// Every storage keeps the deviation f_q - w_q from the rest equilibrium (FP32, FP16 or BF16);
// the kernels compute in deviation form too, so densities and velocities of a nearly
// uniform liquid are not rounded against the O(1) weights.
template <int S> struct Store;
// get_cs / put_cs: streaming accesses (evict first) for the bulk sweep, which passes each PDF
// through once per step; the smaller arrays the latency-bound kernels reuse stay in L2
template <> struct Store<LBM_STORE_F32> {
    using T = float;
    static __device__ __forceinline__ float get(const T* p, size_t i) { return __ldg(p + i); }
    static __device__ __forceinline__ float get_cs(const T* p, size_t i) { return __ldcs(p + i); }
    static __device__ __forceinline__ float get_nc(const T* p, size_t i) { return p[i]; }
    static __device__ __forceinline__ void put(T* p, size_t i, float v) { p[i] = v; }
    static __device__ __forceinline__ void put_cs(T* p, size_t i, float v) { __stcs(p + i, v); }
};
template <> struct Store<LBM_STORE_F16DEV> {
    using T = __half;
    static __device__ __forceinline__ float get(const T* p, size_t i) { return __half2float(__ldg(p + i)); }
    static __device__ __forceinline__ float get_cs(const T* p, size_t i) { return __half2float(__ldcs(p + i)); }
    static __device__ __forceinline__ float get_nc(const T* p, size_t i) { return __half2float(p[i]); }
    static __device__ __forceinline__ void put(T* p, size_t i, float v) { p[i] = __float2half_rn(v); }
    static __device__ __forceinline__ void put_cs(T* p, size_t i, float v) { __stcs(p + i, __float2half_rn(v)); }
};
template <> struct Store<LBM_STORE_BF16DEV> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float get(const T* p, size_t i) { return __bfloat162float(__ldg(p + i)); }
    static __device__ __forceinline__ float get_cs(const T* p, size_t i) { return __bfloat162float(__ldcs(p + i)); }
    static __device__ __forceinline__ float get_nc(const T* p, size_t i) { return __bfloat162float(p[i]); }
    static __device__ __forceinline__ void put(T* p, size_t i, float v) { p[i] = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ void put_cs(T* p, size_t i, float v) { __stcs(p + i, __float2bfloat16_rn(v)); }
};

// ----------------------------------------------------------------- device-side records
struct Sphere {          // FP64 state of one sphere
    double x[3], u[3], w[3];
    double R, rho;
    double F[3], T[3];   // momentum-exchange force and torque of the last step
    double x0[3];        // centre at the start of the step (before the sub-steps)
    double Fl[3];        // lubrication force of the last sub-step
    double hasp;         // 1 once F, T of a previous step exist
    double Fp[3], Tp[3]; // momentum-exchange force and torque of the step before
    double stepped;      // 1 after the first sphere update
    double pad[1];
};
// FP32 copy of what a link needs from its sphere, refreshed after every move: the centre as
// an integer part and a fraction in [0, 1) (cell offsets x - x_P then come out of an exact
// integer difference and one FP32 subtraction), the velocity and angular velocity.  Keeps FP64
// arithmetic, slow on this GPU, out of the per-cell code of the sweep.
struct SphLink {
    int xi[3];
    float xf[3];
    float u[3], w[3];
};
__host__ __device__ inline SphLink sph_link_of(const Sphere& s) {
    SphLink l;
    for (int k = 0; k < 3; k++) {
        const double fl = floor(s.x[k]);
        l.xi[k] = (int)fl;
        l.xf[k] = (float)(s.x[k] - fl);
        l.u[k] = (float)s.u[k];
        l.w[k] = (float)s.w[k];
    }
    return l;
}
// the cells a moved sphere may have covered or uncovered: its box (the union of the old and new
// centres' boxes, a cell of margin), the offsets of the box's first cell from both centres in
// FP32, R^2, and the new centre relative to the old in FP64 for the decisions near the surface
struct TouchBox {
    int lo[3], ext[3];
    float a0[3], a1[3];
    float r2f;
    int go;   // the sphere moved (and its box is sound)
    double off[3];
};
struct SphereAcc {       // per-step momentum-exchange accumulators (zeroed by the sphere update)
    double J[3];         // sum of the deviation part of dj
    double TJ[3];        // sum of (x - x_P) x (deviation part of dj)
    unsigned long long K[3];   // sum of the constant part of dj, times 36 (two's complement)
    unsigned long long XK[3];  // sum of x_img x (constant part), times 36
    double C[3], TC[3];        // force and torque of the links between obstacle nodes of two spheres
};
// one record per bubble id; ids of bubbles that have merged share a root (the smallest id of
// the merged bubble) and hold the merged bubble's V0, V and rho_g
struct Bubble {
    double V0, V, rho_g, Vif;    // reference volume, volume, gas density, interface part of this id's volume
    unsigned long long ngas;     // gas cells carrying this id
    float rho_gf;                // FP32 copy of rho_g for the sweep
    int root;                    // root id (itself until the bubble merges)
    double Vtot[2];              // merged-volume sums at a root, alternating between step closes
    double mg;                   // gas mass rho_g V (conserved; summed when bubbles merge)
    double pad;
};
static_assert(sizeof(Bubble) == 80, "bubble record size");
// distinct pairs of bubbles that may meet in one step (open-addressing table of pairs)
constexpr int kMergeCap = 1024;
// connected parts of bubbles one split step can handle (open-addressing table)
constexpr int kPartCap = 4096;
struct Scalars {
    double pool;          // excess mass waiting to be spread over the interface cells
    double pool_acc;      // excess of this step that found no receiving neighbour
    double S_bb, S_cover, S_uncover;   // mass budget terms
    double share;         // pool / n_iface used by the current sweep
    double mass;          // scratch for the on-demand total-mass reduction
    float share_f;        // FP32 copy of share for the sweep
    float pad0;
    uint32_t n_iface;     // interface cells after the last conversion / covering
    uint32_t n_iface_acc;
    uint32_t status;      // LBM_S_* bits
    uint32_t n_conv, n_newif, n_fromliq, n_touch, n_uncov;
    uint32_t bin_overflow;
    uint32_t n_slow;      // boundary-list length: general cells, at the front of wl_slow
    uint32_t n_liq;       // and liquid cells, at the back
    uint32_t n_rare;      // liquid cells with links into two spheres or into gas (wl_rare)
    uint32_t n_paired;    // spheres with partners this step (sph_list)
    uint32_t n_coupled;   // spheres whose sub-steps feel lubrication this step (sph_cpl)
    uint32_t ticket;      // blocks of the end-of-step scan that have finished
    uint32_t n_fix;       // BULK cells the end of the last step changed or whose neighbours it changed
    uint32_t fix_all;     // the fix list overflowed: the fix pass takes every BULK cell
    uint32_t n_merge;     // distinct pairs of touching bubbles recorded since the last close
    uint32_t merged;      // some bubbles have merged: the close sums volumes per root
    uint32_t vpar;        // which Vtot slot the next close sums into
    uint32_t n_merges;    // merges so far
    uint32_t steps;       // steps closed so far (the split schedule)
    uint32_t n_split;     // parts split off so far
    uint32_t nbub_hw;     // one past the highest bubble id that ever carried cells
    uint32_t split_fail;  // this split step cannot split (part table full, or a find ran too long)
    uint32_t n_split_cells;   // gas and interface cells listed by this split step
    uint32_t obj_on;      // each step adds obj_j . (sum over spheres of F) to obj (lbm_objective)
    double obj_j[3];
    double obj;
};

// status bits (latched; reported through lbm_status and the copy-out calls)
enum : uint32_t { S_UNSTABLE = 1, S_OVERFLOW = 2, S_BUBBLE_GONE = 4, S_BIN_OVERFLOW = 8, S_BAD_OWNER = 16, S_FAST_SPHERE = 32,
                  S_MERGE = 64, S_SPLIT = 128 };

// division of a 32-bit unsigned integer by an invariant divisor d (1 <= d < 2^31) by a
// multiply-high and shifts (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994, the round-up method with the n - t1 correction): exact for every
// 32-bit dividend.  With l = ceil(log2 d): m = floor(2^32 (2^l - d) / d) + 1, s1 = min(l, 1),
// s2 = max(l - 1, 0); n / d = (t + ((n - t) >> s1)) >> s2, t = mulhi(m, n).
struct FastDiv {
    uint32_t m;
    int s1, s2;
};
inline FastDiv make_fastdiv(uint32_t d) {
    int l = 0;
    while ((1ull << l) < d) l++;
    FastDiv f;
    f.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1ull);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l - 1 > 0 ? l - 1 : 0;
    return f;
}
__device__ __forceinline__ uint32_t fast_div(uint32_t n, const FastDiv& f) {
    const uint32_t t = __umulhi(f.m, n);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

// all device pointers of one simulation; passed by value to every kernel
struct Dev {
    int nx, ny, nz;
    int bc[3];                // 1: periodic axis
    uint8_t face[6];          // faces -x, +x, -y, +y, -z, +z of non-periodic axes: FACE_*
    int special;              // some face is free-slip or open
    int split_liq;            // the liquid boundary segment has its own (lean) sweep kernel
    double geo_rmax;          // the largest radius among them
    int ngeo;                 // bubbles given at the start (their geometry); nbub is the table's
                              // size when bubbles split, else ngeo
    int split_every;          // > 0: bubbles split into their connected parts every so many steps
    uint32_t* lab;            // [N] (splitting only) union-find labels of gas / interface cells
    uint32_t* split_list;     // [N] (splitting only) the gas and interface cells of a split step
    uint32_t* part_key;       // [kPartCap] (splitting only) lowest cell index + 1 of each part, 0 free
    uint32_t* part_root;      // [kPartCap] the part's bubble
    double* part_V;           // [kPartCap] the part's volume
    int32_t* part_new;        // [kPartCap] the id the part's cells take, -1: they keep theirs
    uint32_t* bub_cnt;        // [nbub] (splitting only) gas / interface cells per id
    int hydrostatic;          // the liquid starts in hydrostatic equilibrium below the open top
    double gz;                // g_z in FP64 (the hydrostatic start)
    size_t N;                 // cells (< 2^32)
    FastDiv div_nx, div_ny;   // cell index -> coordinates
    int storage;
    int n_sub;
    int sphere_mode;
    int nbub, nsph;
    int max_bub, max_sph;
    int wl_cap;
    float tau, lp, lm;        // tau, lambda_+, lambda_-
    float g[3];
    double gd[3];
    // grid-uniform factors of the collision, from lp, lm and g (set_collision_consts); as kernel
    // arguments they cost the per-cell arithmetic nothing
    struct CollisionConsts {
        float c0;            // 1 + lambda_+ (the rest population)
        float c1, c2;        // 1 + (lambda_+ + lambda_-)/2 and (lambda_+ - lambda_-)/2
        float lp15, cp3;     // 1.5 lambda_+ and 3 (1 + lambda_+/2)
        float lp45;          // 4.5 lambda_+
        float hg[3];         // g / 2
        float K[9], M[9];    // per opposite pair (q = 2k+1, 2k+2): 9 (1 + lambda_+/2) c_q.g, (1 + lambda_-/2) c_q.g
        float cg[9];         // per opposite pair: c_q.g
    } cc;
    float sigma;
    float rho_g0;
    float eps;
    void* f[2];               // PDF grids [19][N]
    uint8_t* flags;           // [N]
    uint8_t* mark;            // [N] conversion marks, zero between steps
    uint8_t* tmark;           // [N] cover / uncover marks (K_TOUCH, K_UNCOV), zero between steps
    float* mass;              // [N]
    float* phi[2];            // [N] fill level, double-buffered with the PDFs
    float* rho[2];            // [N] density of the PDFs in grid g, as the collision (or the
                              // initialisation) that wrote them formed it: the wall density of the
                              // next step's bounce-back links without summing the cell's PDFs
    uint32_t* owner;          // [N] bubble id of gas/interface cells, sphere id of obstacle cells
    float* kappa;             // [N] curvature (sigma > 0 only)
    Bubble* bub;              // [max_bub]
    Sphere* sph;              // [max_sph]
    Sphere* sph_tmp;          // [max_sph] sub-step double buffer
    SphLink* sphl;            // [max_sph] FP32 link data of the current sphere state
    uint32_t* gasflag;        // [2][max_sph] spheres the gas-pressure pass scans, by grid parity
    SphereAcc* acc;           // [max_sph]
    Scalars* sc;
    uint32_t* wl_conv;        // worklists [wl_cap]
    uint32_t* wl_newif;
    uint32_t* wl_fromliq;
    uint32_t* wl_touch;
    uint32_t* wl_slow;        // [N] boundary list: every active cell that is not BULK, in scan order;
                              // liquid cells off the free-slip and open faces from the back
    uint32_t* wl_fix;         // [wl_cap] BULK cells to sweep again after the end-of-step kernels
    uint2* wl_link;           // [N] (many spheres) per liquid-segment entry k: the sphere links of the
                              // cell (bit q: x - c_q is an obstacle cell; bit 31: a link into a second
                              // sphere or a gas cell) and its first sphere; written after the list pass
    uint32_t* wl_rare;        // [wl_cap] the liquid-segment cells with bit 31 (their own sweep)
    // uniform bins of sphere ids for the neighbour searches
    int bin_w, nbx, nby, nbz, bin_cap;
    uint32_t* bin_cnt;        // [nbins]
    uint32_t* bin_ids;        // [nbins][bin_cap]
    uint32_t* npairs;         // [max_sph] partners within lubrication reach this step
    uint32_t* sph_list;       // [max_sph] the spheres with partners this step (n_paired of them)
    uint32_t* sph_cpl;        // [max_sph] the spheres with a partner within lubrication reach (n_coupled)
    uint32_t* sph_near;       // [max_sph][kNearCap] those partners of each listed sphere (sph_nnear of them)
    struct TouchBox* tbox;    // [max_sph] each moved sphere's box for the touch kernel
    int4* sph_bin;            // [max_sph] bin of each sphere's centre (kept with more than 1024 spheres)
    uint32_t* sph_nnear;      // [max_sph]
    uint32_t* pairs;          // [max_sph][kPairCap]
    unsigned long long* merge_keys;   // [kMergeCap] pairs (lo + 1) << 32 | hi of touching roots, 0 = free
    uint32_t* merge_list;     // [kMergeCap] slots of merge_keys in use, in insertion order
};
constexpr int kPairCap = 32;
constexpr int kNearCap = 12;   // partners within lubrication reach (at most 12 equal spheres touch one)
constexpr int kBoundaryGrid = 152 * 2;   // blocks of the general boundary sweep when it runs alone

__device__ __forceinline__ size_t cell_index(const Dev& d, int x, int y, int z) {
    return (size_t)x + (size_t)d.nx * ((size_t)y + (size_t)d.ny * (size_t)z);
}
// coordinates of cell i (N < 2^32: 32-bit division by the grid's invariant extents)
__device__ __forceinline__ void cell_xyz(const Dev& d, size_t i, int& x, int& y, int& z) {
    const uint32_t n = (uint32_t)i;
    const uint32_t r = fast_div(n, d.div_nx);
    x = (int)(n - r * (uint32_t)d.nx);
    const uint32_t q = fast_div(r, d.div_ny);
    y = (int)(r - q * (uint32_t)d.ny);
    z = (int)q;
}
// neighbour index of (x,y,z)+(dx,dy,dz); periodic axes wrap; beyond a wall: returns false
__device__ __forceinline__ bool nbr(const Dev& d, int x, int y, int z, int dx, int dy, int dz, size_t& j) {
    int a = x + dx, b = y + dy, c = z + dz;
    if (a < 0 || a >= d.nx) { if (!d.bc[0]) return false; a = a < 0 ? a + d.nx : a - d.nx; }
    if (b < 0 || b >= d.ny) { if (!d.bc[1]) return false; b = b < 0 ? b + d.ny : b - d.ny; }
    if (c < 0 || c >= d.nz) { if (!d.bc[2]) return false; c = c < 0 ? c + d.nz : c - d.nz; }
    j = cell_index(d, a, b, c);
    return true;
}

// the cell (x, y, z) touches a free-slip or open face
__device__ __forceinline__ bool at_special_face(const Dev& d, int x, int y, int z) {
    if (!d.special) return false;
    const int c[3] = {x, y, z}, L[3] = {d.nx, d.ny, d.nz};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        if (d.bc[k]) continue;
        if (c[k] == 0 && d.face[2 * k] != FACE_WALL) return true;
        if (c[k] == L[k] - 1 && d.face[2 * k + 1] != FACE_WALL) return true;
    }
    return false;
}

// the boundary list in one [N] buffer: the general cells (interface cells and cells on a
// free-slip or open face) from the front, slots [0, n_slow), and the other liquid cells from
// the back, slot N - 1 - k for the k-th (they never overlap: together they are at most N cells)
__device__ __forceinline__ uint32_t blist_len(const Dev& d, uint32_t& ngen) {
    ngen = min(*(volatile const uint32_t*)&d.sc->n_slow, (uint32_t)d.N);
    const uint32_t nliq = min(*(volatile const uint32_t*)&d.sc->n_liq, (uint32_t)d.N - ngen);
    return ngen + nliq;
}
__device__ __forceinline__ uint32_t blist_cell(const Dev& d, uint32_t k, uint32_t ngen) {
    return k < ngen ? d.wl_slow[k] : d.wl_slow[(uint32_t)d.N - 1u - (k - ngen)];
}

// BULK: a liquid cell each of whose 18 neighbours is liquid or interface or lies beyond a
// no-slip wall; the bulk sweep streams it without looking at its neighbours
__device__ __forceinline__ bool bulk_of(const Dev& d, size_t i) {
    if ((d.flags[i] & F_TYPE) != F_LIQ) return false;
    int x, y, z;
    cell_xyz(d, i, x, y, z);
    if (at_special_face(d, x, y, z)) return false;
    uint32_t ok = F_ACTIVE;   // all 18 neighbour loads are independent
#pragma unroll
    for (int q = 1; q < kQ; q++) {
        size_t j;
        if (nbr(d, x, y, z, cx(q), cy(q), cz(q), j)) ok &= (d.flags[j] & F_ACTIVE) ? F_ACTIVE : 0u;
    }
    return ok != 0;
}
// image (per periodic axis, the one nearest to the sphere centre) of cell c and its offset
// c_img - x_P, from the sphere's link data
__device__ __forceinline__ void sph_offset(const Dev& d, const SphLink& l, const int (&c)[3], int (&img)[3],
                                           float (&r)[3]) {
    const int L[3] = {d.nx, d.ny, d.nz};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        int xi = c[k];
        if (d.bc[k]) {
            const float dd = (float)(l.xi[k] - xi) + l.xf[k];   // x_P - c
            if (dd > 0.5f * (float)L[k]) xi += L[k];
            else if (dd < -0.5f * (float)L[k]) xi -= L[k];
        }
        img[k] = xi;
        r[k] = (float)(xi - l.xi[k]) - l.xf[k];
    }
}

// barrier of all threads of the thread-block cluster, ordering their global-memory writes
// before the reads that follow (release / acquire at cluster scope); a hardware barrier, not a
// spin on memory
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
struct ClusterSync {
    __device__ void operator()() const { cluster_sync(); }
};
struct BlockSync {
    __device__ void operator()() const { __syncthreads(); }
};

// two adjacent cells i, j of two bubbles' gas / interface regions: the bubbles touch and are one
// connected gas region from now on (Sec. 2.2: a bubble is a connected gas region).  The pair of
// roots is recorded once per step (the table is probed from a hash of the pair); the step's
// close joins them.  Roots change only at a close, so they are stable here.
__device__ __forceinline__ void merge_check(const Dev& d, size_t i, size_t j) {
    if (!(d.flags[i] & (F_IF | F_GAS)) || !(d.flags[j] & (F_IF | F_GAS))) return;
    const uint32_t a = d.owner[i], b = d.owner[j];
    if (a >= (uint32_t)d.nbub || b >= (uint32_t)d.nbub || a == b) return;
    const uint32_t ra = (uint32_t)d.bub[a].root, rb = (uint32_t)d.bub[b].root;
    if (ra == rb) return;
    const uint32_t lo = min(ra, rb), hi = max(ra, rb);
    const unsigned long long key = ((unsigned long long)(lo + 1u) << 32) | hi;
    uint32_t h = (lo * 0x9E3779B1u ^ hi * 0x85EBCA77u) & (kMergeCap - 1);
    for (int k = 0; k < kMergeCap; k++, h = (h + 1) & (kMergeCap - 1)) {
        const unsigned long long old = atomicCAS(&d.merge_keys[h], 0ull, key);
        if (old == key) return;   // recorded already
        if (old == 0ull) {
            d.merge_list[atomicAdd(&d.sc->n_merge, 1u)] = h;   // at most kMergeCap insertions
            return;
        }
    }
    atomicOr(&d.sc->status, S_MERGE);   // more distinct pairs in one step than the table holds
}

// byte-wise atomic OR / AND on the mark array (4-byte aligned base); returns the old byte
__device__ __forceinline__ uint8_t mark_or(uint8_t* base, size_t i, uint8_t bits) {
    uint32_t* w = reinterpret_cast<uint32_t*>(base + (i & ~(size_t)3));
    const uint32_t sh = (uint32_t)(i & 3) * 8u;
    const uint32_t old = atomicOr(w, (uint32_t)bits << sh);
    return (uint8_t)(old >> sh);
}
__device__ __forceinline__ uint8_t mark_and(uint8_t* base, size_t i, uint8_t bits) {
    uint32_t* w = reinterpret_cast<uint32_t*>(base + (i & ~(size_t)3));
    const uint32_t sh = (uint32_t)(i & 3) * 8u;
    const uint32_t old = atomicAnd(w, ~((uint32_t)bits << sh));
    return (uint8_t)(old >> sh);
}

// BULK bit of cell i from its neighbourhood, set at initialisation
__device__ __forceinline__ void set_bulk_init(const Dev& d, size_t i) {
    const uint8_t t = d.flags[i] & F_TYPE;
    d.flags[i] = (uint8_t)(t | (bulk_of(d, i) ? F_BULK : 0));
}

// BULK bit of cell i from its neighbourhood; the end-of-step kernels call it for every cell
// whose type or PDFs they changed and for those cells' neighbours.  Only that bit changes, by
// an atomic byte AND / OR (other threads update other bytes of the word, or this one).
// The next step's bulk sweep may already be running on the types and PDFs it read before:
// every cell that comes out BULK goes to the fix list, whose cells the sweep takes again once
// these kernels are done.
__device__ __forceinline__ void set_bulk(const Dev& d, size_t i) {
    const bool b = bulk_of(d, i);
    if (b) mark_or(d.flags, i, F_BULK);
    else mark_and(d.flags, i, F_BULK);
    if (b) {
        const unsigned act = __activemask();
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(act) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(&d.sc->n_fix, (uint32_t)__popc(act));
        base = __shfl_sync(act, base, leader);
        const uint32_t slot = base + (uint32_t)__popc(act & ((1u << lane) - 1u));
        if (slot < (uint32_t)d.wl_cap) d.wl_fix[slot] = (uint32_t)i;
        else d.sc->fix_all = 1u;   // no fatal overflow: the fix pass then takes every BULK cell
    }
}

// bubble b's volume bookkeeping when a cell changes: dv to the interface part, dg gas cells,
// di interface cells (any sign)
__device__ __forceinline__ void vol_change(const Dev& d, uint32_t b, double dv, int dg, int di) {
    if (b < (uint32_t)d.nbub) {
        if (dv != 0.0) atomicAdd(&d.bub[b].Vif, dv);
        if (dg) atomicAdd(&d.bub[b].ngas, (unsigned long long)(long long)dg);
    }
    if (di) atomicAdd(&d.sc->n_iface_acc, (uint32_t)di);
}

// full-warp reductions (every lane gets the result)
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ uint32_t warp_min(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// global warp index and warp count of a 1-D launch
__device__ __forceinline__ uint32_t warp_id() { return (blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ uint32_t warp_count() { return (gridDim.x * blockDim.x) >> 5; }

// append to a worklist with warp aggregation; false if the list is full
__device__ __forceinline__ bool wl_push(uint32_t* list, uint32_t* count, uint32_t cap, uint32_t v, uint32_t* status) {
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(act) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(act));
    base = __shfl_sync(act, base, leader);
    const uint32_t slot = base + (uint32_t)__popc(act & ((1u << lane) - 1u));
    if (slot < cap) { list[slot] = v; return true; }
    atomicOr(status, S_OVERFLOW);
    return false;
}

// post-collision moments of cell i from grid f (deviations): rho = 1 + sum d*,
// u = (sum c d* - rho g/2)/rho
// density and velocity of cell i's post-collision PDFs; gw weights the body force the
// collision applied (the cell's fill level for an interface cell, 1 for a liquid cell): the
// velocity the collision used is (sum c f* - rho gw g / 2) / rho
template <int S>
__device__ __forceinline__ void post_moments(const Dev& d, const typename Store<S>::T* f, size_t i, float gw, float& rho, float u[3]) {
    float dr = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int q = 0; q < kQ; q++) {
        const float v = Store<S>::get_nc(f, (size_t)q * d.N + i);
        dr += v;
        jx = cacc(cx(q), jx, v); jy = cacc(cy(q), jy, v); jz = cacc(cz(q), jz, v);
    }
    const float r = 1.f + dr;
    rho = r;
    u[0] = (jx - 0.5f * r * gw * d.g[0]) / r;
    u[1] = (jy - 0.5f * r * gw * d.g[1]) / r;
    u[2] = (jz - 0.5f * r * gw * d.g[2]) / r;
}

// deviation of the equilibrium (Eq. equilibrium) from the weight: e_q(rho,u) - w_q
__device__ __forceinline__ float equilibrium_dev(int q, float rho, const float u[3]) {
    const float cu = cdot(q, u[0], u[1], u[2]);
    const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return wgt(q) * ((rho - 1.f) + rho * (3.f * cu + 4.5f * cu * cu - 1.5f * uu));
}

// the collision's grid-uniform factors (Dev::cc) from d.lp, d.lm and d.g; called wherever those change
inline void set_collision_consts(Dev& d) {
    const double lp = d.lp, lm = d.lm, cp = 1.0 + 0.5 * lp, cm = 1.0 + 0.5 * lm;
    Dev::CollisionConsts& k = d.cc;
    k.c0 = (float)(1.0 + lp);
    k.c1 = (float)(1.0 + 0.5 * (lp + lm));
    k.c2 = (float)(0.5 * (lp - lm));
    k.lp15 = (float)(1.5 * lp);
    k.cp3 = (float)(3.0 * cp);
    k.lp45 = (float)(4.5 * lp);
    for (int a = 0; a < 3; a++) k.hg[a] = (float)(0.5 * (double)d.g[a]);
    for (int p = 0; p < 9; p++) {
        const int q = 2 * p + 1;
        const double cg = cx(q) * (double)d.g[0] + cy(q) * (double)d.g[1] + cz(q) * (double)d.g[2];
        k.K[p] = (float)(9.0 * cp * cg);
        k.M[p] = (float)(cm * cg);
        k.cg[p] = (float)cg;
    }
}

// moments, Guo-shifted velocity and the TRT collision of one cell, all on deviations f - w:
// the post-collision deviations out[].  The body force acts on the cell's liquid mass: rho g in
// a liquid cell, gw = its fill level times that in an interface cell.
// Per opposite pair (q, qb) the relaxation of the symmetric part towards e+ and of the
// antisymmetric part towards e-, with Guo's source split the same way, is gathered as
//   out_q  = c1 f_q + c2 f_qb + alpha + beta,   out_qb = c1 f_qb + c2 f_q + alpha - beta,
//   alpha = w (-lambda_+ drho + rho (1.5 lambda_+ u.u - 3 c+ u.G)) + w rho cu (9 c+ cg - 4.5 lambda_+ cu),
//   beta  = 3 w rho (c- cg - lambda_- cu),
// cu = c_q.u, cg = c_q.G, G = gw g, c+- = 1 + lambda_+-/2, c1 = 1 + (lambda_+ + lambda_-)/2,
// c2 = (lambda_+ - lambda_-)/2: the same collision as f + lambda_+ (f+ - e+) + lambda_- (f- - e-)
// + c+ G+ + c- G- written out per pair, with the grid-uniform factors computed on the host.
__device__ __forceinline__ float trt_collide(const Dev& d, const float (&fin)[kQ], float gw, float (&out)[kQ]) {
    const Dev::CollisionConsts& k = d.cc;
    float drho = 0.f, jx = 0.f, jy = 0.f, jz = 0.f;
#pragma unroll
    for (int q = 0; q < kQ; q++) {
        drho += fin[q];
        jx = cacc(cx(q), jx, fin[q]); jy = cacc(cy(q), jy, fin[q]); jz = cacc(cz(q), jz, fin[q]);
    }
    const float rho = 1.f + drho;
    if (!(rho > 0.f)) atomicOr(&d.sc->status, S_UNSTABLE);
    const float inv = 1.f / rho;
    const float ux = fmaf(jx, inv, gw * k.hg[0]);   // (j + rho G/2) / rho
    const float uy = fmaf(jy, inv, gw * k.hg[1]);
    const float uz = fmaf(jz, inv, gw * k.hg[2]);
    const float usq = ux * ux + uy * uy + uz * uz;
    const float ug = gw * (ux * d.g[0] + uy * d.g[1] + uz * d.g[2]);
    // the part common to every direction of one weight, over that weight
    const float inner = fmaf(-d.lp, drho, rho * (k.lp15 * usq - k.cp3 * ug));
    out[0] = fmaf(k.c0, fin[0], wgt(0) * inner);
    const float af = wgt(1) * inner, ae = wgt(7) * inner;
    const float wrf = wgt(1) * rho, wre = wgt(7) * rho;
    const float wrf3 = 3.f * wrf, wre3 = 3.f * wre;
#pragma unroll
    for (int p = 0; p < 9; p++) {
        const int q = 2 * p + 1, qb = q + 1;
        const bool face = q <= 6;
        const float cu = cdot(q, ux, uy, uz);
        const float al = fmaf((face ? wrf : wre) * cu, fmaf(-k.lp45, cu, gw * k.K[p]), face ? af : ae);
        const float be = (face ? wrf3 : wre3) * fmaf(-d.lm, cu, gw * k.M[p]);
        out[q] = fmaf(k.c1, fin[q], fmaf(k.c2, fin[qb], al + be));
        out[qb] = fmaf(k.c1, fin[qb], fmaf(k.c2, fin[q], al - be));
    }
    return rho;
}

// the collision of one cell, its post-collision deviations stored to grid fb (CS: streaming
// stores) and, with rhob, its density to rhob[i]
template <int S, bool CS = false>
__device__ __forceinline__ void collide_store(const Dev& d, typename Store<S>::T* __restrict__ fb, size_t i, const float (&fin)[kQ],
                                              float gw = 1.f, float* __restrict__ rhob = nullptr) {
    float out[kQ];
    const float rho = trt_collide(d, fin, gw, out);
#pragma unroll
    for (int q = 0; q < kQ; q++) (CS ? Store<S>::put_cs : Store<S>::put)(fb, (size_t)q * d.N + i, out[q]);
    if (rhob) {
        if (CS) __stcs(rhob + i, rho);
        else rhob[i] = rho;
    }
}

// minimum-image difference a - b along axis k (beyond 4 periods, or not finite, the value is
// first reduced with fmod, so no loop runs more than a few times)
__device__ __forceinline__ double min_image(const Dev& d, int k, double a, double b) {
    double v = a - b;
    if (d.bc[k]) {
        const double L = (double)(k == 0 ? d.nx : (k == 1 ? d.ny : d.nz));
        if (!(fabs(v) <= 4.0 * L)) v = fmod(v, L);
        for (int it = 0; it < 8 && v > 0.5 * L; it++) v -= L;
        for (int it = 0; it < 8 && v < -0.5 * L; it++) v += L;
    }
    return v;
}
// periodic position into [-1/2, L - 1/2)
__device__ __forceinline__ double wrap_pos(double x, int L) {
    if (!(fabs(x) <= 4.0 * L)) x = fmod(x, (double)L);
    for (int it = 0; it < 8 && x >= L - 0.5; it++) x -= L;
    for (int it = 0; it < 8 && x < -0.5; it++) x += L;
    return x;
}
__device__ __forceinline__ bool finite3(const double* v) {
    return isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]);
}


// ------------------------------------------------------------ uniform bins of spheres
// bin width >= 2 R_max + 2; the last bin of an axis absorbs the remainder, so every bin is
// at least bin_w wide and a sphere within bin_w of a point lies in the 27 bins around it
__device__ __forceinline__ int bin_coord(const Dev& d, int k, double v) {
    const int n = k == 0 ? d.nbx : (k == 1 ? d.nby : d.nbz);
    int b = (int)floor(v / (double)d.bin_w);
    return b < 0 ? 0 : (b > n - 1 ? n - 1 : b);
}
__device__ __forceinline__ size_t bin_index(const Dev& d, int bx, int by, int bz) {
    return ((size_t)bz * d.nby + by) * d.nbx + bx;
}
// the (at most 3) distinct bin coordinates around b along axis k; returns their count
__device__ __forceinline__ int bin_span(const Dev& d, int k, int b, int out[3]) {
    const int n = k == 0 ? d.nbx : (k == 1 ? d.nby : d.nbz);
    if (n <= 3) { for (int a = 0; a < n; a++) out[a] = a; return n; }
    int c = 0;
    for (int o = -1; o <= 1; o++) {
        int v = b + o;
        if (v < 0 || v >= n) { if (!d.bc[k]) continue; v = v < 0 ? v + n : v - n; }
        out[c++] = v;
    }
    return c;
}
__device__ __forceinline__ bool sphere_covers(const Dev& d, const Sphere& s, int x, int y, int z) {
    const double ddx = min_image(d, 0, (double)x, s.x[0]);
    const double ddy = min_image(d, 1, (double)y, s.x[1]);
    const double ddz = min_image(d, 2, (double)z, s.x[2]);
    return ddx * ddx + ddy * ddy + ddz * ddz <= s.R * s.R;
}
// lowest id of the spheres whose current centre covers cell (x,y,z), or kNone
__device__ __forceinline__ uint32_t covering_sphere(const Dev& d, int x, int y, int z) {
    int sx[3], sy[3], sz[3];
    const int nx_ = bin_span(d, 0, bin_coord(d, 0, (double)x), sx);
    const int ny_ = bin_span(d, 1, bin_coord(d, 1, (double)y), sy);
    const int nz_ = bin_span(d, 2, bin_coord(d, 2, (double)z), sz);
    uint32_t best = kNone;
    for (int c = 0; c < nz_; c++)
        for (int b = 0; b < ny_; b++)
            for (int a = 0; a < nx_; a++) {
                const size_t bi = bin_index(d, sx[a], sy[b], sz[c]);
                uint32_t cnt = d.bin_cnt[bi];
                if (cnt > (uint32_t)d.bin_cap) cnt = (uint32_t)d.bin_cap;
                for (uint32_t e = 0; e < cnt; e++) {
                    const uint32_t P = d.bin_ids[bi * d.bin_cap + e];
                    if (P < best && sphere_covers(d, d.sph[P], x, y, z)) best = P;
                }
            }
    return best;
}

// kernels (defined in the .cu files), launched by lbm_capi.cu
// The bubble model and the bookkeeping that close a step (Sec. 2.2): V_b = gas cells of b +
// sum over b's interface cells of (1 - phi), kept up to date by the sweep (the interface part,
// afresh) and the end-of-step kernels (every change of type or fill level), then
// rho_g,b = rho_g0 V_b(0) / V_b (isothermal gas of conserved mass); the excess pool and the
// share the next sweep spreads over the interface cells; the per-step counters and the
// boundary list are reset;
// moved spheres enter the bins of their new centres.  Run by every thread (t of nt) of the
// step's last kernel, after its last barrier.
// joins the recorded pairs of touching roots (one thread): the larger root joins the smaller
// and passes on its reference volume and gas mass (they add); then every id
// points at its root directly (roots are never larger than the ids below them, so one pass in
// increasing id order suffices)
__device__ inline void merge_apply(const Dev& d, const uint32_t n) {
    Bubble* B = d.bub;
    auto find = [&](int b) { while (B[b].root != b) b = B[b].root; return b; };   // roots: this thread's writes
    for (uint32_t k = 0; k < min(n, (uint32_t)kMergeCap); k++) {
        const uint32_t h = __ldcg(&d.merge_list[k]);
        const unsigned long long key = __ldcg(&d.merge_keys[h]);
        d.merge_keys[h] = 0ull;
        const int ra = find((int)(key >> 32) - 1), rb = find((int)(key & 0xffffffffu));
        if (ra == rb) continue;
        const int lo = min(ra, rb), hi = max(ra, rb);
        B[hi].root = lo;
        B[lo].V0 = __ldcg(&B[lo].V0) + __ldcg(&B[hi].V0);
        B[lo].mg = __ldcg(&B[lo].mg) + __ldcg(&B[hi].mg);
        d.sc->n_merges++;
    }
    for (int b = 0; b < d.nbub; b++) B[b].root = B[B[b].root].root;
    d.sc->n_merge = 0;
    d.sc->merged = 1;
}

// the bubble model at the end of a step (Sec. 2.2): V of each bubble = its gas cells + the
// interface part the sweep summed (both kept per id), rho_g = m_g / V, the gas mass m_g
// conserved (isothermal ideal gas); with init, V0 = V and m_g = rho_g V from the initial gas
// density in rho_g.  Threads t of nt; sync() is a barrier over all of them.  Until
// the first merge every id is its own bubble and no barrier is needed.
template <class Sync>
__device__ inline void bubbles_close(const Dev& d, const uint32_t t, const uint32_t nt, const bool init, Sync sync) {
    Scalars& c = *d.sc;
    // written only by merge_check before the caller's last barrier and by this close's thread 0
    // after the barriers below: every thread reads the same values here
    const uint32_t nm = *(volatile uint32_t*)&c.n_merge;
    if (nm == 0u && *(volatile uint32_t*)&c.merged == 0u) {
        for (uint32_t b = t; b < (uint32_t)d.nbub; b += nt) {
            Bubble& B = d.bub[b];
            const double V = (double)(long long)__ldcg(&B.ngas) + __ldcg(&B.Vif);
            B.V = V;
            if (init) { B.V0 = V; B.mg = B.rho_g * V; }
            else if (V > 0.0) B.rho_g = B.mg / V;
            else if (B.mg > 0.0) atomicOr(&c.status, S_BUBBLE_GONE);   // (a free row holds no gas)
            B.rho_gf = (float)B.rho_g;
            B.Vif = 0.0;
        }
        return;
    }
    const uint32_t par = *(volatile uint32_t*)&c.vpar;
    for (uint32_t b = t; b < (uint32_t)d.nbub; b += nt) {
        Bubble& B = d.bub[b];
        B.V = (double)(long long)__ldcg(&B.ngas) + __ldcg(&B.Vif);   // this id's part
        B.Vif = 0.0;
        if (init) { B.V0 = B.V; B.mg = B.rho_g * B.V; }
        B.Vtot[par ^ 1u] = 0.0;   // read by the last close; summed into by the next
    }
    sync();
    if (t == 0 && nm != 0u) merge_apply(d, nm);
    sync();
    // every thread handles the same ids in every loop: B.V below is its own write
    for (uint32_t b = t; b < (uint32_t)d.nbub; b += nt) atomicAdd(&d.bub[__ldcg(&d.bub[b].root)].Vtot[par], d.bub[b].V);
    sync();
    for (uint32_t b = t; b < (uint32_t)d.nbub; b += nt) {
        Bubble& B = d.bub[b];
        const Bubble& R = d.bub[__ldcg(&B.root)];
        const double V = __ldcg(&R.Vtot[par]);
        B.V = V;
        B.V0 = __ldcg(&R.V0);
        B.mg = __ldcg(&R.mg);
        if (V > 0.0) B.rho_g = B.mg / V;
        else if (B.mg > 0.0) atomicOr(&c.status, S_BUBBLE_GONE);
        B.rho_gf = (float)B.rho_g;
    }
    if (t == 0) c.vpar = par ^ 1u;
}

// the end of a step: bubble model, excess pool and counters, new sphere bins.  Every thread of
// the launch (nt of them) calls it; sync() is a barrier over all of them.
template <class Sync>
__device__ inline void step_close(const Dev& d, const uint32_t t, const uint32_t nt, const bool bin_spheres, Sync sync) {
    bubbles_close(d, t, nt, false, sync);
    if (t == 0) {
        Scalars& c = *d.sc;
        if (c.share != 0.0) c.pool = 0.0;
        c.pool += c.pool_acc;
        c.pool_acc = 0.0;
        c.n_iface = c.n_iface_acc;
        c.n_iface_acc = 0;
        c.share = (c.pool != 0.0 && c.n_iface > 0) ? c.pool / (double)c.n_iface : 0.0;
        c.share_f = (float)c.share;
        c.n_conv = c.n_newif = c.n_fromliq = c.n_touch = c.n_uncov = 0;
        c.n_slow = 0;   // the boundary sweep has consumed its list; the list pass refills it
        c.n_liq = 0;
        c.n_rare = 0;
        c.n_paired = 0;
        c.steps++;
    }
    if (bin_spheres)
        for (uint32_t P = t; P < (uint32_t)d.nsph; P += nt) {
            const Sphere& sp = d.sph[P];
            // (with more than 1024 spheres the touch preparation has found the bins)
            const int4 bb = d.nsph > 1024 ? d.sph_bin[P]
                                          : make_int4(bin_coord(d, 0, sp.x[0]), bin_coord(d, 1, sp.x[1]), bin_coord(d, 2, sp.x[2]), 0);
            const size_t bi = bin_index(d, bb.x, bb.y, bb.z);
            const uint32_t slot = atomicAdd(&d.bin_cnt[bi], 1u);
            if (slot < (uint32_t)d.bin_cap) d.bin_ids[bi * d.bin_cap + slot] = P;
            else atomicOr(&d.sc->status, S_BIN_OVERFLOW);
        }
}

// the bulk sweep of grid cur; `whole`: every warp that holds a BULK cell writes all the cells
// it spans (only where the fix pass and the boundary sweep run after it)
void launch_sweep_bulk(const Dev& d, int cur, cudaStream_t s, bool whole);
void launch_sweep_rest(const Dev& d, int cur, cudaStream_t s, cudaStream_t side, cudaStream_t side2, cudaEvent_t fork,
                       cudaEvent_t join, cudaEvent_t join2);

void launch_conversions(const Dev& d, int nxt, bool close, cudaStream_t s);
void launch_split(const Dev& d, int g, cudaStream_t s);
constexpr int kSplitLaunches = 6;
void launch_init_scan(const Dev& d, cudaStream_t s);
void launch_list_rescan(const Dev& d, cudaStream_t s);
void launch_link_classify(const Dev& d, cudaStream_t s);
void launch_curvature(const Dev& d, int nxt, cudaStream_t s);
void launch_spheres_links(const Dev& d, int g, cudaStream_t s);
void launch_spheres_move(const Dev& d, cudaStream_t s);
void launch_spheres_cover(const Dev& d, int nxt, cudaStream_t s);
void prepare_sphere_kernels();

void launch_bins_insert(const Dev& d, cudaStream_t s);
int spheres_launches(const Dev& d);
int spheres_links_launches(const Dev& d);
void launch_init(const Dev& d, const double* bub_geom_dev, cudaStream_t s);
// rho[g] = 1 + the sum of grid g's PDFs (deviations) of every active cell (after the PDFs of grid
// g were written from outside the sweep)
void launch_rho_of_grid(const Dev& d, int g, cudaStream_t s);
void launch_bulk_all(const Dev& d, cudaStream_t s);
void launch_fields(const Dev& d, int cur, float* rho, float* u, float* phi, uint8_t* flags, cudaStream_t s);
void launch_export(const Dev& d, int cur, float* f, uint8_t* flags, float* m, float* phi, int32_t* owner, float* kappa, cudaStream_t s);
void launch_mass(const Dev& d, int cur, cudaStream_t s);
void launch_frozen_forward(const Dev& d, const float* f_in, float* f_out, cudaStream_t s, cudaStream_t side,
                           cudaEvent_t fork, cudaEvent_t join);

constexpr int kAdjSlots = 512;   // FP64 slots of the adjoint's parameter sums (block id mod slots)
void launch_adjoint(const Dev& d, const float* f_fwd, const float* lam_in, float* lam_out, float* srho,
                    const float jdir[3], double* part, bool moving_walls, cudaStream_t s, cudaStream_t side,
                    cudaEvent_t fork, cudaEvent_t join);

}  // namespace lbm
