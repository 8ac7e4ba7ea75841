// lbm_sweep.cu -- the fused per-step sweep over all cells (one thread per cell).
//
// For every active (liquid or interface) cell x, in one pass over the two PDF grids:
//   pull streaming f_q(x,t+1) = f*_q(x - c_q, t)                         (Sec. 2.1, Eq. LBE1)
//   halfway bounce-back where x - c_q lies beyond a no-slip wall
//   moving-wall bounce-back where x - c_q is an obstacle cell of sphere P (Sec. 2.3, Eq. bbrule):
//       f_q(x,t+1) = f*_q^(x,t) + 6 w_q rho_w c_q.u_w,  u_w = u_P + w_P x (x_w - x_P),
//       x_w = x - c_q/2 the link midpoint, rho_w = sum f*(x,t) the previous-step density,
//     with the momentum exchange dj = c_q^ f*_q^(x,t) - c_q f_q(x,t+1) summed into the
//     force and torque of P (Eqs. netforce, torque, momentum_transfer)
//   free-surface reconstruction where x - c_q is a gas cell of bubble b (Sec. 2.2, Eq. fsk):
//       f_q(x,t+1) = -f*_q^(x,t) + 2 e+_q(rho_w, u_w),  rho_w = rho_g,b + 6 sigma kappa(x),
//       u_w = the velocity of x from its own post-collision state
//   mass exchange of interface cells (Eqs. massExchange, massExchangeb):
//       m(t+1) = m(t) + sum_q s_q (f*_q^(x+c_q,t) - f*_q(x,t)),  s = 1 (liquid neighbour),
//       (phi(x)+phi(x+c_q))/2 (interface neighbour), 0 otherwise;  phi(t+1) = m(t+1)/rho(t+1)
//   TRT collision with lambda_+ = -1/tau, (1/lambda_+ + 1/2)(1/lambda_- + 1/2) = 3/16
//   (Eq. LBE2 and the magic relation of Sec. 2.1) and a Guo body force split into its even
//   and odd parts; u = (sum c f + rho g/2)/rho
//   and the conversion candidates: phi >= 1 + eps (filled) / phi <= -eps (emptied).
//
// The bulk kernel streams and collides every liquid cell whose 18 neighbours are liquid,
// interface or beyond a wall (wall links read the cell's own opposite PDF by an index select),
// with few registers and no branches per link: it is bound by HBM bandwidth, and runs beside
// the previous step's end-of-step kernels.  Every other active cell is on a compact list built
// at the end of the previous step (general and liquid segments), which the boundary kernel
// processes with the full link logic once those kernels are done, beside the fix pass (and,
// for long lists, a lean instance on the liquid segment; streams forked and joined by events,
// captured into the step's CUDA graph): it is bound by memory latency and instruction issue.
//
// Sphere force and torque are reduced in FP64 without cancellation loss: per link the
// momentum is split into the constant part -2 w_q c_q (accumulated exactly as integers,
// times 36) and the small deviation part (FP32 per cell, summed over the warp's lanes of the
// same sphere, then one FP64 atomic per warp and sphere).
#include "lbm_internal.cuh"

namespace lbm {

struct SphAcc {
    uint32_t pid;
    float J[3];
    int K[3];
    float r[3];     // x_img - x_P of this cell
    int xi[3];      // x_img
    float u[3], w[3];   // the sphere's velocity and angular velocity, converted once per cell
};

__device__ __forceinline__ void sph_begin(const Dev& d, SphAcc& a, uint32_t P, int x, int y, int z) {
    a.pid = P;
    a.J[0] = a.J[1] = a.J[2] = 0.f;
    a.K[0] = a.K[1] = a.K[2] = 0;
    const SphLink l = d.sphl[P];
    const int c[3] = {x, y, z};
    sph_offset(d, l, c, a.xi, a.r);
#pragma unroll
    for (int k = 0; k < 3; k++) {
        a.u[k] = l.u[k];
        a.w[k] = l.w[k];
    }
}

// cell's partial sums -> global accumulators of the sphere (used when one cell touches two
// spheres; the common case is reduced over the warp instead)
__device__ __forceinline__ void sph_flush_direct(const Dev& d, const SphAcc& a) {
    if (a.pid == kNone) return;
    SphereAcc& g = d.acc[a.pid];
    const float TJ[3] = {a.r[1] * a.J[2] - a.r[2] * a.J[1], a.r[2] * a.J[0] - a.r[0] * a.J[2], a.r[0] * a.J[1] - a.r[1] * a.J[0]};
    const int XK[3] = {a.xi[1] * a.K[2] - a.xi[2] * a.K[1], a.xi[2] * a.K[0] - a.xi[0] * a.K[2], a.xi[0] * a.K[1] - a.xi[1] * a.K[0]};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        atomicAdd(&g.J[k], (double)a.J[k]);
        atomicAdd(&g.TJ[k], (double)TJ[k]);
        atomicAdd(&g.K[k], (unsigned long long)(long long)a.K[k]);
        atomicAdd(&g.XK[k], (unsigned long long)(long long)XK[k]);
    }
}


// A block's sphere sums of one round of the shell kernels, gathered in shared memory: a table of
// kAccSlots slots keyed by sphere id (slot = id mod kAccSlots), FP32 and integer sums added with
// shared-memory atomics; a cell whose slot another sphere holds adds straight to the global
// accumulators.  In scan order the 32 cells of a warp lie around a dozen or more spheres (a row
// crosses one after another), so a reduction over the warp would take that many rounds; the
// block's 128 cells (four rows or so) meet about as many spheres, each several times.
constexpr int kAccSlots = 64;
struct AccTable {
    uint32_t key[kAccSlots];
    float v[kAccSlots][6];   // J, (x - x_P) x J
    int iv[kAccSlots][6];    // K, x_img x K (integer parts)
};
__device__ __forceinline__ void acc_table_clear(AccTable& t) {
    for (int s = threadIdx.x; s < kAccSlots; s += blockDim.x) {
        t.key[s] = kNone;
#pragma unroll
        for (int c = 0; c < 6; c++) { t.v[s][c] = 0.f; t.iv[s][c] = 0; }
    }
}
__device__ __forceinline__ void acc_table_add(const Dev& d, const SphAcc& acc, AccTable& t) {
    if (acc.pid == kNone) return;
    const float v[6] = {acc.J[0], acc.J[1], acc.J[2], acc.r[1] * acc.J[2] - acc.r[2] * acc.J[1],
                        acc.r[2] * acc.J[0] - acc.r[0] * acc.J[2], acc.r[0] * acc.J[1] - acc.r[1] * acc.J[0]};
    const int iv[6] = {acc.K[0], acc.K[1], acc.K[2], acc.xi[1] * acc.K[2] - acc.xi[2] * acc.K[1],
                       acc.xi[2] * acc.K[0] - acc.xi[0] * acc.K[2], acc.xi[0] * acc.K[1] - acc.xi[1] * acc.K[0]};
    const int s = (int)(acc.pid & (uint32_t)(kAccSlots - 1));
    const uint32_t k = atomicCAS(&t.key[s], kNone, acc.pid);
    if (k == kNone || k == acc.pid) {
#pragma unroll
        for (int c = 0; c < 6; c++) {
            atomicAdd(&t.v[s][c], v[c]);
            atomicAdd(&t.iv[s][c], iv[c]);
        }
    } else {
        SphereAcc& g = d.acc[acc.pid];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            atomicAdd(&g.J[c], (double)v[c]);
            atomicAdd(&g.TJ[c], (double)v[3 + c]);
            atomicAdd(&g.K[c], (unsigned long long)(long long)iv[c]);
            atomicAdd(&g.XK[c], (unsigned long long)(long long)iv[3 + c]);
        }
    }
}
// (after a block barrier) the table's sums to the global accumulators, the table cleared
__device__ __forceinline__ void acc_table_flush(const Dev& d, AccTable& t) {
    for (int s = threadIdx.x; s < kAccSlots; s += blockDim.x) {
        const uint32_t P = t.key[s];
        if (P == kNone) continue;
        SphereAcc& g = d.acc[P];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            if (t.v[s][c] != 0.f) atomicAdd(&g.J[c], (double)t.v[s][c]);
            if (t.v[s][3 + c] != 0.f) atomicAdd(&g.TJ[c], (double)t.v[s][3 + c]);
            if (t.iv[s][c] != 0) atomicAdd(&g.K[c], (unsigned long long)(long long)t.iv[s][c]);
            if (t.iv[s][3 + c] != 0) atomicAdd(&g.XK[c], (unsigned long long)(long long)t.iv[s][3 + c]);
            t.v[s][c] = t.v[s][3 + c] = 0.f;
            t.iv[s][c] = t.iv[s][3 + c] = 0;
        }
        t.key[s] = kNone;
    }
}

// the lanes' sphere accumulators summed over the warp, sphere by sphere, then one FP64 atomic per
// warp and sphere (every lane of the warp takes part)
__device__ __forceinline__ void sph_acc_warp_reduce(const Dev& d, const SphAcc& acc) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float TJ[3] = {0.f, 0.f, 0.f};
    int XK[3] = {0, 0, 0};
    if (acc.pid != kNone) {
        TJ[0] = acc.r[1] * acc.J[2] - acc.r[2] * acc.J[1];
        TJ[1] = acc.r[2] * acc.J[0] - acc.r[0] * acc.J[2];
        TJ[2] = acc.r[0] * acc.J[1] - acc.r[1] * acc.J[0];
        XK[0] = acc.xi[1] * acc.K[2] - acc.xi[2] * acc.K[1];
        XK[1] = acc.xi[2] * acc.K[0] - acc.xi[0] * acc.K[2];
        XK[2] = acc.xi[0] * acc.K[1] - acc.xi[1] * acc.K[0];
    }
    unsigned todo = __ballot_sync(full, acc.pid != kNone);
    while (todo) {
        const int leader = __ffs(todo) - 1;
        const uint32_t P = __shfl_sync(full, acc.pid, leader);
        const bool mine = acc.pid == P;
        todo &= ~__ballot_sync(full, mine);
        float v[6];
        int iv[6];
#pragma unroll
        for (int c = 0; c < 3; c++) {
            v[c] = mine ? acc.J[c] : 0.f;
            v[3 + c] = mine ? TJ[c] : 0.f;
            // the integer parts: one hardware warp reduction each
            iv[c] = __reduce_add_sync(full, mine ? acc.K[c] : 0);
            iv[3 + c] = __reduce_add_sync(full, mine ? XK[c] : 0);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int c = 0; c < 6; c++) v[c] += __shfl_xor_sync(full, v[c], o);
        }
        if (lane == leader) {
            SphereAcc& g = d.acc[P];
#pragma unroll
            for (int c = 0; c < 3; c++) {
                atomicAdd(&g.J[c], (double)v[c]);
                atomicAdd(&g.TJ[c], (double)v[3 + c]);
                atomicAdd(&g.K[c], (unsigned long long)(long long)iv[c]);
                atomicAdd(&g.XK[c], (unsigned long long)(long long)iv[3 + c]);
            }
        }
    }
}

// one link of cell (x, y, z) into an obstacle cell of sphere P that is not the cell's first
// sphere (a cell between two spheres): Eq. bbrule and the link's momentum exchange, summed
// straight into P's accumulators.  Returns the bounce-back correction (f_q(x, t+1) is
// fob + the correction).  Out of line: it is rare.
__device__ __noinline__ float sph_link_other(const Dev& d, int q, uint32_t P, int x, int y, int z, float rho0, float fob) {
    SphAcc a;
    sph_begin(d, a, P, x, y, z);
    const int c[3] = {cx(q), cy(q), cz(q)};
    const float wq = q <= 6 ? (1.0f / 18.0f) : (1.0f / 36.0f);
    const int w72q = q <= 6 ? 4 : 2;
    // c_q . u_w at the link midpoint x - c_q/2 equals c_q . (u_P + w_P x r): c_q . (w x c_q) = 0
    const float ucx = a.u[0] + a.w[1] * a.r[2] - a.w[2] * a.r[1];
    const float ucy = a.u[1] + a.w[2] * a.r[0] - a.w[0] * a.r[2];
    const float ucz = a.u[2] + a.w[0] * a.r[1] - a.w[1] * a.r[0];
    const float corr = 6.f * wq * rho0 * (c[0] * ucx + c[1] * ucy + c[2] * ucz);
    const float dev = 2.f * fob + corr;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        a.J[k] = -c[k] * dev;
        a.K[k] = -w72q * c[k];
    }
    sph_flush_direct(d, a);
    return corr;
}

// a link of cell (x, y, z) whose source x - c_q lies beyond a face of a non-periodic axis,
// not every crossed face being a no-slip wall (Fig. bubbleSetup):
//   - an open face (the top): Eq. fsk with the reference pressure, f_q = -f*_qb + 2 e+_q(1, u),
//     u the cell's own velocity; the mass let in, f_q - f*_qb, is a boundary source (and goes
//     to an interface cell's mass);
//   - free-slip faces only (and periodic axes): specular reflection, the population of the
//     mirrored direction (normal components reversed) from the source moved back across each
//     free-slip face, x' = x - c_q + (its normal components); x' is then an ordinary source:
//     streaming with mass exchange, a sphere's moving wall, or a gas cell (Eq. fsk).
// A no-slip face among those crossed gives halfway bounce-back.  Out of line: face cells are
// few, and only free-slip or open faces get here.
template <int S>
__device__ __noinline__ float face_link(const Dev& d, const typename Store<S>::T* __restrict__ fa, const float* __restrict__ phia,
                                        int cur, int q, int x, int y, int z, float fob, float rho0, float u0x, float u0y,
                                        float u0z, float phix, float kap, bool isIF, bool liq, float& dm, float& sbb) {
    const int c[3] = {cx(q), cy(q), cz(q)};
    const int L[3] = {d.nx, d.ny, d.nz};
    int s[3] = {x - c[0], y - c[1], z - c[2]};
    int m[3] = {c[0], c[1], c[2]};   // velocity of the population that comes back as q
    bool wall = false, open = false;
    for (int k = 0; k < 3; k++) {
        if (s[k] >= 0 && s[k] < L[k]) continue;
        if (d.bc[k]) { s[k] += s[k] < 0 ? L[k] : -L[k]; continue; }
        const uint8_t f = d.face[2 * k + (s[k] >= L[k] ? 1 : 0)];
        if (f == FACE_WALL) wall = true;
        else if (f == FACE_OPEN) open = true;
        else { s[k] += c[k]; m[k] = -c[k]; }
    }
    if (wall) return fob;
    const float u0sq = u0x * u0x + u0y * u0y + u0z * u0z;
    const float cu = c[0] * u0x + c[1] * u0y + c[2] * u0z;
    const float wq = wgt(q);
    if (open) {
        const float fi = 2.f * wq * (4.5f * cu * cu - 1.5f * u0sq) - fob;
        if (isIF) dm += fi - fob;
        sbb += fi - fob;
        return fi;
    }
    const size_t j = cell_index(d, s[0], s[1], s[2]);
    const uint8_t t = d.flags[j];
    if (t & F_ACTIVE) {
        int qm = q;
        for (int p = 1; p < kQ; p++)
            if (cx(p) == m[0] && cy(p) == m[1] && cz(p) == m[2]) qm = p;
        const float fi = Store<S>::get(fa, (size_t)qm * d.N + j);
        if (isIF) {
            const float sw = (t & F_LIQ) ? 1.f : 0.5f * (phix + phia[j]);
            dm += sw * (fi - fob);
        }
        return fi;
    }
    if (t & F_OBS) {
        const uint32_t P = d.owner[j];
        if (P >= (uint32_t)d.nsph) return fob;
        if (isIF) d.gasflag[(size_t)cur * d.max_sph + P] = 1u;
        const float corr = sph_link_other(d, q, P, x, y, z, rho0, fob);
        if (liq) sbb += corr;
        return fob + corr;
    }
    const uint32_t b = d.owner[j];
    const float rg = b < (uint32_t)d.nbub ? d.bub[b].rho_gf : d.rho_g0;
    const float rw = rg + 6.f * d.sigma * kap;
    return 2.f * wq * ((rw - 1.f) + rw * (4.5f * cu * cu - 1.5f * u0sq)) - fob;
}

// the pulled PDFs fin of one BULK cell (x, y, z) = i: every neighbour carries PDFs or lies
// beyond a wall (halfway bounce-back by index select), no neighbour tests.  CS: streaming
// (evict-first) loads.
template <int S, bool CS>
__device__ __forceinline__ void bulk_load(const Dev& d, const typename Store<S>::T* __restrict__ fa, int x, int y, int z,
                                          uint32_t i, float (&fin)[kQ]) {
    using T = typename Store<S>::T;
    const uint32_t nx = (uint32_t)d.nx, nxy = (uint32_t)d.nx * (uint32_t)d.ny;
    if ((x & ~31) > 0 && (x | 31) < d.nx - 1 && y > 0 && y < d.ny - 1 && z > 0 && z < d.nz - 1) {
        // every neighbour inside the grid: the source of direction q is i - c_q . (1, nx, nx ny).
        // Tested on the 32-aligned run of x around x, the warp of the bulk sweep, so that a
        // warp takes one of the two branches (any x in that run is at least 1 and below nx - 1)
#pragma unroll
        for (int q = 0; q < kQ; q++) {
            const int32_t o = cx(q) + cy(q) * (int32_t)nx + cz(q) * (int32_t)nxy;
            const T* plane = fa + (size_t)q * d.N;
            fin[q] = CS ? Store<S>::get_cs(plane, i - (uint32_t)o) : Store<S>::get(plane, i - (uint32_t)o);
        }
        return;
    }
    if (y > 0 && y < d.ny - 1 && z > 0 && z < d.nz - 1) {
        // y and z neighbours inside the grid (the same for a whole warp, which spans x): the
        // source of direction q is i - c_q . (1, nx, nx ny), a grid-uniform offset, except
        // across the x edges (periodic wrap, or bounce-back from a wall)
        const bool edge0 = x == 0, edge1 = x == d.nx - 1;
        const bool perx = d.bc[0] != 0;
#pragma unroll
        for (int q = 0; q < kQ; q++) {
            const int32_t o = cx(q) + cy(q) * (int32_t)nx + cz(q) * (int32_t)nxy;
            bool wall = false;
            int32_t adj = 0;
            if (cx(q) == 1 && edge0) { if (perx) adj = (int32_t)nx; else wall = true; }
            if (cx(q) == -1 && edge1) { if (perx) adj = -(int32_t)nx; else wall = true; }
            const T* plane = fa + (size_t)(wall ? opp(q) : q) * d.N;
            const uint32_t src = wall ? i : i - (uint32_t)o + (uint32_t)adj;   // modulo 2^32
            fin[q] = CS ? Store<S>::get_cs(plane, src) : Store<S>::get(plane, src);
        }
        return;
    }
    const uint32_t xm = x == 0 ? nx - 1 : x - 1, xp = x == d.nx - 1 ? 0 : x + 1;
    const uint32_t ym = (y == 0 ? d.ny - 1 : y - 1) * nx, yp = (y == d.ny - 1 ? 0 : y + 1) * nx, y0 = y * nx;
    const uint32_t zm = (z == 0 ? d.nz - 1 : z - 1) * nxy, zp = (z == d.nz - 1 ? 0 : z + 1) * nxy, z0 = z * nxy;
    const bool wxm = !d.bc[0] && x == 0, wxp = !d.bc[0] && x == d.nx - 1;
    const bool wym = !d.bc[1] && y == 0, wyp = !d.bc[1] && y == d.ny - 1;
    const bool wzm = !d.bc[2] && z == 0, wzp = !d.bc[2] && z == d.nz - 1;
#pragma unroll
    for (int q = 0; q < kQ; q++) {
        const uint32_t sx = cx(q) == 1 ? xm : (cx(q) == -1 ? xp : (uint32_t)x);
        const uint32_t sy = cy(q) == 1 ? ym : (cy(q) == -1 ? yp : y0);
        const uint32_t sz = cz(q) == 1 ? zm : (cz(q) == -1 ? zp : z0);
        const bool wall = (cx(q) == 1 && wxm) || (cx(q) == -1 && wxp) || (cy(q) == 1 && wym) ||
                          (cy(q) == -1 && wyp) || (cz(q) == 1 && wzm) || (cz(q) == -1 && wzp);
        // halfway bounce-back: the cell's own post-collision PDF of the opposite direction
        const T* plane = fa + (size_t)(wall ? opp(q) : q) * d.N;
        const uint32_t src = wall ? i : sx + sy + sz;
        fin[q] = CS ? Store<S>::get_cs(plane, src) : Store<S>::get(plane, src);
    }
}

// pull-stream and collide one BULK cell (x, y, z) = i
template <int S>
__device__ __forceinline__ void bulk_cell(const Dev& d, const typename Store<S>::T* __restrict__ fa,
                                          typename Store<S>::T* __restrict__ fb, int x, int y, int z, uint32_t i,
                                          float* __restrict__ rhob) {
    float fin[kQ];
    bulk_load<S, true>(d, fa, x, y, z, i, fin);
    collide_store<S, true>(d, fb, i, fin, 1.f, rhob);
}

// every liquid cell whose neighbours all carry PDFs or lie beyond a wall; other active cells
// go to the boundary list.  It may run while the end-of-step kernels of the last step are
// still changing types and PDFs near interfaces and spheres: the cells it then reads stale
// inputs for are on the fix list (or leave BULK and go to the boundary list), and the fix pass
// and the boundary sweep, which run after those kernels, overwrite their results.
// With Whole (the forward step, whose fix pass and boundary sweep follow it on the stream), a
// warp that holds a BULK cell writes every cell it spans, so that each 32-byte sector of the
// destination is written whole: a sector written in part costs the memory a read of the
// sector before the write, and in a sphere-dense column most sectors hold a cell beside a
// sphere (16 cells a sector at two bytes a PDF).  The warp's other active cells get a
// provisional update that the fix pass or the boundary sweep replaces; its gas and obstacle
// cells, whose PDFs nothing reads, get the update of a resting population.  Without Whole
// (the adjoint's frozen step, whose boundary kernel runs at the same time) only BULK cells
// are written.
template <int S, bool Whole>
__global__ void __launch_bounds__(128) sweep_bulk_kernel(const Dev d, const int cur) {
    using T = typename Store<S>::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const bool in = x < d.nx && y < d.ny;
    const uint32_t i = (uint32_t)x + (uint32_t)d.nx * (uint32_t)y + (uint32_t)d.nx * (uint32_t)d.ny * (uint32_t)z;
    const uint8_t fl = in ? d.flags[i] : (uint8_t)0;
    const bool bulk = (fl & F_ACTIVE) && (fl & F_BULK);
    const T* __restrict__ fa = static_cast<const T*>(d.f[cur]);
    T* __restrict__ fb = static_cast<T*>(d.f[cur ^ 1]);
    if (!Whole) {   // (the densities are the forward step's: not written)
        if (bulk) bulk_cell<S>(d, fa, fb, x, y, z, i, nullptr);
        return;
    }
    // (all 32 lanes reach the vote: blocks are whole warps and nothing returned before it)
    if (!__any_sync(0xffffffffu, bulk) || !in) return;
    float fin[kQ];
    if (fl & F_ACTIVE) {
        bulk_load<S, true>(d, fa, x, y, z, i, fin);
    } else {
#pragma unroll
        for (int q = 0; q < kQ; q++) fin[q] = 0.f;
    }
    collide_store<S, true>(d, fb, i, fin, 1.f, d.rho[cur ^ 1]);
}

// the fix pass: the listed BULK cells again (or every BULK cell when the list overflowed),
// with the types and PDFs the end-of-step kernels left
template <int S>
__global__ void __launch_bounds__(128) sweep_fix_kernel(const Dev d, const int cur) {
    using T = typename Store<S>::T;
    const T* __restrict__ fa = static_cast<const T*>(d.f[cur]);
    T* __restrict__ fb = static_cast<T*>(d.f[cur ^ 1]);
    const bool all = *(volatile const uint32_t*)&d.sc->fix_all != 0u;
    const uint32_t n = all ? (uint32_t)d.N : min(*(volatile const uint32_t*)&d.sc->n_fix, (uint32_t)d.wl_cap);
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint32_t i = all ? k : d.wl_fix[k];
        const uint8_t fl = d.flags[i];
        if (!(fl & F_LIQ) || !(fl & F_BULK)) continue;
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        bulk_cell<S>(d, fa, fb, x, y, z, i, d.rho[cur ^ 1]);
    }
}

// one active cell that is not BULK: walls, sphere links, gas links, interface mass exchange,
// and the collision (the general instance); with Lean a liquid cell whose links are streaming,
// wall and sphere links (and gas links, should a gas cell sit beside one): no mass exchange,
// no face links.  Sphere sums go to acc, the liquid cells' bounce-back mass to sbb; an
// interface cell reports its bubble (vb) and new fill level (vphi).
template <int S, bool Lean>
__device__ __forceinline__ void boundary_cell(const Dev& d, const typename Store<S>::T* __restrict__ fa,
                                              typename Store<S>::T* __restrict__ fb, const float* __restrict__ phia,
                                              float* __restrict__ phib, const int cur, const size_t i, SphAcc& acc,
                                              float& sbb, uint32_t& vb, float& vphi, bool& isIFc) {
    const size_t N = d.N;
    const float gx = d.g[0], gy = d.g[1], gz = d.g[2];
    const uint8_t fl = d.flags[i];
    int x, y, z;
    cell_xyz(d, i, x, y, z);
    const bool isIF = !Lean && (fl & F_IF) != 0;
    const bool liqc = Lean || (fl & F_LIQ) != 0;
    isIFc = isIF;
    // every load is issued before any link is resolved: neighbour indices and types,
    // then the pulled PDFs, owners and fill levels (predicated on the types)
    float fo[kQ];
    uint32_t src[kQ];
    uint32_t fsv[kQ];   // neighbour type, 0xff beyond a wall
#pragma unroll
    for (int q = 0; q < kQ; q++) fo[q] = Store<S>::get(fa, (size_t)q * N + i);
    {   // neighbour indices with periodic wrap; sources beyond a wall flagged 0xff
        const uint32_t nx = (uint32_t)d.nx, nxy = (uint32_t)d.nx * (uint32_t)d.ny;
        const uint32_t xm = x == 0 ? nx - 1 : x - 1, xp = x == d.nx - 1 ? 0 : x + 1;
        const uint32_t ym = (y == 0 ? d.ny - 1 : y - 1) * nx, yp = (y == d.ny - 1 ? 0 : y + 1) * nx, y0 = y * nx;
        const uint32_t zm = (z == 0 ? d.nz - 1 : z - 1) * nxy, zp = (z == d.nz - 1 ? 0 : z + 1) * nxy, z0 = z * nxy;
        const bool wxm = !d.bc[0] && x == 0, wxp = !d.bc[0] && x == d.nx - 1;
        const bool wym = !d.bc[1] && y == 0, wyp = !d.bc[1] && y == d.ny - 1;
        const bool wzm = !d.bc[2] && z == 0, wzp = !d.bc[2] && z == d.nz - 1;
#pragma unroll
        for (int q = 1; q < kQ; q++) {
            const uint32_t sx = cx(q) == 1 ? xm : (cx(q) == -1 ? xp : (uint32_t)x);
            const uint32_t sy = cy(q) == 1 ? ym : (cy(q) == -1 ? yp : y0);
            const uint32_t sz = cz(q) == 1 ? zm : (cz(q) == -1 ? zp : z0);
            const bool wall = (cx(q) == 1 && wxm) || (cx(q) == -1 && wxp) || (cy(q) == 1 && wym) ||
                              (cy(q) == -1 && wyp) || (cz(q) == 1 && wzm) || (cz(q) == -1 && wzp);
            src[q] = wall ? (uint32_t)i : sx + sy + sz;
            fsv[q] = wall ? 0xffu : (uint32_t)d.flags[sx + sy + sz];
        }
    }
    float fv[kQ];       // pulled PDF (active source) or the source's owner (bit pattern)
    float phn[kQ];      // fill level of an interface source (interface cells only)
#pragma unroll
    for (int q = 1; q < kQ; q++) {
        const uint32_t t = fsv[q];
        fv[q] = 0.f;
        phn[q] = 0.f;
        if (t != 0xffu) {
            if (t & F_ACTIVE) fv[q] = Store<S>::get(fa, (size_t)q * N + src[q]);
            else fv[q] = __uint_as_float(d.owner[src[q]]);
            if (isIF && (t & F_IF)) phn[q] = phia[src[q]];
        }
    }
    float drho0 = 0.f, j0x = 0.f, j0y = 0.f, j0z = 0.f;
#pragma unroll
    for (int q = 0; q < kQ; q++) {
        drho0 += fo[q];
        j0x = cacc(cx(q), j0x, fo[q]); j0y = cacc(cy(q), j0y, fo[q]); j0z = cacc(cz(q), j0z, fo[q]);
    }
    const float rho0 = 1.f + drho0;
    // the force the last collision applied: on the liquid mass, phi g in an interface cell
    const float gw0 = isIF ? phia[i] : 1.f;
    const float u0x = (j0x - 0.5f * rho0 * gw0 * gx) / rho0;
    const float u0y = (j0y - 0.5f * rho0 * gw0 * gy) / rho0;
    const float u0z = (j0z - 0.5f * rho0 * gw0 * gz) / rho0;
    const float u0sq = u0x * u0x + u0y * u0y + u0z * u0z;
    const float phix = isIF ? phia[i] : 0.f;
    const float kap = (isIF && d.kappa) ? d.kappa[i] : 0.f;
    const bool atface = !Lean && at_special_face(d, x, y, z);
    // the cell's sphere: the owner of its first obstacle link (links into a second
    // sphere take sph_link_other); the wall velocity is needed only as c_q . u_w, and
    // c_q . u_w at the link midpoint x - c_q/2 equals c_q . (u_P + w_P x r), r = x - x_P
    // (c_q . (w_P x c_q) = 0): one cell-centre velocity serves every link
    uint32_t P0 = kNone;
#pragma unroll
    for (int q = kQ - 1; q >= 1; q--)
        if (fsv[q] != 0xffu && (fsv[q] & F_OBS)) P0 = __float_as_uint(fv[q]);
    float ucx = 0.f, ucy = 0.f, ucz = 0.f;
    if (P0 < (uint32_t)d.nsph) {
        sph_begin(d, acc, P0, x, y, z);
        ucx = acc.u[0] + acc.w[1] * acc.r[2] - acc.w[2] * acc.r[1];
        ucy = acc.u[1] + acc.w[2] * acc.r[0] - acc.w[0] * acc.r[2];
        ucz = acc.u[2] + acc.w[0] * acc.r[1] - acc.w[1] * acc.r[0];
    }
    float fin[kQ];
    float dm = 0.f;
    fin[0] = fo[0];
#pragma unroll
    for (int q = 1; q < kQ; q++) {
        const int qb = opp(q);
        const uint32_t t = fsv[q];
        if (t == 0xffu) {
            if (atface)
                fin[q] = face_link<S>(d, fa, phia, cur, q, x, y, z, fo[qb], rho0, u0x, u0y, u0z, phix, kap, isIF,
                                      liqc, dm, sbb);
            else
                fin[q] = fo[qb];                                // no-slip wall
        } else if (t & F_ACTIVE) {
            fin[q] = fv[q];                                     // Eq. LBE1
            if (isIF) {  // link to the neighbour x + c_qb: s (f*_q(x+c_qb) - f*_qb(x))
                const float sw = (t & F_LIQ) ? 1.f : 0.5f * (phix + phn[q]);
                dm += sw * (fin[q] - fo[qb]);
            }
        } else if (t & F_OBS) {                                 // Eq. bbrule
            const uint32_t P = __float_as_uint(fv[q]);
            // a sphere beside an interface cell: the next gas-pressure pass scans it
            if (isIF && P < (uint32_t)d.nsph) d.gasflag[(size_t)cur * d.max_sph + P] = 1u;
            if (P == P0) {
                const float corr = 6.f * wgt(q) * rho0 * cdot(q, ucx, ucy, ucz);
                fin[q] = fo[qb] + corr;
                // dj = -c_q (f*_qb + f_q(t+1)) = -c_q (2 w_q) - c_q (2 (f*_qb - w_q) + corr)
                const float dev = 2.f * fo[qb] + corr;
                acc.J[0] = cacc(-cx(q), acc.J[0], dev); acc.J[1] = cacc(-cy(q), acc.J[1], dev); acc.J[2] = cacc(-cz(q), acc.J[2], dev);
                acc.K[0] -= w72(q) * cx(q); acc.K[1] -= w72(q) * cy(q); acc.K[2] -= w72(q) * cz(q);
                if (liqc) sbb += corr;
            } else if (P < (uint32_t)d.nsph) {
                const float corr = sph_link_other(d, q, P, x, y, z, rho0, fo[qb]);
                fin[q] = fo[qb] + corr;
                if (liqc) sbb += corr;
            } else {
                fin[q] = fo[qb];
            }
        } else {                                                // gas: Eq. fsk
            const uint32_t bb = __float_as_uint(fv[q]);
            const float rg = bb < (uint32_t)d.nbub ? d.bub[bb].rho_gf : d.rho_g0;
            const float rw = rg + 6.f * d.sigma * kap;
            const float cu = cdot(q, u0x, u0y, u0z);
            // -f*_qb + 2 e+_q, in deviations: 2 (e+_q - w_q) - (f*_qb - w_q)
            fin[q] = 2.f * wgt(q) * ((rw - 1.f) + rw * (4.5f * cu * cu - 1.5f * u0sq)) - fo[qb];
        }
    }
    float gw = 1.f;   // the body force acts on the liquid mass: phi g in an interface cell
    if (isIF) {
        const float mnew = (d.mass[i] + d.sc->share_f) + dm;
        float drho = 0.f;
#pragma unroll
        for (int q = 0; q < kQ; q++) drho += fin[q];
        const float rho = 1.f + drho;
        d.mass[i] = mnew;
        phib[i] = mnew / rho;
        vb = d.owner[i];
        vphi = mnew / rho;
        gw = vphi;
        // an interface cell is a boundary cell of the liquid with a gas neighbour
        // (Sec. 2.2): one left without any gas neighbour is liquid now (filled).
        // phi >= 1 + eps  <=>  m - rho >= eps rho, taken as (m - 1) - drho so that a
        // density deviation below FP32's resolution of 1 still decides it;
        // phi <= -eps  <=>  m <= -eps rho
        bool gasnb = false;
#pragma unroll
        for (int q = 1; q < kQ; q++) gasnb |= fsv[q] != 0xffu && (fsv[q] & F_GAS);
        uint8_t mk = 0;
        if (!gasnb) mk = K_FILLED;
        else if ((mnew - 1.f) - drho >= d.eps * rho) mk = K_FILLED;
        else if (mnew <= -d.eps * rho) mk = K_EMPTIED;
        if (mk) {
            d.mark[i] = mk;
            wl_push(d.wl_conv, &d.sc->n_conv, (uint32_t)d.wl_cap, (uint32_t)i, &d.sc->status);
        }
    }
    collide_store<S>(d, fb, i, fin, gw, d.rho[cur ^ 1]);
}

// ------------------------------------------------ link words of the liquid segment
// The liquid segment's cells (in practice the spheres' shells) are classified once the list
// pass is done, while the next bulk sweep runs: per entry k, bit q of the word says that the
// link source x - c_q is an obstacle cell, bit 31 that the cell has a link into a second sphere,
// into an obstacle cell of no valid sphere or into a gas cell (it then takes the full path), and
// the second word holds the cell's first sphere (the owner of its lowest-q obstacle link).  The
// lean kernel then needs neither the neighbours' types nor their owners.
constexpr uint32_t kLinkRare = 1u << 31;
__global__ void __launch_bounds__(256) link_classify_kernel(const Dev d) {
    const uint32_t N = (uint32_t)d.N;
    const uint32_t n = min(*(volatile const uint32_t*)&d.sc->n_liq, N);
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint32_t i = d.wl_slow[N - 1u - k];
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        const uint32_t nx = (uint32_t)d.nx, nxy = (uint32_t)d.nx * (uint32_t)d.ny;
        const uint32_t xm = x == 0 ? nx - 1 : x - 1, xp = x == d.nx - 1 ? 0 : x + 1;
        const uint32_t ym = (y == 0 ? d.ny - 1 : y - 1) * nx, yp = (y == d.ny - 1 ? 0 : y + 1) * nx, y0 = y * nx;
        const uint32_t zm = (z == 0 ? d.nz - 1 : z - 1) * nxy, zp = (z == d.nz - 1 ? 0 : z + 1) * nxy, z0 = z * nxy;
        const bool wxm = !d.bc[0] && x == 0, wxp = !d.bc[0] && x == d.nx - 1;
        const bool wym = !d.bc[1] && y == 0, wyp = !d.bc[1] && y == d.ny - 1;
        const bool wzm = !d.bc[2] && z == 0, wzp = !d.bc[2] && z == d.nz - 1;
        uint8_t t[kQ];
        uint32_t src[kQ];
#pragma unroll
        for (int q = 1; q < kQ; q++) {   // every type load first
            const uint32_t sx = cx(q) == 1 ? xm : (cx(q) == -1 ? xp : (uint32_t)x);
            const uint32_t sy = cy(q) == 1 ? ym : (cy(q) == -1 ? yp : y0);
            const uint32_t sz = cz(q) == 1 ? zm : (cz(q) == -1 ? zp : z0);
            const bool wall = (cx(q) == 1 && wxm) || (cx(q) == -1 && wxp) || (cy(q) == 1 && wym) ||
                              (cy(q) == -1 && wyp) || (cz(q) == 1 && wzm) || (cz(q) == -1 && wzp);
            src[q] = sx + sy + sz;
            t[q] = wall ? (uint8_t)F_ACTIVE : d.flags[src[q]];   // (a wall link streams from the cell itself)
        }
        uint32_t mask = 0u, P0 = kNone, first = kNone;
        bool rare = false;
#pragma unroll
        for (int q = kQ - 1; q >= 1; q--) {
            if (t[q] & F_ACTIVE) continue;
            if (t[q] & F_OBS) {
                const uint32_t P = d.owner[src[q]];
                mask |= 1u << q;
                P0 = P;
                if (first == kNone) first = P;
                else if (P != first) rare = true;
                if (P >= (uint32_t)d.nsph) rare = true;
            } else {
                rare = true;   // a gas link
            }
        }
        d.wl_link[k] = make_uint2(mask | (rare ? kLinkRare : 0u), P0);
        if (rare) wl_push(d.wl_rare, &d.sc->n_rare, (uint32_t)d.wl_cap, i, &d.sc->status);
    }
}

// (two blocks per SM: it runs beside the bulk sweep at high priority, and a grid that filled every
// SM's warp slots would hold them from the bulk sweep's blocks for its whole duration; a single
// block per SM leaves it too slow for the chain of end-of-step kernels it ends)
void launch_link_classify(const Dev& d, cudaStream_t s) { link_classify_kernel<<<152 * 2, 256, 0, s>>>(d); }

// a liquid-segment cell whose obstacle links all go into its first sphere P0 (mask: bit q set
// for a link from an obstacle cell), the others streaming or beyond a no-slip wall: the lean
// instance of boundary_cell without any neighbour type or owner load, the same arithmetic.  One
// load per direction: the pulled PDF of a streaming link, the cell's own opposite PDF of a wall
// or sphere link (bounce-back); the wall density (the cell's density of the last step) is the one
// the collision that wrote the cell's PDFs stored in rhoa, not a sum of its 19 PDFs.
template <int S>
__device__ __forceinline__ void lean_cell(const Dev& d, const typename Store<S>::T* __restrict__ fa,
                                          typename Store<S>::T* __restrict__ fb, const float* __restrict__ rhoa,
                                          float* __restrict__ rhob, const size_t i, const uint32_t mask,
                                          const uint32_t P0, SphAcc& acc, float& sbb) {
    const size_t N = d.N;
    int x, y, z;
    cell_xyz(d, i, x, y, z);
    const uint32_t nx = (uint32_t)d.nx, nxy = (uint32_t)d.nx * (uint32_t)d.ny;
    const uint32_t xm = x == 0 ? nx - 1 : x - 1, xp = x == d.nx - 1 ? 0 : x + 1;
    const uint32_t ym = (y == 0 ? d.ny - 1 : y - 1) * nx, yp = (y == d.ny - 1 ? 0 : y + 1) * nx, y0 = y * nx;
    const uint32_t zm = (z == 0 ? d.nz - 1 : z - 1) * nxy, zp = (z == d.nz - 1 ? 0 : z + 1) * nxy, z0 = z * nxy;
    const bool wxm = !d.bc[0] && x == 0, wxp = !d.bc[0] && x == d.nx - 1;
    const bool wym = !d.bc[1] && y == 0, wyp = !d.bc[1] && y == d.ny - 1;
    const bool wzm = !d.bc[2] && z == 0, wzp = !d.bc[2] && z == d.nz - 1;
    float fin[kQ];
    uint32_t wl = 0u;   // bit q: the link comes from beyond a wall
    fin[0] = Store<S>::get(fa, i);
#pragma unroll
    for (int q = 1; q < kQ; q++) {
        const uint32_t sx = cx(q) == 1 ? xm : (cx(q) == -1 ? xp : (uint32_t)x);
        const uint32_t sy = cy(q) == 1 ? ym : (cy(q) == -1 ? yp : y0);
        const uint32_t sz = cz(q) == 1 ? zm : (cz(q) == -1 ? zp : z0);
        const bool wall = (cx(q) == 1 && wxm) || (cx(q) == -1 && wxp) || (cy(q) == 1 && wym) ||
                          (cy(q) == -1 && wyp) || (cz(q) == 1 && wzm) || (cz(q) == -1 && wzp);
        wl |= wall ? 1u << q : 0u;
        const bool bb = wall || (mask & (1u << q)) != 0u;   // bounce-back: the cell's own f*_qb
        fin[q] = Store<S>::get(fa, (size_t)(bb ? opp(q) : q) * N + (bb ? (uint32_t)i : sx + sy + sz));
    }
    float ucx = 0.f, ucy = 0.f, ucz = 0.f, rho0 = 1.f;
    if (mask) {
        rho0 = rhoa[i];
        // c_q . u_w at the link midpoint equals c_q . (u_P + w_P x r) at the cell centre
        sph_begin(d, acc, P0, x, y, z);
        ucx = acc.u[0] + acc.w[1] * acc.r[2] - acc.w[2] * acc.r[1];
        ucy = acc.u[1] + acc.w[2] * acc.r[0] - acc.w[0] * acc.r[2];
        ucz = acc.u[2] + acc.w[0] * acc.r[1] - acc.w[1] * acc.r[0];
    }
#pragma unroll
    for (int q = 1; q < kQ; q++) {
        if (!(wl & (1u << q)) && (mask & (1u << q))) {              // Eq. bbrule
            const float fob = fin[q];                                // f*_qb of the cell
            const float corr = 6.f * wgt(q) * rho0 * cdot(q, ucx, ucy, ucz);
            fin[q] = fob + corr;
            // dj = -c_q (f*_qb + f_q(t+1)) = -c_q (2 w_q) - c_q (2 (f*_qb - w_q) + corr)
            const float dev = 2.f * fob + corr;
            acc.J[0] = cacc(-cx(q), acc.J[0], dev); acc.J[1] = cacc(-cy(q), acc.J[1], dev); acc.J[2] = cacc(-cz(q), acc.J[2], dev);
            acc.K[0] -= w72(q) * cx(q); acc.K[1] -= w72(q) * cy(q); acc.K[2] -= w72(q) * cz(q);
            sbb += corr;
        }
    }
    collide_store<S>(d, fb, i, fin, 1.f, rhob);
}

// every other active cell: walls, sphere links, gas links, interface mass exchange.  Two
// instances: the general one takes the general segment of the list (interface cells and cells
// on a free-slip or open face); the lean one (Lean) the liquid segment, cells whose links are
// streaming, wall and sphere links only (and gas links, should a gas cell sit beside one): no
// mass exchange, no face links; 128 registers a thread against 200, twice the resident warps.
// Mode: kBndGeneral (the general segment, or both), kBndLean (the liquid segment, full link
// logic), kBndLeanFast (the liquid segment's classified cells with links into one sphere
// only), kBndRare (the classified cells with links into two spheres or into gas)
enum { kBndGeneral = 0, kBndLean = 1, kBndLeanFast = 2, kBndRare = 3 };
template <int S, int Mode>
__global__ void __launch_bounds__(128, Mode == kBndLeanFast ? 6 : (Mode != kBndGeneral ? 4 : 1)) sweep_boundary_kernel(const Dev d, const int cur) {
    constexpr bool Lean = Mode != kBndGeneral;
    using T = typename Store<S>::T;
    const T* __restrict__ fa = static_cast<const T*>(d.f[cur]);
    T* __restrict__ fb = static_cast<T*>(d.f[cur ^ 1]);
    const float* __restrict__ phia = d.phi[cur];
    float* __restrict__ phib = d.phi[cur ^ 1];
    const size_t N = d.N;
    // the general kernel takes both segments when no lean kernel runs
    uint32_t ngen = 0, n;
    if (Mode == kBndRare) n = min(*(volatile const uint32_t*)&d.sc->n_rare, (uint32_t)d.wl_cap);
    else if (Lean) n = min(*(volatile const uint32_t*)&d.sc->n_liq, (uint32_t)N);
    else if (d.split_liq) n = ngen = min(*(volatile const uint32_t*)&d.sc->n_slow, (uint32_t)N);
    else n = blist_len(d, ngen);
    const uint32_t* __restrict__ list = d.wl_slow;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    __shared__ uint32_t sNif[4], sVb[4];
    __shared__ double sV[4];
    __shared__ float sS[4];
    __shared__ AccTable sAcc;   // (the shell instances' sphere sums)
    float sbb_t = 0.f;   // Lean: the thread's bounce-back mass over all its rounds
    if (Lean) {
        acc_table_clear(sAcc);
        __syncthreads();
    }

    // every thread of the block runs the same number of rounds (block and warp collectives)
    for (uint32_t base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
        const uint32_t k = base + threadIdx.x;
        SphAcc acc;
        acc.pid = kNone;
        float sbb = 0.f;
        uint32_t vb = kNone;      // the cell's bubble, for an interface cell
        float vphi = 1.f;         // and its new fill level
        bool isIFc = false;
        if (k < n) {
            if (Mode == kBndLeanFast) {
                // a classified liquid cell with links into one sphere only: no neighbour loads
                // (the others are the rare instance's)
                const uint2 lk = d.wl_link[k];
                if (!(lk.x & kLinkRare))
                    lean_cell<S>(d, fa, fb, d.rho[cur], d.rho[cur ^ 1], list[(uint32_t)N - 1u - k], lk.x, lk.y, acc, sbb);
            } else {
                const size_t i = Mode == kBndRare ? d.wl_rare[k] : (Lean ? list[(uint32_t)N - 1u - k] : blist_cell(d, k, ngen));
                boundary_cell<S, Lean>(d, fa, fb, phia, phib, cur, i, acc, sbb, vb, vphi, isIFc);
            }
        }

        if (Lean) {
            sbb_t += sbb;
            acc_table_add(d, acc, sAcc);
            __syncthreads();
            acc_table_flush(d, sAcc);
            __syncthreads();
            continue;
        }
        // ---- per-warp partial sums: interface part of the bubble volumes (1 - phi, FP64),
        // interface count and bounce-back mass; folded per block below (one atomic each)
        const unsigned nifw = __popc(__ballot_sync(full, isIFc));
        const uint32_t lead = __reduce_min_sync(full, vb);
        double vsum = 0.0;
        uint32_t vbub = kNone;
        if (lead < (uint32_t)d.nbub) {
            if (__all_sync(full, vb == lead || vb == kNone)) {
                vsum = warp_sum(vb == lead ? 1.0 - (double)vphi : 0.0);
                vbub = lead;
            } else if (vb < (uint32_t)d.nbub) {   // lanes of several bubbles (rare)
                atomicAdd(&d.bub[vb].Vif, 1.0 - (double)vphi);
            }
        }
        const float sbbw = warp_sum(sbb);
        if (lane == 0) {
            const int w = threadIdx.x >> 5;
            sNif[w] = nifw;
            sV[w] = vsum;
            sVb[w] = vbub;
            sS[w] = sbbw;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t ni = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) ni += sNif[w];
            if (ni) atomicAdd(&d.sc->n_iface_acc, ni);
            double v = 0.0;
            uint32_t vb0 = kNone;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
                if (sVb[w] == kNone) continue;
                if (vb0 != kNone && sVb[w] != vb0) {
                    atomicAdd(&d.bub[vb0].Vif, v);
                    v = 0.0;
                }
                vb0 = sVb[w];
                v += sV[w];
            }
            if (vb0 != kNone) atomicAdd(&d.bub[vb0].Vif, v);
            double sb = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) sb += (double)sS[w];
            if (sb != 0.0) atomicAdd(&d.sc->S_bb, sb);
        }
        if (base + gridDim.x * blockDim.x < n) __syncthreads();   // shared slots reused next round

        sph_acc_warp_reduce(d, acc);
    }
    if (Lean) {
        const double sw = warp_sum((double)sbb_t);
        if (lane == 0 && sw != 0.0) atomicAdd(&d.sc->S_bb, sw);
    }
}

// the bulk sweep of grid cur on stream s
template <bool Whole>
static void sweep_bulk(const Dev& d, int cur, cudaStream_t s) {
    const int bx = d.nx >= 128 ? 128 : ((d.nx + 31) / 32) * 32;
    const int by = 128 / bx;
    dim3 block(bx, by, 1);
    dim3 grid((d.nx + bx - 1) / bx, (d.ny + by - 1) / by, d.nz);
    switch (d.storage) {
        case LBM_STORE_F32: sweep_bulk_kernel<LBM_STORE_F32, Whole><<<grid, block, 0, s>>>(d, cur); break;
        case LBM_STORE_F16DEV: sweep_bulk_kernel<LBM_STORE_F16DEV, Whole><<<grid, block, 0, s>>>(d, cur); break;
        default: sweep_bulk_kernel<LBM_STORE_BF16DEV, Whole><<<grid, block, 0, s>>>(d, cur); break;
    }
}
void launch_sweep_bulk(const Dev& d, int cur, cudaStream_t s, bool whole) {
    if (whole) sweep_bulk<true>(d, cur, s);
    else sweep_bulk<false>(d, cur, s);
}

// the rest of the sweep once the end-of-step kernels are done: the general boundary kernel on
// `side` and the lean one on `side2`, forked from and joined back into `s` by events, the fix
// pass on `s`; all three read grid cur and write disjoint cells of grid cur ^ 1
// (with the lean kernel, one general block per SM, 200 registers a thread: the lean kernel's
// blocks fit beside it)
template <int S>
static void sweep_rest(const Dev& d, int cur, cudaStream_t s, cudaStream_t side, cudaStream_t side2) {
    sweep_boundary_kernel<S, kBndGeneral><<<d.split_liq ? 152 : kBoundaryGrid, 128, 0, side>>>(d, cur);
    if (d.split_liq && d.wl_link) {   // classified: the one-sphere cells, then the rare ones
        sweep_boundary_kernel<S, kBndLeanFast><<<152 * 6, 128, 0, side2>>>(d, cur);
        sweep_boundary_kernel<S, kBndRare><<<152 * 4, 128, 0, side2>>>(d, cur);
    } else if (d.split_liq) {
        sweep_boundary_kernel<S, kBndLean><<<152 * 4, 128, 0, side2>>>(d, cur);
    }
    sweep_fix_kernel<S><<<152 * 2, 128, 0, s>>>(d, cur);
}

void launch_sweep_rest(const Dev& d, int cur, cudaStream_t s, cudaStream_t side, cudaStream_t side2, cudaEvent_t fork,
                       cudaEvent_t join, cudaEvent_t join2) {
    cudaEventRecord(fork, s);
    cudaStreamWaitEvent(side, fork, 0);
    if (d.split_liq) cudaStreamWaitEvent(side2, fork, 0);
    switch (d.storage) {
        case LBM_STORE_F32: sweep_rest<LBM_STORE_F32>(d, cur, s, side, side2); break;
        case LBM_STORE_F16DEV: sweep_rest<LBM_STORE_F16DEV>(d, cur, s, side, side2); break;
        default: sweep_rest<LBM_STORE_BF16DEV>(d, cur, s, side, side2); break;
    }
    cudaEventRecord(join, side);
    cudaStreamWaitEvent(s, join, 0);
    if (d.split_liq) {
        cudaEventRecord(join2, side2);
        cudaStreamWaitEvent(s, join2, 0);
    }
}

}  // namespace lbm
