// lbm_adjoint.cu -- reverse mode of the stream-collide step over a window with frozen cell
// types (liquid cells only: walls, periodic axes and fixed spheres, no free surface), for
// gradients of J = sum over the window's steps of jdir . (total momentum-exchange force on
// the spheres, Eqs. netforce, momentum_transfer) with respect to the relaxation time tau and
// the body force g.
//
// Forward step (lbm_step's sweep, restricted to liquid cells):
//   fin_q(x)  = f*_q(x - c_q)                 source liquid              (Eq. LBE1)
//             = f*_q^(x)                       source beyond a wall
//             = f*_q^(x) + rho0(x) cw_q        source in a sphere          (Eq. bbrule)
//     with rho0 = sum_k f*_k(x), cw_q = 6 w_q c_q . u_w (the fixed sphere's surface velocity)
//   f*(x, t+1) = C(fin(x); tau, g)             TRT + Guo collision          (Eq. LBE2)
//   F(t+1)    = sum over sphere links of -c_q (f*_q^(x) + fin_q(x))
// Reverse step: given lam(t+1) = dL/df*(t+1), with mu = (dC/dfin)^T lam(t+1):
//   lam_q(x - c_q, t) = mu_q(x)                          (one consumer per PDF: unique writer)
//   lam_q^(x, t)      = mu_q(x) [- 2 jdir.c_q at a sphere link]   (wall / sphere sources)
//   lam_k(x, t)      += sum over sphere links of (mu_q(x) - jdir.c_q) cw_q   (for all k)
//   dL/dtheta        += lam(t+1) . dC/dtheta
#include "lbm_internal.cuh"

namespace lbm {

enum : uint8_t { L_FLUID = 0, L_WALL = 1, L_SPHERE = 2 };

// pulled post-collision deviations of liquid cell i at (x,y,z) from grid f (FP32 deviations),
// with the kind of every link, its source index and, for sphere links, cw_q; the same
// arithmetic as the sweep kernels
__device__ __forceinline__ void frozen_pull(const Dev& d, const float* __restrict__ f, uint32_t i, int x, int y, int z,
                                            float (&fin)[kQ], float (&fo)[kQ], uint8_t (&kind)[kQ], uint32_t (&src)[kQ],
                                            float (&cw)[kQ], float& rho0) {
    const size_t N = d.N;
    const uint32_t nx = (uint32_t)d.nx, nxy = (uint32_t)d.nx * (uint32_t)d.ny;
    const uint32_t xm = x == 0 ? nx - 1 : x - 1, xp = x == d.nx - 1 ? 0 : x + 1;
    const uint32_t ym = (y == 0 ? d.ny - 1 : y - 1) * nx, yp = (y == d.ny - 1 ? 0 : y + 1) * nx, y0 = y * nx;
    const uint32_t zm = (z == 0 ? d.nz - 1 : z - 1) * nxy, zp = (z == d.nz - 1 ? 0 : z + 1) * nxy, z0 = z * nxy;
    const bool wxm = !d.bc[0] && x == 0, wxp = !d.bc[0] && x == d.nx - 1;
    const bool wym = !d.bc[1] && y == 0, wyp = !d.bc[1] && y == d.ny - 1;
    const bool wzm = !d.bc[2] && z == 0, wzp = !d.bc[2] && z == d.nz - 1;
    float drho0 = 0.f;
#pragma unroll
    for (int q = 0; q < kQ; q++) {
        fo[q] = f[(size_t)q * N + i];
        drho0 += fo[q];
    }
    rho0 = 1.f + drho0;
    uint32_t pid = kNone;
    float r[3] = {0.f, 0.f, 0.f}, us[3] = {0.f, 0.f, 0.f}, ws[3] = {0.f, 0.f, 0.f};
    fin[0] = fo[0];
    kind[0] = L_FLUID;
    src[0] = i;
    cw[0] = 0.f;
#pragma unroll
    for (int q = 1; q < kQ; q++) {
        const uint32_t sx = cx(q) == 1 ? xm : (cx(q) == -1 ? xp : (uint32_t)x);
        const uint32_t sy = cy(q) == 1 ? ym : (cy(q) == -1 ? yp : y0);
        const uint32_t sz = cz(q) == 1 ? zm : (cz(q) == -1 ? zp : z0);
        const bool wall = (cx(q) == 1 && wxm) || (cx(q) == -1 && wxp) || (cy(q) == 1 && wym) ||
                          (cy(q) == -1 && wyp) || (cz(q) == 1 && wzm) || (cz(q) == -1 && wzp);
        cw[q] = 0.f;
        if (wall) {
            kind[q] = L_WALL;
            src[q] = i;
            fin[q] = fo[opp(q)];
            continue;
        }
        const uint32_t j = sx + sy + sz;
        src[q] = j;
        if (d.flags[j] & F_ACTIVE) {
            kind[q] = L_FLUID;
            fin[q] = f[(size_t)q * N + j];
            continue;
        }
        kind[q] = L_SPHERE;
        const uint32_t P = d.owner[j];
        if (P >= (uint32_t)d.nsph) { fin[q] = fo[opp(q)]; continue; }
        if (P != pid) {   // x - x_P with the image of the cell nearest to the centre
            pid = P;
            const SphLink l = d.sphl[P];
            const int c[3] = {x, y, z};
            int img[3];
            sph_offset(d, l, c, img, r);
            for (int k = 0; k < 3; k++) {
                us[k] = l.u[k];
                ws[k] = l.w[k];
            }
        }
        const float rx = r[0] - 0.5f * cx(q), ry = r[1] - 0.5f * cy(q), rz = r[2] - 0.5f * cz(q);
        const float uwx = us[0] + ws[1] * rz - ws[2] * ry;
        const float uwy = us[1] + ws[2] * rx - ws[0] * rz;
        const float uwz = us[2] + ws[0] * ry - ws[1] * rx;
        cw[q] = 6.f * wgt(q) * cdot(q, uwx, uwy, uwz);
        fin[q] = fo[opp(q)] + 6.f * wgt(q) * rho0 * cdot(q, uwx, uwy, uwz);
    }
}

// the frozen window's cells split as in the forward sweep: BULK liquid cells (every neighbour
// liquid or beyond a wall) in a lean kernel over the grid, the listed others (next to a sphere)
// in a general one; the list is the one the last lbm_step built, valid while no cell changes type

// the boundary cells' forward step (the bulk cells run the forward sweep's own bulk kernel)
__global__ void __launch_bounds__(128) frozen_boundary_kernel(const Dev d, const float* __restrict__ f_in,
                                                              float* __restrict__ f_out) {
    uint32_t ngen;
    const uint32_t n = blist_len(d, ngen);
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint32_t i = blist_cell(d, k, ngen);
        if (i == kNone || !(d.flags[i] & F_LIQ) || (d.flags[i] & F_BULK)) continue;
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        float fin[kQ], fo[kQ], cw[kQ], rho0;
        uint8_t kind[kQ];
        uint32_t src[kQ];
        frozen_pull(d, f_in, i, x, y, z, fin, fo, kind, src, cw, rho0);
        collide_store<LBM_STORE_F32>(d, f_out, i, fin);
    }
}

void launch_frozen_forward(const Dev& d, const float* f_in, float* f_out, cudaStream_t s, cudaStream_t side,
                           cudaEvent_t fork, cudaEvent_t join) {
    Dev dd = d;   // the forward bulk kernel reads grid 0 and writes grid 1
    dd.f[0] = const_cast<float*>(f_in);
    dd.f[1] = f_out;
    cudaEventRecord(fork, s);
    cudaStreamWaitEvent(side, fork, 0);
    frozen_boundary_kernel<<<152 * 2, 128, 0, side>>>(dd, f_in, f_out);
    launch_sweep_bulk(dd, 0, s, false);   // its boundary kernel runs beside it
    cudaEventRecord(join, side);
    cudaStreamWaitEvent(s, join, 0);
}

// ---- reverse step -------------------------------------------------------------------------
// Parameter-gradient partial sums go to kAdjSlots FP64 slots (block id mod kAdjSlots):
// part[slot][0..2] = lam . dC/dg, part[slot][3] = lam . dC/dlambda_+, part[slot][4] = lam . dC/dlambda_-

// (dC/dfin)^T lam of the TRT + Guo collision of one cell, as dL/dfin_q = mu_q(lam) + base +
// (Lu . c_q) inv, mu the direct (pair-local) part; the parameter terms are added to acc
struct AdjOut {
    float base, lx, ly, lz, inv;
};

__device__ __forceinline__ AdjOut collide_adjoint(const Dev& d, const float (&fin)[kQ], const float (&lam)[kQ],
                                                  float (&acc)[5]) {
    const Dev::CollisionConsts& k = d.cc;
    const float gx = d.g[0], gy = d.g[1], gz = d.g[2];
    const float lp = d.lp, lm = d.lm;
    const float cp = 1.f + 0.5f * lp, cm = 1.f + 0.5f * lm;
    // moments from the sums and differences of opposite pairs (reused below)
    float fsum[9], fdif[9];
    float drho = fin[0], jxm = 0.f, jym = 0.f, jzm = 0.f;
#pragma unroll
    for (int p = 0; p < 9; p++) {
        const int q = 2 * p + 1;
        fsum[p] = fin[q] + fin[q + 1];
        fdif[p] = fin[q] - fin[q + 1];
        drho += fsum[p];
        jxm = cacc(cx(q), jxm, fdif[p]); jym = cacc(cy(q), jym, fdif[p]); jzm = cacc(cz(q), jzm, fdif[p]);
    }
    const float rho = 1.f + drho, inv = 1.f / rho;
    const float ux = (jxm + 0.5f * rho * gx) * inv, uy = (jym + 0.5f * rho * gy) * inv, uz = (jzm + 0.5f * rho * gz) * inv;
    const float usq = ux * ux + uy * uy + uz * uz, ug = ux * gx + uy * gy + uz * gz;
    float Lrho, Lux, Luy, Luz;   // lam . dC/drho, lam . dC/du at fixed fin
    float Gx, Gy, Gz;            // lam . dC/dg at fixed u
    float Tp, Tm;                // lam . dC/dlambda_+, lam . dC/dlambda_-
    {
        const float w = wgt(0), L0 = lam[0];
        const float ep = w * (drho - 1.5f * rho * usq), Gp = w * rho * (-3.f * ug);
        Lrho = L0 * (-lp * w * (1.f - 1.5f * usq) + cp * w * (-3.f * ug));
        const float a = L0 * w * rho * 3.f;
        Lux = a * (lp * ux - cp * gx);
        Luy = a * (lp * uy - cp * gy);
        Luz = a * (lp * uz - cp * gz);
        Gx = -a * cp * ux;
        Gy = -a * cp * uy;
        Gz = -a * cp * uz;
        Tp = L0 * ((fin[0] - ep) + 0.5f * Gp);
        Tm = 0.f;
    }
    // The pairs (q, qb), with Lp = lam_q + lam_qb, Lm = lam_q - lam_qb, A = c_q.u, B = c_q.g,
    // s = w rho and R0 = -lp (1 - 1.5 u.u) - 3 cp u.g:
    //   d/drho:  w (Lp (R0 + A (9 cp B - 4.5 lp A)) + 3 Lm (cm B - lm A))
    //   d/du:    c_q s (Lp (9 cp B - 9 lp A) - 3 lm Lm) + 3 s Lp (lp u - cp g)
    //   d/dg:    c_q s (9 cp A Lp + 3 cm Lm) - 3 cp s Lp u
    //   d/dlp:   Lp ((f_q + f_qb)/2 - w drho + s (4.5 A (B - A) + 1.5 (u.u - u.g)))
    //   d/dlm:   Lm ((f_q - f_qb)/2 + 1.5 s (B - 2 A))
    // the terms that do not depend on the pair's direction are summed per weight and applied once
    const float R0 = -lp * (1.f - 1.5f * usq) - 3.f * cp * ug;
    const float lp45 = 4.5f * lp, lp9 = 9.f * lp, lm3 = 3.f * lm, cp9 = 9.f * cp, cm3 = 3.f * cm;
    const float sf = wgt(1) * rho, se = wgt(7) * rho;
    float rxf = 0.f, rxe = 0.f, ryf = 0.f, rye = 0.f;   // sums of Lp (R0 + ...), Lm (cm B - lm A)
    float slf = 0.f, sle = 0.f;                         // sums of Lp
    float taf = 0.f, tae = 0.f, tbf = 0.f, tbe = 0.f;   // sums of Lp A (B - A), Lm (B - 2 A)
    float tfp = 0.f, tfm = 0.f;                         // sums of Lp (f_q + f_qb), Lm (f_q - f_qb)
#pragma unroll
    for (int p = 0; p < 9; p++) {
        const int q = 2 * p + 1, qb = q + 1;
        const bool face = q <= 6;
        const float s = face ? sf : se;
        const float Lp = lam[q] + lam[qb], Lm = lam[q] - lam[qb];
        const float A = cdot(q, ux, uy, uz), B = k.cg[p];
        const float X = fmaf(A, fmaf(-lp45, A, k.K[p]), R0);
        const float Y = fmaf(-lm, A, k.M[p]);
        if (face) { rxf = fmaf(Lp, X, rxf); ryf = fmaf(Lm, Y, ryf); slf += Lp; }
        else { rxe = fmaf(Lp, X, rxe); rye = fmaf(Lm, Y, rye); sle += Lp; }
        const float ap = s * fmaf(-lm3, Lm, Lp * fmaf(-lp9, A, k.K[p]));
        Lux = cacc(cx(q), Lux, ap); Luy = cacc(cy(q), Luy, ap); Luz = cacc(cz(q), Luz, ap);
        const float ag = s * fmaf(cp9 * A, Lp, cm3 * Lm);
        Gx = cacc(cx(q), Gx, ag); Gy = cacc(cy(q), Gy, ag); Gz = cacc(cz(q), Gz, ag);
        const float ta = Lp * (A * (B - A)), tb = Lm * fmaf(-2.f, A, B);
        if (face) { taf += ta; tbf += tb; }
        else { tae += ta; tbe += tb; }
        tfp = fmaf(Lp, fsum[p], tfp);
        tfm = fmaf(Lm, fdif[p], tfm);
    }
    Lrho += wgt(1) * fmaf(3.f, ryf, rxf) + wgt(7) * fmaf(3.f, rye, rxe);
    const float S3 = 3.f * (sf * slf + se * sle);
    Lux += S3 * (lp * ux - cp * gx);
    Luy += S3 * (lp * uy - cp * gy);
    Luz += S3 * (lp * uz - cp * gz);
    Gx -= cp * S3 * ux;
    Gy -= cp * S3 * uy;
    Gz -= cp * S3 * uz;
    const float c15 = 1.5f * (usq - ug);
    Tp += 0.5f * tfp - drho * (wgt(1) * slf + wgt(7) * sle) + sf * fmaf(4.5f, taf, c15 * slf) + se * fmaf(4.5f, tae, c15 * sle);
    Tm += 0.5f * tfm + 1.5f * (sf * tbf + se * tbe);
    // u = (j + rho g/2)/rho: du/dfin_k = (c_k + g/2 - u)/rho, du/dg = I/2
    acc[0] += Gx + 0.5f * Lux;
    acc[1] += Gy + 0.5f * Luy;
    acc[2] += Gz + 0.5f * Luz;
    acc[3] += Tp;
    acc[4] += Tm;
    AdjOut o;
    o.base = Lrho + (Lux * (0.5f * gx - ux) + Luy * (0.5f * gy - uy) + Luz * (0.5f * gz - uz)) * inv;
    o.lx = Lux * inv;
    o.ly = Luy * inv;
    o.lz = Luz * inv;
    o.inv = inv;
    return o;
}

// dL/dfin_q of a cell from its adjoint variables lam and the collision adjoint o
__device__ __forceinline__ float adj_in_q(const Dev& d, int q, const float (&lam)[kQ], const AdjOut& o) {
    float mu;
    if (q == 0) {
        mu = lam[0] * (1.f + d.lp);
    } else {
        const int qa = (q & 1) ? q : q - 1, qb = qa + 1;
        const float Lp = lam[qa] + lam[qb], Lm = lam[qa] - lam[qb];
        mu = lam[q] + 0.5f * d.lp * Lp + ((q & 1) ? 0.5f : -0.5f) * d.lm * Lm;
    }
    return mu + o.base + cdot(q, o.lx, o.ly, o.lz);
}

// the same for all 19 directions, pair by pair: out_q = lam_q + (lp Lp + lm Lm)/2 + base + c_q.l,
// out_qb = lam_qb + (lp Lp - lm Lm)/2 + base - c_q.l
__device__ __forceinline__ void adj_in_all(const Dev& d, const float (&lam)[kQ], const AdjOut& o, float (&out)[kQ]) {
    const float hlp = 0.5f * d.lp, hlm = 0.5f * d.lm;
    out[0] = fmaf(lam[0], 1.f + d.lp, o.base);
#pragma unroll
    for (int p = 0; p < 9; p++) {
        const int q = 2 * p + 1, qb = q + 1;
        const float Lp = lam[q] + lam[qb], Lm = lam[q] - lam[qb];
        const float hp = fmaf(hlp, Lp, o.base);
        const float hm = fmaf(hlm, Lm, cdot(q, o.lx, o.ly, o.lz));
        out[q] = lam[q] + (hp + hm);
        out[qb] = lam[qb] + (hp - hm);
    }
}

// per-block sums of the five parameter terms into one of kAdjSlots FP64 slots
__device__ __forceinline__ void adj_flush(float (&acc)[5], double* part) {
    __shared__ float red[5][32];
    const int lane = threadIdx.x & 31;
    const int nthreads = blockDim.x * blockDim.y;
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    const int wid = tid >> 5;
#pragma unroll
    for (int k = 0; k < 5; k++) {
        const float v = warp_sum(acc[k]);
        if ((tid & 31) == 0) red[k][wid] = v;
    }
    (void)lane;
    __syncthreads();
    if (tid < 5) {
        double t = 0.0;
        for (int w = 0; w < (nthreads + 31) >> 5; w++) t += (double)red[tid][w];
        const unsigned blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
        if (t != 0.0) atomicAdd(&part[(blk % kAdjSlots) * 5 + tid], t);
    }
}

// reverse step of the BULK cells: pull with the wall index select, collision adjoint, and the
// transposed pull (push) with the same select; no sphere links
__global__ void __launch_bounds__(128, 6) adjoint_bulk_kernel(const Dev d, const float* __restrict__ f,
                                                           const float* __restrict__ lam_in,
                                                           float* __restrict__ lam_out, double* part) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (x < d.nx && y < d.ny) {
        const size_t N = d.N;
        const uint32_t nx = (uint32_t)d.nx, nxy = (uint32_t)d.nx * (uint32_t)d.ny;
        const uint32_t i = (uint32_t)x + nx * (uint32_t)y + nxy * (uint32_t)z;
        const uint8_t fl = d.flags[i];
        if ((fl & F_LIQ) && (fl & F_BULK)) {
            // source of direction q: i - c_q . (1, nx, nx ny) (a grid-uniform offset) where y
            // and z stay inside the grid (the same for a whole warp); x edges wrap or bounce
            const bool inner = y > 0 && y < d.ny - 1 && z > 0 && z < d.nz - 1;
            // no x edge in the warp's 32-aligned run of x either: every source at the offset
            const bool plain = inner && (x & ~31) > 0 && (x | 31) < d.nx - 1;
            const bool edge0 = x == 0, edge1 = x == d.nx - 1, perx = d.bc[0] != 0;
            const uint32_t xm = x == 0 ? nx - 1 : x - 1, xp = x == d.nx - 1 ? 0 : x + 1;
            const uint32_t ym = (y == 0 ? d.ny - 1 : y - 1) * nx, yp = (y == d.ny - 1 ? 0 : y + 1) * nx, y0 = y * nx;
            const uint32_t zm = (z == 0 ? d.nz - 1 : z - 1) * nxy, zp = (z == d.nz - 1 ? 0 : z + 1) * nxy, z0 = z * nxy;
            const bool wxm = !d.bc[0] && x == 0, wxp = !d.bc[0] && x == d.nx - 1;
            const bool wym = !d.bc[1] && y == 0, wyp = !d.bc[1] && y == d.ny - 1;
            const bool wzm = !d.bc[2] && z == 0, wzp = !d.bc[2] && z == d.nz - 1;
            // periodic x: the x-edge lanes' sources one period over (0 elsewhere)
            const uint32_t adjp = edge0 ? nx : 0u, adjm = edge1 ? 0u - nx : 0u;
            // (plane, index) of the PDF direction q pulls: its own opposite PDF beyond a wall
            auto link = [&](int q, uint32_t& plane, uint32_t& idx) {
                if (plain) {
                    plane = (uint32_t)q;
                    idx = i - (uint32_t)(cx(q) + cy(q) * (int32_t)nx + cz(q) * (int32_t)nxy);   // modulo 2^32
                } else if (inner && perx) {
                    plane = (uint32_t)q;
                    idx = i - (uint32_t)(cx(q) + cy(q) * (int32_t)nx + cz(q) * (int32_t)nxy) +
                          (cx(q) == 1 ? adjp : (cx(q) == -1 ? adjm : 0u));
                } else if (inner) {
                    const int32_t o = cx(q) + cy(q) * (int32_t)nx + cz(q) * (int32_t)nxy;
                    bool wall = false;
                    int32_t adj = 0;
                    if (cx(q) == 1 && edge0) { if (perx) adj = (int32_t)nx; else wall = true; }
                    if (cx(q) == -1 && edge1) { if (perx) adj = -(int32_t)nx; else wall = true; }
                    plane = wall ? (uint32_t)opp(q) : (uint32_t)q;
                    idx = wall ? i : i - (uint32_t)o + (uint32_t)adj;   // modulo 2^32
                } else {
                    const uint32_t sx = cx(q) == 1 ? xm : (cx(q) == -1 ? xp : (uint32_t)x);
                    const uint32_t sy = cy(q) == 1 ? ym : (cy(q) == -1 ? yp : y0);
                    const uint32_t sz = cz(q) == 1 ? zm : (cz(q) == -1 ? zp : z0);
                    const bool wall = (cx(q) == 1 && wxm) || (cx(q) == -1 && wxp) || (cy(q) == 1 && wym) ||
                                      (cy(q) == -1 && wyp) || (cz(q) == 1 && wzm) || (cz(q) == -1 && wzp);
                    plane = wall ? (uint32_t)opp(q) : (uint32_t)q;
                    idx = wall ? i : sx + sy + sz;
                }
            };
            // each value is read and written once per reverse step: streaming (evict-first)
            // accesses, which keep the small arrays of the boundary kernel beside it in L2
            float fin[kQ], lam[kQ];
#pragma unroll
            for (int q = 0; q < kQ; q++) {
                uint32_t pl, ix;
                link(q, pl, ix);
                fin[q] = __ldcs(f + (size_t)pl * N + ix);
                lam[q] = __ldcs(lam_in + (size_t)q * N + i);
            }
            const AdjOut o = collide_adjoint(d, fin, lam, acc);
            float out[kQ];
            adj_in_all(d, lam, o, out);
#pragma unroll
            for (int q = 0; q < kQ; q++) {
                uint32_t pl, ix;
                link(q, pl, ix);
                __stcs(lam_out + (size_t)pl * N + ix, out[q]);
            }
        }
    }
    adj_flush(acc, part);
}

// reverse step of the listed cells (next to a sphere): general links, the J source of the
// sphere links and, for moving surfaces, the rho0 sums srho
__global__ void __launch_bounds__(128) adjoint_boundary_kernel(const Dev d, const float* __restrict__ f,
                                                               const float* __restrict__ lam_in,
                                                               float* __restrict__ lam_out, float* __restrict__ srho,
                                                               const float jx, const float jy, const float jz,
                                                               const int moving, double* part) {
    const size_t N = d.N;
    uint32_t ngen;
    const uint32_t n = blist_len(d, ngen);
    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint32_t i = blist_cell(d, k, ngen);
        if (i == kNone || !(d.flags[i] & F_LIQ) || (d.flags[i] & F_BULK)) {
            if (moving) srho[k] = 0.f;
            continue;
        }
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        float fin[kQ], fo[kQ], cw[kQ], rho0;
        uint8_t kind[kQ];
        uint32_t src[kQ];
        frozen_pull(d, f, i, x, y, z, fin, fo, kind, src, cw, rho0);
        float lam[kQ];
#pragma unroll
        for (int q = 0; q < kQ; q++) lam[q] = lam_in[(size_t)q * N + i];
        const AdjOut o = collide_adjoint(d, fin, lam, acc);
        float sr = 0.f;
#pragma unroll
        for (int q = 0; q < kQ; q++) {
            const float m = adj_in_q(d, q, lam, o);
            const float jc = jx * cx(q) + jy * cy(q) + jz * cz(q);
            if (q == 0 || kind[q] == L_FLUID) {
                lam_out[(size_t)q * N + src[q]] = m;
            } else if (kind[q] == L_WALL) {
                lam_out[(size_t)opp(q) * N + i] = m;
            } else {   // F gets -c_q (f*_qbar(x) + fin_q(x)), fin_q = f*_qbar(x) + rho0 cw_q
                lam_out[(size_t)opp(q) * N + i] = m - 2.f * jc;
                sr += (m - jc) * cw[q];
            }
        }
        if (moving) srho[k] = sr;
    }
    adj_flush(acc, part);
}

// the rho0 terms of sphere links with a moving surface, added once every link is scattered
__global__ void adjoint_rho_kernel(const Dev d, const float* __restrict__ srho, float* __restrict__ lam_out) {
    uint32_t ngen;
    const uint32_t n = blist_len(d, ngen);
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint32_t i = blist_cell(d, k, ngen);
        if (i == kNone || !(d.flags[i] & F_LIQ) || (d.flags[i] & F_BULK)) continue;
        const float s = srho[k];
        if (s == 0.f) continue;
        for (int q = 0; q < kQ; q++) lam_out[(size_t)q * d.N + i] += s;
    }
}

void launch_adjoint(const Dev& d, const float* f_fwd, const float* lam_in, float* lam_out, float* srho,
                    const float jdir[3], double* part, bool moving_walls, cudaStream_t s, cudaStream_t side,
                    cudaEvent_t fork, cudaEvent_t join) {
    const int bx = d.nx >= 128 ? 128 : ((d.nx + 31) / 32) * 32;
    const int by = 128 / bx;
    const dim3 block(bx, by, 1);
    const dim3 grid((d.nx + bx - 1) / bx, (d.ny + by - 1) / by, d.nz);
    cudaEventRecord(fork, s);
    cudaStreamWaitEvent(side, fork, 0);
    adjoint_boundary_kernel<<<152 * 2, 128, 0, side>>>(d, f_fwd, lam_in, lam_out, srho, jdir[0], jdir[1], jdir[2],
                                                       moving_walls ? 1 : 0, part);
    adjoint_bulk_kernel<<<grid, block, 0, s>>>(d, f_fwd, lam_in, lam_out, part);
    cudaEventRecord(join, side);
    cudaStreamWaitEvent(s, join, 0);
    if (moving_walls) adjoint_rho_kernel<<<152 * 2, 128, 0, s>>>(d, srho, lam_out);
}

}  // namespace lbm
