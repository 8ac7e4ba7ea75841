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
            const Sphere& sp = d.sph[P];
            const int c[3] = {x, y, z};
            const int L[3] = {d.nx, d.ny, d.nz};
            for (int k = 0; k < 3; k++) {
                int xi = c[k];
                if (d.bc[k]) {
                    const double dd = sp.x[k] - (double)xi;
                    if (dd > 0.5 * L[k]) xi += L[k];
                    else if (dd < -0.5 * L[k]) xi -= L[k];
                }
                r[k] = (float)((double)xi - sp.x[k]);
                us[k] = (float)sp.u[k];
                ws[k] = (float)sp.w[k];
            }
        }
        const float rx = r[0] - 0.5f * cx(q), ry = r[1] - 0.5f * cy(q), rz = r[2] - 0.5f * cz(q);
        const float uwx = us[0] + ws[1] * rz - ws[2] * ry;
        const float uwy = us[1] + ws[2] * rx - ws[0] * rz;
        const float uwz = us[2] + ws[0] * ry - ws[1] * rx;
        cw[q] = 6.f * wgt(q) * (cx(q) * uwx + cy(q) * uwy + cz(q) * uwz);
        fin[q] = fo[opp(q)] + 6.f * wgt(q) * rho0 * (cx(q) * uwx + cy(q) * uwy + cz(q) * uwz);
    }
}

// one forward step of the frozen liquid window on FP32 deviation buffers (f_in -> f_out)
__global__ void frozen_forward_kernel(const Dev d, const float* __restrict__ f_in, float* __restrict__ f_out) {
    for (size_t ii = blockIdx.x * (size_t)blockDim.x + threadIdx.x; ii < d.N; ii += (size_t)gridDim.x * blockDim.x) {
        const uint32_t i = (uint32_t)ii;
        if (!(d.flags[i] & F_LIQ)) continue;
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        float fin[kQ], fo[kQ], cw[kQ], rho0;
        uint8_t kind[kQ];
        uint32_t src[kQ];
        frozen_pull(d, f_in, i, x, y, z, fin, fo, kind, src, cw, rho0);
        collide_store<LBM_STORE_F32>(d, f_out, i, fin);
    }
}

void launch_frozen_forward(const Dev& d, const float* f_in, float* f_out, cudaStream_t s) {
    frozen_forward_kernel<<<152 * 16, 256, 0, s>>>(d, f_in, f_out);
}

// reverse step; parameter-gradient partial sums go to kAdjSlots FP64 slots (block id mod
// kAdjSlots, few blocks per slot): part[slot][0..2] = lam . dC/dg, part[slot][3] =
// lam . dC/dlambda_+, part[slot][4] = lam . dC/dlambda_-

__global__ void adjoint_kernel(const Dev d, const float* __restrict__ f, const float* __restrict__ lam_in,
                               float* __restrict__ lam_out, float* __restrict__ srho, const float jx, const float jy,
                               const float jz, const int moving, double* part) {
    const size_t N = d.N;
    const float gx = d.g[0], gy = d.g[1], gz = d.g[2];
    const float lp = d.lp, lm = d.lm;
    const float cp = 1.f + 0.5f * lp, cm = 1.f + 0.5f * lm;
    float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    for (size_t ii = blockIdx.x * (size_t)blockDim.x + threadIdx.x; ii < N; ii += (size_t)gridDim.x * blockDim.x) {
        const uint32_t i = (uint32_t)ii;
        if (!(d.flags[i] & F_LIQ)) continue;
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        float fin[kQ], fo[kQ], cw[kQ], rho0;
        uint8_t kind[kQ];
        uint32_t src[kQ];
        frozen_pull(d, f, i, x, y, z, fin, fo, kind, src, cw, rho0);
        float drho = 0.f, jxm = 0.f, jym = 0.f, jzm = 0.f;
#pragma unroll
        for (int q = 0; q < kQ; q++) {
            drho += fin[q];
            jxm += cx(q) * fin[q]; jym += cy(q) * fin[q]; jzm += cz(q) * fin[q];
        }
        const float rho = 1.f + drho, inv = 1.f / rho;
        const float ux = (jxm + 0.5f * rho * gx) * inv, uy = (jym + 0.5f * rho * gy) * inv, uz = (jzm + 0.5f * rho * gz) * inv;
        const float usq = ux * ux + uy * uy + uz * uz, ug = ux * gx + uy * gy + uz * gz;
        float lam[kQ], mu[kQ];
#pragma unroll
        for (int q = 0; q < kQ; q++) lam[q] = lam_in[(size_t)q * N + i];
        // collision adjoint: direct part, then the parts through rho and u
        float Lrho = 0.f, Lux = 0.f, Luy = 0.f, Luz = 0.f;   // lam . dH/drho, lam . dH/du
        float Gx = 0.f, Gy = 0.f, Gz = 0.f;                  // lam . dH/dg at fixed u
        float Tp = 0.f, Tm = 0.f;                            // lam . df*/dlambda_+, lam . df*/dlambda_-
        {
            const float w = wgt(0);
            const float ep = w * (drho - 1.5f * rho * usq), Gp = w * rho * (-3.f * ug);
            mu[0] = lam[0] * (1.f + lp);
            Lrho += lam[0] * (-lp * w * (1.f - 1.5f * usq) + cp * w * (-3.f * ug));
            Lux += lam[0] * (-lp * w * rho * (-3.f * ux) + cp * w * rho * (-3.f * gx));
            Luy += lam[0] * (-lp * w * rho * (-3.f * uy) + cp * w * rho * (-3.f * gy));
            Luz += lam[0] * (-lp * w * rho * (-3.f * uz) + cp * w * rho * (-3.f * gz));
            Gx += lam[0] * cp * w * rho * (-3.f * ux);
            Gy += lam[0] * cp * w * rho * (-3.f * uy);
            Gz += lam[0] * cp * w * rho * (-3.f * uz);
            Tp += lam[0] * ((fin[0] - ep) + 0.5f * Gp);
        }
#pragma unroll
        for (int q = 1; q < kQ; q += 2) {
            const int qb = q + 1;
            const float w = wgt(q);
            const float Lp = lam[q] + lam[qb], Lm = lam[q] - lam[qb];
            mu[q] = lam[q] + 0.5f * lp * Lp + 0.5f * lm * Lm;
            mu[qb] = lam[qb] + 0.5f * lp * Lp - 0.5f * lm * Lm;
            const float cu = cx(q) * ux + cy(q) * uy + cz(q) * uz;
            const float cg = cx(q) * gx + cy(q) * gy + cz(q) * gz;
            const float ep = w * (drho + rho * (4.5f * cu * cu - 1.5f * usq));
            const float em = w * rho * 3.f * cu;
            const float Gp = w * rho * (9.f * cu * cg - 3.f * ug), Gm = w * rho * 3.f * cg;
            const float fp = 0.5f * (fin[q] + fin[qb]), fm = 0.5f * (fin[q] - fin[qb]);
            // d/drho of e+, e-, G+, G-
            Lrho += Lp * (-lp * w * (1.f + 4.5f * cu * cu - 1.5f * usq) + cp * w * (9.f * cu * cg - 3.f * ug)) +
                    Lm * (-lm * 3.f * w * cu + cm * 3.f * w * cg);
            // d/du: e+ -> w rho (9 cu c - 3 u), e- -> 3 w rho c, G+ -> w rho (9 cg c - 3 g)
            const float ap = -lp * w * rho * 9.f * cu + cp * w * rho * 9.f * cg;
            Lux += Lp * (ap * cx(q) + 3.f * lp * w * rho * ux - 3.f * cp * w * rho * gx) + Lm * (-lm * 3.f * w * rho * cx(q));
            Luy += Lp * (ap * cy(q) + 3.f * lp * w * rho * uy - 3.f * cp * w * rho * gy) + Lm * (-lm * 3.f * w * rho * cy(q));
            Luz += Lp * (ap * cz(q) + 3.f * lp * w * rho * uz - 3.f * cp * w * rho * gz) + Lm * (-lm * 3.f * w * rho * cz(q));
            // d/dg at fixed u: G+ -> w rho (9 cu c - 3 u), G- -> 3 w rho c
            Gx += Lp * cp * w * rho * (9.f * cu * cx(q) - 3.f * ux) + Lm * cm * 3.f * w * rho * cx(q);
            Gy += Lp * cp * w * rho * (9.f * cu * cy(q) - 3.f * uy) + Lm * cm * 3.f * w * rho * cy(q);
            Gz += Lp * cp * w * rho * (9.f * cu * cz(q) - 3.f * uz) + Lm * cm * 3.f * w * rho * cz(q);
            Tp += Lp * ((fp - ep) + 0.5f * Gp);
            Tm += Lm * ((fm - em) + 0.5f * Gm);
        }
        // u = (j + rho g/2)/rho: du/dfin_k = (c_k + g/2 - u)/rho, du/dg = I/2
        const float ax = (0.5f * gx - ux) * inv, ay = (0.5f * gy - uy) * inv, az = (0.5f * gz - uz) * inv;
        const float base = Lrho + Lux * ax + Luy * ay + Luz * az;
        float sr = 0.f;
#pragma unroll
        for (int q = 0; q < kQ; q++) {
            const float m = mu[q] + base + (Lux * cx(q) + Luy * cy(q) + Luz * cz(q)) * inv;
            const float jc = jx * cx(q) + jy * cy(q) + jz * cz(q);
            if (q == 0 || kind[q] == L_FLUID) {
                lam_out[(size_t)q * N + src[q]] = m;
            } else if (kind[q] == L_WALL) {
                lam_out[(size_t)opp(q) * N + i] = m;
            } else {
                lam_out[(size_t)opp(q) * N + i] = m - 2.f * jc;
                sr += (m - jc) * cw[q];
            }
        }
        if (moving) srho[i] = sr;
        acc[0] += Gx + 0.5f * Lux;
        acc[1] += Gy + 0.5f * Luy;
        acc[2] += Gz + 0.5f * Luz;
        acc[3] += Tp;
        acc[4] += Tm;
    }
    // per-block sums into one of kAdjSlots FP64 slots
    __shared__ float red[5][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = 0; k < 5; k++) {
        const float v = warp_sum(acc[k]);
        if (lane == 0) red[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += (double)red[threadIdx.x][w];
        atomicAdd(&part[(blockIdx.x % kAdjSlots) * 5 + threadIdx.x], t);
    }
}

// the rho0 terms of sphere links with a moving surface, added once every link is scattered
__global__ void adjoint_rho_kernel(const Dev d, const float* __restrict__ srho, float* __restrict__ lam_out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < d.N; i += (size_t)gridDim.x * blockDim.x) {
        if (!(d.flags[i] & F_LIQ)) continue;
        const float s = srho[i];
        if (s == 0.f) continue;
        for (int q = 0; q < kQ; q++) lam_out[(size_t)q * d.N + i] += s;
    }
}

void launch_adjoint(const Dev& d, const float* f_fwd, const float* lam_in, float* lam_out, float* srho, const float jdir[3],
                    double* part, bool moving_walls, cudaStream_t s) {
    adjoint_kernel<<<152 * 8, 256, 0, s>>>(d, f_fwd, lam_in, lam_out, srho, jdir[0], jdir[1], jdir[2], moving_walls ? 1 : 0, part);
    if (moving_walls) adjoint_rho_kernel<<<152 * 8, 256, 0, s>>>(d, srho, lam_out);
}

}  // namespace lbm
