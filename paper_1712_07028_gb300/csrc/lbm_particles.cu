// lbm_particles.cu -- the resolved spheres (Sec. 2.3 of the paper): momentum-exchange force
// and torque from the sweep's accumulators, links between obstacle nodes of two spheres,
// lubrication correction and sub-stepped Newton-Euler integration, then the cells that the
// moved spheres cover and uncover, with PDF refill of uncovered cells.
//
// Neighbour searches use uniform bins of sphere ids rebuilt every step; all FP64.
#include "lbm_internal.cuh"

namespace lbm {

constexpr double kPi = 3.14159265358979323846;

__global__ void bins_insert_kernel(const Dev d) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= d.nsph) return;
    const Sphere& s = d.sph[P];
    d.gasflag[P] = d.gasflag[d.max_sph + P] = 1u;   // the first gas-pressure pass scans every sphere
    const int4 bb = make_int4(bin_coord(d, 0, s.x0[0]), bin_coord(d, 1, s.x0[1]), bin_coord(d, 2, s.x0[2]), 0);
    d.sph_bin[P] = bb;
    const size_t bi = bin_index(d, bb.x, bb.y, bb.z);
    const uint32_t slot = atomicAdd(&d.bin_cnt[bi], 1u);
    if (slot < (uint32_t)d.bin_cap) d.bin_ids[bi * d.bin_cap + slot] = (uint32_t)P;
    else atomicOr(&d.sc->status, S_BIN_OVERFLOW);
}

void launch_bins_insert(const Dev& d, cudaStream_t s) {
    if (d.nsph > 0) bins_insert_kernel<<<(d.nsph + 127) / 128, 128, 0, s>>>(d);
}

// Force and torque of the sweep from the split accumulators (constant part exact in
// integers, times 36), plus the links between obstacle nodes of two spheres:
// F = J + K/36 + C,  T = TJ + (XK - x_P x K)/36 + TC.  Then the start-of-step position is
// recorded.
__device__ inline void sph_prepare_one(const Dev& d, const int P) {
    Sphere& s = d.sph[P];
    SphereAcc& a = d.acc[P];
    double K[3], XK[3];
    for (int k = 0; k < 3; k++) {
        K[k] = (double)(long long)a.K[k];
        XK[k] = (double)(long long)a.XK[k];
        s.Fp[k] = s.F[k];   // the step before, kept for the two-step average
        s.Tp[k] = s.T[k];
    }
    s.hasp = s.stepped;
    s.stepped = 1.0;
    const double xK[3] = {s.x[1] * K[2] - s.x[2] * K[1], s.x[2] * K[0] - s.x[0] * K[2], s.x[0] * K[1] - s.x[1] * K[0]};
    const double inv36 = 1.0 / 36.0;
    for (int k = 0; k < 3; k++) {
        s.F[k] = (a.J[k] + K[k] * inv36) + a.C[k];
        s.T[k] = (a.TJ[k] + (XK[k] - xK[k]) * inv36) + a.TC[k];
        a.J[k] = 0.0; a.TJ[k] = 0.0; a.K[k] = 0ull; a.XK[k] = 0ull; a.C[k] = 0.0; a.TC[k] = 0.0;
        s.x0[k] = s.x[k];
    }
    // a differentiated window's objective: jdir . F summed over spheres and steps, on the device
    const Scalars& c = *d.sc;
    if (c.obj_on) atomicAdd(&d.sc->obj, c.obj_j[0] * s.F[0] + c.obj_j[1] * s.F[1] + c.obj_j[2] * s.F[2]);
}
__global__ void sph_prepare_kernel(const Dev d) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P == 0) d.sc->n_coupled = 0u;   // the first sub-step launch lists them anew
    if (P < d.nsph) sph_prepare_one(d, P);
}

// visit every other sphere whose centre lies in the bins around sphere P
template <class Fn>
__device__ __forceinline__ void for_partners(const Dev& d, int P, const double* xp, Fn fn) {
    int sx[3], sy[3], sz[3];
    const int nx_ = bin_span(d, 0, bin_coord(d, 0, xp[0]), sx);
    const int ny_ = bin_span(d, 1, bin_coord(d, 1, xp[1]), sy);
    const int nz_ = bin_span(d, 2, bin_coord(d, 2, xp[2]), sz);
    for (int c = 0; c < nz_; c++)
        for (int b = 0; b < ny_; b++)
            for (int a = 0; a < nx_; a++) {
                const size_t bi = bin_index(d, sx[a], sy[b], sz[c]);
                uint32_t cnt = d.bin_cnt[bi];
                if (cnt > (uint32_t)d.bin_cap) cnt = (uint32_t)d.bin_cap;
                for (uint32_t e = 0; e < cnt; e++) {
                    const uint32_t Q = d.bin_ids[bi * d.bin_cap + e];
                    if ((int)Q != P) fn(Q);
                }
            }
}

// Links from an obstacle node x of sphere Q into an obstacle node of sphere P: the node
// inside Q carries the equilibrium e_q(1, u_Q(x)) of Q's surface velocity (Sec. 2.3, end of
// the momentum-exchange paragraph), reflected by Eq. bbrule with rho_w = 1 at P's surface.
// One block per sphere P; its threads share the cells of each close partner's box, and only
// cells that can be such a node (covered by Q, within R_P + 1.5 of P) are read.
// links between obstacle nodes of sphere P and of its partners, by one warp (lane of 32); the
// warp's sums go to F_P, T_P with one FP64 atomic per sum.  Each partner's box, the cells both
// within R_Q of Q's centre and within R_P + 1.5 of P's, comes from the two spheres' link data
// (integer cell and FP32 fraction of each centre: no FP64 arithmetic, which issues slowly on this
// GPU), one cell wider on every side than the exact box so that its rounding cannot cut a cell
// off; the FP32 distance tests (with margins) and the lattice's types and owners decide, and
// each link's momentum is computed in FP64 from the sphere table.  Every lane forms the box: in a
// warp that costs the same instructions as one lane forming it.
__device__ inline void sph_contact_one(const Dev& d, const int P, const int lane) {
    const Sphere& s = d.sph[P];
    double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
    const int L[3] = {d.nx, d.ny, d.nz};
    const uint32_t np = min(d.npairs[P], (uint32_t)kPairCap);
    const bool valid = finite3(s.x) && s.R > 0.0 && s.R < 64.0;
    const SphLink lp = d.sphl[P];
    const float RP = (float)s.R;
    for (uint32_t pk = 0; valid && pk < np; pk++) {
        const uint32_t Q = d.pairs[(size_t)P * kPairCap + pk];
        const Sphere& o = d.sph[Q];
        if (!(finite3(o.x) && o.R > 0.0 && o.R < 64.0)) continue;
        const SphLink lq = d.sphl[Q];
        const float RQ = (float)o.R;
        float cq[3];   // Q's centre relative to P's integer cell, minimum image
        float dd2 = 0.f;
        for (int k = 0; k < 3; k++) {
            int di = lq.xi[k] - lp.xi[k];
            if (d.bc[k]) {
                if (2 * di > L[k]) di -= L[k];
                else if (2 * di < -L[k]) di += L[k];
            }
            cq[k] = lp.xf[k] + ((float)di + (lq.xf[k] - lp.xf[k]));
            const float v = cq[k] - lp.xf[k];
            dd2 += v * v;
        }
        // beyond R_P + R_Q + 2 two spheres have no adjacent obstacle nodes (the margin covers FP32)
        const float reach = RP + RQ + 2.f;
        if (dd2 > reach * reach + 1e-3f) continue;
        int lo[3], ext[3], total = 1;
        float oq[3], op[3];
        for (int k = 0; k < 3; k++) {
            const int l = (int)floorf(fmaxf(cq[k] - RQ, lp.xf[k] - (RP + 1.5f))) - 1;
            const int h = (int)ceilf(fminf(cq[k] + RQ, lp.xf[k] + (RP + 1.5f))) + 1;
            ext[k] = max(0, h - l + 1);
            lo[k] = lp.xi[k] + l;
            oq[k] = (float)l - cq[k];
            op[k] = (float)l - lp.xf[k];
            total *= ext[k];
        }
        // a necessary condition only (the lattice's owners decide), with a margin for FP32
        const float RQ2 = RQ * RQ + 0.01f, RP2 = (RP + 1.5f) * (RP + 1.5f) + 0.01f;
        {
            for (int e = lane; e < total; e += 32) {
                const int ex[3] = {e % ext[0], (e / ext[0]) % ext[1], e / (ext[0] * ext[1])};
                int w[3] = {lo[0] + ex[0], lo[1] + ex[1], lo[2] + ex[2]};
                float aq = 0.f, ap = 0.f;
                for (int k = 0; k < 3; k++) {
                    aq += (oq[k] + ex[k]) * (oq[k] + ex[k]);
                    ap += (op[k] + ex[k]) * (op[k] + ex[k]);
                }
                if (aq > RQ2 || ap > RP2) continue;
                bool ok = true;
                for (int k = 0; k < 3; k++) {
                    if (w[k] < 0 || w[k] >= L[k]) {
                        if (!d.bc[k]) { ok = false; break; }
                        w[k] = ((w[k] % L[k]) + L[k]) % L[k];
                    }
                }
                if (!ok) continue;
                const size_t xi = cell_index(d, w[0], w[1], w[2]);
                if (!(d.flags[xi] & F_OBS) || d.owner[xi] != Q) continue;
                // surface velocity of Q at x, and x relative to P (minimum image)
                double rq[3], rp[3];
                for (int k = 0; k < 3; k++) {
                    rq[k] = min_image(d, k, (double)w[k], o.x[k]);
                    rp[k] = min_image(d, k, (double)w[k], s.x[k]);
                }
                const double uq[3] = {o.u[0] + o.w[1] * rq[2] - o.w[2] * rq[1],
                                      o.u[1] + o.w[2] * rq[0] - o.w[0] * rq[2],
                                      o.u[2] + o.w[0] * rq[1] - o.w[1] * rq[0]};
                const double uu = uq[0] * uq[0] + uq[1] * uq[1] + uq[2] * uq[2];
                for (int q = 1; q < kQ; q++) {
                    size_t yi;
                    if (!nbr(d, w[0], w[1], w[2], cx(q), cy(q), cz(q), yi)) continue;
                    if (!(d.flags[yi] & F_OBS) || d.owner[yi] != (uint32_t)P) continue;
                    const double c3[3] = {(double)cx(q), (double)cy(q), (double)cz(q)};
                    const double wq = (double)w72(q) / 72.0;
                    const double cu = c3[0] * uq[0] + c3[1] * uq[1] + c3[2] * uq[2];
                    const double fstar = wq * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
                    const double rw[3] = {rp[0] + 0.5 * c3[0], rp[1] + 0.5 * c3[1], rp[2] + 0.5 * c3[2]};
                    const double uw[3] = {s.u[0] + s.w[1] * rw[2] - s.w[2] * rw[1],
                                          s.u[1] + s.w[2] * rw[0] - s.w[0] * rw[2],
                                          s.u[2] + s.w[0] * rw[1] - s.w[1] * rw[0]};
                    const double back = fstar - 6.0 * wq * (c3[0] * uw[0] + c3[1] * uw[1] + c3[2] * uw[2]);
                    const double am = fstar + back;
                    const double dj[3] = {c3[0] * am, c3[1] * am, c3[2] * am};
                    F[0] += dj[0]; F[1] += dj[1]; F[2] += dj[2];
                    T[0] += rp[1] * dj[2] - rp[2] * dj[1];
                    T[1] += rp[2] * dj[0] - rp[0] * dj[2];
                    T[2] += rp[0] * dj[1] - rp[1] * dj[0];
                }
            }
        }
    }
    // (uniform over the warp: only warps with a link sum)
    const bool any = F[0] != 0.0 || F[1] != 0.0 || F[2] != 0.0 || T[0] != 0.0 || T[1] != 0.0 || T[2] != 0.0;
    if (np == 0 || !__any_sync(0xffffffffu, any)) return;
    double v[6] = {F[0], F[1], F[2], T[0], T[1], T[2]};
    for (int c = 0; c < 6; c++) v[c] = warp_sum(v[c]);
    SphereAcc& a = d.acc[P];
    if (lane == 0)
        for (int c = 0; c < 6; c++)
            if (v[c] != 0.0) atomicAdd(c < 3 ? &a.C[c] : &a.TC[c - 3], v[c]);
}

// one warp per sphere with partners (listed by the pair pass)
__global__ void sph_contact_kernel(const Dev d) {
    const uint32_t n = min(*(volatile const uint32_t*)&d.sc->n_paired, (uint32_t)d.nsph);
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t k = warp_id(); k < n; k += nw) sph_contact_one(d, (int)d.sph_list[k], threadIdx.x & 31);
}

// The gas's pressure on the sphere surface the gas touches.  The sweep's links come from
// liquid and interface cells only, and the uniform part of their momentum exchange
// (-2 w_q c_q per link, the reference pressure) cancels over a closed surface; where the gas
// covers part of the surface that part would be missing and the rest of the reference pressure
// would push the sphere.  Every gas cell y beside an obstacle cell o of sphere P (y = o + c_q)
// therefore transfers the momentum of the gas at rest, dj = -2 w_q rho_g c_q into P (rho_g of
// y's bubble, p = rho/3), with the arm y - x_P, as a link from y would.
// Only spheres flagged in flags_in are scanned: those with an interface cell beside them in the
// last sweep (set by the boundary kernel) or gas beside them in the last pass (set here), since
// a cell next to a sphere turns gas only from an interface cell and a sphere covers cells next
// to its surface; the pass clears the flags it read.  One block per sphere.
__global__ void sph_gas_kernel(const Dev d, const int g) {
    const int P = blockIdx.x;
    if (P >= d.nsph) return;
    uint32_t* flags_in = d.gasflag + (size_t)(g ^ 1) * d.max_sph;
    uint32_t* flags_out = d.gasflag + (size_t)g * d.max_sph;
    __shared__ int found;
    const bool scan = flags_in[P] != 0u;
    if (threadIdx.x == 0) found = 0;
    __syncthreads();   // every thread has read the flag before it is cleared
    if (!scan) return;
    const Sphere& s = d.sph[P];
    if (!finite3(s.x) || !(s.R > 0.0 && s.R < 64.0)) return;
    const int L[3] = {d.nx, d.ny, d.nz};
    int lo[3], ext[3];
    for (int k = 0; k < 3; k++) {
        lo[k] = (int)floor(s.x[k] - s.R) - 1;
        ext[k] = (int)ceil(s.x[k] + s.R) + 1 - lo[k] + 1;
    }
    double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
    const int total = ext[0] * ext[1] * ext[2];
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int w[3] = {lo[0] + e % ext[0], lo[1] + (e / ext[0]) % ext[1], lo[2] + e / (ext[0] * ext[1])};
        bool ok = true;
        for (int k = 0; k < 3; k++) {
            if (w[k] < 0 || w[k] >= L[k]) {
                if (!d.bc[k]) { ok = false; break; }
                w[k] = ((w[k] % L[k]) + L[k]) % L[k];
            }
        }
        if (!ok) continue;
        const size_t oi = cell_index(d, w[0], w[1], w[2]);
        if (!(d.flags[oi] & F_OBS) || d.owner[oi] != (uint32_t)P) continue;
        for (int q = 1; q < kQ; q++) {
            size_t yi;
            if (!nbr(d, w[0], w[1], w[2], cx(q), cy(q), cz(q), yi)) continue;
            if (!(d.flags[yi] & F_GAS)) continue;
            found = 1;
            const uint32_t b = d.owner[yi];
            const double rg = b < (uint32_t)d.nbub ? d.bub[b].rho_g : (double)d.rho_g0;
            const double a = 2.0 * (double)w72(q) / 72.0 * rg;
            const double dj[3] = {-a * cx(q), -a * cy(q), -a * cz(q)};
            int y[3];
            cell_xyz(d, yi, y[0], y[1], y[2]);
            double r[3];
            for (int k = 0; k < 3; k++) r[k] = min_image(d, k, (double)y[k], s.x[k]);
            F[0] += dj[0]; F[1] += dj[1]; F[2] += dj[2];
            T[0] += r[1] * dj[2] - r[2] * dj[1];
            T[1] += r[2] * dj[0] - r[0] * dj[2];
            T[2] += r[0] * dj[1] - r[1] * dj[0];
        }
    }
    double v[6] = {F[0], F[1], F[2], T[0], T[1], T[2]};
    for (int c = 0; c < 6; c++) v[c] = warp_sum(v[c]);
    SphereAcc& acc = d.acc[P];
    if ((threadIdx.x & 31) == 0)
        for (int c = 0; c < 6; c++)
            if (v[c] != 0.0) atomicAdd(c < 3 ? &acc.C[c] : &acc.TC[c - 3], v[c]);
    __syncthreads();
    if (threadIdx.x == 0) {
        flags_in[P] = 0u;
        if (found) flags_out[P] = 1u;
    }
}

// partners of sphere P this step: centre distance below R_P + R_Q + 2, which covers the
// lubrication reach (gap < 2/3, the spheres moving less than half a cell per step) and the
// reach of links between obstacle nodes; one warp per sphere, lanes over the 27 bins
__device__ inline void sph_pairs_one(const Dev& d, const uint32_t P, const int lane) {
    const Sphere& s = d.sph[P];
    if (lane == 0) d.npairs[P] = 0;
    __syncwarp();
    int sx[3], sy[3], sz[3];
    // (with more than 1024 spheres the touch preparation has found the sphere's bin)
    const int4 bb = d.nsph > 1024 ? d.sph_bin[P]
                                  : make_int4(bin_coord(d, 0, s.x[0]), bin_coord(d, 1, s.x[1]), bin_coord(d, 2, s.x[2]), 0);
    const int nx_ = bin_span(d, 0, bb.x, sx);
    const int ny_ = bin_span(d, 1, bb.y, sy);
    const int nz_ = bin_span(d, 2, bb.z, sz);
    if (lane < nx_ * ny_ * nz_ && finite3(s.x)) {
        const size_t bi = bin_index(d, sx[lane % nx_], sy[(lane / nx_) % ny_], sz[lane / (nx_ * ny_)]);
        uint32_t cnt = d.bin_cnt[bi];
        if (cnt > (uint32_t)d.bin_cap) cnt = (uint32_t)d.bin_cap;
        for (uint32_t e = 0; e < cnt; e++) {
            const uint32_t Q = d.bin_ids[bi * d.bin_cap + e];
            if (Q == P) continue;
            const Sphere& o = d.sph[Q];
            double dd2 = 0.0;
            for (int k = 0; k < 3; k++) {
                const double v = min_image(d, k, o.x[k], s.x[k]);
                dd2 += v * v;
            }
            const double reach = s.R + o.R + 2.0;
            if (!(dd2 < reach * reach)) continue;
            const uint32_t slot = atomicAdd(&d.npairs[P], 1u);
            if (slot < (uint32_t)kPairCap) d.pairs[(size_t)P * kPairCap + slot] = Q;
            else atomicOr(&d.sc->status, S_BIN_OVERFLOW);
        }
    }
    // the spheres with partners: the only ones the contact-link pass visits
    __syncwarp();
    if (lane == 0 && *(volatile uint32_t*)&d.npairs[P] > 0u) d.sph_list[atomicAdd(&d.sc->n_paired, 1u)] = P;
}

__global__ void sph_pairs_kernel(const Dev d) {
    const uint32_t P = warp_id();
    if (P < (uint32_t)d.nsph) sph_pairs_one(d, P, threadIdx.x & 31);
}

// one Newton-Euler sub-step of sphere P (Sec. 2.3): lubrication (Eq. lubrication, gap
// < 2/3 floored at 0.2 * 2/3, mu = (tau - 1/2)/3) from the sub-step's start state src, then
// u += dt F_tot/m, w += dt T/I, x += dt u into dst.  The hydrodynamic force and torque are
// the mean of this step's and the previous step's momentum exchange (Ladd 1994), which keeps
// light spheres from a two-step oscillation.
// (partners: the np sphere ids of list)
__device__ void substep_one(const Dev& d, const Sphere* src, Sphere* dst, const double dt, const int P,
                            const uint32_t* list, const uint32_t np) {
    const Sphere& s = src[P];
    const double dc = 2.0 / 3.0, mu = ((double)d.tau - 0.5) / 3.0;
    double Fl[3] = {0, 0, 0};
    for (uint32_t k = 0; k < np; k++) {
        const Sphere& o = src[list[k]];
        double dd[3];
        for (int c = 0; c < 3; c++) dd[c] = min_image(d, c, o.x[c], s.x[c]);   // x_12 = x_Q - x_P
        const double dist = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
        double h = dist - s.R - o.R;
        if (!(h < dc) || dist <= 0.0) continue;
        if (h < 0.2 * dc) h = 0.2 * dc;
        const double rr = s.R * o.R, rs = s.R + o.R;
        const double n[3] = {dd[0] / dist, dd[1] / dist, dd[2] / dist};
        const double vn = n[0] * (s.u[0] - o.u[0]) + n[1] * (s.u[1] - o.u[1]) + n[2] * (s.u[2] - o.u[2]);
        const double mag = -6.0 * kPi * mu * rr * rr / (rs * rs) * (1.0 / h - 1.0 / dc) * vn;
        Fl[0] += mag * n[0]; Fl[1] += mag * n[1]; Fl[2] += mag * n[2];
    }
    Sphere o = s;
    const double m = s.rho * 4.0 / 3.0 * kPi * s.R * s.R * s.R, I = 0.4 * m * s.R * s.R;
    const int L[3] = {d.nx, d.ny, d.nz};
    const bool hasp = s.hasp != 0.0;
    for (int k = 0; k < 3; k++) {
        const double Fh = hasp ? 0.5 * (s.F[k] + s.Fp[k]) : s.F[k];
        const double Th = hasp ? 0.5 * (s.T[k] + s.Tp[k]) : s.T[k];
        o.Fl[k] = Fl[k];
        o.u[k] = s.u[k] + dt * (Fh + Fl[k] + m * d.gd[k]) / m;
        o.w[k] = s.w[k] + dt * Th / I;
    }
    for (int k = 0; k < 3; k++) {
        o.x[k] = s.x[k] + dt * o.u[k];
        if (d.bc[k]) o.x[k] = wrap_pos(o.x[k], L[k]);
    }
    dst[P] = o;
}

// Sub-steps of many spheres, one launch per sub-step. The first launch splits them: the partners
// that can come within lubrication reach this step are found by an FP32 prefilter on the
// step-start centres of the link data, with the same margin as the one-block kernel below; a
// sphere with none takes all its sub-steps at once in closed form and writes its final state to
// both buffers; the others keep their near partners, take their first sub-step and are listed,
// and only they run in the later launches, over those partners only (the others cannot come
// within reach; partners are symmetric: a listed sphere reads only listed spheres).
__device__ uint32_t sph_near_partners(const Dev& d, const int P, uint32_t* near) {
    uint32_t nn = 0;
    const SphLink lp = d.sphl[P];
    const float Rp = (float)d.sph[P].R;
    const int L[3] = {d.nx, d.ny, d.nz};
    const uint32_t np = min(d.npairs[P], (uint32_t)kPairCap);
    for (uint32_t k = 0; k < np; k++) {
        const uint32_t Q = d.pairs[(size_t)P * kPairCap + k];
        const SphLink lq = d.sphl[Q];
        float g2 = 0.f;
        for (int c = 0; c < 3; c++) {
            int di = lq.xi[c] - lp.xi[c];
            if (d.bc[c]) {
                if (2 * di > L[c]) di -= L[c];
                else if (2 * di < -L[c]) di += L[c];
            }
            const float v = (float)di + (lq.xf[c] - lp.xf[c]);
            g2 += v * v;
        }
        const float reach = Rp + (float)d.sph[Q].R + 2.f / 3.f + 0.5f;
        if (g2 > reach * reach) continue;
        if (nn < (uint32_t)kNearCap) near[nn++] = Q;
        else atomicOr(&d.sc->status, S_BIN_OVERFLOW);
    }
    return nn;
}
// all n sub-steps of a sphere that feels no lubrication: constant increments, u_k = u_0 + k du,
// x_n = x_0 + dt (n u_0 + n(n+1)/2 du), w_n = w_0 + n dw (the sub-step recurrence up to FP64
// rounding; the same expressions as the one-block kernel)
__device__ Sphere substeps_closed(const Dev& d, const Sphere& s, const double dt) {
    Sphere o = s;
    const double m = s.rho * 4.0 / 3.0 * kPi * s.R * s.R * s.R, I = 0.4 * m * s.R * s.R;
    const int L[3] = {d.nx, d.ny, d.nz};
    const bool hasp = s.hasp != 0.0;
    const double nsub = (double)d.n_sub, tri = 0.5 * nsub * (nsub + 1.0);
    for (int k = 0; k < 3; k++) {
        const double Fh = hasp ? 0.5 * (s.F[k] + s.Fp[k]) : s.F[k];
        const double Th = hasp ? 0.5 * (s.T[k] + s.Tp[k]) : s.T[k];
        const double du = dt * (Fh + 0.0 + m * d.gd[k]) / m, dw = dt * Th / I;
        o.x[k] = s.x[k] + dt * (nsub * s.u[k] + tri * du);
        if (d.bc[k]) o.x[k] = wrap_pos(o.x[k], L[k]);
        o.u[k] = s.u[k] + nsub * du;
        o.w[k] = s.w[k] + nsub * dw;
        o.Fl[k] = 0.0;
    }
    return o;
}
__global__ void sph_substep_first_kernel(const Dev d, Sphere* src, Sphere* dst, const double dt) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= d.nsph) return;
    uint32_t* near = d.sph_near + (size_t)P * kNearCap;
    const uint32_t nn = sph_near_partners(d, P, near);
    if (nn > 0) {
        d.sph_nnear[P] = nn;
        substep_one(d, src, dst, dt, P, near, nn);
        d.sph_cpl[atomicAdd(&d.sc->n_coupled, 1u)] = (uint32_t)P;
    } else {
        const Sphere o = substeps_closed(d, src[P], dt);
        dst[P] = o;
        src[P] = o;   // no listed sphere reads it
    }
}
__global__ void sph_substep_list_kernel(const Dev d, const Sphere* src, Sphere* dst, const double dt) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < *(volatile const uint32_t*)&d.sc->n_coupled) {
        const uint32_t P = d.sph_cpl[t];
        substep_one(d, src, dst, dt, (int)P, d.sph_near + (size_t)P * kNearCap, d.sph_nnear[P]);
    }
}

// All sub-steps in one block (up to 1024 spheres, one per thread): positions and velocities
// of every sphere live in shared memory (double-buffered), the block's barrier separates the
// sub-steps; the same arithmetic as substep_one.  The sub-steps move a sphere by far less than
// a quarter cell per step, so the pair prefilter uses the step-start centres.
__device__ inline void sph_substeps_block(const Dev& d, const double dt, double* smem) {
    const int n = d.nsph;
    double* xs[2] = {smem, smem + 3 * n};
    double* us[2] = {smem + 6 * n, smem + 9 * n};
    double* Rs = smem + 12 * n;
    float* xf = reinterpret_cast<float*>(smem + 13 * n);   // FP32 copy of the centres for the pair prefilter
    const int P = threadIdx.x;
    const bool mine = P < n;
    double x[3] = {0, 0, 0}, u[3] = {0, 0, 0}, w[3] = {0, 0, 0}, Fh[3] = {0, 0, 0}, Th[3] = {0, 0, 0}, Fl[3] = {0, 0, 0};
    double m = 1.0, I = 1.0, R = 0.0;
    if (mine) {
        const Sphere& s = d.sph[P];
        const bool hasp = s.hasp != 0.0;
        for (int k = 0; k < 3; k++) {
            x[k] = s.x[k]; u[k] = s.u[k]; w[k] = s.w[k];
            Fh[k] = hasp ? 0.5 * (s.F[k] + s.Fp[k]) : s.F[k];
            Th[k] = hasp ? 0.5 * (s.T[k] + s.Tp[k]) : s.T[k];
            xs[0][3 * P + k] = x[k];
            us[0][3 * P + k] = u[k];
            xf[3 * P + k] = (float)x[k];
        }
        R = s.R;
        Rs[P] = R;
        m = s.rho * 4.0 / 3.0 * kPi * R * R * R;
        I = 0.4 * m * R * R;
    }
    __syncthreads();
    const double dc = 2.0 / 3.0, mu = ((double)d.tau - 0.5) / 3.0;
    const int L[3] = {d.nx, d.ny, d.nz};
    const uint32_t np = mine ? min(d.npairs[P], (uint32_t)kPairCap) : 0u;
    // the sub-step increments without lubrication are the same every sub-step (the same
    // expressions, so the same bits): computed once
    double du0[3], dw0[3];
    for (int k = 0; k < 3; k++) {
        du0[k] = dt * (Fh[k] + 0.0 + m * d.gd[k]) / m;
        dw0[k] = dt * Th[k] / I;
    }
    // FP32 prefilter on the step-start centres (they move far less than 0.25 per step), once
    // per step: only partners that can come within 2/3 of touching are evaluated in FP64
    uint32_t near[12];   // at most 12 equal spheres touch one (kissing number)
    uint32_t nn = 0;
    for (uint32_t k = 0; k < np; k++) {
        const uint32_t Q = d.pairs[(size_t)P * kPairCap + k];
        float g2 = 0.f;
        for (int c = 0; c < 3; c++) {
            float v = xf[3 * Q + c] - xf[3 * P + c];
            if (d.bc[c]) {
                const float Lc = (float)L[c];
                v -= Lc * rintf(v / Lc);
            }
            g2 += v * v;
        }
        const float reach = (float)(R + Rs[Q]) + 2.f / 3.f + 0.5f;
        if (g2 > reach * reach) continue;
        if (nn < 12) near[nn] = Q;
        else atomicOr(&d.sc->status, S_BIN_OVERFLOW);
        nn++;
    }
    if (nn > 12) nn = 12;
    // a sphere with no partner within reach feels no lubrication: its sub-steps have constant
    // increments, u_k = u_0 + k du, x_n = x_0 + dt (n u_0 + n(n+1)/2 du), w_n = w_0 + n dw
    // (equal to the sub-step recurrence up to FP64 rounding)
    if (mine && nn == 0) {
        const double nsub = (double)d.n_sub, tri = 0.5 * nsub * (nsub + 1.0);
        for (int k = 0; k < 3; k++) {
            x[k] = x[k] + dt * (nsub * u[k] + tri * du0[k]);
            if (d.bc[k]) x[k] = wrap_pos(x[k], L[k]);
            u[k] = u[k] + nsub * du0[k];
            w[k] = w[k] + nsub * dw0[k];
        }
    }
    // the coupled spheres step through the sub-steps together (partners are symmetric: a
    // coupled sphere reads only coupled spheres)
    const int any_coupled = __syncthreads_or(mine && nn > 0);
    for (int sub = 0; any_coupled && sub < d.n_sub; sub++) {
        const int a = sub & 1, b = a ^ 1;
        Fl[0] = Fl[1] = Fl[2] = 0.0;
        for (uint32_t k = 0; k < nn; k++) {
            const uint32_t Q = near[k];
            double dd[3];
            for (int c = 0; c < 3; c++) dd[c] = min_image(d, c, xs[a][3 * Q + c], x[c]);
            const double dist = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
            double h = dist - R - Rs[Q];
            if (!(h < dc) || dist <= 0.0) continue;
            if (h < 0.2 * dc) h = 0.2 * dc;
            const double rr = R * Rs[Q], rs = R + Rs[Q];
            const double nn[3] = {dd[0] / dist, dd[1] / dist, dd[2] / dist};
            const double vn = nn[0] * (u[0] - us[a][3 * Q]) + nn[1] * (u[1] - us[a][3 * Q + 1]) + nn[2] * (u[2] - us[a][3 * Q + 2]);
            const double mag = -6.0 * kPi * mu * rr * rr / (rs * rs) * (1.0 / h - 1.0 / dc) * vn;
            Fl[0] += mag * nn[0]; Fl[1] += mag * nn[1]; Fl[2] += mag * nn[2];
        }
        if (mine && nn > 0) {
            const bool lub = Fl[0] != 0.0 || Fl[1] != 0.0 || Fl[2] != 0.0;
            for (int k = 0; k < 3; k++) {
                u[k] = u[k] + (lub ? dt * (Fh[k] + Fl[k] + m * d.gd[k]) / m : du0[k]);
                w[k] = w[k] + dw0[k];
            }
            for (int k = 0; k < 3; k++) {
                x[k] = x[k] + dt * u[k];
                if (d.bc[k]) x[k] = wrap_pos(x[k], L[k]);
                xs[b][3 * P + k] = x[k];
                us[b][3 * P + k] = u[k];
            }
        }
        __syncthreads();
    }
    if (mine) {
        Sphere& s = d.sph[P];
        double mv = 0.0;
        for (int k = 0; k < 3; k++) {
            const double dk = min_image(d, k, x[k], s.x[k]);
            mv += dk * dk;
            s.x[k] = x[k]; s.u[k] = u[k]; s.w[k] = w[k]; s.Fl[k] = Fl[k];
        }
        // the pair prefilter and partner lists assume less than a quarter cell per step
        if (!(mv <= 0.0625)) atomicOr(&d.sc->status, S_FAST_SPHERE);
    }
}

// the step's force and torque (sph_prepare_one) and all sub-steps in one block
__global__ void sph_substeps_fused_kernel(const Dev d, const double dt) {
    extern __shared__ double smem[];
    if (threadIdx.x < (unsigned)d.nsph) sph_prepare_one(d, threadIdx.x);
    __syncthreads();
    sph_substeps_block(d, dt, smem);
}

__device__ inline void sph_prescribed_one(const Dev& d, const int P) {
    Sphere& s = d.sph[P];
    const int L[3] = {d.nx, d.ny, d.nz};
    for (int k = 0; k < 3; k++) {
        s.x[k] += s.u[k];
        if (d.bc[k]) s.x[k] = wrap_pos(s.x[k], L[k]);
    }
}

__global__ void sph_prescribed_kernel(const Dev d) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P < d.nsph) sph_prescribed_one(d, P);
}

// after an odd number of sub-steps: the listed spheres' final states into the sphere table
// (the others wrote theirs to both buffers)
__global__ void sph_copy_kernel(const Dev d) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < *(volatile const uint32_t*)&d.sc->n_coupled) {
        const uint32_t P = d.sph_cpl[t];
        d.sph[P] = d.sph_tmp[P];
    }
}

// ---------------------------------------------------------------- cover / uncover
constexpr int kTouchWarps = 4;   // spheres per block of the touch kernel
// Each moved sphere's box and offsets, one thread per sphere (its FP64 work then fills every
// lane of a warp, where the touch kernel's warp per sphere would issue it for one lane): FP64
// only splits each centre into an integer cell and an FP32 fraction (as the sweep's link data
// does); the box bounds and offsets follow in integer and FP32 arithmetic (the box has a cell of
// margin on every side, far beyond their rounding).  Also the next sweep's link data.
__device__ void touch_box_prep(const Dev& d, const int P) {
    const Sphere& s = d.sph[P];
    const int L[3] = {d.nx, d.ny, d.nz};
    const SphLink ln = sph_link_of(s);
    d.sphl[P] = ln;   // the next sweep's link data
    d.sph_bin[P] = make_int4(bin_coord(d, 0, s.x[0]), bin_coord(d, 1, s.x[1]), bin_coord(d, 2, s.x[2]), 0);
    TouchBox b;
    b.go = 0;
    if (s.x[0] != s.x0[0] || s.x[1] != s.x0[1] || s.x[2] != s.x0[2]) {
        // a sphere whose centre is not finite or moved more than a cell in one step is left
        // alone (the fluid has gone unstable; the status word says so)
        if (!finite3(s.x) || !finite3(s.x0) || !(s.R > 0.0 && s.R < 64.0)) {
            atomicOr(&d.sc->status, S_UNSTABLE);
        } else {
            const float Rf = (float)s.R;
            const int lim = 2 * (int)ceilf(Rf) + 8;
            b.go = 1;
            for (int k = 0; k < 3; k++) {
                const double f0 = floor(s.x0[k]);
                const int i0 = (int)f0;
                const float x0f = (float)(s.x0[k] - f0);   // old centre = i0 + x0f
                int di = ln.xi[k] - i0;                     // new centre - old: di + (xf - x0f), minimum image
                if (d.bc[k]) {
                    if (2 * di > L[k]) di -= L[k];
                    else if (2 * di < -L[k]) di += L[k];
                }
                const float off = (float)di + (ln.xf[k] - x0f);
                const int lo = i0 + (int)floorf(fminf(x0f, x0f + off) - Rf) - 1;
                const int hi = i0 + (int)ceilf(fmaxf(x0f, x0f + off) + Rf) + 1;
                b.lo[k] = lo;
                b.ext[k] = hi - lo + 1;
                if (hi - lo + 1 > lim) b.go = 0;
                b.a0[k] = (float)(lo - i0) - x0f;   // cell lo minus the old centre
                b.a1[k] = b.a0[k] - off;            // ... minus the new centre
                b.off[k] = min_image(d, k, s.x[k], s.x0[k]);   // for the FP64 decisions
            }
            if (!b.go) atomicOr(&d.sc->status, S_UNSTABLE);
            b.r2f = (float)(s.R * s.R);
        }
    }
    d.tbox[P] = b;
}
__global__ void cover_touch_prep_kernel(const Dev d) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P < d.nsph) touch_box_prep(d, P);
}

// One warp per sphere: the cells of its box whose coverage by this sphere changed are touched
// (deduplicated into a worklist).
__device__ inline void cover_touch_one(const Dev& d, const int P, const int lane) {
    const TouchBox& bx = d.tbox[P];
    const Sphere& s = d.sph[P];
    const int L[3] = {d.nx, d.ny, d.nz};
    if (!bx.go) return;   // (uniform over the warp)
    const double sOffk[3] = {bx.off[0], bx.off[1], bx.off[2]};
    const int lo[3] = {bx.lo[0], bx.lo[1], bx.lo[2]}, ext[3] = {bx.ext[0], bx.ext[1], bx.ext[2]};
    const float a0[3] = {bx.a0[0], bx.a0[1], bx.a0[2]}, a1[3] = {bx.a1[0], bx.a1[1], bx.a1[2]};
    // cell offsets from both centres in FP32 decide wherever |d^2 - R^2| clears their rounding
    // error by far; the few cells closer to the sphere's surface are decided in FP64.  The FP32
    // offsets carry an error under 1e-6 (an exact integer difference less an FP32 fraction), so
    // squared distances near R^2 one of at most a few 1e-6 (1 + R^2): the band is 2e-5 (1 + R^2)
    const float R2f = bx.r2f, band = 2e-5f * (1.f + R2f);
    // each lane takes columns (x, y) of the box and walks them along z
    const int nxy = ext[0] * ext[1];
    for (int exy = lane; exy < nxy; exy += 32) {
        const int ex0 = exy % ext[0], ex1 = exy / ext[0];
        const float ax = a0[0] + (float)ex0, ay = a0[1] + (float)ex1;
        const float bx = a1[0] + (float)ex0, by = a1[1] + (float)ex1;
        const float pxy0 = ax * ax + ay * ay, pxy1 = bx * bx + by * by;
        for (int ex2 = 0; ex2 < ext[2]; ex2++) {
            int w[3] = {lo[0] + ex0, lo[1] + ex1, lo[2] + ex2};
            const float az = a0[2] + (float)ex2, bz = a1[2] + (float)ex2;
            const float f0 = pxy0 + az * az, f1 = pxy1 + bz * bz;
            bool in0 = f0 <= R2f, in1 = f1 <= R2f;
            if (fabsf(f0 - R2f) < band || fabsf(f1 - R2f) < band) {
                const double R2 = s.R * s.R;
                double d0 = 0, d1 = 0;
                for (int k = 0; k < 3; k++) {
                    const double a = (double)w[k] - s.x0[k], b = (double)w[k] - (s.x0[k] + sOffk[k]);
                    d0 += a * a;
                    d1 += b * b;
                }
                in0 = d0 <= R2;
                in1 = d1 <= R2;
            }
            if (in0 == in1) continue;
            bool ok = true;
            for (int k = 0; k < 3; k++) {
                if (w[k] < 0 || w[k] >= L[k]) {
                    if (!d.bc[k]) { ok = false; break; }
                    w[k] = ((w[k] % L[k]) + L[k]) % L[k];
                }
            }
            if (!ok) continue;
            const size_t i = cell_index(d, w[0], w[1], w[2]);
            const uint8_t old = mark_or(d.tmark, i, K_TOUCH);
            if (!(old & K_TOUCH)) wl_push(d.wl_touch, &d.sc->n_touch, (uint32_t)d.wl_cap, (uint32_t)i, &d.sc->status);
        }
    }
}

// Prepared: the boxes were set up by cover_touch_prep_kernel; else lane 0 sets its sphere's up
// (few spheres: one launch less on the step's critical path)
template <bool Prepared>
__global__ void __launch_bounds__(32 * kTouchWarps) cover_touch_kernel(const Dev d) {
    // (a warp's spheres one after another: the loop bound is uniform over the warp)
    for (int P = blockIdx.x * kTouchWarps + (threadIdx.x >> 5); P < d.nsph; P += gridDim.x * kTouchWarps) {
        if (!Prepared) {
            if ((threadIdx.x & 31) == 0) touch_box_prep(d, P);
            __syncwarp();
        }
        cover_touch_one(d, P, threadIdx.x & 31);
    }
}

// touched cells: the lowest id of the spheres covering them now decides; obstacle cells no
// sphere covers any more are uncovered; newly covered cells lose their fluid mass.  One warp
// per cell, its lanes over the 27 neighbouring bins.
template <int S>
__device__ inline void cover_apply_dev(const Dev& d, const int nxt, const uint32_t wid, const uint32_t nw) {
    using T = typename Store<S>::T;
    const T* f = static_cast<const T*>(d.f[nxt]);
    const uint32_t n = min(*(volatile uint32_t*)&d.sc->n_touch, (uint32_t)d.wl_cap);
    const int lane = threadIdx.x & 31;
    for (uint32_t e = wid; e < n; e += nw) {
        const size_t i = d.wl_touch[e];
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        int sx[3], sy[3], sz[3];
        const int nx_ = bin_span(d, 0, bin_coord(d, 0, (double)x), sx);
        const int ny_ = bin_span(d, 1, bin_coord(d, 1, (double)y), sy);
        const int nz_ = bin_span(d, 2, bin_coord(d, 2, (double)z), sz);
        uint32_t best = kNone;
        if (lane < nx_ * ny_ * nz_) {
            const size_t bi = bin_index(d, sx[lane % nx_], sy[(lane / nx_) % ny_], sz[lane / (nx_ * ny_)]);
            uint32_t cnt = d.bin_cnt[bi];
            if (cnt > (uint32_t)d.bin_cap) cnt = (uint32_t)d.bin_cap;
            for (uint32_t k = 0; k < cnt; k++) {
                const uint32_t P = d.bin_ids[bi * d.bin_cap + k];
                if (P < best && sphere_covers(d, d.sph[P], x, y, z)) best = P;
            }
        }
        const uint32_t own = warp_min(best);
        const uint8_t t = d.flags[i] & F_TYPE;
        const float rl = (t & F_LIQ) ? warp_sum(lane < kQ ? Store<S>::get_nc(f, (size_t)lane * d.N + i) : 0.f) : 0.f;
        if (lane != 0) continue;
        if (t & F_OBS) {
            if (own == kNone) mark_or(d.tmark, i, K_UNCOV);
            else d.owner[i] = own;
        } else if (own != kNone) {
            if (t & F_LIQ) {
                atomicAdd(&d.sc->S_cover, (double)(1.f + rl));
            } else if (t & F_IF) {
                atomicAdd(&d.sc->S_cover, (double)d.mass[i]);
                vol_change(d, d.owner[i], -(1.0 - (double)d.phi[nxt][i]), 0, -1);
            } else if (t & F_GAS) {
                vol_change(d, d.owner[i], 0.0, -1, 0);
            }
            d.flags[i] = F_OBS;
            d.owner[i] = own;
            d.mass[i] = 0.f;
        }
    }
}

// uncovered cells take their type from the neighbours that are neither obstacle nor
// uncovered now: only gas -> gas; gas and liquid/interface -> interface with m = mean phi *
// mean rho; else liquid.  f* = e(mean rho, u_P + w_P x (x - x_P)) of the sphere that left.
template <int S>
__device__ inline void cover_refill_dev(const Dev& d, const int nxt, const uint32_t wid, const uint32_t nw) {
    using T = typename Store<S>::T;
    T* f = static_cast<T*>(d.f[nxt]);
    float* phi = d.phi[nxt];
    const uint32_t n = min(*(volatile uint32_t*)&d.sc->n_touch, (uint32_t)d.wl_cap);
    const int lane = threadIdx.x & 31;
    for (uint32_t e = wid; e < n; e += nw) {
        const size_t i = d.wl_touch[e];
        if (!(d.tmark[i] & K_UNCOV)) continue;
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        int isgas = 0, isfl = 0;
        float r = 0.f, ph = 0.f;
        uint32_t myown = kNone;
        size_t j;
        if (lane >= 1 && lane < kQ && nbr(d, x, y, z, cx(lane), cy(lane), cz(lane), j) && !(d.tmark[j] & K_UNCOV)) {
            const uint8_t t = d.flags[j] & F_TYPE;
            if (t & F_GAS) {
                isgas = 1;
                myown = d.owner[j];
            } else if (t & F_ACTIVE) {
                float u[3];
                ph = (t & F_IF) ? phi[j] : 1.f;
                post_moments<S>(d, f, j, ph, r, u);
                isfl = 1;
            }
        }
        const unsigned gmask = __ballot_sync(0xffffffffu, isgas);
        const int ngas = __popc(gmask), nfl = warp_sum(isfl);
        float rs = 0.f, ps = 0.f;
        for (int q = 1; q < kQ; q++) {   // in q order, as a serial sum would take them
            rs += __shfl_sync(0xffffffffu, r, q);
            ps += __shfl_sync(0xffffffffu, ph, q);
        }
        // the bubble of the first gas neighbour in q order
        const uint32_t gown = __shfl_sync(0xffffffffu, myown, gmask ? __ffs(gmask) - 1 : 0);
        const uint32_t P = d.owner[i];
        const Sphere& sp = d.sph[P < (uint32_t)d.nsph ? P : 0];
        double r3[3];
        const int c3[3] = {x, y, z};
        for (int k = 0; k < 3; k++) r3[k] = min_image(d, k, (double)c3[k], sp.x[k]);
        const float uf[3] = {(float)(sp.u[0] + sp.w[1] * r3[2] - sp.w[2] * r3[1]),
                             (float)(sp.u[1] + sp.w[2] * r3[0] - sp.w[0] * r3[2]),
                             (float)(sp.u[2] + sp.w[0] * r3[1] - sp.w[1] * r3[0])};
        if (nfl == 0 && ngas > 0) {
            if (lane == 0) {
                d.flags[i] = F_GAS;
                d.owner[i] = gown;
                d.mass[i] = 0.f;
                phi[i] = 0.f;
                vol_change(d, gown, 0.0, 1, 0);
            }
            continue;
        }
        const float rb = nfl ? rs / (float)nfl : 1.f;
        if (lane < kQ) Store<S>::put(f, (size_t)lane * d.N + i, equilibrium_dev(lane, rb, uf));
        if (lane != 0) continue;
        if (d.rho[nxt]) d.rho[nxt][i] = rb;
        if (ngas > 0) {
            const float pb = ps / (float)nfl;
            d.flags[i] = F_IF;
            d.owner[i] = gown;
            phi[i] = pb;
            d.mass[i] = pb * rb;
            atomicAdd(&d.sc->S_uncover, (double)(pb * rb));
            vol_change(d, gown, 1.0 - (double)pb, 0, 1);
        } else {
            d.flags[i] = F_LIQ;
            d.owner[i] = kNone;
            phi[i] = 1.f;
            d.mass[i] = rb;
            atomicAdd(&d.sc->S_uncover, (double)rb);
        }
    }
}

// BULK bits of every touched cell and its neighbours; marks cleared
__device__ inline void cover_finish_dev(const Dev& d, const uint32_t wid, const uint32_t nw) {
    const uint32_t n = min(*(volatile uint32_t*)&d.sc->n_touch, (uint32_t)d.wl_cap);
    const int lane = threadIdx.x & 31;
    for (uint32_t e = wid; e < n; e += nw) {
        const size_t i = d.wl_touch[e];
        if (lane >= kQ) continue;
        size_t j = i;
        if (lane > 0) {
            int x, y, z;
            cell_xyz(d, i, x, y, z);
            if (!nbr(d, x, y, z, cx(lane), cy(lane), cz(lane), j)) continue;
            merge_check(d, i, j);   // a touched cell against each neighbour
        }
        set_bulk(d, j);
        if (lane == 0) d.tmark[i] = 0;   // BULK reads types only, never marks
    }
}

// the bins are emptied (the end-of-step scan bins the new centres): every bin that holds a
// sphere holds a step-start centre, so clearing them all is clearing those
__device__ inline void bins_clear(const Dev& d, const uint32_t t, const uint32_t nt) {
    const size_t nb = (size_t)d.nbx * (size_t)d.nby * (size_t)d.nbz;
    for (size_t b = t; b < nb; b += nt) d.bin_cnt[b] = 0u;
}

// apply, refill and finish in one launch: one thread-block cluster, the phases separated by
// cluster barriers (the touched cells are few: launches, not work, would set the time); with
// no touched cell it only empties the bins; then the step is closed
constexpr int kCoverCtas = 8, kCoverThreads = 512;
template <int S>
__global__ void __cluster_dims__(kCoverCtas, 1, 1) __launch_bounds__(kCoverThreads) cover_cluster_kernel(const Dev d, const int nxt) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    const uint32_t wid = t >> 5, nw = nt >> 5;
    if (*(volatile const uint32_t*)&d.sc->n_touch != 0u) {   // the same value for every thread
        cover_apply_dev<S>(d, nxt, wid, nw);   // reads the bins
        cluster_sync();
        cover_refill_dev<S>(d, nxt, wid, nw);
        cluster_sync();
        cover_finish_dev(d, wid, nw);
    }
    bins_clear(d, t, nt);
    cluster_sync();
    // the last end-of-step kernel: it closes the step (bubble model, counters, new bins)
    step_close(d, t, nt, true, ClusterSync{});
}

int spheres_links_launches(const Dev& d) { return d.nsph == 0 ? 0 : 3; }

int spheres_launches(const Dev& d) {   // launch_spheres_move + launch_spheres_cover
    if (d.nsph == 0) return 0;
    int n;
    if (d.sphere_mode == LBM_SPHERES_FREE) n = d.nsph <= 1024 ? 1 : 1 + d.n_sub + (d.n_sub & 1);
    else n = 1 + (d.sphere_mode == LBM_SPHERES_PRESCRIBED ? 1 : 0);
    // touch preparation (more than 1024 spheres), touch, cover cluster
    if (d.sphere_mode != LBM_SPHERES_FIXED) n += d.nsph > 1024 ? 3 : 2;
    return n;
}

void prepare_sphere_kernels() {
    // the fused sub-step kernel keeps 13 doubles per sphere in shared memory (<= 1024 spheres)
    cudaFuncSetAttribute(sph_substeps_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (13 * 8 + 3 * 4) * 1024);
}

// the cells whose coverage the move changes (reads only the sphere table; its marks have an
// array of their own, so it may run while the conversions do); with more than 1024 spheres the
// boxes are set up by a kernel of their own
void launch_cover_touch(const Dev& d, cudaStream_t st) {
    if (d.sphere_mode == LBM_SPHERES_FIXED) return;
    const int nb = (d.nsph + kTouchWarps - 1) / kTouchWarps;
    if (d.nsph > 1024) {
        cover_touch_prep_kernel<<<(d.nsph + 127) / 128, 128, 0, st>>>(d);
        // (at most four blocks per SM: it runs beside the bulk sweep at high priority, and a grid of
        // one warp per sphere would take every SM's warp slots while it runs)
        cover_touch_kernel<true><<<nb < 152 * 4 ? nb : 152 * 4, 32 * kTouchWarps, 0, st>>>(d);
    } else {
        cover_touch_kernel<false><<<nb, 32 * kTouchWarps, 0, st>>>(d);
    }
}

// partner lists and the links between obstacle nodes of two spheres: they read only the
// step-start centres (binned), the sphere table and obstacle cells, all final once the cover
// kernel has run, so they run beside the rest of the end-of-step kernels, the next bulk sweep and
// its boundary sweep (their sums wait in the accumulators for sph_prepare_one)
void launch_spheres_links(const Dev& d, int g, cudaStream_t st) {
    if (d.nsph == 0) return;
    sph_pairs_kernel<<<(d.nsph * 32 + 127) / 128, 128, 0, st>>>(d);
    // (many spheres: two blocks per SM, a share of the warp slots beside the bulk sweep)
    sph_contact_kernel<<<d.nsph < 152 * 32 ? (d.nsph + 3) / 4 : 152 * 2, 128, 0, st>>>(d);
    sph_gas_kernel<<<d.nsph, 128, 0, st>>>(d, g);
}

// the step's force and torque, then the motion: sub-stepped Newton-Euler (free spheres) or
// the prescribed velocity, lubrication among the partners; it reads only the sweep's force sums,
// the sphere table and obstacle cells, which the conversions leave alone, so it may run
// concurrently with them
void launch_spheres_move(const Dev& d, cudaStream_t st) {
    if (d.nsph == 0) return;
    const int tb = 128, nb = (d.nsph + tb - 1) / tb;
    if (d.sphere_mode == LBM_SPHERES_FREE && d.nsph <= 1024) {
        const double dt = 1.0 / d.n_sub;
        const size_t shm = sizeof(double) * 13 * (size_t)d.nsph + sizeof(float) * 3 * (size_t)d.nsph;
        sph_substeps_fused_kernel<<<1, d.nsph <= 128 ? 128 : ((d.nsph + 31) / 32) * 32, shm, st>>>(d, dt);
        launch_cover_touch(d, st);
        return;
    }
    sph_prepare_kernel<<<nb, tb, 0, st>>>(d);
    if (d.sphere_mode == LBM_SPHERES_FREE) {
        const double dt = 1.0 / d.n_sub;
        for (int k = 0; k < d.n_sub; k++) {
            Sphere* src = (k & 1) ? d.sph_tmp : d.sph;
            Sphere* dst = (k & 1) ? d.sph : d.sph_tmp;
            if (k == 0) sph_substep_first_kernel<<<nb, tb, 0, st>>>(d, src, dst, dt);
            else sph_substep_list_kernel<<<nb, tb, 0, st>>>(d, src, dst, dt);
        }
        if (d.n_sub & 1) sph_copy_kernel<<<nb, tb, 0, st>>>(d);
    } else if (d.sphere_mode == LBM_SPHERES_PRESCRIBED) {
        sph_prescribed_kernel<<<nb, tb, 0, st>>>(d);
    }
    launch_cover_touch(d, st);
}

// cells covered and uncovered by the moved spheres (after the conversions)
void launch_spheres_cover(const Dev& d, int nxt, cudaStream_t st) {
    if (d.nsph == 0 || d.sphere_mode == LBM_SPHERES_FIXED) return;
    switch (d.storage) {
        case LBM_STORE_F32: cover_cluster_kernel<LBM_STORE_F32><<<kCoverCtas, kCoverThreads, 0, st>>>(d, nxt); break;
        case LBM_STORE_F16DEV: cover_cluster_kernel<LBM_STORE_F16DEV><<<kCoverCtas, kCoverThreads, 0, st>>>(d, nxt); break;
        default: cover_cluster_kernel<LBM_STORE_BF16DEV><<<kCoverCtas, kCoverThreads, 0, st>>>(d, nxt); break;
    }
}

}  // namespace lbm
