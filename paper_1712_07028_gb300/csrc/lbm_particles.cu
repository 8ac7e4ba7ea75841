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
    const size_t bi = bin_index(d, bin_coord(d, 0, s.x0[0]), bin_coord(d, 1, s.x0[1]), bin_coord(d, 2, s.x0[2]));
    const uint32_t slot = atomicAdd(&d.bin_cnt[bi], 1u);
    if (slot < (uint32_t)d.bin_cap) d.bin_ids[bi * d.bin_cap + slot] = (uint32_t)P;
    else atomicOr(&d.sc->status, S_BIN_OVERFLOW);
}

void launch_bins_insert(const Dev& d, cudaStream_t s) {
    if (d.nsph > 0) bins_insert_kernel<<<(d.nsph + 127) / 128, 128, 0, s>>>(d);
}

// Force and torque of the sweep from the split accumulators (constant part exact in
// integers, times 36):  F = J + K/36,  T = TJ + (XK - x_P x K)/36.  Then the start-of-step
// position is recorded and the sphere enters its bin.
__global__ void sph_prepare_kernel(const Dev d) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= d.nsph) return;
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
    for (int k = 0; k < 3; k++) {
        s.F[k] = a.J[k] + K[k] / 36.0;
        s.T[k] = a.TJ[k] + (XK[k] - xK[k]) / 36.0;
        a.J[k] = 0.0; a.TJ[k] = 0.0; a.K[k] = 0ull; a.XK[k] = 0ull;
        s.x0[k] = s.x[k];
    }
    const size_t bi = bin_index(d, bin_coord(d, 0, s.x[0]), bin_coord(d, 1, s.x[1]), bin_coord(d, 2, s.x[2]));
    const uint32_t slot = atomicAdd(&d.bin_cnt[bi], 1u);
    if (slot < (uint32_t)d.bin_cap) d.bin_ids[bi * d.bin_cap + slot] = (uint32_t)P;
    else atomicOr(&d.sc->status, S_BIN_OVERFLOW);
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
// Each thread adds only to its own sphere.
__global__ void sph_contact_kernel(const Dev d) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= d.nsph) return;
    Sphere& s = d.sph[P];
    double F[3] = {0, 0, 0}, T[3] = {0, 0, 0};
    const int L[3] = {d.nx, d.ny, d.nz};
    if (!finite3(s.x) || !(s.R > 0.0 && s.R < 64.0)) return;
    for_partners(d, P, s.x, [&](uint32_t Q) {
        const Sphere& o = d.sph[Q];
        if (!finite3(o.x) || !(o.R > 0.0 && o.R < 64.0)) return;
        double dq[3];
        for (int k = 0; k < 3; k++) dq[k] = min_image(d, k, o.x[k], s.x[k]);
        const double dist2 = dq[0] * dq[0] + dq[1] * dq[1] + dq[2] * dq[2];
        const double reach = s.R + o.R + 2.0;
        if (dist2 > reach * reach) return;
        // cells of Q's box (coordinates unwrapped around P), wrapped when read
        int lo[3], hi[3];
        for (int k = 0; k < 3; k++) {
            const double c = s.x[k] + dq[k];
            lo[k] = (int)floor(c - o.R);
            hi[k] = (int)ceil(c + o.R);
        }
        for (int zz = lo[2]; zz <= hi[2]; zz++)
            for (int yy = lo[1]; yy <= hi[1]; yy++)
                for (int xx = lo[0]; xx <= hi[0]; xx++) {
                    int w[3] = {xx, yy, zz};
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
                        const double a = fstar + back;
                        const double dj[3] = {c3[0] * a, c3[1] * a, c3[2] * a};
                        F[0] += dj[0]; F[1] += dj[1]; F[2] += dj[2];
                        T[0] += rp[1] * dj[2] - rp[2] * dj[1];
                        T[1] += rp[2] * dj[0] - rp[0] * dj[2];
                        T[2] += rp[0] * dj[1] - rp[1] * dj[0];
                    }
                }
    });
    for (int k = 0; k < 3; k++) { s.F[k] += F[k]; s.T[k] += T[k]; }
}

// one Newton-Euler sub-step for every sphere (Sec. 2.3): lubrication (Eq. lubrication, gap
// < 2/3 floored at 0.2 * 2/3, mu = (tau - 1/2)/3) from the sub-step's start state src,
// then u += dt F_tot/m, w += dt T/I, x += dt u into dst
__global__ void sph_substep_kernel(const Dev d, const Sphere* src, Sphere* dst, const double dt) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= d.nsph) return;
    const Sphere& s = src[P];
    const double dc = 2.0 / 3.0, mu = ((double)d.tau - 0.5) / 3.0;
    double Fl[3] = {0, 0, 0};
    for_partners(d, P, s.x0, [&](uint32_t Q) {
        const Sphere& o = src[Q];
        double dd[3];
        for (int k = 0; k < 3; k++) dd[k] = min_image(d, k, o.x[k], s.x[k]);   // x_12 = x_Q - x_P
        const double dist = sqrt(dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2]);
        double h = dist - s.R - o.R;
        if (!(h < dc) || dist <= 0.0) return;
        if (h < 0.2 * dc) h = 0.2 * dc;
        const double rr = s.R * o.R, rs = s.R + o.R;
        const double n[3] = {dd[0] / dist, dd[1] / dist, dd[2] / dist};
        const double vn = n[0] * (s.u[0] - o.u[0]) + n[1] * (s.u[1] - o.u[1]) + n[2] * (s.u[2] - o.u[2]);
        const double mag = -6.0 * kPi * mu * rr * rr / (rs * rs) * (1.0 / h - 1.0 / dc) * vn;
        Fl[0] += mag * n[0]; Fl[1] += mag * n[1]; Fl[2] += mag * n[2];
    });
    Sphere o = s;
    const double m = s.rho * 4.0 / 3.0 * kPi * s.R * s.R * s.R, I = 0.4 * m * s.R * s.R;
    const int L[3] = {d.nx, d.ny, d.nz};
    // the hydrodynamic force and torque are the mean of this step's and the previous step's
    // momentum exchange (Ladd 1994), which keeps light spheres from a two-step oscillation
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

__global__ void sph_prescribed_kernel(const Dev d) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= d.nsph) return;
    Sphere& s = d.sph[P];
    const int L[3] = {d.nx, d.ny, d.nz};
    for (int k = 0; k < 3; k++) {
        s.x[k] += s.u[k];
        if (d.bc[k]) s.x[k] = wrap_pos(s.x[k], L[k]);
    }
}

__global__ void sph_copy_kernel(const Dev d) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P < d.nsph) d.sph[P] = d.sph_tmp[P];
}

// ---------------------------------------------------------------- cover / uncover
// One block per sphere: cells of the union of its old and new boxes whose coverage by this
// sphere changed are touched (deduplicated into a worklist).
__global__ void cover_touch_kernel(const Dev d) {
    const int P = blockIdx.x;
    if (P >= d.nsph) return;
    const Sphere& s = d.sph[P];
    if (s.x[0] == s.x0[0] && s.x[1] == s.x0[1] && s.x[2] == s.x0[2]) return;
    // a sphere whose centre is not finite or moved more than a cell in one step is left alone
    // (the fluid has gone unstable; the status word says so)
    if (!finite3(s.x) || !finite3(s.x0) || !(s.R > 0.0 && s.R < 64.0)) {
        if (threadIdx.x == 0) atomicOr(&d.sc->status, S_UNSTABLE);
        return;
    }
    const int L[3] = {d.nx, d.ny, d.nz};
    int lo[3], ext[3];
    double off[3];
    for (int k = 0; k < 3; k++) {
        off[k] = min_image(d, k, s.x[k], s.x0[k]);           // new centre relative to the old
        const double a = s.x0[k], b = s.x0[k] + off[k];
        lo[k] = (int)floor(fmin(a, b) - s.R) - 1;
        ext[k] = (int)ceil(fmax(a, b) + s.R) + 1 - lo[k] + 1;
    }
    const int lim = 2 * (int)ceil(s.R) + 8;
    if (ext[0] > lim || ext[1] > lim || ext[2] > lim) {
        if (threadIdx.x == 0) atomicOr(&d.sc->status, S_UNSTABLE);
        return;
    }
    const int total = ext[0] * ext[1] * ext[2];
    const double R2 = s.R * s.R;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        int w[3] = {lo[0] + e % ext[0], lo[1] + (e / ext[0]) % ext[1], lo[2] + e / (ext[0] * ext[1])};
        double d0 = 0, d1 = 0;
        for (int k = 0; k < 3; k++) {
            const double a = (double)w[k] - s.x0[k], b = (double)w[k] - (s.x0[k] + off[k]);
            d0 += a * a;
            d1 += b * b;
        }
        if ((d0 <= R2) == (d1 <= R2)) continue;
        bool ok = true;
        for (int k = 0; k < 3; k++) {
            if (w[k] < 0 || w[k] >= L[k]) {
                if (!d.bc[k]) { ok = false; break; }
                w[k] = ((w[k] % L[k]) + L[k]) % L[k];
            }
        }
        if (!ok) continue;
        const size_t i = cell_index(d, w[0], w[1], w[2]);
        const uint8_t old = mark_or(d.mark, i, K_TOUCH);
        if (!(old & K_TOUCH)) wl_push(d.wl_touch, &d.sc->n_touch, (uint32_t)d.wl_cap, (uint32_t)i, &d.sc->status);
    }
}

// touched cells: the lowest id of the spheres covering them now decides; obstacle cells no
// sphere covers any more are uncovered; newly covered cells lose their fluid mass
template <int S>
__global__ void cover_apply_kernel(const Dev d, const int nxt) {
    using T = typename Store<S>::T;
    const T* f = static_cast<const T*>(d.f[nxt]);
    const uint32_t n = min(*(volatile uint32_t*)&d.sc->n_touch, (uint32_t)d.wl_cap);
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const size_t i = d.wl_touch[k];
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        const uint32_t own = covering_sphere(d, x, y, z);
        const uint8_t t = d.flags[i] & F_TYPE;
        if (t & F_OBS) {
            if (own == kNone) mark_or(d.mark, i, K_UNCOV);
            else d.owner[i] = own;
        } else if (own != kNone) {
            if (t & F_LIQ) {
                float dr = 0.f;
                for (int q = 0; q < kQ; q++) dr += Store<S>::get_nc(f, (size_t)q * d.N + i);
                atomicAdd(&d.sc->S_cover, (double)(1.f + dr));
            } else if (t & F_IF) {
                atomicAdd(&d.sc->S_cover, (double)d.mass[i]);
                atomicSub(&d.sc->n_iface_acc, 1u);
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
__global__ void cover_refill_kernel(const Dev d, const int nxt) {
    using T = typename Store<S>::T;
    T* f = static_cast<T*>(d.f[nxt]);
    float* phi = d.phi[nxt];
    const uint32_t n = min(*(volatile uint32_t*)&d.sc->n_touch, (uint32_t)d.wl_cap);
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const size_t i = d.wl_touch[k];
        if (!(d.mark[i] & K_UNCOV)) continue;
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        int ngas = 0, nfl = 0;
        uint32_t gown = kNone;
        float rs = 0.f, ps = 0.f;
        for (int q = 1; q < kQ; q++) {
            size_t j;
            if (!nbr(d, x, y, z, cx(q), cy(q), cz(q), j)) continue;
            if (d.mark[j] & K_UNCOV) continue;
            const uint8_t t = d.flags[j] & F_TYPE;
            if (t & F_OBS) continue;
            if (t & F_GAS) {
                if (gown == kNone) gown = d.owner[j];
                ngas++;
            } else {
                float r, u[3];
                post_moments<S>(d, f, j, r, u);
                rs += r;
                ps += (t & F_IF) ? phi[j] : 1.f;
                nfl++;
            }
        }
        const uint32_t P = d.owner[i];
        const Sphere& sp = d.sph[P < (uint32_t)d.nsph ? P : 0];
        double r3[3];
        for (int k3 = 0; k3 < 3; k3++) r3[k3] = min_image(d, k3, (double)(k3 == 0 ? x : (k3 == 1 ? y : z)), sp.x[k3]);
        const float uf[3] = {(float)(sp.u[0] + sp.w[1] * r3[2] - sp.w[2] * r3[1]),
                             (float)(sp.u[1] + sp.w[2] * r3[0] - sp.w[0] * r3[2]),
                             (float)(sp.u[2] + sp.w[0] * r3[1] - sp.w[1] * r3[0])};
        if (nfl == 0 && ngas > 0) {
            d.flags[i] = F_GAS;
            d.owner[i] = gown;
            d.mass[i] = 0.f;
            phi[i] = 0.f;
            continue;
        }
        const float rb = nfl ? rs / (float)nfl : 1.f;
        if (ngas > 0) {
            const float pb = ps / (float)nfl;
            d.flags[i] = F_IF;
            d.owner[i] = gown;
            phi[i] = pb;
            d.mass[i] = pb * rb;
            atomicAdd(&d.sc->S_uncover, (double)(pb * rb));
            atomicAdd(&d.sc->n_iface_acc, 1u);
        } else {
            d.flags[i] = F_LIQ;
            d.owner[i] = kNone;
            phi[i] = 1.f;
            d.mass[i] = rb;
            atomicAdd(&d.sc->S_uncover, (double)rb);
        }
        for (int q = 0; q < kQ; q++) Store<S>::put(f, (size_t)q * d.N + i, equilibrium_dev(q, rb, uf));
    }
}

__device__ __forceinline__ void set_bulk_p(const Dev& d, size_t i) {
    uint8_t t = d.flags[i] & F_TYPE;
    bool bulk = t == F_LIQ;
    if (bulk) {
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        for (int q = 1; q < kQ && bulk; q++) {
            size_t j;
            if (!nbr(d, x, y, z, cx(q), cy(q), cz(q), j) || !(d.flags[j] & F_ACTIVE)) bulk = false;
        }
    }
    d.flags[i] = (uint8_t)(t | (bulk ? F_BULK : 0));
}

__global__ void cover_finish_kernel(const Dev d) {
    const uint32_t n = min(*(volatile uint32_t*)&d.sc->n_touch, (uint32_t)d.wl_cap);
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const size_t i = d.wl_touch[k];
        int x, y, z;
        cell_xyz(d, i, x, y, z);
        set_bulk_p(d, i);
        for (int q = 1; q < kQ; q++) {
            size_t j;
            if (nbr(d, x, y, z, cx(q), cy(q), cz(q), j)) set_bulk_p(d, j);
        }
        d.mark[i] = 0;
    }
}

int spheres_launches(const Dev& d) {
    if (d.nsph == 0) return 0;
    int n = 2;  // prepare, contact
    if (d.sphere_mode == LBM_SPHERES_FREE) n += d.n_sub + (d.n_sub & 1);
    else if (d.sphere_mode == LBM_SPHERES_PRESCRIBED) n += 1;
    if (d.sphere_mode != LBM_SPHERES_FIXED) n += 4;
    return n;
}

void launch_spheres(const Dev& d, int nxt, cudaStream_t st) {
    if (d.nsph == 0) return;
    const int tb = 128, nb = (d.nsph + tb - 1) / tb;
    sph_prepare_kernel<<<nb, tb, 0, st>>>(d);
    sph_contact_kernel<<<nb, tb, 0, st>>>(d);
    if (d.sphere_mode == LBM_SPHERES_FREE) {
        const double dt = 1.0 / d.n_sub;
        for (int k = 0; k < d.n_sub; k++) {
            const Sphere* src = (k & 1) ? d.sph_tmp : d.sph;
            Sphere* dst = (k & 1) ? d.sph : d.sph_tmp;
            sph_substep_kernel<<<nb, tb, 0, st>>>(d, src, dst, dt);
        }
        if (d.n_sub & 1) sph_copy_kernel<<<nb, tb, 0, st>>>(d);
    } else if (d.sphere_mode == LBM_SPHERES_PRESCRIBED) {
        sph_prescribed_kernel<<<nb, tb, 0, st>>>(d);
    }
    if (d.sphere_mode == LBM_SPHERES_FIXED) return;
    cover_touch_kernel<<<d.nsph, 128, 0, st>>>(d);
    const int lb = 2 * 152;
    switch (d.storage) {
        case LBM_STORE_F32:
            cover_apply_kernel<LBM_STORE_F32><<<lb, 128, 0, st>>>(d, nxt);
            cover_refill_kernel<LBM_STORE_F32><<<lb, 128, 0, st>>>(d, nxt);
            break;
        case LBM_STORE_F16DEV:
            cover_apply_kernel<LBM_STORE_F16DEV><<<lb, 128, 0, st>>>(d, nxt);
            cover_refill_kernel<LBM_STORE_F16DEV><<<lb, 128, 0, st>>>(d, nxt);
            break;
        default:
            cover_apply_kernel<LBM_STORE_BF16DEV><<<lb, 128, 0, st>>>(d, nxt);
            cover_refill_kernel<LBM_STORE_BF16DEV><<<lb, 128, 0, st>>>(d, nxt);
            break;
    }
    cover_finish_kernel<<<lb, 128, 0, st>>>(d);
}

}  // namespace lbm
