/*
 * fslbm_oracle.c -- plain FP64 CPU oracle of one time step of the liquid-gas-solid
 * free-surface lattice Boltzmann method (Bogner, Harting, Ruede, "Direct simulation of
 * liquid-gas-solid flow with a free surface lattice Boltzmann method", Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement of the
 * method against which the CUDA library is checked.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code, header, constant
 * table or helper with the CUDA library; the only thing both sides share is the seeded
 * workload generator, which holds none of the method's arithmetic.
 *
 * Everything is FP64, single threaded, plain loops, in the order of the step below.
 * Lattice units: dx = dt = 1, c_s^2 = 1/3, cell (x,y,z) centred at integer coordinates,
 * linear index i = x + nx*(y + ny*z), PDF q of cell i at f[q*N + i].
 *
 * One step t -> t+1 (state between steps: post-collision f*(t)):
 *   1. sweep over active cells (liquid, interface): pull streaming (Eq. LBE1) with
 *      halfway bounce-back at walls, moving-wall bounce-back at sphere links (Eq. bbrule)
 *      with momentum exchange (Eqs. netforce, torque, momentum_transfer), free-surface
 *      reconstruction from gas neighbours (Eq. fsk), mass exchange of interface cells
 *      (Eqs. massExchange, massExchangeb), moments, TRT collision (Eq. LBE2) with the
 *      "magic" parameter 3/16 (Eq. latticeViscosity and the relation below it) and a
 *      Guo body force (the paper uses gravity without naming a forcing scheme);
 *   2. cell conversions with layer closure, new-interface initialisation from the
 *      equilibrium and excess-mass redistribution (Sec. 2.2, Fig. cellConversions);
 *   3. sphere update: momentum exchange of links between two spheres, lubrication
 *      correction (Eq. lubrication) and n_substeps Newton-Euler sub-steps (Sec. 2.3);
 *   4. cells covered / uncovered by the moved spheres, refill of uncovered cells;
 *   5. bubble model: per-bubble volume and gas density (Sec. 2.2, last paragraph), on the
 *      cells as the step leaves them, for the next step's reconstruction; touching bubbles
 *      merge, and every split_every steps a bubble in several connected parts splits;
 *   6. curvature from fill levels, Parker-Youngs normals (Sec. 2.2, only if sigma > 0).
 *
 * Parity: pinned by the tests (Poiseuille profile, rest-state invariance, exact per-step
 * mass, momentum and angular-momentum balances, Stokes drag in a periodic array, the
 * Laplace pressure jump, the layer invariant, brute-force comparison with a NumPy
 * transcription on tiny grids, and bubble splitting against a restatement with scipy's
 * connectivity labelling).  The conversion details of step 2 (filling wins, layer closure,
 * new-interface initialisation, excess weights along the normal, equal shares, the pool) and
 * the covering / refill rule of step 4 are pinned against an independent set-form NumPy
 * transcription on random states and against values worked out by hand on a flat interface.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NQ 19
#define ORC_PI 3.14159265358979323846

/* D3Q19 velocity set: 0 rest, 1..6 faces, 7..18 edges; q and q^ (opposite) are (odd, odd+1). */
static const int CX[NQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[NQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[NQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

static double wq(int q) { return q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
static int opp(int q) { return q == 0 ? 0 : ((q & 1) ? q + 1 : q - 1); }

/* cell types (the oracle's own codes) */
enum { C_LIQ = 1, C_IF = 2, C_GAS = 4, C_OBS = 8 };
/* transient marks during conversions / covering */
enum { M_FILLED = 1, M_EMPTIED = 2, M_NEWIF = 4, M_FROMLIQ = 8, M_UNCOV = 16, M_RECV = 32 };

/* sphere record layout, doubles */
enum { S_X = 0, S_U = 3, S_W = 6, S_R = 9, S_RHO = 10, S_F = 11, S_T = 14, S_FLUB = 17, S_FP = 20, S_TP = 23,
       S_HASP = 26, S_LEN = 32 };
/* bubble record layout, doubles */
enum { B_C = 0, B_R = 3, B_V0 = 4, B_V = 5, B_RHOG = 6, B_ROOT = 7, B_MG = 8, B_LEN = 10 };
/* scalar slots */
enum { SC_POOL = 0, SC_NIF = 1, SC_SBB = 2, SC_SCOV = 3, SC_SUNC = 4, SC_STEPS = 5, SC_STATUS = 6, SC_NMERGE = 7,
       SC_NBUB = 8, SC_NSPLIT = 9, SC_LEN = 16 };
/* status bits */
enum { ST_UNSTABLE = 1, ST_BUBBLE_GONE = 2, ST_SPLIT_FULL = 4 };

typedef struct {
    int32_t nx, ny, nz;
    int32_t bc[3];          /* 1: periodic axis; else the faces' kinds below */
    int32_t n_substeps;     /* sphere sub-steps per LBM step (Sec. 2.3: up to 10) */
    int32_t sphere_mode;    /* 0: fixed, 1: free Newton-Euler, 2: prescribed constant velocity */
    int32_t nbub, nsph;
    double tau;             /* tau = -1/lambda_plus */
    double g[3];            /* body force per unit mass (gravity) */
    double sigma;           /* surface tension */
    double rho_g0;          /* initial gas density of every bubble */
    double eps;             /* conversion band: fill >= 1+eps -> liquid, fill <= -eps -> gas */
    double near_tol;        /* band logged as "near a conversion threshold" */
    int32_t face[6];        /* faces -x,+x,-y,+y,-z,+z of non-periodic axes: FACE_* */
    int32_t hydrostatic;    /* 1 (open top only): start in hydrostatic equilibrium */
    int32_t max_bub;        /* rows of the bubble table (>= nbub): room for bubbles made by splitting */
    int32_t split_every;    /* > 0: bubbles split every split_every steps (R39); 0: never */
} orc_params;

/* face kinds (Fig. bubbleSetup): no-slip wall, free-slip wall, open at the reference pressure */
enum { FACE_WALL = 0, FACE_SLIP = 1, FACE_OPEN = 2 };
/* what lies beyond a face for a population pulled across it */
enum { FL_WALL = 0, FL_OPEN = 1, FL_SLIP = 2 };

typedef struct {
    double *f, *ft;         /* [19][N] post-collision PDFs; ft is scratch */
    uint8_t *flag;          /* [N] cell type */
    uint8_t *mark;          /* [N] scratch */
    double *m, *phi, *phit; /* [N] interface mass, fill level, scratch */
    double *kappa;          /* [N] curvature of interface cells */
    int32_t *owner;         /* [N] bubble id (gas / interface) or sphere id (obstacle), -1 none */
    int32_t *nown;          /* [N] scratch */
    int32_t *near;          /* [N] steps at which this interface cell was near a threshold */
    double *bub;            /* [max(nbub, max_bub)][B_LEN]; rows in use: scal[SC_NBUB] */
    double *sph;            /* [nsph][S_LEN] */
    double *scal;           /* [SC_LEN] */
} orc_state;

/* ------------------------------------------------------------------------- helpers */

static long ncell(const orc_params *p) { return (long)p->nx * p->ny * p->nz; }
/* rows of the bubble table; ids at or above scal[SC_NBUB] (one past the highest id ever used)
 * carry no cells */
static int bub_cap(const orc_params *p) { return p->max_bub > p->nbub ? p->max_bub : p->nbub; }

/* neighbour of (x,y,z) displaced by (dx,dy,dz); periodic axes wrap, wall axes give -1 */
static long nbr(const orc_params *p, int x, int y, int z, int dx, int dy, int dz)
{
    int a = x + dx, b = y + dy, c = z + dz;
    if (a < 0 || a >= p->nx) { if (!p->bc[0]) return -1; a = (a + p->nx) % p->nx; }
    if (b < 0 || b >= p->ny) { if (!p->bc[1]) return -1; b = (b + p->ny) % p->ny; }
    if (c < 0 || c >= p->nz) { if (!p->bc[2]) return -1; c = (c + p->nz) % p->nz; }
    return (long)a + (long)p->nx * ((long)b + (long)p->ny * c);
}

/* The population that arrives at cell (x,y,z) in direction q comes from x - c_q; when that
 * lies beyond faces of non-periodic axes: FL_WALL if one of them is a no-slip wall (halfway
 * bounce-back), else FL_OPEN if one is open (the reference pressure), else FL_SLIP: free-slip
 * faces reflect specularly, so the population left the cell *src -- x - c_q moved back across
 * each free-slip face -- in the direction *qs, c_q with those faces' normal components reversed. */
static int face_source(const orc_params *p, int x, int y, int z, int q, long *src, int *qs)
{
    const int c[3] = {CX[q], CY[q], CZ[q]}, L[3] = {p->nx, p->ny, p->nz};
    int a[3] = {x - c[0], y - c[1], z - c[2]}, m[3] = {c[0], c[1], c[2]};
    int wall = 0, open = 0;
    for (int k = 0; k < 3; k++) {
        if (a[k] >= 0 && a[k] < L[k]) continue;
        if (p->bc[k]) { a[k] = (a[k] + L[k]) % L[k]; continue; }
        const int f = p->face[2 * k + (a[k] >= L[k] ? 1 : 0)];
        if (f == FACE_WALL) wall = 1;
        else if (f == FACE_OPEN) open = 1;
        else { a[k] += c[k]; m[k] = -c[k]; }
    }
    if (wall) return FL_WALL;
    if (open) return FL_OPEN;
    *src = (long)a[0] + (long)p->nx * ((long)a[1] + (long)p->ny * a[2]);
    *qs = 0;
    for (int r = 1; r < NQ; r++)
        if (CX[r] == m[0] && CY[r] == m[1] && CZ[r] == m[2]) *qs = r;
    return FL_SLIP;
}

/* d = a - b with the minimum-image convention on periodic axes */
static void mindiff(const orc_params *p, const double a[3], const double b[3], double d[3])
{
    const int L[3] = {p->nx, p->ny, p->nz};
    for (int k = 0; k < 3; k++) {
        d[k] = a[k] - b[k];
        if (p->bc[k]) {
            while (d[k] > 0.5 * L[k]) d[k] -= L[k];
            while (d[k] < -0.5 * L[k]) d[k] += L[k];
        }
    }
}

static void cross(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Eq. equilibrium: e_q(rho,u) = rho w_q (1 + c.u/cs2 + u u:(c c - cs2 I)/(2 cs2^2)) */
static double equi(int q, double rho, const double u[3])
{
    double cu = CX[q] * u[0] + CY[q] * u[1] + CZ[q] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return rho * wq(q) * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

/* even part of the equilibrium, e+_q = (e_q + e_q^)/2 */
static double equi_even(int q, double rho, const double u[3])
{
    double cu = CX[q] * u[0] + CY[q] * u[1] + CZ[q] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return rho * wq(q) * (1.0 + 4.5 * cu * cu - 1.5 * uu);
}

/* density and velocity of a post-collision state: rho = sum f*, u = (sum c f* - rho g/2)/rho.
 * With the Guo force the collision adds rho*g to the first moment, so this u is the
 * velocity the collision used. */
/* density and velocity of cell i's post-collision PDFs f; gw weights the body force the
 * collision applied (the body force acts on the liquid mass: the fill level of an interface
 * cell, 1 for a liquid cell), so the velocity the collision used is (sum c f - rho gw g/2)/rho */
static void post_moments(const orc_params *p, const double *f, long N, long i, double gw, double *rho, double u[3])
{
    double r = 0, j[3] = {0, 0, 0};
    for (int q = 0; q < NQ; q++) {
        double v = f[(long)q * N + i];
        r += v;
        j[0] += CX[q] * v; j[1] += CY[q] * v; j[2] += CZ[q] * v;
    }
    *rho = r;
    for (int k = 0; k < 3; k++) u[k] = (j[k] - 0.5 * r * gw * p->g[k]) / r;
}

/* the force weight of cell i in its current state: its fill level if interface, else 1 */
static double force_weight(const orc_state *s, long i)
{
    return (s->flag[i] & C_IF) ? s->phi[i] : 1.0;
}

static void cell_xyz(const orc_params *p, long i, int *x, int *y, int *z)
{
    *x = (int)(i % p->nx);
    *y = (int)((i / p->nx) % p->ny);
    *z = (int)(i / ((long)p->nx * p->ny));
}

/* fill level as seen by the normal / curvature stencils: interface -> phi, liquid -> 1,
 * gas -> 0, sphere cells and cells beyond a wall -> 1 (perfect wetting, Sec. 2.2). */
static double fill_seen(const orc_params *p, const orc_state *s, int x, int y, int z, int dx, int dy, int dz)
{
    long j = nbr(p, x, y, z, dx, dy, dz);
    if (j < 0) return 1.0;
    uint8_t t = s->flag[j];
    if (t & C_IF) return s->phi[j];
    if (t & C_GAS) return 0.0;
    return 1.0;
}

/* Parker-Youngs gradient of the fill level: central difference smoothed by the
 * [1,2,1] x [1,2,1] / 16 weights over the 3x3x3 block.  Points into the liquid. */
static void py_gradient(const orc_params *p, const orc_state *s, int x, int y, int z, double n[3])
{
    static const double w1[3] = {1.0, 2.0, 1.0};
    n[0] = n[1] = n[2] = 0.0;
    for (int a = -1; a <= 1; a++)
        for (int b = -1; b <= 1; b++) {
            double w = w1[a + 1] * w1[b + 1];
            n[0] += w * (fill_seen(p, s, x, y, z, 1, a, b) - fill_seen(p, s, x, y, z, -1, a, b));
            n[1] += w * (fill_seen(p, s, x, y, z, a, 1, b) - fill_seen(p, s, x, y, z, a, -1, b));
            n[2] += w * (fill_seen(p, s, x, y, z, a, b, 1) - fill_seen(p, s, x, y, z, a, b, -1));
        }
    for (int k = 0; k < 3; k++) n[k] /= 32.0;
}

static void unit_normal(const orc_params *p, const orc_state *s, int x, int y, int z, double nh[3])
{
    double n[3];
    py_gradient(p, s, x, y, z, n);
    double l = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int k = 0; k < 3; k++) nh[k] = l > 0 ? n[k] / l : 0.0;
}

/* ------------------------------------------------------------------ step 4: curvature */

/* kappa = -(1/2) div(n^) (the mean curvature, so that a gas sphere of radius R has
 * kappa = -1/R and p_w = p_g - 2 sigma / R on its liquid side).  Central differences of
 * the unit normal; beyond a wall the cell's own normal is used (one-sided difference). */
static void curvature(const orc_params *p, orc_state *s)
{
    const long N = ncell(p);
    for (long i = 0; i < N; i++) {
        s->kappa[i] = 0.0;
        if (!(s->flag[i] & C_IF)) continue;
        int x, y, z;
        cell_xyz(p, i, &x, &y, &z);
        double n0[3];
        unit_normal(p, s, x, y, z, n0);
        double div = 0.0;
        for (int k = 0; k < 3; k++) {
            int d[3] = {0, 0, 0};
            double np[3], nm[3];
            d[k] = 1;
            if (nbr(p, x, y, z, d[0], d[1], d[2]) >= 0) {
                int a = x + d[0], b = y + d[1], c = z + d[2];
                a = (a + p->nx) % p->nx; b = (b + p->ny) % p->ny; c = (c + p->nz) % p->nz;
                unit_normal(p, s, a, b, c, np);
            } else {
                memcpy(np, n0, sizeof np);
            }
            d[k] = -1;
            if (nbr(p, x, y, z, d[0], d[1], d[2]) >= 0) {
                int a = x + d[0], b = y + d[1], c = z + d[2];
                a = (a + p->nx) % p->nx; b = (b + p->ny) % p->ny; c = (c + p->nz) % p->nz;
                unit_normal(p, s, a, b, c, nm);
            } else {
                memcpy(nm, n0, sizeof nm);
            }
            div += 0.5 * (np[k] - nm[k]);
        }
        s->kappa[i] = -0.5 * div;
    }
}

/* ---------------------------------------------------------------- step 3: bubble model */

/* A bubble is a connected gas region (Sec. 2.2).  Every gas or interface cell carries the id
 * of the bubble it was created in; when the regions of two bubbles touch (a gas or interface
 * cell next to one of another bubble) they are one bubble from then on: the ids are joined,
 * the smaller id being the root of the merged bubble.  The merged bubble's gas mass is the sum
 * of the two, and so is its reference volume; its volume is the sum of its members' volumes.
 * With split_every > 0, every split_every steps a bubble whose gas and interface cells form
 * several connected parts (the same D3Q19 adjacency that merges two bubbles) is split
 * (split_bubbles below).
 *
 * V = #gas cells + sum over the interface cells of (1 - phi) of all ids of the bubble;
 * isothermal ideal gas of conserved mass m_g: rho_g = m_g / V, m_g = rho_g(0) V(0).  Every id
 * of a merged bubble holds the merged bubble's V0, V and rho_g. */
static int bubble_root(const orc_state *s, int b)
{
    while ((int)s->bub[b * B_LEN + B_ROOT] != b) b = (int)s->bub[b * B_LEN + B_ROOT];
    return b;
}

static void split_bubbles(const orc_params *p, orc_state *s);

static void bubble_model(const orc_params *p, orc_state *s, int set_reference, int split)
{
    const long N = ncell(p);
    const int nb = bub_cap(p);
    if (nb <= 0) {
        long nif = 0;
        for (long i = 0; i < N; i++) nif += (s->flag[i] & C_IF) != 0;
        s->scal[SC_NIF] = (double)nif;
        return;
    }
    double *own = calloc((size_t)nb, sizeof(double));   /* volume of the cells carrying id b */
    double *Vr = calloc((size_t)nb, sizeof(double));    /* volume of the bubble rooted at b */
    long nif = 0;
    for (long i = 0; i < N; i++) {
        uint8_t t = s->flag[i];
        int b = s->owner[i];
        if (t & C_IF) {
            nif++;
            if (b >= 0 && b < nb) own[b] += 1.0 - s->phi[i];
        } else if (t & C_GAS) {
            if (b >= 0 && b < nb) own[b] += 1.0;
        }
    }
    s->scal[SC_NIF] = (double)nif;
    if (set_reference)   /* the initial gas density of each bubble is in B_RHOG */
        for (int b = 0; b < nb; b++) {
            s->bub[b * B_LEN + B_V0] = own[b];
            s->bub[b * B_LEN + B_MG] = s->bub[b * B_LEN + B_RHOG] * own[b];
        }
    for (int z = 0; z < p->nz; z++)
        for (int y = 0; y < p->ny; y++)
            for (int x = 0; x < p->nx; x++) {
                const long i = (long)x + (long)p->nx * ((long)y + (long)p->ny * z);
                const int b = s->owner[i];
                if (!(s->flag[i] & (C_IF | C_GAS)) || b < 0 || b >= nb) continue;
                for (int q = 1; q < NQ; q++) {
                    const long j = nbr(p, x, y, z, CX[q], CY[q], CZ[q]);
                    if (j < 0 || !(s->flag[j] & (C_IF | C_GAS))) continue;
                    const int bj = s->owner[j];
                    if (bj < 0 || bj >= nb) continue;
                    const int ra = bubble_root(s, b), rb = bubble_root(s, bj);
                    if (ra == rb) continue;
                    const int lo = ra < rb ? ra : rb, hi = ra < rb ? rb : ra;
                    s->bub[hi * B_LEN + B_ROOT] = (double)lo;
                    s->bub[lo * B_LEN + B_V0] += s->bub[hi * B_LEN + B_V0];
                    s->bub[lo * B_LEN + B_MG] += s->bub[hi * B_LEN + B_MG];
                    s->scal[SC_NMERGE] += 1.0;
                }
            }
    for (int b = 0; b < nb; b++) Vr[bubble_root(s, b)] += own[b];
    for (int b = 0; b < nb; b++) {
        double *B = s->bub + b * B_LEN;
        const int r = bubble_root(s, b);
        B[B_V0] = s->bub[r * B_LEN + B_V0];
        B[B_MG] = s->bub[r * B_LEN + B_MG];
        B[B_V] = Vr[r];
        if (Vr[r] > 0.0) {
            B[B_RHOG] = B[B_MG] / Vr[r];
        } else if (B[B_MG] > 0.0) {   /* (a free record holds no gas) */
            s->scal[SC_STATUS] = (double)((int)s->scal[SC_STATUS] | ST_BUBBLE_GONE);
        }
    }
    free(own);
    free(Vr);
    if (split) split_bubbles(p, s);
}

/* R39, splitting (the inverse of the merge above).  First every gas and interface cell takes
 * the id of its bubble's root, so that a bubble carries one id; the ids then left without a
 * cell are free (their records reset).  The cells of each bubble are grouped into connected
 * parts: two cells are in the same part when they are D3Q19 neighbours (or are linked through
 * a chain of such neighbours).  A part is found from its lowest cell index (scanning cells in
 * index order), its volume V_c = #gas cells + sum of (1 - phi) over its interface cells.  If a
 * bubble has several parts, the largest keeps the id (volumes equal to within 1e-9 of each
 * other count as a tie, which goes to the part with the lower lowest index: a sum's rounding
 * depends on its order) and every other part, in the order of their lowest indices, becomes a new
 * bubble with the lowest free id (bubbles taken in increasing id order); its cells take that
 * id.  Gas mass and reference volume are
 * divided in proportion to the parts' volumes, so every part leaves with the gas density of
 * the whole.  A part of zero volume (interface cells that are full) stays with its bubble, and
 * so does a part for which no free id is left (the status says so). */
typedef struct { long rep; int root; double V; } orc_part;

static void split_bubbles(const orc_params *p, orc_state *s)
{
    const long N = ncell(p);
    const int cap = bub_cap(p);
    int32_t *part = s->nown;   /* scratch: the part of each gas / interface cell, -1 elsewhere */
    long *stack = malloc(sizeof(long) * (size_t)N);
    int *root = malloc(sizeof(int) * (size_t)cap), *used = calloc((size_t)cap, sizeof(int));
    long nparts = 0, cparts = 64;
    orc_part *P = malloc(sizeof(orc_part) * (size_t)cparts);
    /* one id per bubble; ids without a cell are free */
    for (int b = 0; b < cap; b++) root[b] = bubble_root(s, b);
    for (long i = 0; i < N; i++) {
        const int b = s->owner[i];
        if (!(s->flag[i] & (C_IF | C_GAS)) || b < 0 || b >= cap) continue;
        s->owner[i] = root[b];
        used[root[b]] = 1;
    }
    for (int b = 0; b < cap; b++) {
        if (used[b]) continue;
        double *B = s->bub + (long)b * B_LEN;
        for (int k = 0; k < B_LEN; k++) B[k] = 0.0;
        B[B_ROOT] = (double)b;
        B[B_RHOG] = p->rho_g0;
    }
    for (long i = 0; i < N; i++) part[i] = -1;
    for (long i0 = 0; i0 < N; i0++) {
        const int r = s->owner[i0];
        if (!(s->flag[i0] & (C_IF | C_GAS)) || r < 0 || r >= cap || part[i0] >= 0) continue;
        if (nparts == cparts) {
            cparts *= 2;
            P = realloc(P, sizeof(orc_part) * (size_t)cparts);
        }
        P[nparts].rep = i0;
        P[nparts].root = r;
        P[nparts].V = 0.0;
        long top = 0;
        stack[top++] = i0;
        part[i0] = (int32_t)nparts;
        while (top > 0) {   /* depth-first over the part */
            const long i = stack[--top];
            P[nparts].V += (s->flag[i] & C_GAS) ? 1.0 : 1.0 - s->phi[i];
            int x, y, z;
            cell_xyz(p, i, &x, &y, &z);
            for (int q = 1; q < NQ; q++) {
                const long j = nbr(p, x, y, z, CX[q], CY[q], CZ[q]);
                if (j < 0 || part[j] >= 0 || !(s->flag[j] & (C_IF | C_GAS)) || s->owner[j] != r) continue;
                part[j] = (int32_t)nparts;
                stack[top++] = j;
            }
        }
        nparts++;
    }
    int *newid = malloc(sizeof(int) * (size_t)(nparts > 0 ? nparts : 1));
    for (long c = 0; c < nparts; c++) newid[c] = -1;
    int next_free = 0;
    for (int r = 0; r < cap; r++) {   /* bubbles in increasing id order */
        long c = -1;   /* r's first part */
        for (long e = 0; e < nparts && c < 0; e++)
            if (P[e].root == r) c = e;
        if (c < 0) continue;
        long keep = c;
        double Vr = 0.0;
        int count = 0;
        for (long e = c; e < nparts; e++) {
            if (P[e].root != r) continue;
            count++;
            Vr += P[e].V;
            if (P[e].V > P[keep].V * (1.0 + 1e-9)) keep = e;   /* (equal to 1e-9: lower index) */
        }
        if (count < 2 || !(Vr > 0.0)) continue;
        double *R = s->bub + (long)r * B_LEN;
        const double V0r = R[B_V0], mgr = R[B_MG];
        double kept_share = 1.0;
        for (long e = c; e < nparts; e++) {
            if (P[e].root != r || e == keep || !(P[e].V > 0.0)) continue;
            while (next_free < cap && used[next_free]) next_free++;
            if (next_free >= cap) {
                s->scal[SC_STATUS] = (double)((int)s->scal[SC_STATUS] | ST_SPLIT_FULL);
                continue;
            }
            const int id = next_free;
            used[id] = 1;
            const double a = P[e].V / Vr;
            double *F = s->bub + (long)id * B_LEN;
            F[B_ROOT] = (double)id;
            F[B_V0] = V0r * a;
            F[B_MG] = mgr * a;
            F[B_V] = P[e].V;
            F[B_RHOG] = F[B_MG] / F[B_V];
            newid[e] = id;
            kept_share -= a;
            if (id + 1 > (int)s->scal[SC_NBUB]) s->scal[SC_NBUB] = (double)(id + 1);
            s->scal[SC_NSPLIT] += 1.0;
        }
        R[B_V0] = V0r * kept_share;
        R[B_MG] = mgr * kept_share;
        R[B_V] = Vr * kept_share;
        if (R[B_V] > 0.0) R[B_RHOG] = R[B_MG] / R[B_V];
    }
    for (long i = 0; i < N; i++)
        if (part[i] >= 0 && newid[part[i]] >= 0) s->owner[i] = newid[part[i]];
    free(newid);
    free(P);
    free(used);
    free(root);
    free(stack);
}

/* ------------------------------------------------------------------ step 1: the sweep */

/* The gas presses on the part of a sphere's surface it touches (the links of the sweep come
 * from liquid and interface cells only, and the uniform part of their momentum exchange, the
 * reference pressure, cancels only over a closed surface): a gas cell y beside an obstacle cell
 * of sphere a (y - c_q covered by a) transfers the momentum of the gas at rest into a, as a
 * link from y would: dj = -2 w_q rho_g c_q, rho_g of y's bubble (p = rho / 3), arm y - x_a. */
static void gas_on_spheres(const orc_params *p, orc_state *s, int x, int y, int z, long i)
{
    const int b = s->owner[i];
    const double rg = (b >= 0 && b < bub_cap(p)) ? s->bub[(long)b * B_LEN + B_RHOG] : p->rho_g0;
    const double xc[3] = {(double)x, (double)y, (double)z};
    for (int q = 1; q < NQ; q++) {
        const long src = nbr(p, x, y, z, -CX[q], -CY[q], -CZ[q]);
        if (src < 0 || !(s->flag[src] & C_OBS)) continue;
        double *S = s->sph + (long)s->owner[src] * S_LEN;
        const double a = 2.0 * wq(q) * rg;
        double dj[3] = {-a * CX[q], -a * CY[q], -a * CZ[q]}, r[3], rxj[3];
        mindiff(p, xc, S + S_X, r);
        cross(r, dj, rxj);
        for (int k = 0; k < 3; k++) {
            S[S_F + k] += dj[k];
            S[S_T + k] += rxj[k];
        }
    }
}

static void sweep(const orc_params *p, orc_state *s, double share)
{
    const long N = ncell(p);
    const double lp = -1.0 / p->tau;                                  /* lambda_+ */
    const double lm = 1.0 / ((3.0 / 16.0) / (1.0 / lp + 0.5) - 0.5);  /* lambda_- from Lambda = 3/16 */
    for (int z = 0; z < p->nz; z++)
        for (int y = 0; y < p->ny; y++)
            for (int x = 0; x < p->nx; x++) {
                const long i = (long)x + (long)p->nx * ((long)y + (long)p->ny * z);
                const uint8_t t = s->flag[i];
                if ((t & C_GAS) && p->nsph > 0) gas_on_spheres(p, s, x, y, z, i);
                if (!(t & (C_LIQ | C_IF))) continue;
                double fo[NQ], fin[NQ];
                for (int q = 0; q < NQ; q++) fo[q] = s->f[(long)q * N + i];
                double rho0, u0[3];
                post_moments(p, s->f, N, i, force_weight(s, i), &rho0, u0);
                const double xc[3] = {(double)x, (double)y, (double)z};

                for (int q = 0; q < NQ; q++) {
                    long src = nbr(p, x, y, z, -CX[q], -CY[q], -CZ[q]);
                    int qs = q;
                    if (src < 0) {
                        const int kind = face_source(p, x, y, z, q, &src, &qs);
                        if (kind == FL_WALL) {           /* no-slip wall: halfway bounce-back */
                            fin[q] = fo[opp(q)];
                            continue;
                        }
                        if (kind == FL_OPEN) {           /* open face: Eq. fsk with rho_w = 1 */
                            fin[q] = -fo[opp(q)] + 2.0 * equi_even(q, 1.0, u0);
                            s->scal[SC_SBB] += fin[q] - fo[opp(q)];
                            continue;
                        }
                    }
                    const uint8_t ts = s->flag[src];
                    if (ts & (C_LIQ | C_IF)) {           /* Eq. LBE1 (specular: direction qs) */
                        fin[q] = s->f[(long)qs * N + src];
                    } else if (ts & C_OBS) {             /* Eq. bbrule at the link midpoint */
                        double *S = s->sph + (long)s->owner[src] * S_LEN;
                        const double cq[3] = {CX[q], CY[q], CZ[q]};
                        double xw[3] = {xc[0] - 0.5 * cq[0], xc[1] - 0.5 * cq[1], xc[2] - 0.5 * cq[2]};
                        double d[3], wxd[3], uw[3];
                        mindiff(p, xw, S + S_X, d);
                        cross(S + S_W, d, wxd);
                        for (int k = 0; k < 3; k++) uw[k] = S[S_U + k] + wxd[k];
                        const double cu = cq[0] * uw[0] + cq[1] * uw[1] + cq[2] * uw[2];
                        /* f_q(x,t+1) = f*_q^(x,t) - 2 e-_q^(rho_w,u_w), e-_q^ = -3 w rho c_q.u */
                        fin[q] = fo[opp(q)] + 6.0 * wq(q) * rho0 * cu;
                        /* Eq. momentum_transfer along the link x -> particle (direction q^):
                         * dj = c_q^ f*_q^(x,t) - c_q f_q(x,t+1) */
                        double a = fo[opp(q)] + fin[q], dj[3], r[3], rxj[3];
                        for (int k = 0; k < 3; k++) dj[k] = -cq[k] * a;
                        mindiff(p, xc, S + S_X, r);
                        cross(r, dj, rxj);
                        for (int k = 0; k < 3; k++) {
                            S[S_F + k] += dj[k];
                            S[S_T + k] += rxj[k];
                        }
                        if (t & C_LIQ) s->scal[SC_SBB] += 6.0 * wq(q) * rho0 * cu;
                    } else {                             /* gas: Eq. fsk */
                        const int b = s->owner[src];
                        const double rg = (b >= 0 && b < bub_cap(p)) ? s->bub[(long)b * B_LEN + B_RHOG] : p->rho_g0;
                        const double rw = rg + 6.0 * p->sigma * s->kappa[i];
                        fin[q] = -fo[opp(q)] + 2.0 * equi_even(q, rw, u0);
                    }
                }

                double mnew = 0.0;
                if (t & C_IF) {                          /* Eqs. massExchange, massExchangeb */
                    double dm = 0.0;
                    for (int q = 1; q < NQ; q++) {
                        long nb = nbr(p, x, y, z, CX[q], CY[q], CZ[q]);
                        int qn = opp(q);   /* the direction the exchanged population arrives in */
                        if (nb < 0) {
                            const int kind = face_source(p, x, y, z, opp(q), &nb, &qn);
                            if (kind == FL_WALL) continue;
                            if (kind == FL_OPEN) {   /* what the open face lets in: as from a liquid cell */
                                dm += fin[opp(q)] - fo[q];
                                continue;
                            }
                        }
                        const uint8_t tn = s->flag[nb];
                        const double ex = s->f[(long)qn * N + nb] - fo[q];
                        if (tn & C_LIQ) dm += ex;
                        else if (tn & C_IF) dm += 0.5 * (s->phi[i] + s->phi[nb]) * ex;
                    }
                    mnew = (s->m[i] + share) + dm;
                }

                /* moments with the Guo half-force shift, then TRT collision (Eq. LBE2) */
                double rho = 0, j[3] = {0, 0, 0};
                for (int q = 0; q < NQ; q++) {
                    rho += fin[q];
                    j[0] += CX[q] * fin[q]; j[1] += CY[q] * fin[q]; j[2] += CZ[q] * fin[q];
                }
                /* the body force acts on the liquid mass: rho g, or phi rho g in an interface cell
                 * (its fill level after this step's mass exchange) */
                const double gw = (t & C_IF) ? mnew / rho : 1.0;
                const double g[3] = {gw * p->g[0], gw * p->g[1], gw * p->g[2]};
                double u[3];
                for (int k = 0; k < 3; k++) u[k] = (j[k] + 0.5 * rho * g[k]) / rho;
                const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                const double ug = u[0] * g[0] + u[1] * g[1] + u[2] * g[2];
                for (int q = 0; q < NQ; q++) {
                    const int qb = opp(q);
                    const double cu = CX[q] * u[0] + CY[q] * u[1] + CZ[q] * u[2];
                    const double cg = CX[q] * g[0] + CY[q] * g[1] + CZ[q] * g[2];
                    const double ep = wq(q) * rho * (1.0 + 4.5 * cu * cu - 1.5 * uu);
                    const double em = wq(q) * rho * 3.0 * cu;
                    const double fp = 0.5 * (fin[q] + fin[qb]);
                    const double fm = 0.5 * (fin[q] - fin[qb]);
                    const double Gp = wq(q) * rho * (9.0 * cu * cg - 3.0 * ug);
                    const double Gm = wq(q) * rho * 3.0 * cg;
                    s->ft[(long)q * N + i] = fin[q] + lp * (fp - ep) + lm * (fm - em)
                                           + (1.0 + 0.5 * lp) * Gp + (1.0 + 0.5 * lm) * Gm;
                }
                if (!(rho > 0.0) || rho != rho)
                    s->scal[SC_STATUS] = (double)((int)s->scal[SC_STATUS] | ST_UNSTABLE);
                if (t & C_IF) {
                    s->m[i] = mnew;
                    s->phit[i] = mnew / rho;
                }
            }
    for (long i = 0; i < N; i++)
        if (s->flag[i] & C_IF) s->phi[i] = s->phit[i];
}

/* ---------------------------------------------------------------- step 2: conversions */

static void conversions(const orc_params *p, orc_state *s)
{
    const long N = ncell(p);
    double *F = s->ft;  /* f*(t+1) */
    memset(s->mark, 0, (size_t)N);

    /* (i) interface cells past a threshold; log cells near one.  An interface cell is a
     * boundary cell of the liquid with a gas neighbour (Sec. 2.2): one left without any gas
     * neighbour is liquid now, whatever its fill level (filled, its mass m - rho the excess) */
    for (long i = 0; i < N; i++) {
        if (!(s->flag[i] & C_IF)) continue;
        const double ph = s->phi[i];
        if (fabs(ph - 1.0) <= p->near_tol || fabs(ph) <= p->near_tol) s->near[i]++;
        int x, y, z, gas = 0;
        cell_xyz(p, i, &x, &y, &z);
        for (int q = 1; q < NQ; q++) {
            const long j = nbr(p, x, y, z, CX[q], CY[q], CZ[q]);
            if (j >= 0 && (s->flag[j] & C_GAS)) gas = 1;
        }
        if (!gas) s->mark[i] = M_FILLED;
        else if (ph >= 1.0 + p->eps) s->mark[i] = M_FILLED;
        else if (ph <= -p->eps) s->mark[i] = M_EMPTIED;
    }
    /* (ii) filled cells: gas neighbours become interface, emptied neighbours stay interface */
    for (long i = 0; i < N; i++) {
        if (!(s->mark[i] & M_FILLED)) continue;
        int x, y, z;
        cell_xyz(p, i, &x, &y, &z);
        for (int q = 1; q < NQ; q++) {
            long j = nbr(p, x, y, z, CX[q], CY[q], CZ[q]);
            if (j < 0) continue;
            if (s->flag[j] & C_GAS) s->mark[j] |= M_NEWIF;
            if (s->mark[j] & M_EMPTIED) s->mark[j] &= (uint8_t)~M_EMPTIED;
        }
    }
    /* (iii) emptied cells: liquid neighbours become interface with m = rho */
    for (long i = 0; i < N; i++) {
        if (!(s->mark[i] & M_EMPTIED)) continue;
        int x, y, z;
        cell_xyz(p, i, &x, &y, &z);
        for (int q = 1; q < NQ; q++) {
            long j = nbr(p, x, y, z, CX[q], CY[q], CZ[q]);
            if (j < 0 || !(s->flag[j] & C_LIQ)) continue;
            if (!(s->mark[j] & M_FROMLIQ)) {
                double r, u[3];
                post_moments(p, F, N, j, force_weight(s, j), &r, u);
                s->mark[j] |= M_FROMLIQ;
                s->m[j] = r;
                s->owner[j] = s->owner[i];
            } else if (s->owner[i] >= 0 && (s->owner[j] < 0 || s->owner[i] < s->owner[j])) {
                s->owner[j] = s->owner[i];
            }
        }
    }
    /* (iv) new interface cells from gas: equilibrium of the mean density and velocity of
     * neighbours that carry PDFs (liquid, interface not emptied, filled) */
    for (long i = 0; i < N; i++) {
        if (!(s->mark[i] & M_NEWIF)) continue;
        int x, y, z;
        cell_xyz(p, i, &x, &y, &z);
        double rs = 0, us[3] = {0, 0, 0};
        int n = 0;
        for (int q = 1; q < NQ; q++) {
            long j = nbr(p, x, y, z, CX[q], CY[q], CZ[q]);
            if (j < 0 || !(s->flag[j] & (C_LIQ | C_IF)) || (s->mark[j] & M_EMPTIED)) continue;
            double r, u[3];
            post_moments(p, F, N, j, force_weight(s, j), &r, u);
            rs += r;
            for (int k = 0; k < 3; k++) us[k] += u[k];
            n++;
        }
        double rb = n ? rs / n : 1.0, ub[3];
        for (int k = 0; k < 3; k++) ub[k] = n ? us[k] / n : 0.0;
        for (int q = 0; q < NQ; q++) F[(long)q * N + i] = equi(q, rb, ub);
        s->m[i] = 0.0;
    }
    /* (v) excess mass of converting cells to the neighbours that will be interface cells,
     * weighted by the interface normal pointing into the gas (n_g = -grad phi):
     * filled -> max(0, n_g.c_q), emptied -> max(0, -n_g.c_q); uniform if all weights vanish;
     * into the global pool if there is no such neighbour.  The normal sees the fill levels
     * and cell types of the sweep result, before any conversion. */
    for (long i = 0; i < N; i++) {
        const uint8_t mk = s->mark[i];
        if (!(mk & (M_FILLED | M_EMPTIED))) continue;
        int x, y, z;
        cell_xyz(p, i, &x, &y, &z);
        double ng[3];
        py_gradient(p, s, x, y, z, ng);
        for (int k = 0; k < 3; k++) ng[k] = -ng[k];
        double r, u[3];
        post_moments(p, F, N, i, force_weight(s, i), &r, u);
        double mex;
        if (mk & M_FILLED) { mex = s->m[i] - r; s->m[i] = r; }
        else { mex = s->m[i]; s->m[i] = 0.0; }
        long rec[NQ];
        double wr[NQ], W = 0.0;
        int nr = 0;
        for (int q = 1; q < NQ; q++) {
            long j = nbr(p, x, y, z, CX[q], CY[q], CZ[q]);
            if (j < 0) continue;
            const uint8_t mj = s->mark[j];
            const int is_rec = ((s->flag[j] & C_IF) && !(mj & (M_FILLED | M_EMPTIED))) ||
                               (mj & (M_NEWIF | M_FROMLIQ));
            if (!is_rec) continue;
            double nc = ng[0] * CX[q] + ng[1] * CY[q] + ng[2] * CZ[q];
            double w = (mk & M_FILLED) ? (nc > 0 ? nc : 0.0) : (nc < 0 ? -nc : 0.0);
            rec[nr] = j;
            wr[nr] = w;
            W += w;
            nr++;
        }
        if (nr == 0) {
            s->scal[SC_POOL] += mex;
            continue;
        }
        for (int k = 0; k < nr; k++) {
            s->m[rec[k]] += W > 0.0 ? mex * (wr[k] / W) : mex / nr;
            s->mark[rec[k]] |= M_RECV;
        }
    }
    /* (vi) finalise types; fill level of every interface cell whose mass changed here */
    for (long i = 0; i < N; i++) {
        const uint8_t mk = s->mark[i];
        if (!mk) continue;
        if (mk & M_FILLED) { s->flag[i] = C_LIQ; s->owner[i] = -1; }
        else if (mk & M_EMPTIED) { s->flag[i] = C_GAS; }
        else if (mk & (M_NEWIF | M_FROMLIQ)) { s->flag[i] = C_IF; }
    }
    for (long i = 0; i < N; i++) {
        const uint8_t mk = s->mark[i];
        if (!(mk & (M_NEWIF | M_FROMLIQ | M_RECV)) || !(s->flag[i] & C_IF)) continue;
        double r, u[3];
        post_moments(p, F, N, i, force_weight(s, i), &r, u);
        s->phi[i] = s->m[i] / r;
    }
}

/* --------------------------------------------------------------- step 5: the spheres */

static double sphere_mass(const double *S) { return S[S_RHO] * 4.0 / 3.0 * ORC_PI * S[S_R] * S[S_R] * S[S_R]; }

static int covers(const orc_params *p, const double *S, int x, int y, int z)
{
    const double xc[3] = {(double)x, (double)y, (double)z};
    double d[3];
    mindiff(p, xc, S + S_X, d);
    return d[0] * d[0] + d[1] * d[1] + d[2] * d[2] <= S[S_R] * S[S_R];
}

/* Links between obstacle nodes of two different spheres: the node inside sphere P' is
 * given the equilibrium e_q(1, u_P'(x)) of its own sphere's surface velocity (Sec. 2.3,
 * end of the momentum-exchange paragraph), reflected by Eq. bbrule with rho_w = 1. */
static void contact_links(const orc_params *p, orc_state *s)
{
    const long N = ncell(p);
    for (long i = 0; i < N; i++) {
        if (!(s->flag[i] & C_OBS)) continue;
        int x, y, z;
        cell_xyz(p, i, &x, &y, &z);
        const double xc[3] = {(double)x, (double)y, (double)z};
        const double *Sp = s->sph + (long)s->owner[i] * S_LEN;
        for (int q = 1; q < NQ; q++) {
            long j = nbr(p, x, y, z, CX[q], CY[q], CZ[q]);
            if (j < 0 || !(s->flag[j] & C_OBS) || s->owner[j] == s->owner[i]) continue;
            double *S = s->sph + (long)s->owner[j] * S_LEN;
            const double cq[3] = {CX[q], CY[q], CZ[q]};
            double d[3], wxd[3], us[3], uw[3];
            mindiff(p, xc, Sp + S_X, d);
            cross(Sp + S_W, d, wxd);
            for (int k = 0; k < 3; k++) us[k] = Sp[S_U + k] + wxd[k];
            const double fstar = equi(q, 1.0, us);
            double xw[3] = {xc[0] + 0.5 * cq[0], xc[1] + 0.5 * cq[1], xc[2] + 0.5 * cq[2]};
            mindiff(p, xw, S + S_X, d);
            cross(S + S_W, d, wxd);
            for (int k = 0; k < 3; k++) uw[k] = S[S_U + k] + wxd[k];
            const double cu = cq[0] * uw[0] + cq[1] * uw[1] + cq[2] * uw[2];
            const double fback = fstar - 6.0 * wq(q) * 1.0 * cu;
            double dj[3], r[3], rxj[3];
            for (int k = 0; k < 3; k++) dj[k] = cq[k] * (fstar + fback);
            mindiff(p, xc, S + S_X, r);
            cross(r, dj, rxj);
            for (int k = 0; k < 3; k++) {
                S[S_F + k] += dj[k];
                S[S_T + k] += rxj[k];
            }
        }
    }
}

/* Eq. lubrication for every pair with gap < Delta_c = 2/3, gap floored at 0.2 Delta_c,
 * mu = rho nu with rho = 1; +F on the first sphere, -F on the second. */
static void lubrication(const orc_params *p, orc_state *s, double *Fl)
{
    const double dc = 2.0 / 3.0, mu = (p->tau - 0.5) / 3.0;
    for (long a = 0; a < 3L * p->nsph; a++) Fl[a] = 0.0;
    for (int a = 0; a < p->nsph; a++)
        for (int b = a + 1; b < p->nsph; b++) {
            const double *A = s->sph + (long)a * S_LEN, *B = s->sph + (long)b * S_LEN;
            double d[3];
            mindiff(p, B + S_X, A + S_X, d);  /* x_12 = x_2 - x_1 */
            const double dist = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double h = dist - A[S_R] - B[S_R];
            if (!(h < dc) || dist <= 0.0) continue;
            if (h < 0.2 * dc) h = 0.2 * dc;
            const double rr = A[S_R] * B[S_R], rs = A[S_R] + B[S_R];
            double n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
            const double vn = n[0] * (A[S_U] - B[S_U]) + n[1] * (A[S_U + 1] - B[S_U + 1]) + n[2] * (A[S_U + 2] - B[S_U + 2]);
            const double mag = -6.0 * ORC_PI * mu * rr * rr / (rs * rs) * (1.0 / h - 1.0 / dc) * vn;
            for (int k = 0; k < 3; k++) {
                Fl[3 * a + k] += mag * n[k];
                Fl[3 * b + k] -= mag * n[k];
            }
        }
}

static void wrap_position(const orc_params *p, double *X)
{
    const int L[3] = {p->nx, p->ny, p->nz};
    for (int k = 0; k < 3; k++)
        if (p->bc[k]) {
            while (X[k] >= L[k] - 0.5) X[k] -= L[k];
            while (X[k] < -0.5) X[k] += L[k];
        }
}

/* Newton-Euler in n_substeps semi-implicit Euler sub-steps: the hydrodynamic force and
 * torque are held over the LBM step, lubrication and gravity are re-evaluated each sub-step.
 * The hydrodynamic force and torque used are the mean of the momentum exchange of this step
 * and of the previous one (Ladd 1994): the explicit coupling of Sec. 2.3 otherwise lets a
 * two-step oscillation of light spheres (density 1.5 - 2) grow from round-off; on the first
 * step of a sphere the current values are used alone. */
static void move_spheres(const orc_params *p, orc_state *s)
{
    if (p->nsph == 0) return;
    if (p->sphere_mode == 2) {
        for (int a = 0; a < p->nsph; a++) {
            double *S = s->sph + (long)a * S_LEN;
            for (int k = 0; k < 3; k++) S[S_X + k] += S[S_U + k];
            wrap_position(p, S + S_X);
        }
        return;
    }
    if (p->sphere_mode != 1) return;
    double *Fl = (double *)calloc((size_t)3 * p->nsph, sizeof(double));
    const double dt = 1.0 / p->n_substeps;
    for (int sub = 0; sub < p->n_substeps; sub++) {
        lubrication(p, s, Fl);
        for (int a = 0; a < p->nsph; a++) {
            double *S = s->sph + (long)a * S_LEN;
            const double mp = sphere_mass(S), I = 0.4 * mp * S[S_R] * S[S_R];
            const int hasp = S[S_HASP] != 0.0;
            for (int k = 0; k < 3; k++) {
                const double Fh = hasp ? 0.5 * (S[S_F + k] + S[S_FP + k]) : S[S_F + k];
                const double Th = hasp ? 0.5 * (S[S_T + k] + S[S_TP + k]) : S[S_T + k];
                S[S_FLUB + k] = Fl[3 * a + k];
                S[S_U + k] += dt * (Fh + Fl[3 * a + k] + mp * p->g[k]) / mp;
                S[S_W + k] += dt * Th / I;
            }
            for (int k = 0; k < 3; k++) S[S_X + k] += dt * S[S_U + k];
            wrap_position(p, S + S_X);
        }
    }
    free(Fl);
}

/* ---------------------------------------------------- step 6: cover / uncover, refill */

static void box_range(const orc_params *p, const double *S, int k, int *lo, int *hi)
{
    const int L[3] = {p->nx, p->ny, p->nz};
    *lo = (int)floor(S[S_X + k] - S[S_R]) - 1;
    *hi = (int)ceil(S[S_X + k] + S[S_R]) + 1;
    if (!p->bc[k]) {
        if (*lo < 0) *lo = 0;
        if (*hi > L[k] - 1) *hi = L[k] - 1;
    }
}

static void cover_uncover(const orc_params *p, orc_state *s)
{
    const long N = ncell(p);
    for (long i = 0; i < N; i++) s->nown[i] = -1;
    for (int a = 0; a < p->nsph; a++) {
        const double *S = s->sph + (long)a * S_LEN;
        int lo[3], hi[3];
        for (int k = 0; k < 3; k++) box_range(p, S, k, lo + k, hi + k);
        for (int zz = lo[2]; zz <= hi[2]; zz++)
            for (int yy = lo[1]; yy <= hi[1]; yy++)
                for (int xx = lo[0]; xx <= hi[0]; xx++) {
                    int x = (xx % p->nx + p->nx) % p->nx, y = (yy % p->ny + p->ny) % p->ny, z = (zz % p->nz + p->nz) % p->nz;
                    long i = (long)x + (long)p->nx * ((long)y + (long)p->ny * z);
                    if (s->nown[i] < 0 && covers(p, S, x, y, z)) s->nown[i] = a;
                }
    }
    memset(s->mark, 0, (size_t)N);
    for (long i = 0; i < N; i++) {
        if (s->flag[i] & C_OBS) {
            if (s->nown[i] < 0) s->mark[i] = M_UNCOV;
            else s->owner[i] = s->nown[i];
        } else if (s->nown[i] >= 0) {
            if (s->flag[i] & C_LIQ) {
                double r, u[3];
                post_moments(p, s->f, N, i, force_weight(s, i), &r, u);
                s->scal[SC_SCOV] += r;
            } else if (s->flag[i] & C_IF) {
                s->scal[SC_SCOV] += s->m[i];
            }
            s->flag[i] = C_OBS;
            s->owner[i] = s->nown[i];
        }
    }
    /* refill: neighbours that are neither obstacle nor uncovered in this step decide the
     * type; PDFs are the equilibrium of their mean density and the sphere's surface velocity */
    for (long i = 0; i < N; i++) {
        if (!(s->mark[i] & M_UNCOV)) continue;
        int x, y, z;
        cell_xyz(p, i, &x, &y, &z);
        int ngas = 0, nfl = 0, gas_owner = -1;
        double rs = 0, ps = 0;
        for (int q = 1; q < NQ; q++) {
            long j = nbr(p, x, y, z, CX[q], CY[q], CZ[q]);
            if (j < 0 || (s->flag[j] & C_OBS) || (s->mark[j] & M_UNCOV)) continue;
            if (s->flag[j] & C_GAS) {
                if (gas_owner < 0) gas_owner = s->owner[j];
                ngas++;
            } else {
                double r, u[3];
                post_moments(p, s->f, N, j, force_weight(s, j), &r, u);
                rs += r;
                ps += (s->flag[j] & C_IF) ? s->phi[j] : 1.0;
                nfl++;
            }
        }
        const double *S = s->sph + (long)s->owner[i] * S_LEN;
        const double xc[3] = {(double)x, (double)y, (double)z};
        double d[3], wxd[3], uf[3];
        mindiff(p, xc, S + S_X, d);
        cross(S + S_W, d, wxd);
        for (int k = 0; k < 3; k++) uf[k] = S[S_U + k] + wxd[k];
        if (nfl == 0 && ngas > 0) {
            s->flag[i] = C_GAS;
            s->owner[i] = gas_owner;
            s->m[i] = 0.0;
            s->phi[i] = 0.0;
            continue;
        }
        const double rb = nfl ? rs / nfl : 1.0;
        if (ngas > 0) {
            const double pb = ps / nfl;
            s->flag[i] = C_IF;
            s->owner[i] = gas_owner;
            s->phi[i] = pb;
            s->m[i] = pb * rb;
            s->scal[SC_SUNC] += s->m[i];
        } else {
            s->flag[i] = C_LIQ;
            s->owner[i] = -1;
            s->phi[i] = 1.0;
            s->m[i] = rb;
            s->scal[SC_SUNC] += rb;
        }
        for (int q = 0; q < NQ; q++) s->f[(long)q * N + i] = equi(q, rb, uf);
    }
}

/* ------------------------------------------------------------------------ public API */

/* Initial state (spherical bubbles in quiescent liquid, then spheres):
 * phi = prod_b clamp(|x - c_b| - (r_b - 1/2), 0, 1); gas if 0, liquid if 1, else interface;
 * liquid cells with a gas neighbour become interface cells (phi = 1) to close the layer;
 * f* = e(1, 0), m = phi; cells with |x - x_P|^2 <= R^2 become obstacle cells of the lowest
 * such sphere id; then the bubble model sets V_b(0) and rho_g = rho_g0. */
/* initial liquid density of layer z: 1, or (hydrostatic) the column's hydrostatic profile
 * dp/dz = rho g_z with p = rho / 3 and rho = 1 on the open top's plane z = nz - 1/2 */
static double rho_initial(const orc_params *p, int z)
{
    return p->hydrostatic ? exp(3.0 * p->g[2] * ((double)z - (p->nz - 0.5))) : 1.0;
}

int orc_init(const orc_params *p, orc_state *s)
{
    const long N = ncell(p);
    for (int b = 0; b < bub_cap(p); b++) s->bub[b * B_LEN + B_ROOT] = (double)b;
    for (int z = 0; z < p->nz; z++)
        for (int y = 0; y < p->ny; y++)
            for (int x = 0; x < p->nx; x++) {
                const long i = (long)x + (long)p->nx * ((long)y + (long)p->ny * z);
                double ph = 1.0;
                int own = -1;
                for (int b = 0; b < p->nbub; b++) {
                    const double *B = s->bub + b * B_LEN;
                    const double xc[3] = {(double)x, (double)y, (double)z};
                    double d[3];
                    mindiff(p, xc, B + B_C, d);
                    double v = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) - (B[B_R] - 0.5);
                    if (v < 0) v = 0;
                    if (v > 1) v = 1;
                    if (v < 1.0 && own < 0) own = b;
                    ph *= v;
                }
                s->phi[i] = ph;
                s->owner[i] = own;
                s->flag[i] = ph <= 0.0 ? C_GAS : (ph >= 1.0 ? C_LIQ : C_IF);
            }
    memset(s->mark, 0, (size_t)N);
    for (int z = 0; z < p->nz; z++)
        for (int y = 0; y < p->ny; y++)
            for (int x = 0; x < p->nx; x++) {
                const long i = (long)x + (long)p->nx * ((long)y + (long)p->ny * z);
                if (!(s->flag[i] & C_LIQ)) continue;
                for (int q = 1; q < NQ; q++) {
                    long j = nbr(p, x, y, z, CX[q], CY[q], CZ[q]);
                    if (j >= 0 && (s->flag[j] & C_GAS)) {
                        s->mark[i] = 1;
                        s->owner[i] = s->owner[j];
                        break;
                    }
                }
            }
    const double u0[3] = {0, 0, 0};
    for (long i = 0; i < N; i++) {
        if (s->mark[i]) { s->flag[i] = C_IF; s->phi[i] = 1.0; }
        if (s->flag[i] & C_LIQ) s->owner[i] = -1;
        const double rho = rho_initial(p, (int)(i / ((long)p->nx * p->ny)));
        s->m[i] = s->phi[i] * rho;
        s->kappa[i] = 0.0;
        s->near[i] = 0;
        for (int q = 0; q < NQ; q++) s->f[(long)q * N + i] = equi(q, rho, u0);
    }
    /* the gas of each bubble at the pressure of the liquid around it: hydrostatic at its
     * centre plus the Laplace jump 2 sigma / r (p = rho / 3) */
    for (int b = 0; b < p->nbub; b++) {
        double *B = s->bub + b * B_LEN;
        B[B_RHOG] = p->hydrostatic ? exp(3.0 * p->g[2] * (B[B_C + 2] - (p->nz - 0.5))) + 6.0 * p->sigma / B[B_R] : p->rho_g0;
    }
    for (int a = 0; a < p->nsph; a++) {
        const double *S = s->sph + (long)a * S_LEN;
        int lo[3], hi[3];
        for (int k = 0; k < 3; k++) box_range(p, S, k, lo + k, hi + k);
        for (int zz = lo[2]; zz <= hi[2]; zz++)
            for (int yy = lo[1]; yy <= hi[1]; yy++)
                for (int xx = lo[0]; xx <= hi[0]; xx++) {
                    int x = (xx % p->nx + p->nx) % p->nx, y = (yy % p->ny + p->ny) % p->ny, z = (zz % p->nz + p->nz) % p->nz;
                    long i = (long)x + (long)p->nx * ((long)y + (long)p->ny * z);
                    if (!(s->flag[i] & C_OBS) && covers(p, S, x, y, z)) {
                        s->flag[i] = C_OBS;
                        s->owner[i] = a;
                        s->m[i] = 0.0;
                        s->phi[i] = 1.0;
                    }
                }
    }
    for (int k = 0; k < SC_LEN; k++) s->scal[k] = 0.0;
    s->scal[SC_NBUB] = (double)p->nbub;
    bubble_model(p, s, 1, 0);
    if (p->sigma > 0.0) curvature(p, s);
    return 0;
}

int orc_step(const orc_params *p, orc_state *s, int nsteps)
{
    const long N = ncell(p);
    for (int it = 0; it < nsteps; it++) {
        /* excess mass that found no receiving neighbour last step, spread evenly */
        double share = 0.0;
        if (s->scal[SC_POOL] != 0.0) {
            long nif = 0;
            for (long i = 0; i < N; i++) nif += (s->flag[i] & C_IF) ? 1 : 0;
            if (nif > 0) {
                share = s->scal[SC_POOL] / (double)nif;
                s->scal[SC_POOL] = 0.0;
            }
        }
        for (int a = 0; a < p->nsph; a++)   /* this step's momentum exchange starts from zero */
            for (int k = 0; k < 6; k++) {
                s->sph[(long)a * S_LEN + S_FP + k] = s->sph[(long)a * S_LEN + S_F + k];
                s->sph[(long)a * S_LEN + S_F + k] = 0.0;
            }
        sweep(p, s, share);                                        /* 1 */
        conversions(p, s);                                         /* 2 */
        memcpy(s->f, s->ft, sizeof(double) * (size_t)NQ * (size_t)N);
        contact_links(p, s);                                       /* 3 */
        move_spheres(p, s);
        for (int a = 0; a < p->nsph; a++) s->sph[(long)a * S_LEN + S_HASP] = 1.0;
        if (p->sphere_mode != 0 && p->nsph > 0) cover_uncover(p, s); /* 4 */
        /* (R39: every split_every steps the bubbles split into their connected parts) */
        const int split = p->split_every > 0 && ((long)s->scal[SC_STEPS] + 1) % p->split_every == 0;
        bubble_model(p, s, 0, split);                              /* 5 */
        if (p->sigma > 0.0) curvature(p, s);                       /* 6 */
        s->scal[SC_STEPS] += 1.0;
    }
    return (int)s->scal[SC_STATUS];
}

/* rho and velocity (Guo-shifted, the one the collision used) of every active cell; 0 elsewhere */
void orc_fields(const orc_params *p, const orc_state *s, double *rho, double *u)
{
    const long N = ncell(p);
    for (long i = 0; i < N; i++) {
        double r = 0, v[3] = {0, 0, 0};
        if (s->flag[i] & (C_LIQ | C_IF)) post_moments(p, s->f, N, i, force_weight(s, i), &r, v);
        rho[i] = r;
        for (int k = 0; k < 3; k++) u[(long)k * N + i] = v[k];
    }
}

/* mass of the liquid: sum over liquid cells of rho plus sum over interface cells of m,
 * plus the undistributed excess pool */
double orc_total_mass(const orc_params *p, const orc_state *s)
{
    const long N = ncell(p);
    double M = 0.0;
    for (long i = 0; i < N; i++) {
        if (s->flag[i] & C_LIQ) {
            double r, u[3];
            post_moments(p, s->f, N, i, force_weight(s, i), &r, u);
            M += r;
        } else if (s->flag[i] & C_IF) {
            M += s->m[i];
        }
    }
    return M + s->scal[SC_POOL];
}

/* the pieces of the method exposed for unit pins */
double orc_equilibrium(int q, double rho, const double *u) { return equi(q, rho, u); }
double orc_lambda_minus(double tau)
{
    const double lp = -1.0 / tau;
    return 1.0 / ((3.0 / 16.0) / (1.0 / lp + 0.5) - 0.5);
}
void orc_lubrication(const orc_params *p, orc_state *s, double *Fl) { lubrication(p, s, Fl); }
void orc_curvature(const orc_params *p, orc_state *s) { curvature(p, s); }
void orc_bubble_model(const orc_params *p, orc_state *s) { bubble_model(p, s, 0, 0); }
void orc_bubble_model_split(const orc_params *p, orc_state *s) { bubble_model(p, s, 0, 1); }
int orc_velocity(int q, int k) { return k == 0 ? CX[q] : (k == 1 ? CY[q] : CZ[q]); }
/* step 2 alone, on the state as it stands: f holds the sweep's result f*(t+1), phi and m its
 * fill levels and masses, flag its types (the conversions work on ft, then f takes it) */
void orc_conversions(const orc_params *p, orc_state *s)
{
    const size_t bytes = sizeof(double) * (size_t)NQ * (size_t)ncell(p);
    memcpy(s->ft, s->f, bytes);
    conversions(p, s);
    memcpy(s->f, s->ft, bytes);
}
/* step 4 alone: cells covered and uncovered by the spheres at their current centres */
void orc_cover_uncover(const orc_params *p, orc_state *s) { cover_uncover(p, s); }

/* ------------------------------------------------ tangent-linear (forward-mode) gradient */

/* One step of the sweep together with its derivative along a parameter direction
 * (dtau, dg): the liquid-only case with frozen cell types (walls, periodic axes, spheres
 * held fixed, their surface velocities as wall velocities), as the differentiated window
 * runs it.  df holds d f* / d(theta) of the post-collision state; dJ accumulates the
 * derivative of J = sum over steps and spheres of jdir . F_P (Eqs. netforce,
 * momentum_transfer).  Every expression is the derivative of the corresponding line of
 * sweep(). */
static int tangent_sweep(const orc_params *p, orc_state *s, double *df, double *dft, double dtau, const double dg[3],
                         const double jdir[3], double *J, double *dJ)
{
    const long N = ncell(p);
    const double tau = p->tau, *g = p->g;
    const double lp = -1.0 / tau, dlp = dtau / (tau * tau);
    const double A = 1.0 / lp + 0.5, dA = -dtau;               /* 1/lambda_+ + 1/2 = 1/2 - tau */
    const double B = (3.0 / 16.0) / A - 0.5, dB = -(3.0 / 16.0) / (A * A) * dA;
    const double lm = 1.0 / B, dlm = -dB / (B * B);
    for (int z = 0; z < p->nz; z++)
        for (int y = 0; y < p->ny; y++)
            for (int x = 0; x < p->nx; x++) {
                const long i = (long)x + (long)p->nx * ((long)y + (long)p->ny * z);
                const uint8_t t = s->flag[i];
                if (t & (C_IF | C_GAS)) return -1;
                if (!(t & C_LIQ)) continue;
                double fo[NQ], dfo[NQ], fin[NQ], dfin[NQ];
                double rho0 = 0.0, drho0 = 0.0;
                for (int q = 0; q < NQ; q++) {
                    fo[q] = s->f[(long)q * N + i];
                    dfo[q] = df[(long)q * N + i];
                    rho0 += fo[q];
                    drho0 += dfo[q];
                }
                const double xc[3] = {(double)x, (double)y, (double)z};
                for (int q = 0; q < NQ; q++) {
                    const long src = nbr(p, x, y, z, -CX[q], -CY[q], -CZ[q]);
                    if (src < 0) { fin[q] = fo[opp(q)]; dfin[q] = dfo[opp(q)]; continue; }
                    if (s->flag[src] & C_LIQ) {
                        fin[q] = s->f[(long)q * N + src];
                        dfin[q] = df[(long)q * N + src];
                        continue;
                    }
                    /* sphere link (Eq. bbrule), wall velocity of the fixed sphere */
                    double *S = s->sph + (long)s->owner[src] * S_LEN;
                    const double cq[3] = {CX[q], CY[q], CZ[q]};
                    double xw[3] = {xc[0] - 0.5 * cq[0], xc[1] - 0.5 * cq[1], xc[2] - 0.5 * cq[2]};
                    double d[3], wxd[3], uw[3];
                    mindiff(p, xw, S + S_X, d);
                    cross(S + S_W, d, wxd);
                    for (int k = 0; k < 3; k++) uw[k] = S[S_U + k] + wxd[k];
                    const double cu = cq[0] * uw[0] + cq[1] * uw[1] + cq[2] * uw[2];
                    fin[q] = fo[opp(q)] + 6.0 * wq(q) * rho0 * cu;
                    dfin[q] = dfo[opp(q)] + 6.0 * wq(q) * drho0 * cu;
                    /* momentum into the sphere and its derivative */
                    const double a = fo[opp(q)] + fin[q], da = dfo[opp(q)] + dfin[q];
                    for (int k = 0; k < 3; k++) {
                        *J += jdir[k] * (-cq[k] * a);
                        *dJ += jdir[k] * (-cq[k] * da);
                    }
                }
                double rho = 0, j[3] = {0, 0, 0}, drho = 0, dj[3] = {0, 0, 0};
                for (int q = 0; q < NQ; q++) {
                    rho += fin[q];
                    drho += dfin[q];
                    j[0] += CX[q] * fin[q]; j[1] += CY[q] * fin[q]; j[2] += CZ[q] * fin[q];
                    dj[0] += CX[q] * dfin[q]; dj[1] += CY[q] * dfin[q]; dj[2] += CZ[q] * dfin[q];
                }
                double u[3], du[3];
                for (int k = 0; k < 3; k++) {
                    u[k] = (j[k] + 0.5 * rho * g[k]) / rho;
                    du[k] = (dj[k] + 0.5 * drho * g[k] + 0.5 * rho * dg[k]) / rho - u[k] * drho / rho;
                }
                const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                const double duu = 2.0 * (u[0] * du[0] + u[1] * du[1] + u[2] * du[2]);
                const double ug = u[0] * g[0] + u[1] * g[1] + u[2] * g[2];
                const double dug = du[0] * g[0] + du[1] * g[1] + du[2] * g[2] + u[0] * dg[0] + u[1] * dg[1] + u[2] * dg[2];
                for (int q = 0; q < NQ; q++) {
                    const int qb = opp(q);
                    const double w = wq(q);
                    const double cu = CX[q] * u[0] + CY[q] * u[1] + CZ[q] * u[2];
                    const double dcu = CX[q] * du[0] + CY[q] * du[1] + CZ[q] * du[2];
                    const double cg = CX[q] * g[0] + CY[q] * g[1] + CZ[q] * g[2];
                    const double dcg = CX[q] * dg[0] + CY[q] * dg[1] + CZ[q] * dg[2];
                    const double ep = w * rho * (1.0 + 4.5 * cu * cu - 1.5 * uu);
                    const double dep = w * drho * (1.0 + 4.5 * cu * cu - 1.5 * uu) + w * rho * (9.0 * cu * dcu - 1.5 * duu);
                    const double em = w * rho * 3.0 * cu, dem = 3.0 * w * (drho * cu + rho * dcu);
                    const double fp = 0.5 * (fin[q] + fin[qb]), dfp = 0.5 * (dfin[q] + dfin[qb]);
                    const double fm = 0.5 * (fin[q] - fin[qb]), dfm = 0.5 * (dfin[q] - dfin[qb]);
                    const double Gp = w * rho * (9.0 * cu * cg - 3.0 * ug);
                    const double dGp = w * drho * (9.0 * cu * cg - 3.0 * ug) + w * rho * (9.0 * (dcu * cg + cu * dcg) - 3.0 * dug);
                    const double Gm = w * rho * 3.0 * cg, dGm = 3.0 * w * (drho * cg + rho * dcg);
                    s->ft[(long)q * N + i] = fin[q] + lp * (fp - ep) + lm * (fm - em) + (1.0 + 0.5 * lp) * Gp + (1.0 + 0.5 * lm) * Gm;
                    dft[(long)q * N + i] = dfin[q] + dlp * (fp - ep) + lp * (dfp - dep) + dlm * (fm - em) + lm * (dfm - dem)
                                         + 0.5 * dlp * Gp + (1.0 + 0.5 * lp) * dGp + 0.5 * dlm * Gm + (1.0 + 0.5 * lm) * dGm;
                }
            }
    memcpy(s->f, s->ft, sizeof(double) * (size_t)NQ * (size_t)N);
    memcpy(df, dft, sizeof(double) * (size_t)NQ * (size_t)N);
    return 0;
}

/* nsteps steps of the frozen liquid window from the current state with the derivative along
 * (dtau, dg): *J = sum_t jdir . sum_P F_P(t) (links between obstacle nodes of two spheres
 * included, constant in the parameters), *dJ its derivative.  df: [19][N] scratch, zero on
 * entry for a state that does not depend on the parameters; dft: [19][N] scratch. */
int orc_tangent_window(const orc_params *p, orc_state *s, double *df, double *dft, double dtau, const double *dg,
                       const double *jdir, int nsteps, double *J, double *dJ)
{
    *J = 0.0;
    *dJ = 0.0;
    for (int it = 0; it < nsteps; it++) {
        for (int a = 0; a < p->nsph; a++)
            for (int k = 0; k < 6; k++) s->sph[(long)a * S_LEN + S_F + k] = 0.0;
        if (tangent_sweep(p, s, df, dft, dtau, dg, jdir, J, dJ)) return -1;
        contact_links(p, s);
        double Fc = 0.0;   /* contact-link part of the forces (the sweep's part is in *J) */
        for (int a = 0; a < p->nsph; a++)
            for (int k = 0; k < 3; k++) Fc += jdir[k] * s->sph[(long)a * S_LEN + S_F + k];
        *J += Fc;
    }
    return 0;
}
