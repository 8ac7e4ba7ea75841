// lbm_capi.cu -- the C ABI (include/lbm.h): arena layout, host-side handle and the launch
// sequence of one time step.  The library allocates no device memory: everything lives in
// the caller's arena.  Work goes to the caller's stream; one step is recorded once into a
// CUDA graph (two steps, for the two grid parities) and replayed.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "lbm_internal.cuh"

using namespace lbm;

struct lbm_ctx {
    lbm_params p;
    Dev d;
    cudaStream_t stream;
    char* arena;
    size_t arena_bytes;
    std::vector<double> bub_geo;     // [nbub][4] centre, radius
    std::vector<Sphere> sph_init;
    std::vector<SphLink> sphl_init;   // staging of the first upload of the link data
    bool started;
    int cur;
    uint64_t launches;
    double* geo_dev;
    float* adj_srho;
    double* adj_part;
    bool moving_walls;
    Sphere* sph_stage;
    Scalars* sc_stage;
    Bubble* bub_stage;
    // graph of two consecutive steps (cur = 0 then 1)
    // two overlapped steps as a CUDA graph; with bubble splitting one graph per combination of
    // the two captured end-of-step passes splitting or not (bit 0: the first, bit 1: the second)
    cudaGraphExec_t graph[4];
    bool graph_ready[4];
    uint64_t closed;   // end-of-step passes enqueued so far (the steps they close)
    bool use_graph;
    // optional timing of the sweep: CUDA events around the bulk kernel and around the rest
    // (fix pass + boundary kernel), on the library's stream
    bool profiling;
    cudaEvent_t ev[4 * 64];
    bool ev_ready;
    bool ev_pending[64];
    int ev_slot;
    double bulk_ms, rest_ms;
    uint64_t sweeps;
    // the end-of-step kernels of the last step not enqueued yet: the next step runs them
    // concurrently with its bulk sweep, any query runs them first
    bool pending;
    // the next step's partner lists / obstacle-node links: not enqueued yet, enqueued on the
    // links stream (to be joined by the sweep's rest), or enqueued and already joined
    int links_state;
    uint64_t h2d_bytes, d2h_bytes;   // host <-> device copies made by the library
    struct { uint32_t on; double j[3]; } obj_stage;   // host side of lbm_objective's upload
    // second stream and fork/join events of the concurrent bulk / boundary sweep
    cudaStream_t side, side2;   // the general and the lean boundary sweep
    cudaEvent_t fork, join, fork2, join2, fork3, join3, fork4, join4, join5;
    cudaStream_t epi;     // the end-of-step kernels when they overlap the next bulk sweep
    cudaStream_t links;   // partner lists and obstacle-node links beside the sweep's rest
    bool side_ready;
};

namespace {

enum { kLinksNone = 0, kLinksForked = 1, kLinksJoined = 2 };
constexpr size_t kAlign = 256;
constexpr int kBinCap = 16;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int check_params(const lbm_params* p) {
    if (!p) return LBM_EINVAL;
    if (p->nx < 3 || p->ny < 3 || p->nz < 3) return LBM_EINVAL;
    if ((double)p->nx * p->ny * p->nz > 4.0e9) return LBM_EINVAL;
    for (int k = 0; k < 3; k++)
        if (p->bc[k] != LBM_BC_WALL && p->bc[k] != LBM_BC_PERIODIC && p->bc[k] != LBM_BC_FREESLIP) return LBM_EINVAL;
    if (p->open_top != 0 && (p->open_top != 1 || p->bc[2] == LBM_BC_PERIODIC)) return LBM_EINVAL;
    if (p->hydrostatic != 0 && (p->hydrostatic != 1 || !p->open_top)) return LBM_EINVAL;
    if (p->split_every < 0) return LBM_EINVAL;
    if (p->storage < LBM_STORE_F32 || p->storage > LBM_STORE_BF16DEV) return LBM_EINVAL;
    if (p->n_substeps < 1 || p->n_substeps > 64) return LBM_EINVAL;
    if (p->sphere_mode < LBM_SPHERES_FIXED || p->sphere_mode > LBM_SPHERES_PRESCRIBED) return LBM_EINVAL;
    if (p->max_bubbles < 1 || p->max_spheres < 1 || p->worklist_cap < 0) return LBM_EINVAL;
    if (!(p->tau > 0.5) || !(p->tau < 100.0)) return LBM_EINVAL;
    if (!(p->sigma >= 0.0) || !(p->rho_gas0 > 0.0) || !(p->eps >= 0.0)) return LBM_EINVAL;
    return LBM_OK;
}

size_t pdf_bytes(const lbm_params* p) { return p->storage == LBM_STORE_F32 ? 4 : 2; }

struct Layout {
    size_t f[2], flags, mark, tmark, wl_link, wl_rare, sph_list, sph_cpl, sph_near, sph_nnear, tbox, sph_bin, mass, phi[2], rho[2], owner, kappa, bub, sph, sph_tmp, sphl, gasflag, acc, sc, wl[4], wl_slow, wl_fix, bin_cnt, bin_ids, npairs, pairs, geo,
        adj_srho, adj_part, merge_keys, merge_list, lab, split_list, part_key, part_root, part_V, part_new, bub_cnt, total;
    size_t N, wl_cap, nbins_max;
};

Layout layout_of(const lbm_params* p) {
    Layout L{};
    L.N = (size_t)p->nx * p->ny * p->nz;
    L.wl_cap = p->worklist_cap > 0 ? (size_t)p->worklist_cap : L.N / 50 + 4096;
    // bins are at least 4 cells wide
    L.nbins_max = (size_t)((p->nx + 3) / 4) * ((p->ny + 3) / 4) * ((p->nz + 3) / 4);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes); return at; };
    L.f[0] = take(19 * L.N * pdf_bytes(p));
    L.f[1] = take(19 * L.N * pdf_bytes(p));
    L.flags = take(L.N + 16);
    L.mark = take(L.N + 16);
    L.tmark = take(L.N + 16);
    L.mass = take(4 * L.N);
    L.phi[0] = take(4 * L.N);
    L.phi[1] = take(4 * L.N);
    L.rho[0] = p->max_spheres > 32 ? take(4 * L.N) : 0;   // (only the lean shell kernel reads them)
    L.rho[1] = p->max_spheres > 32 ? take(4 * L.N) : 0;
    L.owner = take(4 * L.N);
    L.kappa = p->sigma > 0.0 ? take(4 * L.N) : 0;
    L.bub = take(sizeof(Bubble) * (size_t)p->max_bubbles);
    L.sph = take(sizeof(Sphere) * (size_t)p->max_spheres);
    L.sph_tmp = take(sizeof(Sphere) * (size_t)p->max_spheres);
    L.sphl = take(sizeof(SphLink) * (size_t)p->max_spheres);
    L.gasflag = take(sizeof(uint32_t) * 2 * (size_t)p->max_spheres);
    L.acc = take(sizeof(SphereAcc) * (size_t)p->max_spheres);
    L.sc = take(sizeof(Scalars));
    for (int k = 0; k < 4; k++) L.wl[k] = take(4 * L.wl_cap);
    L.wl_slow = take(4 * L.N);
    L.wl_fix = take(4 * L.wl_cap);
    // the lean kernel's link words (only a simulation with many spheres has a liquid segment)
    L.wl_link = p->max_spheres > 32 ? take(8 * L.N) : 0;
    L.wl_rare = p->max_spheres > 32 ? take(4 * L.wl_cap) : 0;
    L.bin_cnt = take(4 * L.nbins_max);
    L.bin_ids = take(4 * L.nbins_max * kBinCap);
    L.npairs = take(4 * (size_t)p->max_spheres);
    L.sph_list = take(4 * (size_t)p->max_spheres);
    L.sph_cpl = take(4 * (size_t)p->max_spheres);
    L.sph_near = take(4 * (size_t)kNearCap * (size_t)p->max_spheres);
    L.sph_nnear = take(4 * (size_t)p->max_spheres);
    L.tbox = take(sizeof(TouchBox) * (size_t)p->max_spheres);
    L.sph_bin = take(sizeof(int4) * (size_t)p->max_spheres);
    L.pairs = take(4 * (size_t)p->max_spheres * kPairCap);
    L.geo = take(sizeof(double) * 4 * (size_t)p->max_bubbles);
    L.adj_srho = take(4 * L.N);
    L.adj_part = take(sizeof(double) * 5 * kAdjSlots);
    L.merge_keys = take(sizeof(unsigned long long) * kMergeCap);
    L.merge_list = take(sizeof(uint32_t) * kMergeCap);
    if (p->split_every > 0) {   // bubble splitting: union-find labels, the part table, counts per id
        L.lab = take(4 * L.N);
        L.split_list = take(4 * L.N);
        L.part_key = take(sizeof(uint32_t) * kPartCap);
        L.part_root = take(sizeof(uint32_t) * kPartCap);
        L.part_V = take(sizeof(double) * kPartCap);
        L.part_new = take(sizeof(int32_t) * kPartCap);
        L.bub_cnt = take(sizeof(uint32_t) * (size_t)p->max_bubbles);
    }
    L.total = o;
    return L;
}

int cuda_fail(cudaError_t e) {
    if (e == cudaSuccess) return LBM_OK;
    std::fprintf(stderr, "lbm: CUDA error %s\n", cudaGetErrorString(e));
    return LBM_ECUDA;
}

int launched(lbm_ctx* c, int n) {
    c->launches += (uint64_t)n;
    return cuda_fail(cudaGetLastError());
}

int status_code(uint32_t st) {
    if (st & S_UNSTABLE) return LBM_EUNSTABLE;
    if (st & (S_OVERFLOW | S_BIN_OVERFLOW)) return LBM_EOVERFLOW;
    if (st & S_SPLIT) return LBM_ESPLIT;
    if (st & S_MERGE) return LBM_EMERGE;
    return LBM_OK;
}

// collect the elapsed times of a recorded slot (bulk start/end, rest start/end)
void prof_collect(lbm_ctx* c, int slot) {
    if (!c->ev_pending[slot]) return;
    cudaEventSynchronize(c->ev[4 * slot + 3]);
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, c->ev[4 * slot], c->ev[4 * slot + 1]) == cudaSuccess &&
        cudaEventElapsedTime(&b, c->ev[4 * slot + 2], c->ev[4 * slot + 3]) == cudaSuccess) {
        c->bulk_ms += a;
        c->rest_ms += b;
        c->sweeps++;
    }
    c->ev_pending[slot] = false;
}

// end-of-step kernels of the step that wrote grid g (Sec. 2.2 conversions and bubble model,
// Sec. 2.3 sphere motion and cover/uncover): the sphere motion on the side stream concurrent
// with the conversions on `e`, then cover/uncover, the end-of-step scan and the curvature on `e`
// the end-of-step pass that closes step k splits bubbles
bool split_due_host(const lbm_ctx* c, uint64_t k) { return c->d.split_every > 0 && k % (uint64_t)c->d.split_every == 0; }

void enqueue_epilogue(lbm_ctx* c, int g, cudaStream_t e, bool split) {
    const Dev& d = c->d;
    if (d.nsph > 0) {
        cudaEventRecord(c->fork4, e);
        cudaStreamWaitEvent(c->side, c->fork4, 0);
        launch_spheres_move(d, c->side);
    }
    // the conversions close the step themselves unless the cover kernel follows
    const bool cover = d.nsph > 0 && d.sphere_mode != LBM_SPHERES_FIXED;
    launch_conversions(d, g, !cover, e);
    if (d.nsph > 0) {
        cudaEventRecord(c->join4, c->side);
        cudaStreamWaitEvent(e, c->join4, 0);
    }
    launch_spheres_cover(d, g, e);
    if (split) launch_split(d, g, e);   // (the step is closed)
    // the next step's partner lists and obstacle-node links need only the moved spheres, their
    // bins and obstacle cells, all final now: they run beside the rest of these kernels and
    // the next bulk sweep, and the next step's sweep joins them
    if (d.nsph > 0) {
        cudaEventRecord(c->fork2, e);
        cudaStreamWaitEvent(c->links, c->fork2, 0);
        launch_spheres_links(d, g, c->links);
        cudaEventRecord(c->join2, c->links);
        c->links_state = kLinksForked;
    }
    if (d.kappa) launch_curvature(d, g, e);
    launch_list_rescan(d, e);   // the next boundary sweep's list, from the final types
    // the liquid segment's links, classified while the next bulk sweep runs
    if (d.split_liq && d.wl_link) launch_link_classify(d, e);
}

int epilogue_launches(const Dev& d, bool split) {
    return 1 + spheres_launches(d) + (d.kappa ? 1 : 0) + 1 + (split ? kSplitLaunches : 0) + (d.split_liq && d.wl_link ? 1 : 0);
}
int step_launches(const Dev& d, bool overlap, bool split) {
    return 3 + d.split_liq + (d.split_liq && d.wl_link ? 1 : 0) + spheres_links_launches(d) + (overlap ? epilogue_launches(d, split) : 0);
}

// one step reading grid cur: the bulk sweep on s and, with `overlap`, the end-of-step kernels
// of the previous step concurrently on the epilogue stream; once both are done the fix pass
// and the boundary sweep.  The step's own end-of-step kernels are left pending.  With `timed`,
// event pairs bracket the bulk sweep and the rest on s.
int enqueue_step(lbm_ctx* c, int cur, cudaStream_t s, bool overlap, bool timed = false, bool split = false) {
    const Dev& d = c->d;
    int slot = 0;
    if (timed) {
        slot = c->ev_slot;
        c->ev_slot = (c->ev_slot + 1) % 64;
        prof_collect(c, slot);
    }
    if (overlap) {
        cudaEventRecord(c->fork3, s);
        cudaStreamWaitEvent(c->epi, c->fork3, 0);
        enqueue_epilogue(c, cur, c->epi, split);
        cudaEventRecord(c->join3, c->epi);
    }
    if (timed) cudaEventRecord(c->ev[4 * slot], s);
    launch_sweep_bulk(d, cur, s, true);
    if (timed) cudaEventRecord(c->ev[4 * slot + 1], s);
    if (overlap) cudaStreamWaitEvent(s, c->join3, 0);
    if (timed) cudaEventRecord(c->ev[4 * slot + 2], s);
    if (d.nsph > 0 && c->links_state == kLinksNone) {   // the first step: nothing forked them
        cudaEventRecord(c->fork2, s);
        cudaStreamWaitEvent(c->links, c->fork2, 0);
        launch_spheres_links(d, cur, c->links);
        cudaEventRecord(c->join2, c->links);
        c->links_state = kLinksForked;
    }
    launch_sweep_rest(d, cur, s, c->side, c->side2, c->fork, c->join, c->join5);
    // the step's force sums need the links (an event recorded in this same call: a graph
    // capture in between would leave an earlier record unusable)
    if (d.nsph > 0 && c->links_state == kLinksForked) cudaStreamWaitEvent(s, c->join2, 0);
    c->links_state = kLinksNone;
    if (timed) {
        cudaEventRecord(c->ev[4 * slot + 3], s);
        c->ev_pending[slot] = true;
    }
    return cuda_fail(cudaGetLastError());
}

// enqueue the pending end-of-step kernels on the library's stream (before any query)
int flush(lbm_ctx* c) {
    if (!c->pending) return LBM_OK;
    const bool split = split_due_host(c, c->closed + 1);
    enqueue_epilogue(c, c->cur, c->stream, split);
    c->closed++;
    // what the caller reads next is ordered after every kernel the library enqueued
    if (c->links_state == kLinksForked) {
        cudaStreamWaitEvent(c->stream, c->join2, 0);
        c->links_state = kLinksJoined;
    }
    c->pending = false;
    return launched(c, epilogue_launches(c->d, split));
}

int first_step(lbm_ctx* c) {
    const lbm_params* p = &c->p;
    Layout L = layout_of(p);
    char* a = c->arena;
    Dev& d = c->d;
    std::memset(&d, 0, sizeof d);
    d.nx = p->nx; d.ny = p->ny; d.nz = p->nz;
    for (int k = 0; k < 3; k++) {
        d.bc[k] = p->bc[k] == LBM_BC_PERIODIC ? 1 : 0;
        d.face[2 * k] = d.face[2 * k + 1] = p->bc[k] == LBM_BC_FREESLIP ? FACE_SLIP : FACE_WALL;
    }
    if (p->open_top) d.face[5] = FACE_OPEN;
    d.hydrostatic = p->hydrostatic;
    d.gz = p->g[2];
    for (int k = 0; k < 6; k++) d.special |= d.face[k] != FACE_WALL && !d.bc[k / 2];
    d.N = L.N;
    d.div_nx = make_fastdiv((uint32_t)p->nx);
    d.div_ny = make_fastdiv((uint32_t)p->ny);
    d.storage = p->storage;
    d.n_sub = p->n_substeps;
    d.sphere_mode = p->sphere_mode;
    d.ngeo = (int)(c->bub_geo.size() / 4);
    d.geo_rmax = 0.0;
    for (int b = 0; b < d.ngeo; b++) d.geo_rmax = std::max(d.geo_rmax, c->bub_geo[4 * b + 3]);
    d.split_every = p->split_every;
    // with splitting, new bubbles take free rows: every row of the table is a bubble id
    d.nbub = p->split_every > 0 ? std::max(p->max_bubbles, d.ngeo) : d.ngeo;
    d.nsph = (int)c->sph_init.size();
    {   // the liquid cells beside the spheres, about 4 pi (R + 1)^2 each: the lean kernel pays
        // for its extra graph branch once they outnumber one round of the general grid
        double shell = 0.0;
        for (const Sphere& sp : c->sph_init) shell += 4.0 * 3.14159265358979 * (sp.R + 1.0) * (sp.R + 1.0);
        d.split_liq = shell > (double)kBoundaryGrid * 128.0 ? 1 : 0;
    }

    d.max_bub = p->max_bubbles;
    d.max_sph = p->max_spheres;
    d.wl_cap = (int)L.wl_cap;
    d.tau = (float)p->tau;
    const double lp = -1.0 / p->tau;
    d.lp = (float)lp;
    d.lm = (float)(1.0 / ((3.0 / 16.0) / (1.0 / lp + 0.5) - 0.5));
    for (int k = 0; k < 3; k++) { d.g[k] = (float)p->g[k]; d.gd[k] = p->g[k]; }
    set_collision_consts(d);
    d.sigma = (float)p->sigma;
    d.rho_g0 = (float)p->rho_gas0;
    d.eps = (float)p->eps;
    d.f[0] = a + L.f[0];
    d.f[1] = a + L.f[1];
    d.flags = (uint8_t*)(a + L.flags);
    d.mark = (uint8_t*)(a + L.mark);
    d.tmark = (uint8_t*)(a + L.tmark);
    d.mass = (float*)(a + L.mass);
    d.phi[0] = (float*)(a + L.phi[0]);
    d.phi[1] = (float*)(a + L.phi[1]);
    // the densities are kept only where the lean shell kernel runs (it alone reads them)
    const bool keep_rho = d.split_liq && p->max_spheres > 32;
    d.rho[0] = keep_rho ? (float*)(a + L.rho[0]) : nullptr;
    d.rho[1] = keep_rho ? (float*)(a + L.rho[1]) : nullptr;
    d.owner = (uint32_t*)(a + L.owner);
    d.kappa = p->sigma > 0.0 ? (float*)(a + L.kappa) : nullptr;
    d.bub = (Bubble*)(a + L.bub);
    d.sph = (Sphere*)(a + L.sph);
    d.sph_tmp = (Sphere*)(a + L.sph_tmp);
    d.gasflag = (uint32_t*)(a + L.gasflag);
    d.sphl = (SphLink*)(a + L.sphl);
    d.acc = (SphereAcc*)(a + L.acc);
    d.sc = (Scalars*)(a + L.sc);
    d.wl_conv = (uint32_t*)(a + L.wl[0]);
    d.wl_newif = (uint32_t*)(a + L.wl[1]);
    d.wl_fromliq = (uint32_t*)(a + L.wl[2]);
    d.wl_touch = (uint32_t*)(a + L.wl[3]);
    d.wl_slow = (uint32_t*)(a + L.wl_slow);
    d.wl_fix = (uint32_t*)(a + L.wl_fix);
    d.wl_link = p->max_spheres > 32 ? (uint2*)(a + L.wl_link) : nullptr;
    d.wl_rare = p->max_spheres > 32 ? (uint32_t*)(a + L.wl_rare) : nullptr;
    double rmax = 1.0;
    for (const Sphere& s : c->sph_init) rmax = std::fmax(rmax, s.R);
    d.bin_w = (int)std::ceil(2.0 * rmax + 2.0);
    if (d.bin_w < 4) d.bin_w = 4;
    d.nbx = p->nx / d.bin_w > 0 ? p->nx / d.bin_w : 1;
    d.nby = p->ny / d.bin_w > 0 ? p->ny / d.bin_w : 1;
    d.nbz = p->nz / d.bin_w > 0 ? p->nz / d.bin_w : 1;
    d.bin_cap = kBinCap;
    d.bin_cnt = (uint32_t*)(a + L.bin_cnt);
    d.bin_ids = (uint32_t*)(a + L.bin_ids);
    d.npairs = (uint32_t*)(a + L.npairs);
    d.sph_list = (uint32_t*)(a + L.sph_list);
    d.sph_cpl = (uint32_t*)(a + L.sph_cpl);
    d.sph_near = (uint32_t*)(a + L.sph_near);
    d.sph_nnear = (uint32_t*)(a + L.sph_nnear);
    d.tbox = (TouchBox*)(a + L.tbox);
    d.sph_bin = (int4*)(a + L.sph_bin);
    d.pairs = (uint32_t*)(a + L.pairs);
    d.merge_keys = (unsigned long long*)(a + L.merge_keys);
    d.merge_list = (uint32_t*)(a + L.merge_list);
    if (p->split_every > 0) {
        d.lab = (uint32_t*)(a + L.lab);
        d.split_list = (uint32_t*)(a + L.split_list);
        d.part_key = (uint32_t*)(a + L.part_key);
        d.part_root = (uint32_t*)(a + L.part_root);
        d.part_V = (double*)(a + L.part_V);
        d.part_new = (int32_t*)(a + L.part_new);
        d.bub_cnt = (uint32_t*)(a + L.bub_cnt);
    }
    c->geo_dev = (double*)(a + L.geo);
    c->adj_srho = (float*)(a + L.adj_srho);
    c->adj_part = (double*)(a + L.adj_part);
    c->moving_walls = false;
    for (const Sphere& sp : c->sph_init)
        for (int k = 0; k < 3; k++) c->moving_walls |= sp.u[k] != 0.0 || sp.w[k] != 0.0;

    cudaStream_t s = c->stream;
    prepare_sphere_kernels();
    if (!c->side_ready) {
        // the boundary sweep is latency-bound and small: on a stream of the highest priority its
        // blocks take their SM slots first and finish inside the bandwidth-bound bulk sweep
        int lo_prio = 0, hi_prio = 0;
        cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
        if (cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi_prio) != cudaSuccess) return LBM_ECUDA;
        if (cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess) return LBM_ECUDA;
        if (cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming) != cudaSuccess) return LBM_ECUDA;
        if (cudaEventCreateWithFlags(&c->fork2, cudaEventDisableTiming) != cudaSuccess) return LBM_ECUDA;
        if (cudaEventCreateWithFlags(&c->join2, cudaEventDisableTiming) != cudaSuccess) return LBM_ECUDA;
        if (cudaEventCreateWithFlags(&c->fork3, cudaEventDisableTiming) != cudaSuccess) return LBM_ECUDA;
        if (cudaEventCreateWithFlags(&c->join3, cudaEventDisableTiming) != cudaSuccess) return LBM_ECUDA;
        if (cudaStreamCreateWithPriority(&c->epi, cudaStreamNonBlocking, hi_prio) != cudaSuccess) return LBM_ECUDA;
        if (cudaStreamCreateWithPriority(&c->links, cudaStreamNonBlocking, hi_prio) != cudaSuccess) return LBM_ECUDA;
        if (cudaEventCreateWithFlags(&c->fork4, cudaEventDisableTiming) != cudaSuccess) return LBM_ECUDA;
        if (cudaEventCreateWithFlags(&c->join4, cudaEventDisableTiming) != cudaSuccess) return LBM_ECUDA;
        if (cudaStreamCreateWithPriority(&c->side2, cudaStreamNonBlocking, hi_prio) != cudaSuccess) return LBM_ECUDA;
        if (cudaEventCreateWithFlags(&c->join5, cudaEventDisableTiming) != cudaSuccess) return LBM_ECUDA;
        c->side_ready = true;
    }
    int rc = cuda_fail(cudaMemsetAsync(a, 0, L.total, s));
    if (rc) return rc;
    if (d.ngeo > 0)
        if ((rc = cuda_fail(cudaMemcpyAsync(c->geo_dev, c->bub_geo.data(), sizeof(double) * c->bub_geo.size(), cudaMemcpyHostToDevice, s)))) return rc;
    if (d.nsph > 0)
        if ((rc = cuda_fail(cudaMemcpyAsync(d.sph, c->sph_init.data(), sizeof(Sphere) * d.nsph, cudaMemcpyHostToDevice, s)))) return rc;
    if (d.nsph > 0) {
        c->sphl_init.resize(d.nsph);
        for (int a2 = 0; a2 < d.nsph; a2++) c->sphl_init[a2] = sph_link_of(c->sph_init[a2]);
        if ((rc = cuda_fail(cudaMemcpyAsync(d.sphl, c->sphl_init.data(), sizeof(SphLink) * d.nsph, cudaMemcpyHostToDevice, s)))) return rc;
        c->h2d_bytes += sizeof(SphLink) * d.nsph;
    }
    c->h2d_bytes += sizeof(double) * c->bub_geo.size() + sizeof(Sphere) * (size_t)d.nsph;
    launch_bins_insert(d, s);
    launch_init(d, c->geo_dev, s);
    launch_bulk_all(d, s);
    launch_init_scan(d, s);
    if (d.split_liq && d.wl_link) launch_link_classify(d, s);
    if (d.kappa) launch_curvature(d, 0, s);
    if ((rc = launched(c, (d.nsph > 0) + 3 + (d.kappa ? 1 : 0) + (d.split_liq && d.wl_link ? 1 : 0)))) return rc;
    c->cur = 0;
    c->pending = false;
    c->links_state = kLinksNone;
    c->started = true;
    return cuda_fail(cudaStreamSynchronize(s));
}

int build_graph(lbm_ctx* c, int variant) {
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return LBM_ECUDA;
    cudaGraph_t g = nullptr;
    int rc = LBM_OK;
    const int links_state = c->links_state;   // host bookkeeping only: captured, not run
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = LBM_ECUDA;
    if (!rc) {
        enqueue_step(c, 0, cap, true, false, (variant & 1) != 0);
        enqueue_step(c, 1, cap, true, false, (variant & 2) != 0);
        c->links_state = links_state;
        if (cudaStreamEndCapture(cap, &g) != cudaSuccess) rc = LBM_ECUDA;
    }
    // per-node priorities: the boundary sweep keeps its stream's priority inside the graph
    if (!rc && cudaGraphInstantiate(&c->graph[variant], g, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess)
        rc = LBM_ECUDA;
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    cudaGetLastError();
    c->graph_ready[variant] = rc == LBM_OK;
    return rc;
}

int sync_tables(lbm_ctx* c) {
    cudaStream_t s = c->stream;
    int rc;
    c->d2h_bytes += sizeof(Scalars) + sizeof(Sphere) * (size_t)c->d.nsph + sizeof(Bubble) * (size_t)c->d.nbub;
    if ((rc = cuda_fail(cudaMemcpyAsync(c->sc_stage, c->d.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s)))) return rc;
    if (c->d.nsph > 0)
        if ((rc = cuda_fail(cudaMemcpyAsync(c->sph_stage, c->d.sph, sizeof(Sphere) * c->d.nsph, cudaMemcpyDeviceToHost, s)))) return rc;
    if (c->d.nbub > 0)
        if ((rc = cuda_fail(cudaMemcpyAsync(c->bub_stage, c->d.bub, sizeof(Bubble) * c->d.nbub, cudaMemcpyDeviceToHost, s)))) return rc;
    return cuda_fail(cudaStreamSynchronize(s));
}

}  // namespace

extern "C" {

int lbm_arena_bytes(const lbm_params* p, size_t* bytes) {
    int rc = check_params(p);
    if (rc) return rc;
    if (!bytes) return LBM_EINVAL;
    *bytes = layout_of(p).total;
    return LBM_OK;
}

int lbm_init(const lbm_params* p, void* arena, size_t arena_bytes, void* cuda_stream, lbm_ctx** out) {
    int rc = check_params(p);
    if (rc) return rc;
    if (!arena || !out || ((uintptr_t)arena % kAlign)) return LBM_EINVAL;
    if (arena_bytes < layout_of(p).total) return LBM_EINVAL;
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_EINVAL;
    c->p = *p;
    c->stream = (cudaStream_t)cuda_stream;
    c->arena = (char*)arena;
    c->arena_bytes = arena_bytes;
    c->started = false;
    c->cur = 0;
    c->launches = 0;
    for (int v = 0; v < 4; v++) c->graph_ready[v] = false;
    c->closed = 0;
    c->use_graph = std::getenv("LBM_NO_GRAPH") == nullptr;
    c->profiling = false;
    c->ev_ready = false;
    for (int k = 0; k < 64; k++) c->ev_pending[k] = false;
    c->ev_slot = 0;
    c->bulk_ms = c->rest_ms = 0.0;
    c->sweeps = 0;
    c->pending = false;
    c->h2d_bytes = 0;
    c->d2h_bytes = 0;
    c->side_ready = false;
    c->sph_stage = (Sphere*)std::malloc(sizeof(Sphere) * (size_t)p->max_spheres);
    c->sc_stage = (Scalars*)std::malloc(sizeof(Scalars));
    c->bub_stage = (Bubble*)std::malloc(sizeof(Bubble) * (size_t)p->max_bubbles);
    if (!c->sph_stage || !c->sc_stage || !c->bub_stage) { lbm_destroy(c); return LBM_EINVAL; }
    *out = c;
    return LBM_OK;
}

int lbm_set_stream(lbm_ctx* c, void* cuda_stream) {
    if (!c) return LBM_EINVAL;
    c->stream = (cudaStream_t)cuda_stream;
    return LBM_OK;
}

int lbm_add_bubble(lbm_ctx* c, const double cen[3], double r, int* id) {
    if (!c || !cen || !(r > 0.0)) return LBM_EINVAL;
    if (c->started) return LBM_ESTATE;
    if ((int)(c->bub_geo.size() / 4) >= c->p.max_bubbles) return LBM_EINVAL;
    if (id) *id = (int)(c->bub_geo.size() / 4);
    c->bub_geo.insert(c->bub_geo.end(), {cen[0], cen[1], cen[2], r});
    return LBM_OK;
}

int lbm_add_sphere(lbm_ctx* c, const double cen[3], double r, double rho_p, const double u[3], const double w[3], int* id) {
    if (!c || !cen || !(r > 0.0) || !(rho_p > 0.0)) return LBM_EINVAL;
    if (c->started) return LBM_ESTATE;
    if ((int)c->sph_init.size() >= c->p.max_spheres) return LBM_EINVAL;
    Sphere s;
    std::memset(&s, 0, sizeof s);
    for (int k = 0; k < 3; k++) {
        s.x[k] = cen[k];
        s.x0[k] = cen[k];
        s.u[k] = u ? u[k] : 0.0;
        s.w[k] = w ? w[k] : 0.0;
    }
    s.R = r;
    s.rho = rho_p;
    if (id) *id = (int)c->sph_init.size();
    c->sph_init.push_back(s);
    return LBM_OK;
}

int lbm_add_spheres(lbm_ctx* c, int n, const double* cen, const double* r, const double* rho_p, const double* u,
                    const double* w, int* first_id) {
    if (!c || n < 0 || (n > 0 && (!cen || !r || !rho_p))) return LBM_EINVAL;
    if (c->started) return LBM_ESTATE;
    if ((long long)c->sph_init.size() + n > (long long)c->p.max_spheres) return LBM_EINVAL;
    for (int a = 0; a < n; a++)
        if (!(r[a] > 0.0) || !(rho_p[a] > 0.0)) return LBM_EINVAL;
    if (first_id) *first_id = (int)c->sph_init.size();
    for (int a = 0; a < n; a++) {
        const int rc = lbm_add_sphere(c, cen + 3 * a, r[a], rho_p[a], u ? u + 3 * a : nullptr, w ? w + 3 * a : nullptr, nullptr);
        if (rc) return rc;
    }
    return LBM_OK;
}

int lbm_step(lbm_ctx* c, int nsteps) {
    if (!c || nsteps < 0) return LBM_EINVAL;
    int rc;
    if (!c->started && (rc = first_step(c))) return rc;
    int left = nsteps;
    auto one = [&](bool timed) {
        const bool ov = c->pending;
        const bool split = ov && split_due_host(c, c->closed + 1);
        int r = enqueue_step(c, c->cur, c->stream, ov, timed, split);
        if (r) return r;
        c->launches += (uint64_t)step_launches(c->d, ov, split);
        if (ov) c->closed++;
        c->pending = true;
        c->cur ^= 1;
        return LBM_OK;
    };
    if (c->profiling) {
        for (; left > 0; left--)
            if ((rc = one(true))) return rc;
        return LBM_OK;
    }
    if (c->use_graph && nsteps >= 2) {
        // the graph holds two overlapped steps from grid 0: align the state to that first
        while (left > 0 && (!c->pending || c->cur == 1)) {
            if ((rc = one(false))) return rc;
            left--;
        }
        for (; left >= 2 && c->use_graph; left -= 2) {
            const bool s1 = split_due_host(c, c->closed + 1), s2 = split_due_host(c, c->closed + 2);
            const int v = (s1 ? 1 : 0) | (s2 ? 2 : 0);
            if (!c->graph_ready[v] && build_graph(c, v)) {
                c->use_graph = false;
                break;
            }
            if ((rc = cuda_fail(cudaGraphLaunch(c->graph[v], c->stream)))) return rc;
            c->launches += (uint64_t)step_launches(c->d, true, s1) + (uint64_t)step_launches(c->d, true, s2);
            c->closed += 2;
        }
    }
    for (; left > 0; left--)
        if ((rc = one(false))) return rc;
    return LBM_OK;
}

int lbm_forces(lbm_ctx* c, double* F, double* T, int n) {
    if (!c || n < 0 || (n > 0 && (!F || !T))) return LBM_EINVAL;
    if (!c->started) return LBM_ESTATE;
    if (int rf = flush(c)) return rf;
    if (n > c->d.nsph) return LBM_EINVAL;
    int rc = sync_tables(c);
    if (rc) return rc;
    for (int a = 0; a < n; a++)
        for (int k = 0; k < 3; k++) {
            F[3 * a + k] = c->sph_stage[a].F[k];
            T[3 * a + k] = c->sph_stage[a].T[k];
        }
    return status_code(c->sc_stage->status);
}

int lbm_spheres(lbm_ctx* c, double* x, double* u, double* w, int n) {
    if (!c || n < 0) return LBM_EINVAL;
    if (!c->started) return LBM_ESTATE;
    if (int rf = flush(c)) return rf;
    if (n > c->d.nsph) return LBM_EINVAL;
    int rc = sync_tables(c);
    if (rc) return rc;
    for (int a = 0; a < n; a++)
        for (int k = 0; k < 3; k++) {
            if (x) x[3 * a + k] = c->sph_stage[a].x[k];
            if (u) u[3 * a + k] = c->sph_stage[a].u[k];
            if (w) w[3 * a + k] = c->sph_stage[a].w[k];
        }
    return LBM_OK;
}

int lbm_lubrication(lbm_ctx* c, double* Fl, int n) {
    if (!c || n < 0 || (n > 0 && !Fl)) return LBM_EINVAL;
    if (!c->started) return LBM_ESTATE;
    if (int rf = flush(c)) return rf;
    if (n > c->d.nsph) return LBM_EINVAL;
    int rc = sync_tables(c);
    if (rc) return rc;
    for (int a = 0; a < n; a++)
        for (int k = 0; k < 3; k++) Fl[3 * a + k] = c->sph_stage[a].Fl[k];
    return LBM_OK;
}

int lbm_bubbles(lbm_ctx* c, double* V0, double* V, double* rho_g, int n) {
    if (!c || n < 0) return LBM_EINVAL;
    if (!c->started) return LBM_ESTATE;
    if (int rf = flush(c)) return rf;
    if (n > c->d.nbub) return LBM_EINVAL;
    int rc = sync_tables(c);
    if (rc) return rc;
    for (int b = 0; b < n; b++) {
        if (V0) V0[b] = c->bub_stage[b].V0;
        if (V) V[b] = c->bub_stage[b].V;
        if (rho_g) rho_g[b] = c->bub_stage[b].rho_g;
    }
    return LBM_OK;
}

int lbm_bubble_roots(lbm_ctx* c, int32_t* root, int n, int* n_merges) {
    if (!c || n < 0) return LBM_EINVAL;
    if (!c->started) return LBM_ESTATE;
    if (int rf = flush(c)) return rf;
    if (n > c->d.nbub) return LBM_EINVAL;
    int rc = sync_tables(c);
    if (rc) return rc;
    for (int b = 0; b < n; b++)
        if (root) root[b] = c->bub_stage[b].root;
    if (n_merges) *n_merges = (int)c->sc_stage->n_merges;
    return LBM_OK;
}


int lbm_bubble_splits(lbm_ctx* c, int* n_ids, int* n_splits) {
    if (!c) return LBM_EINVAL;
    if (!c->started) return LBM_ESTATE;
    if (int rf = flush(c)) return rf;
    int rc = sync_tables(c);
    if (rc) return rc;
    if (n_ids) *n_ids = c->d.split_every > 0 ? (int)c->sc_stage->nbub_hw : c->d.nbub;
    if (n_splits) *n_splits = (int)c->sc_stage->n_split;
    return LBM_OK;
}

int lbm_fields(lbm_ctx* c, float* rho, float* u, float* phi, uint8_t* flags) {
    if (!c) return LBM_EINVAL;
    if (!c->started) return LBM_ESTATE;
    if (int rf = flush(c)) return rf;
    launch_fields(c->d, c->cur, rho, u, phi, flags, c->stream);
    return launched(c, 1);
}

int lbm_export_state(lbm_ctx* c, float* f, uint8_t* flags, float* mass, float* phi, int32_t* owner, float* kappa) {
    if (!c) return LBM_EINVAL;
    if (!c->started) return LBM_ESTATE;
    if (int rf = flush(c)) return rf;
    launch_export(c->d, c->cur, f, flags, mass, phi, owner, kappa, c->stream);
    return launched(c, 1);
}

int lbm_mass_budget(lbm_ctx* c, double out[5]) {
    if (!c || !out) return LBM_EINVAL;
    if (!c->started) return LBM_ESTATE;
    if (int rf = flush(c)) return rf;
    int rc;
    if ((rc = cuda_fail(cudaMemsetAsync(&c->d.sc->mass, 0, sizeof(double), c->stream)))) return rc;
    launch_mass(c->d, c->cur, c->stream);
    if ((rc = launched(c, 1))) return rc;
    if ((rc = sync_tables(c))) return rc;
    const Scalars& sc = *c->sc_stage;
    out[0] = sc.mass + sc.pool;
    out[1] = sc.S_bb;
    out[2] = sc.S_cover;
    out[3] = sc.S_uncover;
    out[4] = sc.pool;
    return LBM_OK;
}

int lbm_status(lbm_ctx* c, uint32_t* status) {
    if (!c || !status) return LBM_EINVAL;
    if (!c->started) { *status = 0; return LBM_OK; }
    int rc = flush(c);
    if (rc) return rc;
    rc = sync_tables(c);
    if (rc) return rc;
    *status = c->sc_stage->status;
    return LBM_OK;
}

// the frozen liquid window the adjoint differentiates: FP32 storage, no bubbles, fixed spheres,
// no-slip or periodic faces
static int adjoint_ready(lbm_ctx* c) {
    if (!c->started) return LBM_ESTATE;
    if (c->p.storage != LBM_STORE_F32 || c->d.ngeo != 0 || c->p.sphere_mode != LBM_SPHERES_FIXED || c->d.special)
        return LBM_ESTATE;
    return flush(c);
}

int lbm_import_state(lbm_ctx* c, const float* f) {
    if (!c || !f) return LBM_EINVAL;
    int rc = adjoint_ready(c);
    if (rc) return rc;
    const size_t bytes = sizeof(float) * kQ * c->d.N;
    if ((rc = cuda_fail(cudaMemcpyAsync(c->d.f[c->cur], f, bytes, cudaMemcpyDeviceToDevice, c->stream)))) return rc;
    if (!c->d.rho[0]) return LBM_OK;
    launch_rho_of_grid(c->d, c->cur, c->stream);   // the densities of the imported PDFs
    return launched(c, 1);
}

int lbm_set_params(lbm_ctx* c, double tau, const double g[3]) {
    if (!c || !g || !(tau > 0.5) || !(tau < 100.0)) return LBM_EINVAL;
    for (int k = 0; k < 3; k++)
        if (!std::isfinite(g[k])) return LBM_EINVAL;
    c->p.tau = tau;
    for (int k = 0; k < 3; k++) c->p.g[k] = g[k];
    if (!c->started) return LBM_OK;   // first_step takes them from p
    int rc = flush(c);   // the last step's end-of-step kernels run with the parameters it had
    if (rc) return rc;
    if ((rc = cuda_fail(cudaStreamSynchronize(c->stream)))) return rc;
    Dev& d = c->d;
    d.tau = (float)tau;
    const double lp = -1.0 / tau;
    d.lp = (float)lp;
    d.lm = (float)(1.0 / ((3.0 / 16.0) / (1.0 / lp + 0.5) - 0.5));
    for (int k = 0; k < 3; k++) { d.g[k] = (float)g[k]; d.gd[k] = g[k]; }
    set_collision_consts(d);
    // the step graphs hold the kernels' arguments: instantiate them again at the next step
    for (int v = 0; v < 4; v++)
        if (c->graph_ready[v]) {
            cudaGraphExecDestroy(c->graph[v]);
            c->graph_ready[v] = false;
        }
    return LBM_OK;
}

int lbm_objective(lbm_ctx* c, const double jdir[3]) {
    if (!c) return LBM_EINVAL;
    if (!c->started) return LBM_ESTATE;
    int rc = flush(c);   // the last step's force belongs to no window opened now
    if (rc) return rc;
    c->obj_stage.on = jdir ? 1u : 0u;
    for (int k = 0; k < 3; k++) c->obj_stage.j[k] = jdir ? jdir[k] : 0.0;
    Scalars* sc = c->d.sc;
    cudaStream_t s = c->stream;
    const double zero = 0.0;
    if ((rc = cuda_fail(cudaMemcpyAsync(&sc->obj_on, &c->obj_stage.on, sizeof(uint32_t), cudaMemcpyHostToDevice, s)))) return rc;
    if ((rc = cuda_fail(cudaMemcpyAsync(sc->obj_j, c->obj_stage.j, sizeof(double) * 3, cudaMemcpyHostToDevice, s)))) return rc;
    if ((rc = cuda_fail(cudaMemcpyAsync(&sc->obj, &zero, sizeof(double), cudaMemcpyHostToDevice, s)))) return rc;
    c->h2d_bytes += sizeof(uint32_t) + 4 * sizeof(double);
    return cuda_fail(cudaStreamSynchronize(s));   // (the host sources are gone after return)
}

int lbm_objective_read(lbm_ctx* c, double* J) {
    if (!c || !J) return LBM_EINVAL;
    if (!c->started) return LBM_ESTATE;
    int rc = flush(c);   // the last step's force
    if (rc) return rc;
    if ((rc = cuda_fail(cudaMemcpyAsync(J, &c->d.sc->obj, sizeof(double), cudaMemcpyDeviceToHost, c->stream)))) return rc;
    c->d2h_bytes += sizeof(double);
    return cuda_fail(cudaStreamSynchronize(c->stream));
}

int lbm_forward_frozen(lbm_ctx* c, const float* f_in, float* f_out) {
    if (!c || !f_in || !f_out || f_in == f_out) return LBM_EINVAL;
    int rc = adjoint_ready(c);
    if (rc) return rc;
    launch_frozen_forward(c->d, f_in, f_out, c->stream, c->side, c->fork, c->join);
    return launched(c, 2);
}

int lbm_adjoint_step(lbm_ctx* c, const float* f_fwd, const float* adj_in, float* adj_out, const double jdir[3],
                     int accumulate, double dJdg[3], double* dJdtau) {
    if (!c || !f_fwd || !adj_in || !adj_out || !jdir || adj_in == adj_out || (!dJdg) != (!dJdtau)) return LBM_EINVAL;
    int rc = adjoint_ready(c);
    if (rc) return rc;
    cudaStream_t s = c->stream;
    if (!accumulate && (rc = cuda_fail(cudaMemsetAsync(c->adj_part, 0, sizeof(double) * 5 * kAdjSlots, s)))) return rc;
    const float jd[3] = {(float)jdir[0], (float)jdir[1], (float)jdir[2]};
    launch_adjoint(c->d, f_fwd, adj_in, adj_out, c->adj_srho, jd, c->adj_part, c->moving_walls, s, c->side, c->fork,
                   c->join);
    if ((rc = launched(c, c->moving_walls ? 3 : 2))) return rc;
    if (!dJdg) return LBM_OK;
    double part[5 * kAdjSlots];
    if ((rc = cuda_fail(cudaMemcpyAsync(part, c->adj_part, sizeof part, cudaMemcpyDeviceToHost, s)))) return rc;
    c->d2h_bytes += sizeof part;
    if ((rc = cuda_fail(cudaStreamSynchronize(s)))) return rc;
    double sum[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < kAdjSlots; k++)
        for (int m = 0; m < 5; m++) sum[m] += part[5 * k + m];
    // lambda_+ = -1/tau; lambda_- = 1/B, B = (3/16)/A - 1/2, A = 1/lambda_+ + 1/2 = 1/2 - tau
    const double tau = c->p.tau, A = 0.5 - tau, B = (3.0 / 16.0) / A - 0.5;
    const double dlp = 1.0 / (tau * tau), dlm = -(3.0 / 16.0) / (A * A * B * B);
    for (int k = 0; k < 3; k++) dJdg[k] = sum[k];
    *dJdtau = sum[3] * dlp + sum[4] * dlm;
    return LBM_OK;
}

int lbm_profile(lbm_ctx* c, int on) {
    if (!c) return LBM_EINVAL;
    if (on && !c->ev_ready) {
        for (int k = 0; k < 4 * 64; k++)
            if (cudaEventCreate(&c->ev[k]) != cudaSuccess) return LBM_ECUDA;
        c->ev_ready = true;
    }
    if (!on && c->ev_ready)
        for (int k = 0; k < 64; k++) prof_collect(c, k);
    c->profiling = on != 0;
    return LBM_OK;
}

int lbm_profile_read(lbm_ctx* c, double ms[2], uint64_t* sweeps) {
    if (!c || !ms || !sweeps) return LBM_EINVAL;
    if (c->ev_ready)
        for (int k = 0; k < 64; k++) prof_collect(c, k);
    ms[0] = c->bulk_ms;
    ms[1] = c->rest_ms;
    *sweeps = c->sweeps;
    c->bulk_ms = c->rest_ms = 0.0;
    c->sweeps = 0;
    return LBM_OK;
}

int lbm_copy_bytes(lbm_ctx* c, uint64_t* h2d, uint64_t* d2h) {
    if (!c || !h2d || !d2h) return LBM_EINVAL;
    *h2d = c->h2d_bytes;
    *d2h = c->d2h_bytes;
    return LBM_OK;
}

int lbm_launch_count(lbm_ctx* c, uint64_t* launches) {
    if (!c || !launches) return LBM_EINVAL;
    *launches = c->launches;
    return LBM_OK;
}

int lbm_destroy(lbm_ctx* c) {
    if (!c) return LBM_EINVAL;
    for (int v = 0; v < 4; v++)
        if (c->graph_ready[v]) cudaGraphExecDestroy(c->graph[v]);
    if (c->ev_ready)
        for (int k = 0; k < 4 * 64; k++) cudaEventDestroy(c->ev[k]);
    if (c->side_ready) {
        // nothing of this simulation may still run once the caller frees the arena
        cudaStreamSynchronize(c->side);
        cudaStreamSynchronize(c->side2);
        cudaStreamSynchronize(c->epi);
        cudaStreamSynchronize(c->links);
        cudaEventDestroy(c->fork);
        cudaEventDestroy(c->join);
        cudaEventDestroy(c->fork2);
        cudaEventDestroy(c->join2);
        cudaEventDestroy(c->fork3);
        cudaEventDestroy(c->join3);
        cudaStreamDestroy(c->side);
        cudaStreamDestroy(c->epi);
        cudaStreamDestroy(c->links);
        cudaEventDestroy(c->fork4);
        cudaEventDestroy(c->join4);
        cudaStreamDestroy(c->side2);
        cudaEventDestroy(c->join5);
    }
    std::free(c->sph_stage);
    std::free(c->sc_stage);
    std::free(c->bub_stage);
    delete c;
    return LBM_OK;
}

const char* lbm_strerror(int code) {
    switch (code) {
        case LBM_OK: return "ok";
        case LBM_EINVAL: return "invalid argument";
        case LBM_ESTATE: return "call not allowed in the current state";
        case LBM_ECUDA: return "CUDA runtime error";
        case LBM_EUNSTABLE: return "density became non-positive or NaN";
        case LBM_EOVERFLOW: return "worklist or neighbour bin overflow";
        case LBM_EMERGE: return "more pairs of bubbles met in one step than the merge table holds";
        case LBM_ESPLIT: return "a bubble could not be split (no free row in the bubble table, or the part table is full)";
        default: return "unknown error";
    }
}

}  // extern "C"
