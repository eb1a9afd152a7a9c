// lbm_batch_api.cu -- the batch entry points of include/gblbm.h: set-up of
// many independent domains in shared device arenas, the tile and argument
// tables of the batched kernels, the step loop (CUDA graphs), the launch
// tuner and read-back.  All arithmetic of the method runs in the kernels of
// lbm_setup.cu, lbm_batch.cu and lbm_link.cu.
//
// Two population buffers alternate: step t reads buffer t % 2 and writes the
// other; the link kernel of step t runs after the collide-stream kernel on the
// same stream, so the buffer of step t-1 is free again once step t is done.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm_batch.cuh"
#include "lbm_host.h"
#include "lbm_internal.cuh"

using namespace gblbm;

namespace {

// Tiles of a launch ordered by code path (1: interior, edge, body; 2: body,
// edge, interior, so that the slower paths do not form the launch's tail) or
// left in domain order (0), per storage (a tuning knob; measured on the
// 256-domain recipe with 128-thread CTAs: FP16 deviations 0.480 in domain
// order, 0.603 in order 1, 0.609 in order 2; FP32 dev 0.879 in domain order,
// 0.857 in order 2, so only FP16 sorts).
#ifndef GBLBM_BATCH_PATH_ORDER_F16
#define GBLBM_BATCH_PATH_ORDER_F16 2
#endif
#ifndef GBLBM_BATCH_PATH_ORDER_F32
#define GBLBM_BATCH_PATH_ORDER_F32 0
#endif
constexpr int BATCH_GRAPH_STEPS = 16;  // steps per captured graph (even: ends on the start buffer)
constexpr int BATCH_GRID_CHOICES[] = {1, 2, 3, 4, 6, 8};  // persistent CTAs per SM tried by the tuner

struct Domain {
    int nx = 0, ny = 0, pitch = 0;
    long long plane = 0;
    double tau = 0;
    int cv[4] = {0, 0, 0, 0};
    long long pop_off = 0;    // elements into each population arena
    long long node_off = 0;   // elements into the nbits arena (plane-sized)
    long long mask_off = 0;   // bytes into the mask arena (nx*ny)
    long long row_off = 0;    // entries into the u_row arena (ny)
    long long inlet_off = 0;  // elements into the inlet arena (9*ny)
    long long link_off = 0, nlinks = 0;
    long long n_bnodes = 0;   // boundary fluid nodes (at link_off in the boundary-node arena)
    double link_base[2] = {0, 0}, flux_base[2] = {0, 0};
    int cvt[BATCH_SHAPES][4];
    int n_cv_tiles[BATCH_SHAPES];
    long long cvp_off[BATCH_SHAPES];  // partial rows into the partials arena
    int tiles_x[BATCH_SHAPES];
    long long tile_base[BATCH_SHAPES];  // first tile in the batch's tile order
    long long cv_base[BATCH_SHAPES];    // first control-volume tile in the batch's order
};

}  // namespace

struct lbm_batch {
    int n = 0, storage = 0, periodic = 0, record_series = 1;
    double rho0 = 1;
    size_t elem = 4;
    int sm_count = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    lbm_alloc_fn alloc_fn = nullptr;
    lbm_free_fn free_fn = nullptr;
    void *alloc_user = nullptr;
    std::vector<Domain> dom;
    long long nodes = 0;
    // device arenas
    void *pop_base[2] = {nullptr, nullptr};
    char *pop[2] = {nullptr, nullptr};
    uint8_t *mask_d = nullptr;
    uint16_t *nbits = nullptr;
    double *u_row = nullptr;
    void *inlet = nullptr;
    int32_t *links = nullptr;
    int32_t *bnodes = nullptr;        // boundary fluid nodes of every domain, at its link offset
    double *partials = nullptr;       // [max over shapes of the partial rows][CV_PARTIAL]
    double *tune_partials = nullptr;  // the tuner's scratch copy of it
    int4 *checked[BATCH_SHAPES] = {nullptr, nullptr, nullptr};     // tile table, batch order
    long long n_tiles[BATCH_SHAPES] = {0, 0, 0};
    int4 *checked_cv[BATCH_SHAPES] = {nullptr, nullptr, nullptr};  // control-volume tiles
    long long n_cv_entries[BATCH_SHAPES] = {0, 0, 0};
    LinkArgs *largs = nullptr;  // [BATCH_SHAPES][3][n]: slots 0/1 = source buffer, 2 = first step (pre-collision)
    double *series = nullptr;   // [series_cap][n][SERIES_ROW]
    long long series_cap = 0;
    double *carry = nullptr;    // [n][8]
    long long *step_ctr = nullptr;
    unsigned int *ticket = nullptr;
    int *status = nullptr;      // [n][2]: flags, first bad step
    int *tune_status = nullptr; // [n][2]
    int *bstatus = nullptr;     // [2]: batch flags (bit 4: series row outside the buffer)
    // state
    long long t = 0, drtt_ready = 0;
    int cur = 0;
    int shape = 0, ctas_per_sm = 0;
    cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    long long launches = 0;
    std::string err;
};

namespace {

thread_local std::string g_batch_err;

lbm_status berr(lbm_batch *b, lbm_status code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (b)
        b->err = buf;
    else
        g_batch_err = buf;
    return code;
}

lbm_status bcuda(lbm_batch *b, cudaError_t e, const char *what)
{
    return berr(b, LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define BCK(b, expr, what)                                   \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return bcuda(b, e_, what);    \
    } while (0)

void *bdev_alloc(lbm_batch *b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (b->alloc_fn) return b->alloc_fn(bytes, (void *)b->stream, b->alloc_user);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void bdev_free(lbm_batch *b, void *p)
{
    if (!p) return;
    if (b->free_fn)
        b->free_fn(p, b->alloc_user);
    else
        cudaFree(p);
}

void drop_graphs(lbm_batch *b)
{
    for (int c = 0; c < 2; ++c)
        for (int k = 0; k < 2; ++k)
            if (b->graph[c][k]) {
                cudaGraphExecDestroy(b->graph[c][k]);
                b->graph[c][k] = nullptr;
            }
}

void free_all(lbm_batch *b)
{
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    void *bufs[] = {b->pop_base[0], b->pop_base[1], b->mask_d, b->nbits, b->u_row, b->inlet,
                    b->links, b->bnodes, b->partials, b->tune_partials, b->checked[0], b->checked[1],
                    b->checked[2], b->checked_cv[0], b->checked_cv[1], b->checked_cv[2], b->largs,
                    b->series, b->carry, b->step_ctr, b->ticket, b->status, b->tune_status,
                    b->bstatus};
    for (void *p : bufs) bdev_free(b, p);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

int n_chunks(const lbm_batch *b) { return (b->n + MAX_BATCH_DOMAINS - 1) / MAX_BATCH_DOMAINS; }

// The kernel parameter of one collide-stream launch: tile shape s, domains of
// chunk c, reading buffer src (-1: the first step, whose state is
// pre-collision in buffer 0).  cv_only: the control-volume tiles only (the
// momentum pass); tune: partial sums and flags into the tuner's scratch.
void make_params(const lbm_batch *b, int s, int src, int c, bool cv_only, bool tune, BatchParams &p)
{
    memset(&p, 0, sizeof(p));
    const int from = src < 0 ? 0 : src;
    p.src = b->pop[from];
    p.dst = b->pop[1 - from];
    p.nbits = b->nbits;
    p.inlet = (const char *)b->inlet;
    p.partials = tune ? b->tune_partials : b->partials;
    p.status = tune ? b->tune_status : b->status;
    p.step_ctr = b->step_ctr;
    const int d0 = c * MAX_BATCH_DOMAINS;
    const int d1 = d0 + MAX_BATCH_DOMAINS < b->n ? d0 + MAX_BATCH_DOMAINS : b->n;
    p.n_dom = d1 - d0;
    p.dom_base = d0;
    const long long base = cv_only ? b->dom[d0].cv_base[s] : b->dom[d0].tile_base[s];
    p.tiles = (cv_only ? b->checked_cv[s] : b->checked[s]) + base;
    long long end = base;
    for (int d = d0; d < d1; ++d) {
        const Domain &m = b->dom[d];
        BatchDomain &q = p.dom[d - d0];
        if (b->storage == LBM_F64)
            q.omega = 1.0 / m.tau;
        else
            q.omega_f = (float)(1.0 / m.tau);  // rounded as the single-domain handles round it
        q.pop_off64 = (int)(m.pop_off / 64);
        q.node_off64 = (int)(m.node_off / 64);
        q.inlet_off64 = (int)(m.inlet_off / 64);
        q.part_off = (int)m.cvp_off[s];
        q.nx = m.nx;
        q.ny = m.ny;
        q.tiles_x = m.tiles_x[s];
        for (int j = 0; j < 4; ++j) {
            q.cv[j] = (short)m.cv[j];
            q.cvt[j] = (short)m.cvt[s][j];
        }
        const int tiles_y = (m.ny + batch_tr(b->storage, s) - 1) / batch_tr(b->storage, s);
        end = (cv_only ? m.cv_base[s] + m.n_cv_tiles[s] : m.tile_base[s] + (long long)m.tiles_x[s] * tiles_y);
    }
    p.n_tiles = (int)(end - base);
    p.periodic = b->periodic;
    p.precollision = src < 0 ? 1 : 0;
    p.cv_only = cv_only ? 1 : 0;
    p.rho0 = b->rho0;
    p.rho0_f = (float)b->rho0;
}

LinkArgs link_args(const lbm_batch *b, int d, int s, int src)
{
    const Domain &m = b->dom[d];
    const int from = src < 0 ? 0 : src;
    LinkArgs a;
    memset(&a, 0, sizeof(a));
    a.src = b->pop[from] + m.pop_off * (long long)b->elem;
    a.dst = b->pop[1 - from] + m.pop_off * (long long)b->elem;
    a.nbits = b->nbits + m.node_off;
    a.links = b->links + m.link_off;
    a.nlinks = m.nlinks;
    a.partials = b->partials + CV_PARTIAL * m.cvp_off[s];
    a.n_partials = m.n_cv_tiles[s];
    a.n_ctas = 1;
    a.status = b->bstatus;
    a.carry = b->carry + 8 * d;
    a.step_ctr = b->step_ctr;
    a.plane = m.plane;
    a.nx = m.nx;
    a.ny = m.ny;
    a.pitch = m.pitch;
    a.periodic = b->periodic;
    a.precollision = src < 0 ? 1 : 0;
    a.record_series = b->record_series;
    a.rho0 = b->rho0;
    a.visc = 1.0 - 0.5 / m.tau;
    a.visc_f = (float)a.visc;
    memcpy(a.link_base, m.link_base, sizeof(a.link_base));
    memcpy(a.flux_base, m.flux_base, sizeof(a.flux_base));
    return a;
}

// Table index of (shape, slot, domain); slot 0/1 = source buffer, 2 = first step.
size_t tix(const lbm_batch *b, int s, int slot) { return ((size_t)s * 3 + slot) * b->n; }

lbm_status upload_tables(lbm_batch *b)
{
    std::vector<LinkArgs> la((size_t)BATCH_SHAPES * 3 * b->n);
    for (int s = 0; s < BATCH_SHAPES; ++s)
        for (int slot = 0; slot < 3; ++slot)
            for (int d = 0; d < b->n; ++d) la[tix(b, s, slot) + d] = link_args(b, d, s, slot == 2 ? -1 : slot);
    BCK(b, cudaMemcpyAsync(b->largs, la.data(), sizeof(LinkArgs) * la.size(), cudaMemcpyHostToDevice,
                           b->stream),
        "H2D link tables");
    BCK(b, cudaStreamSynchronize(b->stream), "sync");
    return LBM_OK;
}

lbm_status ensure_series(lbm_batch *b, long long need)
{
    if (!b->record_series) need = 2;
    if (need <= b->series_cap) return LBM_OK;
    long long cap = b->series_cap ? b->series_cap : 1024;
    while (cap < need) cap *= 2;
    const size_t row = sizeof(double) * SERIES_ROW * b->n;
    double *ns = (double *)bdev_alloc(b, row * cap);
    if (!ns) return berr(b, LBM_ENOMEM, "force series: allocation of %lld steps failed", cap);
    BCK(b, cudaMemsetAsync(ns, 0, row * cap, b->stream), "memset series");
    if (b->series)
        BCK(b, cudaMemcpyAsync(ns, b->series, row * b->series_cap, cudaMemcpyDeviceToDevice, b->stream),
            "copy series");
    BCK(b, cudaStreamSynchronize(b->stream), "sync");
    bdev_free(b, b->series);
    b->series = ns;
    b->series_cap = cap;
    drop_graphs(b);  // captured link launches hold the old series pointer
    return LBM_OK;
}

// Grid of the collide-stream launch: 0 = one CTA per tile, else persistent.
int grid_of(const lbm_batch *b) { return b->ctas_per_sm > 0 ? b->ctas_per_sm * b->sm_count : 0; }

// The collide-stream launches (one per chunk of domains) of a step reading
// buffer src, or of the momentum pass.
cudaError_t launch_collide(lbm_batch *b, int src, bool cv_only, bool tune, int shape, int grid)
{
    BatchParams *p = new (std::nothrow) BatchParams;
    if (!p) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < n_chunks(b) && e == cudaSuccess; ++c) {
        make_params(b, shape, src, c, cv_only, tune, *p);
        e = launch_collide_stream_batch(b->storage, shape, cv_only, *p, cv_only ? 0 : grid, b->stream);
        b->launches += 1;
    }
    delete p;
    return e;
}

BatchLinkArgs link_launch_args(lbm_batch *b, int slot, bool drtt_only)
{
    BatchLinkArgs bl;
    bl.args = b->largs + tix(b, b->shape, slot);
    bl.series = b->series;
    bl.series_rows = b->series_cap;
    bl.n_domains = b->n;
    bl.keep_all = b->record_series;
    bl.drtt_only = drtt_only ? 1 : 0;
    bl.step_ctr = b->step_ctr;
    bl.ticket = b->ticket;
    bl.status = b->bstatus;
    return bl;
}

// One step reading buffer src (-1: the first step from the pre-collision state).
cudaError_t launch_step(lbm_batch *b, int src)
{
    cudaError_t e = launch_collide(b, src, false, false, b->shape, grid_of(b));
    if (e != cudaSuccess) return e;
    e = launch_link_force_batch(b->storage, link_launch_args(b, src < 0 ? 2 : src, false), b->stream);
    b->launches += 1;
    return e;
}

lbm_status build_graph(lbm_batch *b, int c, int k)
{
    const int steps = k == 0 ? BATCH_GRAPH_STEPS : 2;
    cudaGraph_t g = nullptr;
    BCK(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    const long long saved = b->launches;
    cudaError_t le = cudaSuccess;
    int src = c;
    for (int s = 0; s < steps && le == cudaSuccess; ++s) {
        le = launch_step(b, src);
        src = 1 - src;
    }
    b->launches = saved;
    cudaError_t ee = cudaStreamEndCapture(b->stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(b, le, "capture batch steps");
    }
    if (ee != cudaSuccess) return bcuda(b, ee, "end capture");
    cudaError_t ie = cudaGraphInstantiate(&b->graph[c][k], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return bcuda(b, ie, "instantiate graph");
    return LBM_OK;
}

// Complete DRTT(T-1) of every domain: a momentum-only pass over the control-
// volume tiles (J(T) on the pre-collision state), then the link kernel's
// DRTT-only mode.
lbm_status finalize_drtt(lbm_batch *b)
{
    if (b->drtt_ready >= b->t) return LBM_OK;
    if (b->t < 1) return berr(b, LBM_ESTATE, "DRTT needs at least one step");
    BCK(b, launch_collide(b, b->cur, true, false, b->shape, 0), "momentum pass");
    BCK(b, launch_link_force_batch(b->storage, link_launch_args(b, b->cur, true), b->stream), "DRTT finalize");
    BCK(b, cudaStreamSynchronize(b->stream), "sync");
    b->launches += 1;
    b->drtt_ready = b->t;
    return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(const lbm_domain *domains, int n, const lbm_bc *bc_in, lbm_batch **out)
{
    if (!out) return berr(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!domains || n < 1) return berr(nullptr, LBM_EINVAL, "need n >= 1 domains (got %d)", n);
    lbm_bc bc;
    if (bc_in)
        bc = *bc_in;
    else
        lbm_bc_default(&bc);
    if (bc.kind != LBM_BC_CHANNEL && bc.kind != LBM_BC_PERIODIC)
        return berr(nullptr, LBM_EINVAL, "unknown boundary kind %d", bc.kind);
    if (bc.storage < LBM_F64 || bc.storage > LBM_F16_DEV)
        return berr(nullptr, LBM_EINVAL, "unknown storage %d", bc.storage);
    if (!(bc.rho0 > 0) || !std::isfinite(bc.rho0))
        return berr(nullptr, LBM_EINVAL, "rho0 must be finite and > 0");
    if (bc.body_force[0] != 0.0 || bc.body_force[1] != 0.0)
        return berr(nullptr, LBM_EINVAL, "a batch takes no body force");
    if (bc.kernel != 0) return berr(nullptr, LBM_EINVAL, "a batch runs the direct kernel only (kernel = 0)");
    if ((bc.alloc == nullptr) != (bc.free == nullptr))
        return berr(nullptr, LBM_EINVAL, "alloc and free must be given together");
    const int periodic = bc.kind == LBM_BC_PERIODIC;
    std::vector<Domain> dom(n);
    for (int d = 0; d < n; ++d) {
        const lbm_domain &in = domains[d];
        const std::string why =
            check_domain(in.mask, in.nx, in.ny, in.tau, in.u_in, in.n_u_in, periodic, in.cv, dom[d].cv);
        if (!why.empty()) return berr(nullptr, LBM_EINVAL, "domain %d: %s", d, why.c_str());
        if (in.nx > MAX_BATCH_SIDE || in.ny > MAX_BATCH_SIDE)
            return berr(nullptr, LBM_EINVAL, "domain %d: %dx%d: a batch domain has at most %d nodes a side", d,
                        in.nx, in.ny, MAX_BATCH_SIDE);
    }
    int ndev = 0;
    cudaError_t de = cudaGetDeviceCount(&ndev);
    if (de != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return berr(nullptr, LBM_ECUDA, "no CUDA device: %s", cudaGetErrorString(de));
    }

    lbm_batch *b = new (std::nothrow) lbm_batch;
    if (!b) return berr(nullptr, LBM_ENOMEM, "host allocation failed");
    b->n = n;
    b->storage = bc.storage;
    b->periodic = periodic;
    b->record_series = bc.record_series ? 1 : 0;
    b->rho0 = bc.rho0;
    b->elem = storage_bytes(bc.storage);
    b->alloc_fn = bc.alloc;
    b->free_fn = bc.free;
    b->alloc_user = bc.alloc_user;
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            b->sm_count = sms;
        else
            cudaGetLastError();
    }
    auto fail = [&](lbm_status st) {
        g_batch_err = b->err;
        free_all(b);
        delete b;
        return st;
    };
    if (bc.cuda_stream) {
        b->stream = (cudaStream_t)bc.cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            b->stream = nullptr;
            return fail(bcuda(b, e, "stream create"));
        }
        b->own_stream = true;
    }
#define BCKC(expr, what)                                         \
    do {                                                         \
        cudaError_t e_ = (expr);                                 \
        if (e_ != cudaSuccess) return fail(bcuda(b, e_, what));  \
    } while (0)
#define BALLOC(ptr, type, bytes)                                                                   \
    do {                                                                                           \
        ptr = (type)bdev_alloc(b, (bytes));                                                        \
        if (!ptr) return fail(berr(b, LBM_ENOMEM, "device allocation of %zu bytes failed", (size_t)(bytes))); \
    } while (0)

    // layout of the arenas
    long long pop_elems = 0, node_elems = 0, mask_bytes = 0, rows = 0, inlet_elems = 0;
    long long cvp[BATCH_SHAPES] = {0, 0, 0};
    for (int d = 0; d < n; ++d) {
        Domain &m = dom[d];
        const lbm_domain &in = domains[d];
        m.nx = in.nx;
        m.ny = in.ny;
        m.tau = in.tau;
        m.pitch = (in.nx + PITCH_ALIGN - 1) / PITCH_ALIGN * PITCH_ALIGN;
        m.plane = (long long)in.ny * m.pitch;
        m.pop_off = pop_elems;
        pop_elems += 9 * m.plane;
        m.node_off = node_elems;
        node_elems += m.plane;
        m.mask_off = mask_bytes;
        mask_bytes += ((long long)in.nx * in.ny + 255) / 256 * 256;
        m.row_off = rows;
        rows += in.ny;
        m.inlet_off = inlet_elems;
        inlet_elems += ((9LL * in.ny) + 63) / 64 * 64;
        for (int s = 0; s < BATCH_SHAPES; ++s) {
            cv_tile_rect(m.cv, m.nx, m.ny, batch_tx(s), batch_tr(b->storage, s), m.cvt[s]);
            m.n_cv_tiles[s] = (m.cvt[s][1] - m.cvt[s][0] + 1) * (m.cvt[s][3] - m.cvt[s][2] + 1);
            m.cvp_off[s] = cvp[s];
            cvp[s] += m.n_cv_tiles[s];
        }
        if (b->storage == LBM_F32_DEV || b->storage == LBM_F16_DEV)
            base_sums(in.mask, m.nx, m.ny, periodic, m.cv, b->rho0, m.link_base, m.flux_base);
        b->nodes += (long long)m.nx * m.ny;
    }
    b->dom = dom;
    long long cvp_max = 0;
    for (int s = 0; s < BATCH_SHAPES; ++s) cvp_max = cvp[s] > cvp_max ? cvp[s] : cvp_max;

    const size_t guard_front = 256, guard_back = 2048;
    const size_t pop_bytes = (size_t)pop_elems * b->elem;
    for (int c = 0; c < 2; ++c) {
        BALLOC(b->pop_base[c], void *, guard_front + pop_bytes + guard_back);
        b->pop[c] = (char *)b->pop_base[c] + guard_front;
        if ((uintptr_t)b->pop_base[c] & 15)
            return fail(berr(b, LBM_EINVAL, "the allocator returned a pointer that is not 16-byte aligned"));
        BCKC(cudaMemsetAsync(b->pop_base[c], 0, guard_front + pop_bytes + guard_back, b->stream), "memset");
    }
    BALLOC(b->mask_d, uint8_t *, mask_bytes);
    BALLOC(b->nbits, uint16_t *, sizeof(uint16_t) * node_elems);
    BALLOC(b->u_row, double *, sizeof(double) * rows);
    BALLOC(b->inlet, void *, (size_t)inlet_elems * b->elem);
    BALLOC(b->partials, double *, sizeof(double) * CV_PARTIAL * (cvp_max > 0 ? cvp_max : 1));
    BALLOC(b->tune_partials, double *, sizeof(double) * CV_PARTIAL * (cvp_max > 0 ? cvp_max : 1));
    BALLOC(b->largs, LinkArgs *, sizeof(LinkArgs) * BATCH_SHAPES * 3 * n);
    BALLOC(b->carry, double *, sizeof(double) * 8 * n);
    BALLOC(b->step_ctr, long long *, sizeof(long long));
    BALLOC(b->ticket, unsigned int *, sizeof(unsigned int));
    BALLOC(b->status, int *, sizeof(int) * 2 * n);
    BALLOC(b->tune_status, int *, sizeof(int) * 2 * n);
    BALLOC(b->bstatus, int *, sizeof(int) * 2);
    BCKC(cudaMemsetAsync(b->nbits, 0, sizeof(uint16_t) * node_elems, b->stream), "memset");
    BCKC(cudaMemsetAsync(b->partials, 0, sizeof(double) * CV_PARTIAL * (cvp_max > 0 ? cvp_max : 1), b->stream),
         "memset");
    BCKC(cudaMemsetAsync(b->carry, 0, sizeof(double) * 8 * n, b->stream), "memset");
    BCKC(cudaMemsetAsync(b->step_ctr, 0, sizeof(long long), b->stream), "memset");
    BCKC(cudaMemsetAsync(b->ticket, 0, sizeof(unsigned int), b->stream), "memset");
    BCKC(cudaMemsetAsync(b->bstatus, 0, sizeof(int) * 2, b->stream), "memset");
    {
        std::vector<int> st0(2 * n);
        for (int d = 0; d < n; ++d) {
            st0[2 * d] = 0;
            st0[2 * d + 1] = INT_MAX;
        }
        BCKC(cudaMemcpyAsync(b->status, st0.data(), sizeof(int) * 2 * n, cudaMemcpyHostToDevice, b->stream),
             "H2D status");
        BCKC(cudaStreamSynchronize(b->stream), "sync");
    }
    {
        lbm_status st = ensure_series(b, 1024);
        if (st != LBM_OK) return fail(st);
    }

    // per domain: mask, inlet rows, neighbour bits, initial state, link counts
    const cudaStream_t s = b->stream;
    std::vector<int> nb(n);
    long long blk_total = 0;
    for (int d = 0; d < n; ++d) {
        nb[d] = link_blocks(dom[d].nx, dom[d].ny);
        blk_total += nb[d];
    }
    int *blk = nullptr;
    long long *totals_d = nullptr;
    BALLOC(blk, int *, sizeof(int) * blk_total);
    totals_d = (long long *)bdev_alloc(b, sizeof(long long) * n);
    if (!totals_d) {
        bdev_free(b, blk);
        return fail(berr(b, LBM_ENOMEM, "device allocation failed"));
    }
    auto fail_scratch = [&](lbm_status st) {
        cudaStreamSynchronize(s);
        bdev_free(b, blk);
        bdev_free(b, totals_d);
        return fail(st);
    };
    std::vector<double> urow;
    cudaError_t e = cudaSuccess;
    long long blk_off = 0;
    for (int d = 0; d < n && e == cudaSuccess; ++d) {
        const Domain &m = b->dom[d];
        const lbm_domain &in = domains[d];
        urow.assign(m.ny, 0.0);
        for (int y = 0; y < m.ny; ++y) urow[y] = in.n_u_in == 1 ? in.u_in[0] : in.u_in[y];
        e = cudaMemcpyAsync(b->mask_d + m.mask_off, in.mask, (size_t)m.nx * m.ny, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->u_row + m.row_off, urow.data(), sizeof(double) * m.ny, cudaMemcpyHostToDevice, s);
        // (pageable sources: the copies are staged before the calls return, so urow may be reused)
        if (e == cudaSuccess)
            e = launch_node_bits(b->mask_d + m.mask_off, b->nbits + m.node_off, m.nx, m.ny, m.pitch, periodic, s);
        if (e == cudaSuccess)
            e = launch_init(b->storage, b->pop[0] + m.pop_off * (long long)b->elem, m.plane, b->mask_d + m.mask_off,
                            m.nx, m.ny, m.pitch, b->u_row + m.row_off, b->rho0,
                            (char *)b->inlet + m.inlet_off * (long long)b->elem, s, in.n_u_in == 1);
        if (e == cudaSuccess)
            e = launch_link_count(b->nbits + m.node_off, m.nx, m.ny, m.pitch, blk + blk_off, nb[d], s);
        if (e == cudaSuccess) e = launch_scan_blocks(blk + blk_off, nb[d], totals_d + d, s);
        blk_off += nb[d];
        b->launches += 4;
    }
    std::vector<long long> totals(n, 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(totals.data(), totals_d, sizeof(long long) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_scratch(bcuda(b, e, "domain set-up"));
    long long links_total = 0;
    for (int d = 0; d < n; ++d) {
        b->dom[d].link_off = links_total;
        b->dom[d].nlinks = totals[d];
        links_total += totals[d];
    }
    b->links = (int32_t *)bdev_alloc(b, sizeof(int32_t) * (links_total > 0 ? links_total : 1));
    if (!b->links) return fail_scratch(berr(b, LBM_ENOMEM, "device allocation of the link lists failed"));
    blk_off = 0;
    for (int d = 0; d < n && e == cudaSuccess; ++d) {
        const Domain &m = b->dom[d];
        e = launch_link_scatter(b->nbits + m.node_off, m.nx, m.ny, m.pitch, blk + blk_off,
                                b->links + m.link_off, m.nlinks, s);
        blk_off += nb[d];
        b->launches += 1;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_scratch(bcuda(b, e, "link lists"));
    b->bnodes = (int32_t *)bdev_alloc(b, sizeof(int32_t) * (links_total > 0 ? links_total : 1));
    if (!b->bnodes) return fail_scratch(berr(b, LBM_ENOMEM, "device allocation of boundary nodes failed"));
    for (int d = 0; d < n && e == cudaSuccess; ++d) {
        const Domain &m = b->dom[d];
        e = launch_boundary_nodes(b->links + m.link_off, m.nlinks, b->bnodes + m.link_off, totals_d + d, s);
        b->launches += 1;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(totals.data(), totals_d, sizeof(long long) * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    bdev_free(b, blk);
    bdev_free(b, totals_d);
    if (e != cudaSuccess) return fail(bcuda(b, e, "boundary nodes"));
    for (int d = 0; d < n; ++d) b->dom[d].n_bnodes = totals[d];

    // tile flags and tables, every shape
    for (int sh = 0; sh < BATCH_SHAPES; ++sh) {
        const int tw = batch_tx(sh), th = batch_tr(b->storage, sh);
        long long nflags = 0;
        std::vector<long long> foff(n);
        for (int d = 0; d < n; ++d) {
            foff[d] = nflags;
            nflags += (long long)((b->dom[d].nx + tw - 1) / tw) * ((b->dom[d].ny + th - 1) / th);
        }
        uint8_t *flags_d = (uint8_t *)bdev_alloc(b, (size_t)nflags);
        if (!flags_d) return fail(berr(b, LBM_ENOMEM, "device allocation of tile flags failed"));
        for (int d = 0; d < n && e == cudaSuccess; ++d) {
            const Domain &m = b->dom[d];
            e = launch_tile_flags(b->nbits + m.node_off, m.nx, m.ny, m.pitch, periodic, flags_d + foff[d],
                                  (m.nx + tw - 1) / tw, (m.ny + th - 1) / th, tw, th, s);
            b->launches += 1;
        }
        std::vector<uint8_t> flags((size_t)nflags);
        if (e == cudaSuccess) e = cudaMemcpyAsync(flags.data(), flags_d, (size_t)nflags, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        bdev_free(b, flags_d);
        if (e != cudaSuccess) return fail(bcuda(b, e, "tile flags"));
        // per-tile flags in the batch's tile order (domain by domain, row by
        // row), and the same for the control-volume rectangles
        std::vector<int4> chk, chk_cv;
        for (int d = 0; d < n; ++d) {
            Domain &m = b->dom[d];
            const int tiles_x = (m.nx + tw - 1) / tw, tiles_y = (m.ny + th - 1) / th;
            m.tiles_x[sh] = tiles_x;
            m.tile_base[sh] = (long long)chk.size();
            m.cv_base[sh] = (long long)chk_cv.size();
            for (int ty = 0; ty < tiles_y; ++ty)
                for (int tx = 0; tx < tiles_x; ++tx)
                    chk.push_back(make_int4(d % MAX_BATCH_DOMAINS, tx, ty,
                                            flags[foff[d] + (long long)ty * tiles_x + tx] ? 1 : 0));
            for (int ty = m.cvt[sh][2]; ty <= m.cvt[sh][3]; ++ty)
                for (int tx = m.cvt[sh][0]; tx <= m.cvt[sh][1]; ++tx)
                    chk_cv.push_back(make_int4(d % MAX_BATCH_DOMAINS, tx, ty,
                                               flags[foff[d] + (long long)ty * tiles_x + tx] ? 1 : 0));
        }
        // Within each launch (a chunk of domains), the tiles that take the
        // interior path come first, then the edge tiles (top and bottom tile
        // rows, the inlet and outlet tile columns), then the tiles next to a
        // body.  CTAs start roughly in launch order, so co-resident CTAs then
        // mostly run the same code, which keeps the instruction caches warm.
        // Any order gives the same bits: each tile writes its own nodes and
        // its own partial-sum slot.
        const int path_order = b->storage == LBM_F16_DEV ? GBLBM_BATCH_PATH_ORDER_F16 : GBLBM_BATCH_PATH_ORDER_F32;
        for (int c0 = 0; path_order != 0 && c0 < n; c0 += MAX_BATCH_DOMAINS) {
            const int c1 = c0 + MAX_BATCH_DOMAINS < n ? c0 + MAX_BATCH_DOMAINS : n;
            const long long lo = b->dom[c0].tile_base[sh];
            const long long hi = c1 < n ? b->dom[c1].tile_base[sh] : (long long)chk.size();
            auto path = [&](const int4 &t) {
                const Domain &m = b->dom[c0 + t.x];
                if (t.w) return 2;
                const bool edge_row = periodic || t.z == 0 || (t.z + 1) * th >= m.ny;
                const bool edge_col = t.y == 0 || (t.y + 1) * tw >= m.nx - 1;
                return edge_row || edge_col ? 1 : 0;
            };
            std::stable_sort(chk.begin() + lo, chk.begin() + hi, [&](const int4 &u, const int4 &v) {
                return path_order == 1 ? path(u) < path(v) : path(u) > path(v);
            });
        }
        b->n_tiles[sh] = (long long)chk.size();
        b->n_cv_entries[sh] = (long long)chk_cv.size();
        BALLOC(b->checked[sh], int4 *, sizeof(int4) * (chk.size() > 0 ? chk.size() : 1));
        BALLOC(b->checked_cv[sh], int4 *, sizeof(int4) * (chk_cv.size() > 0 ? chk_cv.size() : 1));
        BCKC(cudaMemcpyAsync(b->checked[sh], chk.data(), sizeof(int4) * chk.size(), cudaMemcpyHostToDevice, s),
             "H2D tile table");
        BCKC(cudaMemcpyAsync(b->checked_cv[sh], chk_cv.data(), sizeof(int4) * chk_cv.size(), cudaMemcpyHostToDevice, s),
             "H2D control-volume tile flags");
        BCKC(cudaStreamSynchronize(s), "sync");
    }
    // the tiles of one launch (a chunk of domains) are counted in int
    for (int sh = 0; sh < BATCH_SHAPES; ++sh)
        for (int c = 0; c < n_chunks(b); ++c) {
            const int d0 = c * MAX_BATCH_DOMAINS;
            const int d1 = d0 + MAX_BATCH_DOMAINS < n ? d0 + MAX_BATCH_DOMAINS : n;
            const long long end = d1 < n ? b->dom[d1].tile_base[sh] : b->n_tiles[sh];
            if (end - b->dom[d0].tile_base[sh] > (long long)INT_MAX / 2)
                return fail(berr(b, LBM_EINVAL, "too many tiles in one launch"));
        }
    {
        lbm_status st = upload_tables(b);
        if (st != LBM_OK) return fail(st);
    }
#undef BCKC
#undef BALLOC
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch *b, int n)
{
    if (!b) return berr(nullptr, LBM_EINVAL, "NULL handle");
    if (n < 0) return berr(b, LBM_EINVAL, "n must be >= 0");
    if (n == 0) return LBM_OK;
    lbm_status st = ensure_series(b, b->t + n);
    if (st != LBM_OK) return st;
    while (n > 0) {
        if (b->t == 0 || n < 2) {
            // the first step reads the pre-collision state; single steps run directly
            BCK(b, launch_step(b, b->t == 0 ? -1 : b->cur), "batch step launch");
            b->cur = 1 - b->cur;
            b->t += 1;
            n -= 1;
        } else {
            const int k = n >= BATCH_GRAPH_STEPS ? 0 : 1;
            const int steps = k == 0 ? BATCH_GRAPH_STEPS : 2;
            if (!b->graph[b->cur][k]) {
                st = build_graph(b, b->cur, k);
                if (st != LBM_OK) return st;
            }
            BCK(b, cudaGraphLaunch(b->graph[b->cur][k], b->stream), "graph launch");
            b->launches += (long long)(n_chunks(b) + 1) * steps;
            b->t += steps;
            n -= steps;
        }
    }
    int bst[2];
    std::vector<int> dst((size_t)2 * b->n);
    BCK(b, cudaMemcpyAsync(bst, b->bstatus, sizeof(bst), cudaMemcpyDeviceToHost, b->stream), "D2H status");
    BCK(b, cudaMemcpyAsync(dst.data(), b->status, sizeof(int) * 2 * b->n, cudaMemcpyDeviceToHost, b->stream),
        "D2H status");
    BCK(b, cudaStreamSynchronize(b->stream), "step sync");
    if (b->t - 1 > b->drtt_ready) b->drtt_ready = b->t - 1;
    if (bst[0] & 4) return berr(b, LBM_ESTATE, "a force-series row lay beyond the series buffer");
    int bad = 0, first = -1;
    for (int d = 0; d < b->n; ++d)
        if (dst[2 * d]) {
            if (first < 0) first = d;
            ++bad;
        }
    if (bad)
        return berr(b, LBM_EUNSTABLE, "%d domain(s) flagged unstable (first: domain %d, step %d)", bad, first,
                    dst[2 * first + 1]);
    return LBM_OK;
}

namespace {

lbm_status read_rows(lbm_batch *b, int domain, long first, long count, std::vector<double> &rows)
{
    // rows [count][SERIES_ROW] of one domain (domain >= 0) or [count][n][SERIES_ROW] of all
    const size_t R = SERIES_ROW;
    const size_t stride = R * b->n;
    const int width = domain >= 0 ? 1 : b->n;
    rows.assign((size_t)count * R * width, 0.0);
    for (long k = 0; k < count;) {
        const long long step = first + k;
        const long long slot = b->record_series ? step : (step & 1);
        // contiguous steps when all are kept; one at a time otherwise
        const long run = b->record_series ? count - k : 1;
        const double *src = b->series + stride * slot + (domain >= 0 ? R * domain : 0);
        BCK(b, cudaMemcpy2DAsync(rows.data() + (size_t)k * R * width, sizeof(double) * R * width, src,
                                 sizeof(double) * stride, sizeof(double) * R * width, (size_t)run,
                                 cudaMemcpyDeviceToHost, b->stream),
            "D2H series");
        k += run;
    }
    BCK(b, cudaStreamSynchronize(b->stream), "sync");
    return LBM_OK;
}

lbm_status check_range(lbm_batch *b, int scheme, long first, long count)
{
    if (scheme < 0 || scheme > LBM_FORCE_SI) return berr(b, LBM_EINVAL, "unknown scheme %d", scheme);
    if (count < 0 || first < 0 || first + count > b->t)
        return berr(b, LBM_EINVAL, "steps [%ld, %ld) outside [0, %lld)", first, first + count, b->t);
    if (!b->record_series && first < b->t - 2)
        return berr(b, LBM_EINVAL, "only the last two steps are kept (record_series = 0)");
    if (scheme == LBM_FORCE_DRTT && first + count > b->drtt_ready) return finalize_drtt(b);
    return LBM_OK;
}

}  // namespace

lbm_status lbm_batch_forces(lbm_batch *b, int scheme, long step, double *fx, double *fy)
{
    if (!b) return berr(nullptr, LBM_EINVAL, "NULL handle");
    if (!fx || !fy) return berr(b, LBM_EINVAL, "fx and fy must not be NULL");
    lbm_status st = check_range(b, scheme, step, 1);
    if (st != LBM_OK) return st;
    std::vector<double> rows;
    st = read_rows(b, -1, step, 1, rows);
    if (st != LBM_OK) return st;
    for (int d = 0; d < b->n; ++d) {
        fx[d] = rows[(size_t)SERIES_ROW * d + 2 * scheme];
        fy[d] = rows[(size_t)SERIES_ROW * d + 2 * scheme + 1];
    }
    return LBM_OK;
}

lbm_status lbm_batch_force_series(lbm_batch *b, int domain, int scheme, long first, long count, double *fx,
                                  double *fy)
{
    if (!b) return berr(nullptr, LBM_EINVAL, "NULL handle");
    if (domain < 0 || domain >= b->n) return berr(b, LBM_EINVAL, "no domain %d", domain);
    lbm_status st = check_range(b, scheme, first, count);
    if (st != LBM_OK || count == 0) return st;
    if (!fx || !fy) return berr(b, LBM_EINVAL, "fx and fy must not be NULL");
    std::vector<double> rows;
    st = read_rows(b, domain, first, count, rows);
    if (st != LBM_OK) return st;
    for (long k = 0; k < count; ++k) {
        fx[k] = rows[(size_t)SERIES_ROW * k + 2 * scheme];
        fy[k] = rows[(size_t)SERIES_ROW * k + 2 * scheme + 1];
    }
    return LBM_OK;
}

lbm_status lbm_batch_prepare(lbm_batch *b, long n)
{
    if (!b) return berr(nullptr, LBM_EINVAL, "NULL handle");
    if (n < 0) return berr(b, LBM_EINVAL, "n must be >= 0");
    lbm_status st = ensure_series(b, b->t + n);
    if (st != LBM_OK) return st;
    for (int c = 0; c < 2; ++c)
        for (int k = 0; k < 2; ++k)
            if (!b->graph[c][k]) {
                st = build_graph(b, c, k);
                if (st != LBM_OK) return st;
            }
    return LBM_OK;
}

lbm_status lbm_batch_coefficients(lbm_batch *b, int domain, int scheme, long first, long count, double length,
                                  double u_ref, double *cd, double *cl, double *stats)
{
    if (!b) return berr(nullptr, LBM_EINVAL, "NULL handle");
    if (domain < 0 || domain >= b->n) return berr(b, LBM_EINVAL, "no domain %d", domain);
    if (count < 1) return berr(b, LBM_EINVAL, "the window must hold at least one step");
    if (!(length > 0) || !std::isfinite(length) || !(u_ref != 0) || !std::isfinite(u_ref))
        return berr(b, LBM_EINVAL, "length must be > 0 and u_ref nonzero, both finite");
    lbm_status st = check_range(b, scheme, first, count);
    if (st != LBM_OK) return st;
    const double norm = 2.0 / (b->rho0 * u_ref * u_ref * length);
    const bool per_step = cd || cl;
    double *out = (double *)bdev_alloc(b, sizeof(double) * (4 + (per_step ? 2 * (size_t)count : 0)));
    if (!out) return berr(b, LBM_ENOMEM, "coefficient buffer allocation failed");
    cudaError_t e = launch_coefficients(b->series + (size_t)SERIES_ROW * domain, (long long)SERIES_ROW * b->n,
                                        2 * scheme, first, count, !b->record_series, norm, out, per_step,
                                        b->stream);
    double st4[4];
    if (e == cudaSuccess) e = cudaMemcpyAsync(st4, out, sizeof(st4), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess && cd)
        e = cudaMemcpyAsync(cd, out + 4, sizeof(double) * count, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess && cl)
        e = cudaMemcpyAsync(cl, out + 4 + count, sizeof(double) * count, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    bdev_free(b, out);
    b->launches += 1;
    if (e != cudaSuccess) return bcuda(b, e, "coefficients");
    if (stats) memcpy(stats, st4, sizeof(st4));
    return LBM_OK;
}

lbm_status lbm_batch_populations(lbm_batch *b, int domain, double *out)
{
    if (!b) return berr(nullptr, LBM_EINVAL, "NULL handle");
    if (domain < 0 || domain >= b->n) return berr(b, LBM_EINVAL, "no domain %d", domain);
    if (!out) return berr(b, LBM_EINVAL, "out must not be NULL");
    const Domain &m = b->dom[domain];
    const size_t N = (size_t)m.nx * m.ny;
    double *scratch = (double *)bdev_alloc(b, sizeof(double) * N);
    if (!scratch) return berr(b, LBM_ENOMEM, "scratch allocation failed");
    const char *pop = b->pop[b->cur] + m.pop_off * (long long)b->elem;
    const void *inlet = (const char *)b->inlet + m.inlet_off * (long long)b->elem;
    lbm_status st = LBM_OK;
    for (int i = 0; i < 9 && st == LBM_OK; ++i) {
        cudaError_t e = launch_gather(b->storage, pop, b->nbits + m.node_off, inlet, m.plane, m.nx, m.ny, m.pitch,
                                      b->periodic, b->t == 0 ? 1 : 0, b->rho0, i, scratch, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out + i * N, scratch, sizeof(double) * N, cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) st = bcuda(b, e, "gather populations");
        b->launches += 1;
    }
    bdev_free(b, scratch);
    return st;
}

lbm_status lbm_batch_set_populations(lbm_batch *b, int domain, const double *in)
{
    if (!b) return berr(nullptr, LBM_EINVAL, "NULL handle");
    if (domain < 0 || domain >= b->n) return berr(b, LBM_EINVAL, "no domain %d", domain);
    if (!in) return berr(b, LBM_EINVAL, "in must not be NULL");
    if (b->t != 0) return berr(b, LBM_ESTATE, "populations can be set before the first step only");
    const Domain &m = b->dom[domain];
    const size_t N = (size_t)m.nx * m.ny;
    for (size_t k = 0; k < 9 * N; ++k)
        if (!std::isfinite(in[k])) return berr(b, LBM_EINVAL, "populations must be finite");
    double *scratch = (double *)bdev_alloc(b, sizeof(double) * N);
    if (!scratch) return berr(b, LBM_ENOMEM, "scratch allocation failed");
    char *pop = b->pop[0] + m.pop_off * (long long)b->elem;
    lbm_status st = LBM_OK;
    for (int i = 0; i < 9 && st == LBM_OK; ++i) {
        cudaError_t e = cudaMemcpyAsync(scratch, in + i * N, sizeof(double) * N, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = launch_scatter_pop(b->storage, pop, b->nbits + m.node_off, m.plane, m.nx, m.ny, m.pitch, b->rho0, i,
                                   scratch, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) st = bcuda(b, e, "set populations");
        b->launches += 1;
    }
    bdev_free(b, scratch);
    return st;
}

lbm_status lbm_batch_pressure_coefficient(lbm_batch *b, int domain, double p_inf, double q, int32_t *nodes,
                                          double *cp, long cap, long *count)
{
    if (!b) return berr(nullptr, LBM_EINVAL, "NULL handle");
    if (domain < 0 || domain >= b->n) return berr(b, LBM_EINVAL, "no domain %d", domain);
    if (!std::isfinite(p_inf) || !std::isfinite(q) || q == 0.0)
        return berr(b, LBM_EINVAL, "p_inf must be finite and q finite and nonzero");
    const Domain &m = b->dom[domain];
    if (count) *count = (long)m.n_bnodes;
    const long n = cap < (long)m.n_bnodes ? cap : (long)m.n_bnodes;
    if (n <= 0) return LBM_OK;
    const int32_t *bn = b->bnodes + m.link_off;
    if (nodes) BCK(b, cudaMemcpyAsync(nodes, bn, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->stream), "D2H nodes");
    if (cp) {
        double *d = (double *)bdev_alloc(b, sizeof(double) * m.n_bnodes);
        if (!d) return berr(b, LBM_ENOMEM, "scratch allocation failed");
        cudaError_t e = launch_surface_pressure(b->storage, b->pop[b->cur] + m.pop_off * (long long)b->elem,
                                                b->nbits + m.node_off, bn, m.n_bnodes, m.plane, m.nx, m.ny, m.pitch,
                                                b->periodic, b->t == 0 ? 1 : 0, b->rho0, p_inf, q, d, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cp, d, sizeof(double) * n, cudaMemcpyDeviceToHost, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        bdev_free(b, d);
        b->launches += 1;
        if (e != cudaSuccess) return bcuda(b, e, "surface pressure");
    }
    BCK(b, cudaStreamSynchronize(b->stream), "sync");
    return LBM_OK;
}

lbm_status lbm_batch_status(lbm_batch *b, int *unstable, long *first_bad_step)
{
    if (!b) return berr(nullptr, LBM_EINVAL, "NULL handle");
    std::vector<int> st((size_t)2 * b->n);
    BCK(b, cudaMemcpyAsync(st.data(), b->status, sizeof(int) * 2 * b->n, cudaMemcpyDeviceToHost, b->stream),
        "D2H status");
    BCK(b, cudaStreamSynchronize(b->stream), "sync");
    for (int d = 0; d < b->n; ++d) {
        if (unstable) unstable[d] = st[2 * d] ? 1 : 0;
        if (first_bad_step) first_bad_step[d] = st[2 * d] ? (long)st[2 * d + 1] : -1;
    }
    return LBM_OK;
}

int lbm_batch_num_shapes(void) { return BATCH_SHAPES; }

lbm_status lbm_batch_shape(const lbm_batch *b, int k, int *tile_w, int *tile_h)
{
    if (!b) return berr(nullptr, LBM_EINVAL, "NULL handle");
    if (k < 0 || k >= BATCH_SHAPES) return berr(const_cast<lbm_batch *>(b), LBM_EINVAL, "no tile shape %d", k);
    if (tile_w) *tile_w = batch_tx(k);
    if (tile_h) *tile_h = batch_tr(b->storage, k);
    return LBM_OK;
}

lbm_status lbm_batch_set_launch(lbm_batch *b, int shape, int ctas_per_sm)
{
    if (!b) return berr(nullptr, LBM_EINVAL, "NULL handle");
    if (shape < 0 || shape >= BATCH_SHAPES) return berr(b, LBM_EINVAL, "no tile shape %d", shape);
    if (ctas_per_sm < 0) return berr(b, LBM_EINVAL, "ctas_per_sm must be >= 0");
    if (ctas_per_sm > 0) {
        const int most = batch_max_ctas_per_sm(b->storage, shape);
        if (ctas_per_sm > most)
            return berr(b, LBM_EINVAL, "shape %d holds at most %d CTAs per SM (asked %d)", shape, most, ctas_per_sm);
    }
    if (shape != b->shape || ctas_per_sm != b->ctas_per_sm) {
        BCK(b, cudaStreamSynchronize(b->stream), "sync");
        drop_graphs(b);
        b->shape = shape;
        b->ctas_per_sm = ctas_per_sm;
    }
    return LBM_OK;
}

lbm_status lbm_batch_get_launch(const lbm_batch *b, int *shape, int *ctas_per_sm)
{
    if (!b) return berr(nullptr, LBM_EINVAL, "NULL handle");
    if (shape) *shape = b->shape;
    if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
    return LBM_OK;
}

lbm_status lbm_batch_autotune(lbm_batch *b, int trials, int *shape_out, int *ctas_out, double *best_ms)
{
    if (!b) return berr(nullptr, LBM_EINVAL, "NULL handle");
    if (trials < 1) return berr(b, LBM_EINVAL, "trials must be >= 1");
    const int src = b->t == 0 ? 0 : b->cur;  // timing only: the state is read as if pulled
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BCK(b, cudaEventCreate(&e0), "event create");
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return bcuda(b, e, "event create");
    }
    double best = 1e300;
    int best_s = b->shape, best_k = b->ctas_per_sm;
    for (int s = 0; s < BATCH_SHAPES && e == cudaSuccess; ++s) {
        // the current state as source, the spare buffer as destination, scratch sums and flags
        const int most = batch_max_ctas_per_sm(b->storage, s);
        std::vector<int> choices = {0};
        for (int k : BATCH_GRID_CHOICES)
            if (k <= most) choices.push_back(k);
        for (int k : choices) {
            if (e != cudaSuccess) break;
            const int grid = k * b->sm_count;
            e = launch_collide(b, src, false, true, s, grid);  // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
            for (int r = 0; r < trials && e == cudaSuccess; ++r) e = launch_collide(b, src, false, true, s, grid);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && ms / trials < best) {
                best = ms / trials;
                best_s = s;
                best_k = k;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return bcuda(b, e, "autotune");
    lbm_status st = lbm_batch_set_launch(b, best_s, best_k);
    if (st != LBM_OK) return st;
    if (shape_out) *shape_out = best_s;
    if (ctas_out) *ctas_out = best_k;
    if (best_ms) *best_ms = best;
    return LBM_OK;
}

long lbm_batch_steps_done(const lbm_batch *b) { return b ? (long)b->t : -1; }
int lbm_batch_num_domains(const lbm_batch *b) { return b ? b->n : -1; }
long long lbm_batch_nodes(const lbm_batch *b) { return b ? b->nodes : -1; }
long long lbm_batch_launch_count(const lbm_batch *b) { return b ? b->launches : -1; }

const char *lbm_batch_last_error(const lbm_batch *b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

void lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return;
    free_all(b);
    delete b;
}

}  // extern "C"
