// lbm_api.cu -- the C ABI declared in include/gblbm.h: argument checks, device
// memory, set-up sequence, the step loop (CUDA graphs of whole step pairs) and
// read-back.  All arithmetic of the method runs in the kernels of
// lbm_setup.cu and lbm_step.cu.
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "lbm_host.h"
#include "lbm_internal.cuh"

using namespace gblbm;

namespace {

thread_local std::string g_thread_err;

// Three population buffers rotate: step t reads buffer b(t-1) and writes b(t).
// The link kernel of step t (reading b(t-1) and b(t)) runs on a side stream,
// concurrently with the collide-stream kernel of step t+1 (writing b(t+1));
// the collide-stream kernel of step t+2 waits for it before overwriting b(t-1).
constexpr int NBUF = 3;
#ifndef GBLBM_GRAPH_STEPS
#define GBLBM_GRAPH_STEPS 15
#endif
constexpr int GRAPH_STEPS = GBLBM_GRAPH_STEPS;  // steps per captured graph (a multiple of NBUF)
static_assert(GRAPH_STEPS % NBUF == 0 && GRAPH_STEPS >= NBUF, "GRAPH_STEPS: a multiple of NBUF");
// Share of the free device memory the adjoint may fill with kept forward
// states when the caller leaves the checkpoint interval to it (a tuning knob).
#ifndef GBLBM_ADJ_KEEP_SHARE
#define GBLBM_ADJ_KEEP_SHARE 0.6
#endif
constexpr double ADJ_KEEP_SHARE = GBLBM_ADJ_KEEP_SHARE;
// Dispatch the tile rows that hold bounce-back tiles first (a tuning knob).
#ifndef GBLBM_BODY_ROWS_FIRST
#define GBLBM_BODY_ROWS_FIRST 1
#endif
constexpr int TIMING_BATCH = 64;

}  // namespace

void gblbm::set_thread_error(const char *msg) { g_thread_err = msg; }

struct lbm_ctx {
    int nx = 0, ny = 0, pitch = 0, periodic = 0, storage = 0;
    double tau = 0, omega = 0, rho0 = 1, g[2] = {0, 0};
    int cv[4] = {0, 0, 0, 0}, cvt[4] = {0, 0, 0, 0};
    int tiles_x = 0, tiles_y = 0, n_cv_tiles = 0;
    int record_series = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    lbm_alloc_fn alloc_fn = nullptr;
    lbm_free_fn free_fn = nullptr;
    void *alloc_user = nullptr;
    size_t elem = 4;
    long long plane = 0;
    void *pop[NBUF] = {nullptr, nullptr, nullptr};       // first element of plane 0
    void *pop_base[NBUF] = {nullptr, nullptr, nullptr};  // allocations (with guards)
    alignas(64) CUtensorMap tmap[NBUF];                  // [9][ny][pitch] views for TMA loads
    bool tmap_ok = false;
    int use_bulk = 0, sm_count = 1;
    int pf_rows = 0;                                     // L2 prefetch distance of the direct kernel
    int first_r0 = 1, first_r1 = 0;                      // tile rows holding bounce-back tiles (none: r0 > r1)
    unsigned int wait_limit = WAIT_LIMIT;                // polls of each staged-kernel pipeline wait
    int cur = 0;                 // buffer holding the latest state
    cudaStream_t side = nullptr; // link kernels
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_read[NBUF] = {nullptr, nullptr, nullptr};
    bool ev_live[NBUF] = {false, false, false};
    // The step whose collide-stream kernel is queued and whose link kernel is
    // not yet (lead_src < 0: none): it goes out beside the next step's
    // collide-stream kernel, or when the queue ends.
    int lead_src = -1, lead_pre = 0;
    int link_prio = 0;           // launch priority of the link kernels (the device's highest)
    double adj_budget = 0;       // bytes the adjoint may fill with kept states (0: from free memory)
    uint8_t *mask_d = nullptr;
    uint16_t *nbits = nullptr;
    uint8_t *tile_flag = nullptr;
    int32_t *links = nullptr;
    long long nlinks = 0;
    int32_t *bnodes = nullptr;  // boundary fluid nodes (distinct link nodes, ascending)
    long long n_bnodes = 0;
    double *u_row = nullptr;
    void *inlet = nullptr;
    double *partials = nullptr;  // NBUF slices, one per destination buffer
    double *link_partials = nullptr;
    unsigned int *ticket = nullptr;
    int link_ctas = 1;
    double link_base[2] = {0, 0}, flux_base[2] = {0, 0};
    double *series = nullptr;
    long long series_cap = 0;
    double *carry = nullptr;     // [8]
    long long *step_ctr = nullptr;
    int *status = nullptr;       // [2]
    int status_host[2] = {0, 0};  // the status words read back by settle
    bool status_armed = false;   // status cleared for the queued steps
    bool pending = false;        // steps queued and not yet settled
    long long t = 0;
    int precollision = 1;
    long long carry_from = 0;    // first step of the current DRTT chain
    long long drtt_ready = 0;    // DRTT(s) is final for s < drtt_ready
    // [start buffer][GRAPH_STEPS or NBUF steps][opens with the previous step's link kernel]
    cudaGraphExec_t graph[NBUF][2][2] = {};
    bool timing = false;
    std::vector<cudaEvent_t> events;
    double kt_ms[2] = {0, 0};
    long kt_n[2] = {0, 0};
    long long launches = 0;
    std::string err;
};

namespace {

lbm_status set_err(lbm_ctx *h, lbm_status code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h)
        h->err = buf;
    else
        g_thread_err = buf;
    return code;
}

lbm_status cuda_err(lbm_ctx *h, cudaError_t e, const char *what)
{
    return set_err(h, LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(h, expr, what)                               \
    do {                                                \
        cudaError_t e_ = (expr);                        \
        if (e_ != cudaSuccess) return cuda_err(h, e_, what); \
    } while (0)

void *dev_alloc(lbm_ctx *h, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (h->alloc_fn) return h->alloc_fn(bytes, (void *)h->stream, h->alloc_user);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(lbm_ctx *h, void *p)
{
    if (!p) return;
    if (h->free_fn)
        h->free_fn(p, h->alloc_user);
    else
        cudaFree(p);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    }
    return fn;
}

// Tensor map over one population buffer viewed as [9][ny][pitch], with the
// staged kernel's box: 128 + 2 PAD columns (PAD = 16 bytes of elements), the
// tile rows plus one above and one below, all nine planes.
bool encode_tensor_map(CUtensorMap *m, int storage, void *base, int pitch, int ny)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const size_t elem = storage_bytes(storage);
    const CUtensorMapDataType dt = storage == LBM_F64       ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : storage == LBM_F16_DEV ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                            : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)ny, 9};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * elem, (cuuint64_t)pitch * ny * elem};
    const cuuint32_t box[3] = {(cuuint32_t)(TILE_X + 2 * (16 / elem)),
                               (cuuint32_t)(tile_rows(storage) + 2), 9};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int next_buf(int b) { return b + 1 == NBUF ? 0 : b + 1; }
int prev_buf(int b) { return b == 0 ? NBUF - 1 : b - 1; }

StepArgs step_args(lbm_ctx *h, int src, int dst, int precollision)
{
    StepArgs a;
    memset(&a, 0, sizeof(a));
    a.src = h->pop[src];
    a.dst = h->pop[dst];
    a.nbits = h->nbits;
    a.tile_flag = h->tile_flag;
    a.inlet = h->inlet;
    a.partials = h->partials + (size_t)dst * CV_PARTIAL * h->n_cv_tiles;
    a.status = h->status;
    a.step_ctr = h->step_ctr;
    a.plane = h->plane;
    a.nx = h->nx;
    a.ny = h->ny;
    a.pitch = h->pitch;
    a.periodic = h->periodic;
    a.precollision = precollision;
    a.tiles_x = h->tiles_x;
    set_relaxation(a, h->omega);
    a.rho0 = h->rho0;
    a.gx = h->g[0];
    a.gy = h->g[1];
    a.rho0_f = (float)h->rho0;
    a.gx_f = (float)h->g[0];
    a.gy_f = (float)h->g[1];
    memcpy(a.cv, h->cv, sizeof(a.cv));
    memcpy(a.cvt, h->cvt, sizeof(a.cvt));
    a.use_bulk = h->use_bulk;
    a.sm_count = h->sm_count;
    a.pf_rows = h->pf_rows;
    a.first_r0 = h->first_r0;
    a.first_r1 = h->first_r1;
    a.wait_limit = h->wait_limit;
    return a;
}

LinkArgs link_args(lbm_ctx *h, int src, int dst, int precollision, int drtt_only)
{
    LinkArgs a;
    memset(&a, 0, sizeof(a));
    a.src = h->pop[src];
    a.dst = h->pop[dst];
    a.nbits = h->nbits;
    a.links = h->links;
    a.nlinks = h->nlinks;
    a.partials = h->partials + (size_t)dst * CV_PARTIAL * h->n_cv_tiles;
    a.n_partials = h->n_cv_tiles;
    a.link_partials = h->link_partials;
    a.ticket = h->ticket;
    a.n_ctas = h->link_ctas;
    a.series = h->series;
    a.series_rows = h->series_cap;
    a.status = h->status;
    a.carry = h->carry;
    a.step_ctr = h->step_ctr;
    a.plane = h->plane;
    a.nx = h->nx;
    a.ny = h->ny;
    a.pitch = h->pitch;
    a.periodic = h->periodic;
    a.precollision = precollision;
    a.record_series = h->record_series;
    a.drtt_only = drtt_only;
    a.rho0 = h->rho0;
    a.visc = 1.0 - 0.5 * h->omega;
    a.visc_f = (float)a.visc;
    memcpy(a.link_base, h->link_base, sizeof(a.link_base));
    memcpy(a.flux_base, h->flux_base, sizeof(a.flux_base));
    return a;
}

// The link kernel of the step that read buffer src, on the side stream,
// forked after everything queued so far on the handle's stream (that step's
// collide-stream kernel included); the collide-stream kernel that overwrites
// src next waits for it (ev_read).
cudaError_t launch_link_side(lbm_ctx *h, int src, int precollision)
{
    LinkArgs la = link_args(h, src, next_buf(src), precollision, 0);
    cudaError_t e = cudaEventRecord(h->ev_fork, h->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->ev_fork, 0);
    if (e == cudaSuccess) e = launch_link_force(h->storage, la, h->side, h->link_prio);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev_read[src], h->side);
    h->ev_live[src] = true;
    h->launches += 1;
    return e;
}

// Launches the held link kernel, if any.
cudaError_t flush_link(lbm_ctx *h)
{
    if (h->lead_src < 0) return cudaSuccess;
    const int src = h->lead_src;
    h->lead_src = -1;
    return launch_link_side(h, src, h->lead_pre);
}

// Join the side stream back into the handle's stream.
cudaError_t join_side(lbm_ctx *h)
{
    cudaError_t e = cudaEventRecord(h->ev_join, h->side);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_join, 0);
    for (int b = 0; b < NBUF; ++b) h->ev_live[b] = false;
    return e;
}

// One step t -> t+1 from buffer src into next_buf(src).  Normally the
// collide-stream kernel goes to the handle's stream and its link kernel is
// held (lead_src): it is launched on the side stream beside the next step's
// collide-stream kernel, so that no link kernel waits alone between two
// steps, not even across the end of a captured graph.  The collide-stream
// kernel first waits for the link kernel of step t-2, which read the buffer
// it overwrites.  With timing events (ev != NULL) both kernels run in order
// on the handle's stream, each between events.
cudaError_t launch_one_step(lbm_ctx *h, int src, int precollision, cudaEvent_t *ev)
{
    const int dst = next_buf(src);
    cudaError_t e = cudaSuccess;
    StepArgs sa = step_args(h, src, dst, precollision);
    if (ev) {
        if (h->lead_src >= 0) {
            e = flush_link(h);
            if (e == cudaSuccess) e = join_side(h);
            if (e != cudaSuccess) return e;
        }
        cudaEventRecord(ev[0], h->stream);
        e = launch_collide_stream(h->storage, sa, h->tiles_x, h->tiles_y, false,
                                  h->tmap_ok ? (const void *)&h->tmap[src] : nullptr, h->stream);
        if (e != cudaSuccess) return e;
        LinkArgs la = link_args(h, src, dst, precollision, 0);
        cudaEventRecord(ev[1], h->stream);
        e = launch_link_force(h->storage, la, h->stream);
        cudaEventRecord(ev[2], h->stream);
        h->launches += 2;
        return e;
    }
    e = flush_link(h);
    if (e == cudaSuccess && h->ev_live[dst]) e = cudaStreamWaitEvent(h->stream, h->ev_read[dst], 0);
    if (e != cudaSuccess) return e;
    e = launch_collide_stream(h->storage, sa, h->tiles_x, h->tiles_y, false,
                              h->tmap_ok ? (const void *)&h->tmap[src] : nullptr, h->stream);
    h->lead_src = src;
    h->lead_pre = precollision;
    h->launches += 1;
    return e;
}

void drop_graphs(lbm_ctx *h)
{
    for (int p = 0; p < NBUF; ++p)
        for (int k = 0; k < 2; ++k)
            for (int l = 0; l < 2; ++l)
                if (h->graph[p][k][l]) {
                    cudaGraphExecDestroy(h->graph[p][k][l]);
                    h->graph[p][k][l] = nullptr;
                }
}

// Captures GRAPH_STEPS (k = 0) or NBUF (k = 1) steps from buffer p.  lead = 1:
// the graph opens with the held link kernel of the step before (which read
// prev_buf(p)) beside its first collide-stream kernel.  Either way the graph
// ends with its last step's link kernel held: the caller sets lead_src.
lbm_status build_graph(lbm_ctx *h, int p, int k, int lead)
{
    int steps = k == 0 ? GRAPH_STEPS : NBUF;
    cudaGraph_t g = nullptr;
    for (int b = 0; b < NBUF; ++b) h->ev_live[b] = false;
    const int saved_src = h->lead_src, saved_pre = h->lead_pre;
    h->lead_src = lead ? prev_buf(p) : -1;
    h->lead_pre = 0;
    CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t le = cudaSuccess;
    long long saved = h->launches;
    int b = p;
    for (int s = 0; s < steps && le == cudaSuccess; ++s) {
        le = launch_one_step(h, b, 0, nullptr);
        b = next_buf(b);
    }
    if (le == cudaSuccess) le = join_side(h);
    h->launches = saved;
    h->lead_src = saved_src;
    h->lead_pre = saved_pre;
    cudaError_t ee = cudaStreamEndCapture(h->stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_err(h, le, "capture step kernels");
    }
    if (ee != cudaSuccess) return cuda_err(h, ee, "end capture");
    cudaError_t ie = cudaGraphInstantiateWithFlags(&h->graph[p][k][lead], g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return cuda_err(h, ie, "instantiate graph");
    return LBM_OK;
}

lbm_status ensure_series(lbm_ctx *h, long long need)
{
    if (!h->record_series) need = 2;
    if (need <= h->series_cap) return LBM_OK;
    long long cap = h->series_cap ? h->series_cap : 1024;
    while (cap < need) cap *= 2;
    double *ns = (double *)dev_alloc(h, sizeof(double) * SERIES_ROW * cap);
    if (!ns) return set_err(h, LBM_ENOMEM, "force series: allocation of %lld steps failed", cap);
    CK(h, cudaMemsetAsync(ns, 0, sizeof(double) * SERIES_ROW * cap, h->stream), "memset series");
    if (h->series)
        CK(h, cudaMemcpyAsync(ns, h->series, sizeof(double) * SERIES_ROW * h->series_cap,
                              cudaMemcpyDeviceToDevice, h->stream),
           "copy series");
    CK(h, cudaStreamSynchronize(h->stream), "sync");
    dev_free(h, h->series);
    h->series = ns;
    h->series_cap = cap;
    drop_graphs(h);
    return LBM_OK;
}

lbm_status flush_timing(lbm_ctx *h, int nev)
{
    if (nev == 0) return LBM_OK;
    CK(h, cudaEventSynchronize(h->events[3 * (nev - 1) + 2]), "timing sync");
    for (int k = 0; k < nev; ++k) {
        float a = 0, b = 0;
        CK(h, cudaEventElapsedTime(&a, h->events[3 * k], h->events[3 * k + 1]), "elapsed");
        CK(h, cudaEventElapsedTime(&b, h->events[3 * k + 1], h->events[3 * k + 2]), "elapsed");
        h->kt_ms[0] += a;
        h->kt_ms[1] += b;
        h->kt_n[0] += 1;
        h->kt_n[1] += 1;
    }
    return LBM_OK;
}

// Complete DRTT(T-1) with a momentum-only pass over the control-volume tiles.
lbm_status finalize_drtt(lbm_ctx *h)
{
    if (h->drtt_ready >= h->t) return LBM_OK;
    if (h->t < 1 || h->t - 1 < h->carry_from || h->precollision)
        return set_err(h, LBM_ESTATE, "DRTT of step %lld needs J of step %lld, which is not available",
                       h->t - 1, h->t);
    const int slot = next_buf(h->cur);
    StepArgs sa = step_args(h, h->cur, slot, 0);
    sa.dst = nullptr;  // the momentum-only pass stores nothing
    sa.tile_off_x = h->cvt[0];
    sa.tile_off_y = h->cvt[2];
    CK(h, launch_collide_stream(h->storage, sa, h->cvt[1] - h->cvt[0] + 1, h->cvt[3] - h->cvt[2] + 1,
                                true, nullptr, h->stream),
       "momentum pass");
    LinkArgs la = link_args(h, h->cur, slot, 0, 1);
    CK(h, launch_link_force(h->storage, la, h->stream), "DRTT finalize");
    h->launches += 2;
    h->drtt_ready = h->t;
    return LBM_OK;
}

void free_all(lbm_ctx *h)
{
    drop_graphs(h);
    for (auto e : h->events) cudaEventDestroy(e);
    h->events.clear();
    cudaEvent_t evs[] = {h->ev_fork, h->ev_join, h->ev_read[0], h->ev_read[1], h->ev_read[2]};
    for (auto e : evs)
        if (e) cudaEventDestroy(e);
    if (h->side) cudaStreamDestroy(h->side);
    void *bufs[] = {h->pop_base[0], h->pop_base[1], h->pop_base[2], h->mask_d, h->nbits, h->tile_flag, h->links,
                    h->bnodes,
                    h->u_row, h->inlet, h->partials, h->link_partials, h->ticket, h->series,
                    h->carry, h->step_ctr, h->status};
    for (void *p : bufs) dev_free(h, p);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
}

}  // namespace

extern "C" {

void lbm_bc_default(lbm_bc *bc)
{
    if (!bc) return;
    memset(bc, 0, sizeof(*bc));
    bc->kind = LBM_BC_CHANNEL;
    bc->storage = LBM_F32;
    bc->rho0 = 1.0;
    bc->cv[0] = -1;
    bc->record_series = 1;
}

lbm_status lbm_create(const uint8_t *mask, int nx, int ny, double tau, const double *u_in,
                      int n_u_in, const lbm_bc *bc_in, lbm_ctx **out)
{
    if (!out) return set_err(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    lbm_bc bc;
    if (bc_in)
        bc = *bc_in;
    else
        lbm_bc_default(&bc);
    if (bc.kernel != 0 && bc.kernel != 1)
        return set_err(nullptr, LBM_EINVAL, "unknown kernel choice %d", bc.kernel);
    if (bc.kind != LBM_BC_CHANNEL && bc.kind != LBM_BC_PERIODIC)
        return set_err(nullptr, LBM_EINVAL, "unknown boundary kind %d", bc.kind);
    if (bc.storage < LBM_F64 || bc.storage > LBM_F16_DEV)
        return set_err(nullptr, LBM_EINVAL, "unknown storage %d", bc.storage);
    if (!(bc.rho0 > 0) || !std::isfinite(bc.rho0))
        return set_err(nullptr, LBM_EINVAL, "rho0 must be finite and > 0");
    if (!finite_all(bc.body_force, 2)) return set_err(nullptr, LBM_EINVAL, "body force is not finite");
    if ((bc.alloc == nullptr) != (bc.free == nullptr))
        return set_err(nullptr, LBM_EINVAL, "alloc and free must be given together");
    const int periodic = bc.kind == LBM_BC_PERIODIC;
    // the mask's solid nodes, scanned once for the default box and the base sums
    std::vector<long long> solids;
    const bool need_solids = bc.cv[0] < 0 || bc.storage == LBM_F32_DEV || bc.storage == LBM_F16_DEV;
    if (mask && need_solids && nx > 0 && ny > 0 && (long long)nx * ny * 8 < (1LL << 31))
        solids = solid_nodes(mask, nx, ny);
    int cv[4];
    {
        const std::string why = check_domain(mask, nx, ny, tau, u_in, n_u_in, periodic, bc.cv, cv, &solids);
        if (!why.empty()) return set_err(nullptr, LBM_EINVAL, "%s", why.c_str());
    }
    int ndev = 0;
    cudaError_t de = cudaGetDeviceCount(&ndev);
    if (de != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return set_err(nullptr, LBM_ECUDA, "no CUDA device: %s", cudaGetErrorString(de));
    }

    lbm_ctx *h = new (std::nothrow) lbm_ctx;
    if (!h) return set_err(nullptr, LBM_ENOMEM, "host allocation failed");
    h->nx = nx;
    h->ny = ny;
    h->periodic = periodic;
    h->storage = bc.storage;
    h->tau = tau;
    h->omega = 1.0 / tau;
    h->rho0 = bc.rho0;
    h->g[0] = bc.body_force[0];
    h->g[1] = bc.body_force[1];
    memcpy(h->cv, cv, sizeof(cv));
    h->record_series = bc.record_series ? 1 : 0;
    h->use_bulk = bc.kernel == 1;
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            h->sm_count = sms;
        else
            cudaGetLastError();
    }
    h->alloc_fn = bc.alloc;
    h->free_fn = bc.free;
    h->alloc_user = bc.alloc_user;
    h->elem = storage_bytes(bc.storage);
    h->pitch = (nx + PITCH_ALIGN - 1) / PITCH_ALIGN * PITCH_ALIGN;
    h->plane = (long long)ny * h->pitch;
    h->tiles_x = (nx + TILE_X - 1) / TILE_X;
    h->pf_rows = collide_stream_prefetch_rows(bc.storage, h->sm_count, h->tiles_x);
    h->tiles_y = (ny + tile_rows(h->storage) - 1) / tile_rows(h->storage);
    cv_tile_rect(cv, nx, ny, TILE_X, tile_rows(h->storage), h->cvt);
    h->n_cv_tiles = (h->cvt[1] - h->cvt[0] + 1) * (h->cvt[3] - h->cvt[2] + 1);
    if (bc.cuda_stream) {
        h->stream = (cudaStream_t)bc.cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete h;
            return cuda_err(nullptr, e, "stream create");
        }
        h->own_stream = true;
    }
    {
        int least = 0, greatest = 0;
        cudaError_t e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        h->link_prio = greatest;
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, greatest);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
        for (int b = 0; b < NBUF && e == cudaSuccess; ++b)
            e = cudaEventCreateWithFlags(&h->ev_read[b], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            g_thread_err = std::string("stream/event create: ") + cudaGetErrorString(e);
            free_all(h);
            delete h;
            return LBM_ECUDA;
        }
    }

    lbm_status st = LBM_OK;
    auto fail = [&](lbm_status s) {
        g_thread_err = h->err;
        free_all(h);
        delete h;
        return s;
    };
#define CKC(expr, what)                                  \
    do {                                                 \
        cudaError_t e_ = (expr);                         \
        if (e_ != cudaSuccess) return fail(cuda_err(h, e_, what)); \
    } while (0)
#define ALLOC(ptr, type, bytes)                                                       \
    do {                                                                              \
        ptr = (type)dev_alloc(h, (bytes));                                            \
        if (!ptr) return fail(set_err(h, LBM_ENOMEM, "device allocation of %zu bytes failed", (size_t)(bytes))); \
    } while (0)

    const size_t N = (size_t)nx * ny;
    // The staged kernel copies whole row segments starting 16 bytes before a
    // tile and ending past the last column; guard bytes before and after each
    // buffer keep those copies inside the allocation (their values are never used).
    const size_t pop_bytes = 9 * (size_t)h->plane * h->elem;
    const size_t guard_front = 256, guard_back = 2048;
    for (int b = 0; b < NBUF; ++b) {
        ALLOC(h->pop_base[b], void *, guard_front + pop_bytes + guard_back);
        h->pop[b] = (char *)h->pop_base[b] + guard_front;
        // bulk copies and prefetches of rows start on 16-byte boundaries
        if ((uintptr_t)h->pop_base[b] & 15)
            return fail(set_err(h, LBM_EINVAL, "the allocator returned a pointer that is not 16-byte aligned"));
    }
    if (h->use_bulk) {
        h->tmap_ok = true;
        for (int b = 0; b < NBUF; ++b)
            h->tmap_ok = h->tmap_ok && encode_tensor_map(&h->tmap[b], h->storage, h->pop[b], h->pitch, ny);
        if (!h->tmap_ok)
            return fail(set_err(h, LBM_ECUDA, "tensor maps for the staged kernel could not be encoded"));
    }
    ALLOC(h->mask_d, uint8_t *, N);
    ALLOC(h->nbits, uint16_t *, sizeof(uint16_t) * h->plane);
    ALLOC(h->tile_flag, uint8_t *, (size_t)h->tiles_x * h->tiles_y);
    ALLOC(h->u_row, double *, sizeof(double) * ny);
    ALLOC(h->inlet, void *, 9 * (size_t)ny * h->elem);
    ALLOC(h->partials, double *, sizeof(double) * NBUF * CV_PARTIAL * h->n_cv_tiles);
    ALLOC(h->link_partials, double *, sizeof(double) * LINK_PARTIAL * MAX_LINK_CTAS * LINK_WARPS);
    ALLOC(h->ticket, unsigned int *, sizeof(unsigned int));
    ALLOC(h->carry, double *, sizeof(double) * 8);
    ALLOC(h->step_ctr, long long *, sizeof(long long));
    ALLOC(h->status, int *, sizeof(int) * 2);
    st = ensure_series(h, 1024);
    if (st != LBM_OK) return fail(st);

    std::vector<double> urow(ny);
    for (int y = 0; y < ny; ++y) urow[y] = n_u_in == 1 ? u_in[0] : u_in[y];
    cudaStream_t s = h->stream;
    for (int b = 0; b < NBUF; ++b)
        CKC(cudaMemsetAsync(h->pop_base[b], 0, guard_front + pop_bytes + guard_back, s), "memset");
    CKC(cudaMemsetAsync(h->nbits, 0, sizeof(uint16_t) * h->plane, s), "memset");
    CKC(cudaMemsetAsync(h->partials, 0, sizeof(double) * NBUF * CV_PARTIAL * h->n_cv_tiles, s), "memset");
    CKC(cudaMemsetAsync(h->ticket, 0, sizeof(unsigned int), s), "memset");
    CKC(cudaMemsetAsync(h->carry, 0, sizeof(double) * 8, s), "memset");
    CKC(cudaMemsetAsync(h->step_ctr, 0, sizeof(long long), s), "memset");
    const int status0[2] = {0, INT_MAX};
    CKC(cudaMemcpyAsync(h->status, status0, sizeof(status0), cudaMemcpyHostToDevice, s), "H2D status");
    h->status_armed = true;
    CKC(cudaMemcpyAsync(h->mask_d, mask, N, cudaMemcpyHostToDevice, s), "H2D mask");
    CKC(cudaMemcpyAsync(h->u_row, urow.data(), sizeof(double) * ny, cudaMemcpyHostToDevice, s), "H2D u_in");
    CKC(launch_node_bits(h->mask_d, h->nbits, nx, ny, h->pitch, periodic, s), "node bits");
    CKC(launch_tile_flags(h->nbits, nx, ny, h->pitch, periodic, h->tile_flag, h->tiles_x, h->tiles_y,
                          TILE_X, tile_rows(h->storage), s),
        "tile flags");
    std::vector<uint8_t> flags((size_t)h->tiles_x * h->tiles_y);
    CKC(cudaMemcpyAsync(flags.data(), h->tile_flag, flags.size(), cudaMemcpyDeviceToHost, s), "D2H tile flags");
    // link list: count, scan, scatter
    const int nb = link_blocks(nx, ny);
    int *blk = nullptr;
    long long *total_d = nullptr;
    ALLOC(blk, int *, sizeof(int) * nb);
    total_d = (long long *)dev_alloc(h, sizeof(long long));
    if (!total_d) {
        dev_free(h, blk);
        return fail(set_err(h, LBM_ENOMEM, "device allocation failed"));
    }
    cudaError_t le = launch_link_count(h->nbits, nx, ny, h->pitch, blk, nb, s);
    if (le == cudaSuccess) le = launch_scan_blocks(blk, nb, total_d, s);
    long long total = 0;
    if (le == cudaSuccess) le = cudaMemcpyAsync(&total, total_d, sizeof(total), cudaMemcpyDeviceToHost, s);
    // the host's scan of the mask for the deviation base sums runs while the
    // device builds the node bits and counts the links
    if (bc.storage == LBM_F32_DEV || bc.storage == LBM_F16_DEV)
        base_sums(mask, nx, ny, periodic, h->cv, bc.rho0, h->link_base, h->flux_base, &solids);
    if (le == cudaSuccess) le = cudaStreamSynchronize(s);
    if (le == cudaSuccess) {
        // the tile rows holding bounce-back tiles run first in each step (a
        // body's rows; rows spread over more than half the grid keep their order)
        int r0 = h->tiles_y, r1 = -1;
        for (int ty = 0; ty < h->tiles_y; ++ty)
            for (int tx = 0; tx < h->tiles_x; ++tx)
                if (flags[(size_t)ty * h->tiles_x + tx]) {
                    r0 = ty < r0 ? ty : r0;
                    r1 = ty > r1 ? ty : r1;
                    break;
                }
        if (GBLBM_BODY_ROWS_FIRST && r1 >= r0 && 2 * (r1 - r0 + 1) <= h->tiles_y) {
            h->first_r0 = r0;
            h->first_r1 = r1;
        }
        h->nlinks = total;
        {
            long long work = total > h->n_cv_tiles ? total : h->n_cv_tiles;
            long long c = (work + LINK_THREADS - 1) / LINK_THREADS;
            h->link_ctas = (int)(c < 1 ? 1 : (c > MAX_LINK_CTAS ? MAX_LINK_CTAS : c));
        }
        h->links = (int32_t *)dev_alloc(h, sizeof(int32_t) * (total > 0 ? total : 1));
        if (!h->links) {
            dev_free(h, blk);
            dev_free(h, total_d);
            return fail(set_err(h, LBM_ENOMEM, "device allocation of the link list failed"));
        }
        le = launch_link_scatter(h->nbits, nx, ny, h->pitch, blk, h->links, total, s);
    }
    if (le == cudaSuccess) le = cudaStreamSynchronize(s);
    dev_free(h, blk);
    dev_free(h, total_d);
    if (le != cudaSuccess) return fail(cuda_err(h, le, "link list"));
    {
        ALLOC(h->bnodes, int32_t *, sizeof(int32_t) * (h->nlinks > 0 ? h->nlinks : 1));
        long long *cnt_d = (long long *)dev_alloc(h, sizeof(long long));
        if (!cnt_d) return fail(set_err(h, LBM_ENOMEM, "device allocation failed"));
        cudaError_t be = launch_boundary_nodes(h->links, h->nlinks, h->bnodes, cnt_d, s);
        if (be == cudaSuccess) be = cudaMemcpyAsync(&h->n_bnodes, cnt_d, sizeof(long long), cudaMemcpyDeviceToHost, s);
        if (be == cudaSuccess) be = cudaStreamSynchronize(s);
        dev_free(h, cnt_d);
        if (be != cudaSuccess) return fail(cuda_err(h, be, "boundary nodes"));
    }
    CKC(launch_init(h->storage, h->pop[0], h->plane, h->mask_d, nx, ny, h->pitch, h->u_row, h->rho0,
                    h->inlet, s, n_u_in == 1),
        "initial state");
    CKC(cudaStreamSynchronize(s), "sync");
    h->launches = 7;
#undef CKC
#undef ALLOC
    *out = h;
    return LBM_OK;
}

namespace {

// Clears the status words for the steps about to be queued, unless the last
// settle already did: status[0] = 0 (no flag), status[1] = 0x7f7f7f7f (no bad
// step yet).
lbm_status arm_status(lbm_ctx *h)
{
    if (h->status_armed) return LBM_OK;
    CK(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream), "status reset");
    CK(h, cudaMemsetAsync(h->status + 1, 0x7f, sizeof(int), h->stream), "status reset");
    h->status_armed = true;
    return LBM_OK;
}

// Queues n steps on the handle's stream without waiting for them.  The
// status words are cleared before the first queued step after a settle and
// then collect the flags of every step until the next settle.
lbm_status queue_steps(lbm_ctx *h, int n)
{
    lbm_status st = ensure_series(h, h->t + n);
    if (st == LBM_OK) st = arm_status(h);
    if (st != LBM_OK) return st;
    if (h->timing && (int)h->events.size() < 3 * TIMING_BATCH) {
        h->events.resize(3 * TIMING_BATCH, nullptr);
        for (auto &e : h->events)
            if (!e) CK(h, cudaEventCreate(&e), "event create");
    }
    int nev = 0;
    while (n > 0) {
        if (h->precollision || h->timing || n < NBUF) {
            cudaEvent_t *ev = h->timing ? &h->events[3 * nev] : nullptr;
            CK(h, launch_one_step(h, h->cur, h->precollision, ev), "step launch");
            if (h->timing && ++nev == TIMING_BATCH) {
                st = flush_timing(h, nev);
                if (st != LBM_OK) return st;
                nev = 0;
            }
            h->cur = next_buf(h->cur);
            h->precollision = 0;
            h->t += 1;
            n -= 1;
        } else {
            int k = n >= GRAPH_STEPS ? 0 : 1;
            int steps = k == 0 ? GRAPH_STEPS : NBUF;
            // a held link kernel of the step before opens the graph
            const int lead = h->lead_src == prev_buf(h->cur) && !h->lead_pre ? 1 : 0;
            if (!lead) CK(h, flush_link(h), "link launch");
            // the graph's first steps overwrite buffers that launched link kernels read
            CK(h, join_side(h), "join");
            if (!h->graph[h->cur][k][lead]) {
                st = build_graph(h, h->cur, k, lead);
                if (st != LBM_OK) return st;
            }
            CK(h, cudaGraphLaunch(h->graph[h->cur][k][lead], h->stream), "graph launch");
            h->lead_src = prev_buf(h->cur);  // steps is a multiple of NBUF
            h->lead_pre = 0;
            h->launches += 2 * steps - 1 + lead;  // the last link kernel is held
            h->t += steps;
            n -= steps;
        }
    }
    CK(h, flush_link(h), "link launch");
    CK(h, join_side(h), "join");
    if (h->timing) {
        st = flush_timing(h, nev);
        if (st != LBM_OK) return st;
    }
    h->pending = true;
    return LBM_OK;
}

// Queues n eager steps whose states are kept for a backward sweep: step j
// (0-based) reads slot j and writes slot j + 1 of `slots` (stride bytes
// apart; slot 0 holds a copy of the current state), except the last step,
// which writes the handle's own next buffer.  Each step points the logical
// buffer it writes at its slot, so the kernels, the held link kernels and the
// force series are exactly those of queue_steps; only the population
// addresses differ.  The direct collide-stream kernel serves these steps (the
// staged kernel's tensor maps describe the handle's own buffers).
lbm_status queue_steps_keep(lbm_ctx *h, int n, char *slots, size_t stride)
{
    lbm_status st = ensure_series(h, h->t + n);
    if (st == LBM_OK) st = arm_status(h);
    if (st != LBM_OK) return st;
    void *orig[NBUF];
    for (int b = 0; b < NBUF; ++b) orig[b] = h->pop[b];
    const int bulk = h->use_bulk;
    h->use_bulk = 0;
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < n && e == cudaSuccess; ++j) {
        const int db = next_buf(h->cur);
        // the held link kernel of step j-1 reads buffers prev(cur) and cur,
        // whose addresses stay as they were
        h->pop[db] = j + 1 < n ? (void *)(slots + (size_t)(j + 1) * stride) : orig[db];
        e = launch_one_step(h, h->cur, h->precollision, nullptr);
        h->cur = db;
        h->precollision = 0;
        h->t += 1;
    }
    if (e == cudaSuccess) e = flush_link(h);
    if (e == cudaSuccess) e = join_side(h);
    // launches took their arguments by value: the handle's buffers are its own again
    for (int b = 0; b < NBUF; ++b) h->pop[b] = orig[b];
    h->use_bulk = bulk;
    h->pending = true;
    if (e != cudaSuccess) return cuda_err(h, e, "adjoint forward steps");
    return LBM_OK;
}

// Waits for the queued steps and turns their status words into a result.
lbm_status settle(lbm_ctx *h)
{
    if (!h->pending) return LBM_OK;
    h->pending = false;
    h->status_armed = false;
    CK(h, cudaMemcpyAsync(h->status_host, h->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream),
       "D2H status");
    // clear the words for the next queue here, so that its start waits on nothing
    CK(h, cudaMemsetAsync(h->status, 0, sizeof(int), h->stream), "status reset");
    CK(h, cudaMemsetAsync(h->status + 1, 0x7f, sizeof(int), h->stream), "status reset");
    CK(h, cudaStreamSynchronize(h->stream), "step sync");
    h->status_armed = true;
    const int *status = h->status_host;
    if (h->t - 1 > h->carry_from) h->drtt_ready = h->t - 1 > h->drtt_ready ? h->t - 1 : h->drtt_ready;
    if (status[0] & 4)
        return set_err(h, LBM_ESTATE, "a force-series row lay beyond the series buffer");
    if (status[0] & 2)
        return set_err(h, LBM_ETIMEOUT, "a bounded wait for staged copies expired");
    if (status[0]) return set_err(h, LBM_EUNSTABLE, "rho <= 0 or NaN first seen at step %d", status[1]);
    return LBM_OK;
}

#define SETTLE(h)                          \
    do {                                   \
        lbm_status s_ = settle(h);         \
        if (s_ != LBM_OK) return s_;       \
    } while (0)

}  // namespace

lbm_status lbm_step(lbm_ctx *h, int n)
{
    if (!h) return set_err(nullptr, LBM_EINVAL, "NULL handle");
    if (n < 0) return set_err(h, LBM_EINVAL, "n must be >= 0");
    SETTLE(h);
    if (n == 0) return LBM_OK;
    lbm_status st = queue_steps(h, n);
    if (st != LBM_OK) return st;
    return settle(h);
}

lbm_status lbm_step_async(lbm_ctx *h, int n)
{
    if (!h) return set_err(nullptr, LBM_EINVAL, "NULL handle");
    if (n < 0) return set_err(h, LBM_EINVAL, "n must be >= 0");
    if (n == 0) return LBM_OK;
    return queue_steps(h, n);
}

lbm_status lbm_sync(lbm_ctx *h)
{
    if (!h) return set_err(nullptr, LBM_EINVAL, "NULL handle");
    return settle(h);
}

lbm_status lbm_force_series(lbm_ctx *h, int scheme, long first, long count, double *fx, double *fy)
{
    if (!h) return set_err(nullptr, LBM_EINVAL, "NULL handle");
    SETTLE(h);
    if (scheme < 0 || scheme > LBM_FORCE_SI) return set_err(h, LBM_EINVAL, "unknown scheme %d", scheme);
    if (count < 0 || first < 0 || first + count > h->t)
        return set_err(h, LBM_EINVAL, "steps [%ld, %ld) outside [0, %lld)", first, first + count, h->t);
    if (count == 0) return LBM_OK;
    if (!fx || !fy) return set_err(h, LBM_EINVAL, "fx and fy must not be NULL");
    if (!h->record_series && first < h->t - 2)
        return set_err(h, LBM_EINVAL, "only the last two steps are kept (record_series = 0)");
    if (scheme == LBM_FORCE_DRTT && first + count > h->drtt_ready) {
        lbm_status st = finalize_drtt(h);
        if (st != LBM_OK) return st;
    }
    const size_t R = SERIES_ROW;
    std::vector<double> rows((size_t)count * R);
    if (h->record_series) {
        CK(h, cudaMemcpyAsync(rows.data(), h->series + R * first, sizeof(double) * R * count,
                              cudaMemcpyDeviceToHost, h->stream),
           "D2H series");
    } else {
        for (long k = 0; k < count; ++k)
            CK(h, cudaMemcpyAsync(rows.data() + R * k, h->series + R * ((first + k) & 1),
                                  sizeof(double) * R, cudaMemcpyDeviceToHost, h->stream),
               "D2H series");
    }
    CK(h, cudaStreamSynchronize(h->stream), "sync");
    const int col = 2 * scheme;  // row: A, B, DRTT, A', defect, SI (x, y each)
    for (long k = 0; k < count; ++k) {
        fx[k] = rows[R * k + col];
        fy[k] = rows[R * k + col + 1];
    }
    return LBM_OK;
}

lbm_status lbm_set_kernel(lbm_ctx *h, int kernel)
{
    if (!h) return set_err(nullptr, LBM_EINVAL, "NULL handle");
    SETTLE(h);
    if (kernel != 0 && kernel != 1) return set_err(h, LBM_EINVAL, "unknown kernel choice %d", kernel);
    if (kernel == 1 && !h->tmap_ok)
        return set_err(h, LBM_EINVAL, "the staged kernel needs a handle created with kernel = 1");
    if ((kernel == 1) != (h->use_bulk != 0)) {
        CK(h, cudaStreamSynchronize(h->stream), "sync");
        drop_graphs(h);
        h->use_bulk = kernel;
    }
    return LBM_OK;
}

lbm_status lbm_set_wait_limit(lbm_ctx *h, long polls)
{
    if (!h) return set_err(nullptr, LBM_EINVAL, "NULL handle");
    SETTLE(h);
    const unsigned int lim = polls < 0 ? WAIT_LIMIT : (polls > (long)WAIT_LIMIT ? WAIT_LIMIT : (unsigned int)polls);
    if (lim != h->wait_limit) {
        CK(h, cudaStreamSynchronize(h->stream), "sync");
        drop_graphs(h);
        h->wait_limit = lim;
    }
    return LBM_OK;
}

lbm_status lbm_prepare(lbm_ctx *h, long n)
{
    if (!h) return set_err(nullptr, LBM_EINVAL, "NULL handle");
    SETTLE(h);
    if (n < 0) return set_err(h, LBM_EINVAL, "n must be >= 0");
    lbm_status st = ensure_series(h, h->t + n);
    if (st != LBM_OK) return st;
    for (int p = 0; p < NBUF; ++p)
        for (int k = 0; k < 2; ++k)
            for (int l = 0; l < 2; ++l)
                if (!h->graph[p][k][l]) {
                    st = build_graph(h, p, k, l);
                    if (st != LBM_OK) return st;
                }
    return LBM_OK;
}

lbm_status lbm_coefficients(lbm_ctx *h, int scheme, long first, long count, double length, double u_ref,
                            double *cd, double *cl, double *stats)
{
    if (!h) return set_err(nullptr, LBM_EINVAL, "NULL handle");
    SETTLE(h);
    if (scheme < 0 || scheme > LBM_FORCE_SI) return set_err(h, LBM_EINVAL, "unknown scheme %d", scheme);
    if (count < 1 || first < 0 || first + count > h->t)
        return set_err(h, LBM_EINVAL, "steps [%ld, %ld) outside [0, %lld) or empty", first, first + count, h->t);
    if (!(length > 0) || !std::isfinite(length) || !(u_ref != 0) || !std::isfinite(u_ref))
        return set_err(h, LBM_EINVAL, "length must be > 0 and u_ref nonzero, both finite");
    if (!h->record_series && first < h->t - 2)
        return set_err(h, LBM_EINVAL, "only the last two steps are kept (record_series = 0)");
    if (scheme == LBM_FORCE_DRTT && first + count > h->drtt_ready) {
        lbm_status st = finalize_drtt(h);
        if (st != LBM_OK) return st;
    }
    const double norm = 2.0 / (h->rho0 * u_ref * u_ref * length);
    const bool per_step = cd || cl;
    double *out = (double *)dev_alloc(h, sizeof(double) * (4 + (per_step ? 2 * (size_t)count : 0)));
    if (!out) return set_err(h, LBM_ENOMEM, "coefficient buffer allocation failed");
    cudaError_t e = launch_coefficients(h->series, SERIES_ROW, 2 * scheme, first, count, !h->record_series, norm,
                                        out, per_step, h->stream);
    double st4[4];
    if (e == cudaSuccess) e = cudaMemcpyAsync(st4, out, sizeof(st4), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && cd)
        e = cudaMemcpyAsync(cd, out + 4, sizeof(double) * count, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess && cl)
        e = cudaMemcpyAsync(cl, out + 4 + count, sizeof(double) * count, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dev_free(h, out);
    h->launches += 1;
    if (e != cudaSuccess) return cuda_err(h, e, "coefficients");
    if (stats) memcpy(stats, st4, sizeof(st4));
    return LBM_OK;
}

lbm_status lbm_force(lbm_ctx *h, int scheme, double *fx, double *fy)
{
    if (!h) return set_err(nullptr, LBM_EINVAL, "NULL handle");
    SETTLE(h);
    if (h->t < 1) return set_err(h, LBM_ESTATE, "no step has been taken");
    return lbm_force_series(h, scheme, (long)(h->t - 1), 1, fx, fy);
}

lbm_status lbm_populations(lbm_ctx *h, double *out)
{
    if (!h) return set_err(nullptr, LBM_EINVAL, "NULL handle");
    SETTLE(h);
    if (!out) return set_err(h, LBM_EINVAL, "out must not be NULL");
    const size_t N = (size_t)h->nx * h->ny;
    double *scratch = (double *)dev_alloc(h, sizeof(double) * N);
    if (!scratch) return set_err(h, LBM_ENOMEM, "scratch allocation failed");
    lbm_status st = LBM_OK;
    for (int i = 0; i < 9 && st == LBM_OK; ++i) {
        cudaError_t e = launch_gather(h->storage, h->pop[h->cur], h->nbits, h->inlet, h->plane, h->nx,
                                      h->ny, h->pitch, h->periodic, h->precollision, h->rho0, i,
                                      scratch, h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out + i * N, scratch, sizeof(double) * N, cudaMemcpyDeviceToHost,
                                h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) st = cuda_err(h, e, "gather populations");
        h->launches += 1;
    }
    dev_free(h, scratch);
    return st;
}

lbm_status lbm_set_populations(lbm_ctx *h, const double *in)
{
    if (!h) return set_err(nullptr, LBM_EINVAL, "NULL handle");
    SETTLE(h);
    if (!in) return set_err(h, LBM_EINVAL, "in must not be NULL");
    const size_t N = (size_t)h->nx * h->ny;
    for (size_t k = 0; k < 9 * N; ++k)
        if (!std::isfinite(in[k])) return set_err(h, LBM_EINVAL, "populations must be finite");
    if (h->t >= 1 && h->drtt_ready < h->t && !h->precollision && h->t - 1 >= h->carry_from) {
        lbm_status st = finalize_drtt(h);
        if (st != LBM_OK) return st;
    }
    double *scratch = (double *)dev_alloc(h, sizeof(double) * N);
    if (!scratch) return set_err(h, LBM_ENOMEM, "scratch allocation failed");
    lbm_status st = LBM_OK;
    for (int i = 0; i < 9 && st == LBM_OK; ++i) {
        cudaError_t e = cudaMemcpyAsync(scratch, in + i * N, sizeof(double) * N, cudaMemcpyHostToDevice,
                                        h->stream);
        if (e == cudaSuccess)
            e = launch_scatter_pop(h->storage, h->pop[h->cur], h->nbits, h->plane, h->nx, h->ny,
                                   h->pitch, h->rho0, i, scratch, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) st = cuda_err(h, e, "set populations");
        h->launches += 1;
    }
    dev_free(h, scratch);
    if (st != LBM_OK) return st;
    CK(h, cudaMemsetAsync(h->carry, 0, sizeof(double) * 8, h->stream), "memset carry");
    CK(h, cudaStreamSynchronize(h->stream), "sync");
    h->precollision = 1;
    h->carry_from = h->t;
    if (h->drtt_ready < h->t) h->drtt_ready = h->t;
    return LBM_OK;
}

lbm_status lbm_pressure_coefficient(lbm_ctx *h, double p_inf, double q, int32_t *nodes, double *cp, long cap,
                                    long *count)
{
    if (!h) return set_err(nullptr, LBM_EINVAL, "NULL handle");
    SETTLE(h);
    if (!std::isfinite(p_inf) || !std::isfinite(q) || q == 0.0)
        return set_err(h, LBM_EINVAL, "p_inf must be finite and q finite and nonzero");
    if (count) *count = (long)h->n_bnodes;
    const long n = cap < (long)h->n_bnodes ? cap : (long)h->n_bnodes;
    if (n <= 0) return LBM_OK;
    if (nodes)
        CK(h, cudaMemcpyAsync(nodes, h->bnodes, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, h->stream), "D2H nodes");
    if (cp) {
        double *d = (double *)dev_alloc(h, sizeof(double) * h->n_bnodes);
        if (!d) return set_err(h, LBM_ENOMEM, "scratch allocation failed");
        cudaError_t e = launch_surface_pressure(h->storage, h->pop[h->cur], h->nbits, h->bnodes, h->n_bnodes, h->plane,
                                                h->nx, h->ny, h->pitch, h->periodic, h->precollision, h->rho0, p_inf,
                                                q, d, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cp, d, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        dev_free(h, d);
        h->launches += 1;
        if (e != cudaSuccess) return cuda_err(h, e, "surface pressure");
    }
    CK(h, cudaStreamSynchronize(h->stream), "sync");
    return LBM_OK;
}

lbm_status lbm_links(lbm_ctx *h, int32_t *out, long cap, long *count)
{
    if (!h) return set_err(nullptr, LBM_EINVAL, "NULL handle");
    if (count) *count = (long)h->nlinks;
    long n = cap < (long)h->nlinks ? cap : (long)h->nlinks;
    if (n > 0) {
        if (!out) return set_err(h, LBM_EINVAL, "out must not be NULL");
        CK(h, cudaMemcpyAsync(out, h->links, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, h->stream),
           "D2H links");
        CK(h, cudaStreamSynchronize(h->stream), "sync");
    }
    return LBM_OK;
}

lbm_status lbm_control_volume(lbm_ctx *h, int *cv)
{
    if (!h || !cv) return set_err(h, LBM_EINVAL, "NULL argument");
    memcpy(cv, h->cv, sizeof(h->cv));
    return LBM_OK;
}

lbm_status lbm_naca_mask(int nx, int ny, double chord, double thickness, double alpha_deg,
                         double xc, double yc, int closed_te, uint8_t *out)
{
    if (nx <= 0 || ny <= 0 || !(chord > 0) || !(thickness > 0) || !out || !std::isfinite(alpha_deg) ||
        !std::isfinite(xc) || !std::isfinite(yc))
        return set_err(nullptr, LBM_EINVAL, "bad NACA section arguments");
    double a = alpha_deg * M_PI / 180.0;
    double ca = cos(a), sa = sin(a);
    size_t N = (size_t)nx * ny;
    uint8_t *d = nullptr;
    cudaError_t e = cudaMalloc(&d, N);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_err(nullptr, e, "cudaMalloc mask");
    }
    e = launch_naca_mask(d, nx, ny, chord, thickness, ca, sa, xc, yc, closed_te, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, d, N, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_err(nullptr, e, "NACA mask");
    return LBM_OK;
}

lbm_status lbm_cylinder_mask(int nx, int ny, double xc, double yc, double diameter, uint8_t *out)
{
    if (nx <= 0 || ny <= 0 || !(diameter > 0) || !std::isfinite(diameter) || !out || !std::isfinite(xc) ||
        !std::isfinite(yc))
        return set_err(nullptr, LBM_EINVAL, "bad cylinder arguments");
    const size_t N = (size_t)nx * ny;
    uint8_t *d = nullptr;
    cudaError_t e = cudaMalloc(&d, N);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_err(nullptr, e, "cudaMalloc mask");
    }
    e = launch_cylinder_mask(d, nx, ny, xc, yc, 0.5 * diameter, 0);
    if (e == cudaSuccess) e = cudaMemcpy(out, d, N, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_err(nullptr, e, "cylinder mask");
    return LBM_OK;
}

lbm_status lbm_adjoint(lbm_ctx *h, int steps, int window, double wx, double wy, int checkpoint_every,
                       double *J, double *dJ_dtau, double *dJ_du, double *dJ_df0)
{
    if (!h) return set_err(nullptr, LBM_EINVAL, "NULL handle");
    SETTLE(h);
    if (steps < 1 || window < 1 || window > steps)
        return set_err(h, LBM_EINVAL, "need 1 <= window <= steps (got %d, %d)", window, steps);
    if (h->periodic) return set_err(h, LBM_EINVAL, "the adjoint covers the channel set-up only");
    if (h->g[0] != 0.0 || h->g[1] != 0.0)
        return set_err(h, LBM_EINVAL, "the adjoint does not cover a body force");
    if (!h->record_series) return set_err(h, LBM_EINVAL, "the adjoint needs record_series = 1");
    if (!std::isfinite(wx) || !std::isfinite(wy)) return set_err(h, LBM_EINVAL, "weights not finite");
    const size_t buf_bytes = 9 * (size_t)h->plane * h->elem;
    const size_t comp = h->storage == LBM_F64 ? 8 : 4;
    const size_t comp_bytes = 9 * (size_t)h->plane * comp;
    const int nblk = adjoint_blocks(h->nx, h->ny);
    cudaStream_t st = h->stream;
    auto isqrt_up = [](long long n) {
        long long k = 1;
        while (k * k < n) ++k;
        return (int)k;
    };
    // Plan.  The last L steps keep the states the forward pass writes (no
    // recompute); the first F = steps - L are checkpointed every K steps and
    // recomputed segment by segment.  With checkpoint_every <= 0, L is as
    // large as ADJ_KEEP_SHARE of the free device memory allows, counting the
    // checkpoints and segment buffers the first F steps then need.
    int L = 0;
    if (checkpoint_every <= 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            fr = 0;
        }
        const double reserve = 2.0 * comp_bytes + 72.0 * h->nx * h->ny + (double)(1u << 30);
        const double avail = (h->adj_budget > 0 ? h->adj_budget : ADJ_KEEP_SHARE * (double)fr) - reserve;
        const long long slots = avail > 0 ? (long long)(avail / (double)buf_bytes) : 0;
        auto need = [&](long long keep) {
            const long long f = steps - keep;
            if (f <= 0) return keep;
            const long long k = isqrt_up(f);
            return keep + (f + k - 1) / k + (k - 1);
        };
        for (long long keep = slots < steps ? slots : steps; keep > 0; --keep)
            if (need(keep) <= slots) {
                L = (int)keep;
                break;
            }
    }

    std::vector<void *> owned;
    auto grab = [&](size_t bytes) {
        void *p = dev_alloc(h, bytes);
        if (p) owned.push_back(p);
        return p;
    };
    auto release = [&]() {
        cudaStreamSynchronize(st);
        for (void *p : owned) dev_free(h, p);
        owned.clear();
    };
    // the kept states of the last L steps (slot j: the state step F + j reads)
    char *keep = L > 0 ? (char *)grab(buf_bytes * (size_t)L) : nullptr;
    if (!keep) L = 0;  // no room after all: checkpoints only
    const int F = steps - L;
    int K = checkpoint_every > 0 ? checkpoint_every : isqrt_up(F);
    if (K > F) K = F > 0 ? F : 1;
    const int nck = F > 0 ? (F + K - 1) / K : 0;
    // checkpoints; the recomputed post-collision states of one segment (the
    // first step of a segment reads its checkpoint, step s > 0 the state
    // written by step s-1, so K-1 buffers); the adjoint pair lam(t+1), lam(t)
    char *ck = nck > 0 ? (char *)grab(buf_bytes * nck) : nullptr;
    char *seg = nck > 0 && K > 1 ? (char *)grab(buf_bytes * (K - 1)) : nullptr;
    char *lam_a = (char *)grab(comp_bytes), *lam_b = (char *)grab(comp_bytes);
    double *part = (double *)grab(sizeof(double) * CV_PARTIAL * h->n_cv_tiles);
    double *du_acc = (double *)grab(sizeof(double) * h->ny);
    double *dw_acc = (double *)grab(sizeof(double) * nblk);
    double *dw_out = (double *)grab(sizeof(double));
    if ((nck > 0 && !ck) || (nck > 0 && K > 1 && !seg) || !lam_a || !lam_b || !part || !du_acc || !dw_acc ||
        !dw_out) {
        release();
        return set_err(h, LBM_ENOMEM, "adjoint: allocation of checkpoints / work arrays failed");
    }
    std::vector<int> ckpre(nck);
    const long long T0 = h->t;
    lbm_status rs = LBM_OK;
    // forward: checkpoint, then K steps
    for (int k = 0; k < nck; ++k) {
        cudaError_t e = cudaMemcpyAsync(ck + buf_bytes * k, h->pop[h->cur], buf_bytes,
                                        cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) {
            release();
            return cuda_err(h, e, "adjoint: checkpoint copy");
        }
        ckpre[k] = h->precollision;
        const int n = (k + 1) * K <= F ? K : F - k * K;
        rs = lbm_step(h, n);
        if (rs != LBM_OK) {
            release();
            return rs;
        }
    }
    // the kept steps write their states into the slots as they go
    int keep_pre = 0;
    if (L > 0) {
        cudaError_t e = cudaMemcpyAsync(keep, h->pop[h->cur], buf_bytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) {
            release();
            return cuda_err(h, e, "adjoint: state copy");
        }
        keep_pre = h->precollision;
        rs = queue_steps_keep(h, L, keep, buf_bytes);
        if (rs == LBM_OK) rs = settle(h);
        if (rs != LBM_OK) {
            release();
            return rs;
        }
    }
    // J from the algorithm-B series of the window
    {
        std::vector<double> fx(window), fy(window);
        rs = lbm_force_series(h, LBM_FORCE_MEA_B, (long)(T0 + steps - window), window, fx.data(),
                              fy.data());
        if (rs != LBM_OK) {
            release();
            return rs;
        }
        double s = 0.0;
        for (int k = 0; k < window; ++k) s += wx * fx[k] + wy * fy[k];
        if (J) *J = s / window;
    }
    // backward over the segments, each recomputed from its checkpoint
    cudaError_t e = cudaMemsetAsync(lam_b, 0, comp_bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(lam_a, 0, comp_bytes, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(du_acc, 0, sizeof(double) * h->ny, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dw_acc, 0, sizeof(double) * nblk, st);
    char *lam_next = lam_b, *lam_cur = lam_a;  // lam(T) = 0
    const double obj_x = 2.0 * wx / window, obj_y = 2.0 * wy / window;
    // the kept steps, last to first: their states need no recompute
    for (int j = L - 1; j >= 0 && e == cudaSuccess; --j) {
        const int t = F + j;
        e = launch_adjoint_step(h->storage, keep + buf_bytes * (size_t)j, j == 0 ? keep_pre : 0, lam_next, lam_cur,
                                h->nbits, h->tile_flag, tile_rows(h->storage), h->tiles_x, h->u_row, du_acc, dw_acc,
                                h->plane, h->nx, h->ny, h->pitch, t >= steps - window, h->omega, h->rho0, obj_x,
                                obj_y, st);
        char *tmp = lam_next;
        lam_next = lam_cur;
        lam_cur = tmp;
        h->launches += 1;
    }
    for (int k = nck - 1; k >= 0 && e == cudaSuccess; --k) {
        const int t0 = k * K;
        const int n = (k + 1) * K <= F ? K : F - t0;
        // the state step t0 + s reads
        auto state = [&](int s) { return s == 0 ? ck + buf_bytes * k : seg + buf_bytes * (s - 1); };
        for (int s = 0; s + 1 < n && e == cudaSuccess; ++s) {
            StepArgs sa = step_args(h, h->cur, next_buf(h->cur), s == 0 ? ckpre[k] : 0);
            sa.src = state(s);
            sa.dst = state(s + 1);
            sa.partials = part;
            sa.use_bulk = 0;
            e = launch_collide_stream(h->storage, sa, h->tiles_x, h->tiles_y, false, nullptr, st);
            h->launches += 1;
        }
        for (int s = n - 1; s >= 0 && e == cudaSuccess; --s) {
            const int t = t0 + s;
            e = launch_adjoint_step(h->storage, state(s), s == 0 ? ckpre[k] : 0, lam_next, lam_cur, h->nbits,
                                    h->tile_flag, tile_rows(h->storage), h->tiles_x, h->u_row, du_acc, dw_acc,
                                    h->plane, h->nx, h->ny, h->pitch,
                                    t >= steps - window, h->omega, h->rho0, obj_x, obj_y, st);
            char *tmp = lam_next;
            lam_next = lam_cur;
            lam_cur = tmp;
            h->launches += 1;
        }
    }
    if (e == cudaSuccess) e = launch_sum_fixed(dw_acc, nblk, dw_out, h->storage != LBM_F64, st);
    double dw = 0.0;
    std::vector<double> du(h->ny);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&dw, dw_out, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(du.data(), du_acc, sizeof(double) * h->ny, cudaMemcpyDeviceToHost, st);
    // dJ/df0 = lambda(T0) in FP64, assembled on the device: straight into
    // dJ_df0 when it is device memory, else into a scratch array copied once
    if (e == cudaSuccess && dJ_df0) {
        const size_t N = (size_t)h->nx * h->ny;
        cudaPointerAttributes pa;
        bool on_device = false;
        if (cudaPointerGetAttributes(&pa, dJ_df0) == cudaSuccess)
            on_device = pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged;
        else
            cudaGetLastError();
        double *out = on_device ? dJ_df0 : (double *)grab(sizeof(double) * 9 * N);
        if (!out) {
            release();
            return set_err(h, LBM_ENOMEM, "adjoint: allocation of the dJ/df0 array failed");
        }
        e = launch_adjoint_df0(h->storage, lam_next, h->mask_d, h->plane, h->nx, h->ny, h->pitch, h->sm_count, out,
                               st);
        h->launches += 1;
        if (e == cudaSuccess && !on_device)
            e = cudaMemcpyAsync(dJ_df0, out, sizeof(double) * 9 * N, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    release();
    if (e != cudaSuccess) return cuda_err(h, e, "adjoint");
    if (dJ_dtau) *dJ_dtau = -dw / (h->tau * h->tau);
    if (dJ_du)
        for (int y = 0; y < h->ny; ++y) dJ_du[y] = du[y];
    return LBM_OK;
}

lbm_status lbm_set_adjoint_budget(lbm_ctx *h, double bytes)
{
    if (!h) return set_err(nullptr, LBM_EINVAL, "NULL handle");
    if (!(bytes >= 0) || !std::isfinite(bytes)) return set_err(h, LBM_EINVAL, "budget must be finite and >= 0");
    h->adj_budget = bytes;
    return LBM_OK;
}

long lbm_steps_done(const lbm_ctx *h) { return h ? (long)h->t : -1; }

long lbm_num_links(const lbm_ctx *h) { return h ? (long)h->nlinks : -1; }

lbm_status lbm_set_kernel_timing(lbm_ctx *h, int on)
{
    if (!h) return set_err(nullptr, LBM_EINVAL, "NULL handle");
    SETTLE(h);
    h->timing = on != 0;
    return LBM_OK;
}

lbm_status lbm_kernel_times(lbm_ctx *h, double *ms, long *launches, int reset)
{
    if (!h) return set_err(nullptr, LBM_EINVAL, "NULL handle");
    SETTLE(h);
    for (int k = 0; k < 2; ++k) {
        if (ms) ms[k] = h->kt_ms[k];
        if (launches) launches[k] = h->kt_n[k];
    }
    if (reset) {
        h->kt_ms[0] = h->kt_ms[1] = 0;
        h->kt_n[0] = h->kt_n[1] = 0;
    }
    return LBM_OK;
}

long lbm_launch_count(const lbm_ctx *h) { return h ? (long)h->launches : -1; }

const char *lbm_last_error(const lbm_ctx *h)
{
    return h ? h->err.c_str() : g_thread_err.c_str();
}

void lbm_destroy(lbm_ctx *h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    free_all(h);
    delete h;
}

}  // extern "C"
