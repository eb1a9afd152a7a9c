// lbm_batch.cuh -- declarations of the batched kernels: many independent
// domains (each its own grid, body, relaxation time, inlet and control volume)
// advanced by one collide-stream launch and one link launch per step.
//
// Every domain keeps the single-domain layout ([9][ny][pitch] planes of the
// storage type) at its own offset in two shared population arenas.  The
// collide-stream kernel walks a table of the tiles of all domains of a launch,
// domain by domain; a tile's entry names its domain, whose arguments come from
// the kernel parameter (block-uniform reads of the constant bank).  The link kernel runs
// one CTA per domain.
#pragma once

#include "lbm_internal.cuh"

namespace gblbm {

// Tile shapes the batched collide-stream kernel is compiled for: TX nodes
// along x by TR rows, RPT rows per thread, TX * TR / RPT threads.  All shapes
// hold the same number of nodes; narrower tiles waste less at ragged domain
// edges, wider ones make longer coalesced rows.
#ifndef GBLBM_BATCH_RPT_F32
#define GBLBM_BATCH_RPT_F32 2
#endif
#ifndef GBLBM_BATCH_TRDIV
#define GBLBM_BATCH_TRDIV 1
#endif
constexpr int BATCH_SHAPES = 3;
__host__ __device__ constexpr int batch_tx(int shape) { return shape == 0 ? 128 : (shape == 1 ? 64 : 32); }
// Rows of the 128-wide shape: 2 for FP32 (256-node tiles of 128 threads), 4
// for FP16 deviations (512-node tiles of 128 threads), 4 for FP64.  Small CTAs,
// eight to an SM, overlap more tiles' dependent starts (tile entry, domain
// arguments, populations) than the 1024-node tiles did.
#ifndef GBLBM_BATCH_ROWS_F16
#define GBLBM_BATCH_ROWS_F16 4
#endif
#ifndef GBLBM_BATCH_ROWS_F32
#define GBLBM_BATCH_ROWS_F32 2
#endif
__host__ __device__ constexpr int batch_tr(int storage, int shape)
{
    return (storage == LBM_F16_DEV ? GBLBM_BATCH_ROWS_F16 : (storage == LBM_F64 ? 4 : GBLBM_BATCH_ROWS_F32)) *
           (128 / batch_tx(shape)) / ((storage == LBM_F32 || storage == LBM_F32_DEV) ? GBLBM_BATCH_TRDIV : 1);
}
__host__ __device__ constexpr int batch_rpt(int storage)
{
    return (storage == LBM_F32 || storage == LBM_F32_DEV) ? GBLBM_BATCH_RPT_F32 : direct_rpt(storage);
}

// Per-domain arguments of the batched collide-stream kernel, compact enough
// that MAX_BATCH_DOMAINS of them fit in one kernel parameter block (read from
// the constant bank with a block-uniform index).  Offsets are in units of 64
// elements where the layout guarantees that alignment.
struct BatchDomain {
    union {
        double omega;   // 1/tau (FP64 storage)
        float omega_f;  // 1/tau rounded to FP32 (the other storages: no FP64 conversion per tile)
    };
    int pop_off64;    // population arena offset / 64 (elements)
    int node_off64;   // neighbour-bit arena offset / 64
    int inlet_off64;  // inlet arena offset / 64 (elements)
    int part_off;     // first partial row of the domain (this tile shape)
    int nx, ny;       // grid (nx, ny <= 32767); the pitch is nx rounded up to 64
    int tiles_x;      // tiles per row (this tile shape)
    short cv[4];      // control volume, inclusive
    short cvt[4];     // its tile rectangle (this tile shape)
};
static_assert(sizeof(BatchDomain) == 56, "compact per-domain arguments");
constexpr int MAX_BATCH_SIDE = 32767;

constexpr int MAX_BATCH_DOMAINS = 512;

// The kernel parameter of one batched collide-stream launch (under the
// 32 KB parameter limit): a chunk of at most MAX_BATCH_DOMAINS domains whose
// tiles are numbered domain by domain, row by row.
struct BatchParams {
    const char *src;         // population arena read this step
    char *dst;               // population arena written this step
    const uint16_t *nbits;   // neighbour-bit arena
    const char *inlet;       // inlet arena
    double *partials;        // control-volume partial rows
    int *status;             // [domain][2] of the whole batch
    const long long *step_ctr;
    const int4 *tiles;       // per tile of the launch: {domain within the launch, tx, ty,
                             // 1 = bounce-back-aware path}
    int n_dom;               // domains in this chunk
    int dom_base;            // index of the chunk's first domain in the batch (status rows)
    int n_tiles;             // tiles of this launch
    int periodic;
    int precollision;        // the state is pre-collision (first step)
    int cv_only;             // momentum-only pass over the control-volume tiles
    double rho0;
    float rho0_f;
    BatchDomain dom[MAX_BATCH_DOMAINS];
};
static_assert(sizeof(BatchParams) <= 32000, "kernel parameter block above the 32 KB limit");

struct BatchLinkArgs {
    const LinkArgs *args;     // [n_domains]: this step's link arguments of every domain
    double *series;           // [rows][n_domains][SERIES_ROW]
    long long series_rows;
    int n_domains;
    int keep_all;             // all rows, or the last two (slot = step parity)
    int drtt_only;            // finish DRTT(T-1) only (after a momentum-only pass)
    long long *step_ctr;      // steps done (shared by all domains)
    unsigned int *ticket;     // arrival counter of the CTAs
    int *status;              // [0]: bit 4 = a series row fell outside the buffer
};

// grid > 0: the persistent form with that many CTAs; grid = 0: one CTA per
// tile (the momentum-only pass always takes this form).
cudaError_t launch_collide_stream_batch(int storage, int shape, bool momentum_only,
                                        const BatchParams &p, int grid, cudaStream_t st);
// Resident CTAs per SM of the persistent batched kernel for (storage, shape), or 0.
int batch_max_ctas_per_sm(int storage, int shape);
cudaError_t launch_link_force_batch(int storage, const BatchLinkArgs &b, cudaStream_t st);

}  // namespace gblbm
