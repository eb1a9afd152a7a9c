// lbm_internal.cuh -- declarations shared by the library's translation units.
//
// Layout in HBM (all device buffers owned by the handle):
//   populations  three rotating buffers, each 9 planes [ny][pitch] of the storage type
//                (pitch = nx rounded up to 64 elements, so every row starts on a
//                128-byte boundary for FP16 and wider types);
//   nbits        uint16 [ny][pitch]: bit 0 = node is solid, bit i (1..8) =
//                neighbour n + c_i is solid (y periodic, x periodic only for a
//                fully periodic domain);
//   tile_flag    uint8 per collide-stream tile: nonzero when a solid node lies in
//                the tile or its one-node halo (those tiles take the checked
//                bounce-back path);
//   links        int32 [L], n*8 + (i-1), ascending;
//   inlet        [9][ny] storage-type inlet populations feq(rho0, u_in(y));
//   partials     [3][n_cv_tiles][6] (one slice per destination buffer) per-tile J(t) on the pre- and on the
//                post-collision state, and gained-minus-lost(t); FP64 for FP64
//                storage, float-float pairs otherwise (8 bytes either way);
//   link_partials [n_ctas][12] per-CTA rows of the link kernel, same types;
//   series       double [steps][12]: A, B, DRTT, A', momentum defect, SI (x, y each);
//   carry        double [8]: J_post(t-1), GL(t-1), flag;  step counter int64;
//   ticket       uint32 arrival counter of the link kernel's CTAs.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gblbm.h"

namespace gblbm {

// Collide-stream tiles: 128 nodes along x by tile_rows(storage) rows.
constexpr int TILE_X = 128;
constexpr unsigned int WAIT_LIMIT = 1u << 22;  // default bound on every pipeline mbarrier wait
// bound on each wait for copies already in flight after a pipeline wait gave up
constexpr unsigned int DRAIN_LIMIT = 1u << 26;
constexpr int PITCH_ALIGN = 64;
constexpr int LINK_THREADS = 128;
constexpr int LINK_WARPS = LINK_THREADS / 32;  // partial rows a link-kernel CTA writes
// Threads of the batched link kernel's one CTA per domain (a tuning knob):
// enough that a domain's links take one pass.
#ifndef GBLBM_BATCH_LINK_THREADS
#define GBLBM_BATCH_LINK_THREADS 512
#endif
constexpr int BATCH_LINK_THREADS = GBLBM_BATCH_LINK_THREADS;
constexpr int MAX_LINK_CTAS = 148;
constexpr int CV_PARTIAL = 6;
constexpr int LINK_PARTIAL = 14;
constexpr int SERIES_ROW = 12;

// Tile rows of the FP32 and FP16-deviation kernels (tuning knobs).
#ifndef GBLBM_TR_F16
#define GBLBM_TR_F16 4
#endif
#ifndef GBLBM_TR_F32
#define GBLBM_TR_F32 4
#endif
__host__ __device__ constexpr int tile_rows(int storage)
{
    return (storage == LBM_F32 || storage == LBM_F32_DEV) ? GBLBM_TR_F32 : (storage == LBM_F16_DEV ? GBLBM_TR_F16 : 4);
}
// Adjacent columns per thread of the direct-load kernels: FP16 deviations
// take two, so that loads and stores move 4-byte pairs (a tuning knob).
#ifndef GBLBM_COLS_F16
#define GBLBM_COLS_F16 2
#endif
__host__ __device__ constexpr int cols_per_thread(int storage)
{
    return storage == LBM_F16_DEV ? GBLBM_COLS_F16 : 1;
}
// rows per thread of the direct-load kernel (enough loads in flight per thread:
// 4 nodes a thread for FP16 deviations, 2 for FP32, 1 for FP64)
#ifndef GBLBM_RPT_F16
#define GBLBM_RPT_F16 (4 / GBLBM_COLS_F16)
#endif
__host__ __device__ constexpr int direct_rpt(int storage)
{
    return storage == LBM_F64 ? 1 : (storage == LBM_F16_DEV ? GBLBM_RPT_F16 : 2);
}

// ---- D2Q9 (Section II, Table tabD2Q9) as compile-time functions ----
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
}
template <typename T>
__host__ __device__ constexpr T wgt(int i) {
    return i == 0 ? T(4) / T(9) : (i <= 4 ? T(1) / T(9) : T(1) / T(36));
}

// ---- storage traits ----
template <int S> struct Traits;
template <> struct Traits<LBM_F64> {
    using store_t = double;
    using comp_t = double;
    static constexpr bool dev = false;
};
template <> struct Traits<LBM_F32> {
    using store_t = float;
    using comp_t = float;
    static constexpr bool dev = false;
};
template <> struct Traits<LBM_F32_DEV> {
    using store_t = float;
    using comp_t = float;
    static constexpr bool dev = true;
};
template <> struct Traits<LBM_F16_DEV> {
    using store_t = __half;
    using comp_t = float;
    static constexpr bool dev = true;
};

__device__ __forceinline__ float to_comp(float v) { return v; }
__device__ __forceinline__ double to_comp(double v) { return v; }
__device__ __forceinline__ float to_comp(__half v) { return __half2float(v); }
template <typename ST> __device__ __forceinline__ ST to_store(float v);
template <> __device__ __forceinline__ float to_store<float>(float v) { return v; }
template <> __device__ __forceinline__ __half to_store<__half>(float v) { return __float2half_rn(v); }
template <typename ST> __device__ __forceinline__ ST to_store(double v);
template <> __device__ __forceinline__ double to_store<double>(double v) { return v; }

// ---- kernel arguments ----
struct StepArgs {
    const void *src;         // populations at t-1 (post-collision) or t (pre-collision)
    void *dst;               // post-collision populations at t
    const uint16_t *nbits;
    const uint8_t *tile_flag;
    const void *inlet;       // [9][ny]
    double *partials;        // [n_cv_tiles][CV_PARTIAL]
    int *status;             // [0] flags, [1] first bad step
    const long long *step_ctr;
    long long plane;         // elements per plane = ny * pitch
    int nx, ny, pitch;
    int periodic;
    int precollision;        // src holds f(t) (no pull this step)
    int tiles_x;             // tiles per row band
    int tile_off_x, tile_off_y;  // added to blockIdx (momentum-only pass)
    double omega, rho0, gx, gy;
    float omega_f, rho0_f, gx_f, gy_f;  // the same in FP32 (no FP64 conversions in FP32 kernels)
    int cv[4];               // inclusive control-volume box
    int cvt[4];              // inclusive tile rectangle holding the box and its halo
    int use_bulk;            // staged (TMA) kernel allowed (channel set-up, pulled state)
    int sm_count;            // persistent grid size of the staged kernel
    int pf_rows;             // L2 prefetch distance of the direct kernel in tile rows (0: off)
    int first_r0, first_r1;  // tile rows with bounce-back tiles, dispatched first (r0 > r1: none)
    unsigned int wait_limit; // polls of each pipeline wait of the staged kernel (WAIT_LIMIT)
};

// The relaxation rate of a StepArgs: the FP64 value and its FP32 rounding (a
// kernel reads only the one its storage computes with).
__host__ __device__ inline void set_relaxation_f64(StepArgs &a, double omega) { a.omega = omega; }
__host__ __device__ inline void set_relaxation_f32(StepArgs &a, float omega) { a.omega_f = omega; }
__host__ inline void set_relaxation(StepArgs &a, double omega)
{
    set_relaxation_f64(a, omega);
    set_relaxation_f32(a, (float)omega);
}

struct LinkArgs {
    const void *src, *dst;
    const uint16_t *nbits;
    const int32_t *links;
    long long nlinks;
    const double *partials;
    int n_partials;
    double *link_partials;   // [n_ctas][LINK_PARTIAL]
    unsigned int *ticket;
    int n_ctas;
    double *series;
    long long series_rows;   // rows the series holds; a row beyond sets status bit 4
    int *status;             // [0]: error bits, as in StepArgs
    double *carry;           // J_post(t-1)[2], GL(t-1)[2], have_prev
    long long *step_ctr;
    long long plane;
    int nx, ny, pitch, periodic, precollision;
    int record_series;
    int drtt_only;           // finalise DRTT(T-1) from a momentum-only pass
    double rho0;
    double visc;             // 1 - omega/2: deviatoric stress = -visc * non-equilibrium second moment
    float visc_f;
    double link_base[2];     // deviation storage: 2 rho0 sum_links c_i w_i
    double flux_base[2];     // deviation storage: rho0 (sum_in - sum_out) c_i w_i
};

// Message returned by lbm_last_error(NULL) on the calling thread.
void set_thread_error(const char *msg);

// ---- launchers (defined in the .cu files) ----
cudaError_t launch_naca_mask(uint8_t *mask, int nx, int ny, double chord, double thickness,
                             double ca, double sa, double xc, double yc, int closed_te,
                             cudaStream_t st);
cudaError_t launch_cylinder_mask(uint8_t *mask, int nx, int ny, double xc, double yc, double radius,
                                 cudaStream_t st);
cudaError_t launch_node_bits(const uint8_t *mask, uint16_t *nbits, int nx, int ny, int pitch,
                             int periodic, cudaStream_t st);
cudaError_t launch_link_count(const uint16_t *nbits, int nx, int ny, int pitch, int *block_cnt,
                              int nblocks, cudaStream_t st);
cudaError_t launch_scan_blocks(int *block_cnt, int nblocks, long long *total, cudaStream_t st);
cudaError_t launch_link_scatter(const uint16_t *nbits, int nx, int ny, int pitch,
                                const int *block_off, int32_t *links, long long cap,
                                cudaStream_t st);
// tw x rows tiles (tw <= 1024)
cudaError_t launch_tile_flags(const uint16_t *nbits, int nx, int ny, int pitch, int periodic,
                              uint8_t *flags, int tiles_x, int tiles_y, int tw, int rows,
                              cudaStream_t st);
int link_blocks(int nx, int ny);

// uniform: every row has the same inlet velocity (one row is searched and copied)
cudaError_t launch_init(int storage, void *pop, long long plane, const uint8_t *mask, int nx,
                        int ny, int pitch, const double *u_row, double rho0, void *inlet,
                        cudaStream_t st, int uniform = 0);
// tmap: the tensor map over the source buffer (staged kernel), or NULL
cudaError_t launch_collide_stream(int storage, const StepArgs &a, int tiles_x, int tiles_y,
                                  bool momentum_only, const void *tmap, cudaStream_t st);
size_t tma_stage_bytes(int storage);
// L2 prefetch distance (StepArgs::pf_rows) of the direct kernel for a storage
// type on a device with sm_count SMs and tiles_x tiles per row; 0 where
// prefetching is off.
int collide_stream_prefetch_rows(int storage, int sm_count, int tiles_x);
// priority: the launch's scheduling priority (0: the stream's own; lower
// numbers are served first)
cudaError_t launch_link_force(int storage, const LinkArgs &a, cudaStream_t st, int priority = 0);
cudaError_t launch_gather(int storage, const void *pop, const uint16_t *nbits, const void *inlet,
                          long long plane, int nx, int ny, int pitch, int periodic,
                          int precollision, double rho0, int plane_i, double *out,
                          cudaStream_t st);
cudaError_t launch_boundary_nodes(const int32_t *links, long long nlinks, int32_t *nodes, long long *count,
                                  cudaStream_t st);
cudaError_t launch_surface_pressure(int storage, const void *pop, const uint16_t *nbits, const int32_t *nodes,
                                    long long count, long long plane, int nx, int ny, int pitch, int periodic,
                                    int precollision, double rho0, double p_inf, double q, double *cp,
                                    cudaStream_t st);
// Drag and lift coefficients of a window of a force series (lbm_coeff.cu):
// out[0..3] = mean C_d, mean C_l, std C_d, std C_l; with per_step, C_d and C_l
// of every step follow ([count] each).  norm = 2 / (rho0 U^2 L).
cudaError_t launch_coefficients(const double *series, long long row_stride, int col, long long first,
                                long long count, int wrap, double norm, double *out, bool per_step,
                                cudaStream_t st);
cudaError_t launch_scatter_pop(int storage, void *pop, const uint16_t *nbits, long long plane,
                               int nx, int ny, int pitch, double rho0, int plane_i,
                               const double *in, cudaStream_t st);

// discrete adjoint (lbm_adjoint.cu): one backward step; src holds ft(t-1) in
// the storage type (f(t) itself when precollision), pulled inside the kernel
int adjoint_blocks(int nx, int ny);
// tile_flag: the collide-stream tile flags (tiles of TILE_X x flag_rows nodes,
// flag_tiles_x a row), used when they match the backward step's tiles
cudaError_t launch_adjoint_step(int storage, const void *src, int precollision, const void *lam_next, void *lam,
                                const uint16_t *nbits, const uint8_t *tile_flag, int flag_rows, int flag_tiles_x,
                                const double *u_row, double *du_acc,
                                double *dw_acc, long long plane, int nx, int ny, int pitch,
                                int in_window, double omega, double rho0, double obj_x,
                                double obj_y, cudaStream_t st);
// sum of n slots in a fixed order: FP64 values, or float-float pairs (ff_slots)
cudaError_t launch_sum_fixed(const double *v, long long n, double *out, bool ff_slots, cudaStream_t st);
// lambda (compute type, [9][ny][pitch]) -> dJ/df0 in FP64 [9][ny][nx] in device
// memory, zero on solid nodes (mask) and in the inlet column
cudaError_t launch_adjoint_df0(int storage, const void *lam, const uint8_t *mask, long long plane, int nx, int ny,
                               int pitch, int sm_count, double *out, cudaStream_t st);

}  // namespace gblbm
