// lbm_batch.cu -- the batched collide-stream kernel: one launch advances every
// domain of a batch by one step (Section II, Eq. CollideAdv in pull form, with
// halfway bounce-back, the channel's inlet and outlet columns and the DRTT box
// sums of Eq. rtt7), with exactly the per-node arithmetic of the single-domain
// kernel (collide_tile).
//
// The grid is persistent (a multiple of the SM count, chosen by the host's
// tuner) or one CTA per tile; each CTA walks the launch's tiles with a stride
// of the grid size.  Per tile it finds the tile's domain in the kernel
// parameter block (the tile table names it) and runs the tile.
#include "lbm_batch.cuh"
#include "lbm_collide.cuh"

namespace gblbm {

// Minimum resident CTAs per SM asked of the compiler for the one-CTA-per-tile
// form (0: no bound), per storage: 8 x 128 threads (64 registers) for FP32
// and for FP16 deviations (both measured best).  The persistent form carries no bound: its tile loop
// keeps the domain arguments live across tiles and needs about 128 registers
// a thread.
#ifndef GBLBM_BATCH_MINB_F64
#define GBLBM_BATCH_MINB_F64 0
#endif
#ifndef GBLBM_BATCH_MINB_F32
#define GBLBM_BATCH_MINB_F32 8
#endif
#ifndef GBLBM_BATCH_MINB_F16
#define GBLBM_BATCH_MINB_F16 8
#endif
template <int S> struct BatchMinBlocks {
    static constexpr int value = S == LBM_F64       ? GBLBM_BATCH_MINB_F64
                                 : S == LBM_F16_DEV ? GBLBM_BATCH_MINB_F16
                                                    : GBLBM_BATCH_MINB_F32;
};

// Tile k of the launch: its domain's arguments, its place in the domain, and
// the single-domain tile body.
template <int S, bool MOMENTUM_ONLY, int TX, int TR, int RPT>
__device__ __forceinline__ void batch_tile(const BatchParams &p, int k)
{
    static_assert(TR % RPT == 0, "rows per thread must divide the tile rows");
    const long long elem = (long long)sizeof(typename Traits<S>::store_t);
    {
        // the tile's entry: domain (within the launch), tile column, tile row, checked
        const int4 e = __ldg(p.tiles + k);
        const int d = e.x;
        const BatchDomain &m = p.dom[d];
        StepArgs a;
        a.src = p.src + (long long)m.pop_off64 * 64 * elem;
        a.dst = p.dst + (long long)m.pop_off64 * 64 * elem;
        a.nbits = p.nbits + (long long)m.node_off64 * 64;
        a.tile_flag = nullptr;
        a.inlet = p.inlet + (long long)m.inlet_off64 * 64 * elem;
        a.partials = p.partials + (long long)CV_PARTIAL * m.part_off;
        a.status = p.status + 2 * (p.dom_base + d);
        a.step_ctr = p.step_ctr;
        const int pitch = (m.nx + PITCH_ALIGN - 1) / PITCH_ALIGN * PITCH_ALIGN;
        a.plane = (long long)m.ny * pitch;
        a.nx = m.nx;
        a.ny = m.ny;
        a.pitch = pitch;
        a.periodic = p.periodic;
        a.precollision = p.precollision;
        a.tiles_x = m.tiles_x;
        a.tile_off_x = a.tile_off_y = 0;
        a.pf_rows = 0;
        a.first_r0 = 1;
        a.first_r1 = 0;
        if constexpr (S == LBM_F64)
            set_relaxation_f64(a, m.omega);
        else
            set_relaxation_f32(a, m.omega_f);
        a.rho0 = p.rho0;
        a.gx = a.gy = 0.0;
        a.rho0_f = p.rho0_f;
        a.gx_f = a.gy_f = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            a.cv[j] = m.cv[j];
            a.cvt[j] = m.cvt[j];
        }
        a.use_bulk = 0;
        a.sm_count = 0;
        collide_tile<S, MOMENTUM_ONLY, false, TX, TR, RPT>(a, e.y, e.z, p.precollision || e.w != 0);
    }
}

// PERSIST: a grid of a few CTAs per SM walks the tiles with a stride of the
// grid; otherwise one CTA per tile.
template <int S, bool MOMENTUM_ONLY, bool PERSIST, int TX, int TR, int RPT>
__global__ void __launch_bounds__((TX / cols_per_thread(S)) * (TR / RPT), PERSIST ? 0 : BatchMinBlocks<S>::value)
    k_collide_stream_batch(const __grid_constant__ BatchParams p)
{
    if (PERSIST) {
        for (int k = blockIdx.x; k < p.n_tiles; k += gridDim.x) batch_tile<S, MOMENTUM_ONLY, TX, TR, RPT>(p, k);
    } else if ((int)blockIdx.x < p.n_tiles) {
        batch_tile<S, MOMENTUM_ONLY, TX, TR, RPT>(p, blockIdx.x);
    }
}

template <int S, bool MOM, bool PERSIST, int SHAPE>
struct BatchKernel {
    static constexpr int TX = batch_tx(SHAPE), TR = batch_tr(S, SHAPE), RPT = batch_rpt(S);
    static void *fn() { return (void *)k_collide_stream_batch<S, MOM, PERSIST, TX, TR, RPT>; }
    static cudaError_t launch(const BatchParams &p, int grid, cudaStream_t st)
    {
        k_collide_stream_batch<S, MOM, PERSIST, TX, TR, RPT><<<grid, dim3(TX / cols_per_thread(S), TR / RPT), 0, st>>>(p);
        return cudaGetLastError();
    }
};

template <int S, bool MOM, bool PERSIST>
cudaError_t launch_shape(int shape, const BatchParams &p, int grid, cudaStream_t st)
{
    switch (shape) {
    case 0: return BatchKernel<S, MOM, PERSIST, 0>::launch(p, grid, st);
    case 1: return BatchKernel<S, MOM, PERSIST, 1>::launch(p, grid, st);
    default: return BatchKernel<S, MOM, PERSIST, 2>::launch(p, grid, st);
    }
}

// The momentum-only pass always runs one CTA per tile.
template <int S>
cudaError_t launch_storage(int shape, bool mom, bool persist, const BatchParams &p, int grid, cudaStream_t st)
{
    if (mom) return launch_shape<S, true, false>(shape, p, p.n_tiles, st);
    return persist ? launch_shape<S, false, true>(shape, p, grid, st)
                   : launch_shape<S, false, false>(shape, p, p.n_tiles, st);
}

cudaError_t launch_collide_stream_batch(int storage, int shape, bool momentum_only, const BatchParams &p,
                                        int grid, cudaStream_t st)
{
    if (shape < 0 || shape >= BATCH_SHAPES) return cudaErrorInvalidValue;
    if (p.n_tiles == 0) return cudaSuccess;
    const bool persist = grid > 0;
    switch (storage) {
    case LBM_F64: return launch_storage<LBM_F64>(shape, momentum_only, persist, p, grid, st);
    case LBM_F32: return launch_storage<LBM_F32>(shape, momentum_only, persist, p, grid, st);
    case LBM_F32_DEV: return launch_storage<LBM_F32_DEV>(shape, momentum_only, persist, p, grid, st);
    default: return launch_storage<LBM_F16_DEV>(shape, momentum_only, persist, p, grid, st);
    }
}

template <int S>
void *kernel_of(int shape)
{
    switch (shape) {
    case 0: return BatchKernel<S, false, true, 0>::fn();
    case 1: return BatchKernel<S, false, true, 1>::fn();
    default: return BatchKernel<S, false, true, 2>::fn();
    }
}

int batch_max_ctas_per_sm(int storage, int shape)
{
    void *fn;
    switch (storage) {
    case LBM_F64: fn = kernel_of<LBM_F64>(shape); break;
    case LBM_F32: fn = kernel_of<LBM_F32>(shape); break;
    case LBM_F32_DEV: fn = kernel_of<LBM_F32_DEV>(shape); break;
    default: fn = kernel_of<LBM_F16_DEV>(shape); break;
    }
    const int threads = (batch_tx(shape) / cols_per_thread(storage)) * (batch_tr(storage, shape) / batch_rpt(storage));
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, 0) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace gblbm
