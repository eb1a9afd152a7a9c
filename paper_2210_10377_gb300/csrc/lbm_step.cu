// lbm_step.cu -- the collide-stream kernels, one pass over the grid per time
// step t -> t+1 (Section II, Eq. CollideAdv, written in pull form).
//
// Each fluid node gathers f_i(x, t) = ft_i(x - c_i, t-1), or the bounced
// ft_opp(i)(x, t-1) when x - c_i is solid (halfway bounce-back), takes rho and
// u, relaxes towards feq (second-order equilibrium, theta0 = 1/3) and stores
// ft(x, t).  The channel inlet column stores feq(rho0, u_in(y)); the outlet
// column collides the populations of column nx-2 (zero-gradient copy).  Tiles
// that cover the DRTT control volume also reduce J(t) (Eq. rtt1) and the
// gained-minus-lost flux of ft(t) through the box surface (Eq. rtt7), in a
// fixed order (no floating-point atomics).
//
// Two kernels do the same per-node arithmetic: k_collide_stream loads its
// tile's neighbourhood directly from global memory; k_collide_stream_tma
// (persistent, optional) stages each tile with 3-D tensor-map bulk copies.
#include "lbm_collide.cuh"

namespace gblbm {

// Minimum resident CTAs per SM asked of the compiler for the direct kernel
// (0: no bound); tuning knobs.  FP32 and FP16 storage are occupancy-bound:
// 4 CTAs of 256 threads (FP32) and 8 of 128 (FP16), 64 registers each, run
// them faster than fewer CTAs without spills.
#ifndef GBLBM_DIRECT_MINB_F16
#define GBLBM_DIRECT_MINB_F16 8
#endif
#ifndef GBLBM_DIRECT_MINB_F32
#define GBLBM_DIRECT_MINB_F32 4
#endif
template <int S> struct DirectMinBlocks {
    static constexpr int value = 0;
};
template <> struct DirectMinBlocks<LBM_F32> {
    static constexpr int value = GBLBM_DIRECT_MINB_F32;
};
template <> struct DirectMinBlocks<LBM_F32_DEV> {
    static constexpr int value = GBLBM_DIRECT_MINB_F32;
};
template <> struct DirectMinBlocks<LBM_F16_DEV> {
    static constexpr int value = GBLBM_DIRECT_MINB_F16;
};

// L2 prefetch distance of the direct kernel, in percent of the CTAs that the
// GPU holds at once (0: off); a tuning knob.
#ifndef GBLBM_PF_PERCENT
#define GBLBM_PF_PERCENT 50
#endif

// Asks L2 for the source rows of the tile a.pf_rows tile rows further down
// the same tile column: in the launch's dispatch order (blockIdx.x fastest)
// that tile runs about pf_rows * tiles_x CTAs later, and its CTA then finds
// its lines in L2, so HBM requests no longer wait for a warp's load phase.
// One bulk prefetch per plane and row of that tile, issued by the first 9 TR
// threads.  Each copy lies inside the source buffer (row < ny, columns x0 ..
// min(x0 + 128, pitch) - 1) and starts on a 16-byte boundary (pitch is a
// multiple of 64 elements); the halo rows and columns are the neighbouring
// tiles' own rows.  A prefetch changes no value.
// Tile row of the CTA row `by` of a full-grid launch.  Tiles that take the
// slower paths run first instead of forming the launch's tail: the rows
// [r0, r1] that hold bounce-back tiles (next to a body; several times an
// interior tile's time), then the last and the first tile row, which wrap in
// y and take the general path, then the other rows in order.  The mapping is
// arithmetic, so the L2 prefetch of the tile pf_rows CTA rows ahead finds its
// target without a load (a tuning knob: 0 keeps blockIdx order).
#ifndef GBLBM_WRAP_ROWS_FIRST
#define GBLBM_WRAP_ROWS_FIRST 1
#endif
__device__ __forceinline__ int tile_row_of(int by, int tiles_y, int r0, int r1)
{
    if (!GBLBM_WRAP_ROWS_FIRST || tiles_y < 3) return by;
    // the body's rows strictly inside (the wrap rows come next in any case)
    const int b0 = r0 < 1 ? 1 : r0, b1 = r1 > tiles_y - 2 ? tiles_y - 2 : r1;
    const int nb = b1 >= b0 ? b1 - b0 + 1 : 0;
    if (by < nb) return b0 + by;
    if (by == nb) return tiles_y - 1;
    if (by == nb + 1) return 0;
    const int k = by - nb - 2;  // among the rows 1 .. tiles_y - 2 outside [b0, b1], in order
    return (nb == 0 || 1 + k < b0) ? 1 + k : 1 + k + nb;
}

template <int S>
__device__ __forceinline__ void prefetch_ahead(const StepArgs &a)
{
    using E = typename Traits<S>::store_t;
    constexpr int TR = tile_rows(S);
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int by = (int)blockIdx.y + a.pf_rows;
    if (a.pf_rows <= 0 || t >= 9 * TR || by >= (int)gridDim.y) return;
    const int ty = tile_row_of(by, (int)gridDim.y, a.first_r0, a.first_r1);
    const int y = ty * TR + t % TR;
    if (y >= a.ny) return;
    const int x0 = (int)blockIdx.x * TILE_X;
    const int ncol = min(TILE_X, a.pitch - x0);
    prefetch_l2((const E *)a.src + (long long)(t / TR) * a.plane + (long long)y * a.pitch + x0,
                (unsigned)(ncol * sizeof(E)));
}

// Direct-load collide-stream kernel: one CTA of 128 x (TR/RPT) threads per
// 128 x TR tile; tiles without solids away from the domain's edges take the
// interior path (collide_tile).
template <int S, bool MOMENTUM_ONLY, bool FORCE>
__global__ void __launch_bounds__((TILE_X / cols_per_thread(S)) * (tile_rows(S) / direct_rpt(S)),
                                  DirectMinBlocks<S>::value)
    k_collide_stream(StepArgs a)
{
    if constexpr (!MOMENTUM_ONLY) prefetch_ahead<S>(a);
    // a launch over a sub-rectangle of tiles (the momentum-only pass) keeps plain order
    const int tx = blockIdx.x + a.tile_off_x;
    const int ty = (MOMENTUM_ONLY || a.tile_off_y != 0) ? (int)blockIdx.y + a.tile_off_y
                                                        : tile_row_of((int)blockIdx.y, (int)gridDim.y,
                                                                      a.first_r0, a.first_r1);
    const bool checked = a.precollision || a.tile_flag[(long long)ty * a.tiles_x + tx] != 0;
    collide_tile<S, MOMENTUM_ONLY, FORCE, TILE_X, tile_rows(S), direct_rpt(S)>(a, tx, ty, checked);
}

// ---------------------------------------------------------------------------
// Staged collide-stream kernel (channel set-up, pulled state): persistent CTAs,
// one per SM, walk the 128 x TR tiles round-robin.  For each tile one TMA copy
// (cp.async.bulk.tensor.3d through a tensor map over [9 planes][ny][pitch])
// brings rows y0-1 .. y0+TR of all nine source planes, columns x0-PAD ..
// x0+127+PAD (PAD = 16 bytes of elements, so every copy starts on a 16-byte
// boundary), into shared memory; plane i of node row r is box row r+1-c_iy.
// Rows outside [0, ny) are zero-filled by the copy; on the first and last tile
// rows the threads read those wrapped rows from global memory instead.
// NS tiles are in flight per CTA while its threads collide the current tile
// out of shared memory and store ft(t) with vector stores.  Every mbarrier
// wait is bounded: on expiry the kernel flags status bit 2 (LBM_ETIMEOUT),
// waits boundedly for its copies and returns.
// ---------------------------------------------------------------------------
namespace tma {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait; false when the limit expired.
// At most `limit` polls; false if the phase did not complete within them.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t k = 0; k < limit; ++k)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                        uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

}  // namespace tma

// Shared memory budget (KB) for the staged kernel's stages and the number of
// its CTAs per SM; tuning knobs (two CTAs per SM hide each other's barriers).
#ifndef GBLBM_TMA_SMEM_KB
#define GBLBM_TMA_SMEM_KB 105
#endif
#ifndef GBLBM_TMA_MINB
#define GBLBM_TMA_MINB 2
#endif

template <int S> struct TmaCfg {
    using ST = typename Traits<S>::store_t;
    static constexpr int TR = tile_rows(S);
    static constexpr int BR = TR + 2;                  // box rows: y0-1 .. y0+TR
    static constexpr int PAD = 16 / (int)sizeof(ST);
    static constexpr int SEG = TILE_X + 2 * PAD;       // box columns
    static constexpr int VX = (S == LBM_F64) ? 1 : 2;  // adjacent nodes per thread along x
    static constexpr int XT = TILE_X / VX;
    static constexpr int THREADS = XT * TR;            // one tile row per thread
    static constexpr uint32_t BOX_BYTES = 9u * BR * SEG * (uint32_t)sizeof(ST);
    static constexpr uint32_t STAGE_BYTES = (BOX_BYTES + 127u) & ~127u;
    static constexpr int NS_FIT = (GBLBM_TMA_SMEM_KB * 1024) / STAGE_BYTES;
    static constexpr int NS = NS_FIT < 2 ? 2 : (NS_FIT > 8 ? 8 : NS_FIT);
    static constexpr size_t SMEM = (size_t)NS * STAGE_BYTES + 128 + 8 * NS;
    static_assert(NS >= 2, "at least two stages");
    static_assert(SEG * sizeof(ST) % 16 == 0, "box rows are whole 16-byte units");
    static_assert(THREADS <= 1024, "one tile row per thread");
};

template <int S, bool CHECKED, bool FULL, bool EDGE, bool FORCE>
__device__ __forceinline__ void tma_tile(const StepArgs &a, const typename Traits<S>::store_t *sm,
                                         int tx, int ty, bool cvtile,
                                         typename AccOf<S>::type (&acc)[6], bool &bad)
{
    using C = TmaCfg<S>;
    using ST = typename Traits<S>::store_t;
    using T = typename Traits<S>::comp_t;
    const ST *__restrict__ src = (const ST *)a.src;
    ST *__restrict__ dst = (ST *)a.dst;
    const int t = threadIdx.x;
    const int xl = (t % C::XT) * C::VX;
    const int r = t / C::XT;
    const int x0 = tx * TILE_X, y0 = ty * C::TR;
    const int y = y0 + r;
    if (!FULL && y >= a.ny) return;
    T ft[C::VX][9];
    bool store[C::VX];
#pragma unroll
    for (int v = 0; v < C::VX; ++v) {
        const int x = x0 + xl + v;
        store[v] = FULL || x < a.nx;
        if (!store[v]) continue;
        const long long idx = (long long)y * a.pitch + x;
        const uint16_t nb = CHECKED ? a.nbits[idx] : (uint16_t)0;
        if (nb & 1) {  // solid nodes are not updated
            store[v] = false;
            continue;
        }
        T f[9];
        if (x == 0) {  // equilibrium inlet
            const ST *in = (const ST *)a.inlet;
#pragma unroll
            for (int i = 0; i < 9; ++i) ft[v][i] = to_comp(in[i * a.ny + y]);
        } else {
            // the outlet column x = nx-1 takes the populations of column nx-2
            const int xs = x == a.nx - 1 ? x - 1 : x;
            const uint16_t nbs = CHECKED ? (xs == x ? nb : a.nbits[idx - 1]) : (uint16_t)0;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int sy = y - cy(i);
                if (CHECKED && (nbs & (1u << opp(i)))) {
                    f[i] = to_comp(src[opp(i) * a.plane + (long long)y * a.pitch + xs]);
                } else if (EDGE && (sy < 0 || sy >= a.ny)) {
                    const int wy = sy < 0 ? sy + a.ny : sy - a.ny;
                    f[i] = to_comp(src[i * a.plane + (long long)wy * a.pitch + xs - cx(i)]);
                } else {
                    f[i] = to_comp(sm[(i * C::BR + r + 1 - cy(i)) * C::SEG + (xs - x0) + C::PAD - cx(i)]);
                }
            }
            ST out[9];
            collide_node<S, FORCE>(a, f, out, bad);
#pragma unroll
            for (int i = 0; i < 9; ++i) ft[v][i] = to_comp(out[i]);
        }
        if (cvtile) cv_node<S, false, FORCE>(a, x, y, f, ft[v], nb, acc);
    }
    const long long idx0 = (long long)y * a.pitch + x0 + xl;
    if (C::VX == 2 && !CHECKED && store[0] && store[C::VX - 1]) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            if constexpr (S == LBM_F16_DEV) {
                *(__half2 *)&dst[i * a.plane + idx0] =
                    __halves2half2(to_store<ST>(ft[0][i]), to_store<ST>(ft[C::VX - 1][i]));
            } else if constexpr (S != LBM_F64) {
                *(float2 *)&dst[i * a.plane + idx0] = make_float2(ft[0][i], ft[C::VX - 1][i]);
            }
        }
    } else {
#pragma unroll
        for (int v = 0; v < C::VX; ++v)
            if (store[v])
#pragma unroll
                for (int i = 0; i < 9; ++i) dst[i * a.plane + idx0 + v] = to_store<ST>(ft[v][i]);
    }
}

template <int S, bool FORCE>
__global__ void __launch_bounds__(TmaCfg<S>::THREADS, GBLBM_TMA_MINB)
    k_collide_stream_tma(const StepArgs a, int ntiles, const __grid_constant__ CUtensorMap map)
{
    using C = TmaCfg<S>;
    using ST = typename Traits<S>::store_t;
    using A = typename AccOf<S>::type;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    uint64_t *bar = (uint64_t *)(smem + (size_t)C::NS * C::STAGE_BYTES);
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::NS; ++s) tma::mbar_init(&bar[s], 1);
        tma::fence_barrier_init();
    }
    __syncthreads();
    const int count = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    auto issue = [&](int k, int s) {
        const int tile = blockIdx.x + k * gridDim.x;
        const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
        tma::mbar_expect_tx(&bar[s], C::BOX_BYTES);
        tma::load_3d(smem + (size_t)s * C::STAGE_BYTES, &map, tx * TILE_X - C::PAD, ty * C::TR - 1, 0,
                     &bar[s]);
    };
    if (threadIdx.x == 0)
        for (int k = 0; k < C::NS && k < count; ++k) issue(k, k);
    for (int k = 0; k < count; ++k) {
        const int s = k % C::NS;
        const uint32_t parity = (uint32_t)(k / C::NS) & 1u;
        // one thread waits (bounded) for the stage; the barrier hands the data
        // and the outcome to the whole CTA, so every thread takes the same path
        bool ok = true;
        if (threadIdx.x == 0) ok = tma::mbar_wait(&bar[s], parity, a.wait_limit);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                atomicOr(a.status, 2);
                // The copies issued so far fill the stages of tiles k .. k+NS-1,
                // stage k's (whose wait just gave up) included.  Wait for every one
                // of them, each within its own generous bound, so that no bulk copy
                // is still writing this CTA's shared memory when the CTA exits.
                for (int j = k; j < count && j < k + C::NS; ++j)
                    tma::mbar_wait(&bar[j % C::NS], (uint32_t)(j / C::NS) & 1u, DRAIN_LIMIT);
            }
            return;
        }
        const int tile = blockIdx.x + k * gridDim.x;
        const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
        const bool checked = a.tile_flag[tile] != 0;
        const bool full = (tx + 1) * TILE_X <= a.nx && (ty + 1) * C::TR <= a.ny;
        const bool edge = ty == 0 || (ty + 1) * C::TR >= a.ny;
        const bool cvtile = tx >= a.cvt[0] && tx <= a.cvt[1] && ty >= a.cvt[2] && ty <= a.cvt[3];
        const ST *sm = (const ST *)(smem + (size_t)s * C::STAGE_BYTES);
        A acc[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) acc_zero(acc[j]);
        bool bad = false;
        if (checked || edge || !full)
            tma_tile<S, true, false, true, FORCE>(a, sm, tx, ty, cvtile, acc, bad);
        else
            tma_tile<S, false, true, false, FORCE>(a, sm, tx, ty, cvtile, acc, bad);
        if (cvtile) cv_store<S, false, C::THREADS>(a, tx, ty, acc);
        const int any_bad = __syncthreads_or(bad);  // also: every read of stage s is done
        if (any_bad && threadIdx.x == 0) {
            atomicOr(a.status, 1);
            atomicMin(a.status + 1, (int)*a.step_ctr);
        }
        if (threadIdx.x == 0 && k + C::NS < count) {
            tma::fence_proxy_async();
            issue(k + C::NS, s);
        }
    }
}

template <int S, bool FORCE>
cudaError_t launch_tma_f(const StepArgs &a, int tiles, int sms, const void *map, cudaStream_t st)
{
    using C = TmaCfg<S>;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        e = cudaFuncSetAttribute(k_collide_stream_tma<S, FORCE>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    const int grid = tiles < sms * GBLBM_TMA_MINB ? tiles : sms * GBLBM_TMA_MINB;
    k_collide_stream_tma<S, FORCE><<<grid, C::THREADS, C::SMEM, st>>>(a, tiles, *(const CUtensorMap *)map);
    return cudaGetLastError();
}

template <int S>
cudaError_t launch_tma(const StepArgs &a, int tiles, int sms, const void *map, cudaStream_t st)
{
    if (a.gx != 0.0 || a.gy != 0.0) return launch_tma_f<S, true>(a, tiles, sms, map, st);
    return launch_tma_f<S, false>(a, tiles, sms, map, st);
}

size_t tma_stage_bytes(int storage)
{
    switch (storage) {
    case LBM_F64: return TmaCfg<LBM_F64>::STAGE_BYTES;
    case LBM_F32: return TmaCfg<LBM_F32>::STAGE_BYTES;
    case LBM_F32_DEV: return TmaCfg<LBM_F32_DEV>::STAGE_BYTES;
    default: return TmaCfg<LBM_F16_DEV>::STAGE_BYTES;
    }
}

int collide_stream_prefetch_rows(int storage, int sm_count, int tiles_x)
{
    if (GBLBM_PF_PERCENT <= 0 || storage == LBM_F64 || sm_count <= 0 || tiles_x <= 0) return 0;
    const int threads = (TILE_X / cols_per_thread(storage)) * (tile_rows(storage) / direct_rpt(storage));
    int per_sm = 0;
    cudaError_t e;
    switch (storage) {
    case LBM_F32:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_collide_stream<LBM_F32, false, false>, threads, 0);
        break;
    case LBM_F32_DEV:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_collide_stream<LBM_F32_DEV, false, false>, threads, 0);
        break;
    default:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_collide_stream<LBM_F16_DEV, false, false>, threads, 0);
        break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const long long tiles = (long long)per_sm * sm_count * GBLBM_PF_PERCENT / 100;
    const long long rows = (tiles + tiles_x / 2) / tiles_x;
    return (int)(rows < 1 ? 1 : rows);
}

cudaError_t launch_collide_stream(int storage, const StepArgs &a, int tiles_x, int tiles_y,
                                  bool momentum_only, const void *tmap, cudaStream_t st)
{
    if (!momentum_only && !a.periodic && !a.precollision && a.use_bulk && tmap) {
        const int tiles = tiles_x * tiles_y;
        switch (storage) {
        case LBM_F64: return launch_tma<LBM_F64>(a, tiles, a.sm_count, tmap, st);
        case LBM_F32: return launch_tma<LBM_F32>(a, tiles, a.sm_count, tmap, st);
        case LBM_F32_DEV: return launch_tma<LBM_F32_DEV>(a, tiles, a.sm_count, tmap, st);
        default: return launch_tma<LBM_F16_DEV>(a, tiles, a.sm_count, tmap, st);
        }
    }
    dim3 grid(tiles_x, tiles_y);
    const bool force = a.gx != 0.0 || a.gy != 0.0;
    dim3 block(TILE_X / cols_per_thread(storage), tile_rows(storage) / direct_rpt(storage));
#define GBLBM_CS(S)                                                    \
    if (momentum_only)                                                 \
        k_collide_stream<S, true, false><<<grid, block, 0, st>>>(a);   \
    else if (force)                                                    \
        k_collide_stream<S, false, true><<<grid, block, 0, st>>>(a);   \
    else                                                               \
        k_collide_stream<S, false, false><<<grid, block, 0, st>>>(a);
    switch (storage) {
    case LBM_F64: GBLBM_CS(LBM_F64); break;
    case LBM_F32: GBLBM_CS(LBM_F32); break;
    case LBM_F32_DEV: GBLBM_CS(LBM_F32_DEV); break;
    default: GBLBM_CS(LBM_F16_DEV); break;
    }
#undef GBLBM_CS
    return cudaGetLastError();
}

}  // namespace gblbm
