// lbm_link.cu -- the per-step force kernel and the population read-back.
//
// k_link_force: CTAs share the fluid-solid link list and reduce the momentum
//   exchange of step t for algorithms A, A' and B (Eqs. MEA, rtt4, rtt5), fold
//   the control-volume partials into J(t), and the last CTA to finish completes
//   DRTT(t-1) = J(t-1) - J(t) + GL(t-1) (Eq. rtt7).
// k_link_force_batch: the same for every domain of a batch, one CTA each.
// k_gather / k_scatter: one population plane between the device storage and
//   an FP64 [ny][nx] array (pre-collision f(x, T) reconstructed by a pull).
// k_boundary_nodes / k_surface_pressure: the boundary fluid nodes and their
//   pressure coefficient (Section VI).
//
// Reductions are deterministic (fixed trees, no floating-point atomics).
#include "lbm_batch.cuh"
#include "lbm_device.cuh"

namespace gblbm {

// ---------------------------------------------------------------------------
// Per-link momentum exchange of step t over links [k0, k1) and the sum of the
// control-volume partial rows [p0, p1) (Eqs. MEA, rtt4, rtt5, rtt7), and the
// stress integral (Eq. stress_int) over the axis links:
// v: A(2), B(2), A'(2), J_pre(2), J_post(2), GL(2), SI(2).
//
// Stress integration: an axis link (x_f, i), i = 1..4, is a unit face of the
// voxelised surface with normal -c_i out of the solid; it adds -c_i.T(x_f)
// with T = -p I + sigma on the pre-collision f(x_f, t): p = rho/3 and sigma =
// -(1 - omega/2) (sum_k f_k c_k c_k - rho/3 I - rho u u), the non-equilibrium
// second moment written with the equilibrium's closed-form moments.  The
// pressure enters as (rho - rho0)/3: the faces of any solid come in opposite
// pairs along each axis, so the constant rho0/3 sums to zero, and leaving it
// out keeps the FP32 sums free of its cancellation.
// ---------------------------------------------------------------------------
// NT threads share the ranges.  EARLY: a thread's first partial row is loaded
// before the link loop, so that its latency overlaps the links' (the sums keep
// their order).
template <int S, int NT, bool EARLY>
__device__ __forceinline__ void link_sums(const LinkArgs &a, long long k0, long long k1, int p0, int p1,
                                          typename AccOf<S>::type (&v)[LINK_PARTIAL])
{
    using ST = typename Traits<S>::store_t;
    using T = typename Traits<S>::comp_t;
    using A = typename AccOf<S>::type;
    const ST *__restrict__ src = (const ST *)a.src;
    const ST *__restrict__ dst = (const ST *)a.dst;
    const long long plane = a.plane;
#pragma unroll
    for (int k = 0; k < LINK_PARTIAL; ++k) acc_zero(v[k]);
    const A *part = (const A *)a.partials;
    const int s0 = p0 + (int)threadIdx.x;
    A first[CV_PARTIAL];
#pragma unroll
    for (int k = 0; k < CV_PARTIAL; ++k) {
        if (EARLY && s0 < p1)
            first[k] = part[CV_PARTIAL * (long long)s0 + k];
        else
            acc_zero(first[k]);
    }
    for (long long k = k0 + threadIdx.x; k < k1; k += NT) {
        const int l = a.links[k];
        const int n = l >> 3;
        const int i = (l & 7) + 1;
        const int o = opp(i);
        const int x = n % a.nx, y = n / a.nx;
        const long long idx = (long long)y * a.pitch + x;
        T fi, fo;
        if (a.precollision) {
            fi = to_comp(src[i * plane + idx]);
            fo = to_comp(src[o * plane + idx]);
        } else {
            // f_i(x_f, t): pulled from x_f - c_i, or bounced when that node is solid
            if (a.nbits[idx] & (1u << o)) {
                fi = to_comp(src[o * plane + idx]);
            } else {
                int sx = x - cx(i), sy = y - cy(i);
                if (a.periodic) sx = sx < 0 ? sx + a.nx : (sx >= a.nx ? sx - a.nx : sx);
                sy = sy < 0 ? sy + a.ny : (sy >= a.ny ? sy - a.ny : sy);
                fi = to_comp(src[i * plane + (long long)sy * a.pitch + sx]);
            }
            // f_opp(i)(x_f, t): x_f + c_i is solid, so it is the bounced ft_i(x_f, t-1)
            fo = to_comp(src[i * plane + idx]);
        }
        const T ft = to_comp(dst[i * plane + idx]);
        A sa, sb, sp;
        if constexpr (S == LBM_F64) {
            sa = fi + fo;
            sb = 2.0 * ft;
            sp = fi + ft;
        } else {
            sa = ff_two_sum(fi, fo);
            sb = {2.0f * ft, 0.0f};
            sp = ff_two_sum(fi, ft);
        }
        if (i <= 4) {
            constexpr bool DEV = Traits<S>::dev;
            T g[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                if (a.precollision) {
                    g[q] = to_comp(src[q * plane + idx]);
                } else if (a.nbits[idx] & (1u << opp(q))) {
                    g[q] = to_comp(src[opp(q) * plane + idx]);
                } else {
                    int sx = x - cx(q), sy = y - cy(q);
                    if (a.periodic) sx = sx < 0 ? sx + a.nx : (sx >= a.nx ? sx - a.nx : sx);
                    sy = sy < 0 ? sy + a.ny : (sy >= a.ny ? sy - a.ny : sy);
                    g[q] = to_comp(src[q * plane + (long long)sy * a.pitch + sx]);
                }
            }
            const T r0 = (T)a.rho0;
            const T jx = ((g[1] - g[3]) + (g[5] - g[6])) + (g[8] - g[7]);
            const T jy = ((g[2] - g[4]) + (g[5] + g[6])) - (g[7] + g[8]);
            const T sum = (((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7]))) + g[8];
            // deviation storage holds f - w rho0: sum = rho - rho0, and the base
            // adds rho0/3 to the diagonal second moments
            const T drho = DEV ? sum : sum - r0;
            const T rho = r0 + drho;
            const T inv = T(1) / rho;
            const T ux = jx * inv, uy = jy * inv;
            const T diag = ((g[5] + g[6]) + (g[7] + g[8]));
            const T mxx = (g[1] + g[3]) + diag, myy = (g[2] + g[4]) + diag;
            const T mxy = (g[5] - g[6]) + (g[7] - g[8]);
            // sum f c c - rho/3 I - rho u u, with sum f c_x^2 = mxx (+ rho0/3 for deviations)
            const T third = T(1) / T(3);
            const T pxx = DEV ? (mxx - drho * third) - rho * ux * ux : (mxx - rho * third) - rho * ux * ux;
            const T pyy = DEV ? (myy - drho * third) - rho * uy * uy : (myy - rho * third) - rho * uy * uy;
            const T pxy = mxy - rho * ux * uy;
            const T visc = sizeof(T) == 8 ? (T)a.visc : (T)a.visc_f;
            const T pp = drho * third;
            const T txx = -pp - visc * pxx, tyy = -pp - visc * pyy, txy = -visc * pxy;
            // -c_i . T on the face
            const T fsx = cx(i) != 0 ? (cx(i) > 0 ? -txx : txx) : (cy(i) > 0 ? -txy : txy);
            const T fsy = cx(i) != 0 ? (cx(i) > 0 ? -txy : txy) : (cy(i) > 0 ? -tyy : tyy);
            acc_add(v[12], as_acc(fsx, A()));
            acc_add(v[13], as_acc(fsy, A()));
        }
        const int ex = cx(i), ey = cy(i);
        if (ex != 0) {
            acc_add(v[0], ex > 0 ? sa : -sa);
            acc_add(v[2], ex > 0 ? sb : -sb);
            acc_add(v[4], ex > 0 ? sp : -sp);
        }
        if (ey != 0) {
            acc_add(v[1], ey > 0 ? sa : -sa);
            acc_add(v[3], ey > 0 ? sb : -sb);
            acc_add(v[5], ey > 0 ? sp : -sp);
        }
    }
    if (EARLY && s0 < p1) {
#pragma unroll
        for (int k = 0; k < CV_PARTIAL; ++k) acc_add(v[6 + k], first[k]);
    }
    for (int s = EARLY ? s0 + NT : s0; s < p1; s += NT) {
#pragma unroll
        for (int k = 0; k < CV_PARTIAL; ++k) acc_add(v[6 + k], part[CV_PARTIAL * (long long)s + k]);
    }
}

// Completes the force rows from the reduced sums d, one warp: lane k holds
// d[k] (k < LINK_PARTIAL) and writes the outputs that need it, so that no
// lane runs more than a few FP64 operations (one thread running them all in
// turn took most of the kernel on this GPU's slow FP64 pipe).  prev: the row
// of step t-1, which receives DRTT(t-1) = J(t-1) - J(t) + (gained - lost)(t-1)
// (Eq. rtt7, J(t-1) on the post-collision state, J(t) on the pre-collision
// one); cur: the row of step t (A, B, A', defect, SI), written and the carry
// advanced unless drtt_only.  A null row pointer skips that row's stores.
// Every lane reads the carry before any lane writes it.
__device__ __forceinline__ void finish_rows_warp(const LinkArgs &a, double dk, long long t, double *prev,
                                                 double *cur, bool drtt_only)
{
    const int lane = threadIdx.x & 31;
    const double d6 = shfl_idx(dk, 6), d7 = shfl_idx(dk, 7);
    const double d8 = shfl_idx(dk, 8), d9 = shfl_idx(dk, 9);
    const double c0 = a.carry[0], c1 = a.carry[1], c2 = a.carry[2], c3 = a.carry[3], c4 = a.carry[4];
    __syncwarp();
    if (prev && c4 != 0.0 && t >= 1) {
        if (lane == 6) prev[4] = (c0 - d6) + c2;
        if (lane == 7) prev[5] = (c1 - d7) + c3;
    }
    if (drtt_only) return;
    if (cur) {
        switch (lane) {
        case 0: cur[0] = dk + a.link_base[0]; break;
        case 1: cur[1] = dk + a.link_base[1]; break;
        case 2: cur[2] = dk + a.link_base[0]; break;
        case 3: cur[3] = dk + a.link_base[1]; break;
        case 4: cur[6] = dk + a.link_base[0]; break;
        case 5: cur[7] = dk + a.link_base[1]; break;
        case 6: cur[8] = dk - d8; break;
        case 7: cur[9] = dk - d9; break;
        case 12: cur[10] = dk; break;
        case 13: cur[11] = dk; break;
        default: break;
        }
    }
    switch (lane) {
    case 8: a.carry[0] = dk; break;
    case 9: a.carry[1] = dk; break;
    case 10: a.carry[2] = dk + a.flux_base[0]; break;
    case 11: a.carry[3] = dk + a.flux_base[1]; break;
    case 14: a.carry[4] = 1.0; break;
    default: break;
    }
}

// ---------------------------------------------------------------------------
// Link force + finalisation of one domain.  n_ctas CTAs of LINK_THREADS
// threads share the links (contiguous chunks) and the control-volume
// partials; each writes one partial row.  The last CTA to finish (atomic
// ticket, one per warp) sums the warps' rows in a fixed order, so the result
// does not depend on which warp finishes last, and its lanes complete the
// step's series row and the DRTT of the previous step.
// Series row t: A(2) B(2) DRTT(2) A'(2) defect(2) SI(2), where defect is the
// collision's momentum defect inside the box, J_pre(t) - J_post(t).
// For deviation storage the momentum of the base w_i rho0 over the links and
// over the box-surface crossings is a fixed geometric sum (link_base,
// flux_base, from the host) added at the end.
// ---------------------------------------------------------------------------
// Load each thread's first control-volume row before the link loop (a tuning knob).
#ifndef GBLBM_LINK_EARLY
#define GBLBM_LINK_EARLY 1
#endif
template <int S>
__global__ void __launch_bounds__(LINK_THREADS) k_link_force(LinkArgs a)
{
    using A = typename AccOf<S>::type;
    A v[LINK_PARTIAL];
    {
        const long long nl = a.drtt_only ? 0 : a.nlinks;
        const long long per = (nl + gridDim.x - 1) / gridDim.x;
        const long long k0 = per * blockIdx.x;
        const long long k1 = k0 + per < nl ? k0 + per : nl;
        const int per_p = (a.n_partials + gridDim.x - 1) / gridDim.x;
        const int p0 = per_p * blockIdx.x;
        const int p1 = p0 + per_p < a.n_partials ? p0 + per_p : a.n_partials;
        link_sums<S, LINK_THREADS, GBLBM_LINK_EARLY != 0>(a, k0, k1 > k0 ? k1 : k0, p0, p1 > p0 ? p1 : p0, v);
    }
    // each warp reduces its sums and writes them as one row (slot: CTA, warp);
    // no block barrier, and the last warp to take a ticket completes the step
#pragma unroll
    for (int d = 16; d > 0; d >>= 1)
#pragma unroll
        for (int k = 0; k < LINK_PARTIAL; ++k) acc_add(v[k], shfl_down(v[k], d));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rows = (int)gridDim.x * LINK_WARPS;
    unsigned int ticket = 0;
    if (lane == 0) {
        A *row = (A *)a.link_partials + LINK_PARTIAL * ((long long)blockIdx.x * LINK_WARPS + warp);
#pragma unroll
        for (int k = 0; k < LINK_PARTIAL; ++k) row[k] = v[k];
        __threadfence();
        ticket = atomicAdd(a.ticket, 1u);
    }
    ticket = __shfl_sync(0xffffffffu, ticket, 0);
    if (ticket != (unsigned int)rows - 1) return;
    __threadfence();
    // lane k and lane 16 + k add sum k over the first and the second half of
    // the rows in slot order, then lane k adds the two halves.  The rows are
    // read from L2 (ld.global.cg), where the other warps' stores and fences
    // put them: an SM's L1 is not kept coherent within a launch.
    static_assert(LINK_PARTIAL <= 16, "two lanes per sum");
    const int k = lane & 15, half = (rows + 1) / 2;
    const int r0 = lane < 16 ? 0 : half, r1 = lane < 16 ? half : rows;
    A mine;
    acc_zero(mine);
    if (k < LINK_PARTIAL) {
        const A *col = (const A *)a.link_partials + k;
        for (int b = r0; b < r1; ++b) {
            A r;
            if constexpr (S == LBM_F64)
                r = __ldcg(col + LINK_PARTIAL * (long long)b);
            else
                r = {__ldcg(&col[LINK_PARTIAL * (long long)b].hi), __ldcg(&col[LINK_PARTIAL * (long long)b].lo)};
            acc_add(mine, r);
        }
    }
    {
        const A upper = shfl_down(mine, 16);
        if (lane < 16) acc_add(mine, upper);
    }
    const double dk = acc_double(mine);
    const long long t = *a.step_ctr;
    // Series slot of a step: the step itself, or its parity when only the
    // last two rows are kept.  A slot beyond the buffer (an internal
    // invariant: the host grows the series before every launch) is not
    // written and raises status bit 4.
    const bool keep_all = a.record_series != 0;
    const long long kp = keep_all ? t - 1 : ((t - 1) & 1), kc = keep_all ? t : (t & 1);
    double *prev = nullptr, *cur = nullptr;
    if (t >= 1 && a.carry[4] != 0.0) {
        if (kp < a.series_rows)
            prev = a.series + SERIES_ROW * kp;
        else if (lane == 0)
            atomicOr(a.status, 4);
    }
    if (!a.drtt_only) {
        if (kc < a.series_rows)
            cur = a.series + SERIES_ROW * kc;
        else if (lane == 0)
            atomicOr(a.status, 4);
    }
    finish_rows_warp(a, dk, t, prev, cur, a.drtt_only != 0);
    __syncwarp();
    if (lane == 0) {
        *a.ticket = 0u;
        if (!a.drtt_only) *a.step_ctr = t + 1;
    }
}

cudaError_t launch_link_force(int storage, const LinkArgs &a, cudaStream_t st, int priority)
{
    // The priority travels with the launch, so that a captured graph node
    // keeps it: the link kernel runs beside a collide-stream kernel that
    // fills the GPU, and the collide-stream kernel two steps on waits for it.
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = priority;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.n_ctas);
    cfg.blockDim = dim3(LINK_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = priority != 0 ? 1 : 0;
    switch (storage) {
    case LBM_F64: return cudaLaunchKernelEx(&cfg, k_link_force<LBM_F64>, a);
    case LBM_F32: return cudaLaunchKernelEx(&cfg, k_link_force<LBM_F32>, a);
    case LBM_F32_DEV: return cudaLaunchKernelEx(&cfg, k_link_force<LBM_F32_DEV>, a);
    default: return cudaLaunchKernelEx(&cfg, k_link_force<LBM_F16_DEV>, a);
    }
}

// ---------------------------------------------------------------------------
// Batched link force: one CTA per domain of a batch, the same sums and rows
// as k_link_force.  The series holds rows [step][domain].  Every CTA reads the
// shared step counter before it takes its ticket; the last CTA to arrive
// advances the counter, so no CTA can see the new value.
// ---------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(BATCH_LINK_THREADS) k_link_force_batch(BatchLinkArgs b)
{
    using A = typename AccOf<S>::type;
    static_assert(sizeof(LinkArgs) % 4 == 0, "LinkArgs is copied as 32-bit words");
    constexpr int WORDS = (int)(sizeof(LinkArgs) / 4);
    __shared__ LinkArgs la;
    __shared__ long long t_sh;
    {
        const int *src = (const int *)(b.args + blockIdx.x);
        int *dst = (int *)&la;
        for (int w = threadIdx.x; w < WORDS; w += BATCH_LINK_THREADS) dst[w] = src[w];
        if (threadIdx.x == 0) t_sh = *(volatile long long *)b.step_ctr;
    }
    __syncthreads();
    A v[LINK_PARTIAL];
    link_sums<S, BATCH_LINK_THREADS, true>(la, 0, b.drtt_only ? 0 : la.nlinks, 0, la.n_partials, v);
    block_reduce<A, LINK_PARTIAL, BATCH_LINK_THREADS>(v);
    if (threadIdx.x < 32) {
        // warp 0 finishes the domain's rows, lane k with total k (thread 0
        // holds the totals after the block reduction)
        const int lane = threadIdx.x;
        A mine;
        acc_zero(mine);
#pragma unroll
        for (int k = 0; k < LINK_PARTIAL; ++k) {
            const A tk = shfl_idx(v[k], 0);
            if (lane == k) mine = tk;
        }
        const double dk = acc_double(mine);
        const long long t = t_sh;
        const long long kp = b.keep_all ? t - 1 : ((t - 1) & 1), kc = b.keep_all ? t : (t & 1);
        const long long stride = (long long)b.n_domains * SERIES_ROW;
        double *prev = nullptr, *cur = nullptr;
        if (t >= 1 && la.carry[4] != 0.0) {
            if (kp < b.series_rows)
                prev = b.series + stride * kp + SERIES_ROW * (long long)blockIdx.x;
            else if (lane == 0)
                atomicOr(b.status, 4);
        }
        if (!b.drtt_only) {
            if (kc < b.series_rows)
                cur = b.series + stride * kc + SERIES_ROW * (long long)blockIdx.x;
            else if (lane == 0)
                atomicOr(b.status, 4);
        }
        finish_rows_warp(la, dk, t, prev, cur, b.drtt_only != 0);
        __threadfence();
        __syncwarp();
        if (lane == 0) {
            const unsigned int ticket = atomicAdd(b.ticket, 1u);
            if (ticket == gridDim.x - 1) {
                *b.ticket = 0u;
                if (!b.drtt_only) *b.step_ctr = t + 1;
            }
        }
    }
}

cudaError_t launch_link_force_batch(int storage, const BatchLinkArgs &b, cudaStream_t st)
{
    const int grid = b.n_domains;
    if (grid < 1) return cudaSuccess;
    switch (storage) {
    case LBM_F64: k_link_force_batch<LBM_F64><<<grid, BATCH_LINK_THREADS, 0, st>>>(b); break;
    case LBM_F32: k_link_force_batch<LBM_F32><<<grid, BATCH_LINK_THREADS, 0, st>>>(b); break;
    case LBM_F32_DEV: k_link_force_batch<LBM_F32_DEV><<<grid, BATCH_LINK_THREADS, 0, st>>>(b); break;
    default: k_link_force_batch<LBM_F16_DEV><<<grid, BATCH_LINK_THREADS, 0, st>>>(b); break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Read-back: pre-collision f_i(x, T) of one plane, widened to FP64 [ny][nx].
// After a step the buffer holds ft(T-1); f(T) is its pull with bounce-back,
// the inlet column's stored feq and the outlet copy of column nx-2.
// ---------------------------------------------------------------------------
// f_i(x, y, T) (FP64, the full population for deviation storage) of a fluid node.
template <int S>
__device__ __forceinline__ double pulled_value(const typename Traits<S>::store_t *__restrict__ pop,
                                               const uint16_t *__restrict__ nbits, long long plane, int nx,
                                               int ny, int pitch, int periodic, int precollision, double rho0,
                                               int x, int y, int i)
{
    constexpr bool DEV = Traits<S>::dev;
    const long long idx = (long long)y * pitch + x;
    const bool channel = !periodic;
    double v;
    if (precollision || (channel && x == 0)) {
        v = (double)to_comp(pop[i * plane + idx]);
    } else {
        const int xs = (channel && x == nx - 1) ? nx - 2 : x;
        const long long sidx = (long long)y * pitch + xs;
        const int o = opp(i);
        if (nbits[sidx] & (1u << o)) {
            v = (double)to_comp(pop[o * plane + sidx]);
        } else {
            int sx = xs - cx(i), sy = y - cy(i);
            if (!channel) sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
            sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
            v = (double)to_comp(pop[i * plane + (long long)sy * pitch + sx]);
        }
    }
    if (DEV) v += wgt<double>(i) * rho0;
    return v;
}

template <int S>
__global__ void k_gather(const typename Traits<S>::store_t *__restrict__ pop,
                         const uint16_t *__restrict__ nbits, long long plane, int nx, int ny,
                         int pitch, int periodic, int precollision, double rho0, int i,
                         double *__restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= nx) return;
    const long long idx = (long long)y * pitch + x;
    out[(long long)y * nx + x] =
        (nbits[idx] & 1) ? 0.0 : pulled_value<S>(pop, nbits, plane, nx, ny, pitch, periodic, precollision, rho0, x, y, i);
}

// ---------------------------------------------------------------------------
// Boundary fluid nodes: the distinct nodes of the ascending link list, by one
// CTA walking the list in chunks with a block-wide prefix count.
// ---------------------------------------------------------------------------
constexpr int BNODE_THREADS = 1024;

__global__ void __launch_bounds__(BNODE_THREADS)
    k_boundary_nodes(const int32_t *__restrict__ links, long long nlinks, int32_t *__restrict__ nodes,
                     long long *__restrict__ count)
{
    __shared__ int warp_sum[BNODE_THREADS / 32];
    __shared__ long long base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (long long k0 = 0; k0 < nlinks; k0 += BNODE_THREADS) {
        const long long k = k0 + threadIdx.x;
        int first = 0, node = 0;
        if (k < nlinks) {
            node = links[k] >> 3;
            first = (k == 0 || (links[k - 1] >> 3) != node) ? 1 : 0;
        }
        int incl = first;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += v;
        }
        if (lane == 31) warp_sum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            int w = warp_sum[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += v;
            }
            warp_sum[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        const int before = (warp > 0 ? warp_sum[warp - 1] : 0) + incl - first;
        if (first) nodes[base + before] = node;
        __syncthreads();
        if (threadIdx.x == BNODE_THREADS - 1) base += before + first;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base;
}

cudaError_t launch_boundary_nodes(const int32_t *links, long long nlinks, int32_t *nodes, long long *count,
                                  cudaStream_t st)
{
    k_boundary_nodes<<<1, BNODE_THREADS, 0, st>>>(links, nlinks, nodes, count);
    return cudaGetLastError();
}

// Pressure coefficient at boundary fluid nodes (Section VI):
// cp = (rho/3 - p_inf) / q with rho from the pre-collision populations.
template <int S>
__global__ void k_surface_pressure(const typename Traits<S>::store_t *__restrict__ pop,
                                   const uint16_t *__restrict__ nbits, const int32_t *__restrict__ nodes,
                                   long long count, long long plane, int nx, int ny, int pitch, int periodic,
                                   int precollision, double rho0, double p_inf, double q, double *__restrict__ cp)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int n = nodes[k];
    const int x = n % nx, y = n / nx;
    double rho = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) rho += pulled_value<S>(pop, nbits, plane, nx, ny, pitch, periodic, precollision, rho0, x, y, i);
    cp[k] = (rho / 3.0 - p_inf) / q;
}

cudaError_t launch_surface_pressure(int storage, const void *pop, const uint16_t *nbits, const int32_t *nodes,
                                    long long count, long long plane, int nx, int ny, int pitch, int periodic,
                                    int precollision, double rho0, double p_inf, double q, double *cp,
                                    cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    const int blocks = (int)((count + 127) / 128);
#define GBLBM_SP(S, T)                                                                                   \
    k_surface_pressure<S><<<blocks, 128, 0, st>>>((const T *)pop, nbits, nodes, count, plane, nx, ny, pitch, \
                                                  periodic, precollision, rho0, p_inf, q, cp)
    switch (storage) {
    case LBM_F64: GBLBM_SP(LBM_F64, double); break;
    case LBM_F32: GBLBM_SP(LBM_F32, float); break;
    case LBM_F32_DEV: GBLBM_SP(LBM_F32_DEV, float); break;
    default: GBLBM_SP(LBM_F16_DEV, __half); break;
    }
#undef GBLBM_SP
    return cudaGetLastError();
}

template <int S>
__global__ void k_scatter(typename Traits<S>::store_t *__restrict__ pop,
                          const uint16_t *__restrict__ nbits, long long plane, int nx, int ny,
                          int pitch, double rho0, int i, const double *__restrict__ in)
{
    using ST = typename Traits<S>::store_t;
    using T = typename Traits<S>::comp_t;
    constexpr bool DEV = Traits<S>::dev;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= nx) return;
    const long long idx = (long long)y * pitch + x;
    double v = (nbits[idx] & 1) ? 0.0 : in[(long long)y * nx + x];
    if (DEV && !(nbits[idx] & 1)) v -= wgt<double>(i) * rho0;
    pop[i * plane + idx] = to_store<ST>((T)v);
}

cudaError_t launch_gather(int storage, const void *pop, const uint16_t *nbits, const void *inlet,
                          long long plane, int nx, int ny, int pitch, int periodic,
                          int precollision, double rho0, int plane_i, double *out,
                          cudaStream_t st)
{
    (void)inlet;
    dim3 grid((nx + 255) / 256, ny);
    switch (storage) {
    case LBM_F64:
        k_gather<LBM_F64><<<grid, 256, 0, st>>>((const double *)pop, nbits, plane, nx, ny, pitch,
                                                 periodic, precollision, rho0, plane_i, out);
        break;
    case LBM_F32:
        k_gather<LBM_F32><<<grid, 256, 0, st>>>((const float *)pop, nbits, plane, nx, ny, pitch,
                                                 periodic, precollision, rho0, plane_i, out);
        break;
    case LBM_F32_DEV:
        k_gather<LBM_F32_DEV><<<grid, 256, 0, st>>>((const float *)pop, nbits, plane, nx, ny,
                                                     pitch, periodic, precollision, rho0, plane_i,
                                                     out);
        break;
    default:
        k_gather<LBM_F16_DEV><<<grid, 256, 0, st>>>((const __half *)pop, nbits, plane, nx, ny,
                                                     pitch, periodic, precollision, rho0, plane_i,
                                                     out);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_scatter_pop(int storage, void *pop, const uint16_t *nbits, long long plane,
                               int nx, int ny, int pitch, double rho0, int plane_i,
                               const double *in, cudaStream_t st)
{
    dim3 grid((nx + 255) / 256, ny);
    switch (storage) {
    case LBM_F64:
        k_scatter<LBM_F64><<<grid, 256, 0, st>>>((double *)pop, nbits, plane, nx, ny, pitch,
                                                  rho0, plane_i, in);
        break;
    case LBM_F32:
        k_scatter<LBM_F32><<<grid, 256, 0, st>>>((float *)pop, nbits, plane, nx, ny, pitch,
                                                  rho0, plane_i, in);
        break;
    case LBM_F32_DEV:
        k_scatter<LBM_F32_DEV><<<grid, 256, 0, st>>>((float *)pop, nbits, plane, nx, ny, pitch,
                                                      rho0, plane_i, in);
        break;
    default:
        k_scatter<LBM_F16_DEV><<<grid, 256, 0, st>>>((__half *)pop, nbits, plane, nx, ny, pitch,
                                                      rho0, plane_i, in);
        break;
    }
    return cudaGetLastError();
}

}  // namespace gblbm
