// lbm_step.cu -- the per-step kernels.
//
// k_collide_stream: one pass over the grid per time step t -> t+1 (Section II,
//   Eq. CollideAdv, written in pull form).  Each fluid node gathers
//   f_i(x, t) = ft_i(x - c_i, t-1), or the bounced ft_opp(i)(x, t-1) when
//   x - c_i is solid (halfway bounce-back), takes rho and u, relaxes towards
//   feq (second-order equilibrium, theta0 = 1/3) and stores ft(x, t).  The
//   channel inlet column stores feq(rho0, u_in(y)); the outlet column collides
//   the populations of column nx-2 (zero-gradient copy).  Tiles that cover the
//   DRTT control volume also reduce J(t) (Eq. rtt1, pre-collision) and the
//   gained-minus-lost flux of ft(t) through the box surface (Eq. rtt7).
// k_link_force: one CTA walks the fluid-solid link list and reduces the
//   momentum exchange of step t for algorithms A, A' and B (Eqs. MEA, rtt4,
//   rtt5), folds the control-volume partials into J(t), and completes
//   DRTT(t-1) = J(t-1) - J(t) + GL(t-1) (Eq. rtt7).  Several CTAs share the
//   links; the last one to finish reduces their rows in a fixed order.
//
// All reductions run in FP64 in a fixed order (warp shuffles, then a fixed
// tree over warps), so results are deterministic for a given grid.
#include "lbm_internal.cuh"

namespace gblbm {

// FP64 block reduction; the result is valid in thread 0.  NT threads, NT % 32 == 0.
template <int NV, int NT>
__device__ __forceinline__ void block_reduce(double (&v)[NV])
{
    __shared__ double sm[NT / 32][NV];
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], d);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sm[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = lane < NT / 32 ? sm[lane][k] : 0.0;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
            v[k] = s;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Fused pull-stream + bounce-back + boundary + BGK collision for one node.
// CHECKED: the tile holds solid nodes (bounce-back tests needed).
// ---------------------------------------------------------------------------
template <int S, bool CHECKED, bool MOMENTUM_ONLY>
__device__ __forceinline__ void node_update(const StepArgs &a, int x, int y, double (&acc)[6],
                                            bool cvtile, bool &bad)
{
    using ST = typename Traits<S>::store_t;
    using T = typename Traits<S>::comp_t;
    constexpr bool DEV = Traits<S>::dev;
    const ST *__restrict__ src = (const ST *)a.src;
    ST *__restrict__ dst = (ST *)a.dst;
    const long long plane = a.plane;
    const long long idx = (long long)y * a.pitch + x;
    const bool channel = !a.periodic;
    const uint16_t nb = CHECKED ? a.nbits[idx] : (uint16_t)0;
    if (nb & 1) return;  // solid nodes are not updated

    T f[9];
    T ftr[9];
    T jx = T(0), jy = T(0);
    const bool inlet = channel && x == 0;
    if (inlet) {
        if (MOMENTUM_ONLY) return;  // the inlet column never lies in the control volume
        const ST *in = (const ST *)a.inlet;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            ST sv = in[i * a.ny + y];
            dst[i * plane + idx] = sv;
            ftr[i] = to_comp(sv);
        }
    } else {
        if (a.precollision) {
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = to_comp(src[i * plane + idx]);
        } else {
            // the outlet column x = nx-1 takes the populations of column nx-2
            const int xs = (channel && x == a.nx - 1) ? a.nx - 2 : x;
            const long long sidx = (long long)y * a.pitch + xs;
            const uint16_t nbs = CHECKED ? (xs == x ? nb : a.nbits[sidx]) : (uint16_t)0;
            int xm = xs - 1, xp = xs + 1;
            if (!channel) {
                xm = xm < 0 ? xm + a.nx : xm;
                xp = xp >= a.nx ? xp - a.nx : xp;
            }
            const int ym = y == 0 ? a.ny - 1 : y - 1;
            const int yp = y == a.ny - 1 ? 0 : y + 1;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int sx = cx(i) == 1 ? xm : (cx(i) == -1 ? xp : xs);
                const int sy = cy(i) == 1 ? ym : (cy(i) == -1 ? yp : y);
                if (CHECKED && (nbs & (1u << opp(i))))
                    f[i] = to_comp(src[opp(i) * plane + sidx]);
                else
                    f[i] = to_comp(src[i * plane + (long long)sy * a.pitch + sx]);
            }
        }
        jx = ((f[1] - f[3]) + (f[5] - f[6])) + (f[8] - f[7]);
        jy = ((f[2] - f[4]) + (f[5] + f[6])) - (f[7] + f[8]);
        if (!MOMENTUM_ONLY) {
            // rho = R0 + sum f (R0 = rho0 for deviation storage, 0 otherwise);
            // feq - w R0 = w (drho + rho (3 cu + 4.5 cu^2 - 1.5 u^2))
            const T R0 = DEV ? (T)a.rho0 : T(0);
            const T drho = (((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7]))) + f[8];
            const T rho = R0 + drho;
            if (!(rho > T(0))) bad = true;
            const T inv = T(1) / rho;
            const T ux = jx * inv, uy = jy * inv;
            const T usq = T(1.5) * (ux * ux + uy * uy);
            const T om = (T)a.omega;
            const T gx = (T)a.gx, gy = (T)a.gy;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const T cu = T(cx(i)) * ux + T(cy(i)) * uy;
                const T geq = wgt<T>(i) * (drho + rho * (cu * (T(3) + T(4.5) * cu) - usq));
                T v = f[i] + om * (geq - f[i]);
                if (i != 0) v += T(3) * wgt<T>(i) * (T(cx(i)) * gx + T(cy(i)) * gy);
                const ST sv = to_store<ST>(v);
                dst[i * plane + idx] = sv;
                ftr[i] = to_comp(sv);
            }
        }
    }

    if (!cvtile) return;
    const bool inV = x >= a.cv[0] && x <= a.cv[1] && y >= a.cv[2] && y <= a.cv[3];
    if (inV) {
        // J(t) of the box (Eq. rtt1).  Sums of stored-precision values taken in
        // FP64 are exact for FP32 and FP16 storage (at most ~42 significant bits).
        // acc[0..1]: on the pre-collision f(t), as the Appendix orders it;
        // acc[2..3]: on the stored post-collision ft(t) less the body-force
        // momentum g.  BGK collision conserves momentum, so both are J(t) in
        // exact arithmetic; the second is the one whose streamed values make
        // up J(t+1), so it carries no rounding defect of the collision.
        double d[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) d[i] = (double)f[i];
        acc[0] += ((d[1] - d[3]) + (d[5] - d[6])) + (d[8] - d[7]);
        acc[1] += ((d[2] - d[4]) + (d[5] + d[6])) - (d[7] + d[8]);
        if (!MOMENTUM_ONLY) {
#pragma unroll
            for (int i = 0; i < 9; ++i) d[i] = (double)ftr[i];
            acc[2] += (((d[1] - d[3]) + (d[5] - d[6])) + (d[8] - d[7])) - a.gx;
            acc[3] += (((d[2] - d[4]) + (d[5] + d[6])) - (d[7] + d[8])) - a.gy;
        }
    }
    if (MOMENTUM_ONLY) return;
    // post-collision populations crossing the box surface: + entering, - leaving
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        int x2 = x + cx(i);
        if (x2 < 0 || x2 >= a.nx) {
            if (channel) continue;
            x2 = x2 < 0 ? x2 + a.nx : x2 - a.nx;
        }
        int y2 = y + cy(i);
        y2 = y2 < 0 ? y2 + a.ny : (y2 >= a.ny ? y2 - a.ny : y2);
        const bool in2 = x2 >= a.cv[0] && x2 <= a.cv[1] && y2 >= a.cv[2] && y2 <= a.cv[3];
        if (in2 == inV) continue;
        if (CHECKED && (nb & (1u << i))) continue;  // the neighbour is solid
        double v = (double)ftr[i];
        if (DEV) v += wgt<double>(i) * a.rho0;
        if (inV) v = -v;
        acc[4] += cx(i) * v;
        acc[5] += cy(i) * v;
    }
}

template <int S, bool MOMENTUM_ONLY>
__global__ void __launch_bounds__(TILE_X * 2) k_collide_stream(StepArgs a)
{
    const int tx = blockIdx.x + a.tile_off_x, ty = blockIdx.y + a.tile_off_y;
    const int x = tx * TILE_X + threadIdx.x;
    const bool checked = a.precollision || a.tile_flag[(long long)ty * a.tiles_x + tx] != 0;
    const bool cvtile = tx >= a.cvt[0] && tx <= a.cvt[1] && ty >= a.cvt[2] && ty <= a.cvt[3];
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    bool bad = false;
    const int y0 = ty * TILE_ROWS + threadIdx.y * ROWS_PER_THREAD;
    if (x < a.nx) {
        if (checked) {
#pragma unroll
            for (int r = 0; r < ROWS_PER_THREAD; ++r)
                if (y0 + r < a.ny) node_update<S, true, MOMENTUM_ONLY>(a, x, y0 + r, acc, cvtile, bad);
        } else {
#pragma unroll
            for (int r = 0; r < ROWS_PER_THREAD; ++r)
                if (y0 + r < a.ny) node_update<S, false, MOMENTUM_ONLY>(a, x, y0 + r, acc, cvtile, bad);
        }
    }
    if (cvtile) {
        block_reduce<6, TILE_X * 2>(acc);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            const int slot = (ty - a.cvt[2]) * (a.cvt[1] - a.cvt[0] + 1) + (tx - a.cvt[0]);
            double *p = a.partials + CV_PARTIAL * (long long)slot;
#pragma unroll
            for (int k = 0; k < CV_PARTIAL; ++k) p[k] = (MOMENTUM_ONLY && k >= 2) ? 0.0 : acc[k];
        }
    }
    if (!MOMENTUM_ONLY) {
        const int any_bad = __syncthreads_or(bad);
        if (any_bad && threadIdx.x == 0 && threadIdx.y == 0) {
            atomicOr(a.status, 1);
            atomicMin(a.status + 1, (int)*a.step_ctr);
        }
    }
}

cudaError_t launch_collide_stream(int storage, const StepArgs &a, int tiles_x, int tiles_y,
                                  bool momentum_only, cudaStream_t st)
{
    dim3 grid(tiles_x, tiles_y), block(TILE_X, 2);
#define GBLBM_CS(S)                                                                    \
    if (momentum_only)                                                                 \
        k_collide_stream<S, true><<<grid, block, 0, st>>>(a);                          \
    else                                                                               \
        k_collide_stream<S, false><<<grid, block, 0, st>>>(a);
    switch (storage) {
    case LBM_F64: GBLBM_CS(LBM_F64); break;
    case LBM_F32: GBLBM_CS(LBM_F32); break;
    case LBM_F32_DEV: GBLBM_CS(LBM_F32_DEV); break;
    default: GBLBM_CS(LBM_F16_DEV); break;
    }
#undef GBLBM_CS
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Link force + finalisation.  LINK_CTAS CTAs of LINK_THREADS threads share the
// links (contiguous chunks) and the control-volume partials; each writes one
// FP64 partial row.  The last CTA to finish (atomic ticket) sums the rows in
// slot order, so the result does not depend on which CTA finishes last, and
// completes the step's series row and the DRTT of the previous step.
// Series row t: A(2) B(2) DRTT(2) A'(2) defect(2), where defect is the
// collision's momentum defect inside the box, J_pre(t) - J_post(t).
// ---------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(LINK_THREADS) k_link_force(LinkArgs a)
{
    using ST = typename Traits<S>::store_t;
    constexpr bool DEV = Traits<S>::dev;
    const ST *__restrict__ src = (const ST *)a.src;
    const ST *__restrict__ dst = (const ST *)a.dst;
    const long long plane = a.plane;
    // v: A(2), B(2), A'(2), J_pre(2), J_post(2), GL(2)
    double v[LINK_PARTIAL];
#pragma unroll
    for (int k = 0; k < LINK_PARTIAL; ++k) v[k] = 0.0;
    const long long per = (a.nlinks + gridDim.x - 1) / gridDim.x;
    const long long k0 = per * blockIdx.x;
    const long long k1 = k0 + per < a.nlinks ? k0 + per : a.nlinks;
    if (!a.drtt_only) {
        for (long long k = k0 + threadIdx.x; k < k1; k += LINK_THREADS) {
            const int l = a.links[k];
            const int n = l >> 3;
            const int i = (l & 7) + 1;
            const int o = opp(i);
            const int x = n % a.nx, y = n / a.nx;
            const long long idx = (long long)y * a.pitch + x;
            double fi, fo;
            if (a.precollision) {
                fi = (double)to_comp(src[i * plane + idx]);
                fo = (double)to_comp(src[o * plane + idx]);
            } else {
                // f_i(x_f, t): pulled from x_f - c_i, or bounced when that node is solid
                if (a.nbits[idx] & (1u << o)) {
                    fi = (double)to_comp(src[o * plane + idx]);
                } else {
                    int sx = x - cx(i), sy = y - cy(i);
                    if (a.periodic) sx = sx < 0 ? sx + a.nx : (sx >= a.nx ? sx - a.nx : sx);
                    sy = sy < 0 ? sy + a.ny : (sy >= a.ny ? sy - a.ny : sy);
                    fi = (double)to_comp(src[i * plane + (long long)sy * a.pitch + sx]);
                }
                // f_opp(i)(x_f, t): x_f + c_i is solid, so it is the bounced ft_i(x_f, t-1)
                fo = (double)to_comp(src[i * plane + idx]);
            }
            double ft = (double)to_comp(dst[i * plane + idx]);
            if (DEV) {
                const double base = wgt<double>(i) * a.rho0;  // w_i = w_opp(i)
                fi += base;
                fo += base;
                ft += base;
            }
            const double ex = cx(i), ey = cy(i);
            v[0] += ex * (fi + fo);
            v[1] += ey * (fi + fo);
            v[2] += 2.0 * ex * ft;
            v[3] += 2.0 * ey * ft;
            v[4] += ex * (fi + ft);
            v[5] += ey * (fi + ft);
        }
    }
    {
        const int per_p = (a.n_partials + gridDim.x - 1) / gridDim.x;
        const int p0 = per_p * blockIdx.x;
        const int p1 = p0 + per_p < a.n_partials ? p0 + per_p : a.n_partials;
        for (int s = p0 + threadIdx.x; s < p1; s += LINK_THREADS) {
            const double *p = a.partials + CV_PARTIAL * (long long)s;
#pragma unroll
            for (int k = 0; k < CV_PARTIAL; ++k) v[6 + k] += p[k];
        }
    }
    block_reduce<LINK_PARTIAL, LINK_THREADS>(v);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        double *row = a.link_partials + LINK_PARTIAL * (long long)blockIdx.x;
#pragma unroll
        for (int k = 0; k < LINK_PARTIAL; ++k) row[k] = v[k];
        __threadfence();
        const unsigned int ticket = atomicAdd(a.ticket, 1u);
        last = ticket == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double w[LINK_PARTIAL];
#pragma unroll
    for (int k = 0; k < LINK_PARTIAL; ++k) w[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += LINK_THREADS) {
        const volatile double *row = a.link_partials + LINK_PARTIAL * (long long)b;
#pragma unroll
        for (int k = 0; k < LINK_PARTIAL; ++k) w[k] += row[k];
    }
    block_reduce<LINK_PARTIAL, LINK_THREADS>(w);
    if (threadIdx.x == 0) {
        *a.ticket = 0u;
        const long long t = *a.step_ctr;
        auto row = [&](long long s) {
            return a.series + SERIES_ROW * (a.record_series ? s : (s & 1));
        };
        // DRTT(t-1) = J(t-1) - J(t) + (gained - lost)(t-1), Eq. rtt7, with
        // J(t-1) on the post-collision state and J(t) on the pre-collision one
        if (a.carry[4] != 0.0 && t >= 1) {
            double *q = row(t - 1);
            q[4] = (a.carry[0] - w[6]) + a.carry[2];
            q[5] = (a.carry[1] - w[7]) + a.carry[3];
        }
        if (!a.drtt_only) {
            double *r = row(t);
            r[0] = w[0];
            r[1] = w[1];
            r[2] = w[2];
            r[3] = w[3];
            r[6] = w[4];
            r[7] = w[5];
            r[8] = w[6] - w[8];
            r[9] = w[7] - w[9];
            a.carry[0] = w[8];
            a.carry[1] = w[9];
            a.carry[2] = w[10];
            a.carry[3] = w[11];
            a.carry[4] = 1.0;
            *a.step_ctr = t + 1;
        }
    }
}

cudaError_t launch_link_force(int storage, const LinkArgs &a, cudaStream_t st)
{
    const int grid = a.n_ctas;
    switch (storage) {
    case LBM_F64: k_link_force<LBM_F64><<<grid, LINK_THREADS, 0, st>>>(a); break;
    case LBM_F32: k_link_force<LBM_F32><<<grid, LINK_THREADS, 0, st>>>(a); break;
    case LBM_F32_DEV: k_link_force<LBM_F32_DEV><<<grid, LINK_THREADS, 0, st>>>(a); break;
    default: k_link_force<LBM_F16_DEV><<<grid, LINK_THREADS, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Read-back: pre-collision f_i(x, T) of one plane, widened to FP64 [ny][nx].
// After a step the buffer holds ft(T-1); f(T) is its pull with bounce-back,
// the inlet column's stored feq and the outlet copy of column nx-2.
// ---------------------------------------------------------------------------
template <int S>
__global__ void k_gather(const typename Traits<S>::store_t *__restrict__ pop,
                         const uint16_t *__restrict__ nbits, long long plane, int nx, int ny,
                         int pitch, int periodic, int precollision, double rho0, int i,
                         double *__restrict__ out)
{
    constexpr bool DEV = Traits<S>::dev;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= nx) return;
    const long long idx = (long long)y * pitch + x;
    double v;
    if (nbits[idx] & 1) {
        out[(long long)y * nx + x] = 0.0;
        return;
    }
    const bool channel = !periodic;
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
    out[(long long)y * nx + x] = v;
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
