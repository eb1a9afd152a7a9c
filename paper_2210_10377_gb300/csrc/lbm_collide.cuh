// lbm_collide.cuh -- the per-node work of one collide-stream step (Section
// II, Eq. CollideAdv in pull form, halfway bounce-back, the channel's inlet and
// outlet columns, the DRTT box sums of Eq. rtt7) and one tile of it,
// collide_tile, for any tile shape.  Included by the single-domain kernels
// (lbm_step.cu) and the batched kernel (lbm_batch.cu): both run exactly this
// arithmetic per node.
#pragma once

#include "lbm_device.cuh"

namespace gblbm {

// ---------------------------------------------------------------------------
// Per-node pieces shared by the two collide-stream kernels.
// ---------------------------------------------------------------------------

// BGK collision of one node: rho = R0 + sum f (R0 = rho0 for deviation storage,
// 0 otherwise), u = (sum c f)/rho, and with theta0 = 1/3 the second-order
// equilibrium of Section II, less the base w_i R0,
//   feq_i - w_i R0 = w_i (drho + rho (3 c_i.u + 4.5 (c_i.u)^2 - 1.5 u^2)),
// evaluated for opposite directions together: they share the even part
// s = drho - 1.5 rho u^2 + 4.5 rho (c.u)^2 and differ in the sign of the odd
// part 3 rho c.u.  ft = f + (feq - f)/tau, plus 3 w_i c_i.g with a body force.
// out receives ft rounded to the storage type (the values that are stored).
__device__ __forceinline__ float recip(float v) { return __frcp_rn(v); }
__device__ __forceinline__ double recip(double v) { return 1.0 / v; }

template <int S, bool FORCE>
__device__ __forceinline__ void collide_node(const StepArgs &a, const typename Traits<S>::comp_t (&g)[9],
                                             typename Traits<S>::store_t (&out)[9], bool &bad)
{
    using ST = typename Traits<S>::store_t;
    using T = typename Traits<S>::comp_t;
    constexpr bool DEV = Traits<S>::dev;
    const T R0 = DEV ? param<T>(a.rho0, a.rho0_f) : T(0);
    const T jx = ((g[1] - g[3]) + (g[5] - g[6])) + (g[8] - g[7]);
    const T jy = ((g[2] - g[4]) + (g[5] + g[6])) - (g[7] + g[8]);
    const T drho = (((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7]))) + g[8];
    const T rho = R0 + drho;
    if (!(rho > T(0))) bad = true;
    const T inv = recip(rho);
    const T ux = jx * inv, uy = jy * inv;
    const T base = drho - rho * (T(1.5) * (ux * ux + uy * uy));
    const T r45 = T(4.5) * rho, r3 = T(3) * rho;
    const T om = param<T>(a.omega, a.omega_f);
    const T w0 = wgt<T>(0), w1 = wgt<T>(1), w5 = wgt<T>(5);
    T v[9];
    v[0] = g[0] + om * (w0 * base - g[0]);
    {  // directions 1 (+x) and 3 (-x): c.u = ux
        const T se = base + r45 * ux * ux, so = r3 * ux;
        v[1] = g[1] + om * (w1 * (se + so) - g[1]);
        v[3] = g[3] + om * (w1 * (se - so) - g[3]);
    }
    {  // directions 2 (+y) and 4 (-y): c.u = uy
        const T se = base + r45 * uy * uy, so = r3 * uy;
        v[2] = g[2] + om * (w1 * (se + so) - g[2]);
        v[4] = g[4] + om * (w1 * (se - so) - g[4]);
    }
    {  // directions 5 (+x+y) and 7 (-x-y): c.u = ux + uy
        const T c = ux + uy;
        const T se = base + r45 * c * c, so = r3 * c;
        v[5] = g[5] + om * (w5 * (se + so) - g[5]);
        v[7] = g[7] + om * (w5 * (se - so) - g[7]);
    }
    {  // directions 6 (-x+y) and 8 (+x-y): c.u = uy - ux
        const T c = uy - ux;
        const T se = base + r45 * c * c, so = r3 * c;
        v[6] = g[6] + om * (w5 * (se + so) - g[6]);
        v[8] = g[8] + om * (w5 * (se - so) - g[8]);
    }
    if (FORCE) {
        const T gx = param<T>(a.gx, a.gx_f), gy = param<T>(a.gy, a.gy_f);
#pragma unroll
        for (int i = 1; i < 9; ++i) v[i] += T(3) * wgt<T>(i) * (T(cx(i)) * gx + T(cy(i)) * gy);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) out[i] = to_store<ST>(v[i]);
}

// Control-volume contributions of one fluid node (x, y).
// acc[0..1]: J(t) of the box (Eq. rtt1) on the pre-collision f(t), as the
// Appendix orders it; acc[2..3]: J(t) on the stored post-collision ft(t) less
// the body-force momentum g.  BGK collision conserves momentum, so both are J(t)
// in exact arithmetic; the second is the one whose streamed values make up
// J(t+1), so it carries no rounding defect of the reduced-precision collision.
// (Deviation storage: the base w_i rho0 carries no momentum, sum_i c_i w_i = 0.)
// acc[4..5]: post-collision populations crossing the box surface, + entering,
// - leaving (Eq. rtt7); for deviation storage the fixed base parts w_i rho0 are
// added once by the link kernel.  nb: the node's neighbour bits (0 in tiles
// without solids).
template <int S, bool MOMENTUM_ONLY, bool FORCE = false>
__device__ __forceinline__ void cv_node(const StepArgs &a, int x, int y,
                                        const typename Traits<S>::comp_t *f,
                                        const typename Traits<S>::comp_t *ftr, uint16_t nb,
                                        typename AccOf<S>::type (&acc)[6])
{
    using T = typename Traits<S>::comp_t;
    using A = typename AccOf<S>::type;
    const bool channel = !a.periodic;
    const bool inV = x >= a.cv[0] && x <= a.cv[1] && y >= a.cv[2] && y <= a.cv[3];
    if (inV) {
        acc_add(acc[0], mom_x(f));
        acc_add(acc[1], mom_y(f));
        if (!MOMENTUM_ONLY) {
            acc_add(acc[2], mom_x(ftr));
            acc_add(acc[3], mom_y(ftr));
            if (FORCE) {
                acc_add(acc[2], as_acc(-param<T>(a.gx, a.gx_f), A()));
                acc_add(acc[3], as_acc(-param<T>(a.gy, a.gy_f), A()));
            }
        }
    }
    if (MOMENTUM_ONLY) return;
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
        if (nb & (1u << i)) continue;  // the neighbour is solid
        const T v = inV ? -ftr[i] : ftr[i];
        if (cx(i) != 0) acc_add(acc[4], as_acc(cx(i) > 0 ? v : -v, A()));
        if (cy(i) != 0) acc_add(acc[5], as_acc(cy(i) > 0 ? v : -v, A()));
    }
}

// Block-reduce the control-volume accumulators of a tile and store its slot.
template <int S, bool MOMENTUM_ONLY, int NT>
__device__ __forceinline__ void cv_store(const StepArgs &a, int tx, int ty,
                                         typename AccOf<S>::type (&acc)[6])
{
    using A = typename AccOf<S>::type;
    block_reduce<A, 6, NT>(acc);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const int slot = (ty - a.cvt[2]) * (a.cvt[1] - a.cvt[0] + 1) + (tx - a.cvt[0]);
        A *p = (A *)a.partials + CV_PARTIAL * (long long)slot;
#pragma unroll
        for (int k = 0; k < CV_PARTIAL; ++k) {
            if (MOMENTUM_ONLY && k >= 2)
                acc_zero(p[k]);
            else
                p[k] = acc[k];
        }
    }
}

// ---------------------------------------------------------------------------
// One thread's column of RPT rows: all loads are issued before the collisions.
// This general form serves the first step after the state was set
// (pre-collision state, no pull), fully periodic domains, tiles at a periodic
// edge and the momentum-only pass.
// CHECKED: the tile holds solid nodes (bounce-back tests needed).
// ---------------------------------------------------------------------------
template <int S, bool CHECKED, bool MOMENTUM_ONLY, int RPT, bool FORCE>
__device__ __forceinline__ void column_update(const StepArgs &a, int x, int y0,
                                              typename AccOf<S>::type (&acc)[6], bool cvtile,
                                              bool &bad)
{
    using ST = typename Traits<S>::store_t;
    using T = typename Traits<S>::comp_t;
    const ST *__restrict__ src = (const ST *)a.src;
    ST *__restrict__ dst = (ST *)a.dst;
    const long long plane = a.plane;
    const bool channel = !a.periodic;
    const bool inlet = channel && x == 0;
    if (inlet && MOMENTUM_ONLY) return;  // the inlet column never lies in the control volume
    // the outlet column x = nx-1 takes the populations of column nx-2
    const int xs = (channel && x == a.nx - 1 && !a.precollision) ? a.nx - 2 : x;
    int xm = xs - 1, xp = xs + 1;
    if (!channel) {
        xm = xm < 0 ? xm + a.nx : xm;
        xp = xp >= a.nx ? xp - a.nx : xp;
    }

    T f[RPT][9];
    uint16_t nb[RPT];
    bool live[RPT];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        const int y = y0 + r;
        live[r] = y < a.ny;
        const long long idx = (long long)y * a.pitch + x;
        nb[r] = (CHECKED && live[r]) ? a.nbits[idx] : (uint16_t)0;
        if (nb[r] & 1) live[r] = false;  // solid nodes are not updated
        if (!live[r] || inlet) continue;
        if (a.precollision) {
#pragma unroll
            for (int i = 0; i < 9; ++i) f[r][i] = to_comp(src[i * plane + idx]);
        } else {
            const long long sidx = (long long)y * a.pitch + xs;
            const uint16_t nbs = CHECKED ? (xs == x ? nb[r] : a.nbits[sidx]) : (uint16_t)0;
            const int ym = y == 0 ? a.ny - 1 : y - 1;
            const int yp = y == a.ny - 1 ? 0 : y + 1;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const int sx = cx(i) == 1 ? xm : (cx(i) == -1 ? xp : xs);
                const int sy = cy(i) == 1 ? ym : (cy(i) == -1 ? yp : y);
                if (CHECKED && (nbs & (1u << opp(i))))
                    f[r][i] = to_comp(src[opp(i) * plane + sidx]);
                else
                    f[r][i] = to_comp(src[i * plane + (long long)sy * a.pitch + sx]);
            }
        }
    }

#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        if (!live[r]) continue;
        const int y = y0 + r;
        const long long idx = (long long)y * a.pitch + x;
        T ftr[9];
        if (inlet) {
            const ST *in = (const ST *)a.inlet;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const ST sv = in[i * a.ny + y];
                dst[i * plane + idx] = sv;
                ftr[i] = to_comp(sv);
            }
        } else if (!MOMENTUM_ONLY) {
            ST out[9];
            collide_node<S, FORCE>(a, f[r], out, bad);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                dst[i * plane + idx] = out[i];
                ftr[i] = to_comp(out[i]);
            }
        }
        if (cvtile) cv_node<S, MOMENTUM_ONLY, FORCE>(a, x, y, f[r], ftr, nb[r], acc);
    }
}

// Interior tiles (no solid node in or next to the tile, no wrap in y, channel
// set-up, pulled state): every load of a thread is its own base address plus a
// warp-uniform offset i*plane - c_iy*pitch - c_ix, every store its own base plus
// i*plane, so the address arithmetic stays out of the per-node work.
template <int S, bool MOMENTUM_ONLY, int RPT, bool FORCE>
__device__ __forceinline__ void column_update_interior(const StepArgs &a, int x, int y0,
                                                       typename AccOf<S>::type (&acc)[6],
                                                       bool cvtile, bool &bad)
{
    using ST = typename Traits<S>::store_t;
    using T = typename Traits<S>::comp_t;
    const long long pitch = a.pitch, plane = a.plane;
    const bool inlet = x == 0;
    if (inlet && MOMENTUM_ONLY) return;
    // the outlet column x = nx-1 takes the populations of column nx-2
    const int xs = x == a.nx - 1 ? x - 1 : x;
    const ST *__restrict__ b = (const ST *)a.src + (long long)y0 * pitch + xs;
    ST *__restrict__ o = (ST *)a.dst + (long long)y0 * pitch + x;
    T f[RPT][9];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
        for (int i = 0; i < 9; ++i)
            f[r][i] = to_comp(b[r * pitch + i * plane - cy(i) * pitch - cx(i)]);
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        T ftr[9];
        if (inlet) {
            const ST *in = (const ST *)a.inlet;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const ST sv = in[i * a.ny + y0 + r];
                o[r * pitch + i * plane] = sv;
                ftr[i] = to_comp(sv);
            }
        } else if (!MOMENTUM_ONLY) {
            ST out[9];
            collide_node<S, FORCE>(a, f[r], out, bad);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                o[r * pitch + i * plane] = out[i];
                if (cvtile) ftr[i] = to_comp(out[i]);
            }
        }
        if (cvtile) cv_node<S, MOMENTUM_ONLY, FORCE>(a, x, y0 + r, f[r], ftr, 0, acc);
    }
}

// ---------------------------------------------------------------------------
// One tile of TX x TR nodes with TX x (TR/RPT) threads (threadIdx.x: column,
// threadIdx.y: group of RPT rows).  `checked` selects the bounce-back-aware
// path (solid nodes in or next to the tile, or a pre-collision state).  A
// block that met rho <= 0 or NaN sets status bit 0 and the first bad step.
// All threads of the block must call it (it synchronises).
// ---------------------------------------------------------------------------
template <int S, bool MOMENTUM_ONLY, bool FORCE, int TX, int TR, int RPT>
__device__ __forceinline__ void collide_tile(const StepArgs &a, int tx, int ty, bool checked)
{
    using A = typename AccOf<S>::type;
    const int x = tx * TX + threadIdx.x;
    const bool cvtile = tx >= a.cvt[0] && tx <= a.cvt[1] && ty >= a.cvt[2] && ty <= a.cvt[3];
    A acc[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) acc_zero(acc[k]);
    bool bad = false;
    const int y0 = ty * TR + threadIdx.y * RPT;
    const bool interior = !checked && !a.periodic && ty > 0 && (ty + 1) * TR < a.ny;
    if (x < a.nx) {
        if (interior)
            column_update_interior<S, MOMENTUM_ONLY, RPT, FORCE>(a, x, y0, acc, cvtile, bad);
        else if (checked)
            column_update<S, true, MOMENTUM_ONLY, RPT, FORCE>(a, x, y0, acc, cvtile, bad);
        else
            column_update<S, false, MOMENTUM_ONLY, RPT, FORCE>(a, x, y0, acc, cvtile, bad);
    }
    if (cvtile) cv_store<S, MOMENTUM_ONLY, TX *(TR / RPT)>(a, tx, ty, acc);
    if (!MOMENTUM_ONLY) {
        const int any_bad = __syncthreads_or(bad);
        if (any_bad && threadIdx.x == 0 && threadIdx.y == 0) {
            atomicOr(a.status, 1);
            atomicMin(a.status + 1, (int)*a.step_ctr);
        }
    }
}

}  // namespace gblbm
