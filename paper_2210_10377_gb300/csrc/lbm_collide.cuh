// lbm_collide.cuh -- the per-node work of one collide-stream step (Section
// II, Eq. CollideAdv in pull form, halfway bounce-back, the channel's inlet and
// outlet columns, the DRTT box sums of Eq. rtt7) and one tile of it,
// collide_tile, for any tile shape.  Included by the single-domain kernels
// (lbm_step.cu) and the batched kernel (lbm_batch.cu): both run exactly this
// arithmetic per node.
#pragma once

#include "lbm_device.cuh"

namespace gblbm {

// Asks L2 for `bytes` bytes of global memory from p (a bulk prefetch through
// the copy engine; p and bytes multiples of 16).  It changes no value.
__device__ __forceinline__ void prefetch_l2(const void *p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes));
}

// ---------------------------------------------------------------------------
// Per-node pieces shared by the two collide-stream kernels.
// ---------------------------------------------------------------------------

// BGK collision (Section II, Eq. CollideAdv): rho = R0 + sum g (R0 = rho0 for
// deviation storage, g = f - w rho0; R0 = 0 and g = f otherwise), j = sum c g,
// u = j / rho, and with theta0 = 1/3 the second-order equilibrium less its
// base, written with rho u = j,
//   feq_i - w_i R0 = w_i (base + 4.5 (c_i.j)(c_i.u)) + 3 w_i c_i.j,
//   base = drho - 1.5 j.u,
// evaluated for opposite directions together (they share the even part and
// differ in the sign of the odd one).  The relaxation is ft = g + omega (feq -
// g), plus 3 w_i c_i.g with a body force.  In exact arithmetic every such
// form is the same map; in FP32 this one conserves momentum to the last
// rounding (see Lat and relax_pair_j), which keeps reduced-precision runs on
// the FP64 trajectory far longer.
//
// The FP32 arithmetic is spelled out operation by operation, each rounded
// once, in one template over the value type: one node (float) or two nodes at
// once in the packed FP32 pairs of this GPU (float2, two results per
// instruction); FP64 (double) runs the same expression.  A subtraction of packed pairs is an fma with -1, which is
// exact, so every lane of the packed form computes exactly the bits of the
// one-node form: which form a node takes (a pair of rows in interior tiles,
// single nodes elsewhere) never changes its result.
template <typename V> struct Arith;
template <> struct Arith<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    static __device__ __forceinline__ float splat(float c) { return c; }
    static __device__ __forceinline__ float rcp(float v) { return __frcp_rn(v); }
    static __device__ __forceinline__ float neg(float v) { return -v; }
};
// FP64 has no packed form, so its operations are left to the compiler (it
// may fuse a product into the following sum), as in any FP64 expression.
template <> struct Arith<double> {
    static __device__ __forceinline__ double add(double a, double b) { return a + b; }
    static __device__ __forceinline__ double sub(double a, double b) { return a - b; }
    static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return a * b + c; }
    static __device__ __forceinline__ double splat(double c) { return c; }
    static __device__ __forceinline__ double rcp(double v) { return 1.0 / v; }
    static __device__ __forceinline__ double neg(double v) { return -v; }
};
// Packed FP32 pairs.  The code generator may fuse a packed product that feeds
// a packed sum into one packed fma (measured: it does, whatever rounding
// modifier the two carry), which the one-node form never does; so the
// collision below never lets a product feed a sum: it writes such pairs as
// explicit fmas.
template <> struct Arith<float2> {
    static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ float2 sub(float2 a, float2 b)
    {
        return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
    }
    static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ float2 splat(float c) { return make_float2(c, c); }
    static __device__ __forceinline__ float2 rcp(float2 v) { return make_float2(__frcp_rn(v.x), __frcp_rn(v.y)); }
    static __device__ __forceinline__ float2 neg(float2 v) { return make_float2(-v.x, -v.y); }
};


// Lattice constants of the momentum-exact form, in the compute type T:
// w0 = 4/9, w1 = 1/9, w5 = 1/36, and the odd-part weights 3 w1 = A1 and
// 3 w5 = A5 chosen so that 2 A1 + 4 A5 = 1 holds exactly in T (the D2Q9
// identity sum_i w_i c_ix c_ix = theta0 = 1/3, times 3).  With rounded 1/3 and
// 1/12 the identity is off by a few units in the last place, and every
// collision of a uniform-flow region then makes or destroys the same small
// momentum at every node, a coherent drift of the whole flow.
template <typename T> struct Lat {
    static constexpr T W0 = T(4) / T(9), W1 = T(1) / T(9), W5 = T(1) / T(36);
    static constexpr T A1 = T(1) / T(3);
    static constexpr T A5 = (T(1) - T(2) * A1) * T(0.25);  // exact: 1 - 2 A1 and / 4 round nothing
};

// One pair of opposite directions: cj = c.j and cu = c.u of the direction
// with the + sign.  The equilibrium deviations are
//   eq+- = w (base + 4.5 (c.j)(c.u)) +- A (c.j)
// (second order in u, theta0 = 1/3, rho u = j), and the relaxation is
// ft = g + omega (eq - g), so that the old value enters with weight exactly
// one.  eq - g is formed as w (...) + (+-A (c.j) - g): the large odd part and
// the old value meet inside one fma, whose small result rounds far below the
// storage precision, and the even part joins it in a second fma, so that the
// only rounding at the size of g is the last.
template <typename V, typename T>
__device__ __forceinline__ void relax_pair_j(V cj, V cu, V w, V A, V om, V base, V gp, V gm, V &vp, V &vm)
{
    using O = Arith<V>;
    const V se = O::fma(O::mul(cj, O::splat(T(4.5))), cu, base);
    const V dp = O::fma(w, se, O::fma(A, cj, O::neg(gp)));
    const V dm = O::fma(w, se, O::fma(O::neg(A), cj, O::neg(gm)));
    vp = O::fma(om, dp, gp);
    vm = O::fma(om, dm, gm);
}

// The collision of one node (V = T) or of two (V = float2, T = float); T is
// the compute type of the uniform constants.  rho receives the density.
template <typename V, typename T, bool DEV, bool FORCE>
__device__ __forceinline__ void collide_core(const StepArgs &a, const V (&g)[9], V (&v)[9], V &rho)
{
    using O = Arith<V>;
    using L = Lat<T>;
    const V om = O::splat(param<T>(a.omega, a.omega_f));
    const V jx = O::add(O::add(O::sub(g[1], g[3]), O::sub(g[5], g[6])), O::sub(g[8], g[7]));
    const V jy = O::sub(O::add(O::sub(g[2], g[4]), O::add(g[5], g[6])), O::add(g[7], g[8]));
    const V jpd = O::add(jx, jy), jmd = O::sub(jy, jx);
    const V drho = O::add(O::add(O::add(O::add(g[0], g[1]), O::add(g[2], g[3])),
                                 O::add(O::add(g[4], g[5]), O::add(g[6], g[7]))),
                          g[8]);
    rho = DEV ? O::add(O::splat(param<T>(a.rho0, a.rho0_f)), drho) : drho;
    const V inv = O::rcp(rho);
    const V ux = O::mul(jx, inv), uy = O::mul(jy, inv);
    // base = drho - 1.5 rho u^2 = drho - 1.5 j.u
    const V base = O::fma(O::fma(jx, ux, O::mul(jy, uy)), O::splat(T(-1.5)), drho);
    v[0] = O::fma(om, O::fma(O::splat(L::W0), base, O::neg(g[0])), g[0]);
    const V w1 = O::splat(L::W1), w5 = O::splat(L::W5), a1 = O::splat(L::A1), a5 = O::splat(L::A5);
    // directions 1 (+x) and 3 (-x); 2 (+y) and 4 (-y); 5 (+x+y) and 7 (-x-y);
    // 6 (-x+y) and 8 (+x-y)
    relax_pair_j<V, T>(jx, ux, w1, a1, om, base, g[1], g[3], v[1], v[3]);
    relax_pair_j<V, T>(jy, uy, w1, a1, om, base, g[2], g[4], v[2], v[4]);
    relax_pair_j<V, T>(jpd, O::add(ux, uy), w5, a5, om, base, g[5], g[7], v[5], v[7]);
    relax_pair_j<V, T>(jmd, O::sub(uy, ux), w5, a5, om, base, g[6], g[8], v[6], v[8]);
    if constexpr (FORCE) {
        const T gx = param<T>(a.gx, a.gx_f), gy = param<T>(a.gy, a.gy_f);
#pragma unroll
        for (int i = 1; i < 9; ++i)
            v[i] = O::add(v[i], O::splat(T(3) * wgt<T>(i) * (T(cx(i)) * gx + T(cy(i)) * gy)));
    }
}

// One node; out receives ft rounded to the storage type (the stored values).
template <int S, bool FORCE>
__device__ __forceinline__ void collide_node(const StepArgs &a, const typename Traits<S>::comp_t (&g)[9],
                                             typename Traits<S>::store_t (&out)[9], bool &bad)
{
    using ST = typename Traits<S>::store_t;
    using T = typename Traits<S>::comp_t;
    T v[9], rho;
    collide_core<T, T, Traits<S>::dev, FORCE>(a, g, v, rho);
    if (!(rho > T(0))) bad = true;
#pragma unroll
    for (int i = 0; i < 9; ++i) out[i] = to_store<ST>(v[i]);
}

// Two nodes in packed FP32 pairs from their populations already paired.
template <int S, bool FORCE>
__device__ __forceinline__ void collide_pair2(const StepArgs &a, const float2 (&g)[9],
                                              typename Traits<S>::store_t (&out0)[9],
                                              typename Traits<S>::store_t (&out1)[9], bool &bad)
{
    using ST = typename Traits<S>::store_t;
    float2 v[9], rho;
    collide_core<float2, float, Traits<S>::dev, FORCE>(a, g, v, rho);
    if (!(rho.x > 0.0f) || !(rho.y > 0.0f)) bad = true;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        out0[i] = to_store<ST>(v[i].x);
        out1[i] = to_store<ST>(v[i].y);
    }
}

// Two nodes in packed FP32 pairs (FP32 compute types only).
template <int S, bool FORCE>
__device__ __forceinline__ void collide_pair(const StepArgs &a, const float (&g0)[9], const float (&g1)[9],
                                             typename Traits<S>::store_t (&out0)[9],
                                             typename Traits<S>::store_t (&out1)[9], bool &bad)
{
    using ST = typename Traits<S>::store_t;
    float2 g[9], v[9], rho;
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = make_float2(g0[i], g1[i]);
    collide_core<float2, float, Traits<S>::dev, FORCE>(a, g, v, rho);
    if (!(rho.x > 0.0f) || !(rho.y > 0.0f)) bad = true;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        out0[i] = to_store<ST>(v[i].x);
        out1[i] = to_store<ST>(v[i].y);
    }
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
    if constexpr (MOMENTUM_ONLY) return;
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
    if constexpr (S == LBM_F16_DEV && RPT % 2 == 0 && !MOMENTUM_ONLY) {
        if (!inlet) {
            // FP16 deviations: the populations of a thread's row pairs are held
            // packed two to a register until the pair collision widens them
            __half2 h[RPT / 2][9];
#pragma unroll
            for (int q = 0; q < RPT / 2; ++q)
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const long long off = i * plane - cy(i) * pitch - cx(i);
                    h[q][i] = __halves2half2(b[(2 * q) * pitch + off], b[(2 * q + 1) * pitch + off]);
                }
#pragma unroll
            for (int q = 0; q < RPT / 2; ++q) {
                float2 g[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) g[i] = __half22float2(h[q][i]);
                ST out0[9], out1[9];
                collide_pair2<S, FORCE>(a, g, out0, out1, bad);
                const int r = 2 * q;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    o[r * pitch + i * plane] = out0[i];
                    o[(r + 1) * pitch + i * plane] = out1[i];
                }
                if (cvtile) {
                    T f0[9], f1[9], ftr[9];
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        f0[i] = g[i].x;
                        f1[i] = g[i].y;
                        ftr[i] = to_comp(out0[i]);
                    }
                    cv_node<S, MOMENTUM_ONLY, FORCE>(a, x, y0 + r, f0, ftr, 0, acc);
#pragma unroll
                    for (int i = 0; i < 9; ++i) ftr[i] = to_comp(out1[i]);
                    cv_node<S, MOMENTUM_ONLY, FORCE>(a, x, y0 + r + 1, f1, ftr, 0, acc);
                }
            }
            return;
        }
    }
    T f[RPT][9];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
        for (int i = 0; i < 9; ++i)
            f[r][i] = to_comp(b[r * pitch + i * plane - cy(i) * pitch - cx(i)]);
    constexpr bool PAIRS = sizeof(T) == 4 && RPT % 2 == 0 && !MOMENTUM_ONLY;
    // FP32 storages: the inlet lane runs the same instructions as its warp on
    // its (unused) pulls and then takes the inlet's values, so that its warp
    // does not split into two paths (its collision raises no instability
    // flag).  FP16 deviations reach this form only off their column-pair path
    // and keep the inlet apart: on their tighter register budget the inlet in
    // the pair paths cost them 4-15 % (measured).
    constexpr bool INLET_IN_PAIRS = S != LBM_F16_DEV;
    if constexpr (PAIRS) {
      if (INLET_IN_PAIRS || !inlet) {
        // two rows at a time in packed FP32 pairs (identical bits to one node at a time)
#pragma unroll
        for (int r = 0; r < RPT; r += 2) {
            ST out0[9], out1[9];
            bool bad2 = false;
            collide_pair<S, FORCE>(a, f[r], f[r + 1], out0, out1, bad2);
            if (INLET_IN_PAIRS && inlet) {
                const ST *in = (const ST *)a.inlet;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    out0[i] = in[i * a.ny + y0 + r];
                    out1[i] = in[i * a.ny + y0 + r + 1];
                }
            } else if (bad2) {
                bad = true;
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                o[r * pitch + i * plane] = out0[i];
                o[(r + 1) * pitch + i * plane] = out1[i];
            }
            if (cvtile) {
                T ftr[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) ftr[i] = to_comp(out0[i]);
                cv_node<S, MOMENTUM_ONLY, FORCE>(a, x, y0 + r, f[r], ftr, 0, acc);
#pragma unroll
                for (int i = 0; i < 9; ++i) ftr[i] = to_comp(out1[i]);
                cv_node<S, MOMENTUM_ONLY, FORCE>(a, x, y0 + r + 1, f[r + 1], ftr, 0, acc);
            }
        }
        return;
      }
    }
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

// Interior tiles of FP16 deviations, two adjacent columns x, x+1 (x even, both
// strictly inside (0, nx-1)) and RPT rows per thread: the directions with
// c_x = 0 load both columns as one aligned __half2, the others load their two
// halves; the two columns collide together as the lanes of the packed pair and
// every direction stores both as one __half2.  The same bits as one column at a
// time.
template <int S, bool MOMENTUM_ONLY, int RPT, bool FORCE>
__device__ __forceinline__ void column_pair_update_interior(const StepArgs &a, int x, int y0,
                                                            typename AccOf<S>::type (&acc)[6],
                                                            bool cvtile, bool &bad)
{
    static_assert(S == LBM_F16_DEV, "column pairs are the FP16-deviation layout");
    const long long pitch = a.pitch, plane = a.plane;
    const __half *__restrict__ b = (const __half *)a.src + (long long)y0 * pitch + x;
    __half *__restrict__ o = (__half *)a.dst + (long long)y0 * pitch + x;
    __half2 h[RPT][9];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const long long off = r * pitch + i * plane - cy(i) * pitch;
            if (cx(i) == 0)
                h[r][i] = *(const __half2 *)(b + off);
            else
                h[r][i] = __halves2half2(b[off - cx(i)], b[off + 1 - cx(i)]);
        }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
        float2 g[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = __half22float2(h[r][i]);
        if constexpr (!MOMENTUM_ONLY) {
            float2 v[9], rho;
            collide_core<float2, float, true, FORCE>(a, g, v, rho);
            if (!(rho.x > 0.0f) || !(rho.y > 0.0f)) bad = true;
            __half2 out[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                out[i] = __float22half2_rn(v[i]);
                *(__half2 *)(o + r * pitch + i * plane) = out[i];
            }
            if (cvtile) {
                float f0[9], f1[9], t0[9], t1[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    f0[i] = g[i].x;
                    f1[i] = g[i].y;
                    const float2 w = __half22float2(out[i]);
                    t0[i] = w.x;
                    t1[i] = w.y;
                }
                cv_node<S, MOMENTUM_ONLY, FORCE>(a, x, y0 + r, f0, t0, 0, acc);
                cv_node<S, MOMENTUM_ONLY, FORCE>(a, x + 1, y0 + r, f1, t1, 0, acc);
            }
        } else if (cvtile) {
            float f0[9], f1[9], none[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                f0[i] = g[i].x;
                f1[i] = g[i].y;
                none[i] = 0.0f;
            }
            cv_node<S, MOMENTUM_ONLY, FORCE>(a, x, y0 + r, f0, none, 0, acc);
            cv_node<S, MOMENTUM_ONLY, FORCE>(a, x + 1, y0 + r, f1, none, 0, acc);
        }
    }
}

// ---------------------------------------------------------------------------
// One tile of TX x TR nodes with (TX/COLS) x (TR/RPT) threads (threadIdx.x:
// COLS adjacent columns, threadIdx.y: group of RPT rows).  `checked` selects the bounce-back-aware
// path (solid nodes in or next to the tile, or a pre-collision state).  A
// warp that met rho <= 0 or NaN sets status bit 0 and the first bad step.
// All threads of the block must call it: control-volume tiles synchronise the
// block, and the vote needs every lane of a warp.
// ---------------------------------------------------------------------------
template <int S, bool MOMENTUM_ONLY, bool FORCE, int TX, int TR, int RPT>
__device__ __forceinline__ void collide_tile(const StepArgs &a, int tx, int ty, bool checked)
{
    using A = typename AccOf<S>::type;
    constexpr int COLS = cols_per_thread(S);
    const int x = tx * TX + COLS * threadIdx.x;
    const bool cvtile = tx >= a.cvt[0] && tx <= a.cvt[1] && ty >= a.cvt[2] && ty <= a.cvt[3];
    A acc[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) acc_zero(acc[k]);
    bool bad = false;
    const int y0 = ty * TR + threadIdx.y * RPT;
    const bool interior = !checked && !a.periodic && ty > 0 && (ty + 1) * TR < a.ny;
    if constexpr (COLS == 2) {
        if (interior && x >= 1 && x + 1 <= a.nx - 2) {
            column_pair_update_interior<S, MOMENTUM_ONLY, RPT, FORCE>(a, x, y0, acc, cvtile, bad);
        } else {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                if (x + c >= a.nx) continue;
                if (interior)
                    column_update_interior<S, MOMENTUM_ONLY, RPT, FORCE>(a, x + c, y0, acc, cvtile, bad);
                else if (checked)
                    column_update<S, true, MOMENTUM_ONLY, RPT, FORCE>(a, x + c, y0, acc, cvtile, bad);
                else
                    column_update<S, false, MOMENTUM_ONLY, RPT, FORCE>(a, x + c, y0, acc, cvtile, bad);
            }
        }
    } else if (x < a.nx) {
        if (interior)
            column_update_interior<S, MOMENTUM_ONLY, RPT, FORCE>(a, x, y0, acc, cvtile, bad);
        else if (checked)
            column_update<S, true, MOMENTUM_ONLY, RPT, FORCE>(a, x, y0, acc, cvtile, bad);
        else
            column_update<S, false, MOMENTUM_ONLY, RPT, FORCE>(a, x, y0, acc, cvtile, bad);
    }
    if (cvtile) cv_store<S, MOMENTUM_ONLY, (TX / COLS) * (TR / RPT)>(a, tx, ty, acc);
    if (!MOMENTUM_ONLY) {
        // one vote per warp rather than per block: no barrier, so a warp that
        // is done leaves at once (the flags are idempotent: OR and MIN)
        const unsigned any_bad = __ballot_sync(0xffffffffu, bad);
        if (any_bad && ((threadIdx.y * blockDim.x + threadIdx.x) & 31) == 0) {
            atomicOr(a.status, 1);
            atomicMin(a.status + 1, (int)*a.step_ctr);
        }
    }
}

}  // namespace gblbm
