// lbm_adjoint.cu -- discrete adjoint of the channel step, for gradients of the
// window-averaged algorithm-B force (Eq. rtt5 with bounce-back)
//   J = (1/M) sum_{t in window} (wx Fx(t) + wy Fy(t)),  F(t) = 2 sum_links c_i ft_i(x_f, t),
// with respect to the relaxation time, the inlet velocity of every row and the
// pre-collision state at the start.
//
// With lt = dJ/d(ft(t)) and lam = dJ/d(f(t)), one backward step is
//   lt_j(y) = L_j(y + c_j)      if y + c_j is a fluid node in the domain,
//           = L_opp(j)(y)       if y + c_j is solid (halfway bounce-back),
//           + (2/M)(wx c_jx + wy c_jy) on links inside the window,
//   L = lam(t+1) with the inlet and outlet columns zero and the outlet column
//   added to column nx-2 (the outlet copies it);
//   lam_k(y) = (1 - w) lt_k + w (A + B . c_k),  w = 1/tau,
//   A = sum_i lt_i dfeq_i/drho = sum_i lt_i w_i (1 - 4.5 (c_i.u)^2 + 1.5 u^2),
//   B = sum_i lt_i dfeq_i/dj   = sum_i lt_i w_i (3 c_i + 9 (c_i.u) c_i - 3 u),
//   dJ/dw += sum_i lt_i (feq_i - f_i);  at the inlet, where ft = feq(rho0, u_in(y)),
//   dJ/du_in(y) += sum_i lt_i rho0 w_i (3 c_ix + 9 c_ix^2 u - 3 u) and lam = 0.
// (feq here is the second-order equilibrium of Section II written in rho and
// j = rho u; BGK: ft = f + w (feq - f).)
#include "lbm_collide.cuh"

namespace gblbm {

struct AdjArgs {
    const void *src;       // [9][ny][pitch] storage type: ft(t-1) (f(t) itself when precollision)
    int precollision;
    const void *lam_next;  // [9][ny][pitch] compute type: lam(t+1)
    void *lam;             // [9][ny][pitch] compute type: lam(t)
    const uint16_t *nbits;
    const uint8_t *tile_flag;  // per tile of the grid: 0 = every node's bits are 0 (or NULL)
    const double *u_row;
    double *du_acc;        // [ny] running dJ/du_in
    double *dw_acc;        // [blocks * ADJ_WARPS] running per-warp dJ/domega: FP64, or a
                           // float-float pair in the same 8 bytes below FP64 storage
    long long plane;
    int nx, ny, pitch;
    int in_window;
    double omega, rho0;
    float omega_f, rho0_f;
    double obj[9];         // (2/M)(wx c_ix + wy c_iy): the objective's source on a link of direction i
    float obj_f[9];        // the same rounded to FP32
    int pf_rows;           // L2 prefetch distance in tile rows (0: off)
};

template <typename T>
__device__ __forceinline__ T lam_fold(const T *__restrict__ lam, long long plane, int pitch, int nx,
                                      int i, int x, int y)
{
    // L = lam(t+1) with inlet/outlet columns zero, outlet added to column nx-2
    if (x == 0 || x == nx - 1) return T(0);
    const long long idx = (long long)y * pitch + x;
    T v = lam[i * plane + idx];
    if (x == nx - 2) v += lam[i * plane + idx + 1];
    return v;
}

// Tiles of the backward step: 128 nodes along x by ADJ_TR rows, ADJ_RPT rows
// a thread (all loads of a thread issued before its arithmetic).
constexpr int ADJ_TX = 128, ADJ_TR = 4, ADJ_RPT = 2;
constexpr int ADJ_THREADS = ADJ_TX * (ADJ_TR / ADJ_RPT);
constexpr int ADJ_WARPS = ADJ_THREADS / 32;

// Minimum resident CTAs per SM asked of the compiler (a tuning knob: 4 CTAs
// of 256 threads, 64 registers, measured fastest of 0, 3 and 4).
#ifndef GBLBM_ADJ_MINB
#define GBLBM_ADJ_MINB 4
#endif

// The inputs of one node of the backward step: lt = lambda(t+1) gathered
// along the transposed streaming (L = lambda(t+1) folded at the outlet, bounce-
// back on links, the objective's source on links inside the window) and the
// pre-collision f(t) pulled from the stored ft(t-1).  Returns false for solid
// nodes and the inlet column (whose results need no collision Jacobian).
template <int S>
__device__ __forceinline__ bool adj_node_inputs(const AdjArgs &a, int x, int y, uint16_t nb,
                                                typename Traits<S>::comp_t (&lt)[9],
                                                typename Traits<S>::comp_t (&g)[9])
{
    using T = typename Traits<S>::comp_t;
    using ST = typename Traits<S>::store_t;
    const T *__restrict__ lamn = (const T *)a.lam_next;
    const ST *__restrict__ src = (const ST *)a.src;
    const long long plane = a.plane, pitch = a.pitch;
    const long long idx = (long long)y * pitch + x;
    const int ym = y == 0 ? a.ny - 1 : y - 1, yp = y == a.ny - 1 ? 0 : y + 1;
    if (nb & 1) return false;
    // a node away from solids, the inlet and the outlet (and their neighbour
    // columns), in a pulled state: every load is a plain shift
    if (!a.precollision && nb == 0 && x >= 2 && x <= a.nx - 4) {
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const int y2 = cy(j) == 1 ? yp : (cy(j) == -1 ? ym : y);
            lt[j] = lamn[j * plane + (long long)y2 * pitch + x + cx(j)];
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int sy = cy(i) == 1 ? ym : (cy(i) == -1 ? yp : y);
            g[i] = to_comp(src[i * plane + (long long)sy * pitch + x - cx(i)]);
        }
        return true;
    }
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        const int x2 = x + cx(j);
        const int y2 = cy(j) == 1 ? yp : (cy(j) == -1 ? ym : y);
        T v;
        if (x2 < 0 || x2 >= a.nx) {
            v = T(0);
        } else if (j != 0 && (nb & (1u << j))) {
            v = lam_fold(lamn, plane, a.pitch, a.nx, opp(j), x, y);
            if (a.in_window) v += param<T>(a.obj[j], a.obj_f[j]);
        } else {
            v = lam_fold(lamn, plane, a.pitch, a.nx, j, x2, y2);
        }
        lt[j] = v;
    }
    if (x == 0) return false;
    if (a.precollision) {
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = to_comp(src[i * plane + idx]);
        return true;
    }
    // halfway bounce-back from the node's own opposite population, and the
    // outlet column x = nx-1 taking the pull of column nx-2
    const int xs = x == a.nx - 1 ? a.nx - 2 : x;
    const long long sidx = (long long)y * pitch + xs;
    const uint16_t nbs = xs == x ? nb : a.nbits[sidx];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const int sy = cy(i) == 1 ? ym : (cy(i) == -1 ? yp : y);
        g[i] = (nbs & (1u << opp(i))) ? to_comp(src[opp(i) * plane + sidx])
                                      : to_comp(src[i * plane + (long long)sy * pitch + (xs - cx(i))]);
    }
    return true;
}

// One node's lambda(t) and its dJ/domega term from lt and f(t).
template <int S>
__device__ __forceinline__ typename Traits<S>::comp_t adj_node(const AdjArgs &a, long long idx,
                                                               const typename Traits<S>::comp_t (&lt)[9],
                                                               const typename Traits<S>::comp_t (&g)[9])
{
    using T = typename Traits<S>::comp_t;
    constexpr bool DEV = Traits<S>::dev;
    T *__restrict__ lam = (T *)a.lam;
    const T R0 = DEV ? param<T>(a.rho0, a.rho0_f) : T(0);
    const T jx = ((g[1] - g[3]) + (g[5] - g[6])) + (g[8] - g[7]);
    const T jy = ((g[2] - g[4]) + (g[5] + g[6])) - (g[7] + g[8]);
    const T drho = (((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7]))) + g[8];
    const T rho = R0 + drho;
    const T inv = T(1) / rho;
    const T ux = jx * inv, uy = jy * inv;
    const T usq = ux * ux + uy * uy;
    const T om = param<T>(a.omega, a.omega_f);
    // weighted moments of lt: L0 = sum w lt, L_a = sum w lt c_a,
    // L_ab = sum w lt c_a c_b; with them, for cu = c.u,
    //   sum w lt cu = ux Lx + uy Ly,  sum w lt cu^2 = ux^2 Lxx + 2 ux uy Lxy + uy^2 Lyy,
    // so that A, B and sum lt feq take a few operations each
    const T w1 = wgt<T>(1), w5 = wgt<T>(5);
    const T d13 = lt[1] - lt[3], d24 = lt[2] - lt[4], s13 = lt[1] + lt[3], s24 = lt[2] + lt[4];
    const T sd = (lt[5] + lt[6]) + (lt[7] + lt[8]);
    const T L0 = wgt<T>(0) * lt[0] + w1 * (s13 + s24) + w5 * sd;
    const T Lx = w1 * d13 + w5 * ((lt[5] - lt[6]) + (lt[8] - lt[7]));
    const T Ly = w1 * d24 + w5 * ((lt[5] + lt[6]) - (lt[7] + lt[8]));
    const T Lxx = w1 * s13 + w5 * sd, Lyy = w1 * s24 + w5 * sd;
    const T Lxy = w5 * ((lt[5] - lt[6]) + (lt[7] - lt[8]));
    const T P = ux * Lx + uy * Ly;
    const T Q = ux * ux * Lxx + T(2) * ux * uy * Lxy + uy * uy * Lyy;
    // A = sum lt dfeq/drho, B = sum lt dfeq/dj (per unit rho)
    const T A = L0 - T(4.5) * Q + T(1.5) * usq * L0;
    const T Bx = T(3) * Lx + T(9) * (ux * Lxx + uy * Lxy) - T(3) * ux * L0;
    const T By = T(3) * Ly + T(9) * (ux * Lxy + uy * Lyy) - T(3) * uy * L0;
#pragma unroll
    for (int k = 0; k < 9; ++k)
        lam[k * a.plane + idx] = (T(1) - om) * lt[k] + om * (A + Bx * T(cx(k)) + By * T(cy(k)));
    // sum lt (feq - f), feq less its base for deviation storage
    T lg = T(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) lg += lt[i] * g[i];
    return (drho * L0 + rho * (T(3) * P + T(4.5) * Q - T(1.5) * usq * L0)) - lg;
}

// Asks L2 for the rows of the tile a.pf_rows tile rows further down (as the
// forward kernel does): the state rows y0-1 .. y0+TR and the lambda(t+1) rows
// y0-1 .. y0+TR of all nine planes, one bulk prefetch per plane and row, each
// inside its buffer (row in [0, ny), columns x0 .. min(x0 + 128, pitch) - 1)
// and on a 16-byte boundary (pitch is a multiple of 64 elements).
template <int S>
__device__ __forceinline__ void adj_prefetch(const AdjArgs &a)
{
    using T = typename Traits<S>::comp_t;
    using ST = typename Traits<S>::store_t;
    constexpr int ROWS = ADJ_TR + 2;
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
    const int ty = (int)blockIdx.y + a.pf_rows;
    if (a.pf_rows <= 0 || t >= 2 * 9 * ROWS || ty >= (int)gridDim.y) return;
    const int which = t / (9 * ROWS), k = t % (9 * ROWS);
    int y = ty * ADJ_TR - 1 + k % ROWS;
    y = y < 0 ? y + a.ny : (y >= a.ny ? y - a.ny : y);
    const int i = k / ROWS;
    const int x0 = (int)blockIdx.x * ADJ_TX;
    const int ncol = min(ADJ_TX, a.pitch - x0);
    if (which == 0)
        prefetch_l2((const ST *)a.src + (long long)i * a.plane + (long long)y * a.pitch + x0,
                    (unsigned)(ncol * sizeof(ST)));
    else
        prefetch_l2((const T *)a.lam_next + (long long)i * a.plane + (long long)y * a.pitch + x0,
                    (unsigned)(ncol * sizeof(T)));
}

template <int S>
__global__ void __launch_bounds__(ADJ_THREADS, GBLBM_ADJ_MINB) k_adjoint_step(AdjArgs a)
{
    using T = typename Traits<S>::comp_t;
    using Acc = typename AccOf<S>::type;
    T *__restrict__ lam = (T *)a.lam;
    adj_prefetch<S>(a);
    const int x = blockIdx.x * ADJ_TX + threadIdx.x;
    const int y0 = blockIdx.y * ADJ_TR + threadIdx.y * ADJ_RPT;
    // a tile whose nodes all have zero bits (no solid in or next to it) skips
    // the per-node bit loads, so its population loads start at once
    const bool plain_tile =
        a.tile_flag && !a.precollision && a.tile_flag[(long long)blockIdx.y * gridDim.x + blockIdx.x] == 0;
    Acc dw;
    acc_zero(dw);
    if (x < a.nx) {
        T lt[ADJ_RPT][9], g[ADJ_RPT][9];
        bool live[ADJ_RPT];
        uint16_t nb[ADJ_RPT];
#pragma unroll
        for (int r = 0; r < ADJ_RPT; ++r) {
            const int y = y0 + r;
            nb[r] = (plain_tile || y >= a.ny) ? (uint16_t)0 : a.nbits[(long long)y * a.pitch + x];
        }
#pragma unroll
        for (int r = 0; r < ADJ_RPT; ++r) {
            const int y = y0 + r;
            live[r] = false;
            if (y >= a.ny) continue;
            live[r] = adj_node_inputs<S>(a, x, y, nb[r], lt[r], g[r]);
        }
#pragma unroll
        for (int r = 0; r < ADJ_RPT; ++r) {
            const int y = y0 + r;
            if (y >= a.ny) continue;
            const long long idx = (long long)y * a.pitch + x;
            if (live[r]) {
                acc_add(dw, as_acc(adj_node<S>(a, idx, lt[r], g[r]), Acc()));
            } else {
                if (x == 0 && !(nb[r] & 1)) {  // inlet: ft = feq(rho0, (u_in(y), 0))
                    // in the compute type: FP64 instructions are slow on this
                    // GPU even with one lane active, and this warp's siblings wait
                    const T u = (T)a.u_row[y];
                    const T r0 = param<T>(a.rho0, a.rho0_f);
                    T s = T(0);
#pragma unroll
                    for (int j = 0; j < 9; ++j)
                        s += lt[r][j] * wgt<T>(j) * r0 * (T(3 * cx(j)) + T(9 * cx(j) * cx(j)) * u - T(3) * u);
                    a.du_acc[y] += (double)s;
                }
#pragma unroll
                for (int i = 0; i < 9; ++i) lam[i * a.plane + idx] = T(0);
            }
        }
    }
    // running sums of dJ/domega, one slot per warp (fixed order within the
    // warp; float-float below FP64 storage, the running slot included, so
    // that no FP64 instruction runs per step, and no barrier between warps)
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc_add(dw, shfl_down(dw, d));
    const int warp = (threadIdx.y * blockDim.x + threadIdx.x) >> 5;
    if ((threadIdx.x & 31) == 0) {
        Acc *slot = (Acc *)a.dw_acc + ((long long)blockIdx.y * gridDim.x + blockIdx.x) * ADJ_WARPS + warp;
        acc_add(*slot, dw);
    }
}

// Sum of n doubles in a fixed order (the final reduction): thread t of one
// CTA adds slots t, t + 256, ... in turn, then the CTA's tree.
template <typename A>
__global__ void __launch_bounds__(256) k_sum_fixed(const A *__restrict__ v, long long n, double *__restrict__ out)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (long long k = threadIdx.x; k < n; k += 256) s += acc_double(v[k]);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int d = 128; d > 0; d >>= 1) {
        if ((int)threadIdx.x < d) sh[threadIdx.x] += sh[threadIdx.x + d];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// slots of the per-warp dJ/domega sums
int adjoint_blocks(int nx, int ny)
{
    return ((nx + ADJ_TX - 1) / ADJ_TX) * ((ny + ADJ_TR - 1) / ADJ_TR) * ADJ_WARPS;
}

cudaError_t launch_adjoint_step(int storage, const void *src, int precollision, const void *lam_next, void *lam,
                                const uint16_t *nbits, const uint8_t *tile_flag, int flag_rows, int flag_tiles_x,
                                const double *u_row, double *du_acc,
                                double *dw_acc, long long plane, int nx, int ny, int pitch,
                                int in_window, double omega, double rho0, double obj_x,
                                double obj_y, cudaStream_t st)
{
    AdjArgs a;
    a.src = src;
    a.precollision = precollision;
    a.lam_next = lam_next;
    a.lam = lam;
    a.nbits = nbits;
    a.u_row = u_row;
    a.du_acc = du_acc;
    a.dw_acc = dw_acc;
    a.plane = plane;
    a.nx = nx;
    a.ny = ny;
    a.pitch = pitch;
    a.in_window = in_window;
    a.omega = omega;
    a.rho0 = rho0;
    a.omega_f = (float)omega;
    a.rho0_f = (float)rho0;
    for (int i = 0; i < 9; ++i) {
        a.obj[i] = obj_x * cx(i) + obj_y * cy(i);
        a.obj_f[i] = (float)a.obj[i];
    }
    dim3 grid((nx + ADJ_TX - 1) / ADJ_TX, (ny + ADJ_TR - 1) / ADJ_TR);
    dim3 block(ADJ_TX, ADJ_TR / ADJ_RPT);
    // the collide-stream tile flags serve when their tiles are these tiles
    a.tile_flag = (tile_flag && TILE_X == ADJ_TX && flag_rows == ADJ_TR && flag_tiles_x == (int)grid.x) ? tile_flag
                                                                                                        : nullptr;
    // prefetch half the CTAs the GPU holds at once ahead, in tile rows
    int pf_rows = 0;
    if (storage != LBM_F64) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const void *fn = storage == LBM_F32 ? (const void *)k_adjoint_step<LBM_F32>
                         : storage == LBM_F32_DEV ? (const void *)k_adjoint_step<LBM_F32_DEV>
                                                  : (const void *)k_adjoint_step<LBM_F16_DEV>;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, ADJ_THREADS, 0) == cudaSuccess && sms > 0)
            pf_rows = (int)(((long long)per_sm * sms / 2 + grid.x / 2) / grid.x);
        cudaGetLastError();
        if (pf_rows < 1) pf_rows = 1;
    }
    a.pf_rows = pf_rows;
    switch (storage) {
    case LBM_F64: k_adjoint_step<LBM_F64><<<grid, block, 0, st>>>(a); break;
    case LBM_F32: k_adjoint_step<LBM_F32><<<grid, block, 0, st>>>(a); break;
    case LBM_F32_DEV: k_adjoint_step<LBM_F32_DEV><<<grid, block, 0, st>>>(a); break;
    default: k_adjoint_step<LBM_F16_DEV><<<grid, block, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_sum_fixed(const double *v, long long n, double *out, bool ff_slots, cudaStream_t st)
{
    if (ff_slots)
        k_sum_fixed<ff><<<1, 256, 0, st>>>((const ff *)v, n, out);
    else
        k_sum_fixed<double><<<1, 256, 0, st>>>(v, n, out);
    return cudaGetLastError();
}

// dJ/df(x, T0) = lambda(T0) in FP64, [9][ny][nx] without the row pitch: zero on
// solid nodes and in the inlet column, which do not enter J.  One thread per
// (direction, node); the conversion from FP32 is exact.
template <typename C>
__global__ void __launch_bounds__(256) k_adjoint_df0(const C *__restrict__ lam, const uint8_t *__restrict__ mask,
                                                     long long plane, int nx, int ny, int pitch,
                                                     double *__restrict__ out)
{
    const long long n = (long long)nx * ny;
    for (long long k = blockIdx.x * 256LL + threadIdx.x; k < 9 * n; k += (long long)gridDim.x * 256) {
        const int i = (int)(k / n);
        const long long node = k - i * n;
        const int y = (int)(node / nx), x = (int)(node - (long long)y * nx);
        const double v = (double)lam[i * plane + (long long)y * pitch + x];
        out[k] = (mask[node] || x == 0) ? 0.0 : v;
    }
}

cudaError_t launch_adjoint_df0(int storage, const void *lam, const uint8_t *mask, long long plane, int nx, int ny,
                               int pitch, int sm_count, double *out, cudaStream_t st)
{
    const long long total = 9LL * nx * ny;
    long long blocks = (total + 255) / 256;
    const long long cap = 8LL * (sm_count > 0 ? sm_count : 1);
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (storage == LBM_F64)
        k_adjoint_df0<double><<<(int)blocks, 256, 0, st>>>((const double *)lam, mask, plane, nx, ny, pitch, out);
    else
        k_adjoint_df0<float><<<(int)blocks, 256, 0, st>>>((const float *)lam, mask, plane, nx, ny, pitch, out);
    return cudaGetLastError();
}

}  // namespace gblbm
