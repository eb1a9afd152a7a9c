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
#include "lbm_device.cuh"

namespace gblbm {

struct AdjArgs {
    const void *src;       // [9][ny][pitch] storage type: ft(t-1) (f(t) itself when precollision)
    int precollision;
    const void *lam_next;  // [9][ny][pitch] compute type: lam(t+1)
    void *lam;             // [9][ny][pitch] compute type: lam(t)
    const uint16_t *nbits;
    const double *u_row;
    double *du_acc;        // [ny] running dJ/du_in
    double *dw_acc;        // [gridDim.x * gridDim.y] running per-block dJ/domega
    long long plane;
    int nx, ny, pitch;
    int in_window;
    double omega, rho0, obj_x, obj_y;  // obj = (2/M) (wx, wy)
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

template <int S>
__global__ void __launch_bounds__(256) k_adjoint_step(AdjArgs a)
{
    using T = typename Traits<S>::comp_t;
    constexpr bool DEV = Traits<S>::dev;
    const T *__restrict__ lamn = (const T *)a.lam_next;
    T *__restrict__ lam = (T *)a.lam;
    using ST = typename Traits<S>::store_t;
    const ST *__restrict__ src = (const ST *)a.src;
    using Acc = typename AccOf<S>::type;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    Acc dw;
    acc_zero(dw);
    if (x < a.nx) {
        const long long idx = (long long)y * a.pitch + x;
        const uint16_t nb = a.nbits[idx];
        if (nb & 1) {
#pragma unroll
            for (int i = 0; i < 9; ++i) lam[i * a.plane + idx] = T(0);
        } else {
            T lt[9];
            const int ym = y == 0 ? a.ny - 1 : y - 1, yp = y == a.ny - 1 ? 0 : y + 1;
#pragma unroll
            for (int j = 0; j < 9; ++j) {
                const int x2 = x + cx(j);
                const int y2 = cy(j) == 1 ? yp : (cy(j) == -1 ? ym : y);
                T v;
                if (x2 < 0 || x2 >= a.nx) {
                    v = T(0);
                } else if (j != 0 && (nb & (1u << j))) {
                    v = lam_fold(lamn, a.plane, a.pitch, a.nx, opp(j), x, y);
                    if (a.in_window) v += (T)(a.obj_x * cx(j) + a.obj_y * cy(j));
                } else {
                    v = lam_fold(lamn, a.plane, a.pitch, a.nx, j, x2, y2);
                }
                lt[j] = v;
            }
            if (x == 0) {  // inlet: ft = feq(rho0, (u_in(y), 0))
                const double u = a.u_row[y];
                double s = 0.0;
#pragma unroll
                for (int j = 0; j < 9; ++j)
                    s += (double)lt[j] * wgt<double>(j) * a.rho0 *
                         (3.0 * cx(j) + 9.0 * cx(j) * cx(j) * u - 3.0 * u);
                a.du_acc[y] += s;
#pragma unroll
                for (int i = 0; i < 9; ++i) lam[i * a.plane + idx] = T(0);
            } else {
                // f(t) of the step, pulled from the stored ft(t-1) of the
                // segment's recomputed forward: halfway bounce-back from the
                // node's own opposite population, and the outlet column
                // x = nx-1 taking the pull of column nx-2
                T g[9];
                if (a.precollision) {
#pragma unroll
                    for (int i = 0; i < 9; ++i) g[i] = to_comp(src[i * a.plane + idx]);
                } else {
                    const int xs = x == a.nx - 1 ? a.nx - 2 : x;
                    const long long sidx = (long long)y * a.pitch + xs;
                    const uint16_t nbs = xs == x ? nb : a.nbits[sidx];
#pragma unroll
                    for (int i = 0; i < 9; ++i) {
                        const int sy = cy(i) == 1 ? ym : (cy(i) == -1 ? yp : y);
                        g[i] = (nbs & (1u << opp(i)))
                                   ? to_comp(src[opp(i) * a.plane + sidx])
                                   : to_comp(src[i * a.plane + (long long)sy * a.pitch + (xs - cx(i))]);
                    }
                }
                const T R0 = DEV ? (T)a.rho0 : T(0);
                const T jx = ((g[1] - g[3]) + (g[5] - g[6])) + (g[8] - g[7]);
                const T jy = ((g[2] - g[4]) + (g[5] + g[6])) - (g[7] + g[8]);
                const T drho = (((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7]))) + g[8];
                const T rho = R0 + drho;
                const T inv = T(1) / rho;
                const T ux = jx * inv, uy = jy * inv;
                const T usq = ux * ux + uy * uy;
                const T om = (T)a.omega;
                T A = T(0), Bx = T(0), By = T(0), dwt = T(0);
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    const T cu = T(cx(i)) * ux + T(cy(i)) * uy;
                    const T w = wgt<T>(i);
                    const T feq = w * (drho + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq));
                    A += lt[i] * w * (T(1) - T(4.5) * cu * cu + T(1.5) * usq);
                    Bx += lt[i] * w * (T(3) * cx(i) + T(9) * cu * cx(i) - T(3) * ux);
                    By += lt[i] * w * (T(3) * cy(i) + T(9) * cu * cy(i) - T(3) * uy);
                    dwt += lt[i] * (feq - g[i]);
                }
#pragma unroll
                for (int k = 0; k < 9; ++k)
                    lam[k * a.plane + idx] = (T(1) - om) * lt[k] + om * (A + Bx * T(cx(k)) + By * T(cy(k)));
                dw = as_acc(dwt, Acc());
            }
        }
    }
    // per-block running sum of dJ/domega (fixed order: warp shuffles, then
    // warps); float-float below FP64 storage, so that the one-per-node part
    // of the sum stays off this GPU's few FP64 units
    __shared__ double ws[8];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc_add(dw, shfl_down(dw, d));
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc_double(dw);
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += ws[k];
        a.dw_acc[(long long)blockIdx.y * gridDim.x + blockIdx.x] += s;
    }
}

// Sum of n doubles in index order by one thread (the final reduction).
__global__ void k_sum_serial(const double *__restrict__ v, long long n, double *__restrict__ out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (long long k = 0; k < n; ++k) s += v[k];
    *out = s;
}

int adjoint_blocks(int nx, int ny) { return ((nx + 255) / 256) * ny; }

cudaError_t launch_adjoint_step(int storage, const void *src, int precollision, const void *lam_next, void *lam,
                                const uint16_t *nbits, const double *u_row, double *du_acc,
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
    a.obj_x = obj_x;
    a.obj_y = obj_y;
    dim3 grid((nx + 255) / 256, ny);
    switch (storage) {
    case LBM_F64: k_adjoint_step<LBM_F64><<<grid, 256, 0, st>>>(a); break;
    case LBM_F32: k_adjoint_step<LBM_F32><<<grid, 256, 0, st>>>(a); break;
    case LBM_F32_DEV: k_adjoint_step<LBM_F32_DEV><<<grid, 256, 0, st>>>(a); break;
    default: k_adjoint_step<LBM_F16_DEV><<<grid, 256, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_sum_serial(const double *v, long long n, double *out, cudaStream_t st)
{
    k_sum_serial<<<1, 32, 0, st>>>(v, n, out);
    return cudaGetLastError();
}

}  // namespace gblbm
