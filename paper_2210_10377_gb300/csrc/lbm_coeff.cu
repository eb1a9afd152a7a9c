// lbm_coeff.cu -- drag and lift coefficients of a window of the force series
// (Section V: C_d = 2 F_x / (rho0 U^2 L), C_l = 2 F_y / (rho0 U^2 L), signed,
// with L the chord (or the cylinder's diameter, Section VI) and U the inflow
// speed), per step and as the window's mean and standard deviation.
#include "lbm_internal.cuh"

namespace gblbm {
namespace {

constexpr int COEFF_THREADS = 256;

// Sum of one value per thread over the CTA, in a fixed tree order (the same
// bits for the same inputs on every run).
__device__ double cta_sum(double v, double *sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = COEFF_THREADS / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// One CTA.  Row `slot` of the series holds the force of one step at
// series[slot * row_stride + col] (x) and the next element (y); with wrap,
// only two rows are kept and step s sits in row s & 1.
// out: [0..3] = mean C_d, mean C_l, std C_d, std C_l (population standard
// deviation, two passes: mean first, then the squared deviations), then
// per-step C_d [count] and C_l [count] when per_step is set.
__global__ void __launch_bounds__(COEFF_THREADS)
k_coefficients(const double *__restrict__ series, long long row_stride, int col, long long first,
               long long count, int wrap, double norm, double *__restrict__ out, int per_step)
{
    __shared__ double sh[COEFF_THREADS];
    double sx = 0.0, sy = 0.0;
    for (long long k = threadIdx.x; k < count; k += COEFF_THREADS) {
        const long long step = first + k;
        const long long slot = wrap ? (step & 1) : step;
        // __dmul_rn: the same rounded product in both passes (never fused
        // with the subtraction of the second pass)
        const double cd = __dmul_rn(norm, series[slot * row_stride + col]);
        const double cl = __dmul_rn(norm, series[slot * row_stride + col + 1]);
        if (per_step) {
            out[4 + k] = cd;
            out[4 + count + k] = cl;
        }
        sx += cd;
        sy += cl;
    }
    const double mx = cta_sum(sx, sh) / (double)count;
    const double my = cta_sum(sy, sh) / (double)count;
    double vx = 0.0, vy = 0.0;
    for (long long k = threadIdx.x; k < count; k += COEFF_THREADS) {
        const long long step = first + k;
        const long long slot = wrap ? (step & 1) : step;
        const double dx = __dmul_rn(norm, series[slot * row_stride + col]) - mx;
        const double dy = __dmul_rn(norm, series[slot * row_stride + col + 1]) - my;
        vx += dx * dx;
        vy += dy * dy;
    }
    const double qx = cta_sum(vx, sh) / (double)count;
    const double qy = cta_sum(vy, sh) / (double)count;
    if (threadIdx.x == 0) {
        out[0] = mx;
        out[1] = my;
        out[2] = sqrt(qx);
        out[3] = sqrt(qy);
    }
}

}  // namespace

cudaError_t launch_coefficients(const double *series, long long row_stride, int col, long long first,
                                long long count, int wrap, double norm, double *out, bool per_step,
                                cudaStream_t st)
{
    k_coefficients<<<1, COEFF_THREADS, 0, st>>>(series, row_stride, col, first, count, wrap, norm, out,
                                                per_step ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace gblbm
