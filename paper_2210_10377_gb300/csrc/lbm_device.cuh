// lbm_device.cuh -- device helpers shared by the collide-stream and the link
// kernels: float-float (compensated FP32) sums, the per-storage accumulator
// type, warp and block reductions in a fixed order, and node momentum sums.
//
// For FP64 storage the accumulators are FP64; for FP32 and FP16 storage they
// are pairs of FP32 values (hi + lo, about 48 significant bits) built from
// error-free two-sums, so that the reductions stay off the FP64 units.
#pragma once

#include "lbm_internal.cuh"

namespace gblbm {

// ---- float-float arithmetic (error-free sums of FP32 values) ----
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ ff ff_addf(ff a, float b)
{
    const ff s = ff_two_sum(a.hi, b);
    return ff_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    const ff s = ff_two_sum(a.hi, b.hi);
    return ff_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ff operator-(ff a) { return {-a.hi, -a.lo}; }

// Accumulator per storage: FP64 for FP64 storage, float-float otherwise.
template <int S> struct AccOf {
    using type = ff;
};
template <> struct AccOf<LBM_F64> {
    using type = double;
};

__device__ __forceinline__ void acc_zero(double &a) { a = 0.0; }
__device__ __forceinline__ void acc_zero(ff &a) { a = {0.0f, 0.0f}; }
__device__ __forceinline__ void acc_add(double &a, double b) { a += b; }
__device__ __forceinline__ void acc_add(ff &a, ff b) { a = ff_add(a, b); }
__device__ __forceinline__ double acc_double(double a) { return a; }
__device__ __forceinline__ double acc_double(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double shfl_down(double v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double shfl_idx(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ ff shfl_idx(ff v, int src)
{
    return {__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}
__device__ __forceinline__ ff shfl_down(ff v, int d)
{
    return {__shfl_down_sync(0xffffffffu, v.hi, d), __shfl_down_sync(0xffffffffu, v.lo, d)};
}

// Signed sums of a node's populations: x-momentum f1 - f3 + f5 - f6 - f7 + f8,
// y-momentum f2 - f4 + f5 + f6 - f7 - f8.  Exact in float-float for FP32 values.
__device__ __forceinline__ double mom_x(const double *f)
{
    return ((f[1] - f[3]) + (f[5] - f[6])) + (f[8] - f[7]);
}
__device__ __forceinline__ double mom_y(const double *f)
{
    return ((f[2] - f[4]) + (f[5] + f[6])) - (f[7] + f[8]);
}
__device__ __forceinline__ ff mom_x(const float *f)
{
    ff s = ff_two_sum(f[1], -f[3]);
    s = ff_addf(s, f[5]);
    s = ff_addf(s, -f[6]);
    s = ff_addf(s, -f[7]);
    return ff_addf(s, f[8]);
}
__device__ __forceinline__ ff mom_y(const float *f)
{
    ff s = ff_two_sum(f[2], -f[4]);
    s = ff_addf(s, f[5]);
    s = ff_addf(s, f[6]);
    s = ff_addf(s, -f[7]);
    return ff_addf(s, -f[8]);
}
__device__ __forceinline__ double as_acc(double v, double) { return v; }
__device__ __forceinline__ ff as_acc(float v, ff) { return {v, 0.0f}; }

// Block reduction; the result is valid in thread 0.  NT threads, NT % 32 == 0.
template <typename A, int NV, int NT>
__device__ __forceinline__ void block_reduce(A (&v)[NV])
{
    __shared__ A sm[NT / 32][NV];
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) acc_add(v[k], shfl_down(v[k], d));
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sm[warp][k] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            if (lane < NT / 32)
                v[k] = sm[lane][k];
            else
                acc_zero(v[k]);
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1)
#pragma unroll
            for (int k = 0; k < NV; ++k) acc_add(v[k], shfl_down(v[k], d));
    }
    __syncthreads();
}

template <typename T> __device__ __forceinline__ T param(double d, float f);
template <> __device__ __forceinline__ double param<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float param<float>(double, float f) { return f; }

}  // namespace gblbm
