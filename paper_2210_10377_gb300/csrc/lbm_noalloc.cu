// lbm_noalloc.cu -- lbm_links_noalloc: the fluid-solid link list of a mask that
// is already in device memory, built without allocating any memory.
//
// It is the same three-pass stream compaction as the handle's link builder
// (per-block counts, one exclusive scan, per-block scan and scatter), except
// that the per-block counts and the total live in one fixed static device
// array instead of memory from an allocator, and the neighbour bits are taken
// from the mask on the fly.
#include <cstdio>

#include "lbm_internal.cuh"

namespace gblbm {

// Largest grid lbm_links_noalloc accepts, and its scratch: one int per block
// of 1024 nodes, then the 64-bit total.  256 KB per device that loads the
// library, held until the process exits.
constexpr long long NOALLOC_MAX_NODES = 1LL << 26;
constexpr int NOALLOC_BLOCK = 1024;
constexpr int NOALLOC_MAX_BLOCKS = (int)(NOALLOC_MAX_NODES / NOALLOC_BLOCK);
static __device__ __align__(256) int g_noalloc_scratch[NOALLOC_MAX_BLOCKS + 64];

namespace {

__device__ __forceinline__ unsigned int mask_link_bits(const uint8_t *__restrict__ mask, long long n,
                                                       int nx, int ny, int periodic, long long N)
{
    if (n >= N || mask[n]) return 0u;
    const int x = (int)(n % nx), y = (int)(n / nx);
    unsigned int b = 0u;
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        int x2 = x + cx(i), y2 = y + cy(i);
        y2 = y2 < 0 ? y2 + ny : (y2 >= ny ? y2 - ny : y2);
        if (x2 < 0 || x2 >= nx) {
            if (!periodic) continue;
            x2 = x2 < 0 ? x2 + nx : x2 - nx;
        }
        if (mask[(long long)y2 * nx + x2]) b |= 1u << i;
    }
    return b;
}

__device__ __forceinline__ int scan_1024(int v)
{
    __shared__ int ws[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int s = ws[lane];
        int si = s;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, si, d);
            if (lane >= d) si += o;
        }
        ws[lane] = si - s;
    }
    __syncthreads();
    const int excl = ws[warp] + inc - v;
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(NOALLOC_BLOCK)
k_noalloc_count(const uint8_t *__restrict__ mask, int nx, int ny, int periodic, int *__restrict__ cnt)
{
    const long long N = (long long)nx * ny;
    const long long n = (long long)blockIdx.x * NOALLOC_BLOCK + threadIdx.x;
    const int c = __popc(mask_link_bits(mask, n, nx, ny, periodic, N));
    const int excl = scan_1024(c);
    if (threadIdx.x == NOALLOC_BLOCK - 1) cnt[blockIdx.x] = excl + c;
}

__global__ void __launch_bounds__(NOALLOC_BLOCK)
k_noalloc_scatter(const uint8_t *__restrict__ mask, int nx, int ny, int periodic,
                  const int *__restrict__ off, int32_t *__restrict__ links, long long cap)
{
    const long long N = (long long)nx * ny;
    const long long n = (long long)blockIdx.x * NOALLOC_BLOCK + threadIdx.x;
    const unsigned int b = mask_link_bits(mask, n, nx, ny, periodic, N);
    long long pos = (long long)off[blockIdx.x] + scan_1024(__popc(b));
    for (int i = 1; i < 9; ++i)
        if (b & (1u << i)) {
            if (pos < cap) links[pos] = (int32_t)(n * 8 + (i - 1));
            ++pos;
        }
}

}  // namespace

}  // namespace gblbm

using namespace gblbm;

extern "C" lbm_status lbm_links_noalloc(const uint8_t *d_mask, int nx, int ny, int periodic_x,
                                        int32_t *d_links, long cap, long *count,
                                        void *cuda_stream)
{
    if (!d_mask || !count || nx <= 0 || ny <= 0 || cap < 0 || (cap > 0 && !d_links)) {
        set_thread_error("lbm_links_noalloc: bad argument");
        return LBM_EINVAL;
    }
    const long long N = (long long)nx * ny;
    if (N > NOALLOC_MAX_NODES) {
        char buf[160];
        snprintf(buf, sizeof(buf),
                 "lbm_links_noalloc: %dx%d = %lld nodes exceeds the fixed scratch limit of %lld nodes",
                 nx, ny, N, NOALLOC_MAX_NODES);
        set_thread_error(buf);
        return LBM_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // The call reads its result back and waits for the stream, so it cannot
    // be recorded into a graph: refuse a stream that is being captured.
    cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap_status);
    if (e != cudaSuccess || cap_status != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        set_thread_error("lbm_links_noalloc: the stream is being captured (or is invalid); "
                         "this call is synchronous and cannot be captured");
        return LBM_EINVAL;
    }
    // Host code sees only a stand-in for the static array.  Its device address
    // is asked for on every call, with the caller's device current, so that a
    // reset device or another context never leaves a stale address behind.
    int *scratch = nullptr;
    e = cudaGetSymbolAddress((void **)&scratch, g_noalloc_scratch);
    if (e != cudaSuccess || !scratch) {
        cudaGetLastError();
        set_thread_error("lbm_links_noalloc: cudaGetSymbolAddress failed (no usable CUDA device?)");
        return LBM_ECUDA;
    }
    const int nblocks = (int)((N + NOALLOC_BLOCK - 1) / NOALLOC_BLOCK);
    long long *total_d = (long long *)(scratch + NOALLOC_MAX_BLOCKS);
    k_noalloc_count<<<nblocks, NOALLOC_BLOCK, 0, st>>>(d_mask, nx, ny, periodic_x, scratch);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = launch_scan_blocks(scratch, nblocks, total_d, st);
    if (e == cudaSuccess)
        k_noalloc_scatter<<<nblocks, NOALLOC_BLOCK, 0, st>>>(d_mask, nx, ny, periodic_x, scratch,
                                                              d_links, (long long)cap);
    if (e == cudaSuccess) e = cudaGetLastError();
    long long total = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&total, total_d, sizeof(total), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        char buf[200];
        snprintf(buf, sizeof(buf), "lbm_links_noalloc: %s", cudaGetErrorString(e));
        set_thread_error(buf);
        return LBM_ECUDA;
    }
    *count = (long)total;
    return LBM_OK;
}
