// lbm_setup.cu -- set-up kernels: body voxelisation, neighbour bits, the
// fluid-solid link list, tile flags and the initial equilibrium.
#include "lbm_internal.cuh"

namespace gblbm {

// ---------------------------------------------------------------------------
// NACA 4-digit symmetric section (the paper's NACA0012, Section V; the
// thickness law is the standard closed form, not printed in the paper).
// Every operation is an explicitly rounded FP64 intrinsic, in the order
//   xi  = ((dx*ca) - (dy*sa)) + (0.5*C)
//   eta = (dx*sa) + (dy*ca)
//   s   = xi / C
//   p   = ((((0.2969*sqrt(s)) - (0.1260*s)) - ((0.3516*s)*s)) + (((0.2843*s)*s)*s))
//         - ((((a4*s)*s)*s)*s)
//   y_t = ((5*t)*C)*p
// so that no contraction into fused multiply-adds changes the predicate.
// ---------------------------------------------------------------------------
__global__ void k_naca_mask(uint8_t *__restrict__ mask, int nx, int ny, double chord, double t,
                            double ca, double sa, double xc, double yc, double a4)
{
    long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (long long)nx * ny) return;
    int x = (int)(n % nx), y = (int)(n / nx);
    double dx = __dsub_rn((double)x, xc);
    double dy = __dsub_rn((double)y, yc);
    double xi = __dadd_rn(__dsub_rn(__dmul_rn(dx, ca), __dmul_rn(dy, sa)), __dmul_rn(0.5, chord));
    double eta = __dadd_rn(__dmul_rn(dx, sa), __dmul_rn(dy, ca));
    uint8_t solid = 0;
    if (xi >= 0.0 && xi <= chord) {
        double s = __ddiv_rn(xi, chord);
        double s2 = __dmul_rn(__dmul_rn(0.3516, s), s);
        double s3 = __dmul_rn(__dmul_rn(__dmul_rn(0.2843, s), s), s);
        double s4 = __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(a4, s), s), s), s);
        double p = __dsub_rn(__dmul_rn(0.2969, __dsqrt_rn(s)), __dmul_rn(0.1260, s));
        p = __dsub_rn(p, s2);
        p = __dadd_rn(p, s3);
        p = __dsub_rn(p, s4);
        double yt = __dmul_rn(__dmul_rn(__dmul_rn(5.0, t), chord), p);
        solid = fabs(eta) <= yt;
    }
    mask[n] = solid;
}

// Circular cylinder (Section VI): solid iff dx*dx + dy*dy <= r*r, with
// separately rounded FP64 operations in that order (no contraction), so the
// mask matches a plain C evaluation bit for bit.
__global__ void k_cylinder_mask(uint8_t *__restrict__ mask, int nx, int ny, double xc, double yc, double r2)
{
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= (long long)nx * ny) return;
    const int x = (int)(n % nx), y = (int)(n / nx);
    const double dx = __dsub_rn((double)x, xc);
    const double dy = __dsub_rn((double)y, yc);
    mask[n] = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= r2;
}

cudaError_t launch_cylinder_mask(uint8_t *mask, int nx, int ny, double xc, double yc, double radius,
                                 cudaStream_t st)
{
    const long long N = (long long)nx * ny;
    const int blocks = (int)((N + 255) / 256);
    k_cylinder_mask<<<blocks, 256, 0, st>>>(mask, nx, ny, xc, yc, radius * radius);
    return cudaGetLastError();
}

cudaError_t launch_naca_mask(uint8_t *mask, int nx, int ny, double chord, double thickness,
                             double ca, double sa, double xc, double yc, int closed_te,
                             cudaStream_t st)
{
    long long N = (long long)nx * ny;
    int blocks = (int)((N + 255) / 256);
    k_naca_mask<<<blocks, 256, 0, st>>>(mask, nx, ny, chord, thickness, ca, sa, xc, yc,
                                         closed_te ? 0.1036 : 0.1015);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Neighbour bits.  bit 0: node solid.  bit i: neighbour n + c_i solid, with y
// periodic and x periodic only for a periodic domain (a neighbour outside the
// channel in x is never solid).  Solid nodes keep only bit 0.
// ---------------------------------------------------------------------------
__global__ void k_node_bits(const uint8_t *__restrict__ mask, uint16_t *__restrict__ nbits,
                            int nx, int ny, int pitch, int periodic)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (x >= nx) return;
    uint16_t b;
    if (mask[(long long)y * nx + x]) {
        b = 1;
    } else {
        b = 0;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            int x2 = x + cx(i), y2 = y + cy(i);
            y2 = y2 < 0 ? y2 + ny : (y2 >= ny ? y2 - ny : y2);
            if (x2 < 0 || x2 >= nx) {
                if (!periodic) continue;
                x2 = x2 < 0 ? x2 + nx : x2 - nx;
            }
            if (mask[(long long)y2 * nx + x2]) b |= (uint16_t)(1u << i);
        }
    }
    nbits[(long long)y * pitch + x] = b;
}

cudaError_t launch_node_bits(const uint8_t *mask, uint16_t *nbits, int nx, int ny, int pitch,
                             int periodic, cudaStream_t st)
{
    dim3 grid((nx + 255) / 256, ny);
    k_node_bits<<<grid, 256, 0, st>>>(mask, nbits, nx, ny, pitch, periodic);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Link list by stream compaction over nodes in row-major order n = y*nx + x.
// A node's links are its set bits 1..8 taken in increasing direction, so the
// list comes out sorted without a sort.  Three passes, all deterministic:
// per-block counts, one exclusive scan of the block counts, then a per-block
// scan and scatter.
// ---------------------------------------------------------------------------
constexpr int LB = 1024;  // nodes (= threads) per link block

int link_blocks(int nx, int ny) { return (int)(((long long)nx * ny + LB - 1) / LB); }

__device__ __forceinline__ int node_links(const uint16_t *nbits, long long n, int nx, int pitch,
                                          long long N, uint16_t *bits)
{
    if (n >= N) {
        *bits = 0;
        return 0;
    }
    int x = (int)(n % nx), y = (int)(n / nx);
    uint16_t b = nbits[(long long)y * pitch + x];
    b = (b & 1) ? 0 : (uint16_t)(b & 0x1FE);
    *bits = b;
    return __popc(b);
}

// Block-wide exclusive scan of one int per thread (1024 threads = 32 warps).
__device__ __forceinline__ int block_exclusive_scan(int v)
{
    __shared__ int warp_sums[32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += o;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int s = warp_sums[lane];
        int si = s;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int o = __shfl_up_sync(0xffffffffu, si, d);
            if (lane >= d) si += o;
        }
        warp_sums[lane] = si - s;
    }
    __syncthreads();
    int excl = warp_sums[warp] + inc - v;
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(LB) k_link_count(const uint16_t *__restrict__ nbits, int nx,
                                                   int ny, int pitch, int *__restrict__ block_cnt)
{
    long long N = (long long)nx * ny;
    long long n = (long long)blockIdx.x * LB + threadIdx.x;
    uint16_t b;
    int c = node_links(nbits, n, nx, pitch, N, &b);
    // block sum by warp shuffles then one warp
    __shared__ int ws[32];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) c += __shfl_down_sync(0xffffffffu, c, d);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        int s = ws[threadIdx.x];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
        if (threadIdx.x == 0) block_cnt[blockIdx.x] = s;
    }
}

// Exclusive scan of nblocks counts in place by one CTA; total to *total.
__global__ void __launch_bounds__(LB) k_scan_blocks(int *__restrict__ cnt, int nblocks,
                                                    long long *__restrict__ total)
{
    __shared__ long long carry_s;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < nblocks; base += LB) {
        int i = base + threadIdx.x;
        int v = i < nblocks ? cnt[i] : 0;
        int excl = block_exclusive_scan(v);
        long long c = carry_s;
        if (i < nblocks) cnt[i] = (int)(c + excl);
        __syncthreads();
        if (threadIdx.x == LB - 1) carry_s = c + excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry_s;
}

__global__ void __launch_bounds__(LB) k_link_scatter(const uint16_t *__restrict__ nbits, int nx,
                                                     int ny, int pitch,
                                                     const int *__restrict__ block_off,
                                                     int32_t *__restrict__ links, long long cap)
{
    long long N = (long long)nx * ny;
    long long n = (long long)blockIdx.x * LB + threadIdx.x;
    uint16_t b;
    int c = node_links(nbits, n, nx, pitch, N, &b);
    int excl = block_exclusive_scan(c);
    long long pos = (long long)block_off[blockIdx.x] + excl;
    for (int i = 1; i < 9; ++i) {
        if (b & (1u << i)) {
            if (pos < cap) links[pos] = (int32_t)(n * 8 + (i - 1));
            ++pos;
        }
    }
}

cudaError_t launch_link_count(const uint16_t *nbits, int nx, int ny, int pitch, int *block_cnt,
                              int nblocks, cudaStream_t st)
{
    k_link_count<<<nblocks, LB, 0, st>>>(nbits, nx, ny, pitch, block_cnt);
    return cudaGetLastError();
}

cudaError_t launch_scan_blocks(int *block_cnt, int nblocks, long long *total, cudaStream_t st)
{
    k_scan_blocks<<<1, LB, 0, st>>>(block_cnt, nblocks, total);
    return cudaGetLastError();
}

cudaError_t launch_link_scatter(const uint16_t *nbits, int nx, int ny, int pitch,
                                const int *block_off, int32_t *links, long long cap,
                                cudaStream_t st)
{
    k_link_scatter<<<link_blocks(nx, ny), LB, 0, st>>>(nbits, nx, ny, pitch, block_off, links,
                                                        cap);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tile flags: a collide-stream tile needs the checked path when any node of
// the tile is solid or has a solid neighbour.  In a channel the outlet column
// collides the populations pulled for column nx-2, so that column's bits count
// for the tile holding the outlet too.
// ---------------------------------------------------------------------------
__global__ void k_tile_flags(const uint16_t *__restrict__ nbits, int nx, int ny, int pitch,
                             int periodic, uint8_t *__restrict__ flags, int tiles_x, int rows)
{
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int any = 0;
    for (int r = 0; r < rows; ++r) {
        int y = blockIdx.y * rows + r;
        if (x < nx && y < ny) {
            any |= nbits[(long long)y * pitch + x] != 0;
            if (!periodic && x == nx - 1) any |= nbits[(long long)y * pitch + nx - 2] != 0;
        }
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) flags[(long long)blockIdx.y * tiles_x + blockIdx.x] = (uint8_t)any;
}

cudaError_t launch_tile_flags(const uint16_t *nbits, int nx, int ny, int pitch, int periodic,
                              uint8_t *flags, int tiles_x, int tiles_y, int tw, int rows,
                              cudaStream_t st)
{
    dim3 grid(tiles_x, tiles_y);
    k_tile_flags<<<grid, tw, 0, st>>>(nbits, nx, ny, pitch, periodic, flags, tiles_x, rows);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Initial state f = feq(rho0, (u(y), 0)) (FP64, then rounded to storage; for
// deviation storage the base w_i rho0 is subtracted in FP64 first), and the
// inlet table of the same values.  Solid nodes hold 0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double feq_row(int i, double rho0, double u)
{
    double cu = cx(i) * u;
    return wgt<double>(i) * rho0 * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * u * u);
}

// Storage values next to v: the nearest (lo) and its neighbour on the other
// side of v (hi; equal to lo when v is representable).
__device__ void bracket(double v, float &lo, float &hi)
{
    lo = (float)v;
    if ((double)lo == v) {
        hi = lo;
        return;
    }
    hi = nextafterf(lo, (double)lo < v ? INFINITY : -INFINITY);
}
__device__ void bracket(double v, __half &lo, __half &hi)
{
    lo = __double2half(v);
    const double l = (double)__half2float(lo);
    if (l == v) {
        hi = lo;
        return;
    }
    // one step along the 16-bit pattern towards v
    unsigned short b = __half_as_ushort(lo);
    const bool up = l < v;
    if ((b & 0x7fff) == 0)
        b = up ? 0x0001 : 0x8001;
    else if (((b & 0x8000) == 0) == up)
        b = (unsigned short)(b + 1);
    else
        b = (unsigned short)(b - 1);
    hi = __ushort_as_half(b);
}
__device__ double as_double(float v) { return (double)v; }
__device__ double as_double(__half v) { return (double)__half2float(v); }

// The inlet state of each row, feq(rho0, (u_in(y), 0)) (less w_i rho0 for
// deviation storage), rounded to the storage type.  Rounding each value to
// nearest by itself changes the row's density and momentum by up to a few
// half-units in the last place of the storage type (for FP16 deviations about
// 2e-4 of rho0 u_in in the momentum, which the whole flow then carries).  So
// each value takes the nearer or the farther of its two bracketing storage
// values, whichever of the 2^9 choices keeps the mass and both momentum
// components closest to the exact ones (sum of squared errors; ties go to the
// choice nearer element by element).  FP64 storage stores the values as they are.
template <int S>
__global__ void k_inlet_rows(const double *__restrict__ u_row, double rho0, int ny, int rows,
                             typename Traits<S>::store_t *__restrict__ inlet)
{
    using ST = typename Traits<S>::store_t;
    // one warp per row of the first `rows` (the table's rows are ny apart);
    // lane l tries the choices l, l + 32, ... of the 2^9
    const int y = blockIdx.x * (blockDim.x / 32) + (int)(threadIdx.x / 32);
    const int lane = threadIdx.x & 31;
    if (y >= rows) return;
    const double u = u_row[y];
    double v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        v[i] = feq_row(i, rho0, u);
        if (Traits<S>::dev) v[i] -= wgt<double>(i) * rho0;
    }
    if constexpr (S == LBM_F64) {
        if (lane == 0)
#pragma unroll
            for (int i = 0; i < 9; ++i) inlet[i * ny + y] = v[i];
    } else {
        ST lo[9], hi[9];
        double dl[9], dh[9];
        for (int i = 0; i < 9; ++i) {
            bracket(v[i], lo[i], hi[i]);
            dl[i] = as_double(lo[i]) - v[i];
            dh[i] = as_double(hi[i]) - v[i];
        }
        unsigned best = 0;
        double best_e = INFINITY, best_a = INFINITY;
        for (unsigned c = lane; c < 512u; c += 32) {
            double dr = 0.0, jx = 0.0, jy = 0.0, ab = 0.0;
            for (int i = 0; i < 9; ++i) {
                const double d = (c >> i) & 1u ? dh[i] : dl[i];
                dr += d;
                jx += cx(i) * d;
                jy += cy(i) * d;
                ab += fabs(d);
            }
            const double e = dr * dr + jx * jx + jy * jy;
            if (e < best_e || (e == best_e && ab < best_a)) {
                best_e = e;
                best_a = ab;
                best = c;
            }
        }
        // the warp's best: least error, then least total rounding, then the
        // lowest choice index (the same winner as a serial search)
        for (int d = 16; d > 0; d >>= 1) {
            const double oe = __shfl_xor_sync(0xffffffffu, best_e, d);
            const double oa = __shfl_xor_sync(0xffffffffu, best_a, d);
            const unsigned oc = __shfl_xor_sync(0xffffffffu, best, d);
            if (oe < best_e || (oe == best_e && (oa < best_a || (oa == best_a && oc < best)))) {
                best_e = oe;
                best_a = oa;
                best = oc;
            }
        }
        if (lane == 0)
            for (int i = 0; i < 9; ++i) inlet[i * ny + y] = (best >> i) & 1u ? hi[i] : lo[i];
    }
}

// Initial state: every fluid node of row y holds the row's inlet state.  With
// a uniform inlet only row 0 of the table was computed: every row reads it,
// and the thread at x = 0 of each other row copies it into its own row (no
// thread writes row 0, so no read meets a write).
template <int S>
__global__ void k_init(typename Traits<S>::store_t *__restrict__ pop, long long plane,
                       const uint8_t *__restrict__ mask, int nx, int ny, int pitch,
                       typename Traits<S>::store_t *__restrict__ inlet, int uniform)
{
    using ST = typename Traits<S>::store_t;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (x >= nx) return;
    const int ys = uniform ? 0 : y;
    bool solid = mask[(long long)y * nx + x] != 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const ST v = inlet[i * ny + ys];
        pop[i * plane + (long long)y * pitch + x] = solid ? to_store<ST>((typename Traits<S>::comp_t)0) : v;
        if (uniform && x == 0 && y > 0) inlet[i * ny + y] = v;
    }
}

cudaError_t launch_init(int storage, void *pop, long long plane, const uint8_t *mask, int nx,
                        int ny, int pitch, const double *u_row, double rho0, void *inlet,
                        cudaStream_t st, int uniform)
{
    dim3 grid((nx + 255) / 256, ny);
    const int rows = uniform ? 1 : ny;  // a uniform inlet has one distinct row
    const int rb = (rows + 3) / 4;      // four rows (warps) a block
    switch (storage) {
    case LBM_F64:
        k_inlet_rows<LBM_F64><<<rb, 128, 0, st>>>(u_row, rho0, ny, rows, (double *)inlet);
        k_init<LBM_F64><<<grid, 256, 0, st>>>((double *)pop, plane, mask, nx, ny, pitch, (double *)inlet, uniform);
        break;
    case LBM_F32:
        k_inlet_rows<LBM_F32><<<rb, 128, 0, st>>>(u_row, rho0, ny, rows, (float *)inlet);
        k_init<LBM_F32><<<grid, 256, 0, st>>>((float *)pop, plane, mask, nx, ny, pitch, (float *)inlet, uniform);
        break;
    case LBM_F32_DEV:
        k_inlet_rows<LBM_F32_DEV><<<rb, 128, 0, st>>>(u_row, rho0, ny, rows, (float *)inlet);
        k_init<LBM_F32_DEV><<<grid, 256, 0, st>>>((float *)pop, plane, mask, nx, ny, pitch, (float *)inlet, uniform);
        break;
    default:
        k_inlet_rows<LBM_F16_DEV><<<rb, 128, 0, st>>>(u_row, rho0, ny, rows, (__half *)inlet);
        k_init<LBM_F16_DEV><<<grid, 256, 0, st>>>((__half *)pop, plane, mask, nx, ny, pitch, (__half *)inlet,
                                                   uniform);
        break;
    }
    return cudaGetLastError();
}

}  // namespace gblbm
