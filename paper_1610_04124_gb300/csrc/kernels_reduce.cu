// kernels_reduce.cu -- column reduction and transpose (paper Sec. 5.1).
//
// Every stixel-width column of the H x W disparity map becomes one column of
// H Q4 codes: each pixel is clamped to [0, dmax] (NaN -> 0) and rounded to the
// 1/16-px grid, then the s codes of a row are reduced to their lower median
// (rank (s-1)/2; the median commutes with the monotone quantisation) or to
// their mean rounded half up (the paper's average).  On the whole-pixel grid
// (the paper's LUT_cost variant, Sec. 3.4) the reduced code is then rounded
// to the nearest multiple of 16, halves up.  The output is stored
// column-major and bottom-up (q[c * H + v], v = H-1-r) -- the layout the LUT
// and DP stages read.
//
// A 512-thread CTA reduces a tile of 32 columns x 16 rows, one output per
// thread: a warp reads 32 consecutive groups of s pixels of one row (32 s
// contiguous floats, so the warp's loads cover whole cache lines), the 32 x 16
// results are transposed through shared memory, and each half-warp then writes
// 16 consecutive bottom-up rows of one column (a contiguous 32-byte store).  The kernel moves 4 W H
// bytes in and 2 ncols H bytes out and is bandwidth / launch bound.
#include "internal.h"

namespace stx {
namespace {

__device__ __forceinline__ int q4_code(float d, int dmax)
{
    if (!(d > 0.0f)) return 0;               // NaN, negative, zero
    if (d >= (float)dmax) return 16 * dmax;
    return __float2int_rn(16.0f * d);        // 16 d is exact; halves to even
}

template <int S, int MODE>
__device__ __forceinline__ int reduce_q4(const float* __restrict__ px, int dmax)
{
    int v[S];
#pragma unroll
    for (int i = 0; i < S; ++i) v[i] = q4_code(__ldg(px + i), dmax);
    if (MODE == 1) {
        int sum = 0;
#pragma unroll
        for (int i = 0; i < S; ++i) sum += v[i];
        return (2 * sum + S) / (2 * S);      // mean, halves up
    }
    // lower median by rank selection: v[i] is the answer iff
    // #{v < v[i]} <= m < #{v <= v[i]}, m = (S-1)/2
    constexpr int m = (S - 1) / 2;
    int out = 0;
#pragma unroll
    for (int i = 0; i < S; ++i) {
        int lt = 0, le = 0;
#pragma unroll
        for (int j = 0; j < S; ++j) {
            lt += v[j] < v[i];
            le += v[j] <= v[i];
        }
        if (lt <= m && m < le) out = v[i];
    }
    return out;
}

// MODE bit 0: mean (else lower median); bit 1: round the result to whole pixels.
template <int S, int MODE>
__device__ __forceinline__ int reduce_group(const float* __restrict__ px, int dmax)
{
    const int r = reduce_q4<S, MODE & 1>(px, dmax);
    return (MODE & 2) ? ((r + 8) >> 4) << 4 : r;
}

template <int S, int MODE>
__global__ void __launch_bounds__(512) reduce_transpose_kernel(const float* __restrict__ disp, int H, int W,
                                                               int ncols, int dmax, int16_t* __restrict__ q)
{
    // the LUT kernel that follows may be scheduled now (it waits for these codes)
    grid_dependents_may_launch();
    __shared__ int16_t tile[32][18];                 // [column][row], padded
    const int tx = threadIdx.x, ty = threadIdx.y;    // 32 x 16
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 16;
    const int c = c0 + tx, r = r0 + ty;
    int val = 0;
    if (c < ncols && r < H) val = reduce_group<S, MODE>(disp + (size_t)r * W + (size_t)c * S, dmax);
    tile[tx][ty] = (int16_t)val;
    __syncthreads();
    // warp ty writes columns 2 ty and 2 ty + 1 of the tile: 16 bottom-up rows each
    const int cc = c0 + 2 * ty + (tx >> 4);
    const int rr = r0 + (tx & 15);
    if (cc < ncols && rr < H) q[(size_t)cc * H + (H - 1 - rr)] = tile[2 * ty + (tx >> 4)][tx & 15];
}

// Batch form: blockIdx.x indexes a list of (frame, column tile, row tile)
// items of frames that share stixel width S and reduction mode.
template <int S, int MODE>
__global__ void __launch_bounds__(512) reduce_transpose_batch_kernel(const ReduceArgs* __restrict__ frames,
                                                                     const int4* __restrict__ tiles)
{
    __shared__ int16_t tile[32][18];
    const int4 w = tiles[blockIdx.x];                // (frame, first column, first row, -)
    const ReduceArgs a = frames[w.x];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int c0 = w.y, r0 = w.z;
    const int c = c0 + tx, r = r0 + ty;
    int val = 0;
    if (c < a.ncols && r < a.H) val = reduce_group<S, MODE>(a.disp + (size_t)r * a.W + (size_t)c * S, a.dmax);
    tile[tx][ty] = (int16_t)val;
    __syncthreads();
    const int cc = c0 + 2 * ty + (tx >> 4);
    const int rr = r0 + (tx & 15);
    if (cc < a.ncols && rr < a.H) a.q[(size_t)cc * a.H + (a.H - 1 - rr)] = tile[2 * ty + (tx >> 4)][tx & 15];
}

template <int S>
cudaError_t launch_batch_s(const ReduceArgs* frames, const int4* tiles, int ntiles, int mode, cudaStream_t st)
{
    dim3 block(32, 16);
    switch (mode) {
        case 0: reduce_transpose_batch_kernel<S, 0><<<ntiles, block, 0, st>>>(frames, tiles); break;
        case 1: reduce_transpose_batch_kernel<S, 1><<<ntiles, block, 0, st>>>(frames, tiles); break;
        case 2: reduce_transpose_batch_kernel<S, 2><<<ntiles, block, 0, st>>>(frames, tiles); break;
        case 3: reduce_transpose_batch_kernel<S, 3><<<ntiles, block, 0, st>>>(frames, tiles); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int S>
cudaError_t launch_s(const float* disp, const FrameGeom& g, int dmax, int mode, int16_t* q, cudaStream_t st)
{
    dim3 block(32, 16), grid((g.ncols + 31) / 32, (g.H + 15) / 16);
    switch (mode) {
        case 0: reduce_transpose_kernel<S, 0><<<grid, block, 0, st>>>(disp, g.H, g.W, g.ncols, dmax, q); break;
        case 1: reduce_transpose_kernel<S, 1><<<grid, block, 0, st>>>(disp, g.H, g.W, g.ncols, dmax, q); break;
        case 2: reduce_transpose_kernel<S, 2><<<grid, block, 0, st>>>(disp, g.H, g.W, g.ncols, dmax, q); break;
        case 3: reduce_transpose_kernel<S, 3><<<grid, block, 0, st>>>(disp, g.H, g.W, g.ncols, dmax, q); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_reduce(const float* disp, const FrameGeom& g, int dmax, int mode, int16_t* q,
                          cudaStream_t st)
{
    if (g.H <= 0 || g.ncols <= 0) return cudaSuccess;
    switch (g.s) {
        case 1: return launch_s<1>(disp, g, dmax, mode, q, st);
        case 2: return launch_s<2>(disp, g, dmax, mode, q, st);
        case 3: return launch_s<3>(disp, g, dmax, mode, q, st);
        case 4: return launch_s<4>(disp, g, dmax, mode, q, st);
        case 5: return launch_s<5>(disp, g, dmax, mode, q, st);
        case 6: return launch_s<6>(disp, g, dmax, mode, q, st);
        case 7: return launch_s<7>(disp, g, dmax, mode, q, st);
        case 8: return launch_s<8>(disp, g, dmax, mode, q, st);
        case 9: return launch_s<9>(disp, g, dmax, mode, q, st);
        case 10: return launch_s<10>(disp, g, dmax, mode, q, st);
        case 11: return launch_s<11>(disp, g, dmax, mode, q, st);
        case 12: return launch_s<12>(disp, g, dmax, mode, q, st);
        case 13: return launch_s<13>(disp, g, dmax, mode, q, st);
        case 14: return launch_s<14>(disp, g, dmax, mode, q, st);
        case 15: return launch_s<15>(disp, g, dmax, mode, q, st);
        case 16: return launch_s<16>(disp, g, dmax, mode, q, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_reduce_batch(const ReduceArgs* d_frames, const int4* d_tiles, int ntiles, int s, int mode,
                                cudaStream_t st)
{
    if (ntiles <= 0) return cudaSuccess;
    switch (s) {
        case 1: return launch_batch_s<1>(d_frames, d_tiles, ntiles, mode, st);
        case 2: return launch_batch_s<2>(d_frames, d_tiles, ntiles, mode, st);
        case 3: return launch_batch_s<3>(d_frames, d_tiles, ntiles, mode, st);
        case 4: return launch_batch_s<4>(d_frames, d_tiles, ntiles, mode, st);
        case 5: return launch_batch_s<5>(d_frames, d_tiles, ntiles, mode, st);
        case 6: return launch_batch_s<6>(d_frames, d_tiles, ntiles, mode, st);
        case 7: return launch_batch_s<7>(d_frames, d_tiles, ntiles, mode, st);
        case 8: return launch_batch_s<8>(d_frames, d_tiles, ntiles, mode, st);
        case 9: return launch_batch_s<9>(d_frames, d_tiles, ntiles, mode, st);
        case 10: return launch_batch_s<10>(d_frames, d_tiles, ntiles, mode, st);
        case 11: return launch_batch_s<11>(d_frames, d_tiles, ntiles, mode, st);
        case 12: return launch_batch_s<12>(d_frames, d_tiles, ntiles, mode, st);
        case 13: return launch_batch_s<13>(d_frames, d_tiles, ntiles, mode, st);
        case 14: return launch_batch_s<14>(d_frames, d_tiles, ntiles, mode, st);
        case 15: return launch_batch_s<15>(d_frames, d_tiles, ntiles, mode, st);
        case 16: return launch_batch_s<16>(d_frames, d_tiles, ntiles, mode, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace stx
