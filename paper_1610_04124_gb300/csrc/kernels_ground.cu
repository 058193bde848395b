// kernels_ground.cu -- the frame's ground line from its v-disparity (the step
// before the path: the paper takes the ground slope and horizon as known for
// every image, Sec. 3).
//
// On the 1/16-px grid of the reduced codes (image row r = H-1-v):
//   hist[r][e]  columns whose code at row r is e, for e in [16, 16 dmax]
//               (codes below 1 px -- sky, invalid pixels -- carry no ground);
//   S[r][e]     sum over |t| <= 16 of (17 - |t|) hist[r][e + t], a triangular
//               kernel of half-width 1 px so that noisy ground still votes;
//   line (k, h) code (k (r - h) + 8) >> 4 at rows r > h: slope k / 256 px of
//               disparity per image row (k = 1..256), horizon at image row h;
//   votes(k, h) sum of S[r][code] over the rows r > h with code in [16, 16 dmax];
// the line with the most votes wins, ties to the smaller k, then the smaller h.
// Its codes (rounded half away from zero above the horizon) replace the
// camera's ground line for the frame, and the ground K of each row comes from
// a table over the clamped code built at create time.  With no vote at all
// the camera's line is kept.
//
// Kernels: one CTA per image row builds and smooths its histogram in shared
// memory; one thread per (k, h) sums its votes, 16 rows' loads at a time (the
// smoothed rows are read from L1 / L2 -- neighbouring k read neighbouring
// codes) and a 64-bit
// atomic max over (votes, 256 - k, 65535 - h) picks the winner whatever the
// order; one CTA then writes the frame's row tables.
#include "internal.h"

namespace stx {
namespace {

// per image row: histogram of the codes, smoothed
__global__ void __launch_bounds__(256) vdisp_kernel(const int16_t* __restrict__ q, int H, int ncols, int dmax,
                                                    int32_t* __restrict__ smooth)
{
    extern __shared__ int32_t s_h[];               // [E]
    const int E = 16 * dmax + 1;
    const int r = blockIdx.x, v = H - 1 - r;
    for (int e = threadIdx.x; e < E; e += blockDim.x) s_h[e] = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
        const int code = q[(size_t)c * H + v];
        if (code >= 16 && code < E) atomicAdd(&s_h[code], 1);
    }
    __syncthreads();
    int32_t* out = smooth + (size_t)r * E;
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        int32_t acc = 0;
        if (e >= 16)
            for (int t = -16; t <= 16; ++t) {
                const int x = e + t;
                if (x >= 16 && x < E) acc += (17 - abs(t)) * s_h[x];
            }
        out[e] = acc;
    }
}

// one thread per candidate: k = threadIdx.x + 1, h = blockIdx.x
__global__ void __launch_bounds__(256) vote_kernel(const int32_t* __restrict__ smooth, int H, int dmax,
                                                   unsigned long long* __restrict__ best)
{
    const int E = 16 * dmax + 1;
    const int k = threadIdx.x + 1, h = blockIdx.x;
    int32_t votes = 0;
    // rows in chunks of 16 independent loads (the codes grow with r, so the
    // first chunk that starts beyond the table ends the line)
    for (int r0 = h + 1; r0 < H; r0 += 16) {
        if (((k * (r0 - h) + 8) >> 4) >= E) break;
        int32_t part[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int r = r0 + i;
            const int code = (k * (r - h) + 8) >> 4;
            part[i] = (r < H && code >= 16 && code < E) ? __ldg(smooth + (size_t)r * E + code) : 0;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) votes += part[i];
    }
    unsigned long long key = ((unsigned long long)(uint32_t)votes << 32) |
                             ((unsigned long long)(256 - k) << 16) | (unsigned long long)(65535 - h);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
        key = other > key ? other : key;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(best, key);
}

// the frame's row tables from the winning line (or the camera's when nothing voted)
__global__ void __launch_bounds__(256) ground_rows_kernel(const unsigned long long* __restrict__ best, int H,
                                                          int dmax, const int32_t* __restrict__ kg_tab,
                                                          RowsDev cam, int32_t* __restrict__ rows,
                                                          int32_t* __restrict__ line)
{
    const unsigned long long key = *best;
    const int votes = (int)(key >> 32);
    const int k = 256 - (int)((key >> 16) & 0xffff);
    const int h = 65535 - (int)(key & 0xffff);
    const int emax = 16 * dmax;
    for (int v = threadIdx.x; v < H; v += blockDim.x) {
        int32_t fgq, kg;
        if (votes > 0) {
            const int x = k * (H - 1 - v - h);
            fgq = x >= 0 ? (x + 8) >> 4 : -((8 - x) >> 4);
            kg = kg_tab[min(max(fgq, 0), emax)];
        } else {
            fgq = cam.fgq[v];
            kg = cam.k_ground[v];
        }
        rows[v] = fgq;
        rows[H + v] = kg;
    }
    if (threadIdx.x == 0 && line) {
        line[0] = k;
        line[1] = h;
        line[2] = votes;
    }
}

}  // namespace

size_t ground_work_bytes(int H, int dmax)
{
    const size_t E = 16 * (size_t)dmax + 1;
    return ((sizeof(int32_t) * H * E + 255) / 256 * 256) + 256 + ((sizeof(int32_t) * (2 * (size_t)H + 3) + 255) / 256 * 256);
}

cudaError_t launch_ground(const int16_t* q, const FrameGeom& g, const ModelDev& m, RowsDev cam, char* work,
                          RowsDev* frame_rows, int32_t* line, cudaStream_t st)
{
    // cam is a copy: frame_rows may be the caller's camera rows themselves
    const size_t E = 16 * (size_t)m.dmax + 1;
    int32_t* smooth = (int32_t*)work;
    unsigned long long* best = (unsigned long long*)(work + (sizeof(int32_t) * g.H * E + 255) / 256 * 256);
    int32_t* rows = (int32_t*)((char*)best + 256);
    frame_rows->fgq = rows;
    frame_rows->k_ground = rows + g.H;
    frame_rows->g_ground = nullptr;
    cudaError_t e = cudaMemsetAsync(best, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    vdisp_kernel<<<g.H, 256, sizeof(int32_t) * E, st>>>(q, g.H, g.ncols, m.dmax, smooth);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    vote_kernel<<<g.H, 256, 0, st>>>(smooth, g.H, m.dmax, best);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ground_rows_kernel<<<1, 256, 0, st>>>(best, g.H, m.dmax, m.kg_tab, cam, rows, line ? line : rows + 2 * g.H);
    return cudaGetLastError();
}

}  // namespace stx
