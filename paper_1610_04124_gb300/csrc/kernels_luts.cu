// kernels_luts.cu -- per-column prefix look-up tables (paper Sec. 3.4, Sec. 5.2).
//
// For every reduced column (Q4 codes q[v], v = 0 bottom) the kernel writes the
// prefix sums, with a leading zero, of
//   - the disparities themselves (PD, Q4 units)             -> mean of any stixel in O(1)
//   - the ground and sky per-pixel costs of Eq. 4 (PG, PS)
//   - the object per-pixel cost at every integer model disparity f in [0, dmax]
//     (PO, the paper's LUT_object: (dmax+1) rows per column)
// so that any stixel's data cost is the difference of two table entries.
// Per-pixel cost: min(C_out, K + G[min(|q - 16 f|, 16 dmax)]), all int32 in
// 2^-14 units (see stixels.h); G is the per-class residual table built at
// create time.
//
// Work split: one warp per LUT row (as in the paper's Sec. 5.2), 16 rows per
// 256-thread CTA, grid = (ncols, ceil((dmax + 4) / 16)).  A lane owns 4
// consecutive outputs, so one chunk of the row is 128 entries: 4 in-register
// adds, a 5-step shuffle scan of the lane totals, and one 16-byte store per
// lane (512 contiguous bytes per warp store).  Rows are padded to a multiple
// of 4 entries (pitch P) so every store is aligned.  The kernel is bound by
// the write bandwidth of the ncols x (dmax + 4) x P x 4-byte output.
#include "internal.h"

namespace stx {
namespace {

constexpr int kRowsPerCta = 16;

enum RowKind { kObject = 0, kDisp = 1, kGround = 2, kSky = 3 };

__global__ void __launch_bounds__(256) prefix_lut_kernel(const int16_t* __restrict__ q, int H, int P, int F,
                                                         ModelDev m, RowsDev rows, int32_t* __restrict__ pd,
                                                         int32_t* __restrict__ pg, int32_t* __restrict__ ps,
                                                         int32_t* __restrict__ po)
{
    extern __shared__ __align__(16) int32_t sm[];
    const int HP = (H + 3) & ~3;
    int32_t* s_q = sm;            // [HP]
    int32_t* s_g = sm + HP;       // [emax + 1] object residual table
    const int col = blockIdx.x;
    const int row0 = blockIdx.y * kRowsPerCta;
    const int R = F + 3;

    for (int v = threadIdx.x; v < H; v += blockDim.x) s_q[v] = q[(size_t)col * H + v];
    if (row0 < F)
        for (int e = threadIdx.x; e <= m.emax; e += blockDim.x) s_g[e] = __ldg(m.g_obj + e);
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int rr = warp; rr < kRowsPerCta; rr += 8) {
        const int row = row0 + rr;
        if (row >= R) break;
        int kind, f = 0;
        int32_t kf = 0;
        int32_t* out;
        if (row < F) {
            kind = kObject; f = row; kf = __ldg(m.k_obj + f);
            out = po + ((size_t)col * F + f) * P;
        } else if (row == F) {
            kind = kDisp; out = pd + (size_t)col * P;
        } else if (row == F + 1) {
            kind = kGround; out = pg + (size_t)col * P;
        } else {
            kind = kSky; out = ps + (size_t)col * P;
        }
        const int f16 = 16 * f;
        int32_t carry = 0;
        for (int base = 0; base < P; base += 128) {
            const int j0 = base + 4 * lane;              // outputs j0 .. j0+3 hold sums over v < j
            int32_t c[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int v = j0 + i - 1;                 // pixel that enters at output j
                int32_t x = 0;
                if (v >= 0 && v < H) {
                    const int32_t qv = s_q[v];
                    if (kind == kObject) {
                        const int e = min(abs(qv - f16), m.emax);
                        x = min(m.c_out, kf + s_g[e]);
                    } else if (kind == kDisp) {
                        x = qv;
                    } else if (kind == kGround) {
                        const int e = min(abs(qv - __ldg(rows.fgq + v)), m.emax);
                        x = min(m.c_out, __ldg(rows.k_ground + v) + __ldg(m.g_ground + e));
                    } else {
                        x = min(m.c_out, m.k_sky + __ldg(m.g_sky + min(abs(qv), m.emax)));
                    }
                }
                c[i] = x;
            }
            c[1] += c[0];
            c[2] += c[1];
            c[3] += c[2];
            int32_t tot = c[3];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t t = __shfl_up_sync(0xffffffffu, tot, o);
                if (lane >= o) tot += t;
            }
            const int32_t add = carry + tot - c[3];       // exclusive prefix of this lane
            if (j0 < P) {
                int4 w = make_int4(c[0] + add, c[1] + add, c[2] + add, c[3] + add);
                *reinterpret_cast<int4*>(out + j0) = w;
            }
            carry += __shfl_sync(0xffffffffu, tot, 31);
        }
    }
}

}  // namespace

cudaError_t launch_luts(const int16_t* q, const FrameGeom& g, const ModelDev& m, const RowsDev& r,
                        int32_t* pd, int32_t* pg, int32_t* ps, int32_t* po, cudaStream_t st)
{
    if (g.H <= 0 || g.ncols <= 0) return cudaSuccess;
    const int F = m.dmax + 1;
    const int HP = (g.H + 3) & ~3;
    const size_t smem = sizeof(int32_t) * ((size_t)HP + m.emax + 1);
    dim3 grid(g.ncols, (F + 3 + kRowsPerCta - 1) / kRowsPerCta);
    prefix_lut_kernel<<<grid, 256, smem, st>>>(q, g.H, g.P, F, m, r, pd, pg, ps, po);
    return cudaGetLastError();
}

}  // namespace stx
