// kernels_luts.cu -- per-column prefix look-up tables (paper Sec. 3.4, Sec. 5.2).
//
// For every reduced column (Q4 codes q[v], v = 0 bottom) the kernel writes the
// prefix sums, with a leading zero, of
//   - the disparities themselves (PD, Q4 units)             -> mean of any stixel in O(1)
//   - the ground and sky per-pixel costs of Eq. 4 (PG, PS)
//   - the object per-pixel cost at every integer model disparity f in [0, dmax]
//     (PO, the paper's LUT_object: (dmax+1) rows per column)
// so that any stixel's data cost is the difference of two table entries.
// On the whole-pixel grid the object pixel cost is instead read from the
// off-line (f, d) table (the paper's LUT_cost, Sec. 3.4), which holds the same
// values.  Per-pixel cost: min(C_out, K + G[min(|q - 16 f|, esat)]), all int32 in
// 2^-14 units (see stixels.h); G is the per-class residual table built at
// create time and esat the residual from which every pixel of the class costs
// C_out (so the clamp changes no cost and the staged table is small: ~64
// entries for sigma = 1 px).
//
// Work split: one warp per LUT row (as in the paper's Sec. 5.2), 32 rows per
// 256-thread CTA (48 when only the code range is written with the default
// model), grid = (ncols, ceil((dmax + 4) / rows)).  A lane owns 8
// consecutive outputs, so one chunk of the row is 256 entries: 7 in-register
// adds, a 5-step shuffle scan of the lane totals, and two 16-byte stores per
// lane.  Rows are padded to a multiple
// of 4 entries (pitch P) so every store is aligned.  The kernel is bound by
// the write bandwidth of the ncols x (dmax + 4) x P x 4-byte output.
#include <climits>

#include "internal.h"

namespace stx {
namespace {

constexpr int kRowsPerCta = 32;               // rows per CTA, whole tables
constexpr int kRowsPerCtaRange = 48;          // rows per CTA, code range only (default model)
constexpr int kMaxRowsPerCta = 48;
constexpr int kLutThreads = 256;             // threads of every LUT CTA (8 warps)
constexpr int kPerLane = 8;                    // consecutive outputs per lane
constexpr int kChunk = 32 * kPerLane;          // outputs per warp iteration

// Half-width (whole pixels) of the window of the LUT_cost row of disparity f
// outside which every pixel costs C_out: |d - f| >= ceil(esat / 16).
__host__ __device__ inline int lc_radius(int esat_obj) { return (esat_obj + 15) >> 4; }

// One LUT row: out[j] = sum over pixels v < j of cost(q[v], v), j = 0 .. P-1,
// by one warp; s_q[j] = q[j - 1].  A lane owns kPerLane consecutive outputs
// of each 256-entry chunk: in-register adds, a shuffle scan of the lane
// totals, two 16-byte stores.  Pixels outside [0, H) contribute nothing
// (cost is evaluated for them and discarded, so the loop has no branch).
// kSplit: a chunk whose pixels all lie in [0, H), but the one before output
// 0, skips the per-pixel test (measured: 32 1024x440 frames batched 13.06 ->
// 13.47 K frames/s); off where the extra code path spills registers (the
// whole-pixel grid's 32-register shape).
template <bool kSplit, class Cost>
__device__ __forceinline__ void scan_row(int32_t* __restrict__ out, const int32_t* s_q, int P, int H, int lane,
                                         Cost cost)
{
    int32_t carry = 0;
    for (int base = 0; base < P; base += kChunk) {
        const int j0 = base + kPerLane * lane;
        // the lane's 8 codes in two 16-byte reads (conflict-free)
        const int4 qa = *reinterpret_cast<const int4*>(s_q + j0);
        const int4 qb = *reinterpret_cast<const int4*>(s_q + j0 + 4);
        const int32_t qs[kPerLane] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
        int32_t c[kPerLane];
        if (kSplit && base + kChunk <= H + 1) {
            // every pixel of the chunk lies in [0, H) but the one before
            // output 0 (the leading zero): one test for the whole chunk
#pragma unroll
            for (int i = 0; i < kPerLane; ++i) c[i] = cost(qs[i], max(j0 + i - 1, 0));
            if (base == 0 && lane == 0) c[0] = 0;
        } else {
#pragma unroll
            for (int i = 0; i < kPerLane; ++i) {
                const int v = j0 + i - 1;                 // pixel that enters at output j
                const int32_t x = cost(qs[i], min(max(v, 0), H - 1));
                c[i] = (unsigned)v < (unsigned)H ? x : 0;
            }
        }
#pragma unroll
        for (int i = 1; i < kPerLane; ++i) c[i] += c[i - 1];
        int32_t tot = c[kPerLane - 1];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, tot, o);
            if (lane >= o) tot += t;
        }
        const int32_t add = carry + tot - c[kPerLane - 1];   // exclusive prefix of this lane
#pragma unroll
        for (int h = 0; h < kPerLane; h += 4) {
            if (j0 + h < P) {
                int4 w = make_int4(c[h] + add, c[h + 1] + add, c[h + 2] + add, c[h + 3] + add);
                *reinterpret_cast<int4*>(out + j0 + h) = w;
            }
        }
        carry += __shfl_sync(0xffffffffu, tot, 31);
    }
}

// Rows [row0, row0 + a.rows_per_cta) of column `col`'s LUTs (row f < F: object
// at disparity f; F: disparities; F + 1: ground; F + 2: sky), by one CTA.
// kIntGrid: codes are whole pixels and object costs come from the staged
// window [f - r, f + r] of LUT_cost row f (d outside it is clamped to its
// edge, where the cost is already C_out, so every saturated pixel of a warp
// reads the same word).  kVarSigma: sigma depends on the model disparity, so
// each object row f reads its own residual row (global, L1-resident) and each
// ground pixel its row's table; the constant-sigma tables are not staged.
template <bool kIntGrid, bool kVarSigma>
__device__ __forceinline__ void lut_rows(const LutArgs& a, const int col, const int row0, int32_t* sm)
{
    const int16_t* __restrict__ q = a.q;
    const int H = a.H, P = a.P, F = a.F;
    const ModelDev& m = a.m;
    const RowsDev& rows = a.rows;
    int32_t* __restrict__ pd = a.pd;
    int32_t* __restrict__ pg = a.pg;
    int32_t* __restrict__ ps = a.ps;
    int32_t* __restrict__ po = a.po;
    const int QP = (P + kChunk - 1) / kChunk * kChunk;
    int32_t* s_q = sm;                           // [QP]: s_q[j] = q[j - 1] (j = 1..H), 0 elsewhere
    const int ngo = kVarSigma ? 0 : m.esat_obj + 1;
    const int E = m.emax + 1;
    int32_t* s_go = s_q + QP;                    // [ngo]   residual tables, clamped at saturation
    int32_t* s_gs = s_go + ngo;                  // [esat_sky + 1]
    int32_t* s_lc = s_gs + m.esat_sky + 1;       // whole-pixel grid: [rows per CTA][2 r + 1] windows
    const int RC = a.rows_per_cta;
    const int R = F + 3;
    const int lr = lc_radius(m.esat_obj), lw = 2 * lr + 1;

    if ((unsigned)(F + 1 - row0) < (unsigned)RC) {
        // the ground row reads its row tables, then its residual windows, at
        // every pixel: start bringing both into L2 now, behind the codes' loads
        const char* pb = reinterpret_cast<const char*>(rows.gpool);
        const int np = 4 * rows.gn;
        for (int o = 128 * threadIdx.x; o < np; o += 128 * kLutThreads) asm volatile("prefetch.global.L2 [%0];" ::"l"(pb + o));
        const char* rb = reinterpret_cast<const char*>(rows.fg);
        const int nr = 36 * H;
        for (int o = 128 * threadIdx.x; o < nr; o += 128 * kLutThreads) asm volatile("prefetch.global.L2 [%0];" ::"l"(rb + o));
    }
    for (int e = threadIdx.x; e < ngo; e += blockDim.x) s_go[e] = __ldg(m.g_obj + e);
    for (int e = threadIdx.x; e <= m.esat_sky; e += blockDim.x) s_gs[e] = __ldg(m.g_sky + e);
    if (kIntGrid) {
        // the windows of the LUT_cost rows of this CTA's object disparities
        // (entries beyond [0, dmax] are never read: d is clamped to [0, dmax] first)
        const int nf = min(RC, F - row0);
        for (int i = threadIdx.x; i < nf * lw; i += blockDim.x) {
            const int ff = row0 + i / lw, d = ff - lr + i % lw;
            s_lc[i] = (d >= 0 && d < F) ? __ldg(m.lut_cost + (size_t)ff * F + d) : m.c_out;
        }
    }
    // the codes: from here on this kernel reads what the reduction wrote and
    // writes the tables the previous frame's DP may have read
    grid_dependency_wait();
    for (int j = threadIdx.x; j < QP; j += blockDim.x) s_q[j] = (j >= 1 && j <= H) ? q[(size_t)col * H + j - 1] : 0;
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the object rows a stixel of this column can use: its rounded mean lies
    // between round(min q / 16) and round(max q / 16)
    int f_lo = 0, f_hi = F - 1;
    if (a.range_only && row0 < F) {
        __shared__ int s_ext[2][kLutThreads / 32];
        int lo = INT_MAX, hi = INT_MIN;
        for (int j = 1 + threadIdx.x; j <= H; j += blockDim.x) {
            lo = min(lo, s_q[j]);
            hi = max(hi, s_q[j]);
        }
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        if (lane == 0) {
            s_ext[0][warp] = lo;
            s_ext[1][warp] = hi;
        }
        __syncthreads();
        lo = INT_MAX;
        hi = INT_MIN;
#pragma unroll
        for (int w = 0; w < kLutThreads / 32; ++w) {
            lo = min(lo, s_ext[0][w]);
            hi = max(hi, s_ext[1][w]);
        }
        f_lo = max((lo + 8) >> 4, 0);
        f_hi = min((hi + 8) >> 4, F - 1);
    }
    for (int rr = warp; rr < RC; rr += 8) {
        const int row = row0 + rr;
        if (row >= R) break;
        if (row < F && (row < f_lo || row > f_hi)) continue;     // never read
        // one row kind per call, so the per-pixel cost below is branch-free
        if (row < F) {
            const int f = row, f16 = 16 * f;
            const int32_t kf = __ldg(m.k_obj + f);
            int32_t* out = po + ((size_t)col * F + f) * P;
            if (kIntGrid) {
                // one read of the off-line table (codes are 16 d; the unsigned
                // clamp keeps malformed caller codes in [0, dmax])
                const int32_t* lc = s_lc + rr * lw + lr;
                scan_row<false>(out, s_q, P, H, lane, [&](int32_t qv, int) {
                    const int d = (int)(min((uint32_t)qv, (uint32_t)m.emax) >> 4);
                    return lc[min(max(d - f, -lr), lr)];
                });
            } else if (kVarSigma) {
                const int32_t* g = m.g_obj + (size_t)f * E;
                scan_row<true>(out, s_q, P, H, lane, [&](int32_t qv, int) {
                    return min(m.c_out, kf + __ldg(g + min(abs(qv - f16), m.emax)));
                });
            } else {
                const int es = m.esat_obj;
                const int32_t co = m.c_out;
                scan_row<true>(out, s_q, P, H, lane, [&](int32_t qv, int) {
                    return min(co, kf + s_go[min(abs(qv - f16), es)]);
                });
            }
        } else if (row == F) {
            scan_row<!kIntGrid>(pd + (size_t)col * P, s_q, P, H, lane, [&](int32_t qv, int) { return qv; });
        } else if (row == F + 1) {
            // the ground line is not on the Q4 grid: each row has its own
            // window of residuals (RowsDev), past which a pixel costs C_out
            const int32_t* __restrict__ kg = rows_kg(rows.fg, H);
            const int32_t* __restrict__ gf = rows_gf(rows.fg, H);
            const int32_t* __restrict__ goff = rows_goff(rows.fg, H);
            const int32_t* __restrict__ gpool = rows.gpool;
            const int gw = rows.gw, er = (rows.gw - 2) >> 1;
            const int32_t co = m.c_out;
            scan_row<!kIntGrid>(pg + (size_t)col * P, s_q, P, H, lane, [&](int32_t qv, int v) {
                const int j = qv - __ldg(gf + v) + er;
                return (unsigned)j < (unsigned)gw ? min(co, __ldg(kg + v) + __ldg(gpool + __ldg(goff + v) + j)) : co;
            });
        } else {
            scan_row<!kIntGrid>(ps + (size_t)col * P, s_q, P, H, lane, [&](int32_t qv, int) {
                return min(m.c_out, m.k_sky + s_gs[min(abs(qv), m.esat_sky)]);
            });
        }
    }
}

template <bool kIntGrid, bool kVarSigma>
__global__ void __launch_bounds__(256, kVarSigma ? 6 : 8) prefix_lut_kernel(LutArgs a)
{
    extern __shared__ __align__(16) int32_t sm[];
    // the DP kernel that follows may be scheduled now (it waits for the tables)
    grid_dependents_may_launch();
    lut_rows<kIntGrid, kVarSigma>(a, blockIdx.x, blockIdx.y * a.rows_per_cta, sm);
}

// Batch form: blockIdx.x indexes a list of (frame, column) items, blockIdx.y
// the row group; groups beyond a frame's F + 3 rows return at once.
__global__ void __launch_bounds__(256) prefix_lut_batch_kernel(const LutArgs* __restrict__ frames,
                                                               const int2* __restrict__ items)
{
    extern __shared__ __align__(16) int32_t sm[];
    __shared__ LutArgs s_args;
    const int2 w = items[blockIdx.x];
    const int* src = reinterpret_cast<const int*>(frames + w.x);
    int* dst = reinterpret_cast<int*>(&s_args);
    for (int i = threadIdx.x; i < (int)(sizeof(LutArgs) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    if ((int)blockIdx.y * s_args.rows_per_cta >= s_args.F + 3) return;
    const int row0 = blockIdx.y * s_args.rows_per_cta;
    if (s_args.m.var_sigma) {
        if (s_args.m.int_grid) lut_rows<true, true>(s_args, w.y, row0, sm);
        else lut_rows<false, true>(s_args, w.y, row0, sm);
    } else {
        if (s_args.m.int_grid) lut_rows<true, false>(s_args, w.y, row0, sm);
        else lut_rows<false, false>(s_args, w.y, row0, sm);
    }
}

}  // namespace

size_t lut_shared_bytes(int H, const ModelDev& m)
{
    const int P = lut_pitch(H);
    const int QP = (P + kChunk - 1) / kChunk * kChunk;
    const size_t lc = m.int_grid ? (size_t)kMaxRowsPerCta * (2 * lc_radius(m.esat_obj) + 1) : 0;
    const size_t tabs = m.var_sigma ? (size_t)m.esat_sky + 1 : (size_t)m.esat_obj + m.esat_sky + 2;
    return sizeof(int32_t) * ((size_t)QP + tabs + lc);
}

// (measured with the code range written, 1024x440: 32 rows 106.8 us per
// stixels_compute, 48 rows 105.5, 64 rows 107.1; 32 batched frames 14.67 /
// 14.99 / 14.98 K frames/s; with whole tables, the whole-pixel grid or the
// variable sigma 48 rows were slower: 18.4 -> 22.5 us per LUT launch)
int lut_rows_per_cta(const ModelDev& m, int range_only)
{
    return range_only && !m.int_grid && !m.var_sigma ? kRowsPerCtaRange : kRowsPerCta;
}

int lut_row_groups(int F, int rows_per_cta) { return (F + 3 + rows_per_cta - 1) / rows_per_cta; }

cudaError_t launch_luts(const int16_t* q, const FrameGeom& g, const ModelDev& m, const RowsDev& r,
                        int32_t* pd, int32_t* pg, int32_t* ps, int32_t* po, cudaStream_t st, int range_only)
{
    if (g.H <= 0 || g.ncols <= 0) return cudaSuccess;
    LutArgs a;
    a.q = q; a.H = g.H; a.P = g.P; a.F = m.dmax + 1; a.m = m; a.rows = r;
    a.pd = pd; a.pg = pg; a.ps = ps; a.po = po;
    a.range_only = range_only;
    a.rows_per_cta = lut_rows_per_cta(m, range_only);
    dim3 grid(g.ncols, lut_row_groups(a.F, a.rows_per_cta));
    const size_t smem = lut_shared_bytes(g.H, m);
    // a programmatic dependent of the reduction before it on the stream
    if (m.var_sigma)
        return m.int_grid ? launch_dependent(prefix_lut_kernel<true, true>, grid, dim3(256), smem, st, a)
                          : launch_dependent(prefix_lut_kernel<false, true>, grid, dim3(256), smem, st, a);
    return m.int_grid ? launch_dependent(prefix_lut_kernel<true, false>, grid, dim3(256), smem, st, a)
                      : launch_dependent(prefix_lut_kernel<false, false>, grid, dim3(256), smem, st, a);
}

cudaError_t launch_luts_batch(const LutArgs* d_frames, const int2* d_items, int nitems, int max_groups,
                              size_t smem, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    dim3 grid(nitems, max_groups);
    prefix_lut_batch_kernel<<<grid, 256, smem, st>>>(d_frames, d_items);
    return cudaGetLastError();
}

}  // namespace stx
