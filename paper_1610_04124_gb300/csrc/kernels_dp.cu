// kernels_dp.cu -- the stixel dynamic program (paper Eq. 5-6, Sec. 3.3, Sec. 5.3)
// with fused backtracking (Sec. 5.4).
//
// Recurrence, per column, for every end row k and class c in {object, ground, sky}:
//   V_c[k] = min over start b <= k and previous class p of
//            data_c(b, k) + prior(c | p, b, k) + V_p[b - 1]      (b = 0: first-stixel prior)
// data_c(b, k) is a difference of two prefix-LUT entries; for objects the LUT
// row is the rounded mean f = floor((S + 8 n) / (16 n)) of the stixel's Q4
// codes (S from the disparity prefix, n = k - b + 1).  Ties are broken by
// (cost, previous class, start row): the previous class's code sits in the two
// low bits of every candidate cost (all costs are multiples of 4), so one
// integer min orders (cost, class) and a strict "<" over ascending starts keeps
// the earliest start.
//
// Ground and sky stixels depend on the start b only through V[b - 1], the
// transition prior and the prefix entry at b, so for them
//   V_c[k] = PC[k + 1] + min_{b <= k} ( min_p (V_p[b - 1] + T_cp) - PC[b] )
// is a running minimum: O(1) per row.  Objects are the O(H^2) part.
//
// Parallel scheme (a redesign of the paper's one-thread-per-row CTA): rows are
// cut into blocks of 32.  For block t,
//   1. all warps gather the data terms of the block's 528 intra-block (b, k)
//      pairs into shared memory (no dependence on the DP),
//   2. warp 0 solves the block's triangle: 32 sequential starts, lane l owns
//      end row 32 t + l; after each start the owner's running minimum is
//      broadcast with a shuffle and every lane derives the next start's
//      context (no shared-memory round trip on the dependency chain),
//   3. all warps apply the 32 starts of block t to every later end row
//      (rectangles of 32 x 32 independent candidates, one per lane and start;
//      chunk j of end rows always goes to the same warp, so updates of one cell
//      happen in start order).
// The data terms come from the object LUT in global memory (L2-resident).
#include <climits>

#include "internal.h"

namespace stx {
namespace {

struct DpArgs {
    const int32_t* pd;
    const int32_t* pg;
    const int32_t* ps;
    const int32_t* po;
    int H, P, F;
    ModelDev m;
    RowsDev rows;
    stixel_t* stixels;
    int32_t* counts;
    float* cost;
    int32_t* cost_fixed;
    int cap;
    uint32_t* err;
};

// Context of one start row b, shared by every end row k >= b.
struct __align__(16) StartCtx {
    int32_t pdb;        // PD[b]
    int32_t bo, bg, bs; // V_p[b-1] + T(object | p) + code(p), p = object, ground, sky
    int32_t ford;       // ordering penalty iff f > ford
    int32_t fhi;        // gravity penalty iff f > fhi
    int32_t flo;        // diving penalty iff f < flo
    int32_t b;
};

__device__ __forceinline__ int32_t min3(int32_t a, int32_t b, int32_t c) { return min(min(a, b), c); }

// floor(x / (16 n)) for 0 <= x < 2^31 via a multiply-high: M = ceil(2^(32+s) / d),
// s = floor(log2 d), d = 16 n (M = 2^31, s - 1 when d is a power of two).
__device__ __forceinline__ uint2 div_magic(int n)
{
    const uint32_t d = 16u * (uint32_t)n;
    const int s = 31 - __clz(d);
    if ((d & (d - 1)) == 0) return make_uint2(1u << 31, (uint32_t)(s - 1));
    const unsigned long long num = 1ull << (32 + s);
    return make_uint2((uint32_t)((num + d - 1) / d), (uint32_t)s);
}

// Rounded mean disparity of a stixel, clamped to the LUT's rows: valid Q4 input
// always gives f <= dmax; the clamp only keeps malformed caller-built LUTs
// (stixels_solve) inside the table.
__device__ __forceinline__ int mean_f(int32_t S, int n, const uint2* s_div, int dmax)
{
    const uint2 dm = s_div[n];
    return (int)min(__umulhi((uint32_t)(S + 8 * n), dm.x) >> dm.y, (uint32_t)dmax);
}

// Object candidate of start context c for a stixel with rounded mean f and data cost d.
__device__ __forceinline__ int32_t obj_cand(const StartCtx& c, int f, int32_t d, const ModelDev& m)
{
    const int32_t co = c.bo + (f > c.ford ? m.pen_ord : 0);
    const int32_t cg = c.bg + (f > c.fhi ? m.pen_grav : 0) + (f < c.flo ? m.pen_div : 0);
    return min3(co, cg, c.bs) + d;
}

template <int NW>
__global__ void __launch_bounds__(NW * 32) stixel_dp_kernel(DpArgs a)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int col = blockIdx.x;
    const int H = a.H, P = a.P, F = a.F;
    const int HP = (H + 3) & ~3;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const ModelDev& m = a.m;

    extern __shared__ __align__(16) int32_t sm[];
    StartCtx* s_ctx = reinterpret_cast<StartCtx*>(sm);          // [HP]
    int32_t* s_pd = sm + 8 * HP;                                 // [P]
    int32_t* s_pg = s_pd + P;                                    // [P]
    int32_t* s_ps = s_pg + P;                                    // [P]
    uint2* s_div = reinterpret_cast<uint2*>(s_ps + P);           // [HP + 4], index n = 1..H
    int32_t* s_fhi = reinterpret_cast<int32_t*>(s_div + HP + 4); // [HP]
    int32_t* s_flo = s_fhi + HP;
    int32_t* s_bp = s_flo + HP;                                  // [3][HP] back-pointers b << 2 | p
    int32_t* s_runv = s_bp + 3 * HP;                             // [HP] object running minimum
    int32_t* s_runb = s_runv + HP;
    int32_t* s_runf = s_runb + HP;
    int32_t* s_tri_d = s_runf + HP;                              // [32][32]
    int32_t* s_tri_f = s_tri_d + 1024;                           // [32][32]

    const int32_t* po_col = a.po + (size_t)col * F * P;
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
        s_pd[j] = a.pd[(size_t)col * P + j];
        s_pg[j] = a.pg[(size_t)col * P + j];
        s_ps[j] = a.ps[(size_t)col * P + j];
    }
    for (int v = threadIdx.x; v < H; v += blockDim.x) {
        const int32_t g = a.rows.fgq[v];
        s_fhi[v] = (g + m.eps_g) >> 4;              // 16 f > g + eps  <=>  f > floor((g + eps) / 16)
        s_flo[v] = -((m.eps_d - g) >> 4);           // 16 f < g - eps  <=>  f < ceil((g - eps) / 16)
        s_runv[v] = INT_MAX;
        s_runb[v] = -1;
        s_runf[v] = 0;
    }
    for (int n = 1 + threadIdx.x; n <= H; n += blockDim.x) s_div[n] = div_magic(n);
    __syncthreads();

    const int ord_off = m.eps_o >> 4;               // 16 f > 16 f' + eps  <=>  f > f' + floor(eps / 16)
    const int NB = (H + 31) >> 5;

    // warp 0's carried state: V of the last finalised row, f of its best object
    // stixel, and the ground / sky running minima (all uniform across lanes)
    int32_t vo_p = 0, vg_p = 0, vs_p = 0, fo_p = 0;
    int32_t rg = INT_MAX, rgb = 0, rs = INT_MAX, rsb = 0;

    for (int t = 0; t < NB; ++t) {
        const int B = 32 * t;
        const int nb = min(32, H - B);
        // 1. intra-block data terms
        for (int idx = threadIdx.x; idx < 1024; idx += blockDim.x) {
            const int i = idx >> 5, l = idx & 31;
            if (i <= l && l < nb) {
                const int b = B + i, k = B + l, n = k - b + 1;
                const int f = mean_f(s_pd[k + 1] - s_pd[b], n, s_div, m.dmax);
                const int32_t* row = po_col + (size_t)f * P;
                s_tri_d[idx] = __ldg(row + k + 1) - __ldg(row + b);
                s_tri_f[idx] = f;
            }
        }
        __syncthreads();
        // 2. triangle
        if (warp == 0) {
            const int k = B + lane;
            const bool kv = lane < nb;
            int32_t run = kv ? s_runv[k] : INT_MAX;
            int32_t runb = kv ? s_runb[k] : -1;
            int32_t runf = kv ? s_runf[k] : 0;
            for (int i = 0; i < nb; ++i) {
                const int b = B + i;
                StartCtx c;
                int32_t ag, as;
                c.pdb = s_pd[b];
                c.b = b;
                if (b == 0) {
                    c.bo = m.first[0] + kNoneCode;
                    c.bg = kBig;
                    c.bs = kBig;
                    c.ford = INT_MAX; c.fhi = INT_MAX; c.flo = INT_MIN;
                    ag = m.first[1] + kNoneCode;
                    as = m.first[2] + kNoneCode;
                } else {
                    c.bo = vo_p + m.trans[0][0];
                    c.bg = vg_p + m.trans[0][1] + 1;
                    c.bs = vs_p + m.trans[0][2] + 2;
                    c.ford = fo_p + ord_off;
                    c.fhi = s_fhi[b];
                    c.flo = s_flo[b];
                    ag = min3(vo_p + m.trans[1][0], vg_p + m.trans[1][1] + 1, vs_p + m.trans[1][2] + 2);
                    as = min3(vo_p + m.trans[2][0], vg_p + m.trans[2][1] + 1, vs_p + m.trans[2][2] + 2);
                }
                if (lane == 0) s_ctx[b] = c;
                ag -= s_pg[b];
                as -= s_ps[b];
                if (ag < rg) { rg = ag; rgb = b; }
                if (as < rs) { rs = as; rsb = b; }
                if (kv && lane >= i) {
                    const int f = s_tri_f[i * 32 + lane];
                    const int32_t cand = obj_cand(c, f, s_tri_d[i * 32 + lane], m);
                    if (cand < run) { run = cand; runb = b; runf = f; }
                }
                // row b is complete: every lane derives its values
                const int32_t r = __shfl_sync(FULL, run, i);
                const int32_t rb = __shfl_sync(FULL, runb, i);
                const int32_t rf = __shfl_sync(FULL, runf, i);
                const int32_t gr = s_pg[b + 1] + rg;
                const int32_t sk = s_ps[b + 1] + rs;
                vo_p = min(r & ~3, kBig);
                vg_p = min(gr & ~3, kBig);
                vs_p = min(sk & ~3, kBig);
                fo_p = rf;
                if (lane == 0) {
                    s_bp[b] = (rb << 2) | (r & 3);
                    s_bp[HP + b] = (rgb << 2) | (gr & 3);
                    s_bp[2 * HP + b] = (rsb << 2) | (sk & 3);
                }
                __syncwarp();
            }
        }
        __syncthreads();
        // 3. rectangles: starts of block t applied to end rows of blocks j > t
        for (int j = t + 1 + warp; j < NB; j += NW) {
            const int k = 32 * j + lane;
            const bool kv = k < H;
            int32_t run = INT_MAX, runb = -1, runf = 0, pdk1 = 0;
            if (kv) { run = s_runv[k]; runb = s_runb[k]; runf = s_runf[k]; pdk1 = s_pd[k + 1]; }
#pragma unroll 4
            for (int i = 0; i < 32; ++i) {
                const StartCtx c = s_ctx[B + i];
                if (kv) {
                    const int n = k + 1 - c.b;
                    const int f = mean_f(pdk1 - c.pdb, n, s_div, m.dmax);
                    const int32_t* row = po_col + (size_t)f * P;
                    const int32_t d = __ldg(row + k + 1) - __ldg(row + c.b);
                    const int32_t cand = obj_cand(c, f, d, m);
                    if (cand < run) { run = cand; runb = c.b; runf = f; }
                }
            }
            if (kv) { s_runv[k] = run; s_runb[k] = runb; s_runf[k] = runf; }
        }
        __syncthreads();
    }

    // backtracking from the top row (Sec. 3.3, Sec. 5.4)
    if (threadIdx.x == 0) {
        int c = 0;
        int32_t best = vo_p;
        if (vg_p < best) { best = vg_p; c = 1; }
        if (vs_p < best) { best = vs_p; c = 2; }
        if (best >= kBig) {
            a.counts[col] = 0;
            if (a.cost) a.cost[col] = __int_as_float(0x7f800000);
            if (a.cost_fixed) a.cost_fixed[col] = kBig;
            atomicOr(a.err, STIXELS_ERR_INFEASIBLE);
            return;
        }
        int n = 0;
        for (int k = H - 1, cc = c; k >= 0 && cc < 3;) {
            const int32_t bp = s_bp[cc * HP + k];
            ++n;
            k = (bp >> 2) - 1;
            cc = bp & 3;
        }
        int idx = n - 1;
        stixel_t* out = a.stixels + (size_t)col * a.cap;
        for (int k = H - 1, cc = c; k >= 0 && cc < 3; --idx) {
            const int32_t bp = s_bp[cc * HP + k];
            const int b = bp >> 2;
            if (idx < a.cap) {
                const int32_t S = s_pd[k + 1] - s_pd[b];
                stixel_t st;
                st.row_top = (int16_t)(H - 1 - k);
                st.row_bottom = (int16_t)(H - 1 - b);
                st.cls = (uint8_t)cc;
                st.flags = 0;
                st.reserved = 0;
                st.disparity = __fdiv_rn(__int2float_rn(S), __int2float_rn(16 * (k - b + 1)));
                out[idx] = st;
            }
            k = b - 1;
            cc = bp & 3;
        }
        a.counts[col] = n;
        if (n > a.cap) atomicOr(a.err, STIXELS_ERR_CAPACITY);
        if (a.cost) a.cost[col] = __int2float_rn(best) * (1.0f / (float)kUnitsPerCost);
        if (a.cost_fixed) a.cost_fixed[col] = best;
    }
}

constexpr int kDpWarps = 4;

size_t dp_smem_bytes(int H, int P)
{
    const size_t HP = (size_t)((H + 3) & ~3);
    return sizeof(int32_t) * (8 * HP + 3 * (size_t)P + 2 * (HP + 4) + 2 * HP + 3 * HP + 3 * HP + 2048);
}

}  // namespace

cudaError_t launch_dp(const int32_t* pd, const int32_t* pg, const int32_t* ps, const int32_t* po,
                      const FrameGeom& g, const ModelDev& m, const RowsDev& r, const stixels_output_t& out,
                      uint32_t* err, cudaStream_t st)
{
    if (g.H <= 0 || g.ncols <= 0) return cudaSuccess;
    // opt in to large dynamic shared memory once per device
    static bool configured[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!configured[dev]) {
        e = cudaFuncSetAttribute(stixel_dp_kernel<kDpWarps>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 227 * 1024);
        if (e != cudaSuccess) return e;
        configured[dev] = true;
    }
    DpArgs a;
    a.pd = pd; a.pg = pg; a.ps = ps; a.po = po;
    a.H = g.H; a.P = g.P; a.F = m.dmax + 1;
    a.m = m; a.rows = r;
    a.stixels = out.stixels; a.counts = out.counts; a.cost = out.column_cost; a.cost_fixed = out.column_cost_fixed;
    a.cap = out.capacity;
    a.err = err;
    const size_t smem = dp_smem_bytes(g.H, g.P);
    stixel_dp_kernel<kDpWarps><<<g.ncols, kDpWarps * 32, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace stx
