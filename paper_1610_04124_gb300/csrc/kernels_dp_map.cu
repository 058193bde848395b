// kernels_dp_map.cu -- the global MAP (global_map = 1): the DP of Eq. 5-6 with
// the ordering prior exact.  Eq. 6 keeps one best stixel per (row, class), so
// the ordering penalty of an object is judged against the best object below
// it, not against every object that could be below it; here the object state
// also carries the disparity f of its stixel:
//   O[k][f]  best cost of rows 0..k whose top stixel is an object of mean f,
//   G[k], S[k] the same for ground / sky tops,
// and an object [b, k] of mean f' above an object state (b-1, f) pays the
// ordering penalty iff f' > f + floor(eps / 16).  Over f that is a prefix
// (penalised) and a suffix (free) of row b-1, so with the prefix and suffix
// minima of O[b-1][.] every candidate costs O(1): O(H^2 + H F) per column.
//
// Ties: lexicographic (cost, previous class, start row, previous f), the
// previous class's code in the cost's two low bits as everywhere in this
// library; a candidate is one 64-bit key (cost | code) << 32 | start << 8 | f,
// so one integer minimum orders them (shared-memory atomicMin per object bin).
//
// Parallel scheme (correctness first): one 256-thread CTA per column, rows in
// order; at row k the threads take the starts b <= k, the object candidates
// go to their bin f' by atomic minimum, ground and sky by warp minima then one
// atomic each; then the CTA turns row k's bins into prefix / suffix minima
// (a block scan over f) in global scratch, which row k + 1 onwards reads.
#include <climits>

#include "internal.h"

namespace stx {
namespace {

constexpr unsigned long long kNoKey = ~0ull;

__device__ __forceinline__ unsigned long long make_key(int32_t cost_code, int b, int f)
{
    return ((unsigned long long)(uint32_t)cost_code << 32) | (unsigned long long)((uint32_t)b << 8 | (uint32_t)f);
}
__device__ __forceinline__ int32_t key_cost(unsigned long long k) { return (int32_t)(k >> 32); }
__device__ __forceinline__ int key_start(unsigned long long k) { return (int)((k >> 8) & 0xffffff); }
__device__ __forceinline__ int key_f(unsigned long long k) { return (int)(k & 255); }

// value of a state for the states above it: the cost without the code, capped
__device__ __forceinline__ int32_t state_value(unsigned long long k)
{
    return k == kNoKey ? kBig : min(key_cost(k) & ~3, kBig);
}

__device__ __forceinline__ unsigned long long warp_min(unsigned long long x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
        x = y < x ? y : x;
    }
    return x;
}

struct MapScratch {
    unsigned long long* keyo;   // [H][F] best key of each object state
    unsigned long long* pre;    // [H][F] (min over f' <= x of value) << 32 | argmin f'
    unsigned long long* suf;    // [H][F] (min over f' >= x) << 32 | argmin f'
};

__global__ void __launch_bounds__(256) stixel_map_kernel(DpArgs a, unsigned long long* scratch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int H = a.H, P = a.P, F = a.F;
    const int col = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const ModelDev& m = a.m;
    const size_t HF = (size_t)H * F;
    MapScratch sc;
    sc.keyo = scratch + (size_t)col * 3 * HF;
    sc.pre = sc.keyo + HF;
    sc.suf = sc.pre + HF;

    int32_t* s_pd = reinterpret_cast<int32_t*>(smem);                 // [H + 1]
    int32_t* s_pg = s_pd + (H + 1);                                   // [H + 1]
    int32_t* s_ps = s_pg + (H + 1);                                   // [H + 1]
    int32_t* s_fhi = s_ps + (H + 1);                                  // [H]
    int32_t* s_flo = s_fhi + H;                                       // [H]
    unsigned long long* s_kg = reinterpret_cast<unsigned long long*>(s_flo + H + ((2 * H + 3 * (H + 1)) & 1));  // [H]
    unsigned long long* s_ks = s_kg + H;                              // [H]
    unsigned long long* s_bin = s_ks + H;                             // [F]
    unsigned long long* s_red = s_bin + F;                            // [8] warp partials
    __shared__ unsigned long long s_rowg, s_rows;

    const int32_t* po_col = a.po + (size_t)col * F * P;
    for (int v = tid; v <= H; v += blockDim.x) {
        s_pd[v] = a.pd[(size_t)col * P + v];
        s_pg[v] = a.pg[(size_t)col * P + v];
        s_ps[v] = a.ps[(size_t)col * P + v];
        if (v < H) {
            const int32_t g = a.rows.fgq[v];
            s_fhi[v] = (g + m.eps_g) >> 4;            // gravity iff f > fhi
            s_flo[v] = -((m.eps_d - g) >> 4);         // diving iff f < flo
        }
    }
    __syncthreads();
    const int ord_off = m.eps_o >> 4;               // ordering iff f' > f + ord_off
    const int32_t T_oo = m.trans[0][0], T_og = m.trans[0][1] + 1, T_os = m.trans[0][2] + 2;
    const int32_t T_go = m.trans[1][0], T_gg = m.trans[1][1] + 1, T_gs = m.trans[1][2] + 2;
    const int32_t T_so = m.trans[2][0], T_sg = m.trans[2][1] + 1, T_ss = m.trans[2][2] + 2;

    for (int k = 0; k < H; ++k) {
        for (int f = tid; f < F; f += blockDim.x) s_bin[f] = kNoKey;
        if (tid == 0) { s_rowg = kNoKey; s_rows = kNoKey; }
        __syncthreads();
        unsigned long long bg = kNoKey, bs = kNoKey;   // this thread's best ground / sky candidates
        for (int b = tid; b <= k; b += blockDim.x) {
            const int n = k - b + 1;
            const int32_t S = s_pd[k + 1] - s_pd[b];
            const int fo = min((S + 8 * n) / (16 * n), m.dmax);
            const int32_t d_o = __ldg(po_col + (size_t)fo * P + k + 1) - __ldg(po_col + (size_t)fo * P + b);
            const int32_t d_g = s_pg[k + 1] - s_pg[b], d_s = s_ps[k + 1] - s_ps[b];
            unsigned long long ko, kg, ks;
            if (b == 0) {
                ko = make_key(d_o + m.first[0] + kNoneCode, 0, 0);
                kg = make_key(d_g + m.first[1] + kNoneCode, 0, 0);
                ks = make_key(d_s + m.first[2] + kNoneCode, 0, 0);
            } else {
                const size_t row = (size_t)(b - 1) * F;
                // object above object: free for previous f >= fo - ord_off, penalised below
                const int x = fo - ord_off;
                ko = kNoKey;
                if (x <= F - 1) {
                    const unsigned long long su = sc.suf[row + max(x, 0)];
                    const int32_t v = min((int32_t)(su >> 32), kBig);
                    const unsigned long long c = make_key(d_o + v + T_oo, b, (int)(su & 255));
                    ko = c < ko ? c : ko;
                }
                if (x - 1 >= 0) {
                    const unsigned long long pr = sc.pre[row + min(x - 1, F - 1)];
                    const int32_t v = min((int32_t)(pr >> 32), kBig);
                    const unsigned long long c = make_key(d_o + v + T_oo + m.pen_ord, b, (int)(pr & 255));
                    ko = c < ko ? c : ko;
                }
                const int32_t vg = state_value(s_kg[b - 1]), vs = state_value(s_ks[b - 1]);
                const int32_t gpen = (fo > s_fhi[b] ? m.pen_grav : 0) + (fo < s_flo[b] ? m.pen_div : 0);
                const unsigned long long cg = make_key(d_o + vg + T_og + gpen, b, 0);
                const unsigned long long cs = make_key(d_o + vs + T_os, b, 0);
                ko = cg < ko ? cg : ko;
                ko = cs < ko ? cs : ko;
                // ground / sky above: the best object of row b-1 (any f), ground, sky
                const unsigned long long mo = sc.pre[row + F - 1];
                const int32_t vo = min((int32_t)(mo >> 32), kBig);
                const int fm = (int)(mo & 255);
                kg = make_key(d_g + vo + T_go, b, fm);
                const unsigned long long g2 = make_key(d_g + vg + T_gg, b, 0), g3 = make_key(d_g + vs + T_gs, b, 0);
                kg = g2 < kg ? g2 : kg;
                kg = g3 < kg ? g3 : kg;
                ks = make_key(d_s + vo + T_so, b, fm);
                const unsigned long long s2 = make_key(d_s + vg + T_sg, b, 0), s3 = make_key(d_s + vs + T_ss, b, 0);
                ks = s2 < ks ? s2 : ks;
                ks = s3 < ks ? s3 : ks;
            }
            atomicMin(&s_bin[fo], ko);
            bg = kg < bg ? kg : bg;
            bs = ks < bs ? ks : bs;
        }
        bg = warp_min(bg);
        bs = warp_min(bs);
        if (lane == 0) {
            atomicMin(&s_rowg, bg);
            atomicMin(&s_rows, bs);
        }
        __syncthreads();
        // row k: object keys, and their prefix / suffix minima over f (value << 32 | f)
        const size_t row = (size_t)k * F;
        for (int base = 0; base < F; base += blockDim.x) {
            const int f = base + tid;
            if (f < F) sc.keyo[row + f] = s_bin[f];
        }
        if (tid == 0) {
            s_kg[k] = s_rowg;
            s_ks[k] = s_rows;
        }
        // F <= 256 = blockDim: one value per thread, block-wide inclusive scans
        const int f = tid;
        const unsigned long long mine = f < F ? ((unsigned long long)(uint32_t)state_value(s_bin[f]) << 32) | f : kNoKey;
        unsigned long long pmin = mine, smin = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long up = __shfl_up_sync(0xffffffffu, pmin, o);
            const unsigned long long dn = __shfl_down_sync(0xffffffffu, smin, o);
            if (lane >= o) pmin = up < pmin ? up : pmin;
            if (lane + o < 32) smin = dn < smin ? dn : smin;
        }
        __syncthreads();                              // s_bin no longer read below: reuse s_red
        if (lane == 31) s_red[warp] = pmin;           // warp totals for the prefix
        __syncthreads();
        unsigned long long pcarry = kNoKey;
        for (int w = 0; w < warp; ++w) pcarry = s_red[w] < pcarry ? s_red[w] : pcarry;
        __syncthreads();
        if (lane == 0) s_red[warp] = smin;            // warp totals for the suffix
        __syncthreads();
        unsigned long long scarry = kNoKey;
        for (int w = warp + 1; w < 8; ++w) scarry = s_red[w] < scarry ? s_red[w] : scarry;
        pmin = pcarry < pmin ? pcarry : pmin;
        smin = scarry < smin ? scarry : smin;
        if (f < F) {
            sc.pre[row + f] = pmin;
            sc.suf[row + f] = smin;
        }
        __threadfence_block();
        __syncthreads();
    }

    // top row (lexicographic cost, class, f) and backtracking
    if (tid == 0) {
        int c = -1, fb = 0;
        int32_t best = kBig;
        for (int f = 0; f < F; ++f) {
            const int32_t v = state_value(sc.keyo[(size_t)(H - 1) * F + f]);
            if (v < best) { best = v; c = 0; fb = f; }
        }
        if (state_value(s_kg[H - 1]) < best) { best = state_value(s_kg[H - 1]); c = 1; fb = 0; }
        if (state_value(s_ks[H - 1]) < best) { best = state_value(s_ks[H - 1]); c = 2; fb = 0; }
        if (c < 0 || best >= kBig) {
            a.counts[col] = 0;
            if (a.cost) a.cost[col] = __int_as_float(0x7f800000);
            if (a.cost_fixed) a.cost_fixed[col] = kBig;
            atomicOr(a.err, STIXELS_ERR_INFEASIBLE);
            return;
        }
        // count, then write bottom -> top
        int n = 0;
        for (int k = H - 1, cc = c, ff = fb; k >= 0 && cc < 3 && n <= H;) {
            const unsigned long long key = cc == 0 ? sc.keyo[(size_t)k * F + ff] : (cc == 1 ? s_kg[k] : s_ks[k]);
            ++n;
            const int b = key_start(key);
            if (b > k) break;
            k = b - 1;
            cc = key_cost(key) & 3;
            ff = key_f(key);
        }
        int idx = n - 1;
        stixel_t* out = a.stixels + (size_t)col * a.cap;
        for (int k = H - 1, cc = c, ff = fb; k >= 0 && cc < 3 && idx >= 0; --idx) {
            const unsigned long long key = cc == 0 ? sc.keyo[(size_t)k * F + ff] : (cc == 1 ? s_kg[k] : s_ks[k]);
            const int b = key_start(key);
            if (idx < a.cap) {
                const int nrows = k - b + 1;
                const int32_t S = s_pd[k + 1] - s_pd[b];
                stixel_t st;
                st.row_top = (int16_t)(H - 1 - k);
                st.row_bottom = (int16_t)(H - 1 - b);
                st.cls = (uint8_t)cc;
                st.flags = 0;
                st.reserved = 0;
                st.disparity = __fdiv_rn(__int2float_rn(S), __int2float_rn(16 * nrows));
                out[idx] = st;
            }
            if (b > k) break;
            k = b - 1;
            cc = key_cost(key) & 3;
            ff = key_f(key);
        }
        a.counts[col] = n;
        if (n > a.cap) atomicOr(a.err, STIXELS_ERR_CAPACITY);
        if (a.cost) a.cost[col] = __int2float_rn(best) * (1.0f / (float)kUnitsPerCost);
        if (a.cost_fixed) a.cost_fixed[col] = best;
    }
}

size_t map_smem_bytes(int H, int F)
{
    const size_t ints = 3 * (size_t)(H + 1) + 2 * (size_t)H;
    return sizeof(int32_t) * (ints + (ints & 1)) + sizeof(unsigned long long) * (2 * (size_t)H + F + 8);
}

}  // namespace

size_t map_scratch_bytes(int H, int ncols, int F) { return sizeof(unsigned long long) * 3 * (size_t)H * F * ncols; }

cudaError_t launch_dp_map(const int32_t* pd, const int32_t* pg, const int32_t* ps, const int32_t* po,
                          const FrameGeom& g, const ModelDev& m, const RowsDev& r, const stixels_output_t& out,
                          uint32_t* err, void* scratch, cudaStream_t st)
{
    if (g.H <= 0 || g.ncols <= 0) return cudaSuccess;
    if (g.H > STIXELS_MAX_HEIGHT || m.dmax + 1 > 256) return cudaErrorInvalidValue;
    DpArgs a;
    dp_frame_args(pd, pg, ps, po, g, m, r, out, err, &a);
    const size_t smem = map_smem_bytes(g.H, m.dmax + 1);
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        e = cudaFuncSetAttribute(stixel_map_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    stixel_map_kernel<<<g.ncols, 256, smem, st>>>(a, (unsigned long long*)scratch);
    return cudaGetLastError();
}

}  // namespace stx
