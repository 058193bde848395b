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
// Parallel scheme: one 256-thread CTA per column, rows in blocks of 32.  For
// block j (rows K0 ..): phase A, every warp evaluates the starts b < K0 (their
// rows are final) for the block's rows, lane = row, warps over the starts;
// object candidates go to their bin (row, f') in shared memory by atomic
// minimum (a lane merges consecutive candidates of the same f' first), ground
// and sky stay in registers until one atomic per lane.  Phase B, one warp,
// the block's rows in order: row k adds its starts inside the block (lane =
// start), then the warp turns the row's bins into prefix / suffix minima over
// f (one lane owns 8 consecutive f) in global scratch, which the rows above
// read; at the block's end all warps copy its bins (the object state keys,
// for the backtracking) to global memory.  Three CTA barriers per block
// instead of several per row.
#include <climits>

#include "internal.h"
#include "real_cost.cuh"

namespace stx {
namespace {

constexpr unsigned long long kNoKey = ~0ull;
__device__ const DivTable kDivTable = make_div_table();

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

// Minimum of a 64-bit key over the warp: the high words' minimum, then the
// low words' minimum among the lanes that hold it (two warp reductions).
__device__ __forceinline__ unsigned long long warp_min(unsigned long long x)
{
    const unsigned hi = (unsigned)(x >> 32), lo = (unsigned)x;
    const unsigned mh = __reduce_min_sync(0xffffffffu, hi);
    const unsigned ml = __reduce_min_sync(0xffffffffu, hi == mh ? lo : 0xffffffffu);
    return ((unsigned long long)mh << 32) | ml;
}

constexpr int kMapRows = 32;                 // rows per block
constexpr size_t kMapSmemMax = 227 * 1024;   // dynamic shared memory one CTA may use
constexpr int kMapWarps = 8;

// What one column's candidate evaluation needs (shared memory and the LUT).
struct MapCol {
    const int32_t* s_pd8;        // [H + 1] PD[v] + 8 v
    const int32_t* s_pg;         // [H + 1]
    const int32_t* s_ps;         // [H + 1]
    const int32_t* s_fhi;        // [H] gravity iff f > fhi
    const int32_t* s_flo;        // [H] diving iff f < flo
    const uint2* s_div;          // [H + 1] rounded-mean constants
    const unsigned long long* s_kg;   // [H] ground state keys
    const unsigned long long* s_ks;   // [H] sky state keys
    const unsigned long long* s_bo;   // [H] best object state of each row, value << 32 | f
    const int32_t* po;           // the column's object LUT, [F][P]
    int P, F, dmax, ord_off;
    int32_t T_oo, T_og, T_os, T_go, T_gg, T_gs, T_so, T_sg, T_ss;
};

// The candidate keys of the stixel [b, k]: object (for the state (k, fo)),
// ground and sky; every key is (cost | previous class code) << 32 | b << 8 |
// previous object f, so one integer minimum is the tie order.
// prer / sufr: the prefix / suffix minima of row b - 1 (unused for b = 0).
__device__ __forceinline__ void map_cands(const MapCol& c, const ModelDev& m, int b, int k,
                                          const unsigned long long* prer, const unsigned long long* sufr, int& fo,
                                          unsigned long long& ko, unsigned long long& kg, unsigned long long& ks)
{
    const int n = k - b + 1;
    const uint2 dm = c.s_div[n];
    fo = (int)min(__umulhi((uint32_t)(c.s_pd8[k + 1] - c.s_pd8[b]), dm.x) >> dm.y, (uint32_t)c.dmax);
    const int32_t* row = c.po + (size_t)fo * c.P;
    const int32_t d_o = __ldg(row + k + 1) - __ldg(row + b);
    const int32_t d_g = c.s_pg[k + 1] - c.s_pg[b], d_s = c.s_ps[k + 1] - c.s_ps[b];
    if (b == 0) {
        ko = make_key(d_o + m.first[0] + kNoneCode, 0, 0);
        kg = make_key(d_g + m.first[1] + kNoneCode, 0, 0);
        ks = make_key(d_s + m.first[2] + kNoneCode, 0, 0);
        return;
    }
    // object above object: free for previous f >= fo - ord_off, penalised below
    const int x = fo - c.ord_off;
    ko = kNoKey;
    if (x <= c.F - 1) {
        const unsigned long long su = sufr[max(x, 0)];
        const int32_t v = min((int32_t)(su >> 32), kBig);
        const unsigned long long t = make_key(d_o + v + c.T_oo, b, (int)(su & 255));
        ko = t < ko ? t : ko;
    }
    if (x - 1 >= 0) {
        const unsigned long long pr = prer[min(x - 1, c.F - 1)];
        const int32_t v = min((int32_t)(pr >> 32), kBig);
        const unsigned long long t = make_key(d_o + v + c.T_oo + m.pen_ord, b, (int)(pr & 255));
        ko = t < ko ? t : ko;
    }
    const int32_t vg = state_value(c.s_kg[b - 1]), vs = state_value(c.s_ks[b - 1]);
    const int32_t gpen = (fo > c.s_fhi[b] ? m.pen_grav : 0) + (fo < c.s_flo[b] ? m.pen_div : 0);
    const unsigned long long cg = make_key(d_o + vg + c.T_og + gpen, b, 0);
    const unsigned long long cs = make_key(d_o + vs + c.T_os, b, 0);
    ko = cg < ko ? cg : ko;
    ko = cs < ko ? cs : ko;
    // ground / sky above: the best object of row b-1 (any f), ground, sky
    const unsigned long long mo = c.s_bo[b - 1];
    const int32_t vo = min((int32_t)(mo >> 32), kBig);
    const int fm = (int)(mo & 255);
    kg = make_key(d_g + vo + c.T_go, b, fm);
    const unsigned long long g2 = make_key(d_g + vg + c.T_gg, b, 0), g3 = make_key(d_g + vs + c.T_gs, b, 0);
    kg = g2 < kg ? g2 : kg;
    kg = g3 < kg ? g3 : kg;
    ks = make_key(d_s + vo + c.T_so, b, fm);
    const unsigned long long s2 = make_key(d_s + vg + c.T_sg, b, 0), s3 = make_key(d_s + vs + c.T_ss, b, 0);
    ks = s2 < ks ? s2 : ks;
    ks = s3 < ks ? s3 : ks;
}

__global__ void __launch_bounds__(kMapWarps * 32) stixel_map_kernel(DpArgs a, unsigned long long* scratch)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int H = a.H, P = a.P, F = a.F;
    const int col = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const ModelDev& m = a.m;
    const size_t HF = (size_t)H * F;
    unsigned long long* keyo = scratch + (size_t)col * 3 * HF;   // [H][F] best key of each object state
    unsigned long long* pre = keyo + HF;
    unsigned long long* suf = pre + HF;

    unsigned long long* s_kg = reinterpret_cast<unsigned long long*>(smem);      // [H]
    unsigned long long* s_ks = s_kg + H;                                         // [H]
    unsigned long long* s_bo = s_ks + H;                                         // [H]
    unsigned long long* s_bin = s_bo + H;                                        // [2][kMapRows][F]
    unsigned long long* s_gbin = s_bin + 2 * (size_t)kMapRows * F;               // [2][kMapRows]
    unsigned long long* s_sbin = s_gbin + 2 * kMapRows;                          // [2][kMapRows]
    uint2* s_div = reinterpret_cast<uint2*>(s_sbin + 2 * kMapRows);              // [H + 1]
    int32_t* s_pd8 = reinterpret_cast<int32_t*>(s_div + H + 1);                  // [H + 1]
    int32_t* s_pg = s_pd8 + (H + 1);                                             // [H + 1]
    int32_t* s_ps = s_pg + (H + 1);                                              // [H + 1]
    int32_t* s_fhi = s_ps + (H + 1);                                             // [H]
    int32_t* s_flo = s_fhi + H;                                                  // [H]

    for (int v = tid; v <= H; v += blockDim.x) {
        s_pd8[v] = a.pd[(size_t)col * P + v] + 8 * v;
        s_pg[v] = a.pg[(size_t)col * P + v];
        s_ps[v] = a.ps[(size_t)col * P + v];
        if (v >= 1) {
            const DivMagic dm = kDivTable.v[v];
            s_div[v] = make_uint2(dm.m, dm.s);
        }
        if (v < H) {
            const int32_t t = rows_thr(a.rows.fg, H)[v];
            s_fhi[v] = (int32_t)(int16_t)(t & 0xffff);    // gravity iff f > fhi
            s_flo[v] = t >> 16;                           // diving iff f < flo
        }
    }
    MapCol c;
    c.s_pd8 = s_pd8; c.s_pg = s_pg; c.s_ps = s_ps; c.s_fhi = s_fhi; c.s_flo = s_flo; c.s_div = s_div;
    c.s_kg = s_kg; c.s_ks = s_ks; c.s_bo = s_bo;
    c.po = a.po + (size_t)col * F * P;
    c.P = P; c.F = F; c.dmax = m.dmax; c.ord_off = m.ord_off;       // ordering iff f' > f + ord_off
    c.T_oo = m.trans[0][0]; c.T_og = m.trans[0][1] + 1; c.T_os = m.trans[0][2] + 2;
    c.T_go = m.trans[1][0]; c.T_gg = m.trans[1][1] + 1; c.T_gs = m.trans[1][2] + 2;
    c.T_so = m.trans[2][0]; c.T_sg = m.trans[2][1] + 1; c.T_ss = m.trans[2][2] + 2;

    const int NB = (H + kMapRows - 1) / kMapRows;
    constexpr int kPer = 8;                       // object states per lane in the row scan (F <= 256)
    const size_t BF = (size_t)kMapRows * F;

    // Phase A for the rows K + lane (lane < nr) and the starts b = b0, b0 + step,
    // ... < b1 (rows of earlier blocks, all final), into one block's bins.  Two
    // starts are evaluated together so that their loads overlap; a lane keeps
    // its object candidates for one bin until f changes (consecutive starts
    // mostly share f), its ground / sky minima in registers.
    auto phase_a = [&](unsigned long long* bins, unsigned long long* gbin, unsigned long long* sbin, int K, int nr,
                       int b0, int b1, int step) {
        if (lane >= nr || b0 >= b1) return;
        const int k = K + lane;
        unsigned long long rg = kNoKey, rs = kNoKey, ck = kNoKey;
        int cf = -1;
        auto merge = [&](int fo, unsigned long long ko, unsigned long long kg, unsigned long long ks) {
            rg = kg < rg ? kg : rg;
            rs = ks < rs ? ks : rs;
            if (fo != cf) {
                if (cf >= 0) atomicMin(&bins[lane * F + cf], ck);
                cf = fo;
                ck = ko;
            } else {
                ck = ko < ck ? ko : ck;
            }
        };
        int b = b0;
        for (; b + step < b1; b += 2 * step) {
            int f0, f1;
            unsigned long long o0, g0, s0, o1, g1, s1;
            map_cands(c, m, b, k, pre + (size_t)(b - 1) * F, suf + (size_t)(b - 1) * F, f0, o0, g0, s0);
            map_cands(c, m, b + step, k, pre + (size_t)(b + step - 1) * F, suf + (size_t)(b + step - 1) * F, f1, o1,
                      g1, s1);
            merge(f0, o0, g0, s0);
            merge(f1, o1, g1, s1);
        }
        if (b < b1) {
            int f0;
            unsigned long long o0, g0, s0;
            map_cands(c, m, b, k, pre + (size_t)(b - 1) * F, suf + (size_t)(b - 1) * F, f0, o0, g0, s0);
            merge(f0, o0, g0, s0);
        }
        if (cf >= 0) atomicMin(&bins[lane * F + cf], ck);
        atomicMin(&gbin[lane], rg);
        atomicMin(&sbin[lane], rs);
    };

    // bins of blocks 0 and 1 (the bins are double-buffered by block parity)
    for (int i = tid; i < 2 * (int)BF; i += blockDim.x) s_bin[i] = kNoKey;
    if (tid < 2 * kMapRows) { s_gbin[tid] = kNoKey; s_sbin[tid] = kNoKey; }
    __syncthreads();
    for (int j = 0; j < NB; ++j) {
        const int K0 = kMapRows * j, nb = min(kMapRows, H - K0);
        const int K1 = K0 + kMapRows, nb1 = j + 1 < NB ? min(kMapRows, H - K1) : 0;
        unsigned long long* bin_j = s_bin + (j & 1) * BF;
        unsigned long long* gbin_j = s_gbin + (j & 1) * kMapRows;
        unsigned long long* sbin_j = s_sbin + (j & 1) * kMapRows;
        unsigned long long* bin_n = s_bin + ((j + 1) & 1) * BF;
        unsigned long long* gbin_n = s_gbin + ((j + 1) & 1) * kMapRows;
        unsigned long long* sbin_n = s_sbin + ((j + 1) & 1) * kMapRows;

        if (warp == 0) {
            // Phase B: the block's rows in order; row k adds its starts within
            // the block (lane = start K0 + lane <= k), then its object states
            // become prefix / suffix minima over f for the rows above.
            for (int r = 0; r < nb; ++r) {
                const int k = K0 + r;
                unsigned long long kg = kNoKey, ks = kNoKey;
                if (lane <= r) {
                    const int b = K0 + lane;
                    int fo;
                    unsigned long long ko;
                    map_cands(c, m, b, k, pre + (size_t)(b - 1) * F, suf + (size_t)(b - 1) * F, fo, ko, kg, ks);
                    atomicMin(&bin_j[r * F + fo], ko);
                }
                kg = warp_min(kg);
                ks = warp_min(ks);
                __syncwarp();
                const unsigned long long* bin = bin_j + (size_t)r * F;
                // lane l owns f = kPer l .. kPer l + kPer - 1: local prefix / suffix, then warp scans
                unsigned long long pv[kPer], sv[kPer];
#pragma unroll
                for (int i = 0; i < kPer; ++i) {
                    const int f = kPer * lane + i;
                    pv[i] = f < F ? ((unsigned long long)(uint32_t)state_value(bin[f]) << 32) | (unsigned)f : kNoKey;
                    sv[i] = pv[i];
                }
#pragma unroll
                for (int i = 1; i < kPer; ++i) pv[i] = pv[i - 1] < pv[i] ? pv[i - 1] : pv[i];
#pragma unroll
                for (int i = kPer - 2; i >= 0; --i) sv[i] = sv[i + 1] < sv[i] ? sv[i + 1] : sv[i];
                unsigned long long pt = pv[kPer - 1], st = sv[0];       // lane totals
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned long long up = __shfl_up_sync(0xffffffffu, pt, o);
                    const unsigned long long dn = __shfl_down_sync(0xffffffffu, st, o);
                    if (lane >= o) pt = up < pt ? up : pt;
                    if (lane + o < 32) st = dn < st ? dn : st;
                }
                // exclusive carries from the lanes below / above
                unsigned long long pc = __shfl_up_sync(0xffffffffu, pt, 1);
                unsigned long long sc = __shfl_down_sync(0xffffffffu, st, 1);
                if (lane == 0) pc = kNoKey;
                if (lane == 31) sc = kNoKey;
                const size_t rw = (size_t)k * F;
#pragma unroll
                for (int i = 0; i < kPer; ++i) {
                    const int f = kPer * lane + i;
                    if (f < F) {
                        pre[rw + f] = pc < pv[i] ? pc : pv[i];
                        suf[rw + f] = sc < sv[i] ? sc : sv[i];
                    }
                }
                if (lane == 0) {
                    s_kg[k] = kg < gbin_j[r] ? kg : gbin_j[r];
                    s_ks[k] = ks < sbin_j[r] ? ks : sbin_j[r];
                }
                // the row's best object state (over every f): the last prefix
                const unsigned long long best = __shfl_sync(0xffffffffu, pt, 31);
                if (lane == 0) s_bo[k] = best;
                // the rows above in this block are read by this warp only:
                // the warp barrier orders its lanes' stores and loads
                __syncwarp();
            }
        } else if (warp != 4) {
            // meanwhile: the next block's candidates whose starts lie in the
            // blocks before this one (their rows are final), on the warps that
            // do not share warp 0's scheduler (warp 4 does), so that the
            // sequential rows keep its issue slots
            phase_a(bin_n, gbin_n, sbin_n, K1, nb1, warp - 1 - (warp > 4), K0, kMapWarps - 2);
        }
        __syncthreads();                          // block j's rows are final and visible
        // the next block's starts inside this block; then this block's bins
        // (its object state keys) go to global memory for the backtracking,
        // coalesced, and are reset for block j + 2
        phase_a(bin_n, gbin_n, sbin_n, K1, nb1, K0 + warp, K0 + nb, kMapWarps);
        for (int i = tid; i < (int)BF; i += blockDim.x) {
            if (i < nb * F) keyo[(size_t)K0 * F + i] = bin_j[i];
            bin_j[i] = kNoKey;
        }
        if (tid < kMapRows) { gbin_j[tid] = kNoKey; sbin_j[tid] = kNoKey; }
        __syncthreads();
    }

    // top row (lexicographic cost, class, f) and backtracking, by warp 0: lane
    // 0 walks the path, then the warp reports its cost in real arithmetic
    if (warp != 0) return;
    int n = 0, feasible = 1;
    int32_t* s_seg = s_pg;                        // free after the last block; [H + 1] >= n
    if (lane == 0) {
        int cc0 = -1, fb = 0;
        int32_t best = kBig;
        for (int f = 0; f < F; ++f) {
            const int32_t v = state_value(keyo[(size_t)(H - 1) * F + f]);
            if (v < best) { best = v; cc0 = 0; fb = f; }
        }
        if (state_value(s_kg[H - 1]) < best) { best = state_value(s_kg[H - 1]); cc0 = 1; fb = 0; }
        if (state_value(s_ks[H - 1]) < best) { best = state_value(s_ks[H - 1]); cc0 = 2; fb = 0; }
        if (cc0 < 0 || best >= kBig) {
            a.counts[col] = 0;
            if (a.cost) a.cost[col] = __int_as_float(0x7f800000);
            if (a.cost_fixed) a.cost_fixed[col] = kBig;
            atomicOr(a.err, STIXELS_ERR_INFEASIBLE);
            feasible = 0;
        } else {
            // count, then write bottom -> top
            for (int k = H - 1, cc = cc0, ff = fb; k >= 0 && cc < 3 && n <= H;) {
                const unsigned long long key = cc == 0 ? keyo[(size_t)k * F + ff] : (cc == 1 ? s_kg[k] : s_ks[k]);
                ++n;
                const int b = key_start(key);
                if (b > k) break;
                k = b - 1;
                cc = key_cost(key) & 3;
                ff = key_f(key);
            }
            int idx = n - 1;
            stixel_t* out = a.stixels + (size_t)col * a.cap;
            for (int k = H - 1, cc = cc0, ff = fb; k >= 0 && cc < 3 && idx >= 0; --idx) {
                const unsigned long long key = cc == 0 ? keyo[(size_t)k * F + ff] : (cc == 1 ? s_kg[k] : s_ks[k]);
                const int b = key_start(key);
                s_seg[idx] = (min(b, k) << 13) | (k << 2) | cc;
                if (idx < a.cap) {
                    const int nrows = k - b + 1;
                    const int32_t S = s_pd8[k + 1] - s_pd8[b] - 8 * nrows;
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
            if (a.cost_fixed) a.cost_fixed[col] = best;
        }
    }
    n = __shfl_sync(0xffffffffu, n, 0);
    feasible = __shfl_sync(0xffffffffu, feasible, 0);
    __syncwarp();
    if (feasible && a.cost) {
        // (the scratch covers s_fhi / s_flo: the thresholds come from the row tables)
        const int32_t* thr_row = rows_thr(a.rows.fg, H);
        auto thr = [&](int b) {
            const int32_t t = __ldg(thr_row + b);
            return make_int2((int32_t)(int16_t)(t & 0xffff), t >> 16);
        };
        const long long rc = real_segmentation_cost(s_seg, n, s_pd8, s_div, a, H, lane, thr);
        if (lane == 0) a.cost[col] = __ll2float_rn(rc) * (1.0f / kReportUnits);
    }
}

size_t map_smem_bytes(int H, int F)
{
    return sizeof(unsigned long long) * (3 * (size_t)H + 2 * (size_t)kMapRows * F + 4 * kMapRows) +
           sizeof(uint2) * (size_t)(H + 1) + sizeof(int32_t) * (3 * (size_t)(H + 1) + 2 * (size_t)H);
}

}  // namespace

size_t map_scratch_bytes(int H, int ncols, int F) { return sizeof(unsigned long long) * 3 * (size_t)H * F * ncols; }

bool map_fits(int H, int F) { return map_smem_bytes(H, F) <= kMapSmemMax; }

cudaError_t launch_dp_map(const int32_t* pd, const int32_t* pg, const int32_t* ps, const int32_t* po,
                          const FrameGeom& g, const ModelDev& m, const RowsDev& r, const RealParams& rp,
                          int32_t pixel_floor, const stixels_output_t& out, uint32_t* err, void* scratch,
                          cudaStream_t st)
{
    if (g.H <= 0 || g.ncols <= 0) return cudaSuccess;
    if (g.H > STIXELS_MAX_HEIGHT || m.dmax + 1 > 256 || !map_fits(g.H, m.dmax + 1)) return cudaErrorInvalidValue;
    DpArgs a;
    dp_frame_args(pd, pg, ps, po, g, m, r, rp, pixel_floor, out, err, &a);
    const size_t smem = map_smem_bytes(g.H, m.dmax + 1);
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        e = cudaFuncSetAttribute(stixel_map_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMapSmemMax);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    stixel_map_kernel<<<g.ncols, 256, smem, st>>>(a, (unsigned long long*)scratch);
    return cudaGetLastError();
}

}  // namespace stx
