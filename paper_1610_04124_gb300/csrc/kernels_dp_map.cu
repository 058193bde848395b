// kernels_dp_map.cu -- the global MAP (global_map = 1): the DP of Eq. 5-6 with
// the ordering prior exact.  Eq. 6 keeps one best stixel per (row, class), so
// the ordering penalty of an object is judged against the best object below
// it, not against every object that could be below it; here the object state
// also carries the disparity f of its stixel:
//   O[k][f]  best cost of rows 0..k whose top stixel is an object of mean f,
//   G[k], S[k] the same for ground / sky tops,
// and an object [b, k] of mean f' above an object state (b-1, f) pays the
// ordering penalty iff f' > f + floor(eps / 16).  Over f that splits row b-1
// into a penalised prefix f < x and a free suffix f >= x (x = f' - floor(eps
// / 16)), so the best object-below term of every candidate is one entry of
//   M[b-1][x] = min(min_{f >= x} O[b-1][f], min_{f < x} O[b-1][f] + penalty),
// x clamped to [0, F]: O(H^2 + H F) per column.
//
// Ties: lexicographic (cost, previous class, start row, previous f), the
// previous class's code in the cost's two low bits as everywhere in this
// library.  A state holds only its cost and code (int32, one atomic minimum
// per update); the backtracking recovers the rest for the states on the
// path: the lowest start whose candidate reaches the state's value, and for
// an object below, the lowest f at the minimum (the penalised side's if it
// reaches the minimum, else the free side's).
//
// Parallel scheme: one 256-thread CTA per column, rows in blocks of 32.  For
// block j (rows K0 ..): phase A, six warps evaluate the next block's rows
// against the starts of the blocks before this one (their rows are final;
// lane = row, warps over the starts) and gather the next block's own
// triangle of object cells (mean and data cost) into shared memory; object
// candidates go to their bin (row, f') by atomic minimum (a lane merges
// consecutive candidates of the same f' first), ground and sky stay in
// registers until one atomic per lane.  Phase B, two warps, the block's
// rows in order, from shared memory only: one warp adds row k + 1's starts
// inside the block up to k (lane = start; lanes of equal f' combine first)
// while the other finishes row k: it adds the start k, the one candidate
// that reads row k - 1, and turns the row's bins into the row M[k][.] (one
// lane owns 8 consecutive f; a suffix scan over f, since the penalty is not
// negative), kept in a shared ring of the block's rows; a 64-thread barrier
// per row.  Then every warp adds this block's starts to the next block's
// rows, and the block's states and rows of M go to global memory.  Three CTA
// barriers per block instead of several per row.
#include <climits>

#include "internal.h"
#include "real_cost.cuh"

namespace stx {
namespace {

constexpr int32_t kNone = INT_MAX;           // a state no candidate has reached

// value of a state for the states above it: the cost without the code, capped
__device__ __forceinline__ int32_t state_value(int32_t k) { return min(k & ~3, kBig); }

constexpr int kMapRows = 32;                 // rows per block
constexpr size_t kMapSmemMax = 226 * 1024;   // dynamic shared memory one CTA may use (227 KB less the static)
constexpr int kMapWarps = 8;
constexpr int kPer = 8;
// phase B's two warps (on different schedulers); phase A runs on the rest
// (measured against phase A on five warps with the first one's scheduler
// partner idle, and against the second phase-B warp on that partner: 1024x440
// 315 / 324 / 324 us, 2048x880 1564 / 1763 / 1593 us)
constexpr int kWarpS = 0, kWarpC = 1;
constexpr int kPhaseAWarps = kMapWarps - 2;
__device__ __forceinline__ int phase_a_index(int w) { return w - 2; }                      // object states per lane in a row's scan (F <= 256)
constexpr int kTri = 528;                    // cells (b, k), b <= k, of one block
__device__ __forceinline__ int tri_slot(int i) { return (i * (65 - i)) >> 1; }

__device__ const DivTable kDivTable = make_div_table();

// the stride of a row of M (F + 1 entries, x = 0 .. F), a multiple of 4
__host__ __device__ inline int m_stride(int F) { return (F + 1 + 3) & ~3; }

// What one column's candidate evaluation needs (shared memory and the LUT).
struct MapCol {
    const int32_t* s_pd8;        // [H + 1] PD[v] + 8 v
    const int32_t* s_pg;         // [H + 1]
    const int32_t* s_ps;         // [H + 1]
    const int32_t* s_thr;        // [H] gravity iff f > fhi (low half), diving iff f < flo (high half)
    const uint2* div;            // rounded-mean constants (the global table, L1-resident)
    const int32_t* s_gv;         // [H] ground state values
    const int32_t* s_sv;         // [H] sky state values
    const int32_t* s_bo;         // [H] best object state value of each row (over f)
    const int32_t* po;           // the column's object LUT, [F][P]
    int P, F, dmax, ord_off;
    int32_t T_oo, T_og, T_os, T_go, T_gg, T_gs, T_so, T_sg, T_ss;
};

// the 64-thread barrier of the two phase-B warps
__device__ __forceinline__ void pair_sync() { asm volatile("bar.sync 1, 64;" ::: "memory"); }

// rounded mean of the stixel [b, k]
__device__ __forceinline__ int map_mean(const MapCol& c, int b, int k)
{
    const uint2 dm = __ldg(c.div + k - b + 1);
    return (int)min(__umulhi((uint32_t)(c.s_pd8[k + 1] - c.s_pd8[b]), dm.x) >> dm.y, (uint32_t)c.dmax);
}

// the entry of row b - 1 of M that an object of mean fo reads
__device__ __forceinline__ int m_index(const MapCol& c, int fo) { return min(max(fo - c.ord_off, 0), c.F); }

// The candidates (cost | previous class code) of the stixel [b, k] with mean
// fo and object data cost d_o: object (for the state (k, fo)), ground and
// sky.  mx = M[b - 1][x] (any value for b = 0).
__device__ __forceinline__ void map_cands(const MapCol& c, const ModelDev& m, int b, int k, int fo, int32_t d_o,
                                          int32_t mx, int32_t& ko, int32_t& kg, int32_t& ks)
{
    const int32_t d_g = c.s_pg[k + 1] - c.s_pg[b], d_s = c.s_ps[k + 1] - c.s_ps[b];
    if (b == 0) {
        ko = d_o + m.first[0] + kNoneCode;
        kg = d_g + m.first[1] + kNoneCode;
        ks = d_s + m.first[2] + kNoneCode;
        return;
    }
    // object above object (ordering exact through M), above ground, above sky
    const int32_t vg = c.s_gv[b - 1], vs = c.s_sv[b - 1];
    const int32_t t = c.s_thr[b];
    const int32_t gpen = (fo > (int32_t)(int16_t)(t & 0xffff) ? m.pen_grav : 0) + (fo < (t >> 16) ? m.pen_div : 0);
    ko = min(min(d_o + mx + c.T_oo, d_o + vg + c.T_og + gpen), d_o + vs + c.T_os);
    // ground / sky above: the best object of row b-1 (any f), ground, sky
    const int32_t vo = c.s_bo[b - 1];
    kg = min(min(d_g + vo + c.T_go, d_g + vg + c.T_gg), d_g + vs + c.T_gs);
    ks = min(min(d_s + vo + c.T_so, d_s + vg + c.T_sg), d_s + vs + c.T_ss);
}

// The lowest f at the minimum value of a row of object states (global) over
// f in [lo, hi), by the whole warp: {value, f} ({kBig, -1} when every state
// there is unreached).
__device__ __forceinline__ int2 row_argmin(const int32_t* row, int lo, int hi, int lane)
{
    int32_t bv = kBig;
    int bf = INT_MAX;
    for (int f = lo + lane; f < hi; f += 32) {
        const int32_t v = state_value(row[f]);
        if (v < bv) { bv = v; bf = f; }            // ascending f: the first at the minimum
    }
    const int32_t mv = __reduce_min_sync(0xffffffffu, bv);
    const int mf = (int)__reduce_min_sync(0xffffffffu, (unsigned)(bv == mv ? bf : INT_MAX));
    return make_int2(mv, mf == INT_MAX ? -1 : mf);
}

// Shared-memory layout of one CTA: a head that lives through the whole
// kernel, and a body that the DP uses and the cost report then takes over.
struct MapLayout {
    size_t gv, sv, bo, pd8, thr, pg, ps;             // head
    size_t bin, gbin, sbin, ring, trid, trif;        // body
    size_t body, total;
};

__host__ __device__ inline size_t up16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline MapLayout map_layout(int H, int F)
{
    MapLayout L;
    size_t o = 0;
    L.gv = o;   o += 4 * (size_t)H;
    L.sv = o;   o += 4 * (size_t)H;
    L.bo = o;   o += 4 * (size_t)H;
    L.pd8 = o;  o += 4 * (size_t)(H + 1);
    L.thr = o;  o += 4 * (size_t)H;
    L.pg = o;   o += 4 * (size_t)(H + 1);
    L.ps = o;   o += 4 * (size_t)(H + 1);
    o = up16(o);
    L.body = o;
    L.bin = o;  o += 4 * 2 * (size_t)kMapRows * m_stride(F);
    L.gbin = o; o += 4 * 2 * kMapRows;
    L.sbin = o; o += 4 * 2 * kMapRows;
    o = up16(o);
    L.ring = o; o += 4 * (size_t)(kMapRows + 1) * m_stride(F);
    L.trid = o; o += 4 * 2 * (size_t)kTri;
    L.trif = o; o += 2 * (size_t)kTri;
    // the report stages 4 H words in the body
    L.total = up16(L.body + (o - L.body > 16 * (size_t)H ? o - L.body : 16 * (size_t)H));
    return L;
}

// Backtracking from the top state (class cc0, mean fb, value best) by one
// warp: the path's stixels, the output records and counts, and the stixel
// part of the cost report (priors and per-stixel constants staged in s_rep[H
// ..4H), the stixel list bottom -> top in s_rep[0..n)); *s_n receives n, or
// -1 when no cost is reported, *s_acc the priors' sum.
__device__ __forceinline__ void walk_and_stage(const MapCol& c, const ModelDev& m, const DpArgs& a, int col, int H,
                                            const int32_t* keyo, const int32_t* kgs, const int32_t* mv,
                                            int32_t* s_rep, int cc0, int fb, int32_t best, int lane, int* s_n,
                                            unsigned long long* s_acc)
{
    const int F = c.F, P = c.P, MS = m_stride(F);
    const int32_t pen_ord = m.pen_ord;
    // The lowest start b <= k whose candidate for the state (k, class cc,
    // mean f) is v, the state's value (cost | code), by the whole warp: four
    // rounds of 32 starts per pass, their loads in flight together.
    auto find_start = [&](int k, int cc, int f, int32_t v) -> int {
        constexpr int kR = 4;
        for (int b0 = 0; b0 <= k; b0 += 32 * kR) {
            int fo[kR];
            int32_t lo[kR], hi[kR], mx[kR];
#pragma unroll
            for (int u = 0; u < kR; ++u) {
                const int b = min(b0 + 32 * u + lane, k);
                fo[u] = map_mean(c, b, k);
                const int32_t* row = c.po + (size_t)fo[u] * P;
                const bool need = cc != 0 || fo[u] == f;
                lo[u] = need ? __ldg(row + b) : 0;
                hi[u] = need ? __ldg(row + k + 1) : 0;
                mx[u] = need && b > 0 ? mv[(size_t)(b - 1) * MS + m_index(c, fo[u])] : 0;
            }
#pragma unroll
            for (int u = 0; u < kR; ++u) {
                const int b = b0 + 32 * u + lane;
                bool hit = false;
                if (b <= k && (cc != 0 || fo[u] == f)) {
                    int32_t ko, kg, ks;
                    map_cands(c, m, b, k, fo[u], hi[u] - lo[u], mx[u], ko, kg, ks);
                    hit = (cc == 0 ? ko : (cc == 1 ? kg : ks)) == v;
                }
                const unsigned hits = __ballot_sync(0xffffffffu, hit);
                if (hits) return b0 + 32 * u + __ffs(hits) - 1;
            }
        }
        return -1;
    };
    int32_t* top_down = s_rep + 3 * H;
    int n = 0;
    for (int k = H - 1, cc = cc0, ff = fb; k >= 0 && cc < 3 && n < H;) {
        const int32_t v = cc == 0 ? keyo[(size_t)k * F + ff] : kgs[(cc == 1 ? 0 : H) + k];
        const int bs = find_start(k, cc, ff, v);
        const int b = bs < 0 ? 0 : bs;                 // (every reached state has a start)
        if (lane == 0) top_down[n] = (b << 13) | (k << 2) | cc;
        ++n;
        const int p = bs < 0 ? 3 : (v & 3);
        int fp = 0;
        if (p == 0 && b >= 1) {
            const int32_t* prow = keyo + (size_t)(b - 1) * F;
            if (cc == 0) {
                // the penalised side (f < x) wins ties: its f are the lower
                const int x = m_index(c, ff);
                const int2 pr = x > 0 ? row_argmin(prow, 0, x, lane) : make_int2(kBig, -1);
                const int2 su = x < F ? row_argmin(prow, x, F, lane) : make_int2(kBig, -1);
                fp = x == 0 ? su.y : (x == F ? pr.y : (pr.x + pen_ord <= su.x ? pr.y : su.y));
            } else {
                fp = row_argmin(prow, 0, F, lane).y;
            }
            fp = max(fp, 0);
        }
        k = b - 1;
        cc = p;
        ff = fp;
    }
    __syncwarp();
    stixel_t* out = a.stixels + (size_t)col * a.cap;
    for (int i = lane; i < n; i += 32) {
        const int w = top_down[n - 1 - i];
        s_rep[i] = w;
        if (i < a.cap) {
            const int b = w >> 13, k = (w >> 2) & 2047;
            const int nrows = k - b + 1;
            const int32_t S = c.s_pd8[k + 1] - c.s_pd8[b] - 8 * nrows;
            stixel_t st;
            st.row_top = (int16_t)(H - 1 - k);
            st.row_bottom = (int16_t)(H - 1 - b);
            st.cls = (uint8_t)(w & 3);
            st.flags = 0;
            st.reserved = 0;
            st.disparity = __fdiv_rn(__int2float_rn(S), __int2float_rn(16 * nrows));
            out[i] = st;
        }
    }
    if (lane == 0) {
        a.counts[col] = n;
        if (n > a.cap) atomicOr(a.err, STIXELS_ERR_CAPACITY);
        if (a.cost_fixed) a.cost_fixed[col] = best;
    }
    __syncwarp();
    if (!a.cost) {
        if (lane == 0) *s_n = -1;
        return;
    }
    const float* __restrict__ k_obj = real_k_obj(a.rows.real_model);
    const float* __restrict__ inv_obj = k_obj + F;
    auto kinv = [&](int f, bool valid) {
        return valid ? make_float2(__ldg(k_obj + f), __ldg(inv_obj + f)) : make_float2(0.f, 0.f);
    };
    auto thr = [&](int b) {
        const int32_t t = c.s_thr[b];
        return make_int2((int32_t)(int16_t)(t & 0xffff), t >> 16);
    };
    const long long pri = warp_sum64(report_stixels(s_rep, n, c.s_pd8, c.div, a, H, lane, kinv, thr));
    if (lane == 0) {
        *s_acc = (unsigned long long)pri;
        *s_n = n;
    }
}

// Column `col` of the frame `a` (its arguments in shared memory) by one CTA.
__device__ __forceinline__ void map_column(const DpArgs& a, const int col, int32_t* keyo_all, int32_t* kgs_all,
                                           int32_t* mv_all)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int H = a.H, P = a.P, F = a.F, MS = m_stride(F);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const ModelDev& m = a.m;
    int32_t* keyo = keyo_all + (size_t)col * H * F;       // [H][F] object states (backtracking)
    int32_t* kgs = kgs_all + (size_t)col * 2 * H;          // [2][H] ground, sky states
    int32_t* mv = mv_all + (size_t)col * H * MS;           // [H][MS] the rows of M

    const MapLayout L = map_layout(H, F);
    int32_t* s_gv = reinterpret_cast<int32_t*>(smem + L.gv);
    int32_t* s_sv = reinterpret_cast<int32_t*>(smem + L.sv);
    int32_t* s_bo = reinterpret_cast<int32_t*>(smem + L.bo);
    int32_t* s_pd8 = reinterpret_cast<int32_t*>(smem + L.pd8);
    int32_t* s_thr = reinterpret_cast<int32_t*>(smem + L.thr);
    int32_t* s_pg = reinterpret_cast<int32_t*>(smem + L.pg);
    int32_t* s_ps = reinterpret_cast<int32_t*>(smem + L.ps);
    int32_t* s_bin = reinterpret_cast<int32_t*>(smem + L.bin);     // [2][kMapRows][MS]
    int32_t* s_gbin = reinterpret_cast<int32_t*>(smem + L.gbin);   // [2][kMapRows]
    int32_t* s_sbin = reinterpret_cast<int32_t*>(smem + L.sbin);   // [2][kMapRows]
    int32_t* s_ring = reinterpret_cast<int32_t*>(smem + L.ring);   // [kMapRows + 1][MS]: ring i = row K0 - 1 + i
    int32_t* s_trid = reinterpret_cast<int32_t*>(smem + L.trid);   // [2][kTri] object data cost of the block's cells
    uint8_t* s_trif = smem + L.trif;                                // [2][kTri] their means
    const uint2* div = reinterpret_cast<const uint2*>(kDivTable.v);

    for (int v = tid; v <= H; v += blockDim.x) {
        s_pd8[v] = a.pd[(size_t)col * P + v] + 8 * v;
        s_pg[v] = a.pg[(size_t)col * P + v];
        s_ps[v] = a.ps[(size_t)col * P + v];
        if (v < H) s_thr[v] = rows_thr(a.rows.fg, H)[v];
    }
    MapCol c;
    c.s_pd8 = s_pd8; c.s_pg = s_pg; c.s_ps = s_ps; c.s_thr = s_thr; c.div = div;
    c.s_gv = s_gv; c.s_sv = s_sv; c.s_bo = s_bo;
    c.po = a.po + (size_t)col * F * P;
    c.P = P; c.F = F; c.dmax = m.dmax; c.ord_off = m.ord_off;       // ordering iff f' > f + ord_off
    c.T_oo = m.trans[0][0]; c.T_og = m.trans[0][1] + 1; c.T_os = m.trans[0][2] + 2;
    c.T_go = m.trans[1][0]; c.T_gg = m.trans[1][1] + 1; c.T_gs = m.trans[1][2] + 2;
    c.T_so = m.trans[2][0]; c.T_sg = m.trans[2][1] + 1; c.T_ss = m.trans[2][2] + 2;
    const int32_t pen_ord = m.pen_ord;

    const int NB = (H + kMapRows - 1) / kMapRows;
    const size_t BF = (size_t)kMapRows * MS;           // bins of one block, rows at the stride of M

    // The object cells (K + i, K + l), i <= l < nr, of the block at rows K:
    // mean and data cost, into triangle buffer `buf` (slot tri_slot(i) + l - i),
    // by the warps w, w + nw, ... (start i per warp, lane = end row).
    auto gather_tri = [&](int buf, int K, int nr, int w, int nw) {
        int32_t* td = s_trid + buf * kTri;
        uint8_t* tf = s_trif + buf * kTri;
        const int k = K + lane;
        for (int i = w; i < nr; i += nw) {
            if (lane >= i && lane < nr) {
                const int b = K + i;
                const int fo = map_mean(c, b, k);
                const int32_t* row = c.po + (size_t)fo * P;
                const int e = tri_slot(i) + lane - i;
                td[e] = __ldg(row + k + 1) - __ldg(row + b);
                tf[e] = (uint8_t)fo;
            }
        }
    };

    // Phase A for the rows K + lane (lane < nr) and the starts b = b0, b0 +
    // step, ... < b1 (rows of earlier blocks, all final), into one block's
    // bins.  M of row b - 1 comes from the ring (whose row 0 is row ring_base)
    // when use_ring, else from global memory.  Four starts are evaluated
    // together so that their loads overlap; a lane keeps its object
    // candidates for one bin until f changes (consecutive starts mostly share
    // f), its ground / sky minima in registers.
    auto phase_a = [&](int32_t* bins, int32_t* gbin, int32_t* sbin, int K, int nr, int b0, int b1, int step,
                       bool use_ring, int ring_base) {
        if (lane >= nr || b0 >= b1) return;
        const int k = K + lane;
        int32_t rg = kNone, rs = kNone, ck = kNone;
        int cf = -1;
        for (int bb = b0; bb < b1; bb += 4 * step) {
            int fo[4];
            int32_t lo[4], hi[4], mx[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int b = min(bb + u * step, b1 - 1);   // past b1: repeats a valid start, not merged
                fo[u] = map_mean(c, b, k);
                const int32_t* row = c.po + (size_t)fo[u] * P;
                lo[u] = __ldg(row + b);
                hi[u] = __ldg(row + k + 1);
                const int x = m_index(c, fo[u]);
                mx[u] = b == 0 ? 0 : (use_ring ? s_ring[(b - 1 - ring_base) * MS + x] : mv[(size_t)(b - 1) * MS + x]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int b = bb + u * step;
                if (b < b1) {
                    int32_t ko, kg, ks;
                    map_cands(c, m, b, k, fo[u], hi[u] - lo[u], mx[u], ko, kg, ks);
                    rg = min(rg, kg);
                    rs = min(rs, ks);
                    if (fo[u] != cf) {
                        if (cf >= 0) atomicMin(&bins[lane * MS + cf], ck);
                        cf = fo[u];
                        ck = ko;
                    } else {
                        ck = min(ck, ko);
                    }
                }
            }
        }
        if (cf >= 0) atomicMin(&bins[lane * MS + cf], ck);
        atomicMin(&gbin[lane], rg);
        atomicMin(&sbin[lane], rs);
    };

    // bins of blocks 0 and 1 (double-buffered by block parity), then block 0's
    // triangle (which reads the prefix arrays staged above)
    for (int i = tid; i < 2 * (int)BF; i += blockDim.x) s_bin[i] = kNone;
    if (tid < 2 * kMapRows) { s_gbin[tid] = kNone; s_sbin[tid] = kNone; }
    __syncthreads();
    gather_tri(0, 0, min(kMapRows, H), warp, kMapWarps);
    __syncthreads();
    for (int j = 0; j < NB; ++j) {
        const int K0 = kMapRows * j, nb = min(kMapRows, H - K0);
        const int K1 = K0 + kMapRows, nb1 = j + 1 < NB ? min(kMapRows, H - K1) : 0;
        int32_t* bin_j = s_bin + (j & 1) * BF;
        int32_t* gbin_j = s_gbin + (j & 1) * kMapRows;
        int32_t* sbin_j = s_sbin + (j & 1) * kMapRows;
        int32_t* bin_n = s_bin + ((j + 1) & 1) * BF;
        int32_t* gbin_n = s_gbin + ((j + 1) & 1) * kMapRows;
        int32_t* sbin_n = s_sbin + ((j + 1) & 1) * kMapRows;
        const int32_t* tri_d = s_trid + (j & 1) * kTri;
        const uint8_t* tri_f = s_trif + (j & 1) * kTri;

        if (warp == kWarpS || warp == kWarpC) {
            // Phase B: the block's rows in order, on two warps.  In step r,
            // warp C evaluates row K0 + r + 1 against the starts K0 .. K0 + r
            // (they read rows of M up to K0 + r - 1) into that row's bins,
            // while warp S finishes row k = K0 + r: it
            // adds the one start that reads row k - 1 (the stixel [k, k]) and
            // turns the row's bins into M[k].  One 64-thread barrier per step
            // orders the two.  The previous block's last row opens the ring
            // (ring row i = row K0 - 1 + i).
            if (j > 0)
                for (int x = (warp == kWarpC ? 32 : 0) + lane; x < MS; x += 64) s_ring[x] = s_ring[kMapRows * MS + x];
            pair_sync();
            for (int r = 0; r < nb; ++r) {
                if (warp == kWarpC) {
                    if (r + 1 < nb) {
                        // row k1's starts K0 + lane <= k1 - 1
                        const int k1 = K0 + r + 1;
                        int32_t ko = kNone, kg = kNone, ks = kNone;
                        int fo = -1 - lane;              // lanes past the row: no candidate, no peer
                        if (lane <= r) {
                            const int b = K0 + lane;
                            const int e = tri_slot(lane) + r + 1 - lane;
                            fo = tri_f[e];
                            const int32_t mx = b == 0 ? 0 : s_ring[lane * MS + m_index(c, fo)];
                            map_cands(c, m, b, k1, fo, tri_d[e], mx, ko, kg, ks);
                        }
                        // consecutive starts mostly share their mean: two
                        // rounds of a scan over the lanes combine the
                        // candidates of equal f within aligned groups of four
                        // lanes (a lane takes a lane below it only if that one
                        // has its f, which keeps every minimum in its bin), so
                        // that one lane per group and run updates the bin
#pragma unroll
                        for (int o = 1; o < 4; o <<= 1) {
                            const int32_t u = __shfl_up_sync(0xffffffffu, ko, o);
                            const int fu = __shfl_up_sync(0xffffffffu, fo, o);
                            if (lane >= o && fu == fo) ko = min(ko, u);
                        }
                        const int fn = __shfl_down_sync(0xffffffffu, fo, 1);
                        if (lane <= r && (lane == 31 || fn != fo || (lane & 3) == 3))
                            atomicMin(&bin_j[(r + 1) * MS + fo], ko);
                        kg = __reduce_min_sync(0xffffffffu, kg);
                        ks = __reduce_min_sync(0xffffffffu, ks);
                        if (lane == 0) {
                            gbin_j[r + 1] = min(gbin_j[r + 1], kg);
                            sbin_j[r + 1] = min(sbin_j[r + 1], ks);
                        }
                    }
                } else {
                    const int k = K0 + r;
                    // the row's object states without the start k, as values;
                    // lane l owns f = 8 l .. 8 l + 7: local suffix minima, then
                    // a warp scan of the lane totals.  With the penalty >= 0,
                    // M[k][x] = min(min_{f >= x} O, best + penalty): where the
                    // penalised prefix holds the row's best that is the
                    // prefix's term, and where the suffix holds it the
                    // penalised term cannot win.
                    int32_t* bin = bin_j + (size_t)r * MS;
                    int32_t sv[kPer];
                    {
                        // two 16-byte loads per lane
                        const int x0 = kPer * lane;
                        int4 u0 = make_int4(kNone, kNone, kNone, kNone), u1 = u0;
                        if (x0 < MS) u0 = *reinterpret_cast<const int4*>(bin + x0);
                        if (x0 + 4 < MS) u1 = *reinterpret_cast<const int4*>(bin + x0 + 4);
                        sv[0] = u0.x; sv[1] = u0.y; sv[2] = u0.z; sv[3] = u0.w;
                        sv[4] = u1.x; sv[5] = u1.y; sv[6] = u1.z; sv[7] = u1.w;
#pragma unroll
                        for (int i = 0; i < kPer; ++i) sv[i] = x0 + i < F ? state_value(sv[i]) : INT_MAX;
                    }
                    // meanwhile the start k (the stixel [k, k]), the same on
                    // every lane: its one object state joins M[k] at the end
                    const int e = tri_slot(r);
                    const int fn = tri_f[e];
                    const int32_t mxn = k == 0 ? 0 : s_ring[r * MS + m_index(c, fn)];
                    int32_t kon, kg, ks;
                    map_cands(c, m, k, k, fn, tri_d[e], mxn, kon, kg, ks);
                    kg = min(kg, gbin_j[r]);
                    ks = min(ks, sbin_j[r]);
                    if (lane == fn / kPer) bin[fn] = min(bin[fn], kon);
                    const int32_t vn = state_value(kon);
#pragma unroll
                    for (int i = kPer - 2; i >= 0; --i) sv[i] = min(sv[i + 1], sv[i]);
                    int32_t st = sv[0];
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int32_t dn = __shfl_down_sync(0xffffffffu, st, o);
                        if (lane + o < 32) st = min(st, dn);
                    }
                    // the exclusive carry from the lanes above; the row's best
                    // object state (with the start k's)
                    int32_t sc = __shfl_down_sync(0xffffffffu, st, 1);
                    if (lane == 31) sc = INT_MAX;
                    const int32_t best = min(__shfl_sync(0xffffffffu, st, 0), vn);
                    const int32_t capped = best + pen_ord;
                    // M[k][x], x = 8 lane + i (shared memory only: the block's
                    // rows go to global memory at its end); the start k's state
                    // is in the suffixes of x <= fn
                    int32_t mr[kPer];
#pragma unroll
                    for (int i = 0; i < kPer; ++i) {
                        const int x = kPer * lane + i;
                        const int32_t suf = min(min(sc, sv[i]), x <= fn ? vn : INT_MAX);
                        mr[i] = min(suf, capped);
                    }
                    int32_t* rrow = s_ring + (r + 1) * MS;
                    const int x0 = kPer * lane;
                    if (x0 + 3 < MS) *reinterpret_cast<int4*>(rrow + x0) = make_int4(mr[0], mr[1], mr[2], mr[3]);
                    if (x0 + 7 < MS) *reinterpret_cast<int4*>(rrow + x0 + 4) = make_int4(mr[4], mr[5], mr[6], mr[7]);
                    if (F == 32 * kPer && lane == 31) rrow[F] = capped;     // x = F past the lanes' ranges
                    if (lane == 0) {
                        gbin_j[r] = kg;
                        sbin_j[r] = ks;
                        s_gv[k] = state_value(kg);
                        s_sv[k] = state_value(ks);
                        s_bo[k] = best;
                    }
                }
                pair_sync();
            }
        } else {
            // meanwhile: the next block's candidates whose starts lie in the
            // blocks before this one (their rows are final), and the next
            // block's own object cells
            const int wa = phase_a_index(warp);
            phase_a(bin_n, gbin_n, sbin_n, K1, nb1, wa, K0, kPhaseAWarps, false, 0);
            if (nb1 > 0) gather_tri((j + 1) & 1, K1, nb1, wa, kPhaseAWarps);
        }
        __syncthreads();                          // block j's rows are final and visible
        // the next block's starts inside this block (M from the ring); then
        // this block's states and rows of M go to global memory, coalesced,
        // and its bins are reset for block j + 2
        phase_a(bin_n, gbin_n, sbin_n, K1, nb1, K0 + warp, K0 + nb, kMapWarps, true, K0 - 1);
        // (the padding past F and the rows past nb are never written)
        for (int r = warp; r < nb; r += kMapWarps)
            for (int f = lane; f < F; f += 32) {
                keyo[(size_t)(K0 + r) * F + f] = bin_j[r * MS + f];
                bin_j[r * MS + f] = kNone;
            }
        for (int i = tid; i < nb * MS; i += blockDim.x) mv[(size_t)K0 * MS + i] = s_ring[MS + i];
        if (tid < kMapRows) {
            if (tid < nb) {
                kgs[K0 + tid] = gbin_j[tid];
                kgs[H + K0 + tid] = sbin_j[tid];
            }
            gbin_j[tid] = kNone;
            sbin_j[tid] = kNone;
        }
        __syncthreads();
    }

    // top row (lexicographic cost, class, f) and backtracking by warp 0, its
    // records and the stixel part of the cost report; then every warp takes
    // its blocks of rows of the report
    __shared__ int s_n;                              // stixels on the path (-1: no report)
    __shared__ unsigned long long s_acc;             // the report's sum, 2^-24 units
    int32_t* s_rep = reinterpret_cast<int32_t*>(smem + L.body);    // the report's 4 H words
    if (warp == 0) {
        const int2 ob = row_argmin(keyo + (size_t)(H - 1) * F, 0, F, lane);
        int cc0 = ob.x < kBig ? 0 : -1, fb = max(ob.y, 0);
        int32_t best = ob.x;
        if (s_gv[H - 1] < best) { best = s_gv[H - 1]; cc0 = 1; fb = 0; }
        if (s_sv[H - 1] < best) { best = s_sv[H - 1]; cc0 = 2; fb = 0; }
        if (cc0 < 0 || best >= kBig) {
            if (lane == 0) {
                a.counts[col] = 0;
                if (a.cost) a.cost[col] = __int_as_float(0x7f800000);
                if (a.cost_fixed) a.cost_fixed[col] = kBig;
                atomicOr(a.err, STIXELS_ERR_INFEASIBLE);
                s_n = -1;
            }
        } else {
            walk_and_stage(c, a.m, a, col, H, keyo, kgs, mv, s_rep, cc0, fb, best, lane, &s_n, &s_acc);
        }
    }
    __syncthreads();
    const int n = s_n;
    if (n < 0) return;
    const long long sum = warp_sum64(report_rows(s_rep, n, s_pd8, a, H, lane, warp, kMapWarps, nullptr));
    if (lane == 0) atomicAdd(&s_acc, (unsigned long long)sum);
    __syncthreads();
    if (tid == 0) a.cost[col] = __ll2float_rn((long long)s_acc) * (1.0f / kReportUnits);
}

// copies the arguments (DpArgs words) to shared memory
__device__ __forceinline__ void stage_args(const DpArgs* src, DpArgs* dst)
{
    const int* s = reinterpret_cast<const int*>(src);
    int* d = reinterpret_cast<int*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(DpArgs) / sizeof(int)); i += blockDim.x) d[i] = s[i];
}

// One frame, one CTA per column.  The column reads its arguments from a
// shared copy (measured against the kernel parameters with only the tail on
// the copy: 1024x440 277 / 285 us, 2048x880 1446 / 1551 us).
__global__ void __launch_bounds__(kMapWarps * 32) stixel_map_kernel(DpArgs a, int32_t* keyo_all, int32_t* kgs_all,
                                                                   int32_t* mv_all)
{
    __shared__ DpArgs s_args;
    stage_args(&a, &s_args);
    __syncthreads();
    map_column(s_args, blockIdx.x, keyo_all, kgs_all, mv_all);
}

// Batch form: one CTA per (frame, column) item of the list (the tallest
// frames' first); each frame's arguments and scratch come from its table row.
__global__ void __launch_bounds__(kMapWarps * 32) stixel_map_batch_kernel(const DpArgs* __restrict__ frames,
                                                                         const MapScratch* __restrict__ scratch,
                                                                         const int2* __restrict__ items)
{
    __shared__ DpArgs s_args;
    const int2 w = items[blockIdx.x];
    stage_args(frames + w.x, &s_args);
    __syncthreads();
    const MapScratch sc = scratch[w.x];
    map_column(s_args, w.y, sc.keyo, sc.kgs, sc.mv);
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// global scratch: object states [ncols][H][F], ground / sky states
// [ncols][2][H], the rows of M [ncols][H][m_stride(F)] (int32 each)
size_t map_scratch_bytes(int H, int ncols, int F)
{
    return up256(sizeof(int32_t) * (size_t)H * F * ncols) + up256(sizeof(int32_t) * 2 * (size_t)H * ncols) +
           sizeof(int32_t) * (size_t)H * m_stride(F) * ncols;
}

MapScratch map_scratch_carve(void* scratch, int H, int ncols, int F)
{
    char* sp = static_cast<char*>(scratch);
    MapScratch r;
    r.keyo = reinterpret_cast<int32_t*>(sp);
    sp += up256(sizeof(int32_t) * (size_t)H * F * ncols);
    r.kgs = reinterpret_cast<int32_t*>(sp);
    sp += up256(sizeof(int32_t) * 2 * (size_t)H * ncols);
    r.mv = reinterpret_cast<int32_t*>(sp);
    return r;
}

size_t map_smem_bytes(int H, int F) { return map_layout(H, F).total; }

bool map_fits(int H, int F) { return F <= 32 * kPer && map_layout(H, F).total <= kMapSmemMax; }

cudaError_t prepare_map_kernel()
{
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        e = cudaFuncSetAttribute(stixel_map_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMapSmemMax);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(stixel_map_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kMapSmemMax);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    return cudaSuccess;
}

cudaError_t launch_dp_map(const int32_t* pd, const int32_t* pg, const int32_t* ps, const int32_t* po,
                          const FrameGeom& g, const ModelDev& m, const RowsDev& r, const RealParams& rp,
                          int32_t pixel_floor, const stixels_output_t& out, uint32_t* err, void* scratch,
                          cudaStream_t st)
{
    if (g.H <= 0 || g.ncols <= 0) return cudaSuccess;
    const int F = m.dmax + 1;
    if (g.H > STIXELS_MAX_HEIGHT || !map_fits(g.H, F)) return cudaErrorInvalidValue;
    DpArgs a;
    dp_frame_args(pd, pg, ps, po, g, m, r, rp, pixel_floor, out, err, &a);
    const size_t smem = map_layout(g.H, F).total;
    cudaError_t e = prepare_map_kernel();
    if (e != cudaSuccess) return e;
    const MapScratch sc = map_scratch_carve(scratch, g.H, g.ncols, F);
    // a plain launch (as a programmatic dependent of the LUT kernel, scheduled
    // while the LUT's CTAs still held the SMs, it measured 292 -> 358 us per
    // 1024x440 call)
    stixel_map_kernel<<<g.ncols, kMapWarps * 32, smem, st>>>(a, sc.keyo, sc.kgs, sc.mv);
    return cudaGetLastError();
}

cudaError_t launch_dp_map_batch(const DpArgs* d_frames, const MapScratch* d_scratch, const int2* d_items, int nitems,
                                size_t smem, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    if (smem > kMapSmemMax) return cudaErrorInvalidValue;
    cudaError_t e = prepare_map_kernel();
    if (e != cudaSuccess) return e;
    stixel_map_batch_kernel<<<nitems, kMapWarps * 32, smem, st>>>(d_frames, d_scratch, d_items);
    return cudaGetLastError();
}

}  // namespace stx
