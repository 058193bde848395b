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
// Parallel scheme (a redesign of the paper's one-thread-per-row CTA with a
// barrier per row), one 256-thread CTA per column, rows cut into blocks of 32:
//   - the chain warp finalises the blocks in order.  For block j it applies the
//     32 starts of block j-1 to block j's end rows, then solves the block's
//     triangle: 32 sequential starts, lane l owning end row 32 j + l; after each
//     start the owner's running minimum is broadcast with a shuffle and every
//     lane derives the next start's context in registers.  Lane l keeps row
//     32 j + l's results in registers (predicated selects, no per-row stores)
//     and the warp writes the block's back-pointers and start contexts with one
//     coalesced store each at the end of the block.  The chain's data terms
//     (with the input-only gravity / diving penalties already added) were
//     gathered into shared memory beforehand, so the sequential chain never
//     waits on global memory.
//   - the 7 bulk warps apply the starts of every finalised block t to the end
//     rows of blocks t+2, t+3, ... (independent 32 x 32 tiles).  End-row block c
//     receives c - 1 tiles; blocks are dealt to the bulk warps largest first
//     to the least-loaded warp, and a block always stays with its warp, so a
//     cell's updates happen in start order.  Right after block t is final they
//     first do what the chain needs next -- the tile (t, t+2) and, shared among
//     all of them, the chain's data gathers for block t+2 -- and only then the
//     tiles of later blocks.
// The two sides synchronise through progress counters in shared memory
// instead of CTA barriers, so neither waits for the other's non-critical work.
// Every wait is a bounded spin: on expiry the CTA records STIXELS_ERR_TIMEOUT,
// leaves the column empty and exits (no wait can hang the device).
// The object LUT is read from global memory (L2-resident).
//
// The kernel is specialised for the standard staggering constraints (ground
// never directly above ground or sky, sky never directly above sky): those
// transitions then drop out of the ground / sky running minima.  Any other
// transition table uses the general instantiation.
#include <climits>

#include "internal.h"

namespace stx {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxBlocks = (STIXELS_MAX_HEIGHT + 31) / 32;
constexpr int kSpinLimit = 1 << 24;  // polls (~20 ns apart) before a wait gives up

// Context of one start row b, shared by every end row k >= b: the three
// previous-class terms V_p[b-1] + T(object | p) + code(p) and the ordering
// threshold (penalty iff f > ford).
struct __align__(16) StartCtx {
    int32_t bo, bg, bs, ford;
};

// Input-only data of row v: pd8 = PD[v] + 8 v (so that S + 8 n of a stixel
// [b, k] is pd8[k + 1] - pd8[b]) and the gravity / diving thresholds at row v
// (penalty iff f > fhi, iff f < flo).
struct __align__(16) RowInfo {
    int32_t pd8, fhi, flo, pad;
};

// Ground and sky prefix entries of rows v and v + 1, read by the chain in one load.
struct __align__(16) GS4 {
    int32_t pg0, ps0, pg1, ps1;
};

// Chain data of one block: for each (start i, end row l) slot e = 32 i + l,
// {d, e_g} = the object data cost and the same plus the ground-below
// penalties, and f = the rounded mean; part 0 = starts of the previous block,
// part 1 = the block's own triangle.
struct ChainBuf {
    int2 de[2][1024];
    uint8_t f[2][1024];
};

struct SyncState {
    int final_blocks;            // blocks the chain warp has finalised
    int abort;                   // set when a wait gave up
    int ready[kMaxBlocks];       // ready[c]: bulk tiles applied to end-row block c
    int gathered[kMaxBlocks];    // gathered[j]: bulk warps done gathering block j's chain data
    int owner[kMaxBlocks];       // bulk warp that owns end-row block c
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

// Rounded mean disparity of a stixel of n rows from x = S + 8 n, clamped to
// the LUT's rows: valid Q4 input always gives f <= dmax; the clamp only keeps
// malformed caller-built LUTs (stixels_solve) inside the table.
__device__ __forceinline__ int mean_f(int32_t x, int n, const uint2* s_div, int dmax)
{
    const uint2 dm = s_div[n];
    return (int)min(__umulhi((uint32_t)x, dm.x) >> dm.y, (uint32_t)dmax);
}

// Minimum of N candidates (cost, start << 8 | f) listed in ascending start
// order, ties to the earlier start, by a pairwise tree (depth log2 N instead of
// a serial chain of N compare-selects).  Result in v[0], bf[0].
template <int N>
__device__ __forceinline__ void tree_min(int32_t (&v)[N], int32_t (&bf)[N])
{
#pragma unroll
    for (int s = 1; s < N; s *= 2)
#pragma unroll
        for (int i = 0; i + s < N; i += 2 * s) {
            const bool take = v[i + s] < v[i];
            v[i] = take ? v[i + s] : v[i];
            bf[i] = take ? bf[i + s] : bf[i];
        }
}

// Gravity / diving penalties of an object with rounded mean f directly above
// ground, base row thresholds r (input-only).
__device__ __forceinline__ int32_t ground_pen(const RowInfo& r, int f, const ModelDev& m)
{
    return (f > r.fhi ? m.pen_grav : 0) + (f < r.flo ? m.pen_div : 0);
}

// Warp-wide bounded wait until *p >= target (lane 0 polls).  Returns false if
// the wait gave up or another warp did; the caller then stops.
__device__ __forceinline__ bool wait_geq(volatile int* p, int target, volatile int* abort_flag)
{
    int ok = 1;
    if ((threadIdx.x & 31) == 0) {
        int it = 0;
        while (*p < target) {
            if (*abort_flag) { ok = 0; break; }
            if (++it > kSpinLimit) { *abort_flag = 1; ok = 0; break; }
            __nanosleep(20);
        }
    }
    ok = __shfl_sync(kFull, ok, 0);
    __threadfence_block();
    return ok != 0;
}

size_t dp_smem_bytes(int H)
{
    const size_t HP = (size_t)((H + 3) & ~3);
    return sizeof(StartCtx) * HP + sizeof(RowInfo) * (HP + 4) + sizeof(GS4) * HP + sizeof(uint2) * (HP + 4) +
           sizeof(int32_t) * 5 * HP + sizeof(ChainBuf) * 2 + sizeof(SyncState);
}

// Solves column `col` of frame `a` with all NW warps of the CTA (one chain
// warp, NW - 1 bulk warps); `sm` is the CTA's dynamic shared memory
// (dp_smem_bytes).  Every warp returns from here; the caller synchronises
// before reusing `sm`.
template <int NW, bool kStdTrans>
__device__ __forceinline__ void dp_column(const DpArgs& a, const int col, int32_t* sm)
{
    constexpr int kWarps = NW;
    constexpr int kThreads = NW * 32;
    constexpr int kBulk = NW - 1;                   // warps besides the chain warp
    const int H = a.H, P = a.P, F = a.F;
    const int HP = (H + 3) & ~3;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const ModelDev& m = a.m;
    // rotate the chain warp between CTAs so that two CTAs sharing an SM are
    // less likely to put their chain warps on the same scheduler; the other
    // warps are bulk warps 0 .. kBulk-1
    const int chain = col & 3;
    const int bulk_id = (warp - chain - 1 + kWarps) % kWarps;

    StartCtx* s_ctx = reinterpret_cast<StartCtx*>(sm);                // [HP]
    RowInfo* s_row = reinterpret_cast<RowInfo*>(s_ctx + HP);          // [HP + 4], row H holds pd8[H]
    GS4* s_gs = reinterpret_cast<GS4*>(s_row + HP + 4);               // [HP]
    uint2* s_div = reinterpret_cast<uint2*>(s_gs + HP);               // [HP + 4], index n = 1..H
    int32_t* s_bp = reinterpret_cast<int32_t*>(s_div + HP + 4);        // [3][HP] back-pointers b << 2 | p
    int32_t* s_runv = s_bp + 3 * HP;                                   // [HP] object running minimum
    int32_t* s_runbf = s_runv + HP;                                    // [HP] its start << 8 | f
    ChainBuf* s_cb = reinterpret_cast<ChainBuf*>(s_runbf + HP);        // [2]
    SyncState* sync = reinterpret_cast<SyncState*>(s_cb + 2);
    volatile int* v_final = &sync->final_blocks;
    volatile int* v_abort = &sync->abort;
    const int NB = (H + 31) >> 5;

    const int32_t* po_col = a.po + (size_t)col * F * P;
    const int32_t* pg_col = a.pg + (size_t)col * P;
    const int32_t* ps_col = a.ps + (size_t)col * P;
    for (int v = threadIdx.x; v <= H; v += kThreads) {
        RowInfo r;
        r.pd8 = a.pd[(size_t)col * P + v] + 8 * v;
        r.fhi = r.flo = r.pad = 0;
        if (v < H) {
            const int32_t g = a.rows.fgq[v];
            r.fhi = (g + m.eps_g) >> 4;             // 16 f > g + eps  <=>  f > floor((g + eps) / 16)
            r.flo = -((m.eps_d - g) >> 4);          // 16 f < g - eps  <=>  f < ceil((g - eps) / 16)
            GS4 q;
            q.pg0 = pg_col[v]; q.ps0 = ps_col[v]; q.pg1 = pg_col[v + 1]; q.ps1 = ps_col[v + 1];
            s_gs[v] = q;
            s_runv[v] = INT_MAX;
            s_runbf[v] = 0;
        }
        s_row[v] = r;
    }
    for (int n = 1 + threadIdx.x; n <= H; n += kThreads) s_div[n] = div_magic(n);
    if (threadIdx.x < kMaxBlocks) {
        sync->ready[threadIdx.x] = 0;
        sync->gathered[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) {
        sync->final_blocks = 0;
        sync->abort = 0;
        // end-row block c receives c - 1 bulk tiles; hand the blocks, largest
        // first, to the least-loaded bulk warp (balanced per-warp work)
        int load[kBulk];
        for (int w = 0; w < kBulk; ++w) load[w] = 0;
        for (int c = NB - 1; c >= 2; --c) {
            int best = 0;
            for (int w = 1; w < kBulk; ++w)
                if (load[w] < load[best]) best = w;
            sync->owner[c] = best;
            load[best] += c - 1;
        }
        // start 0 carries the first-stixel prior (code 3 = no previous stixel)
        s_ctx[0] = StartCtx{m.first[0] + kNoneCode, kBig, kBig, INT_MAX};
    }
    __syncthreads();

    // Gather the data terms the chain warp needs for block jn into chain buffer
    // jn & 1: part 0 = starts of block jn-1 x end rows of block jn, part 1 =
    // starts and end rows of block jn (start <= end row).  All loads of a pass
    // are issued before any store.
    auto gather_chain = [&](int jn, int tid, int nthreads) {
        ChainBuf* cb = s_cb + (jn & 1);
        for (int base = tid; base < 2048; base += 5 * nthreads) {
            int32_t lo[5], hi[5], fv[5];
            bool ok[5];
#pragma unroll
            for (int r = 0; r < 5; ++r) {
                const int idx = base + r * nthreads;
                const int part = idx >> 10, e = idx & 1023, i = e >> 5, l = e & 31;
                const int k = 32 * jn + l;
                const int b = part == 0 ? 32 * (jn - 1) + i : 32 * jn + i;
                ok[r] = idx < 2048 && k < H && (part == 0 ? jn >= 1 : i <= l);
                lo[r] = hi[r] = fv[r] = 0;
                if (ok[r]) {
                    const int f = mean_f(s_row[k + 1].pd8 - s_row[b].pd8, k - b + 1, s_div, m.dmax);
                    const int32_t* row = po_col + (size_t)f * P;
                    lo[r] = __ldg(row + b);
                    hi[r] = __ldg(row + k + 1);
                    fv[r] = f;
                }
            }
#pragma unroll
            for (int r = 0; r < 5; ++r) {
                const int idx = base + r * nthreads;
                if (ok[r]) {
                    const int part = idx >> 10, e = idx & 1023;
                    const int b = part == 0 ? 32 * (jn - 1) + (e >> 5) : 32 * jn + (e >> 5);
                    const int32_t d = hi[r] - lo[r];
                    cb->de[part][e] = make_int2(d, d + ground_pen(s_row[b], fv[r], m));
                    cb->f[part][e] = (uint8_t)fv[r];
                }
            }
        }
    };

    // Apply the 32 starts of finalised block t to end-row block jc (a bulk tile).
    auto bulk_tile = [&](int t, int jc) {
        const int k = 32 * jc + lane;
        const bool kv = k < H;
        const int kk = kv ? k : H - 1;
        int32_t run = INT_MAX, runbf = 0;
        if (kv) { run = s_runv[k]; runbf = s_runbf[k]; }
        const int32_t x1 = s_row[kk + 1].pd8;
#pragma unroll
        for (int h = 0; h < 2; ++h) {          // two groups of 16 starts: 32 gathers in flight
            int32_t lo[16], hi[16], fv[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int b = 32 * t + 16 * h + i;
                const int f = mean_f(x1 - s_row[b].pd8, kk + 1 - b, s_div, m.dmax);
                const int32_t* row = po_col + (size_t)f * P;
                lo[i] = __ldg(row + b);
                hi[i] = __ldg(row + kk + 1);
                fv[i] = f;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int b = 32 * t + 16 * h + i;
                const StartCtx c = s_ctx[b];
                const int32_t d = hi[i] - lo[i];
                const int f = fv[i];
                const int32_t cand = min3(c.bo + d + (f > c.ford ? m.pen_ord : 0),
                                          c.bg + d + ground_pen(s_row[b], f, m), c.bs + d);
                if (cand < run) { run = cand; runbf = (b << 8) | f; }
            }
        }
        if (kv) { s_runv[k] = run; s_runbf[k] = runbf; }
    };

    // chain data of blocks 0 and 1 depend on the input only
    gather_chain(0, threadIdx.x, kThreads);
    if (NB > 1) gather_chain(1, threadIdx.x, kThreads);
    __syncthreads();

    if (warp != chain) {
        // ---------------------------------------------------------------- bulk warps
        for (int t = 0; t + 2 < NB; ++t) {
            if (!wait_geq(v_final, t + 1, v_abort)) break;          // block t is final
            const int jn = t + 2;
            if (sync->owner[jn] == bulk_id) {                         // the tile the chain needs next
                bulk_tile(t, jn);
                __threadfence_block();
                __syncwarp();
                if (lane == 0) sync->ready[jn] = t + 1;
            }
            gather_chain(jn, bulk_id * 32 + lane, kBulk * 32);        // the chain's data for block t+2
            __threadfence_block();
            __syncwarp();
            if (lane == 0) atomicAdd(&sync->gathered[jn], 1);
            for (int jc = jn + 1; jc < NB; ++jc) {                    // tiles of later blocks
                if (sync->owner[jc] != bulk_id) continue;
                bulk_tile(t, jc);
                __threadfence_block();
                __syncwarp();
                if (lane == 0) sync->ready[jc] = t + 1;
            }
        }
        return;
    }

    // -------------------------------------------------------------------- chain warp
    // transition priors with the previous-class codes folded in
    const int32_t T_oo = m.trans[0][0], T_og = m.trans[0][1] + 1, T_os = m.trans[0][2] + 2;
    const int32_t T_go = m.trans[1][0], T_gg = m.trans[1][1] + 1, T_gs = m.trans[1][2] + 2;
    const int32_t T_so = m.trans[2][0], T_sg = m.trans[2][1] + 1, T_ss = m.trans[2][2] + 2;
    const int ord_off = m.eps_o >> 4;               // 16 f > 16 f' + eps  <=>  f > f' + floor(eps / 16)
    // carried state (uniform across lanes): V of the last finalised row, f of
    // its best object stixel, and the ground / sky running minima
    int32_t vo_p = 0, vg_p = 0, vs_p = 0, fo_p = 0;
    int32_t rg = INT_MAX, rgb = 0, rs = INT_MAX, rsb = 0;
    bool aborted = false;

    for (int j = 0; j < NB; ++j) {
        const int B = 32 * j;
        if (j >= 2) {
            if (!wait_geq(&sync->ready[j], j - 1, v_abort) || !wait_geq(&sync->gathered[j], kBulk, v_abort)) {
                aborted = true;
                break;
            }
        }
        const ChainBuf* cb = s_cb + (j & 1);
        const int nb = min(32, H - B);
        const int k = B + lane;
        const bool kv = lane < nb;
        int32_t run = kv ? s_runv[k] : INT_MAX;
        int32_t runbf = kv ? s_runbf[k] : 0;
        if (j > 0) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int32_t cv[16], cbf[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int e = (16 * h + i) * 32 + lane;
                    const int b = B - 32 + 16 * h + i;
                    const StartCtx c = s_ctx[b];
                    const int2 de = cb->de[0][e];
                    const int f = cb->f[0][e];
                    cv[i] = min3(c.bo + de.x + (f > c.ford ? m.pen_ord : 0), c.bg + de.y, c.bs + de.x);
                    cbf[i] = (b << 8) | f;
                }
                tree_min<16>(cv, cbf);
                if (cv[0] < run) { run = cv[0]; runbf = cbf[0]; }
            }
        }
        // lane l's copy of row B + l's results
        int32_t my_r = 0, my_bf = 0, my_gr = 0, my_rgb = 0, my_sk = 0, my_rsb = 0;
        // one start of the triangle, start row b = B + i; `first` is set only for
        // b = 0, whose candidates carry the first-stixel prior
        auto step = [&](int i, bool first) {
            const int b = B + i;
            const GS4 gs = s_gs[b];
            const int2 de = cb->de[1][i * 32 + lane];
            const int ff = cb->f[1][i * 32 + lane];
            int32_t bo, bg, bs, ford, ag, as;
            if (first) {
                bo = m.first[0] + kNoneCode; bg = kBig; bs = kBig; ford = INT_MAX;
                ag = m.first[1] + kNoneCode - gs.pg0;
                as = m.first[2] + kNoneCode - gs.ps0;
            } else {
                bo = vo_p + T_oo; bg = vg_p + T_og; bs = vs_p + T_os; ford = fo_p + ord_off;
                if (kStdTrans) {
                    ag = vo_p + T_go - gs.pg0;
                    as = min(vo_p + T_so, vg_p + T_sg) - gs.ps0;
                } else {
                    ag = min3(vo_p + T_go, vg_p + T_gg, vs_p + T_gs) - gs.pg0;
                    as = min3(vo_p + T_so, vg_p + T_sg, vs_p + T_ss) - gs.ps0;
                }
            }
            if (ag < rg) { rg = ag; rgb = b; }
            if (as < rs) { rs = as; rsb = b; }
            const int32_t cand = min3(bo + de.x + (ff > ford ? m.pen_ord : 0), bg + de.y, bs + de.x);
            if (cand < run) { run = cand; runbf = (b << 8) | ff; }
            // row b is complete: every lane derives its values, lane i keeps them
            const int32_t r = __shfl_sync(kFull, run, i);
            const int32_t bf = __shfl_sync(kFull, runbf, i);
            const int32_t gr = gs.pg1 + rg;
            const int32_t sk = gs.ps1 + rs;
            vo_p = min(r & ~3, kBig);
            vg_p = min(gr & ~3, kBig);
            vs_p = min(sk & ~3, kBig);
            fo_p = bf & 255;
            const bool mine = lane == i;
            my_r = mine ? r : my_r;
            my_bf = mine ? bf : my_bf;
            my_gr = mine ? gr : my_gr;
            my_rgb = mine ? rgb : my_rgb;
            my_sk = mine ? sk : my_sk;
            my_rsb = mine ? rsb : my_rsb;
        };
        int i0 = 0;
        if (j == 0) { step(0, true); i0 = 1; }
        if (nb == 32) {
#pragma unroll 8
            for (int i = i0; i < 32; ++i) step(i, false);
        } else {
#pragma unroll 1
            for (int i = i0; i < nb; ++i) step(i, false);
        }
        // the block's back-pointers and the contexts of the starts that follow its rows
        if (kv) {
            s_bp[k] = ((my_bf >> 8) << 2) | (my_r & 3);
            s_bp[HP + k] = (my_rgb << 2) | (my_gr & 3);
            s_bp[2 * HP + k] = (my_rsb << 2) | (my_sk & 3);
            if (k + 1 < H)
                s_ctx[k + 1] = StartCtx{min(my_r & ~3, kBig) + T_oo, min(my_gr & ~3, kBig) + T_og,
                                        min(my_sk & ~3, kBig) + T_os, (my_bf & 255) + ord_off};
        }
        __threadfence_block();
        __syncwarp();
        if (lane == 0) *v_final = j + 1;
    }

    // backtracking from the top row (Sec. 3.3, Sec. 5.4)
    if (lane == 0) {
        if (aborted) {
            a.counts[col] = 0;
            if (a.cost) a.cost[col] = __int_as_float(0x7f800000);
            if (a.cost_fixed) a.cost_fixed[col] = kBig;
            atomicOr(a.err, STIXELS_ERR_TIMEOUT);
            return;
        }
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
                const int nrows = k - b + 1;
                const int32_t S = s_row[k + 1].pd8 - s_row[b].pd8 - 8 * nrows;
                stixel_t st;
                st.row_top = (int16_t)(H - 1 - k);
                st.row_bottom = (int16_t)(H - 1 - b);
                st.cls = (uint8_t)cc;
                st.flags = 0;
                st.reserved = 0;
                st.disparity = __fdiv_rn(__int2float_rn(S), __int2float_rn(16 * nrows));
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

template <int NW, bool kStd>
__global__ void __launch_bounds__(NW * 32, 16 / NW) stixel_dp_kernel(DpArgs a)
{
    extern __shared__ __align__(16) int32_t sm[];
    dp_column<NW, kStd>(a, blockIdx.x, sm);
}

// Persistent form: each CTA takes columns from a work list (one shared atomic
// counter, reset before the launch) until the list is empty.  The list is
// ordered longest column first, so the last columns to start are the short ones.
template <int NW, bool kStd>
__global__ void __launch_bounds__(NW * 32, 16 / NW)
    stixel_dp_batch_kernel(const DpArgs* __restrict__ frames, const int2* __restrict__ items, int nitems,
                           int* counter)
{
    extern __shared__ __align__(16) int32_t sm[];
    __shared__ DpArgs s_args;
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const int2 w = items[it];                        // (frame, column)
        // the frame's arguments, staged in shared memory for the whole CTA
        const int* src = reinterpret_cast<const int*>(frames + w.x);
        int* dst = reinterpret_cast<int*>(&s_args);
        for (int i = threadIdx.x; i < (int)(sizeof(DpArgs) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
        __syncthreads();
        dp_column<NW, kStd>(s_args, w.y, sm);
        __syncthreads();
    }
}

}  // namespace

int sm_count()
{
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!cached[dev]) cudaDeviceGetAttribute(&cached[dev], cudaDevAttrMultiProcessorCount, dev);
    return cached[dev];
}

namespace {

// opt a kernel in to large dynamic shared memory once per device
template <typename K>
cudaError_t allow_smem(K kernel, bool* done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!done[dev]) {
        // the per-block limit (227 KB) covers static + dynamic shared memory
        cudaFuncAttributes attr;
        e = cudaFuncGetAttributes(&attr, kernel);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 227 * 1024 - (int)attr.sharedSizeBytes);
        if (e != cudaSuccess) return e;
        done[dev] = true;
    }
    return cudaSuccess;
}

// per-instantiation "attribute set" flags, one per device
template <int NW, bool kStd>
bool* frame_flags() { static bool f[64] = {false}; return f; }
template <int NW, bool kStd>
bool* batch_flags() { static bool f[64] = {false}; return f; }

template <int NW, bool kStd>
cudaError_t launch_frame(const DpArgs& a, int ncols, size_t smem, cudaStream_t st)
{
    cudaError_t e = allow_smem(stixel_dp_kernel<NW, kStd>, frame_flags<NW, kStd>());
    if (e != cudaSuccess) return e;
    stixel_dp_kernel<NW, kStd><<<ncols, NW * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int NW, bool kStd>
cudaError_t launch_batch(const DpArgs* frames, const int2* items, int nitems, int* counter, int grid, size_t smem,
                         cudaStream_t st)
{
    cudaError_t e = allow_smem(stixel_dp_batch_kernel<NW, kStd>, batch_flags<NW, kStd>());
    if (e != cudaSuccess) return e;
    stixel_dp_batch_kernel<NW, kStd><<<grid, NW * 32, smem, st>>>(frames, items, nitems, counter);
    return cudaGetLastError();
}

bool standard_transitions(const ModelDev& m)
{
    return m.trans[1][1] >= kBig && m.trans[1][2] >= kBig && m.trans[2][2] >= kBig;
}

}  // namespace

size_t dp_shared_bytes(int H) { return dp_smem_bytes(H); }

void dp_frame_args(const int32_t* pd, const int32_t* pg, const int32_t* ps, const int32_t* po, const FrameGeom& g,
                   const ModelDev& m, const RowsDev& r, const stixels_output_t& out, uint32_t* err, DpArgs* a)
{
    a->pd = pd; a->pg = pg; a->ps = ps; a->po = po;
    a->H = g.H; a->P = g.P; a->F = m.dmax + 1;
    a->m = m; a->rows = r;
    a->stixels = out.stixels; a->counts = out.counts; a->cost = out.column_cost; a->cost_fixed = out.column_cost_fixed;
    a->cap = out.capacity;
    a->err = err;
}

cudaError_t launch_dp(const int32_t* pd, const int32_t* pg, const int32_t* ps, const int32_t* po,
                      const FrameGeom& g, const ModelDev& m, const RowsDev& r, const stixels_output_t& out,
                      uint32_t* err, cudaStream_t st)
{
    if (g.H <= 0 || g.ncols <= 0) return cudaSuccess;
    if (g.H > STIXELS_MAX_HEIGHT) return cudaErrorInvalidValue;
    DpArgs a;
    dp_frame_args(pd, pg, ps, po, g, m, r, out, err, &a);
    const size_t smem = dp_smem_bytes(g.H);
    // with no more columns than SMs, each column gets a whole SM: 16 warps
    // (15 bulk); otherwise two 8-warp CTAs share an SM
    const bool wide = g.ncols <= sm_count();
    if (standard_transitions(m))
        return wide ? launch_frame<16, true>(a, g.ncols, smem, st) : launch_frame<8, true>(a, g.ncols, smem, st);
    return wide ? launch_frame<16, false>(a, g.ncols, smem, st) : launch_frame<8, false>(a, g.ncols, smem, st);
}

cudaError_t prepare_dp_kernels()
{
    // attribute changes are not stream operations: do them before any capture
    cudaError_t e = allow_smem(stixel_dp_batch_kernel<8, true>, batch_flags<8, true>());
    if (e == cudaSuccess) e = allow_smem(stixel_dp_batch_kernel<8, false>, batch_flags<8, false>());
    if (e == cudaSuccess) e = allow_smem(stixel_dp_batch_kernel<16, true>, batch_flags<16, true>());
    if (e == cudaSuccess) e = allow_smem(stixel_dp_batch_kernel<16, false>, batch_flags<16, false>());
    if (e == cudaSuccess) e = allow_smem(stixel_dp_kernel<8, true>, frame_flags<8, true>());
    if (e == cudaSuccess) e = allow_smem(stixel_dp_kernel<8, false>, frame_flags<8, false>());
    if (e == cudaSuccess) e = allow_smem(stixel_dp_kernel<16, true>, frame_flags<16, true>());
    if (e == cudaSuccess) e = allow_smem(stixel_dp_kernel<16, false>, frame_flags<16, false>());
    if (e == cudaSuccess && sm_count() <= 0) e = cudaErrorInvalidDevice;
    return e;
}

cudaError_t launch_dp_batch(const DpArgs* d_frames, const int2* d_items, int nitems, int* d_counter, int maxH,
                            int warps, bool std_trans, int grid, cudaStream_t st)
{
    if (nitems <= 0) return cudaSuccess;
    if (maxH <= 0 || maxH > STIXELS_MAX_HEIGHT || grid <= 0) return cudaErrorInvalidValue;
    const size_t smem = dp_smem_bytes(maxH);
    if (warps == 16)
        return std_trans ? launch_batch<16, true>(d_frames, d_items, nitems, d_counter, grid, smem, st)
                         : launch_batch<16, false>(d_frames, d_items, nitems, d_counter, grid, smem, st);
    return std_trans ? launch_batch<8, true>(d_frames, d_items, nitems, d_counter, grid, smem, st)
                     : launch_batch<8, false>(d_frames, d_items, nitems, d_counter, grid, smem, st);
}

}  // namespace stx
